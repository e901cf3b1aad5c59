"""GPU parity of Alg. 1's padded search window (CMIF_FLAG_WINDOW) and of the
two-stage rigid search (cmif_align_two_stage) against the oracle.

The oracle pads A literally (Alg. 1's ZERO-PAD step) and runs the direct method on the
padded pair; the library computes only the window rows of the unpadded map.
Count parity for rotations uses the device-warped B (see test_gpu_rotations).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tolerances import MI_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def cm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_14699_gb300 as cm
    from paper_2106_14699_gb300 import build
    build.build()
    cm.lib()
    return cm


def _dev(x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _case(shape_a, shape_b, K, masked, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(0, K, shape_a).astype(np.int32)
    A[: shape_a[0] // 2, : shape_a[1] // 3] = 1
    y0, x0 = (shape_a[0] - shape_b[0]) // 2, (shape_a[1] - shape_b[1]) // 3
    if shape_b[0] <= shape_a[0] and shape_b[1] <= shape_a[1]:
        B = A[y0:y0 + shape_b[0], x0:x0 + shape_b[1]].copy()
    else:
        B = rng.integers(0, K, shape_b).astype(np.int32)
    B[rng.random(B.shape) < 0.1] = 0
    MB = (rng.random(B.shape) > 0.15).astype(np.uint8) if masked else None
    return A, B, MB


@pytest.mark.parametrize("shapes,K,masked,gamma", [
    (((96, 80), (96, 80)), 8, False, 0.5),
    (((130, 150), (130, 150)), 16, True, 0.3),
    (((200, 180), (64, 72)), 8, True, 0.6),     # template matching
    (((77, 90), (77, 45)), 4, False, 0.0),       # gamma = 0: the window is the whole map
])
def test_compute_window_vs_oracle(cm, shapes, K, masked, gamma):
    A, B, MB = _case(shapes[0], shapes[1], K, masked, seed=sum(shapes[0]) + K)
    HA, WA = A.shape
    HB, WB = B.shape
    R, C = HA + HB - 1, WA + WB - 1
    plan = cm.Plan(HA, WA, HB, WB, K, K, cm.FP32, window=True)
    mi = torch.full((R, C), float("nan"), dtype=torch.float64, device="cuda:0")
    n = torch.full((R, C), -7, dtype=torch.int32, device="cuda:0")
    pk = torch.empty(24, dtype=torch.uint8, device="cuda:0")
    plan.compute(_dev(A), None, _dev(B), _dev(MB), mi, n, None, gamma, pk)
    st = plan.status()
    assert st[0] == "OK", st
    ref = oracle.alg1_padded(A, None, B, MB, K, K, gamma)
    full = oracle.cmif(A, None, B, MB, K, K)
    dy_lo, dy_hi, dx_lo, dx_hi = ref["window"]
    r0, r1 = max(0, dy_lo + HA - 1), min(R, dy_hi + HA)
    g_mi, g_n = mi.cpu().numpy(), n.cpu().numpy()
    # window rows: the unpadded map (every column); other rows: zero
    assert float(np.abs(g_mi[r0:r1] - full["mi"][r0:r1]).max()) <= MI_TOL
    assert np.array_equal(g_n[r0:r1], full["n"][r0:r1])
    assert not g_mi[:r0].any() and not g_mi[r1:].any() and not g_n[:r0].any() and not g_n[r1:].any()
    a, dy, dx, gn, gmi = cm.peaks_from_bytes(pk, 1)[0]
    assert abs(gmi - ref["mi"]) <= MI_TOL, ((dy, dx, gn, gmi), ref)
    if (dy, dx) != (ref["dy"], ref["dx"]):   # FP near tie: the oracle's MI at our choice is its best
        assert abs(full["mi"][dy + HA - 1, dx + WA - 1] - ref["mi"]) <= MI_TOL
        assert dy_lo <= dy <= dy_hi and dx_lo <= dx <= dx_hi
    else:
        assert gn == ref["n"]
    plan.close()


def _dev_warp(cm):
    def warp(B, MB, theta):
        dB, dM = _dev(B), _dev(MB)
        oB = torch.empty_like(dB)
        oM = torch.empty(B.shape, dtype=torch.uint8, device="cuda:0")
        cm.rotate_nn(dB, dM, theta, oB, oM)
        torch.cuda.synchronize()
        return oB.cpu().numpy(), oM.cpu().numpy()
    return warp


def test_align_rotations_window_vs_oracle(cm):
    cfg = synth.make_workload("rotation-512x512-K16-64angles", scale=80 / 512)
    A, B = cfg["A"], cfg["B"]
    H, W = A.shape
    angles = cfg["angles"][::8]
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, window=True)
    top = torch.empty(24 * len(angles), dtype=torch.uint8, device="cuda:0")
    plan.align_rotations(_dev(A), None, _dev(B), None, angles, 0.5, len(angles), top)
    assert plan.status()[0] == "OK"
    got = cm.peaks_from_bytes(top, len(angles))
    warp = _dev_warp(cm)
    recs = []
    for t, th in enumerate(angles):
        wB, wM = warp(B, None, th)
        r = oracle.alg1_padded(A, None, wB, wM, 16, 16, 0.5)
        recs.append((t, r["dy"], r["dx"], r["n"], r["mi"]))
    recs.sort(key=lambda x: (-x[4], x[0]))
    for g, r in zip(got, recs):
        assert abs(g[4] - r[4]) <= MI_TOL, (g, r)
    assert got[0][0] == recs[0][0]
    plan.close()


def test_two_stage_vs_oracle(cm):
    cfg = synth.make_workload("rotation-512x512-K16-64angles", scale=64 / 512)
    A, B = cfg["A"], cfg["B"]
    H, W = A.shape
    u = [0.11, 0.5, 0.73, 0.94, 0.28, 0.6]
    for window in (False, True):
        plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, window=window)
        (a, dy, dx, n, mi), theta = plan.align_two_stage(_dev(A), None, _dev(B), None, 16, u, 0.5)
        assert plan.status()[0] == "OK"
        (ra, rdy, rdx, rn, rmi), rtheta = oracle.align_two_stage(A, None, B, None, 16, 16, 16, u, 0.5,
                                                                 padded=window, warp=_dev_warp(cm))
        assert abs(mi - rmi) <= MI_TOL, (window, (a, dy, dx, n, mi), (ra, rdy, rdx, rn, rmi))
        assert a == ra and abs(theta - rtheta) < 1e-12
        plan.close()


def test_rotation512_two_stage_refines_planted_angle(cm):
    """512^2, B = A rotated by 37.5 deg (off the 5.625 deg grid) and shifted by
    (-23, 61): the refinement draws (evenly spaced here) bring the angle within
    2 deg of 37.5 deg and never lower I."""
    cfg = synth.make_workload("rotation-512x512-K16-64angles")
    A, B = cfg["A"], cfg["B"]
    H, W = A.shape
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, window=True)
    (a1, _, _, _, mi1), th1 = plan.align_two_stage(_dev(A), None, _dev(B), None, 64, [], 0.5)
    u = [(i + 0.5) / 16 for i in range(16)]
    (a2, dy, dx, n, mi2), th2 = plan.align_two_stage(_dev(A), None, _dev(B), None, 64, u, 0.5)
    assert plan.status()[0] == "OK"
    assert mi2 >= mi1
    assert abs(math.degrees(th2) - 37.5) <= 2.0, math.degrees(th2)
    assert abs(dy - cfg["shift"][0]) <= 3 and abs(dx - cfg["shift"][1]) <= 3
    plan.close()
