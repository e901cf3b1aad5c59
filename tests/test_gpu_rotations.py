"""GPU parity for Alg. 1 over rotations: the NN warp (cmif_rotate_nn) and
cmif_align_rotations against the oracle.

Count parity does not depend on floating-point ties of the warp: the oracle's
maps are computed on the device-warped images (downloaded); the warp itself is
checked separately against the oracle's FP64 warp, allowing a pixel or 1e-4 of
the pixels to differ where a source coordinate sits on a rounding tie.
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


def _warp_dev(cm, B, MB, theta):
    dB, dM = _dev(B), _dev(MB)
    oB = torch.empty_like(dB)
    oM = torch.empty(B.shape, dtype=torch.uint8, device="cuda:0")
    cm.rotate_nn(dB, dM, theta, oB, oM)
    torch.cuda.synchronize()
    return oB.cpu().numpy(), oM.cpu().numpy()


@pytest.mark.parametrize("theta", [0.0, math.pi / 2, math.radians(37.5), math.pi, 2.1, -0.7, 5.9])
def test_rotate_nn_matches_oracle(cm, theta):
    rng = np.random.default_rng(3)
    B = rng.integers(0, 13, (301, 257)).astype(np.int32)
    MB = (rng.random(B.shape) > 0.2).astype(np.uint8)
    gB, gM = _warp_dev(cm, B, MB, theta)
    rB, rM = oracle.warp_nn(B, MB, theta)
    diff = int(((gB != rB) | (gM != rM)).sum())
    assert diff <= 1 + 1e-4 * B.size, diff
    if theta in (0.0, math.pi / 2, math.pi):
        assert diff == 0


def test_align_rotations_vs_oracle(cm):
    cfg = synth.make_workload("rotation-512x512-K16-64angles", scale=96 / 512)
    A, B = cfg["A"], cfg["B"]
    H, W = A.shape
    K = 16
    angles = cfg["angles"][::4]  # 16 of the 64 angles
    n_ang = len(angles)
    R, C = 2 * H - 1, 2 * W - 1
    plan = cm.Plan(H, W, H, W, K, K, cm.FP32)
    maps = torch.empty((n_ang, R, C), dtype=torch.float64, device="cuda:0")
    topk = torch.empty(24 * n_ang, dtype=torch.uint8, device="cuda:0")
    plan.align_rotations(_dev(A), None, _dev(B), None, angles, 0.5, n_ang, topk, maps)
    st = plan.status()
    assert st[0] == "OK", st
    got_maps = maps.cpu().numpy()
    per_angle = []
    for i, th in enumerate(angles):
        wB, wM = _warp_dev(cm, B, None, th)
        ref = oracle.cmif(A, None, wB, wM, K, K)
        err = float(np.abs(got_maps[i] - ref["mi"]).max())
        assert err <= MI_TOL, (i, err)
        per_angle.append((ref["mi"], ref["n"]))
    best, top = oracle.align(per_angle, 0.5, top_k=n_ang)
    got = cm.peaks_from_bytes(topk, n_ang)
    for (ga, gdy, gdx, gn, gmi), (ra, ridx, rmi, rn) in zip(got, top):
        rdy, rdx = divmod(ridx, C)
        rdy -= H - 1
        rdx -= W - 1
        if (ga, gdy, gdx) != (ra, rdy, rdx):
            # a floating-point near tie: the oracle's MI at our choice must equal its best
            mi_o = per_angle[ga][0][gdy + H - 1, gdx + W - 1]
            assert abs(mi_o - rmi) <= MI_TOL
        assert abs(gmi - rmi) <= MI_TOL
    assert got[0][0] == best[0]
    plan.close()


def test_rotation512_planted_angle_and_shift(cm):
    """512^2, K = 16, 64 angles over 360 degrees; B is A rotated by 37.5 deg and
    shifted by (-23, 61).  37.5 deg is off the 5.625 deg grid: the best angle
    must be a grid neighbour and the shift within 3 px of the planted one."""
    cfg = synth.make_workload("rotation-512x512-K16-64angles")
    A, B = cfg["A"], cfg["B"]
    H, W = A.shape
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32)
    topk = torch.empty(24 * 5, dtype=torch.uint8, device="cuda:0")
    plan.align_rotations(_dev(A), None, _dev(B), None, cfg["angles"], 0.5, 5, topk)
    st = plan.status()
    assert st[0] == "OK" and st[1] < 0.25, st
    top = cm.peaks_from_bytes(topk, 5)
    ang_deg = math.degrees(cfg["angles"][top[0][0]])
    assert min(abs(ang_deg - 33.75), abs(ang_deg - 39.375)) < 1e-9, top
    assert abs(top[0][1] - cfg["shift"][0]) <= 3 and abs(top[0][2] - cfg["shift"][1]) <= 3, top
    mis = [t[4] for t in top]
    assert all(mis[i] >= mis[i + 1] for i in range(4))
    plan.close()


def test_sharded_entry_single_rank_equals_direct(cm):
    """shard.align_rotations_sharded without a process group = one rank holding
    every angle: its merged top-k equals cmif_align_rotations' device top-k."""
    from paper_2106_14699_gb300 import shard
    cfg = synth.make_workload("rotation-512x512-K16-64angles", scale=64 / 512)
    A, B = _dev(cfg["A"]), _dev(cfg["B"])
    H, W = cfg["A"].shape
    angles = list(cfg["angles"][::4])
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32)
    top = torch.empty(24 * 5, dtype=torch.uint8, device="cuda:0")
    plan.align_rotations(A, None, B, None, angles, 0.5, 5, top)
    direct = cm.peaks_from_bytes(top, 5)
    merged = shard.align_rotations_sharded(plan, A, None, B, None, angles, 0.5, 5)
    assert merged == direct
    plan.close()


@pytest.mark.parametrize("window", [False, True])
def test_batched_angles_equal_angle_by_angle(cm, window, monkeypatch):
    """CMIF_FLAG_BATCH_ANGLES: the angles run as units of one launch per stage
    (chunks of at most 5 here, so 16 angles take 5 + 5 + 5 + 1); maps, N maps and
    the top-k equal the angle-by-angle run bit for bit, with unequal image sizes
    and label counts."""
    monkeypatch.setenv("CMIF_ANGLE_BATCH", "5")
    rng = np.random.default_rng(77)
    HA, WA, HB, WB, KA, KB = 70, 90, 61, 77, 6, 9
    A = synth.make_field(rng, HA, WA, 60, KA).image(HA, WA)
    B = synth.make_field(rng, HB, WB, 50, KB).image(HB, WB)
    MB = (rng.random((HB, WB)) > 0.1).astype(np.uint8)
    angles = np.linspace(0.0, 2 * math.pi, 16, endpoint=False) + 0.1
    R, C = HA + HB - 1, WA + WB - 1
    out = []
    for batched in (False, True):
        plan = cm.Plan(HA, WA, HB, WB, KA, KB, cm.FP32, window=window, batch_angles=batched)
        maps = torch.full((16, R, C), float("nan"), dtype=torch.float64, device="cuda:0")
        nmaps = torch.full((16, R, C), -1, dtype=torch.int32, device="cuda:0")
        top = torch.zeros(24 * 16, dtype=torch.uint8, device="cuda:0")
        plan.align_rotations(_dev(A), None, _dev(B), _dev(MB), angles, 0.5, 16, top, maps, n_maps=nmaps)
        st = plan.status()
        assert st[0] == "OK", st
        out.append((maps, nmaps, top))
        plan.close()
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(torch.nan_to_num(out[0][0], nan=-7.0), torch.nan_to_num(out[1][0], nan=-7.0))
    assert torch.equal(out[0][2], out[1][2])


def test_batched_angles_vs_oracle(cm):
    """Batched angles at 96^2 (the rotation workload scaled down), 16 angles in one
    launch per stage: every map equals the oracle's on the device-warped B."""
    cfg = synth.make_workload("rotation-512x512-K16-64angles", scale=96 / 512)
    A, B = cfg["A"], cfg["B"]
    H, W = A.shape
    angles = cfg["angles"][::4]
    n_ang = len(angles)
    R, C = 2 * H - 1, 2 * W - 1
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, batch_angles=True)
    maps = torch.empty((n_ang, R, C), dtype=torch.float64, device="cuda:0")
    nmaps = torch.empty((n_ang, R, C), dtype=torch.int32, device="cuda:0")
    topk = torch.empty(24 * n_ang, dtype=torch.uint8, device="cuda:0")
    plan.align_rotations(_dev(A), None, _dev(B), None, angles, 0.5, n_ang, topk, maps, n_maps=nmaps)
    assert plan.status()[0] == "OK"
    gm, gn = maps.cpu().numpy(), nmaps.cpu().numpy()
    per = []
    for i, th in enumerate(angles):
        wB, wM = _warp_dev(cm, B, None, th)
        ref = oracle.cmif(A, None, wB, wM, 16, 16)
        np.testing.assert_array_equal(gn[i], ref["n"])
        assert float(np.abs(gm[i] - ref["mi"]).max()) <= MI_TOL
        per.append((ref["mi"], ref["n"]))
    best, top = oracle.align(per, 0.5, top_k=n_ang)
    got = cm.peaks_from_bytes(topk, n_ang)
    assert got[0][0] == best[0]
    for (ga, gdy, gdx, gnn, gmi), (ra, ridx, rmi, rn) in zip(got, top):
        assert abs(gmi - rmi) <= MI_TOL
    plan.close()
