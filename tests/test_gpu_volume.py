"""GPU parity of the CMIF of label VOLUMES (cmif_plan_create_3d) against the
oracle's direct 3-D method: N bit-exact, MI within 1e-6, the peak (dz, dy, dx);
and a depth-1 volume plan equal to the image plan."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MI_TOL = 1e-6


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


def _run(cm, A, MA, B, MB, K, prec, gamma=0.5):
    plan = cm.VolumePlan(*A.shape, *B.shape, K, K, prec)
    mi = torch.full((plan.R, plan.C), float("nan"), dtype=torch.float64, device="cuda:0")
    n = torch.full((plan.R, plan.C), -1, dtype=torch.int32, device="cuda:0")
    pk = torch.empty(24, dtype=torch.uint8, device="cuda:0")
    plan.compute(_dev(A), _dev(MA), _dev(B), _dev(MB), mi, n, None, gamma, pk)
    st = plan.status()
    plan.close()
    return mi.cpu().numpy(), n.cpu().numpy(), cm.peaks_from_bytes(pk, 1)[0], st


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
@pytest.mark.parametrize("shape_a,shape_b,K", [((4, 9, 10), (3, 8, 11), 4), ((6, 12, 7), (6, 12, 7), 5),
                                               ((2, 30, 20), (5, 17, 24), 3)])
def test_volume_vs_oracle(cm, prec, shape_a, shape_b, K):
    rng = np.random.default_rng(sum(shape_a) * 7 + K)
    A = rng.integers(0, K, shape_a).astype(np.int32)
    A[: shape_a[0] // 2, : shape_a[1] // 2] = 1
    B = rng.integers(0, K, shape_b).astype(np.int32)
    MA = (rng.random(shape_a) > 0.1).astype(np.uint8)
    MB = (rng.random(shape_b) > 0.15).astype(np.uint8)
    A[MA == 0] = 99
    mi, n, pk, st = _run(cm, A, MA, B, MB, K, getattr(cm, prec))
    assert st[0] == "OK", st
    ref = oracle.cmif3(A, MA, B, MB, K, K)
    np.testing.assert_array_equal(n, ref["n"])
    assert float(np.abs(mi - ref["mi"]).max()) <= MI_TOL
    idx, best, _ = oracle.gamma_argmax(ref["mi"], ref["n"], 0.5)
    dz, dy, dx, pn, pv = pk
    R2 = shape_a[1] + shape_b[1] - 1
    row = (dz + shape_a[0] - 1) * R2 + dy + shape_a[1] - 1
    col = dx + shape_a[2] - 1
    assert abs(pv - best) <= MI_TOL and abs(ref["mi"][row, col] - best) <= MI_TOL


def test_volume_planted_shift_and_depth1(cm):
    rng = np.random.default_rng(21)
    A = rng.integers(0, 6, (8, 20, 22)).astype(np.int32)
    A[:, :10, :11] = 2
    B = np.roll(A, (2, -3, 4), axis=(0, 1, 2))
    B[rng.random(B.shape) < 0.1] = 0
    mi, n, pk, st = _run(cm, A, None, B, None, 6, cm.FP32)
    assert st[0] == "OK"
    assert tuple(pk[:3]) == (2, -3, 4), pk
    # depth 1: a volume plan is the image plan
    A2, B2 = A[0], B[0]
    mi1, n1, pk1, _ = _run(cm, A2[None], None, B2[None], None, 6, cm.FP32)
    ref = cm.cmif(_dev(A2), None, _dev(B2), None, 6, 6, precision=cm.FP32, gamma=0.5)
    assert np.array_equal(mi1, ref["mi"].cpu().numpy()) and np.array_equal(n1, ref["n"].cpu().numpy())
