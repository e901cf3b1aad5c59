"""GPU parity of the CMIF of label VOLUMES (cmif_plan_create_3d) against the
oracle's direct 3-D method: N bit-exact, MI within MI_TOL, the peak (dz, dy, dx);
and a depth-1 volume plan equal to the image plan."""
import numpy as np
import pytest

import oracle
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



def test_volume_host_entry_auto_and_nmi(cm):
    """Volume plans through the host-buffer entry point (copies of D*H*W voxels)
    with AUTO precision, and NMI maps of a volume plan against the oracle's
    (H_A + H_B) / H_AB: each entropy is within ~1.1e-6 bits, so the NMI error is
    at most 4.4e-6 / H_AB (5e-6 / H_AB allowed), exact 0 where H_AB = 0."""
    rng = np.random.default_rng(31)
    A = rng.integers(0, 4, (3, 10, 12)).astype(np.int32)
    A[:2, :5] = 2
    B = rng.integers(0, 4, (4, 9, 11)).astype(np.int32)
    MB = (rng.random(B.shape) > 0.1).astype(np.uint8)
    ref = oracle.cmif3(A, None, B, MB, 4, 4)
    plan = cm.VolumePlan(3, 10, 12, 4, 9, 11, 4, 4, cm.AUTO)
    mi = np.full((plan.R, plan.C), np.nan)
    n = np.full((plan.R, plan.C), -1, np.int32)
    pk = cm.Peak()
    plan.compute_host(A, None, B, MB, mi, n, 0.5, pk)
    assert plan.status()[0] == "OK"
    plan.close()
    np.testing.assert_array_equal(n, ref["n"])
    assert float(np.abs(mi - ref["mi"]).max()) <= MI_TOL
    _, best, _ = oracle.gamma_argmax(ref["mi"], ref["n"], 0.5)
    row = (pk.angle_idx + 3 - 1) * (10 + 9 - 1) + pk.dy + 10 - 1
    col = pk.dx + 12 - 1
    assert abs(pk.mi - best) <= MI_TOL and abs(ref["mi"][row, col] - best) <= MI_TOL
    assert pk.n == ref["n"][row, col]

    nplan = cm.VolumePlan(3, 10, 12, 4, 9, 11, 4, 4, cm.FP32, nmi=True)
    m = torch.full((nplan.R, nplan.C), float("nan"), dtype=torch.float64, device="cuda:0")
    nplan.compute(_dev(A), None, _dev(B), _dev(MB), m)
    torch.cuda.synchronize()
    assert nplan.status()[0] == "OK"
    nplan.close()
    got = m.cpu().numpy()
    hab = ref["h_ab"]
    zero = hab == 0
    assert np.all(got[zero] == 0.0)
    err = np.abs(got[~zero] - ref["nmi"][~zero])
    assert np.all(err <= 5e-6 / hab[~zero])


def test_volume_auto_every_pair_listed(cm, monkeypatch):
    """Volume plan with CMIF_AUTO and every pair sent to the second precision
    (CMIF_AUTO_PREDICATE=all): the listed pairs' depth-summed products and exact
    counts come from the two-term transforms; N and MI equal the oracle's."""
    monkeypatch.setenv("CMIF_AUTO_PREDICATE", "all")
    rng = np.random.default_rng(41)
    A = rng.integers(0, 3, (4, 9, 10)).astype(np.int32)
    B = rng.integers(0, 3, (3, 8, 11)).astype(np.int32)
    MB = (rng.random(B.shape) > 0.2).astype(np.uint8)
    mi, n, pk, st = _run(cm, A, None, B, MB, 3, cm.AUTO)
    assert st[0] == "OK" and st[2] == 9, st       # all 3 x 3 pairs in the second precision
    ref = oracle.cmif3(A, None, B, MB, 3, 3)
    np.testing.assert_array_equal(n, ref["n"])
    assert float(np.abs(mi - ref["mi"]).max()) <= MI_TOL
