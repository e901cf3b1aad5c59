"""GPU parity of the NMI map (CMIF_FLAG_NMI) against the oracle's
(H_A + H_B) / H_AB from the direct method's entropies.

Tolerance: each entropy of the fixed-point reduction is within ~1.1e-6 bits
(the MI bound), so |dNMI| <= (|dH_A| + |dH_B| + NMI |dH_AB|) / H_AB
<= 4.4e-6 / H_AB; the test allows 5e-6 / H_AB, and exact 0 where H_AB = 0.
"""
import numpy as np
import pytest

import oracle
import synth

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


def _check(got, ref):
    hab = ref["h_ab"]
    zero = hab == 0
    assert np.all(got[zero] == 0.0)
    tol = 5e-6 / np.maximum(hab[~zero], 1e-300)
    err = np.abs(got[~zero] - ref["nmi"][~zero])
    assert np.all(err <= tol), float((err / tol).max())


@pytest.mark.parametrize("shape,K,prec", [
    ((150, 200), 8, "FP32"),     # TMEM row kernel (Q = 512)
    ((96, 520), 8, "FP32"),      # TMEM row kernel (Q = 2048)
    ((40, 1100), 6, "FP32"),     # generic FP32 row kernel (Q = 3072)
    ((70, 66), 6, "FP64"),
    ((70, 66), 6, "SPLIT32"),
])
def test_nmi_map_vs_oracle(cm, shape, K, prec):
    rng = np.random.default_rng(sum(shape) + K)
    A = rng.integers(0, K, shape).astype(np.int32)
    A[: shape[0] // 2, : shape[1] // 3] = 2
    B = np.roll(A, (5, -9), axis=(0, 1))
    B[rng.random(B.shape) < 0.25] = 1
    MB = (rng.random(B.shape) > 0.1).astype(np.uint8)
    H, W = shape
    R, C = 2 * H - 1, 2 * W - 1
    plan = cm.Plan(H, W, H, W, K, K, getattr(cm, prec), nmi=True)
    m = torch.empty((R, C), dtype=torch.float64, device="cuda:0")
    n = torch.empty((R, C), dtype=torch.int32, device="cuda:0")
    pk = torch.empty(24, dtype=torch.uint8, device="cuda:0")
    plan.compute(_dev(A), None, _dev(B), _dev(MB), m, n, None, 0.5, pk)
    assert plan.status()[0] == "OK"
    ref = oracle.nmi(A, None, B, MB, K, K)
    got = m.cpu().numpy()
    _check(got, ref)
    assert np.array_equal(n.cpu().numpy(), ref["n"])
    # Alg. 1 on the NMI map: the peak is the gated argmax of NMI
    idx, v, nn = oracle.gamma_argmax(ref["nmi"], ref["n"], 0.5)
    a, dy, dx, gn, gv = cm.peaks_from_bytes(pk, 1)[0]
    assert abs(gv - v) <= 5e-6 / max(ref["h_ab"].flat[idx], 1e-3)
    plan.close()


def test_nmi_single256_full_map(cm):
    cfg = synth.make_workload("single-256x256-K16")
    A, B, MA, MB = cfg["A"], cfg["B"], cfg["M_A"], cfg["M_B"]
    H, W = A.shape
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, nmi=True)
    m = torch.empty((2 * H - 1, 2 * W - 1), dtype=torch.float64, device="cuda:0")
    plan.compute(_dev(A), _dev(MA), _dev(B), _dev(MB), m)
    assert plan.status()[0] == "OK"
    _check(m.cpu().numpy(), oracle.nmi(A, MA, B, MB, 16, 16))
    plan.close()
