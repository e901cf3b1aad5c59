"""GPU parity of spatially weighted MI (cmif_compute_weighted, FP64 transforms)
against the oracle's direct weighted histogram.

The weighted counts are real, so there is no rounding and no exact-integer
contract: the tolerance on MI is 1e-9 bits (FP64 transforms: relative count
errors ~1e-13), on N 1e-9 relative.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MI_TOL = 1e-9


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


def _run(cm, A, WA, B, WB, KA, KB, gamma, window=False):
    HA, WdA = A.shape
    HB, WdB = B.shape
    R, C = HA + HB - 1, WdA + WdB - 1
    plan = cm.Plan(HA, WdA, HB, WdB, KA, KB, cm.FP64, weighted=True, window=window)
    mi = torch.full((R, C), float("nan"), dtype=torch.float64, device="cuda:0")
    nw = torch.full((R, C), float("nan"), dtype=torch.float64, device="cuda:0")
    pk = torch.empty(24, dtype=torch.uint8, device="cuda:0")
    plan.compute_weighted(_dev(A), _dev(WA), _dev(B), _dev(WB), mi, nw, gamma, pk)
    st = plan.status()
    plan.close()
    return mi.cpu().numpy(), nw.cpu().numpy(), cm.peaks_from_bytes(pk, 1)[0], st


@pytest.mark.parametrize("shape_a,shape_b,K", [((20, 24), (20, 24), 5), ((33, 17), (21, 30), 7), ((9, 300), (8, 280), 4)])
def test_swmi_vs_oracle(cm, shape_a, shape_b, K):
    rng = np.random.default_rng(sum(shape_a) + sum(shape_b))
    A = rng.integers(0, K, shape_a).astype(np.int32)
    A[: shape_a[0] // 2, : shape_a[1] // 2] = 1
    B = rng.integers(0, K, shape_b).astype(np.int32)
    WA = rng.random(shape_a) * (rng.random(shape_a) > 0.1)   # some zero weights (mask 0)
    WB = rng.gamma(2.0, 1.0, shape_b)
    A[WA == 0] = 777                                           # ignored where the weight is 0
    mi, nw, pk, st = _run(cm, A, WA, B, WB, K, K, 0.4)
    assert st[0] == "OK", st
    ref = oracle.swmi(A, WA, B, WB, K, K)
    assert float(np.abs(mi - ref["mi"]).max()) <= MI_TOL
    assert np.allclose(nw, ref["nw"], rtol=1e-9, atol=1e-9)
    idx, best, _ = oracle.gamma_argmax(ref["mi"], ref["nw"], 0.4)
    a, dy, dx, n, v = pk
    assert abs(v - best) <= MI_TOL
    r, c = dy + shape_a[0] - 1, dx + shape_a[1] - 1
    assert ref["nw"][r, c] >= 0.4 * ref["nw"].max() * (1 - 1e-12)


def test_swmi_unit_weights_equal_mi_and_window(cm):
    """Unit weights: the weighted path equals the integer MI map of cmif_compute;
    with the padded window, rows outside it are zero and the rest unchanged."""
    rng = np.random.default_rng(5)
    A = rng.integers(0, 6, (40, 36)).astype(np.int32)
    B = np.roll(A, (3, -4), axis=(0, 1))
    B[rng.random(B.shape) < 0.2] = 2
    mi, nw, pk, st = _run(cm, A, None, B, None, 6, 6, 0.5)
    ref = oracle.cmif(A, None, B, None, 6, 6)
    assert float(np.abs(mi - ref["mi"]).max()) <= MI_TOL
    assert np.allclose(nw, ref["n"], rtol=1e-12, atol=1e-9)  # real N from FP64 transforms: not rounded
    assert (pk[1], pk[2]) == (3, -4)
    miw, nww, pkw, st = _run(cm, A, None, B, None, 6, 6, 0.5, window=True)
    py = int(np.ceil(40 * 0.5))
    r0, r1 = 40 - 1 - py, 40 - 1 + py + 1
    assert float(np.abs(miw[r0:r1] - ref["mi"][r0:r1]).max()) <= MI_TOL
    assert not miw[:r0].any() and not miw[r1:].any()
    assert (pkw[1], pkw[2]) == (3, -4)
