"""The epilogue's per-count entropy term, checked over every count a map can hold.

The MI of a shift is (sum_joint T(c) - sum_A T - sum_B T + T(N)) / N with
T(c) = c log2 c (Eq. finalentropy rearranged; the joint counts, each marginal
family and N all sum to N).  The row kernels evaluate T(c) = c * L(c) in fixed
point, so |dMI| <= 4 * max_c |L(c) 2^-F - log2 c|.  This test reads L(c) back
through cmif_entropy_terms for every c in [0, 2^22] (the largest N a plan
allows) and compares it with log2 c in FP64: the maximum it finds is the
per-count bound behind the MI tolerance the parity tests assert.
"""
import numpy as np
import pytest

from tolerances import MI_TOL, TERM_EPS

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


def test_entropy_term_every_count(cm):
    n = (1 << 22) + 1
    out = torch.empty(n, dtype=torch.int64, device="cuda:0")
    cm.entropy_terms(0, n, out)
    torch.cuda.synchronize()
    T = out.cpu().numpy()
    assert T[0] == 0 and T[1] == 0                      # 0 log 0 = 0 (Sec. 3.2), 1 log 1 = 0
    c = np.arange(1, n, dtype=np.int64)
    assert np.all(T[1:] % c == 0)                       # T(c) = c * L(c), L an integer
    L = T[1:] // c
    err = np.abs(L.astype(np.float64) * 2.0 ** -cm.ENTROPY_FIX_BITS - np.log2(c.astype(np.float64)))
    worst = int(np.argmax(err)) + 1
    print(f"[entropy-term] max |L(c) 2^-{cm.ENTROPY_FIX_BITS} - log2 c| = {err.max():.4e} "
          f"(= 2^{np.log2(err.max()):.3f}) at c = {worst}; 4x = {4 * err.max():.4e}")
    assert err.max() <= TERM_EPS
    assert 4 * TERM_EPS <= MI_TOL                      # the parity tolerance covers the worst case
    assert np.all(np.diff(T[1:]) > 0)                   # c log2 c is increasing for c >= 1


def test_entropy_term_range_checks(cm):
    out = torch.empty(4, dtype=torch.int64, device="cuda:0")
    with pytest.raises(cm.CmifError):
        cm.entropy_terms(-1, 4, out)
    with pytest.raises(cm.CmifError):
        cm.entropy_terms((1 << 22) - 2, 4, out)          # beyond the largest count
