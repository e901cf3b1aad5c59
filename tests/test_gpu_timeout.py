"""The bounded device waits of the Tensor-Memory row kernel run out cleanly.

The row kernel fetches each team's next row of column-inverted products with a
bulk copy completed on an mbarrier; every wait gives up after a poll limit,
records a timeout in the device status word and ends the kernel's work without
touching memory it does not own.  Here the plan's diagnostics withhold the copy
of one output row (the mbarrier phase that nothing completes), with a short
poll limit: the call must report TIMEOUT, and the same plan must then compute
a correct map again (the context stays usable).  Nothing faults or hangs.
"""
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


def test_row_kernel_wait_times_out_then_recovers(cm):
    H = W = 512          # transform width 1024: the Tensor-Memory row kernel
    K = 4
    rng = np.random.default_rng(21)
    A, B = synth.planted_pair(rng, H, W, 300, K, K, (7, -11), 0.1, same_labels=True)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    R, C = 2 * H - 1, 2 * W - 1
    plan = cm.Plan(H, W, H, W, K, K, cm.FP32)
    mi = torch.zeros((R, C), dtype=torch.float64, device="cuda:0")
    n = torch.zeros((R, C), dtype=torch.int32, device="cuda:0")
    plan.set_wait_test(1 << 12, 700)           # short limit; row 700's first copy never issued
    plan.compute(dA, None, dB, None, mi, n, None, 0.5)
    st = plan.status()
    assert st[0] == "TIMEOUT", st
    assert int(n[700].abs().sum()) == 0        # the row whose wait ran out is not written
    plan.set_wait_test(0, -1)                  # back to the default limit, nothing withheld
    mi.fill_(float("nan"))
    plan.compute(dA, None, dB, None, mi, n, None, 0.5)
    st = plan.status()
    assert st[0] == "OK" and st[1] < 0.25, st
    got_mi, got_n = mi.cpu().numpy(), n.cpu().numpy()
    dys = np.array([0, 7, -511, 511, 189, -300], dtype=np.int32)
    dxs = np.array([0, -11, 511, -511, 17, 402], dtype=np.int32)
    ref = oracle.cmif_at(A, None, B, None, K, K, dys, dxs)
    np.testing.assert_array_equal(got_n[dys + H - 1, dxs + W - 1], ref["n"])
    assert np.abs(got_mi[dys + H - 1, dxs + W - 1] - ref["mi"]).max() <= MI_TOL
    plan.close()
