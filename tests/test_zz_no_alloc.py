"""The no-allocation entry point (cmif_compute_noalloc) against cmif_compute and the oracle.

It serves callers that may not allocate device memory (a host framework that
owns all device memory, code that must not synchronise the device); its
scratch is a fixed array inside the library.  Two calls in a row, on inputs of
different sizes, must each match the plan-based entry point (N and the peak
exactly, MI within the parity tolerance) and the CPU oracle (N bit-exact, MI
within the parity tolerance).  The optional outputs are exercised too: N kept
inside the fixed array (no n_map) with a peak, and a status-only call.  Around
a repeated call the device's free memory must not change.  This file is
collected last so that a failure here leaves every other test run.
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


def _dev(x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _cases():
    cfg = synth.make_workload("plain-64x64-K8")
    yield cfg["A"], cfg["M_A"], cfg["B"], cfg["M_B"], 8, 8
    rng = np.random.default_rng(77)
    A = synth.make_field(rng, 45, 70, 30, 12).image(45, 70)
    B = synth.make_field(rng, 60, 38, 30, 9).image(60, 38)
    MB = (rng.random(B.shape) > 0.1).astype(np.uint8)
    yield A, None, B, MB, 12, 9


def test_noalloc_matches_compute_and_oracle_twice(cm):
    for A, MA, B, MB, KA, KB in _cases():
        dA, dB, dMA, dMB = _dev(A), _dev(B), _dev(MA), _dev(MB)
        ref = cm.cmif(dA, dMA, dB, dMB, KA, KB, precision=cm.FP32, gamma=0.5)
        orc = oracle.cmif(A, MA, B, MB, KA, KB)
        R, C = A.shape[0] + B.shape[0] - 1, A.shape[1] + B.shape[1] - 1
        mi = torch.full((R, C), float("nan"), dtype=torch.float64, device="cuda:0")
        n = torch.full((R, C), -1, dtype=torch.int32, device="cuda:0")
        peak = torch.zeros(24, dtype=torch.uint8, device="cuda:0")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
        cm.compute_noalloc(dA, dMA, dB, dMB, KA, KB, mi, n, 0.5, peak, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(n, ref["n"])
        assert float((mi - ref["mi"]).abs().max()) <= MI_TOL
        np.testing.assert_array_equal(n.cpu().numpy(), orc["n"])
        assert float(np.abs(mi.cpu().numpy() - orc["mi"]).max()) <= MI_TOL
        pk = cm.Peak.from_buffer_copy(peak.cpu().numpy().tobytes())
        assert (pk.dy, pk.dx, pk.n) == ref["peak"][1:4]


def test_noalloc_optional_outputs_and_no_allocation(cm):
    cfg = synth.make_workload("plain-64x64-K8")
    A, MA, B, MB = (_dev(cfg[k]) for k in ("A", "M_A", "B", "M_B"))
    ref = cm.cmif(A, MA, B, MB, 8, 8, precision=cm.FP32, gamma=0.5)
    mi = torch.empty((127, 127), dtype=torch.float64, device="cuda:0")
    peak = torch.zeros(24, dtype=torch.uint8, device="cuda:0")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
    # N kept in the fixed array: the gamma gate and the peak still use it
    cm.compute_noalloc(A, MA, B, MB, 8, 8, mi, None, 0.5, peak, None)
    torch.cuda.synchronize()
    pk = cm.Peak.from_buffer_copy(peak.cpu().numpy().tobytes())
    assert (pk.dy, pk.dx, pk.n) == ref["peak"][1:4] and abs(pk.mi - ref["peak"][4]) <= MI_TOL
    assert float((mi - ref["mi"]).abs().max()) <= MI_TOL
    # status only, no peak, no N map; the free device memory must not move
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    mi.fill_(float("nan"))
    cm.compute_noalloc(A, MA, B, MB, 8, 8, mi, None, 0.5, None, status)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(status.item()) == 0
    assert float((mi - ref["mi"]).abs().max()) <= MI_TOL


def test_noalloc_rejects_oversize_and_bad_tensors(cm):
    A = torch.zeros((512, 512), dtype=torch.int32, device="cuda:0")
    mi = torch.empty((1023, 1023), dtype=torch.float64, device="cuda:0")
    with pytest.raises(cm.CmifError) as ei:
        cm.compute_noalloc(A, None, A, None, 16, 16, mi)
    assert ei.value.code == 8  # CMIF_ERR_UNSUPPORTED: workspace beyond the fixed array
    a = torch.zeros((16, 16), dtype=torch.int32, device="cuda:0")
    with pytest.raises(cm.CmifError) as ei:  # MI map of the wrong dtype: refused before the C call
        cm.compute_noalloc(a, None, a, None, 2, 2, torch.empty((31, 31), dtype=torch.float32, device="cuda:0"))
    assert ei.value.code == 1
    with pytest.raises(cm.CmifError) as ei:  # wrong shape
        cm.compute_noalloc(a, None, a, None, 2, 2, torch.empty((30, 31), dtype=torch.float64, device="cuda:0"))
    assert ei.value.code == 1
