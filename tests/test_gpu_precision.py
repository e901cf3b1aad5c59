"""The three transform precisions side by side at the benchmark size
(1024^2, K = 16): FP32, two-term FP32 (split) and FP64.  For each: time of one
map, max pre-rounding residual, count mismatches and MI error against the
oracle on sampled shifts (all K_A*K_B + K_A + K_B counts there), and count
mismatches of the whole map against the FP64 map."""
import time

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


def test_single1024_three_precisions(cm, capsys):
    cfg = synth.make_workload("single-1024x1024-K16")
    A, B = cfg["A"], cfg["B"]
    H = 1024
    K = 16
    R = C = 2 * H - 1
    nmaps = K * K + 2 * K
    dev = torch.device("cuda:0")
    dA, dB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    rng = np.random.default_rng(5)
    dys = rng.integers(-(H - 1), H, 48).astype(np.int32)
    dxs = rng.integers(-(H - 1), H, 48).astype(np.int32)
    dys[0], dxs[0] = cfg["shift"]
    ref = oracle.cmif_at(A, None, B, None, K, K, dys, dxs, counts=True)
    rows, cols = dys + H - 1, dxs + H - 1
    report, counts_by = [], {}
    for name in ("FP64", "SPLIT32", "FP32"):
        prec = getattr(cm, name)
        plan = cm.Plan(H, H, H, H, K, K, prec, debug_counts=True)
        mi = torch.empty((R, C), dtype=torch.float64, device=dev)
        n = torch.empty((R, C), dtype=torch.int32, device=dev)
        counts = torch.empty((nmaps, R, C), dtype=torch.int32, device=dev)
        plan.compute(dA, None, dB, None, mi, n, counts, 0.5, None)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.compute(dA, None, dB, None, mi, n, None, 0.5, None)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        st = plan.status()
        joint = counts[:K * K][:, torch.from_numpy(rows).long().to(dev), torch.from_numpy(cols).long().to(dev)]
        joint = joint.cpu().numpy().T  # [shift][pair]
        mism = int((joint != ref["joint"]).sum())
        err = float(np.abs(mi.cpu().numpy()[rows, cols] - ref["mi"]).max())
        if name == "FP64":
            counts_by["FP64"] = counts
            full_mism = 0
        else:
            full_mism = int((counts != counts_by["FP64"]).sum().item())
        report.append((name, ms, st[1], mism, full_mism, err, st[0]))
        assert st[0] == "OK" and st[1] < 0.25
        assert mism == 0 and full_mism == 0
        assert err <= MI_TOL
        if name != "FP64":
            del counts
        plan.close()
    with capsys.disabled():
        print("\n[precision] 1024^2, K=16: name, ms/map (debug counts off), max residual, "
              "count mismatches vs oracle at 48 shifts x 256 pairs, count mismatches vs FP64 over the whole map, "
              "max |dMI| at the sampled shifts, status")
        for r in report:
            print(f"[precision] {r[0]:8s} {r[1]:9.2f} ms  residual={r[2]:.3e}  mism_oracle={r[3]}  "
                  f"mism_fp64={r[4]}  max|dMI|={r[5]:.3e}  {r[6]}")
