"""The autotuner (cmif_plan_autotune): it times the launch-shape candidates of a
plan's FP32 transforms and keeps the fastest; the choice does not change the
results (the same counts, and the same MI, which is computed from exact integer
sums), it is cached per process and in the JSON-lines cache file."""
import json

import numpy as np
import pytest

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


@pytest.mark.parametrize("H,K", [(512, 8), (300, 5)])
def test_autotune_keeps_results_and_caches(cm, tmp_path, H, K):
    rng = np.random.default_rng(H + K)
    A, B = synth.planted_pair(rng, H, H, 200, K, K, (5, -9), 0.1, same_labels=True)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    R = 2 * H - 1
    plan = cm.Plan(H, H, H, H, K, K, cm.FP32)
    mi0 = torch.empty((R, R), dtype=torch.float64, device="cuda:0")
    n0 = torch.empty((R, R), dtype=torch.int32, device="cuda:0")
    plan.compute(dA, None, dB, None, mi0, n0, None, 0.5)
    cache = tmp_path / "tune.jsonl"
    t = plan.autotune(str(cache))
    print(f"[autotune] {H}^2 K={K}: {t}")
    assert t["col_lanes"] in (16, 32) and t["tmem_rows"] in (0, 1)
    assert t["from_cache"] in (0, 1) and (t["from_cache"] == 1 or t["candidates"] >= 2)
    mi1, n1 = torch.empty_like(mi0), torch.empty_like(n0)
    plan.compute(dA, None, dB, None, mi1, n1, None, 0.5)
    assert plan.status()[0] == "OK"
    assert torch.equal(n0, n1) and torch.equal(mi0, mi1)
    again = plan.autotune(str(cache))
    assert again["from_cache"] == 1 and again["col_lanes"] == t["col_lanes"]
    if t["from_cache"] == 0:
        line = json.loads(cache.read_text().strip().splitlines()[-1])
        assert line["key"].startswith("P") and f".KA{K}.KB{K}." in line["key"] and line["col_m"] in (0, 16)
    plan.close()
