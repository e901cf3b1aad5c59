"""GPU tests of CUDA-graph replay and of the batch API (uneven pairs, several
K, rotation angles), against direct calls and the oracle."""
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


def test_graph_replay_matches_direct(cm):
    cfg = synth.make_workload("single-256x256-K16", scale=0.5)
    A, B, MA, MB = (_dev(cfg[k]) for k in ("A", "B", "M_A", "M_B"))
    H, W = cfg["A"].shape
    R, C = 2 * H - 1, 2 * W - 1
    direct = cm.cmif(A, MA, B, MB, 16, 16, precision=cm.FP32, gamma=0.5)
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, graph=True)
    mi = torch.empty((R, C), dtype=torch.float64, device="cuda:0")
    n = torch.empty((R, C), dtype=torch.int32, device="cuda:0")
    pk = torch.empty(24, dtype=torch.uint8, device="cuda:0")
    for _ in range(3):  # capture once, replay twice
        mi.fill_(float("nan"))
        plan.compute(A, MA, B, MB, mi, n, None, 0.5, pk)
        torch.cuda.synchronize()
        assert torch.equal(mi, direct["mi"]) and torch.equal(n, direct["n"])
        assert cm.peaks_from_bytes(pk, 1)[0][:4] == direct["peak"][:4]
    # new arguments -> a new capture
    B2 = torch.roll(B, shifts=(3, -2), dims=(0, 1))
    direct2 = cm.cmif(A, MA, B2, MB, 16, 16, precision=cm.FP32, gamma=0.5)
    plan.compute(A, MA, B2, MB, mi, n, None, 0.5, pk)
    torch.cuda.synchronize()
    assert torch.equal(mi, direct2["mi"])
    assert plan.status()[0] == "OK"
    plan.close()


def test_graph_align_rotations(cm):
    cfg = synth.make_workload("rotation-512x512-K16-64angles", scale=64 / 512)
    A, B = _dev(cfg["A"]), _dev(cfg["B"])
    H, W = cfg["A"].shape
    angles = cfg["angles"][::8]
    ref_plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32)
    ref_top = torch.empty(24 * len(angles), dtype=torch.uint8, device="cuda:0")
    ref_plan.align_rotations(A, None, B, None, angles, 0.5, len(angles), ref_top)
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, graph=True)
    top = torch.empty_like(ref_top)
    for _ in range(2):
        top.zero_()
        plan.align_rotations(A, None, B, None, angles, 0.5, len(angles), top)
        torch.cuda.synchronize()
        assert torch.equal(top, ref_top)
    plan.close()
    ref_plan.close()


def _pair_oracle(cm, p):
    """Alg. 1 over the pair's angles by the oracle, on device-warped floating images."""
    A, MA, B, MB = p["A"], p["M_A"], p["B"], p["M_B"]
    per = []
    for th in p["angles"]:
        dB, dM = _dev(B), _dev(MB)
        oB = torch.empty_like(dB)
        oM = torch.empty(B.shape, dtype=torch.uint8, device="cuda:0")
        cm.rotate_nn(dB, dM, th, oB, oM)
        torch.cuda.synchronize()
        ref = oracle.cmif(A, MA, oB.cpu().numpy(), oM.cpu().numpy(), p["K_A"], p["K_B"])
        per.append((ref["mi"], ref["n"]))
    best, _ = oracle.align(per, 0.5, top_k=1)
    return best, per


@pytest.mark.parametrize("graph", [False, True])
def test_batch_vs_oracle(cm, graph):
    cfg = synth.make_workload("uneven-batch-128pairs", scale=0.1)
    pairs = cfg["pairs"]
    dev_pairs = [dict(A=_dev(p["A"]), M_A=_dev(p["M_A"]), B=_dev(p["B"]), M_B=_dev(p["M_B"]), K_A=p["K_A"],
                      K_B=p["K_B"], angles=p["angles"], gamma=0.5) for p in pairs]
    # one translation-only pair as well
    dev_pairs.append(dict(A=dev_pairs[0]["A"], M_A=dev_pairs[0]["M_A"], B=dev_pairs[0]["B"], M_B=dev_pairs[0]["M_B"],
                          K_A=pairs[0]["K_A"], K_B=pairs[0]["K_B"], angles=[], gamma=0.5))
    batch = cm.Batch(dev_pairs, cm.FP32, graph=graph)
    res = torch.empty(24 * len(dev_pairs), dtype=torch.uint8, device="cuda:0")
    stat = torch.full((len(dev_pairs),), -1, dtype=torch.int32, device="cuda:0")
    for _ in range(2 if graph else 1):
        res.zero_()
        batch.run(res, stat)
        torch.cuda.synchronize()
    assert batch.status()[0] == "OK"
    assert torch.all(stat == 0)
    got = cm.peaks_from_bytes(res, len(dev_pairs))
    for i, p in enumerate(pairs):
        best, per = _pair_oracle(cm, p)
        H, W = p["A"].shape
        ga, gdy, gdx, gn, gmi = got[i]
        assert abs(gmi - best[2]) <= MI_TOL, (i, got[i], best)
        mi_at = per[ga][0][gdy + H - 1, gdx + W - 1]
        assert abs(mi_at - best[2]) <= MI_TOL
    # the translation-only pair equals a direct cmif_compute
    p0 = pairs[0]
    direct = cm.cmif(dev_pairs[0]["A"], dev_pairs[0]["M_A"], dev_pairs[0]["B"], dev_pairs[0]["M_B"], p0["K_A"],
                     p0["K_B"], gamma=0.5)
    assert got[-1][1:4] == direct["peak"][1:4] and abs(got[-1][4] - direct["peak"][4]) <= MI_TOL
    batch.close()


@pytest.mark.parametrize("flag", ["window", "nmi"])
def test_batch_with_window_or_nmi(cm, flag):
    """Batch plans inherit CMIF_FLAG_WINDOW / CMIF_FLAG_NMI: each pair's result
    equals a single-pair plan with the same flag."""
    cfg = synth.make_workload("uneven-batch-128pairs", scale=0.08)
    pairs = cfg["pairs"][:4]
    dev_pairs = [dict(A=_dev(p["A"]), M_A=_dev(p["M_A"]), B=_dev(p["B"]), M_B=_dev(p["M_B"]), K_A=p["K_A"],
                      K_B=p["K_B"], angles=p["angles"][:2], gamma=0.5) for p in pairs]
    kw = {flag: True}
    batch = cm.Batch(dev_pairs, cm.FP32, graph=True, **kw)
    res = torch.empty(24 * len(dev_pairs), dtype=torch.uint8, device="cuda:0")
    batch.run(res)
    torch.cuda.synchronize()
    assert batch.status()[0] == "OK"
    got = cm.peaks_from_bytes(res, len(dev_pairs))
    for i, (p, dp) in enumerate(zip(pairs, dev_pairs)):
        HA, WA = p["A"].shape
        HB, WB = p["B"].shape
        plan = cm.Plan(HA, WA, HB, WB, p["K_A"], p["K_B"], cm.FP32, **kw)
        top = torch.empty(24, dtype=torch.uint8, device="cuda:0")
        plan.align_rotations(dp["A"], dp["M_A"], dp["B"], dp["M_B"], dp["angles"], 0.5, 1, top)
        ref = cm.peaks_from_bytes(top, 1)[0]
        assert got[i] == ref, (i, got[i], ref)
        plan.close()
    batch.close()


def test_weighted_graph_replay(cm):
    """cmif_compute_weighted under graph replay: replays equal the direct call."""
    rng = np.random.default_rng(4)
    A = rng.integers(0, 5, (30, 26)).astype(np.int32)
    B = rng.integers(0, 5, (28, 24)).astype(np.int32)
    WA, WB = _dev(rng.random(A.shape)), _dev(rng.random(B.shape))
    R, C = 57, 49
    outs = []
    for graph in (False, True):
        plan = cm.Plan(30, 26, 28, 24, 5, 5, cm.FP64, graph=graph, weighted=True)
        mi = torch.empty((R, C), dtype=torch.float64, device="cuda:0")
        for _ in range(2 if graph else 1):
            mi.fill_(float("nan"))
            plan.compute_weighted(_dev(A), WA, _dev(B), WB, mi, None, 0.3)
            torch.cuda.synchronize()
        outs.append(mi.clone())
        assert plan.status()[0] == "OK"
        plan.close()
    assert torch.equal(outs[0], outs[1])


def test_sharded_batch_single_rank_equals_direct(cm):
    """compute_batch_sharded without a process group (one rank) runs every pair
    and returns, in pair order, the records and statuses of one Batch run."""
    from paper_2106_14699_gb300 import shard
    cfg = synth.make_workload("uneven-batch-128pairs", scale=0.08)
    pairs = cfg["pairs"][:6]
    dev_pairs = [dict(A=_dev(p["A"]), M_A=_dev(p["M_A"]), B=_dev(p["B"]), M_B=_dev(p["M_B"]), K_A=p["K_A"],
                      K_B=p["K_B"], angles=p["angles"], gamma=0.5) for p in pairs]
    recs, stats = shard.compute_batch_sharded(dev_pairs, cm.FP32, graph=False)
    batch = cm.Batch(dev_pairs, cm.FP32, graph=False)
    res = torch.empty(24 * len(dev_pairs), dtype=torch.uint8, device="cuda:0")
    stat = torch.full((len(dev_pairs),), -1, dtype=torch.int32, device="cuda:0")
    batch.run(res, stat)
    torch.cuda.synchronize()
    batch.close()
    assert recs == cm.peaks_from_bytes(res, len(dev_pairs))
    assert stats == stat.cpu().tolist() == [0] * len(dev_pairs)


def test_batch_with_batched_angles_and_autotune(cm, tmp_path, monkeypatch):
    """A batch whose pairs run their angles as units of one launch per stage and
    whose size classes were autotuned gives the same per-pair records as the plain
    batch."""
    monkeypatch.setenv("CMIF_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    cfg = synth.make_workload("uneven-batch-128pairs", scale=0.08)
    pairs = cfg["pairs"][:6]
    dev_pairs = [dict(A=_dev(p["A"]), M_A=_dev(p["M_A"]), B=_dev(p["B"]), M_B=_dev(p["M_B"]), K_A=p["K_A"],
                      K_B=p["K_B"], angles=p["angles"], gamma=0.5) for p in pairs]
    recs = []
    for kw in ({}, {"batch_angles": True, "autotune": True}):
        batch = cm.Batch(dev_pairs, cm.FP32, graph=True, **kw)
        res = torch.empty(24 * len(dev_pairs), dtype=torch.uint8, device="cuda:0")
        for _ in range(2):
            res.zero_()
            batch.run(res)
            torch.cuda.synchronize()
        assert batch.status()[0] == "OK"
        recs.append(cm.peaks_from_bytes(res, len(dev_pairs)))
        batch.close()
    assert recs[0] == recs[1]
    assert (tmp_path / "tune.jsonl").exists()
