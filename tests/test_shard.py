"""Alg. 1 sharded over ranks (CPU, gloo): shares, merge order, and a world-size-2
run whose merged top-k equals the single-process Alg. 1 of the oracle.

The per-angle maps inside the ranks come from the oracle (no GPU here); what is
under test is the product's sharding and merge logic (paper_2106_14699_gb300.shard).
"""
import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2106_14699_gb300 import shard

torch = pytest.importorskip("torch")


def test_shard_range_covers_once():
    for n in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            seen = []
            sizes = []
            for r in range(world):
                lo, hi = shard.shard_range(n, world, r)
                seen.extend(range(lo, hi))
                sizes.append(hi - lo)
            assert seen == list(range(n))
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(4, 2, 2)


def test_merge_order_and_ties():
    recs = [(3, 0, 0, 9, 0.5), (1, 2, 2, 9, 0.5), (0, 1, 1, 9, 0.25), shard.EMPTY, (2, 5, 5, 9, 0.75)]
    m = shard.merge_topk(recs, 3)
    assert [r[0] for r in m] == [2, 1, 3]            # MI descending, lower angle first among equals
    assert shard.merge_topk(recs, 6)[-2:] == [shard.EMPTY, shard.EMPTY]
    assert shard.alg1_choice(m)[0] == 2
    assert shard.alg1_choice([(0, 0, 0, 1, 0.0)]) == shard.EMPTY  # I starts at 0, strict >


def _case():
    rng = np.random.default_rng(11)
    H = W = 20
    A = rng.integers(0, 4, (H, W)).astype(np.int32)
    A[:10, :10] = 1
    A[10:, 10:] = 2
    angles = [2 * math.pi * t / 7 for t in range(7)]
    B, MB = oracle.warp_nn(A, None, angles[3])
    return A, B, MB, angles


def _per_angle_records(A, B, MB, angles, lo, hi, gamma):
    recs = []
    C = 2 * A.shape[1] - 1
    for t in range(lo, hi):
        wB, wM = oracle.warp_nn(B, MB, angles[t])
        ref = oracle.cmif(A, None, wB, wM, 4, 4)
        idx, mi, n = oracle.gamma_argmax(ref["mi"], ref["n"], gamma)
        dy, dx = divmod(idx, C)
        recs.append((t, dy - (A.shape[0] - 1), dx - (A.shape[1] - 1), n, mi))
    return recs


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, B, MB, angles = _case()
        lo, hi = shard.shard_range(len(angles), world, rank)
        local = shard.merge_topk(_per_angle_records(A, B, MB, angles, lo, hi, 0.5), 3)
        merged = shard.gather_merge([r for r in local if r[0] >= 0], 3)
        np.save(f"{out_path}.{rank}.npy", np.array(merged, dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gloo_world2_merge_equals_single_process(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    out = str(tmp_path / "merged")
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    got = [list(map(tuple, np.load(f"{out}.{r}.npy", allow_pickle=True))) for r in range(world)]
    assert got[0] == got[1]                      # every rank holds the same merge
    A, B, MB, angles = _case()
    per = []
    C = 2 * A.shape[1] - 1
    for t in range(len(angles)):
        wB, wM = oracle.warp_nn(B, MB, angles[t])
        ref = oracle.cmif(A, None, wB, wM, 4, 4)
        per.append((ref["mi"], ref["n"]))
    best, top = oracle.align(per, 0.5, top_k=3)
    for (ga, gdy, gdx, gn, gmi), (ra, ridx, rmi, rn) in zip(got[0], top):
        rdy, rdx = divmod(ridx, C)
        assert (ga, gdy, gdx, gn) == (ra, rdy - (A.shape[0] - 1), rdx - (A.shape[1] - 1), rn)
        assert gmi == rmi
    # B is A turned by angles[3]; turning B by angles[4] = 2 pi - angles[3] undoes it
    assert shard.alg1_choice(got[0])[0] == best[0] == 4


# ---- batch pairs as units --------------------------------------------------

def test_shard_pairs_partition_and_balance():
    rng = np.random.default_rng(4)
    works = [int(w) for w in rng.integers(1, 1000, 37)] + [5000, 5000]
    for world in (1, 2, 3, 8, 50):
        shares = [shard.shard_pairs(works, world, r) for r in range(world)]
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(works)))                 # every pair exactly once
        loads = [sum(works[i] for i in s) for s in shares]
        assert max(loads) <= sum(works) / world + max(works)   # longest-first bound
        assert all(s == sorted(s) for s in shares)
    assert shard.shard_pairs([], 2, 1) == []
    with pytest.raises(ValueError):
        shard.shard_pairs(works, 2, 2)
    # the model: a pair's work grows with K_A K_B, its angles and its transform grid
    w = shard.pair_work(100, 100, 100, 100, 8, 8, 4)
    assert shard.pair_work(100, 100, 100, 100, 16, 16, 4) > 3 * w
    assert shard.pair_work(100, 100, 100, 100, 8, 8, 8) > 1.9 * w
    assert shard.pair_work(200, 100, 200, 100, 8, 8, 4) == 2 * w


def _batch_pairs():
    rng = np.random.default_rng(17)
    out = []
    for H, W, K, n_ang in [(12, 14, 3, 2), (9, 10, 2, 1), (16, 11, 4, 3), (8, 8, 3, 0), (13, 9, 2, 2)]:
        A = rng.integers(0, K, (H, W)).astype(np.int32)
        A[: H // 2, : W // 2] = 0
        B = np.roll(A, (1, -2), axis=(0, 1))
        angles = [2 * math.pi * t / 5 for t in range(n_ang)]
        out.append(dict(A=A, B=B, K=K, angles=angles))
    return out


def _pair_record(p, gamma=0.5):
    """Alg. 1's choice for one pair by the oracle (angle index 0 without angles)."""
    per = []
    for th in (p["angles"] or [None]):
        wB, wM = (p["B"], None) if th is None else oracle.warp_nn(p["B"], None, th)
        ref = oracle.cmif(p["A"], None, wB, wM, p["K"], p["K"])
        per.append((ref["mi"], ref["n"]))
    (a, idx, mi, n), _ = oracle.align(per, gamma)
    if a < 0:
        return shard.EMPTY
    dy, dx = divmod(idx, 2 * p["A"].shape[1] - 1)
    return (a, dy - (p["A"].shape[0] - 1), dx - (p["A"].shape[1] - 1), n, mi)


def _works(pairs):
    return [shard.pair_work(*p["A"].shape, *p["B"].shape, p["K"], p["K"], len(p["angles"])) for p in pairs]


def _pairs_rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pairs = _batch_pairs()
        ran = []

        def run_local(idx):
            ran.extend(idx)
            return [(_pair_record(pairs[i]), 0) for i in idx]
        recs, stats = shard.run_pairs_sharded(_works(pairs), run_local)
        np.save(f"{out_path}.{rank}.npy", np.array([recs, stats, ran], dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_gloo_world2_pairs_equal_single_process(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    out = str(tmp_path / "pairs")
    mp.start_processes(_pairs_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    got = [np.load(f"{out}.{r}.npy", allow_pickle=True) for r in range(world)]
    recs0, stats0, ran0 = got[0]
    recs1, stats1, ran1 = got[1]
    assert list(recs0) == list(recs1) and list(stats0) == list(stats1)   # every rank holds all results
    assert sorted(list(ran0) + list(ran1)) == list(range(5))              # each pair computed once
    assert ran0 and ran1                                                  # both ranks worked
    pairs = _batch_pairs()
    assert [tuple(r) for r in recs0] == [_pair_record(p) for p in pairs]
    assert list(stats0) == [0] * 5
