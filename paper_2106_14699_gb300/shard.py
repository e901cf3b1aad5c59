"""Alg. 1 over several GPUs: independent units, one top-k merge.

The units of Alg. 1 -- one rotation angle T of one image pair -- are
independent (each is a full CMIF map and its gamma-gated argmax).  A rank
computes the per-angle bests of a contiguous share of the angle list with
``cmif_align_rotations`` on its own GPU; the ranks then exchange only their k
best records and merge them in the order of the device top-k: MI descending,
the lower global angle index first among equals.  Alg. 1's choice is the first
merged record when its MI is > 0 (I starts at 0, a transform replaces it only
when strictly greater), else the identity.

Records are ``(angle_idx, dy, dx, n, mi)`` tuples as returned by
``peaks_from_bytes``; ``angle_idx < 0`` marks an empty slot.

A batch of image pairs shards the same way one level up: every pair (all its
angles) is one unit.  Pairs differ widely in cost, so they are split by a work
model, longest first onto the least-loaded rank; each rank runs one
``cmif_compute_batch`` over its pairs and the ranks exchange only the one
result record and status of each pair.
"""
from __future__ import annotations

EMPTY = (-1, 0, 0, 0, 0.0)


def shard_range(n_units: int, world: int, rank: int):
    """Contiguous share [lo, hi) of n_units for rank (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError(f"bad shard request: n_units={n_units}, world={world}, rank={rank}")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_topk(records, k: int):
    """The k best of records (any order, empty slots ignored), padded with EMPTY."""
    live = [tuple(r) for r in records if r[0] >= 0]
    live.sort(key=lambda r: (-r[4], r[0]))
    out = live[:k]
    return out + [EMPTY] * (k - len(out))


def alg1_choice(merged):
    """Alg. 1's (angle_idx, dy, dx, n, mi) from merged records, or EMPTY (identity)."""
    return merged[0] if merged and merged[0][0] >= 0 and merged[0][4] > 0.0 else EMPTY


def gather_merge(local_records, k: int, group=None):
    """All-gather every rank's records (global angle indices) and merge them.

    Every rank of the process group must call this; all receive the same result.
    Without an initialised process group it merges the local records only.
    """
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return merge_topk(local_records, k)
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, [tuple(r) for r in local_records], group=group)
    return merge_topk([r for p in parts for r in p], k)


def align_rotations_sharded(plan, A, M_A, B, M_B, angles_rad, gamma: float, top_k: int, group=None):
    """Alg. 1 over angles_rad, this rank's share on this rank's GPU, merged over the group.

    A, M_A, B, M_B are CUDA tensors on this rank's device (masks may be None).
    Returns the merged top_k records (global angle indices) on every rank.
    """
    import torch
    import torch.distributed as dist
    from . import peaks_from_bytes
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    lo, hi = shard_range(len(angles_rad), world, rank)
    local = []
    if hi > lo:
        k_loc = min(top_k, hi - lo)
        buf = torch.empty(24 * k_loc, dtype=torch.uint8, device=A.device)
        plan.align_rotations(A, M_A, B, M_B, list(angles_rad[lo:hi]), gamma, k_loc, buf)
        torch.cuda.synchronize(A.device)
        for (a, dy, dx, n, mi) in peaks_from_bytes(buf, k_loc):
            if a >= 0:
                local.append((a + lo, dy, dx, n, mi))
    return gather_merge(local, top_k, group)


def _pow2_at_least(n: int) -> int:
    return 1 << max(4, (max(1, n) - 1).bit_length())


def pair_work(H_A: int, W_A: int, H_B: int, W_B: int, K_A: int, K_B: int, n_angles: int) -> int:
    """Work model of one batch pair: transform points of A's forward planes once,
    and per angle B's forward planes and the K_A x K_B pair transforms, on the
    power-of-two P x Q grid that holds the full shift range."""
    PQ = _pow2_at_least(H_A + H_B - 1) * _pow2_at_least(W_A + W_B - 1)
    return K_A * PQ + max(1, n_angles) * (K_B + K_A * K_B) * PQ


def shard_pairs(works, world: int, rank: int):
    """This rank's pair indices (ascending) under a longest-first greedy split:
    pairs in decreasing work (lower index first among equals) each go to the
    least-loaded rank (lower rank first among equals).  Every pair lands on
    exactly one rank, and no rank's load exceeds the mean load by more than the
    largest single work."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad shard request: world={world}, rank={rank}")
    load = [0] * world
    owner = [0] * len(works)
    for i in sorted(range(len(works)), key=lambda i: (-works[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += works[i]
    return [i for i in range(len(works)) if owner[i] == rank]


def gather_pair_results(local, n_pairs: int, group=None):
    """All-gather every rank's ``(pair_index, record, status)`` triples and return
    (records, statuses) in pair order; a pair that no rank reported keeps EMPTY
    and status None.  Every rank of the process group must call this."""
    import torch.distributed as dist
    parts = [list(local)]
    if dist.is_available() and dist.is_initialized():
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, [(int(i), tuple(r), s) for i, r, s in local], group=group)
    records, statuses = [EMPTY] * n_pairs, [None] * n_pairs
    for part in parts:
        for i, r, s in part:
            records[i], statuses[i] = tuple(r), s
    return records, statuses


def run_pairs_sharded(works, run_local, group=None):
    """Shard pairs with the given works over the group, call ``run_local(indices)``
    on this rank's share (it returns one (record, status) per index, in order)
    and gather all pairs' results on every rank."""
    import torch.distributed as dist
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    mine = shard_pairs(works, world, rank)
    local = []
    if mine:
        out = run_local(mine)
        if len(out) != len(mine):
            raise RuntimeError(f"run_local returned {len(out)} results for {len(mine)} pairs")
        local = [(i, r, s) for i, (r, s) in zip(mine, out)]
    return gather_pair_results(local, len(works), group)


def compute_batch_sharded(pairs, precision, group=None, **batch_kw):
    """cmif_compute_batch over pairs (dicts as for ``Batch``, device tensors on this
    rank's GPU), this rank's share on this rank's GPU.  Returns (records,
    statuses) of all pairs in order on every rank; statuses are cmif_status codes."""
    import torch
    from . import Batch, peaks_from_bytes
    works = [pair_work(*p["A"].shape, *p["B"].shape, p["K_A"], p["K_B"], len(p.get("angles", [])))
             for p in pairs]

    def run_local(idx):
        dev = pairs[idx[0]]["A"].device
        b = Batch([pairs[i] for i in idx], precision, **batch_kw)
        try:
            res = torch.empty(24 * len(idx), dtype=torch.uint8, device=dev)
            stat = torch.empty(len(idx), dtype=torch.int32, device=dev)
            b.run(res, stat)
            torch.cuda.synchronize(dev)
            return list(zip(peaks_from_bytes(res, len(idx)), stat.cpu().tolist()))
        finally:
            b.close()

    return run_pairs_sharded(works, run_local, group)
