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
