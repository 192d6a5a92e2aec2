"""Multi-process form of the path: every rank owns whole events (or disjoint Philox counter
ranges of one event), so the data path needs no collective.  The only exchanges are the
job's wall time (the maximum over ranks) and, when one event's batches are spread over
ranks, the associative merge of the reducer states (max log w, S1, S2, N) -- 32 bytes per
event, gathered once and merged with mbis_merge_summaries.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """The items rank `rank` of `world` owns: a strided split, so every rank gets an equal
    share (to within one) of a list ordered by any key."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return list(items)[rank::world]


def counter_range(n_total: int, rank: int, world: int):
    """[start, stop) of the Philox counters rank `rank` draws when n_total samples of one
    event are spread over `world` ranks (contiguous, sizes differ by at most one)."""
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(seconds: float, device=None) -> float:
    """The job's time: the largest of the ranks' times."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


_FIELDS = ("max_logw", "s1", "s2", "n")


def merge_over_ranks(summary: dict, merge=None, device=None) -> dict:
    """Merge one reducer state per rank into the state of all the ranks' samples.
    summary: a dict with max_logw, s1, s2, n (as mbis_reduce returns).  merge: the
    two-state merge (defaults to the library's mbis_merge_summaries)."""
    import torch
    import torch.distributed as tdist
    if merge is None:
        from . import mbis_merge_summaries as merge
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return dict(summary)
    mine = torch.tensor([float(summary[k]) for k in _FIELDS], dtype=torch.float64, device=device)
    parts = [torch.empty_like(mine) for _ in range(tdist.get_world_size())]
    tdist.all_gather(parts, mine)
    states = [dict(zip(_FIELDS, p.cpu().numpy().tolist())) for p in parts]
    out = states[0]
    out["n"] = int(out["n"])
    for s in states[1:]:
        s["n"] = int(s["n"])
        out = merge(out, s)
    return out
