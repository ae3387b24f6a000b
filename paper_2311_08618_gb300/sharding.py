"""Multi-GPU k-range sharding: one H^2 replica per rank, the target indices
split equally (the first parallel algorithm of Sec. 4.2), no data-path
collective; results are gathered once at the end.  The per-rank solve is a
multi-k h2_kth_eig, which reuses inertia across that rank's indices
(its extreme eigenvalues bracket the inner ones, Sec. 4.2)."""
from __future__ import annotations


def equal_distribution(ks, world: int):
    """Contiguous, equally sized shares of the sorted index list (sizes differ
    by at most one), rank r gets share r."""
    ks = sorted(ks)
    n = len(ks)
    base, extra = divmod(n, world)
    out, i = [], 0
    for r in range(world):
        m = base + (1 if r < extra else 0)
        out.append(ks[i:i + m])
        i += m
    return out


def solve_sharded(solver, ks, rank: int, world: int, dist=None):
    """solver(list_of_k) -> list_of_values on this rank's share; returns the
    dict k -> value for all ks on every rank (one all_gather_object)."""
    mine = equal_distribution(ks, world)[rank]
    vals = list(solver(mine)) if mine else []
    local = dict(zip(mine, vals))
    if dist is None or world == 1:
        return local
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    out = {}
    for g in gathered:
        out.update(g)
    return out


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (the bench's timing rule)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
