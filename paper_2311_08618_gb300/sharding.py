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


# ---------------------------------------------------------------------------
# The second parallel algorithm of Sec. 4.2: a master keeps the free intervals
# and gives each idle worker one of them with its range of eigenvalue indices.
# A worker computes every eigenvalue of an item holding at most 2m of them;
# otherwise it picks the inner m indices, computes the smallest and largest of
# those first, hands the two outer intervals back to the master, then computes
# the rest of its m between those two.
#
# Work items are (lo, hi, k_lo, k_hi): the interval [lo, hi] holds the
# eigenvalues k_lo..k_hi (nu(lo) < k_lo and k_hi <= nu(hi)).  Eigenvalues come
# back as brackets (mid, half-width): the final interval of Algorithm 1.  The
# outer items use the bracket ends, so they still hold their indices
# (nu(hi_s) >= k_s > k_s - 1 and nu(lo_e) < k_e <= k_e + 1).
# ---------------------------------------------------------------------------

def split_item(item, m):
    """The inner m indices of an item and its two outer index ranges, or None
    when the item holds at most 2m indices (the worker takes all of them)."""
    lo, hi, k_lo, k_hi = item
    cnt = k_hi - k_lo + 1
    if cnt <= 2 * m:
        return None
    ks = k_lo + (cnt - m) // 2
    ke = ks + m - 1
    return ks, ke, (k_lo, ks - 1), (ke + 1, k_hi)


def work_item(item, m, solve, notify):
    """One worker's handling of an item.  solve(ks, lo, hi) -> (mids,
    half_widths) for the indices ks inside [lo, hi]; notify(item) hands an
    outer item to the master.  Returns {k: value}."""
    lo, hi, k_lo, k_hi = item
    sp = split_item(item, m)
    if sp is None:
        ks = list(range(k_lo, k_hi + 1))
        mids, _ = solve(ks, lo, hi)
        return dict(zip(ks, (float(v) for v in mids)))
    ks, ke, left, right = sp
    mids, hw = solve([ks, ke], lo, hi)
    notify((lo, float(mids[0] + hw[0]), left[0], left[1]))
    notify((float(mids[1] - hw[1]), hi, right[0], right[1]))
    out = {ks: float(mids[0]), ke: float(mids[1])}
    inner = list(range(ks + 1, ke))
    if inner:
        vals, _ = solve(inner, float(mids[0] - hw[0]), float(mids[1] + hw[1]))
        out.update(zip(inner, (float(v) for v in vals)))
    return out


def master_worker_local(solvers, lo, hi, k0, k1, m):
    """The master-worker schedule with the workers' solves run in turn in this
    process (one solver per worker, e.g. one resident replica each).  Returns
    ({k: value}, number of items handed out)."""
    from collections import deque
    free = deque([(lo, hi, k0, k1)])
    out = {}
    handed = 0
    w = 0
    while free:
        item = free.popleft()
        handed += 1
        out.update(work_item(item, m, solvers[w % len(solvers)], free.append))
        w += 1
    return out, handed


_IDLE, _OUTER, _DONE = 0.0, 1.0, 2.0


def master_worker_dist(solve, lo, hi, k0, k1, m, rank, world, dist):
    """The master-worker schedule over torch.distributed ranks: rank 0 is the
    master (free list, hands out items as workers become idle), ranks >= 1 are
    workers with their own replica (solve as in work_item).  Point-to-point
    messages of float64 tensors only.  Returns {k: value} on every rank."""
    import torch
    if world < 2:
        return master_worker_local([solve], lo, hi, k0, k1, m)[0]
    msg = torch.zeros(6, dtype=torch.float64)
    if rank == 0:
        from collections import deque
        free = deque([(lo, hi, k0, k1)])
        idle = deque()
        out = {}
        total = k1 - k0 + 1
        while len(out) < total or len(idle) < world - 1:
            src = dist.recv(msg)
            kind = msg[0].item()
            if kind == _IDLE:
                idle.append(src)
            elif kind == _OUTER:
                free.append((msg[1].item(), msg[2].item(), int(msg[3].item()), int(msg[4].item())))
            else:                                   # results follow as (k, value) pairs
                buf = torch.zeros(2 * int(msg[1].item()), dtype=torch.float64)
                dist.recv(buf, src=src)
                for j in range(0, buf.numel(), 2):
                    out[int(buf[j].item())] = buf[j + 1].item()
            while free and idle:
                it = free.popleft()
                dist.send(torch.tensor([it[0], it[1], it[2], it[3], 0.0, 0.0], dtype=torch.float64), dst=idle.popleft())
            if len(out) == total and not free and len(idle) == world - 1:
                break
        for r in range(1, world):                   # stop every worker
            dist.send(torch.tensor([float("nan")] * 6, dtype=torch.float64), dst=r)
        res = [out]
    else:
        while True:
            dist.send(torch.tensor([_IDLE, 0, 0, 0, 0, 0], dtype=torch.float64), dst=0)
            dist.recv(msg, src=0)
            if torch.isnan(msg[0]):
                break
            item = (msg[0].item(), msg[1].item(), int(msg[2].item()), int(msg[3].item()))

            def notify(it):
                dist.send(torch.tensor([_OUTER, it[0], it[1], it[2], it[3], 0.0], dtype=torch.float64), dst=0)

            got = work_item(item, m, solve, notify)
            dist.send(torch.tensor([_DONE, len(got), 0, 0, 0, 0], dtype=torch.float64), dst=0)
            flat = [v for kv in sorted(got.items()) for v in kv]
            dist.send(torch.tensor(flat, dtype=torch.float64), dst=0)
        res = [None]
    dist.broadcast_object_list(res, src=0)
    return res[0]
