"""The multi-rank path on CPU: world_size 2 over gloo (127.0.0.1).  Each rank
solves its equal share of the k-range with a host stand-in solver (exact
dense eigenvalues from the oracle); the gathered result equals the
single-process solve, and the timing reduction returns the slowest rank."""
import os

import numpy as np
import pytest

from paper_2311_08618_gb300 import sharding


def test_equal_distribution_shapes():
    parts = sharding.equal_distribution(list(range(10, 0, -1)), 3)
    assert parts == [[1, 2, 3, 4], [5, 6, 7], [8, 9, 10]]
    assert sharding.equal_distribution([5], 4) == [[5], [], [], []]
    assert sum(len(p) for p in sharding.equal_distribution(list(range(100)), 7)) == 100


def _worker(rank, world, port, ks, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as W
    from oracle import dense
    X = W.uniform_cube(64, 2, 61)
    ev = dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), X))
    res = sharding.solve_sharded(lambda mine: [ev[k - 1] for k in mine], ks, rank, world, dist)
    slow = sharding.max_over_ranks(float(rank + 1), dist)
    out_q.put((rank, res, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_solve_matches_single_process():
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ks = [1, 5, 17, 32, 33, 50, 64]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ks, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import workloads as W
    from oracle import dense
    X = W.uniform_cube(64, 2, 61)
    ev = dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), X))
    for rank, res, slow in got:
        assert sorted(res) == ks
        assert all(res[k] == ev[k - 1] for k in ks)
        assert slow == 2.0


def _standin(ev, tol, seen=None):
    """Worker solve stand-in: exact eigenvalues as brackets of half-width
    tol/2; asserts that the interval it is given holds every requested index
    (lambda_k in [lo, hi), i.e. nu(lo) < k <= nu(hi))."""
    def solve(ks, lo, hi):
        for k in ks:
            assert lo <= ev[k - 1] < hi, (k, lo, hi, ev[k - 1])
            if seen is not None:
                seen.append(k)
        return [ev[k - 1] for k in ks], [0.5 * tol] * len(ks)
    return solve


def _circle_eigs():
    import workloads as W
    from oracle import dense
    X = W.unit_circle(256, 5)
    return dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), X))


def test_master_worker_splits_and_covers_every_index():
    ev = _circle_eigs()
    seen = []
    k0, k1, m = 60, 190, 8
    out, handed = sharding.master_worker_local([_standin(ev, 1e-9, seen)] * 3, ev[0] - 1.0, ev[-1] + 1.0,
                                               k0, k1, m)
    assert sorted(out) == list(range(k0, k1 + 1))
    assert all(out[k] == ev[k - 1] for k in out)
    assert handed > 3                            # the range was split into free intervals
    assert sorted(seen) == list(range(k0, k1 + 1))   # every index solved exactly once
    assert sharding.split_item((0.0, 1.0, 1, 16), 8) is None
    assert sharding.split_item((0.0, 1.0, 1, 17), 8) == (5, 12, (1, 4), (13, 17))


def _mw_worker(rank, world, port, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ev = _circle_eigs()
    res = sharding.master_worker_dist(_standin(ev, 1e-9), ev[0] - 1.0, ev[-1] + 1.0, 20, 120, 6, rank, world, dist)
    out_q.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_three_rank_gloo_master_worker():
    """Rank 0 is the master, ranks 1 and 2 are workers (Sec. 4.2, second
    algorithm): every rank ends with every eigenvalue of the index range."""
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_mw_worker, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(3)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ev = _circle_eigs()
    for rank, res in got:
        assert sorted(res) == list(range(20, 121))
        assert all(res[k] == ev[k - 1] for k in res)
