"""Host logic of the serving layer (no GPU): how a round's shifts are planned
over a matrix's lanes, how brackets narrow with every evaluated (mu, nu) pair
(Algorithm 1), and how new requests start from the tightest bracket in the
matrix's table (inertia reuse, Sec. 4.2).  Counts come from a known spectrum:
nu(mu) = #{lambda_j < mu} for the tridiagonal Toeplitz closed form."""
import bisect

import numpy as np

from paper_2311_08618_gb300.serving import narrow, plan_shifts, tightest_bracket


def toeplitz_eigs(n):
    j = np.arange(1, n + 1)
    return np.sort(2.0 - 2.0 * np.cos(j * np.pi / (n + 1)))


def test_plan_shifts_sections_and_sharing():
    assert plan_shifts([], 8) == []
    s = plan_shifts([(0.0, 1.0)], 4)                      # 5-section of one interval
    assert np.allclose(s, [0.2, 0.4, 0.6, 0.8])
    s = plan_shifts([(0.0, 1.0), (2.0, 3.0)], 5)          # 3 + 2 lanes
    assert np.allclose(s, [0.25, 0.5, 0.75, 2.0 + 1 / 3, 2.0 + 2 / 3])
    s = plan_shifts([(0.0, 1.0), (0.0, 1.0), (2.0, 4.0)], 2)   # duplicates share
    assert np.allclose(s, [0.5, 3.0])
    s = plan_shifts([(float(i), i + 1.0) for i in range(6)], 4)  # more intervals than lanes
    assert np.allclose(s, [0.5, 1.5, 2.5, 3.5])
    for lanes in (1, 3, 16):
        s = plan_shifts([(0.0, 1.0), (5.0, 9.0)], lanes)
        assert len(s) == lanes and all(0.0 < x < 1.0 or 5.0 < x < 9.0 for x in s)


def test_narrow_keeps_the_eigenvalue_inside():
    ev = toeplitz_eigs(40)
    nu = lambda mu: int(np.sum(ev < mu))
    for k in (1, 7, 20, 40):
        lo, hi = -1.0, 5.0
        mus = list(np.linspace(-0.5, 4.5, 23))
        lo, hi = narrow(lo, hi, k, mus, [nu(m) for m in mus])
        assert nu(lo) < k <= nu(hi)
        assert lo < ev[k - 1] < hi
    # a pair outside the bracket changes nothing
    assert narrow(1.0, 2.0, 3, [0.5, 2.5], [0, 40]) == (1.0, 2.0)


def test_tightest_bracket_from_table():
    ev = toeplitz_eigs(30)
    nu = lambda mu: int(np.sum(ev < mu))
    mus = sorted([-1.0, 5.0] + list(np.linspace(0.0, 4.0, 17)))
    nus = [nu(m) for m in mus]
    for k in range(1, 31):
        lo, hi = tightest_bracket(-1.0, 5.0, mus, nus, k)
        assert nu(lo) < k <= nu(hi)
        i = bisect.bisect_left(mus, ev[k - 1])
        assert lo == mus[i - 1] and hi == mus[i]       # the neighbouring table entries


def test_rounds_of_shared_lanes_reach_tolerance_with_reuse():
    """The server's round logic, replayed on the host: requests for several k
    share 8 lanes per round; every pair narrows every request and enters the
    table; a request arriving later starts from the table and needs fewer
    rounds than the first ones."""
    ev = toeplitz_eigs(64)
    nu = lambda mu: int(np.sum(ev < mu))
    lo0, hi0, lanes, tol = -0.1, 4.1, 8, 1e-9
    table_mu, table_nu = [lo0, hi0], [0, 64]

    def run(ks):
        reqs = [[k, *tightest_bracket(lo0, hi0, table_mu, table_nu, k), 0] for k in ks]
        active = [r for r in reqs if r[2] - r[1] >= tol]
        while active:
            shifts = plan_shifts([(r[1], r[2]) for r in active], lanes)
            counts = [nu(m) for m in shifts]
            for m, c in zip(shifts, counts):
                i = bisect.bisect_left(table_mu, m)
                table_mu.insert(i, m)
                table_nu.insert(i, c)
            for r in active:
                r[1], r[2] = narrow(r[1], r[2], r[0], shifts, counts)
                r[3] += 1
            active = [r for r in active if r[2] - r[1] >= tol]
        return reqs

    first = run([10, 32, 33])
    for k, lo, hi, rounds in first:
        assert abs(0.5 * (lo + hi) - ev[k - 1]) < 0.5 * tol
    later = run([32])
    assert abs(0.5 * (later[0][1] + later[0][2]) - ev[31]) < 0.5 * tol
    assert later[0][3] < min(r[3] for r in first)
