"""Edge and degenerate cases of the CUDA path against the oracle, and parity at
the benchmark's own launch configuration (n = 1024 workload, 256 lanes)."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import dense, h2 as oh2

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_08618_gb300 as p
    from paper_2311_08618_gb300 import build
    build.build()
    return p


def _dense_counts(A, shifts):
    ev = dense.eigenvalues(A)
    return np.array([np.sum(ev < s) for s in shifts]), ev


def test_bench_launch_configuration_sampled_against_oracle(pkg):
    """The bench times 256-lane batches of the n = 1024 workload: sampled lanes
    of such a batch equal the H^2 oracle's counts one by one."""
    X = W.uniform_cube(1024, 2, 1)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=16, max_lanes=256)
    info = M.h2_info()
    lo, hi = info["gershgorin_lo"], info["gershgorin_hi"]
    u = W.uniform(7, 256)
    shifts = lo + (hi - lo) * (np.arange(256) + u) / 256        # the bench's first batch recipe
    got, mp = M.h2_inertia(shifts)
    ref = oh2.construct(X, W.LAPLACE_EPS, kp, 64, 16, 1.0)
    for i in range(0, 256, 37):
        want, wmp, _ = oh2.h2_inertia(ref, shifts[i])
        if min(mp[i], wmp) > 1e-10 * ref.scale:
            assert got[i] == want, (i, shifts[i])
    assert np.all(np.diff(got) >= 0)


@pytest.mark.parametrize("prec", [2, 1])
def test_bench_launch_configuration_other_precisions(pkg, prec):
    """The bench also times FP64_TC and mixed 256-lane batches of the n = 1024
    workload.  FP64_TC: sampled lanes equal the H^2 oracle's counts one by one.
    Mixed: the lanes farther than Delta = 64 * 2^-24 ||A||_inf from the dense
    spectrum (where a mixed count is exact, see h2_kth_eig) equal the dense
    counts."""
    X = W.uniform_cube(1024, 2, 1)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=16, max_lanes=256, precision=prec)
    info = M.h2_info()
    lo, hi = info["gershgorin_lo"], info["gershgorin_hi"]
    u = W.uniform(7, 256)
    shifts = lo + (hi - lo) * (np.arange(256) + u) / 256
    import torch
    d_sh = torch.tensor(shifts, dtype=torch.float64, device="cuda")
    d_c = torch.zeros(256, dtype=torch.int64, device="cuda")
    d_mp = torch.zeros(256, dtype=torch.float64, device="cuda")
    M.h2_inertia_device(d_sh, 256, d_c, d_mp)       # the bench's path (no FP64 re-run)
    torch.cuda.synchronize()
    got, mp = d_c.cpu().numpy(), d_mp.cpu().numpy()
    if prec == 2:
        ref = oh2.construct(X, W.LAPLACE_EPS, kp, 64, 16, 1.0)
        checked = 0
        for i in range(0, 256, 37):
            want, wmp, _ = oh2.h2_inertia(ref, shifts[i])
            if min(mp[i], wmp) > 1e-10 * ref.scale:
                assert got[i] == want, (i, shifts[i])
                checked += 1
        assert checked >= 5
    else:
        A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
        want, ev = _dense_counts(A, shifts)
        delta = 64 * 2.0 ** -24 * info["norm_inf"]
        far = np.abs(shifts[:, None] - ev[None, :]).min(axis=1) > delta
        assert far.sum() >= 64
        assert np.array_equal(got[far], want[far])
    assert M.h2_status()[0] == 0


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_matrices(pkg, n):
    X = W.uniform_cube(n, 2, 70 + n)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=2, rank=1, max_lanes=4)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    shifts = np.array([-1e4, 0.0, 999.0, 1001.0, 1e5])
    want, ev = _dense_counts(A, shifts)
    got, _ = M.h2_inertia(shifts)
    assert np.array_equal(got, want)
    lam, eb = M.h2_kth_eig(list(range(1, n + 1)), 1e-9)
    assert np.max(np.abs(lam - ev)) <= 1e-9 + 1e-8 * np.abs(ev).max()


def test_duplicate_points(pkg):
    """Coincident points: A has repeated rows, eigenvalue f(0) - f(0) = 0 ... the
    counts must still match the dense oracle away from the spectrum."""
    base = W.uniform_cube(60, 2, 81)
    X = np.vstack([base, base[:20]])
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=16, rank=8, max_lanes=16)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    shifts = 0.5 * (ev[1:] + ev[:-1])[::7]
    got, mp = M.h2_inertia(shifts)
    ok = mp > 1e-10 * np.abs(A).sum(1).max()
    assert np.array_equal(got[ok], np.array([np.sum(ev < s) for s in shifts])[ok])


def test_rank_zero_and_weak_admissibility(pkg):
    X = W.uniform_cube(200, 2, 82)
    kp = (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    shifts = 0.5 * (ev[1:] + ev[:-1])[::11]
    # rank 0: no far field kept -> every far block is dropped; compare with the oracle of the same A~
    M0 = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=25, rank=0, max_lanes=32)
    r0 = oh2.construct(X, W.LAPLACE_EPS, kp, 25, 0, 1.0)
    g0, m0 = M0.h2_inertia(shifts)
    for s, c, p in zip(shifts, g0, m0):
        w, wp, _ = oh2.h2_inertia(r0, s)
        if min(p, wp) > 1e-10 * r0.scale:
            assert c == w
    # eta large: everything admissible except the diagonal (weak admissibility, HSS-like)
    Mw = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=25, rank=24, eta=1e6, max_lanes=32)
    rw = oh2.construct(X, W.LAPLACE_EPS, kp, 25, 24, 1e6)
    gw, mw = Mw.h2_inertia(shifts)
    for s, c, p in zip(shifts, gw, mw):
        w, wp, _ = oh2.h2_inertia(rw, s)
        if min(p, wp) > 1e-10 * rw.scale:
            assert c == w


def test_center_admissibility_option(pkg):
    X = W.uniform_cube(256, 2, 83)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=32, rank=16, max_lanes=16, admissibility=pkg.H2_ADM_CENTER)
    ref = oh2.construct(X, W.LAPLACE_EPS, kp, 32, 16, 1.0, rule=oh2.ADM_CENTER)
    assert np.array_equal(M.h2_tree_perm(), ref.st.perm)
    shifts = np.linspace(950, 1050, 9)
    got, mp = M.h2_inertia(shifts)
    for s, c, p in zip(shifts, got, mp):
        w, wp, _ = oh2.h2_inertia(ref, s)
        if min(p, wp) > 1e-10 * ref.scale:
            assert c == w


def test_extreme_k_and_many_k(pkg):
    g = json.load(open(os.path.join(HERE, "golden", "c1_laplace2d_n1024.json")))
    X = W.uniform_cube(1024, 2, 1)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=64, rank=16, max_lanes=64)
    ks = list(range(500, 525))
    lam, eb = M.h2_kth_eig(ks, 1e-8)
    dense_ev = np.array(g["dense_eigs_500_524"])
    assert np.max(np.abs(lam - dense_ev)) <= 1e-8 + 1e-8 * g["norm2"]
    assert np.all(np.diff(lam) >= -1e-8)


def test_invalid_inputs_rejected(pkg):
    X = W.uniform_cube(64, 2, 84)
    with pytest.raises(pkg.H2Error):
        pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=1, rank=4)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=16, rank=4, max_lanes=4)
    with pytest.raises(pkg.H2Error):
        M.h2_inertia(np.array([np.nan]))
    with pytest.raises(pkg.H2Error):
        M.h2_kth_eig([1], -1.0)
    c, _ = M.h2_inertia(np.zeros(0))
    assert c.size == 0
    rc, info = M.h2_status()
    assert rc == 0 and info[0] == 0
