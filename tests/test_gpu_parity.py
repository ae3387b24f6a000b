"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: counts bit-exact with the H^2 oracle for every shift whose
smallest |pivot| exceeds 1e-10 * ||A||; closed-form matrices exactly; k-th
eigenvalues within tol + 1e-8 ||A|| of the dense oracle.
"""
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


def toeplitz_eigs(n):
    j = np.arange(1, n + 1)
    return np.sort(2.0 - 2.0 * np.cos(j * np.pi / (n + 1)))


def min_eigs(n):
    j = np.arange(1, n + 1)
    return np.sort(1.0 / (4.0 * np.sin((2 * j - 1) * np.pi / (4 * n + 2)) ** 2))


def shifts_between(ev, step=1):
    return np.array(list(0.5 * (ev[1:] + ev[:-1]))[::step] + [ev[0] - 1.0, ev[-1] + 1.0])


@pytest.mark.parametrize("n,leaf,lanes", [(100, 16, 64), (37, 5, 8), (128, 8, 200)])
def test_tridiagonal_closed_form(pkg, n, leaf, lanes):
    M = pkg.H2Matrix(W.line_points(n) - 1.0, W.TRIDIAG_TEST, (0, 0, 0, 0), leaf=leaf, rank=4,
                     max_lanes=lanes)
    ev = toeplitz_eigs(n)
    s = shifts_between(ev)
    got, mp = M.h2_inertia(s)
    assert np.array_equal(got, np.array([np.sum(ev < x) for x in s]))


@pytest.mark.parametrize("n,leaf", [(128, 16), (90, 12)])
def test_min_matrix_closed_form(pkg, n, leaf):
    M = pkg.H2Matrix(W.line_points(n), W.MIN_TEST, (0, 0, 0, 0), leaf=leaf, rank=8, max_lanes=32)
    assert M.h2_info()["max_rank"] == 2
    ev = min_eigs(n)
    s = shifts_between(ev, 2)
    got, mp = M.h2_inertia(s)
    assert np.array_equal(got, np.array([np.sum(ev < x) for x in s]))


def _compare_with_oracle(pkg, X, kind, kp, leaf, rank, shifts, lanes=64):
    M = pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=lanes)
    ref = oh2.construct(X, kind, kp, leaf, rank, 1.0)
    # same tree and same build ranks
    assert np.array_equal(M.h2_tree_perm(), ref.st.perm)
    for l in range(ref.st.L + 1):
        assert list(M.h2_level_ranks(l)) == list(ref.ranks[l]), l
    info = M.h2_info()
    assert info["norm_inf"] == pytest.approx(ref.scale, rel=1e-12)
    got, mp = M.h2_inertia(shifts)
    thr = 1e-10 * ref.scale
    checked = 0
    for s, c, p in zip(shifts, got, mp):
        want, wmp, _ = oh2.h2_inertia(ref, s)
        if min(p, wmp) > thr:
            assert c == want, (s, c, want, p, wmp)
            checked += 1
    assert checked >= len(shifts) // 2
    return M, ref


def test_laplace2d_counts_match_oracle(pkg):
    X = W.uniform_cube(256, 2, 21)
    kp = (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 9)
    _compare_with_oracle(pkg, X, W.LAPLACE_EPS, kp, 32, 16, s)


def test_laplace2d_counts_next_to_eigenvalues(pkg):
    """Shifts within 1e-7 ||A~|| of the eigenvalues of the oracle's A~ (every
    8th one, both sides): far above the factorization error of either side,
    far below the effect of a wrong recompression (the oracle's planted
    mistakes flip such counts), so the GPU's recompression and rotation are
    pinned, not only its pivots."""
    X = W.uniform_cube(256, 2, 21)
    kp = (1e-3, 0, 0, 0)
    ref = oh2.construct(X, W.LAPLACE_EPS, kp, 32, 16, 1.0)
    At = oh2.dense_approximation(ref)
    evt = np.linalg.eigvalsh(At)
    d = 1e-7 * np.abs(At).sum(axis=1).max()
    s = np.concatenate([evt[::8] - d, evt[::8] + d])
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=32, rank=16, max_lanes=64)
    got, mp = M.h2_inertia(s)
    want = np.array([np.sum(evt < x) for x in s])
    sure = mp > 1e-10 * ref.scale
    assert sure.sum() >= 0.9 * len(s)
    assert np.array_equal(got[sure], want[sure])
    assert M.h2_status()[0] == 0
    M.close()


def test_yukawa3d_ragged_counts_match_oracle(pkg):
    X = W.uniform_cube(300, 3, 22)          # leaves of 37 and 38 points
    kp = (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(W.YUKAWA_EPS, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 13)
    _compare_with_oracle(pkg, X, W.YUKAWA_EPS, kp, 40, 20, s, lanes=16)


def test_single_cluster_is_dense_ldl(pkg):
    X = W.uniform_cube(50, 2, 23)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=8, max_lanes=8)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 3)
    got, _ = M.h2_inertia(s)
    assert np.array_equal(got, [dense.inertia_dense(A, x)[0] for x in s])


def test_gaussian_kernel_counts(pkg):
    X = W.cylinder_lattice(400, 4)
    kp = (1e-2, 0.1, 0, 0)
    A = dense.kernel_matrix(W.GAUSS_PLUS_INV, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 23)
    _compare_with_oracle(pkg, X, W.GAUSS_PLUS_INV, kp, 32, 16, s, lanes=32)


def test_determinism_and_batching(pkg):
    X = W.uniform_cube(256, 2, 24)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=32, rank=16, max_lanes=7)
    s = np.linspace(900, 1100, 23)
    a, _ = M.h2_inertia(s)
    b, _ = M.h2_inertia(s)
    c, _ = M.h2_inertia(s[::-1])
    assert np.array_equal(a, b) and np.array_equal(a, c[::-1])
    assert np.all(np.diff(a) >= 0)
    info = M.h2_info()
    lo, hi = info["gershgorin_lo"], info["gershgorin_hi"]
    e, _ = M.h2_inertia([lo - 1e-6 * info["norm_inf"], hi + 1e-6 * info["norm_inf"]])
    assert list(e) == [0, 256]


def test_c1_kth_eigenvalue_against_dense_oracle(pkg):
    g = json.load(open(os.path.join(HERE, "golden", "c1_laplace2d_n1024.json")))
    X = W.uniform_cube(1024, 2, 1)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=64, rank=16, max_lanes=64)
    info = M.h2_info()
    assert info["norm_inf"] == pytest.approx(g["norm_inf"], rel=1e-12)
    assert [info["gershgorin_lo"], info["gershgorin_hi"]] == pytest.approx(g["gershgorin"], rel=1e-12)
    tol = 1e-8
    lam, eb = M.h2_kth_eig([512], tol)
    assert eb[0] < 0.5 * tol
    lam_dense = g["dense_eigs_500_524"][512 - 500]
    assert abs(lam[0] - lam_dense) <= tol + 1e-8 * g["norm2"]
    assert abs(lam[0] - g["h2_lambda_512_tol1e-8"]) <= tol


def test_multi_k_with_reuse(pkg):
    X = W.uniform_cube(200, 2, 25)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=25, rank=12, max_lanes=16)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    ks = [1, 2, 50, 100, 101, 199, 200]
    tol = 1e-7
    lam, eb = M.h2_kth_eig(ks, tol)
    nrm = np.max(np.abs(ev))
    for k, x in zip(ks, lam):
        assert abs(x - ev[k - 1]) <= tol + 1e-8 * nrm, (k, x, ev[k - 1])


def test_kth_rejects_bad_k(pkg):
    X = W.uniform_cube(64, 2, 26)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=16, rank=8, max_lanes=4)
    with pytest.raises(pkg.H2Error):
        M.h2_kth_eig([0], 1e-8)
    with pytest.raises(pkg.H2Error):
        M.h2_kth_eig([65], 1e-8)
