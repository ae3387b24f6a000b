"""Pins of the dense oracle against closed forms, brute force and invariants.

Closed forms used:
* tridiagonal Toeplitz (2, -1) of order n: lambda_j = 2 - 2 cos(j pi / (n+1));
* min(i, j) on 1..n: lambda_j = 1 / (4 sin^2((2j-1) pi / (4n+2))) (its inverse
  is the (2,-1) tridiagonal whose last diagonal entry is 1).
The error bound of Algorithm 1 is |lambda_k - lambda~_k| < eps_ev / 2 (Eq. error-bound).
"""
import math

import numpy as np
import pytest

from oracle import dense
import workloads as W


def toeplitz_eigs(n):
    j = np.arange(1, n + 1)
    return np.sort(2.0 - 2.0 * np.cos(j * np.pi / (n + 1)))


def min_eigs(n):
    j = np.arange(1, n + 1)
    return np.sort(1.0 / (4.0 * np.sin((2 * j - 1) * np.pi / (4 * n + 2)) ** 2))


def toeplitz(n):
    return 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def rand_sym(n, seed):
    A = W.gaussian(seed, n * n).reshape(n, n)
    return A + A.T


def test_sturm_matches_closed_form():
    n = 200
    ev = toeplitz_eigs(n)
    d, e = 2.0 * np.ones(n), -np.ones(n - 1)
    for mu in np.linspace(-0.5, 4.5, 41):
        assert dense.sturm_count(d, e, mu) == int(np.sum(ev < mu))


@pytest.mark.parametrize("n", [1, 2, 7, 64, 129])
def test_bk_count_tridiagonal_closed_form(n):
    ev = toeplitz_eigs(n)
    A = toeplitz(n)
    # shifts midway between consecutive eigenvalues and at the ends
    mids = list(0.5 * (ev[1:] + ev[:-1])) + [ev[0] - 0.1, ev[-1] + 0.1]
    for mu in mids:
        assert dense.inertia_dense(A, mu)[0] == int(np.sum(ev < mu))


def test_jacobi_against_closed_forms():
    for n in (5, 32, 100):
        assert np.max(np.abs(dense.jacobi_eigenvalues(toeplitz(n)) - toeplitz_eigs(n))) < 1e-12
    n = 64
    M = np.minimum.outer(np.arange(1.0, n + 1), np.arange(1.0, n + 1))
    ev = dense.jacobi_eigenvalues(M)
    # backward-stable accuracy: absolute error a small multiple of eps * ||M||
    assert np.max(np.abs(ev - min_eigs(n))) < 1e-13 * min_eigs(n)[-1]


def test_min_formula_at_256_by_jacobi():
    """The min(i,j) closed form is itself checked by brute force before use."""
    n = 256
    M = np.minimum.outer(np.arange(1.0, n + 1), np.arange(1.0, n + 1))
    ev = np.linalg.eigvalsh(M)
    assert np.max(np.abs(ev - min_eigs(n))) < 1e-13 * min_eigs(n)[-1]
    ev_j = dense.jacobi_eigenvalues(M[:128, :128])
    assert np.max(np.abs(ev_j - min_eigs(128))) < 1e-13 * min_eigs(128)[-1]


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_bk_reconstruction_and_inertia_random(seed):
    n = 48
    A = rand_sym(n, seed)
    perm, L, blocks = dense.bk_ldl(A)
    D = np.zeros_like(A)
    for s, z, E in blocks:
        D[s:s + z, s:s + z] = E
    assert np.allclose(np.tril(L), L) and np.allclose(np.diag(L), 1.0)
    assert np.max(np.abs(L @ D @ L.T - A[np.ix_(perm, perm)])) < 1e-10 * np.max(np.abs(A))
    assert any(z == 2 for _, z, _ in blocks), "random indefinite matrices exercise 2x2 pivots"
    ev = dense.jacobi_eigenvalues(A)
    for mu in list(0.5 * (ev[1:] + ev[:-1]))[::5]:
        assert dense.inertia_dense(A, mu)[0] == int(np.sum(ev < mu))


def test_bk_zero_matrix_and_exact_zero_pivot():
    # all-zero: every pivot is 0, counted non-negative (strict <)
    assert dense.inertia_dense(np.zeros((4, 4)), 0.0)[0] == 0
    # shift exactly at an eigenvalue of a diagonal matrix: strict count
    A = np.diag([1.0, 2.0, 3.0])
    assert dense.inertia_dense(A, 2.0)[0] == 1


def test_block_inertia_2x2_rules():
    assert dense.block_inertia(np.array([[0.0, 1.0], [1.0, 0.0]]))[0] == 1      # det<0
    assert dense.block_inertia(np.array([[-2.0, 1.0], [1.0, -3.0]]))[0] == 2    # det>0, tr<0
    assert dense.block_inertia(np.array([[2.0, 1.0], [1.0, 3.0]]))[0] == 0
    neg, mn = dense.block_inertia(np.array([[0.0, 2.0], [2.0, 0.0]]))
    assert neg == 1 and abs(mn - 2.0) < 1e-15


def test_kernel_matrix_definitions():
    X = np.array([[0.0, 0.0], [3.0, 4.0]])
    A = dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), X)
    assert A[0, 0] == pytest.approx(1e3) and A[0, 1] == pytest.approx(1.0 / 5.001)
    A = dense.kernel_matrix(W.YUKAWA_EPS, (1e-3, 0, 0, 0), X)
    assert A[0, 1] == pytest.approx(math.exp(-5.0) / 5.001) and A[1, 1] == pytest.approx(1e3)
    A = dense.kernel_matrix(W.GAUSS_PLUS_INV, (1e-2, 0.1, 0, 0), X)
    assert A[0, 1] == pytest.approx(math.exp(-12.5) + 1e-2 / 5.1) and A[0, 0] == pytest.approx(1.1)
    T = dense.kernel_matrix(W.TRIDIAG_TEST, (0, 0, 0, 0), W.line_points(6))
    assert np.array_equal(T, toeplitz(6))
    M = dense.kernel_matrix(W.MIN_TEST, (0, 0, 0, 0), W.line_points(5))
    assert np.array_equal(M, np.minimum.outer(np.arange(1.0, 6), np.arange(1.0, 6)))


def test_gershgorin_contains_spectrum():
    X = W.uniform_cube(150, 2, 5)
    A = dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), X)
    a, b = dense.gershgorin(A)
    ev = np.linalg.eigvalsh(A)
    assert a <= ev[0] and ev[-1] <= b
    assert dense.inertia_dense(A, a)[0] == 0 and dense.inertia_dense(A, b + 1e-9)[0] == 150


def test_count_monotone_and_permutation_invariant():
    X = W.uniform_cube(120, 3, 6)
    A = dense.kernel_matrix(W.YUKAWA_EPS, (1e-3, 0, 0, 0), X)
    p = np.argsort(W.uniform(99, 120))
    Ap = dense.kernel_matrix(W.YUKAWA_EPS, (1e-3, 0, 0, 0), X[p])
    prev = -1
    for mu in np.linspace(900.0, 1100.0, 25):
        c = dense.inertia_dense(A, mu)[0]
        assert c >= prev
        assert dense.inertia_dense(Ap, mu)[0] == c      # congruence by a permutation
        prev = c


@pytest.mark.parametrize("k", [1, 17, 50, 100])
def test_bisection_error_bound_tridiagonal(k):
    n, tol = 100, 1e-10
    ev = toeplitz_eigs(n)
    d, e = 2.0 * np.ones(n), -np.ones(n - 1)
    lam, a, b, steps = dense.bisect_kth(lambda mu: dense.sturm_count(d, e, mu), k, 0.0, 4.0, tol)
    assert abs(lam - ev[k - 1]) < 0.5 * tol
    assert b - a < tol and steps == math.ceil(math.log2(4.0 / tol))


def test_bisect_many_inertia_reuse_and_trace():
    n, tol = 40, 1e-9
    X = W.uniform_cube(n, 2, 8)
    A = dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), X)
    ev = dense.jacobi_eigenvalues(A)
    a, b = dense.gershgorin(A)
    calls = []

    def count(mu):
        calls.append(mu)
        return dense.inertia_dense(A, mu)[0]

    mids, lo, hi, evals = dense.bisect_many(count, list(range(1, n + 1)), a, b, tol)
    assert np.max(np.abs(np.array(mids) - ev)) < 0.5 * tol
    # trace = sum of eigenvalues (every k computed), within n * tol / 2
    assert abs(sum(mids) - np.trace(A)) < n * 0.5 * tol + 1e-9 * abs(np.trace(A))
    # reuse: far fewer evaluations than n independent bisections
    assert evals < n * math.ceil(math.log2((b - a) / tol))


def test_planted_sign_error_is_caught(monkeypatch):
    """A wrong sign in the Schur update of the oracle's BK must fail the pins."""
    orig = np.outer

    def bad_outer(a, b):
        return -orig(a, b)

    monkeypatch.setattr(dense.np, "outer", bad_outer)
    n = 30
    ev = toeplitz_eigs(n)
    wrong = 0
    for mu in 0.5 * (ev[1:] + ev[:-1]):
        wrong += dense.inertia_dense(toeplitz(n), mu)[0] != int(np.sum(ev < mu))
    assert wrong > 0
