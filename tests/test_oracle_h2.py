"""Pins of the H^2 oracle (generalized H^2-LDL^T, Sec. 3-4) against closed
forms, the dense oracle and structural invariants.

* TRIDIAG_TEST on integer points: far blocks are exactly zero (rank 0), so the
  factorization is exact and nu must equal the closed form 2 - 2cos(j pi/(n+1)).
* MIN_TEST on 1..n: far blocks are exactly rank 1, nested row spans {1, x} need
  rank 2, fill-ins exist (distance-2 leaves); counts must equal the closed form
  1/(4 sin^2((2j-1) pi/(4n+2))).
* Kernel matrices: nu(A~ - mu I) from the generalized LDL equals the dense count
  of the written-out A~, and of A itself when mu is far from the spectrum
  relative to ||A - A~||.
"""
import math

import numpy as np
import pytest

from oracle import dense, h2
import workloads as W


def toeplitz_eigs(n):
    j = np.arange(1, n + 1)
    return np.sort(2.0 - 2.0 * np.cos(j * np.pi / (n + 1)))


def min_eigs(n):
    j = np.arange(1, n + 1)
    return np.sort(1.0 / (4.0 * np.sin((2 * j - 1) * np.pi / (4 * n + 2)) ** 2))


def gaps_shifts(ev, step=1):
    return list(0.5 * (ev[1:] + ev[:-1]))[::step] + [ev[0] - 1.0, ev[-1] + 1.0]


@pytest.mark.parametrize("n,leaf", [(64, 8), (100, 16), (37, 5)])
def test_tridiagonal_exact(n, leaf):
    h = h2.construct(W.line_points(n), W.TRIDIAG_TEST, (0, 0, 0, 0), leaf, 4, 1.0)
    assert h.stats["max_rank"] == 0
    ev = toeplitz_eigs(n)
    for mu in gaps_shifts(ev, 3):
        assert h2.h2_inertia(h, mu)[0] == int(np.sum(ev < mu))


@pytest.mark.parametrize("n,leaf", [(128, 16), (90, 12)])
def test_min_matrix_exact(n, leaf):
    h = h2.construct(W.line_points(n), W.MIN_TEST, (0, 0, 0, 0), leaf, 8, 1.0)
    assert h.stats["max_rank"] == 2 and h.stats["fill_pairs_leaf"] > 0
    A = dense.kernel_matrix(W.MIN_TEST, (0, 0, 0, 0), h.X)
    assert np.linalg.norm(A - h2.dense_approximation(h)) < 1e-12 * np.linalg.norm(A)
    ev = min_eigs(n)
    for mu in gaps_shifts(ev, 4):
        c, mp, info = h2.h2_inertia(h, mu)
        assert c == int(np.sum(ev < mu))


@pytest.fixture(scope="module")
def lap2d():
    X = W.uniform_cube(256, 2, 21)
    h = h2.construct(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), 32, 16, 1.0)
    A = dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), h.X)
    At = h2.dense_approximation(h)
    return h, A, At


def test_structure_invariants(lap2d):
    h = lap2d[0]
    st = h.st
    n = st.n
    cover = np.zeros((n, n), dtype=np.int64)
    L = st.L
    for c, d in zip(*np.nonzero(st.near[L])):
        a, b = st.rng(L, c)
        a2, b2 = st.rng(L, d)
        cover[a:b, a2:b2] += 1
    for l in range(1, L + 1):
        for c, d in zip(*np.nonzero(st.far[l])):
            a, b = st.rng(l, c)
            a2, b2 = st.rng(l, d)
            cover[a:b, a2:b2] += 1
    assert np.all(cover == 1), "every entry lies in exactly one near or far block"
    for l in range(L + 1):
        assert np.array_equal(st.near[l], st.near[l].T)
        assert not np.any(st.near[l] & st.fill[l])
        if l > 0:
            assert np.all(st.far[l][st.fill[l]])
        adj = st.near[l].copy()
        np.fill_diagonal(adj, False)
        two = adj | ((adj.astype(int) @ adj.astype(int)) > 0)
        col = st.colors[l]
        for c, d in zip(*np.nonzero(two)):
            if c != d:
                assert col[c] != col[d], "same-colour clusters are >= 3 apart"


def test_bases_orthogonal_and_nested(lap2d):
    h = lap2d[0]
    for l in range(h.st.L + 1):
        for Qc in h.Q[l]:
            assert np.allclose(Qc.T @ Qc, np.eye(Qc.shape[0]), atol=1e-13)
        for Ec in h.E[l]:
            assert np.allclose(Ec.T @ Ec, np.eye(Ec.shape[1]), atol=1e-12)


def test_compression_error(lap2d):
    h, A, At = lap2d
    assert np.linalg.norm(A - At, 2) <= 1e-8 * np.linalg.norm(A, 2)


def test_counts_equal_dense_counts(lap2d):
    h, A, At = lap2d
    ev, evt = np.linalg.eigvalsh(A), np.linalg.eigvalsh(At)
    err = np.linalg.norm(A - At, 2)
    for mu in gaps_shifts(evt, 17):
        c, mp, info = h2.h2_inertia(h, mu)
        assert c == int(np.sum(evt < mu))
        if np.min(np.abs(ev - mu)) > 2 * err:
            assert c == int(np.sum(ev < mu))


def test_count_monotone_and_gershgorin_ends(lap2d):
    h = lap2d[0]
    a, b = h.gershgorin
    assert h2.h2_inertia(h, a - 1e-6 * h.scale)[0] == 0
    assert h2.h2_inertia(h, b + 1e-6 * h.scale)[0] == h.st.n
    prev = 0
    for mu in np.linspace(950.0, 1100.0, 12):
        c = h2.h2_inertia(h, mu)[0]
        assert c >= prev
        prev = c


def test_same_colour_order_commutes(lap2d):
    """Eliminations inside one colour touch disjoint blocks, so reversing the
    order within every colour leaves the count unchanged."""
    h = lap2d[0]
    st = h.st
    mus = [960.0, 990.0, 1010.0]
    base = [h2.h2_inertia(h, mu)[0] for mu in mus]
    saved = [list(o) for o in st.order]
    try:
        for l in range(st.L + 1):
            st.order[l] = sorted(saved[l], key=lambda c: (st.colors[l][c], -c))
        assert [h2.h2_inertia(h, mu)[0] for mu in mus] == base
    finally:
        st.order = saved


def test_permuted_points_same_count():
    X = W.uniform_cube(200, 2, 31)
    p = np.argsort(W.uniform(77, 200))
    h1 = h2.construct(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), 32, 16, 1.0)
    h2b = h2.construct(X[p], W.LAPLACE_EPS, (1e-3, 0, 0, 0), 32, 16, 1.0)
    for mu in (970.0, 1000.0, 1040.0):
        assert h2.h2_inertia(h1, mu)[0] == h2.h2_inertia(h2b, mu)[0]


def test_kth_eigenvalue_3d_within_tolerance():
    X = W.uniform_cube(320, 3, 41)
    h = h2.construct(X, W.YUKAWA_EPS, (1e-3, 0, 0, 0), 40, 24, 1.0)
    A = dense.kernel_matrix(W.YUKAWA_EPS, (1e-3, 0, 0, 0), h.X)
    ev = np.linalg.eigvalsh(A)
    err = np.linalg.norm(A - h2.dense_approximation(h), 2)
    tol = 1e-6
    ks = [1, 160, 320]
    mids, lo, hi, evals = h2.kth_eigenvalues(h, ks, tol)
    for k, lam in zip(ks, mids):
        assert abs(lam - ev[k - 1]) <= 0.5 * tol + err


def test_pivoted_qr_basis_exact_rank():
    rng = W.gaussian(5, 40 * 3).reshape(40, 3)
    Y = rng @ W.gaussian(6, 3 * 20).reshape(3, 20)         # rank 3
    Q, k = h2.pivoted_qr_basis(Y, 1e-10, 10)
    assert k == 3
    assert np.linalg.norm(Y - Q[:, :3] @ (Q[:, :3].T @ Y)) < 1e-12 * np.linalg.norm(Y)
    Q2, k2 = h2.pivoted_qr_basis(Y, 1e-10, 2)                # cap binds
    assert k2 == 2


def test_sketch_matrix_moments():
    Om = h2.sketch_matrix(4000, 8, 3)
    assert np.allclose(Om.T @ Om / 4000 * 8, np.eye(8), atol=0.1)
    assert np.all(np.abs(Om) <= math.sqrt(3.0 / 8))


# ---- weak admissibility (HSS structure, Sec. 3.3) ---------------------------
@pytest.mark.parametrize("n,leaf", [(64, 8), (100, 16)])
def test_weak_tridiagonal_exact(n, leaf):
    """Under weak admissibility every off-diagonal block is far; a cluster's
    far row of the (2, -1) tridiagonal holds its first and last point's -1
    entries (rank 2, exact).  Counts equal the closed form; no fill-ins, one
    colour per level."""
    h = h2.construct(W.line_points(n), W.TRIDIAG_TEST, (0, 0, 0, 0), leaf, 4, 1.0, rule=h2.ADM_WEAK)
    assert h.stats["max_rank"] == 2 and h.stats["fill_pairs_leaf"] == 0
    assert h.stats["near_pairs_leaf"] == len(h.st.offsets[-1]) - 1       # diagonal blocks only
    assert all(len(set(c)) == 1 for c in h.st.colors)
    A = dense.kernel_matrix(W.TRIDIAG_TEST, (0, 0, 0, 0), h.X)
    assert np.linalg.norm(A - h2.dense_approximation(h)) < 1e-12 * np.linalg.norm(A)
    ev = toeplitz_eigs(n)
    for mu in gaps_shifts(ev, 3):
        assert h2.h2_inertia(h, mu)[0] == int(np.sum(ev < mu))


def test_weak_min_matrix_exact():
    n = 128
    h = h2.construct(W.line_points(n), W.MIN_TEST, (0, 0, 0, 0), 16, 8, 1.0, rule=h2.ADM_WEAK)
    A = dense.kernel_matrix(W.MIN_TEST, (0, 0, 0, 0), h.X)
    assert np.linalg.norm(A - h2.dense_approximation(h)) < 1e-12 * np.linalg.norm(A)
    ev = min_eigs(n)
    for mu in gaps_shifts(ev, 4):
        assert h2.h2_inertia(h, mu)[0] == int(np.sum(ev < mu))


def test_weak_unit_circle_counts():
    """The paper's synthetic Laplace matrix (points on the unit circle) in HSS
    form: rank 40 reproduces the dense counts at midpoints between eigenvalues."""
    X = W.unit_circle(256, 5)
    kp = (1e-3, 0, 0, 0)
    h = h2.construct(X, W.LAPLACE_EPS, kp, 32, 40, 1.0, rule=h2.ADM_WEAK)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, h.X)
    err = np.linalg.norm(A - h2.dense_approximation(h), 2) / np.linalg.norm(A, 2)
    assert err < 1e-6, err
    ev = dense.eigenvalues(A)
    shifts = gaps_shifts(ev, 17)
    gap = np.array([np.abs(ev - mu).min() for mu in shifts])
    for mu, g in zip(shifts, gap):
        if g > 1e-3:
            assert h2.h2_inertia(h, mu)[0] == int(np.sum(ev < mu))



def _near_eigenvalue_shifts(At):
    """Shifts at lambda_j(A~) -+ 1e-7 ||A~||_inf for every 16th j: the
    factorization error of the generalized LDL (truncation 1e-10 ||A||) is far
    below that distance, while a wrong recompression is not."""
    evt = np.linalg.eigvalsh(At)
    d = 1e-7 * np.abs(At).sum(axis=1).max()
    return evt, np.concatenate([evt[::16] - d, evt[::16] + d])


def test_counts_next_to_eigenvalues(lap2d):
    """nu(A~ - mu I) equals the dense count of A~ for shifts within
    1e-7 ||A~|| of its eigenvalues (the fill-ins of this matrix are
    recompressed at several levels)."""
    h, A, At = lap2d
    evt, sel = _near_eigenvalue_shifts(At)
    for mu in sel:
        assert h2.h2_inertia(h, mu)[0] == int(np.sum(evt < mu))


def _lap2d_wrong_counts(h, At):
    evt, sel = _near_eigenvalue_shifts(At)
    return sum(h2.h2_inertia(h, mu)[0] != int(np.sum(evt < mu)) for mu in sel)


def _min_matrix_wrong_counts(h, n):
    ev = min_eigs(n)
    return sum(h2.h2_inertia(h, mu)[0] != int(np.sum(ev < mu)) for mu in gaps_shifts(ev, 2))


@pytest.mark.parametrize("mistake", ["schur_sign", "no_recompression", "transposed_solve", "rotation_side"])
def test_planted_mistakes_are_caught(monkeypatch, lap2d, mistake):
    """A plausible mistake planted in the H^2 oracle (a wrong sign in the
    Schur update, the recompression left out, the triangular solve with the
    transposed factor, the rotation by V^T instead of V) must break a pin: the
    closed form of the min(i, j) matrix, or the dense counts of the 2D Laplace
    A~ next to its eigenvalues (recompression of the min matrix's fill-ins
    adds no columns, so only the second pin sees the last two)."""
    n = 90
    h = h2.construct(W.line_points(n), W.MIN_TEST, (0, 0, 0, 0), 12, 8, 1.0)
    hl, _, At = lap2d
    assert _min_matrix_wrong_counts(h, n) == 0 and _lap2d_wrong_counts(hl, At) == 0
    if mistake == "schur_sign":
        def add(self, a, b, ra, rb, delta):
            if a >= b:
                self.blk[(a, b)][np.ix_(ra, rb)] += delta
            else:
                self.blk[(b, a)][np.ix_(rb, ra)] += delta.T
        monkeypatch.setattr(h2._Level, "sub", add)
    elif mistake == "no_recompression":
        monkeypatch.setattr(h2, "_recompress", lambda *a, **k: None)
    elif mistake == "transposed_solve":
        orig = h2.solve_triangular
        monkeypatch.setattr(h2, "solve_triangular",
                            lambda L, B, lower=True, unit_diagonal=False: orig(L.T, B, lower=not lower,
                                                                               unit_diagonal=unit_diagonal))
    else:
        orig_qr = h2.pivoted_qr_basis

        def qr_transposed(Y, tol, cap):
            V, t = orig_qr(Y, tol, cap)
            return V.T.copy(), t
        monkeypatch.setattr(h2, "pivoted_qr_basis", qr_transposed)

    def caught(check):      # wrong counts, or the oracle breaking down, fail the pin
        try:
            return check() > 0
        except np.linalg.LinAlgError:
            return True
    assert caught(lambda: _min_matrix_wrong_counts(h, n)) or caught(lambda: _lap2d_wrong_counts(hl, At))


def test_center_admissibility_counts_equal_dense_counts_of_a_tilde():
    """Under the centre-distance rule (ADM_CENTER) the generalized LDL still
    counts the eigenvalues of its own (symmetric) A~ exactly, at the midpoints
    of A~'s spectrum."""
    X = W.uniform_cube(256, 2, 21)
    h = h2.construct(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), 32, 16, 1.0, rule=h2.ADM_CENTER)
    At = h2.dense_approximation(h)
    assert np.allclose(At, At.T, atol=1e-12 * np.abs(At).max())
    evt = np.linalg.eigvalsh(At)
    for mu in gaps_shifts(evt, 23):
        assert h2.h2_inertia(h, mu)[0] == int(np.sum(evt < mu))
