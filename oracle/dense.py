"""Dense FP64 oracle: the plain definitions the H^2 method approximates.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``kernel_matrix``     A_ij = f(|x_i - x_j|) for the kernels of Sec. 5.
* ``bk_ldl``            Bunch-Kaufman LDL^T (partial pivoting, alpha=(1+sqrt17)/8).
* ``inertia_dense``     nu(A - mu I) = #{j : D_jj < 0}  (Sec. 2, Sylvester).
* ``sturm_count``       the same count for a symmetric tridiagonal matrix.
* ``jacobi_eigenvalues`` cyclic Jacobi, brute force for small n.
* ``gershgorin``        an interval [a, b] holding every eigenvalue.
* ``bisect_kth``        Algorithm 1 (slicing the spectrum) for one k.
* ``bisect_many``       Algorithm 1 for several k with inertia reuse (Sec. 4.2).
"""
from __future__ import annotations

import math

import numpy as np

LAPLACE_EPS, YUKAWA_EPS, GAUSS_PLUS_INV, TRIDIAG_TEST, MIN_TEST = 0, 1, 2, 3, 4

BK_ALPHA = (1.0 + math.sqrt(17.0)) / 8.0


def kernel_values(kind: int, p, r: np.ndarray, xi=None, xj=None) -> np.ndarray:
    """f(r) for the kernel ``kind`` (Sec. 5.1 and the configs' variants).

    LAPLACE_EPS   1/(r + p0)                 (Sec. 5.1 with p0 = 1e-3)
    YUKAWA_EPS    exp(-r)/(r + p0)
    GAUSS_PLUS_INV exp(-r^2/2) + p0/(r + p1)
    TRIDIAG_TEST  2 at r = 0, -1 at r = 1, 0 otherwise (points on integers)
    MIN_TEST      min(x_i, x_j) of the first coordinates (not radial)
    """
    if kind == LAPLACE_EPS:
        return 1.0 / (r + p[0])
    if kind == YUKAWA_EPS:
        return np.exp(-r) / (r + p[0])
    if kind == GAUSS_PLUS_INV:
        return np.exp(-0.5 * r * r) + p[0] / (r + p[1])
    if kind == TRIDIAG_TEST:
        out = np.zeros_like(r)
        out[r < 0.5] = 2.0
        out[np.abs(r - 1.0) < 0.5] = -1.0
        return out
    if kind == MIN_TEST:
        return np.minimum(xi[:, None], xj[None, :])
    raise ValueError("unknown kernel kind %r" % kind)


def kernel_block(kind: int, p, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """The block A(X, Y) with rows at points X and columns at points Y."""
    diff = X[:, None, :] - Y[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    return kernel_values(kind, p, r, X[:, 0], Y[:, 0])


def kernel_matrix(kind: int, p, X: np.ndarray) -> np.ndarray:
    return kernel_block(kind, p, X, X)


def bk_ldl(A: np.ndarray, zero_pivot: float = 0.0):
    """Bunch-Kaufman LDL^T of a symmetric matrix (Bunch & Kaufman 1977).

    ``zero_pivot``: value stored for a 1x1 pivot that is exactly zero (its
    column is then zero too, so nothing is eliminated).  The dense count keeps
    0; the generalized H^2 factorization passes eps * ||A||_inf so that its
    block elimination S^{xR} D^{-1} stays finite when a cluster's redundant
    block is exactly singular (a perturbation of size eps ||A||).

    Returns (perm, L, blocks) with A[perm][:, perm] = L D L^T, L unit lower
    triangular and D block diagonal; ``blocks`` lists (start, size, E) for every
    1x1 or 2x2 diagonal block E of D.  Pivot rule, per elimination step k on the
    trailing matrix S:
      lam = max_{i>k} |S_ik| (row r = first index attaining it);
      1x1 at k          if |S_kk| >= alpha*lam  (or lam == 0);
      otherwise sig = max_{j>=k, j!=r} |S_jr|, and
      1x1 at k          if |S_kk|*sig >= alpha*lam^2,
      1x1 at r (swap)   if |S_rr| >= alpha*sig,
      2x2 at (k, r)     otherwise (r swapped to k+1).
    """
    S = np.array(A, dtype=np.float64, copy=True)
    n = S.shape[0]
    perm = np.arange(n)
    L = np.eye(n)
    blocks = []

    def swap(i, j):
        if i == j:
            return
        S[[i, j], :] = S[[j, i], :]
        S[:, [i, j]] = S[:, [j, i]]
        L[[i, j], :i] = L[[j, i], :i]
        perm[[i, j]] = perm[[j, i]]

    k = 0
    while k < n:
        akk = abs(S[k, k])
        if k + 1 < n:
            col = np.abs(S[k + 1:, k])
            r = k + 1 + int(np.argmax(col))
            lam = col[r - k - 1]
        else:
            r, lam = k, 0.0
        size = 1
        if lam == 0.0 or akk >= BK_ALPHA * lam:
            pass
        else:
            colr = np.abs(S[k:, r]).copy()
            colr[r - k] = 0.0
            sig = float(np.max(colr))
            if akk * sig >= BK_ALPHA * lam * lam:
                pass
            elif abs(S[r, r]) >= BK_ALPHA * sig:
                swap(k, r)
            else:
                swap(k + 1, r)
                size = 2
        if size == 1:
            d = S[k, k]
            if d == 0.0 and zero_pivot != 0.0:
                d = zero_pivot
                S[k, k] = d
            blocks.append((k, 1, np.array([[d]])))
            if d != 0.0 and k + 1 < n:
                l = S[k + 1:, k] / d
                L[k + 1:, k] = l
                S[k + 1:, k + 1:] -= np.outer(l, S[k + 1:, k])
            k += 1
        else:
            E = S[k:k + 2, k:k + 2].copy()
            blocks.append((k, 2, E))
            if k + 2 < n:
                C = S[k + 2:, k:k + 2]
                Lc = np.linalg.solve(E, C.T).T          # C E^{-1}
                L[k + 2:, k:k + 2] = Lc
                S[k + 2:, k + 2:] -= Lc @ C.T
            k += 2
    return perm, L, blocks


def block_inertia(E: np.ndarray):
    """(#negative eigenvalues, min |eigenvalue|) of a 1x1 or 2x2 block of D.

    A 2x2 block counts 1 if det < 0, else 2 if trace < 0, else 0.
    """
    if E.shape[0] == 1:
        d = float(E[0, 0])
        return (1 if d < 0.0 else 0), abs(d)
    a, b, c = float(E[0, 0]), float(E[1, 0]), float(E[1, 1])
    det = a * c - b * b
    tr = a + c
    neg = 1 if det < 0.0 else (2 if tr < 0.0 else 0)
    disc = math.sqrt(max(0.0, 0.25 * (a - c) ** 2 + b * b))
    eig = (0.5 * tr - disc, 0.5 * tr + disc)
    return neg, min(abs(eig[0]), abs(eig[1]))


def inertia_from_blocks(blocks):
    neg, mn = 0, math.inf
    for _, _, E in blocks:
        c, m = block_inertia(E)
        neg += c
        mn = min(mn, m)
    return neg, mn


def inertia_dense(A: np.ndarray, mu: float):
    """nu(A - mu I) = #{j : D_jj < 0} from the BK LDL^T (Sec. 2, Eq. 2);
    also returns min |pivot| (smallest |eigenvalue| of a D block)."""
    n = A.shape[0]
    _, _, blocks = bk_ldl(A - mu * np.eye(n))
    return inertia_from_blocks(blocks)


def sturm_count(diag: np.ndarray, off: np.ndarray, mu: float) -> int:
    """#{lambda < mu} of the symmetric tridiagonal (diag, off) by the Sturm
    sequence q_i = (d_i - mu) - e_{i-1}^2 / q_{i-1}; a zero q is nudged to
    a tiny negative-free value (-eps) as in LAPACK's dstebz."""
    cnt = 0
    q = 1.0
    for i in range(len(diag)):
        e2 = off[i - 1] ** 2 if i > 0 else 0.0
        q = (diag[i] - mu) - (e2 / q if i > 0 else 0.0)
        if q == 0.0:
            q = -1e-300
        if q < 0.0:
            cnt += 1
    return cnt


def jacobi_eigenvalues(A: np.ndarray, sweeps: int = 60, tol: float = 1e-15) -> np.ndarray:
    """All eigenvalues by the cyclic Jacobi method (rotations zero each
    off-diagonal entry in turn until the off-diagonal norm is negligible)."""
    S = np.array(A, dtype=np.float64, copy=True)
    n = S.shape[0]
    for _ in range(sweeps):
        off = math.sqrt(max(0.0, float(np.sum(S * S) - np.sum(np.diag(S) ** 2))))
        if off <= tol * math.sqrt(float(np.sum(S * S))):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = S[p, q]
                if apq == 0.0:
                    continue
                diff = float(S[q, q] - S[p, p])
                if abs(diff) > 1e150 * abs(apq):
                    t = float(apq) / diff                  # tiny rotation, theta ~ inf
                else:
                    theta = diff / (2.0 * float(apq))
                    t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                rp, rq = S[p, :].copy(), S[q, :].copy()
                S[p, :] = c * rp - s * rq
                S[q, :] = s * rp + c * rq
                cp, cq = S[:, p].copy(), S[:, q].copy()
                S[:, p] = c * cp - s * cq
                S[:, q] = s * cp + c * cq
    return np.sort(np.diag(S))


def eigenvalues(A: np.ndarray) -> np.ndarray:
    """All eigenvalues of the symmetric A by LAPACK (numpy eigvalsh), the
    dense comparison solver of Sec. 5 (dsyev); pinned against Jacobi in tests."""
    return np.linalg.eigvalsh(A)


def gershgorin(A: np.ndarray):
    """[min_i (A_ii - R_i), max_i (A_ii + R_i)], R_i = sum_{j != i} |A_ij|."""
    d = np.diag(A)
    R = np.sum(np.abs(A), axis=1) - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


def bisect_kth(count, k: int, a: float, b: float, tol: float):
    """Algorithm 1: while b_k - a_k >= tol: mu = midpoint; nu = count(mu);
    nu >= k -> b_k = mu else a_k = mu.  Returns ((a_k + b_k)/2, a_k, b_k, steps)."""
    ak, bk = a, b
    steps = 0
    while bk - ak >= tol:
        mu = 0.5 * (ak + bk)
        if count(mu) >= k:
            bk = mu
        else:
            ak = mu
        steps += 1
    return 0.5 * (ak + bk), ak, bk, steps


def bisect_many(count, ks, a: float, b: float, tol: float):
    """Algorithm 1 for several k at once with the inertia reuse of Sec. 4.2:
    each evaluated (mu, nu) narrows every k's interval (k <= nu -> [a, mu),
    k > nu -> [mu, b]).  Each round evaluates the distinct midpoints of the
    intervals still wider than tol.  Returns (midpoints, lo, hi, #evaluations)."""
    ks = list(ks)
    lo = {k: a for k in ks}
    hi = {k: b for k in ks}
    table = {}
    evals = 0
    while True:
        active = [k for k in ks if hi[k] - lo[k] >= tol]
        if not active:
            break
        mus = sorted({0.5 * (lo[k] + hi[k]) for k in active})
        for mu in mus:
            table[mu] = count(mu)
            evals += 1
        for k in active:
            for mu, nu in table.items():
                if lo[k] < mu < hi[k]:
                    if nu >= k:
                        hi[k] = mu
                    else:
                        lo[k] = mu
    mids = [0.5 * (lo[k] + hi[k]) for k in ks]
    return mids, [lo[k] for k in ks], [hi[k] for k in ks], evals
