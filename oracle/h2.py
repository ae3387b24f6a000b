"""Plain FP64 CPU oracle of the generalized H^2-LDL^T factorization and its
inertia count (Apriansyah & Yokota, Sec. 3-4).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written for a reader
who checks it against the paper: every step is a loop over clusters with
numpy/scipy primitives, no blocking, batching or fusion.

Readings taken where the paper is silent (each also listed in the design notes):

* Tree: binary; a cluster is split at its median (sizes floor/ceil of half)
  along the longest axis of its points' bounding box (first axis on ties), the
  points ordered by that coordinate with a stable sort.  All leaves sit at
  depth L = ceil(log2(n / leaf)).
* Admissibility of a cluster pair (c, d), c != d, on point bounding boxes:
  ADM_BOX    max(diam c, diam d) <= eta * dist(box c, box d);
  ADM_CENTER (diam c + diam d) / 2 <= eta * |center c - center d|;
  ADM_WEAK   always (weak admissibility: the HSS structure of Sec. 3.3, where
             every off-diagonal block is low-rank; no fill-ins arise).
  The block tree is built top-down from the root pair; a leaf pair that is not
  admissible is "near" (dense).
* Fill-in closure: eliminating cluster p updates every pair (a, b) of its near
  neighbours (Eq. blr2-diag-schur applied to the dense off-diagonal blocks,
  Sec. 3.4).  Each such pair that is not near is a fill-in block.  So that the
  recompressed fill-ins can always be merged into the parent level (Sec. 3.4),
  the parent pair of every near-or-fill pair is made inadmissible ("forced
  near"), bottom-up; the far pairs with explicit couplings at a level are the
  non-near pairs whose parents are near.
* Bases: the shared basis of cluster c spans its far row A_{l;c,+} (all
  columns outside its near clusters, which includes every ancestor's far
  field, so the bases nest) -- Eq. shared-bases / transfer-matrices.  The
  rank-revealing QR is Householder QR with column pivoting of the randomized
  sketch A_{l;c,+} Omega (Halko-Martinsson-Tropp range finder), Omega drawn
  from SplitMix64, stopped when the Frobenius norm of the unpivoted remainder
  is <= tol = eps_h2 * ||A||_inf, or at the rank cap.
* Elimination order within a level: colour-major order of a greedy
  distance-2 colouring of the near graph (same-colour clusters share no near
  neighbour, so their eliminations commute).
* Recompression (Sec. 3.4): just before cluster p is factorized, the fill-in
  blocks of row p are concatenated; since [U^R U^S] is square orthogonal and
  the far field lies in U^S, only their redundant rows can leave the
  skeleton span.  A pivoted QR of those rows (same tolerance, capped at
  ``fill_cap`` total skeleton columns) gives an orthogonal rotation of p's
  redundant coordinates; its leading t columns join the skeleton, and the
  remaining redundant rows of the fill-in blocks (norm <= tol) are dropped.
* Local pivoting: Bunch-Kaufman within each cluster's redundant block.  A 1x1
  pivot that is exactly zero (the cluster's redundant block is exactly
  singular while it still couples to other blocks) is replaced by
  eps * ||A||_inf, a perturbation of that size; min |pivot| then flags the shift.
* Inertia: nu = total number of negative pivots over all levels (Sec. 4,
  Sylvester); a 2x2 pivot counts by det and trace.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular

from . import dense
from workloads import splitmix64

ADM_BOX, ADM_CENTER, ADM_WEAK = 0, 1, 2


# ----------------------------------------------------------------------------
# Cluster tree and block structure (Sec. 3.1 notation: A_{level; row, col})
# ----------------------------------------------------------------------------

@dataclass
class Structure:
    n: int
    L: int
    perm: np.ndarray                    # tree position -> original point index
    offsets: list                       # offsets[l] : (nc+1,) ranges in tree order
    near: list                          # near[l] : bool (nc, nc), dense blocks
    fill: list                          # fill[l] : bool, non-near pairs with a common near neighbour
    far: list                           # far[l]  : bool, explicit couplings (parents near)
    order: list                         # order[l]: elimination order (colour-major)
    colors: list                        # colors[l]: colour of each cluster

    def nclusters(self, l):
        return len(self.offsets[l]) - 1

    def rng(self, l, c):
        return self.offsets[l][c], self.offsets[l][c + 1]


def build_tree(points: np.ndarray, leaf: int):
    n = points.shape[0]
    L = int(math.ceil(math.log2(n / leaf))) if n > leaf else 0
    order = np.arange(n)
    offsets = [np.array([0, n])]
    for _ in range(L):
        prev = offsets[-1]
        nxt = [0]
        for c in range(len(prev) - 1):
            s, e = prev[c], prev[c + 1]
            sub = order[s:e]
            X = points[sub]
            ext = X.max(axis=0) - X.min(axis=0)
            ax = int(np.argmax(ext))
            o = np.argsort(X[:, ax], kind="stable")
            order[s:e] = sub[o]
            h = (e - s) // 2
            nxt += [s + h, e]
        offsets.append(np.array(nxt))
    return L, order, offsets


def _boxes(points, perm, offs):
    nc = len(offs) - 1
    lo = np.empty((nc, points.shape[1]))
    hi = np.empty((nc, points.shape[1]))
    for c in range(nc):
        X = points[perm[offs[c]:offs[c + 1]]]
        lo[c], hi[c] = X.min(axis=0), X.max(axis=0)
    return lo, hi


def admissible(lo, hi, c, d, eta, rule):
    """Strong admissibility of the cluster pair (c, d) (readings above)."""
    if c == d:
        return False
    if rule == ADM_WEAK:
        return True
    dc = math.sqrt(float(np.sum((hi[c] - lo[c]) ** 2)))
    dd = math.sqrt(float(np.sum((hi[d] - lo[d]) ** 2)))
    if rule == ADM_BOX:
        gap = np.maximum(0.0, np.maximum(lo[c] - hi[d], lo[d] - hi[c]))
        return max(dc, dd) <= eta * math.sqrt(float(np.sum(gap * gap)))
    cc, cd = 0.5 * (lo[c] + hi[c]), 0.5 * (lo[d] + hi[d])
    return 0.5 * (dc + dd) <= eta * math.sqrt(float(np.sum((cc - cd) ** 2)))


def distance2_coloring(near: np.ndarray):
    """Greedy colouring in cluster-index order: a cluster takes the smallest
    colour unused within graph distance <= 2 in the near graph."""
    nc = near.shape[0]
    adj = near.copy()
    np.fill_diagonal(adj, False)
    two = adj | ((adj.astype(np.int64) @ adj.astype(np.int64)) > 0)
    np.fill_diagonal(two, False)
    colors = -np.ones(nc, dtype=np.int64)
    for c in range(nc):
        used = set(colors[two[c]].tolist())
        k = 0
        while k in used:
            k += 1
        colors[c] = k
    order = sorted(range(nc), key=lambda c: (colors[c], c))
    return colors, order


def build_structure(points: np.ndarray, leaf: int, eta: float, rule: int = ADM_BOX) -> Structure:
    n = points.shape[0]
    L, perm, offsets = build_tree(points, leaf)
    boxes = [_boxes(points, perm, offsets[l]) for l in range(L + 1)]
    # top-down block tree: children of a near pair are near or far
    near = [np.ones((1, 1), dtype=bool)]
    for l in range(1, L + 1):
        nc = len(offsets[l]) - 1
        lo, hi = boxes[l]
        m = np.zeros((nc, nc), dtype=bool)
        P, Q = np.nonzero(near[l - 1])
        for p, q in zip(P, Q):
            for c in (2 * p, 2 * p + 1):
                for d in (2 * q, 2 * q + 1):
                    if not admissible(lo, hi, c, d, eta, rule):
                        m[c, d] = True
        near.append(m)
    # bottom-up fill-in closure: parents of near-or-fill pairs are forced near
    fill = [None] * (L + 1)
    for l in range(L, 0, -1):
        N = near[l].astype(np.int64)
        X = near[l] | ((N @ N) > 0)
        fill[l] = X & ~near[l]
        P, Q = np.nonzero(X)
        near[l - 1][P // 2, Q // 2] = True
    fill[0] = np.zeros((1, 1), dtype=bool)
    far = [np.zeros((1, 1), dtype=bool)]
    for l in range(1, L + 1):
        nc = len(offsets[l]) - 1
        par = np.arange(nc) // 2
        far.append(near[l - 1][par[:, None], par[None, :]] & ~near[l])
    order, colors = [], []
    for l in range(L + 1):
        col, o = distance2_coloring(near[l])
        colors.append(col)
        order.append(o)
    return Structure(n, L, perm, offsets, near, fill, far, order, colors)


# ----------------------------------------------------------------------------
# Construction (Sec. 3.1): nested orthogonal bases, couplings, near blocks
# ----------------------------------------------------------------------------

def pivoted_qr_basis(Y: np.ndarray, tol: float, cap: int):
    """Householder QR with column pivoting of Y (m x s), stopped when the
    Frobenius norm of the not-yet-pivoted remainder is <= tol or after ``cap``
    steps.  Returns (Q, k): Q = H_1 ... H_k (m x m orthogonal), whose first k
    columns are the skeleton basis U^S and the rest the redundant basis U^R."""
    m = Y.shape[0]
    R = np.array(Y, dtype=np.float64, copy=True)
    s = R.shape[1]
    vs = []
    k = 0
    while k < min(m, s, cap):
        norms = np.sum(R[k:, k:] ** 2, axis=0)
        if math.sqrt(float(np.sum(norms))) <= tol:
            break
        j = k + int(np.argmax(norms))
        R[:, [k, j]] = R[:, [j, k]]
        x = R[k:, k]
        nx = math.sqrt(float(x @ x))
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = math.sqrt(float(v @ v))
        if nv > 0.0:
            v /= nv
            R[k:, k:] -= 2.0 * np.outer(v, v @ R[k:, k:])
        vs.append((k, v, nv > 0.0))
        k += 1
    Q = np.eye(m)
    for j, v, used in reversed(vs):
        if used:
            Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    return Q, k


def sketch_matrix(n: int, s: int, seed: int) -> np.ndarray:
    """Omega (n x s), entries (2u - 1) * sqrt(3/s) with u the top 53 bits of
    SplitMix64 output number i*s + c (state ``seed``): E[Omega Omega^T] = I."""
    u = (splitmix64(seed, n * s) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return ((2.0 * u - 1.0) * math.sqrt(3.0 / s)).reshape(n, s)


@dataclass
class H2Matrix:
    st: Structure
    kind: int
    kparams: tuple
    X: np.ndarray                  # points in tree order
    scale: float                   # ||A||_inf
    tol: float                     # eps_h2 * ||A||_inf
    fill_cap: int
    ranks: list                    # ranks[l][c] = build skeleton rank
    Q: list                        # Q[l][c] : orthogonal basis (leaf: m x m; upper: transfer)
    E: list                        # E[l][c] : expanded skeleton basis in point space
    coupling: list                 # coupling[l][(c, d)] for far pairs (c > d and c < d)
    near_blocks: dict              # leaf near blocks Q_c^T A_cd Q_d for c >= d
    gershgorin: tuple = (0.0, 0.0)
    stats: dict = field(default_factory=dict)


def construct(points, kind, kparams, leaf, rank, eta, eps_h2=1e-10, rule=ADM_BOX,
              sketch_cols=None, seed=0x5EED, fill_cap=None) -> H2Matrix:
    """Level-by-level H^2 construction (Eqs. shared-bases, transfer-matrices,
    dense_skeleton, lr_skeleton)."""
    st = build_structure(points, leaf, eta, rule)
    X = np.asarray(points, dtype=np.float64)[st.perm]
    n, L = st.n, st.L
    A = dense.kernel_matrix(kind, kparams, X)            # plain definition, O(n^2)
    scale = float(np.max(np.sum(np.abs(A), axis=1)))
    ga, gb = dense.gershgorin(A)
    tol = eps_h2 * scale
    s = sketch_cols if sketch_cols is not None else rank + 16
    Om = sketch_matrix(n, s, seed)
    if fill_cap is None:
        fill_cap = 2 * rank
    ranks = [None] * (L + 1)
    Q = [None] * (L + 1)
    E = [None] * (L + 1)
    for l in range(L, -1, -1):
        nc = st.nclusters(l)
        ranks[l], Q[l], E[l] = [], [], []
        for c in range(nc):
            a, b = st.rng(l, c)
            nearcols = np.zeros(n, dtype=bool)
            for d in np.nonzero(st.near[l][c])[0]:
                a2, b2 = st.rng(l, d)
                nearcols[a2:b2] = True
            farc = ~nearcols
            Y = A[a:b][:, farc] @ Om[farc]               # A_{l;c,+} Omega
            if l < L:
                c1, c2 = 2 * c, 2 * c + 1
                a1, b1 = st.rng(l + 1, c1)
                Y = np.vstack([E[l + 1][c1].T @ Y[:b1 - a], E[l + 1][c2].T @ Y[b1 - a:]])
            Qc, r = pivoted_qr_basis(Y, tol, rank)
            ranks[l].append(r)
            Q[l].append(Qc)
            if l == L:
                E[l].append(Qc[:, :r])
            else:
                c1, c2 = 2 * c, 2 * c + 1
                r1, r2 = ranks[l + 1][c1], ranks[l + 1][c2]
                Ec1, Ec2 = E[l + 1][c1], E[l + 1][c2]
                blk = np.zeros((Ec1.shape[0] + Ec2.shape[0], r1 + r2))
                blk[:Ec1.shape[0], :r1] = Ec1
                blk[Ec1.shape[0]:, r1:] = Ec2
                E[l].append(blk @ Qc[:, :r])
    coupling = [dict() for _ in range(L + 1)]
    for l in range(1, L + 1):
        P, Qi = np.nonzero(st.far[l])
        for c, d in zip(P, Qi):
            a, b = st.rng(l, c)
            a2, b2 = st.rng(l, d)
            coupling[l][(int(c), int(d))] = E[l][c].T @ A[a:b, a2:b2] @ E[l][d]
    near_blocks = {}
    P, Qi = np.nonzero(st.near[L])
    for c, d in zip(P, Qi):
        if c >= d:
            a, b = st.rng(L, c)
            a2, b2 = st.rng(L, d)
            near_blocks[(int(c), int(d))] = Q[L][c].T @ A[a:b, a2:b2] @ Q[L][d]
    h = H2Matrix(st, kind, tuple(kparams), X, scale, tol, fill_cap, ranks, Q, E, coupling,
                 near_blocks, (ga, gb))
    h.stats = {"max_rank": max(max(r) if r else 0 for r in ranks),
               "near_pairs_leaf": int(st.near[L].sum()),
               "fill_pairs_leaf": int(st.fill[L].sum()) if L > 0 else 0}
    return h


def dense_approximation(h: H2Matrix) -> np.ndarray:
    """The H^2 matrix A~ written out densely (tree order): near blocks at the
    leaves plus E_c C_cd E_d^T for every far pair at every level."""
    st = h.st
    L = st.L
    out = np.zeros((st.n, st.n))
    for (c, d), B in h.near_blocks.items():
        a, b = st.rng(L, c)
        a2, b2 = st.rng(L, d)
        blk = h.Q[L][c] @ B @ h.Q[L][d].T
        out[a:b, a2:b2] = blk
        out[a2:b2, a:b] = blk.T
    for l in range(1, L + 1):
        for (c, d), C in h.coupling[l].items():
            a, b = st.rng(l, c)
            a2, b2 = st.rng(l, d)
            out[a:b, a2:b2] = h.E[l][c] @ C @ h.E[l][d].T
    return out


# ----------------------------------------------------------------------------
# Generalized H^2-LDL^T of A~ - sigma I and its inertia (Sec. 3.2-3.4, Sec. 4)
# ----------------------------------------------------------------------------

class _Level:
    """Blocks of one level: dense near and fill-in blocks stored for c >= d."""

    def __init__(self, dims, ranks):
        self.dim = list(dims)
        self.rk = list(ranks)
        self.elim = [False] * len(dims)
        self.blk = {}

    def get(self, a, b):
        return self.blk[(a, b)] if a >= b else self.blk[(b, a)].T

    def sub(self, a, b, ra, rb, delta):
        """blk(a, b)[ra, rb] -= delta (symmetric storage)."""
        if a >= b:
            self.blk[(a, b)][np.ix_(ra, rb)] -= delta
        else:
            self.blk[(b, a)][np.ix_(rb, ra)] -= delta.T

    def live(self, a):
        """Coordinates of cluster a still in the trailing matrix."""
        return np.arange(self.rk[a]) if self.elim[a] else np.arange(self.dim[a])


def _bk_solve_parts(Braw, zero_pivot):
    perm, Lf, blocks = dense.bk_ldl(Braw, zero_pivot)
    Dm = np.zeros_like(Braw)
    for s0, sz, Eb in blocks:
        Dm[s0:s0 + sz, s0:s0 + sz] = Eb
    return perm, Lf, Dm, blocks


def _recompress(lv: _Level, st: Structure, l: int, p: int, tol: float, cap: int, info):
    """Sec. 3.4 recompression of row/column p just before its factorization."""
    nc = st.nclusters(l)
    fq = [q for q in range(nc) if st.fill[l][p, q]]
    r0, m = lv.rk[p], lv.dim[p]
    Rs = np.arange(r0, m)
    if not fq or len(Rs) == 0:
        return
    Z = np.hstack([lv.get(p, q)[np.ix_(Rs, lv.live(q))] for q in fq])
    V, t = pivoted_qr_basis(Z, tol, max(0, min(cap, m) - r0))
    resid = Z - V[:, :t] @ (V[:, :t].T @ Z)
    info["trunc"] = max(info["trunc"], float(np.linalg.norm(resid)))
    # rotate the redundant coordinates of p in every block of row/column p
    for key in list(lv.blk.keys()):
        a, b = key
        B = lv.blk[key]
        if a == p:
            B[Rs, :] = V.T @ B[Rs, :]
        if b == p:
            B[:, Rs] = B[:, Rs] @ V
    # drop the remaining redundant rows of the fill-in blocks (norm <= tol)
    for q in fq:
        if p >= q:
            lv.blk[(p, q)][r0 + t:, :] = 0.0
        else:
            lv.blk[(q, p)][:, r0 + t:] = 0.0
    lv.rk[p] = r0 + t
    info["max_skel"] = max(info["max_skel"], lv.rk[p])


def _eliminate(lv: _Level, st: Structure, l: int, p: int, info, zero_pivot):
    """Eqs. blr2-diag-ldl, -elimination, -schur for cluster p: LDL^T of
    S_pp^RR, L^{xR} = S^{xR} L^{-T} D^{-1} for every live block x coupled to
    p's redundant part, and S_xy -= L^{xR} D L^{yR T} on all such pairs."""
    Rs = np.arange(lv.rk[p], lv.dim[p])
    lv.elim[p] = True
    if len(Rs) == 0:
        return
    BRR = lv.get(p, p)[np.ix_(Rs, Rs)]
    perm, Lf, Dm, blocks = _bk_solve_parts(BRR, zero_pivot)
    neg, mn = dense.inertia_from_blocks(blocks)
    info["neg"] += neg
    info["minpiv"] = min(info["minpiv"], mn)
    nc = st.nclusters(l)
    targets = [p] + [a for a in range(nc) if a != p and st.near[l][p, a]]
    LxR = {}
    rows = {}
    for a in targets:
        ra = lv.live(a)                     # for a == p: its skeleton only
        rows[a] = ra
        C = lv.get(a, p)[np.ix_(ra, Rs)][:, perm]
        W = solve_triangular(Lf, C.T, lower=True, unit_diagonal=True).T   # S^{xR} L^{-T}
        LxR[a] = np.linalg.solve(Dm, W.T).T if W.size else W             # ... D^{-1}
    for i, a in enumerate(targets):
        for b in targets[:i + 1]:
            if LxR[a].size == 0 or LxR[b].size == 0:
                continue
            lv.sub(a, b, rows[a], rows[b], LxR[a] @ Dm @ LxR[b].T)


def _merge(h: H2Matrix, st: Structure, l: int, lv: _Level) -> _Level:
    """Merge children's skeleton blocks into the parent level (Sec. 3.3) and
    transform them with the parents' transfer bases."""
    ncp = st.nclusters(l - 1)
    r_build = h.ranks[l]
    # parent coordinates: [orig skel c1, orig skel c2, new skel c1, new skel c2]
    place = {}
    dims = []
    for P in range(ncp):
        c1, c2 = 2 * P, 2 * P + 1
        o1, o2 = r_build[c1], r_build[c2]
        t1, t2 = lv.rk[c1] - o1, lv.rk[c2] - o2
        idx1 = np.concatenate([np.arange(o1), o1 + o2 + np.arange(t1)])
        idx2 = np.concatenate([o1 + np.arange(o2), o1 + o2 + t1 + np.arange(t2)])
        place[c1], place[c2] = idx1, idx2
        dims.append(o1 + o2 + t1 + t2)
    up = _Level(dims, h.ranks[l - 1])
    for P in range(ncp):
        for Qc in range(P + 1):
            if not st.near[l - 1][P, Qc]:
                continue
            S = np.zeros((dims[P], dims[Qc]))
            for c in (2 * P, 2 * P + 1):
                for d in (2 * Qc, 2 * Qc + 1):
                    if st.near[l][c, d] or st.fill[l][c, d]:
                        src = lv.get(c, d)[:lv.rk[c], :lv.rk[d]]
                    else:
                        src = np.zeros((lv.rk[c], lv.rk[d]))
                        Cc = h.coupling[l][(c, d)]
                        src[:Cc.shape[0], :Cc.shape[1]] = Cc
                    S[np.ix_(place[c], place[d])] = src
            TP = _transfer_full(h.Q[l - 1][P], dims[P])
            TQ = _transfer_full(h.Q[l - 1][Qc], dims[Qc])
            up.blk[(P, Qc)] = TP.T @ S @ TQ
    _init_fill(h, st, l - 1, up)
    return up


def _transfer_full(T, dim):
    """[[T, 0], [0, I]]: the transfer on the build skeleton coordinates and the
    identity on coordinates added by recompression (all redundant above)."""
    out = np.eye(dim)
    k = T.shape[0]
    out[:k, :k] = T
    return out


def _init_fill(h, st, l, lv):
    nc = st.nclusters(l)
    for c in range(nc):
        for d in range(c + 1):
            if st.fill[l][c, d]:
                B = np.zeros((lv.dim[c], lv.dim[d]))
                C = h.coupling[l][(c, d)]
                B[:C.shape[0], :C.shape[1]] = C
                lv.blk[(c, d)] = B


def h2_inertia(h: H2Matrix, sigma: float):
    """nu(A~ - sigma I) by the generalized H^2-LDL^T (Eq. h2-generalized-ldl)
    and Sylvester's law (Sec. 4).  Returns (count, min |pivot|, info)."""
    st = h.st
    L = st.L
    nc = st.nclusters(L)
    lv = _Level([st.rng(L, c)[1] - st.rng(L, c)[0] for c in range(nc)], h.ranks[L])
    for key, B in h.near_blocks.items():
        lv.blk[key] = B.copy()
    for c in range(nc):
        lv.blk[(c, c)] -= sigma * np.eye(lv.dim[c])      # Q^T (A - sigma I) Q
    _init_fill(h, st, L, lv)
    info = {"neg": 0, "minpiv": math.inf, "trunc": 0.0, "max_skel": 0}
    for l in range(L, -1, -1):
        for p in st.order[l]:
            _recompress(lv, st, l, p, h.tol, h.fill_cap, info)
            _eliminate(lv, st, l, p, info, np.finfo(np.float64).eps * h.scale)
        if l > 0:
            lv = _merge(h, st, l, lv)
    return info["neg"], info["minpiv"], info


def kth_eigenvalues(h: H2Matrix, ks, tol: float, interval=None):
    """Algorithm 1 with inertia reuse on nu(A~ - mu I); start interval is the
    Gershgorin interval padded by 1e-6 * ||A||_inf."""
    a, b = interval if interval is not None else (
        h.gershgorin[0] - 1e-6 * h.scale, h.gershgorin[1] + 1e-6 * h.scale)
    return dense.bisect_many(lambda mu: h2_inertia(h, mu)[0], ks, a, b, tol)
