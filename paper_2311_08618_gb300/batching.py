"""k-th eigenvalues of many independent H^2 matrices in shared batches (a
scheduling layer above the C ABI; every inertia evaluation runs in the
library's kernels, as one h2_group batch per round).

Each matrix i has its own k_i and bracket [a_i, b_i], starting from its
Gershgorin interval widened by 1e-6 ||A_i||_inf (nu(a_i) = 0, nu(b_i) = n_i).
A round places the matrix's max_lanes shifts at equally spaced interior points
of its bracket ((q+1)-section, Algorithm 1 with spare lanes), evaluates the
shifts of all unfinished matrices in one group batch (one launch per tree
level and colour over all of them), and narrows every bracket with all of its
matrix's (mu, nu) pairs: nu >= k_i moves b_i down, nu < k_i moves a_i up.  A
matrix is done when b_i - a_i < tol; its result is the midpoint, so
|lambda_k - result| < tol / 2 (Eq. error-bound).
"""
from __future__ import annotations

import numpy as np

from .binding import H2Group


def bracket_rounds(a, b, ks, tol, lanes, evaluate):
    """The host side of the rounds: brackets [a_i, b_i] of lambda_{k_i},
    narrowed until b_i - a_i < tol.  evaluate(mu, ns) returns the counts
    nu(mu[i, j]) for j < ns[i] (mu: matrices x lanes array, ns: shifts per
    matrix, 0 for finished ones).  Returns (midpoints, rounds, shifts)."""
    a = np.array(a, dtype=np.float64)
    b = np.array(b, dtype=np.float64)
    k = np.asarray(ks, dtype=np.int64)
    frac = np.arange(1, lanes + 1) / (lanes + 1.0)
    rounds = shifts = 0
    while True:
        act = (b - a) >= tol
        if not act.any():
            break
        mu = a[:, None] + (b - a)[:, None] * frac[None, :]
        ns = np.where(act, lanes, 0)
        nu = evaluate(mu, ns)
        for i in np.nonzero(act)[0]:
            hi_side = nu[i] >= k[i]
            if hi_side.any():
                b[i] = min(b[i], mu[i][hi_side].min())
            if (~hi_side).any():
                a[i] = max(a[i], mu[i][~hi_side].max())
        rounds += 1
        shifts += int(ns.sum())
    return 0.5 * (a + b), rounds, shifts


def kth_group(mats, ks, tol, stream, group=None, start=None):
    """lambda_{k_i}(A_i) for every handle in ``mats`` (equal max_lanes and
    precision, all on ``stream``, a torch.cuda.Stream).  ``start`` = (a, b)
    replaces the widened Gershgorin intervals (the caller guarantees
    nu(a_i) < k_i <= nu(b_i)).  Returns (values, rounds, shifts evaluated)."""
    import torch
    G = group if group is not None else H2Group(mats)
    nh = len(mats)
    lanes = int(mats[0].h2_info()["lanes"])
    a = np.zeros(nh)
    b = np.zeros(nh)
    for i, M in enumerate(mats):
        inf = M.h2_info()
        a[i] = inf["gershgorin_lo"] - 1e-6 * inf["norm_inf"]
        b[i] = inf["gershgorin_hi"] + 1e-6 * inf["norm_inf"]
    if start is not None:
        a[:] = start[0]
        b[:] = start[1]
    h_sh = torch.zeros((nh, lanes), dtype=torch.float64).pin_memory()
    h_c = torch.zeros((nh, lanes), dtype=torch.int64).pin_memory()
    d_sh = torch.zeros((nh, lanes), dtype=torch.float64, device="cuda")
    d_c = torch.zeros((nh, lanes), dtype=torch.int64, device="cuda")

    def evaluate(mu, ns):
        with torch.cuda.stream(stream):
            h_sh.numpy()[:] = mu
            d_sh.copy_(h_sh, non_blocking=True)
            G.h2_group_inertia_device(d_sh, ns, d_c)
            h_c.copy_(d_c, non_blocking=True)
        stream.synchronize()
        return h_c.numpy()

    out = bracket_rounds(a, b, ks, tol, lanes, evaluate)
    if group is None:
        G.close()
    return out
