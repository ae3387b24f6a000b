"""Fill-in recompression on a thread-block cluster (k_recomp_cluster) against
the CPU oracle and against the one-CTA kernel.

The clustered pivoted QR splits the columns of Z over 8 CTAs; its pivots follow
the same rule (largest norm, then smallest index), so its counts must equal the
oracle's wherever the smallest |pivot| clears 1e-10 ||A||, exactly as the
one-CTA path's do.  recomp_cluster_cols=1 sends every level with fill-ins to
the clustered kernel.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense, h2 as oh2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_08618_gb300 as p
    from paper_2311_08618_gb300 import build
    build.build()
    return p


def shifts_between(ev, count):
    idx = np.linspace(1, len(ev) - 2, count).astype(int)
    return np.array([0.5 * (ev[i] + ev[i + 1]) for i in idx])


@pytest.mark.parametrize("d,n,seed,leaf,rank,kind", [
    (2, 256, 21, 32, 16, W.LAPLACE_EPS),
    (3, 800, 22, 32, 16, W.YUKAWA_EPS),
])
def test_clustered_recompression_matches_oracle(pkg, d, n, seed, leaf, rank, kind):
    X = W.uniform_cube(n, d, seed)
    kp = (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(kind, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 11)
    Mc = pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=16, recomp_cluster_cols=1)
    assert Mc.h2_info()["fill_pairs"] > 0          # the recompression runs
    ref = oh2.construct(X, kind, kp, leaf, rank, 1.0)
    got, mp = Mc.h2_inertia(s)
    thr = 1e-10 * ref.scale
    checked = 0
    for x, c, p in zip(s, got, mp):
        want, wmp, _ = oh2.h2_inertia(ref, x)
        if min(p, wmp) > thr:
            assert c == want, (x, c, want, p, wmp)
            checked += 1
    assert checked >= len(s) // 2
    assert Mc.h2_status()[0] == 0


def test_clustered_and_single_cta_paths_agree(pkg):
    """n=1024 2D (leaf 64, rank 16): the same counts and pivots (up to the
    stopping sum's addition order) from both recompression kernels, FP64 and
    mixed, and the golden dense eigenvalue for k = 512."""
    X = W.uniform_cube(1024, 2, 1)
    kp = (1e-3, 0, 0, 0)
    lo_hi = None
    out = {}
    for prec in (pkg.H2_PREC_FP64, pkg.H2_PREC_MIXED):
        for cols in (-1, 1):
            M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=16, max_lanes=64, precision=prec,
                             recomp_cluster_cols=cols)
            info = M.h2_info()
            if lo_hi is None:
                lo_hi = (info["gershgorin_lo"], info["gershgorin_hi"])
            s = np.linspace(lo_hi[0], lo_hi[1], 67)[1:-1]
            c, p = M.h2_inertia(s)
            lam, eb = M.h2_kth_eig([512], 1e-8)
            out[(prec, cols)] = (c, p, lam[0])
            assert M.h2_status()[0] == 0
            M.close()
    for prec in (pkg.H2_PREC_FP64, pkg.H2_PREC_MIXED):
        c1, p1, l1 = out[(prec, -1)]
        c2, p2, l2 = out[(prec, 1)]
        assert np.array_equal(c1, c2)
        np.testing.assert_allclose(p1, p2, rtol=1e-6)
        assert abs(l1 - l2) <= 1e-8
    # lambda_512 of the dense matrix (golden file): within tol + 1e-8 ||A||_2
    assert abs(out[(pkg.H2_PREC_FP64, 1)][2] - 965.7169369317037) <= 1e-8 + 1e-8 * 4109.95


def test_autotuned_handle(pkg):
    """autotune=1: every level reports a valid choice, and the tuned handle's
    counts equal the dense oracle's at midpoints between eigenvalues (FP64 and
    mixed)."""
    X = W.uniform_cube(800, 3, 22)
    kp = (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(W.YUKAWA_EPS, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 15)
    gap = np.abs(s[:, None] - ev[None, :]).min(axis=1)
    sure = gap > 1e-6 * np.abs(ev).max()
    want = np.array([np.sum(ev < x) for x in s])
    for prec in (pkg.H2_PREC_FP64, pkg.H2_PREC_MIXED):
        M = pkg.H2Matrix(X, W.YUKAWA_EPS, kp, leaf=32, rank=16, max_lanes=16, precision=prec, autotune=1)
        L = M.h2_info()["levels"] - 1
        for l in range(L + 1):
            t, c = M.h2_autotune_choice(l)
            assert t in (32, 128, 256) and c in (0, 1)
        got, mp = M.h2_inertia(s)
        assert np.array_equal(got[sure], want[sure])
        assert M.h2_status()[0] == 0
        M.close()
