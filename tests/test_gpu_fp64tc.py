"""H2_PREC_FP64_TC: the Schur-update products W_a Y_b^T on the tensor cores
(exact BF16 products of 7-bit integer digits of the FP64 entries, integer
accumulation, one FP64 rounding per entry) against the CPU oracles.

The emulated product's error is below one FP64 rounding of the exact result
plus 2^-56 K of the row-scale products, the same order as an FP64 dot product;
so the bar is the FP64 path's: counts equal to the H^2 oracle's wherever the
smallest |pivot| clears 1e-10 ||A||, and k-th eigenvalues within tol + 1e-8 ||A||
of the dense oracle.
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


def shifts_between(ev, count):
    idx = np.linspace(1, len(ev) - 2, count).astype(int)
    return np.array([0.5 * (ev[i] + ev[i + 1]) for i in idx])


@pytest.mark.parametrize("d,n,seed,leaf,rank,kind", [
    (2, 256, 21, 32, 16, W.LAPLACE_EPS),
    (3, 800, 22, 32, 16, W.YUKAWA_EPS),
    (3, 400, 4, 32, 16, W.GAUSS_PLUS_INV),        # cylinder lattice
])
def test_fp64tc_counts_match_oracle(pkg, d, n, seed, leaf, rank, kind):
    if kind == W.GAUSS_PLUS_INV:
        X, kp = W.cylinder_lattice(n, seed), (1e-2, 0.1, 0, 0)
    else:
        X, kp = W.uniform_cube(n, d, seed), (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(kind, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 11)
    M = pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=16, precision=pkg.H2_PREC_FP64_TC)
    ref = oh2.construct(X, kind, kp, leaf, rank, 1.0)
    got, mp = M.h2_inertia(s)
    thr = 1e-10 * ref.scale
    checked = 0
    for x, c, p in zip(s, got, mp):
        want, wmp, _ = oh2.h2_inertia(ref, x)
        if min(p, wmp) > thr:
            assert c == want, (x, c, want, p, wmp)
            checked += 1
    assert checked >= len(s) // 2
    assert M.h2_status()[0] == 0


def test_fp64tc_c1_against_fp64_and_dense(pkg):
    """n=1024 2D (leaf 64, rank 16; K up to 48: two digit chunks): counts equal
    to the DFMA path's, pivots within 1e-9, lambda_512 within tol + 1e-8 ||A||
    of the dense eigenvalue in the golden file."""
    X = W.uniform_cube(1024, 2, 1)
    kp = (1e-3, 0, 0, 0)
    g = json.load(open(os.path.join(HERE, "golden", "c1_laplace2d_n1024.json")))
    F = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=16, max_lanes=64)
    T = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=16, max_lanes=64, precision=pkg.H2_PREC_FP64_TC)
    info = F.h2_info()
    s = np.linspace(info["gershgorin_lo"], info["gershgorin_hi"], 130)[1:-1]
    cf, pf = F.h2_inertia(s)
    ct, pt = T.h2_inertia(s)
    assert np.array_equal(cf, ct)
    np.testing.assert_allclose(pt, pf, rtol=1e-9)
    ks = [1, 256, 500, 512, 524, 1024]
    lf, _ = F.h2_kth_eig(ks, 1e-8)
    lt, ebt = T.h2_kth_eig(ks, 1e-8)
    assert np.all(ebt < 0.5e-8)
    assert np.max(np.abs(lt - lf)) <= 1e-8
    for k, lam in zip(ks, lt):
        if 500 <= k <= 524:
            assert abs(lam - g["dense_eigs_500_524"][k - 500]) <= 1e-8 + 1e-8 * g["norm2"]
    assert T.h2_status()[0] == 0


def test_fp64tc_wide_redundant_blocks(pkg):
    """Leaves of 128 points (build ranks up to 26, below the cap of 32): about
    100 redundant columns, four 32-wide digit chunks per product; counts equal
    to the DFMA path's and to the dense oracle's at midpoints between
    eigenvalues."""
    X = W.uniform_cube(2048, 2, 31)
    kp = (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    s = shifts_between(ev, 25)
    F = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=128, rank=32, max_lanes=32)
    T = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=128, rank=32, max_lanes=32, precision=pkg.H2_PREC_FP64_TC)
    cf, pf = F.h2_inertia(s)
    ct, pt = T.h2_inertia(s)
    assert np.array_equal(cf, ct)
    # pivots of 100-wide redundant blocks amplify rounding-level differences
    # of the Schur products (any two FP64 summation orders differ as much):
    # compare them on the scale of ||A||, as the count criterion does
    assert np.max(np.abs(pt - pf)) <= 1e-9 * T.h2_info()["norm_inf"]
    gap = np.minimum(np.abs(s[:, None] - ev[None, :]).min(axis=1), np.inf)
    sure = gap > 1e-6 * np.abs(ev).max()
    assert sure.sum() >= len(s) // 2
    want = np.array([np.sum(ev < x) for x in s])
    assert np.array_equal(ct[sure], want[sure])


@pytest.mark.parametrize("n,d,leaf,rank,lanes", [(1024, 2, 64, 16, 256), (600, 3, 40, 16, 16), (2048, 2, 32, 12, 64)])
def test_tcgen05_schur_bit_identical_to_mma_sync(pkg, n, d, leaf, rank, lanes):
    """The tcgen05 digit Schur kernel (tensor-memory accumulators, 128-row
    panels) and the mma.sync one form the same exact integer level sums and
    round once the same way: counts and min |pivot| agree bit for bit."""
    import torch
    X = W.uniform_cube(n, d, 91)
    kp = (1e-3, 0, 0, 0)
    mats = [pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=leaf, rank=rank, max_lanes=lanes,
                         precision=pkg.H2_PREC_FP64_TC, tc_schur=t) for t in (1, 0)]
    info = mats[0].h2_info()
    sh = torch.tensor(info["gershgorin_lo"] + (info["gershgorin_hi"] - info["gershgorin_lo"]) *
                      (np.arange(lanes) + 0.37) / lanes, dtype=torch.float64, device="cuda")
    out = []
    for M in mats:
        c = torch.zeros(lanes, dtype=torch.int64, device="cuda")
        mp = torch.zeros(lanes, dtype=torch.float64, device="cuda")
        M.h2_inertia_device(sh, lanes, c, mp)
        torch.cuda.synchronize()
        assert M.h2_status()[0] == 0
        out.append((c.cpu().numpy(), mp.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1].view(np.int64), out[1][1].view(np.int64))
    for M in mats:
        M.close()
