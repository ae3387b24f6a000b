"""Mixed precision (FP32 Schur/rotation products, FP64 storage, pivots, counts
and interval updates) against the FP64 path and the dense oracle.

Certified rule under test: mixed rounds stop at bracket width
Delta = 64 * 2^-24 * ||A||_inf; the widened bracket is checked in FP64 and
FP64 rounds finish, so every k-th eigenvalue must match the FP64 path within
tol and the dense oracle within tol + 1e-8 ||A||.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import dense

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


@pytest.fixture(scope="module")
def c1(pkg):
    X = W.uniform_cube(1024, 2, 1)
    kp = (1e-3, 0, 0, 0)
    F = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=16, max_lanes=64)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=16, max_lanes=64, precision=pkg.H2_PREC_MIXED)
    g = json.load(open(os.path.join(HERE, "golden", "c1_laplace2d_n1024.json")))
    return X, F, M, g


def test_mixed_kth_matches_fp64_and_dense(c1):
    X, F, M, g = c1
    tol = 1e-8
    ks = [1, 256, 512, 513, 1024]
    lf, ebf = F.h2_kth_eig(ks, tol)
    lm, ebm = M.h2_kth_eig(ks, tol)
    info = M.h2_info()
    assert info["last_mixed_rounds"] > 0
    assert info["bracket_resets"] == 0
    assert np.all(ebm < 0.5 * tol)
    assert np.max(np.abs(lm - lf)) <= tol
    lam_dense = g["dense_eigs_500_524"][512 - 500]
    assert abs(lm[2] - lam_dense) <= tol + 1e-8 * g["norm2"]


def test_mixed_counts_away_from_spectrum(c1):
    """Shifts farther than Delta from every eigenvalue: mixed counts are exact."""
    X, F, M, g = c1
    A = dense.kernel_matrix(W.LAPLACE_EPS, (1e-3, 0, 0, 0), X)
    ev = dense.eigenvalues(A)
    info = M.h2_info()
    delta = 64 * 2.0 ** -24 * info["norm_inf"]
    gaps = np.nonzero(np.diff(ev) > 4 * delta)[0]
    shifts = 0.5 * (ev[gaps] + ev[gaps + 1])[::4][:256]
    cm, mm = M.h2_inertia(shifts)
    cf, mf = F.h2_inertia(shifts)
    assert len(shifts) >= 64
    assert np.array_equal(cm, cf)
    assert np.array_equal(cf, [np.sum(ev < s) for s in shifts])


def test_mixed_guard_reruns_low_pivot_shifts(pkg):
    """A shift placed on a (dense) eigenvalue is guarded and re-run in FP64;
    every certified count equals the FP64 count."""
    X = W.uniform_cube(128, 2, 33)
    kp = (1e-3, 0, 0, 0)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=32, rank=12, max_lanes=16,
                     precision=pkg.H2_PREC_MIXED, pivot_guard=1e-3)
    F = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=32, rank=12, max_lanes=16)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    shifts = np.array([0.5 * (ev[10] + ev[11]), ev[40] + 1e-9, 0.5 * (ev[90] + ev[91])])
    cm, mm = M.h2_inertia(shifts)
    info = M.h2_info()
    assert info["guard_reruns"] >= 1 and info["guard_checked"] == 3
    cf, mf = F.h2_inertia(shifts)
    assert np.array_equal(cm, cf)


def test_mixed_wide_blocks_counts_away_from_spectrum(pkg):
    """Blocks of up to 128 rows (leaf 128): the FP32 Schur tiles are 64 wide,
    so diagonal blocks span 2 x 2 tiles and their upper tile is written as the
    transpose of the lower one.  Counts more than Delta from the spectrum equal
    the dense oracle's."""
    X = W.uniform_cube(2048, 2, 31)
    kp = (1e-3, 0, 0, 0)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=128, rank=32, max_lanes=64, precision=pkg.H2_PREC_MIXED)
    delta = 64 * 2.0 ** -24 * M.h2_info()["norm_inf"]
    gaps = np.nonzero(np.diff(ev) > 4 * delta)[0]
    shifts = 0.5 * (ev[gaps] + ev[gaps + 1])[::7][:64]
    assert len(shifts) >= 32
    cm, _ = M.h2_inertia(shifts)
    assert np.array_equal(cm, [np.sum(ev < s) for s in shifts])
    assert M.h2_status()[0] == 0
    M.close()
