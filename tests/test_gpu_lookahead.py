"""The lookahead schedule within a level (h2_options.lookahead): once colour
c's Schur updates of the blocks in rows and columns of colour c + 1's clusters
are done, colour c + 1's recompression, rotation, LDL^T and solves run on a
second stream beside colour c's remaining updates.

Every block receives its updates in the order of the one-stream schedule (the
distance-2 colouring gives each block at most one update per colour), and the
two colours' factors sit in separate scratch halves, so the counts, the
smallest pivots and the k-th eigenvalues are the same bit for bit.
"""
import numpy as np
import pytest

import workloads as W

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


def _points(shape):
    if shape == "laplace2d_1024":
        return W.uniform_cube(1024, 2, 1), W.LAPLACE_EPS, (1e-3, 0, 0, 0), 64, 16
    if shape == "yukawa3d_800":
        return W.uniform_cube(800, 3, 22), W.YUKAWA_EPS, (1e-3, 0, 0, 0), 32, 16
    return W.cylinder_lattice(400, 4), W.GAUSS_PLUS_INV, (1e-2, 0.1, 0, 0), 32, 16


def _batch(M, sh, lanes):
    import torch
    c = torch.zeros(lanes, dtype=torch.int64, device="cuda")
    mp = torch.zeros(lanes, dtype=torch.float64, device="cuda")
    M.h2_inertia_device(sh, lanes, c, mp)
    torch.cuda.synchronize()
    assert M.h2_status()[0] == 0
    return c.cpu().numpy(), mp.cpu().numpy()


@pytest.mark.parametrize("shape", ["laplace2d_1024", "yukawa3d_800", "cylinder_400"])
@pytest.mark.parametrize("prec", ["FP64", "FP64_TC", "MIXED"])
def test_lookahead_bit_identical(pkg, shape, prec):
    import torch
    X, kind, kp, leaf, rank = _points(shape)
    lanes = 48
    p = getattr(pkg, "H2_PREC_" + prec)
    mats = [pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=lanes, precision=p, lookahead=la)
            for la in (1, 0)]
    info = mats[0].h2_info()
    lo, hi = info["gershgorin_lo"], info["gershgorin_hi"]
    sh = torch.tensor(lo + (hi - lo) * (np.arange(lanes) + 0.41) / lanes, dtype=torch.float64, device="cuda")
    out = [_batch(M, sh, lanes) for M in mats]
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1].view(np.int64), out[1][1].view(np.int64))
    # the one-stream graph and the plain launches agree with it too
    plain = pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=lanes, precision=p, graphs=0)
    c, mp = _batch(plain, sh, lanes)
    assert np.array_equal(c, out[0][0])
    assert np.array_equal(mp.view(np.int64), out[0][1].view(np.int64))
    # k-th eigenvalues through the device-resident loop
    ks = [1, X.shape[0] // 3, X.shape[0] // 2, X.shape[0]]
    lam = [M.h2_kth_eig(ks, 1e-9) for M in mats]
    assert np.array_equal(np.asarray(lam[0][0]).view(np.int64), np.asarray(lam[1][0]).view(np.int64))
    for M in mats + [plain]:
        M.close()


def test_lookahead_scratch_and_kernels(pkg):
    """The schedule takes a second scratch half and splits each colour's
    Schur launch (but the last of a level) in two."""
    X, kind, kp, leaf, rank = _points("laplace2d_1024")
    on = pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=16, lookahead=1)
    off = pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=16, lookahead=0)
    a, b = on.h2_info(), off.h2_info()
    assert a["workspace_bytes"] > b["workspace_bytes"]
    assert a["kernels_per_batch"] > b["kernels_per_batch"]
    on.close()
    off.close()
