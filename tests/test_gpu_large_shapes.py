"""Parity at the block shapes of the large configurations (Sec. 3.4 with leaf
256): the 3D Yukawa shape (leaf 256, rank 32) and the cylindrical-lattice
shape (leaf 256, rank 48, exp(-r^2/2) + 1e-2/(r + 0.1)), at n = 8192 where
the dense eigenvalues are computable on the host.

Counts of all three precisions must equal the dense counts of A at shifts
farther than 2 (||A - A~||_2 + 1e-10 ||A||) from its spectrum (Weyl: the
eigenvalues of A~ are within ||A - A~||_2 of those of A); the FP64 count of a
sampled shift must equal the H^2 oracle's (bit-exact bar, min |pivot| >
1e-10 ||A||).
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense, h2 as oh2

pytestmark = pytest.mark.gpu

SHAPES = {
    "yukawa3d_n8192_leaf256_rank32": (lambda: W.uniform_cube(8192, 3, 2), W.YUKAWA_EPS, (1e-3, 0.0, 0.0, 0.0),
                                      256, 32),
    "cylinder_n8192_leaf256_rank48": (lambda: W.cylinder_lattice(8192, 4), W.GAUSS_PLUS_INV,
                                      (1e-2, 0.1, 0.0, 0.0), 256, 48),
}


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_08618_gb300 as p
    from paper_2311_08618_gb300 import build
    build.build()
    return p


@pytest.fixture(scope="module", params=sorted(SHAPES))
def shape(request, pkg):
    pts, kind, kp, leaf, rank = SHAPES[request.param]
    X = pts()
    A = dense.kernel_matrix(kind, kp, X)
    ev = np.linalg.eigvalsh(A)
    del A
    F = pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, eta=1.0, max_lanes=64)
    err, nrm = F.h2_compression_error(30)
    info = F.h2_info()
    thr = 1e-10 * info["norm_inf"]
    # midpoints of gaps wider than 4 (err + thr), spread over the spectrum,
    # plus both ends
    gaps = np.nonzero(np.diff(ev) > 4.0 * (err + thr))[0]
    mids = 0.5 * (ev[gaps] + ev[gaps + 1])
    pick = mids[np.linspace(0, len(mids) - 1, min(62, len(mids))).astype(int)]
    shifts = np.unique(np.concatenate([pick, [ev[0] - 1.0, ev[-1] + 1.0]]))
    want = np.searchsorted(ev, shifts)
    yield dict(name=request.param, X=X, kind=kind, kp=kp, leaf=leaf, rank=rank, F=F, err=err, nrm=nrm,
               shifts=shifts, want=want, info=info)
    F.close()


def test_compression_and_structure(shape):
    info = shape["info"]
    assert shape["err"] / shape["nrm"] <= 1e-8, (shape["name"], shape["err"] / shape["nrm"])
    assert info["leaves"] == 32 and info["max_rank"] <= shape["rank"]
    assert len(shape["shifts"]) >= 32


@pytest.mark.parametrize("prec", ["FP64", "FP64_TC", "MIXED"])
def test_counts_equal_dense_away_from_spectrum(pkg, shape, prec):
    code = getattr(pkg, "H2_PREC_" + prec)
    if code == pkg.H2_PREC_FP64:
        M = shape["F"]
    else:
        M = pkg.H2Matrix(shape["X"], shape["kind"], shape["kp"], leaf=shape["leaf"], rank=shape["rank"], eta=1.0,
                         max_lanes=64, precision=code)
    got, mp = M.h2_inertia(shape["shifts"])
    assert np.array_equal(got, shape["want"]), (shape["name"], prec, np.nonzero(got != shape["want"]))
    assert M.h2_status()[0] == 0
    if M is not shape["F"]:
        M.close()


def test_fp64_count_equals_h2_oracle(shape):
    """One shift in the interior of the spectrum through the oracle's
    generalized LDL^T (about half a minute of host time)."""
    ref = oh2.construct(shape["X"], shape["kind"], shape["kp"], shape["leaf"], shape["rank"], 1.0)
    assert [max(r) for r in ref.ranks] == [max(shape["F"].h2_level_ranks(l)) for l in range(ref.st.L + 1)]
    mid = len(shape["shifts"]) // 2
    s = shape["shifts"][mid]
    want, wmp, _ = oh2.h2_inertia(ref, s)
    got, mp = shape["F"].h2_inertia([s])
    assert min(wmp, mp[0]) > 1e-10 * ref.scale
    assert got[0] == want == shape["want"][mid]
