"""The many-eigenvalue experiments of Sec. 5.1 and Sec. 4.2 on the GPU.

E2 (Sec. 5.1, second accuracy experiment): every eigenvalue of the unit-circle
Laplace matrix (n = 1024, the paper's E1 geometry) at decreasing eps_ev, with
eps_H2 = 1e-2 eps_ev; the largest error over all n eigenvalues against the
dense oracle stays below eps_ev/2 + ||A - A~||_2 (Eq. error-bound plus Weyl).

Master-worker (Sec. 4.2, second parallel algorithm): an interior index range
split into free intervals and solved by two resident replicas through
h2_kth_eig_in equals one h2_kth_eig call over the whole range within tol.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense

pytestmark = pytest.mark.gpu
KP = (1e-3, 0.0, 0.0, 0.0)


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
def circle():
    X = W.unit_circle(1024, 5)
    return X, dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, KP, X))


@pytest.mark.parametrize("eps_ev", [1e-4, 1e-6, 1e-8])
def test_all_eigenvalues_error_sweep(pkg, circle, eps_ev):
    X, ev = circle
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=48, eta=1.0, eps_h2=1e-2 * eps_ev, max_lanes=256)
    err, _ = M.h2_compression_error(40)
    lam, eb = M.h2_kth_eig(np.arange(1, 1025), eps_ev)
    assert np.all(eb < 0.5 * eps_ev)
    assert np.all(np.diff(lam) >= -eps_ev)
    assert np.max(np.abs(lam - ev)) <= 0.5 * eps_ev + 1.5 * err, (np.max(np.abs(lam - ev)), err)
    M.close()


def test_master_worker_on_replicas(pkg, circle):
    from paper_2311_08618_gb300 import sharding
    X, ev = circle
    tol = 1e-8
    reps = [pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=32, eta=1.0, eps_h2=1e-9, max_lanes=16)
            for _ in range(2)]
    info = reps[0].h2_info()
    lo = info["gershgorin_lo"] - 1e-6 * info["norm_inf"]
    hi = info["gershgorin_hi"] + 1e-6 * info["norm_inf"]
    solvers = [lambda ks, a, b, M=M: M.h2_kth_eig_in(ks, a, b, tol) for M in reps]
    k0, k1 = 462, 561                           # 100 interior eigenvalues (the Sec. 5.1 parallel workload)
    out, handed = sharding.master_worker_local(solvers, lo, hi, k0, k1, 8)
    assert sorted(out) == list(range(k0, k1 + 1)) and handed > 2
    ref, _ = reps[0].h2_kth_eig(np.arange(k0, k1 + 1), tol)
    got = np.array([out[k] for k in range(k0, k1 + 1)])
    assert np.max(np.abs(got - ref)) <= tol
    # an interval that does not hold the indices is refused
    with pytest.raises(pkg.H2Error) as e:
        reps[0].h2_kth_eig_in([k0], ev[k0 + 5], hi, tol)
    assert e.value.code == -5
    for M in reps:
        M.close()


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_shifts_per_interval_cap(pkg, prec):
    """The round cap of h2_kth_eig (at most shifts_per_interval shifts per
    unfinished bracket): a few k on a 64-lane handle converge to the same
    eigenvalues within tol as with every lane per round, using at most
    16 shifts per bracket and round."""
    X = W.uniform_cube(1024, 2, 1)
    ev = dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, KP, X))
    ks = [1, 512, 700]
    tol = 1e-8
    out = {}
    for per in (16, 0):
        M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=64,
                         precision=getattr(pkg, "H2_PREC_" + prec), shifts_per_interval=per)
        lam, eb = M.h2_kth_eig(ks, tol)
        info = M.h2_info()
        out[per] = (lam, info)
        M.close()
        assert np.all(np.abs(lam - ev[np.array(ks) - 1]) <= tol / 2 + 1e-8 * np.abs(ev).max())
    lam16, info16 = out[16]
    lam0, info0 = out[0]
    assert np.all(np.abs(lam16 - lam0) <= tol)
    if prec == "FP64":
        assert info16["last_shifts"] <= 16 * len(ks) * info16["last_rounds"]
        assert info16["last_shifts"] < info0["last_shifts"]
