"""Multi-matrix batches (h2_group_*): one launch per tree level and colour
over several resident matrices of different sizes.

Each handle keeps its own workspace, so a group batch must reproduce every
handle's own batch exactly (counts and pivots), and through them the oracle.
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


MEMBERS = [   # (points, kernel, kparams, leaf, rank): uneven sizes, depths and dimensions
    (lambda: W.uniform_cube(300, 2, 41), W.LAPLACE_EPS, (1e-3, 0, 0, 0), 32, 16),
    (lambda: W.uniform_cube(1024, 2, 1), W.LAPLACE_EPS, (1e-3, 0, 0, 0), 64, 16),
    (lambda: W.uniform_cube(800, 3, 22), W.YUKAWA_EPS, (1e-3, 0, 0, 0), 32, 16),
    (lambda: W.cylinder_lattice(400, 4), W.GAUSS_PLUS_INV, (1e-2, 0.1, 0, 0), 32, 16),
    (lambda: W.uniform_cube(2048, 2, 31), W.LAPLACE_EPS, (1e-3, 0, 0, 0), 64, 16),
]


def _build(pkg, stream, lanes, precision):
    mats, pts = [], []
    for mk, kind, kp, leaf, rank in MEMBERS:
        X = mk()
        pts.append((X, kind, kp, leaf, rank))
        mats.append(pkg.H2Matrix(X, kind, kp, leaf=leaf, rank=rank, max_lanes=lanes, stream=stream.cuda_stream,
                                 precision=precision))
    return mats, pts


@pytest.mark.parametrize("prec", [0, 2, 1])
def test_group_equals_each_handles_own_batch(pkg, prec):
    import torch
    st = torch.cuda.Stream()
    lanes = 16
    with torch.cuda.stream(st):
        mats, _ = _build(pkg, st, lanes, prec)
        G = pkg.H2Group(mats)
        nh = len(mats)
        ns = [16, 5, 0, 11, 16]
        sh = np.zeros((nh, lanes))
        for i, M in enumerate(mats):
            inf = M.h2_info()
            sh[i] = np.linspace(inf["gershgorin_lo"], inf["gershgorin_hi"], lanes + 2)[1:-1] + 1e-3 * i
        d_sh = torch.tensor(sh, dtype=torch.float64, device="cuda")
        d_c = torch.full((nh, lanes), -1, dtype=torch.int64, device="cuda")
        d_mp = torch.zeros((nh, lanes), dtype=torch.float64, device="cuda")
        for _ in range(2):                     # the batch is repeatable
            G.h2_group_inertia_device(d_sh, ns, d_c, d_mp)
        torch.cuda.synchronize()
        gc, gm = d_c.cpu().numpy(), d_mp.cpu().numpy()
        for i, M in enumerate(mats):
            if ns[i] == 0:
                assert np.all(gc[i] == -1)     # nothing written for an idle handle
                continue
            own_c = torch.zeros(lanes, dtype=torch.int64, device="cuda")
            own_m = torch.zeros(lanes, dtype=torch.float64, device="cuda")
            M.h2_inertia_device(d_sh[i], ns[i], own_c, own_m)
            torch.cuda.synchronize()
            assert np.array_equal(gc[i, :ns[i]], own_c.cpu().numpy()[:ns[i]]), i
            assert np.array_equal(gm[i, :ns[i]], own_m.cpu().numpy()[:ns[i]]), i
            assert M.h2_status()[0] == 0
        assert G.launches() > 0
        G.close()
        for M in mats:
            M.close()


def test_group_counts_match_oracle(pkg):
    """The smallest member's group counts against the H^2 oracle, the others
    against the dense oracle at midpoints between eigenvalues."""
    import torch
    st = torch.cuda.Stream()
    lanes = 16
    with torch.cuda.stream(st):
        mats, pts = _build(pkg, st, lanes, 0)
        G = pkg.H2Group(mats)
        nh = len(mats)
        sh = np.zeros((nh, lanes))
        evs = []
        for i, (X, kind, kp, leaf, rank) in enumerate(pts):
            ev = dense.eigenvalues(dense.kernel_matrix(kind, kp, X))
            evs.append(ev)
            idx = np.linspace(1, len(ev) - 2, lanes).astype(int)
            sh[i] = 0.5 * (ev[idx] + ev[idx + 1])
        d_sh = torch.tensor(sh, dtype=torch.float64, device="cuda")
        d_c = torch.zeros((nh, lanes), dtype=torch.int64, device="cuda")
        d_mp = torch.zeros((nh, lanes), dtype=torch.float64, device="cuda")
        G.h2_group_inertia_device(d_sh, [lanes] * nh, d_c, d_mp)
        torch.cuda.synchronize()
        gc, gm = d_c.cpu().numpy(), d_mp.cpu().numpy()
        X, kind, kp, leaf, rank = pts[0]
        ref = oh2.construct(X, kind, kp, leaf, rank, 1.0)
        thr = 1e-10 * ref.scale
        checked = 0
        for x, c, p in zip(sh[0], gc[0], gm[0]):
            want, wmp, _ = oh2.h2_inertia(ref, x)
            if min(p, wmp) > thr:
                assert c == want
                checked += 1
        assert checked >= lanes // 2
        for i in range(1, nh):
            ev = evs[i]
            gap = np.abs(sh[i][:, None] - ev[None, :]).min(axis=1)
            sure = gap > 1e-6 * np.abs(ev).max()
            want = np.array([np.sum(ev < x) for x in sh[i]])
            assert np.array_equal(gc[i][sure], want[sure]), i
        G.close()
        for M in mats:
            M.close()


def test_group_rejects_unequal_lanes(pkg):
    import torch
    st = torch.cuda.Stream()
    X = W.uniform_cube(300, 2, 41)
    a = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=32, rank=16, max_lanes=8, stream=st.cuda_stream)
    b = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=32, rank=16, max_lanes=16, stream=st.cuda_stream)
    with pytest.raises(pkg.H2Error) as e:
        pkg.H2Group([a, b])
    assert e.value.code == -1


def test_group_kth_driver_against_dense(pkg):
    """batching.kth_group: every matrix's own k to tol 1e-8 in shared group
    rounds; within tol of the handle's own h2_kth_eig.  Against the dense
    oracle's eigenvalue the bound is tol + 1e-7 ||A||_inf: these members' rank
    caps (16) leave compression errors above 1e-8 ||A||, and by Weyl's
    inequality an eigenvalue moves by at most ||A - A~||_2."""
    import torch
    from paper_2311_08618_gb300 import batching
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        mats, pts = _build(pkg, st, 8, 0)
        ks = [1, 512, 400, 200, 1500]
        lam, rounds, shifts = batching.kth_group(mats, ks, 1e-8, st)
        assert rounds > 0 and shifts > 0
        for i, (M, (X, kind, kp, leaf, rank)) in enumerate(zip(mats, pts)):
            own, eb = M.h2_kth_eig([ks[i]], 1e-8)
            assert abs(lam[i] - own[0]) <= 1e-8, i
            A = dense.kernel_matrix(kind, kp, X)
            ev = dense.eigenvalues(A)
            assert abs(lam[i] - ev[ks[i] - 1]) <= 1e-8 + 1e-7 * np.abs(A).sum(axis=1).max(), i
        for M in mats:
            M.close()
