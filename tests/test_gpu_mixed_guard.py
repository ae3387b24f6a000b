"""The certified mixed-precision counts (Sec. 4.1, Parlett's criterion, and
the FP64 re-run of small-pivot shifts) on every entry point that returns counts:
h2_inertia, h2_inertia_device, group batches, and the serving and batching
layers above them.

Shifts are placed 1e-8 from eigenvalues of A~, far inside the FP32 product
error of the mixed factorization (about 1e-4 at n = 1024) and far outside the
FP64 one: raw mixed counts flip there (shown with the unguarded mixed batch of
h2_profile_batch), certified counts must not.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense, h2 as oh2

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
def c1(pkg):
    X = W.uniform_cube(1024, 2, 1)
    ref = oh2.construct(X, W.LAPLACE_EPS, KP, 64, 16, 1.0)
    evt = np.linalg.eigvalsh(oh2.dense_approximation(ref))
    sel = evt[::8]
    shifts = np.sort(np.concatenate([sel - 1e-8, sel + 1e-8]))
    F = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=64)
    want, _ = F.h2_inertia(shifts)
    F.close()
    return X, shifts, want


def test_raw_mixed_flips_are_caught(pkg, c1):
    import torch
    X, shifts, want = c1
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=64, precision=pkg.H2_PREC_MIXED)
    # raw mixed counts: the mixed batch alone, without the guard
    raw = np.zeros(len(shifts), dtype=np.int64)
    for b0 in range(0, len(shifts), 64):
        nb = min(64, len(shifts) - b0)
        d_sh = torch.tensor(shifts[b0:b0 + nb], dtype=torch.float64, device="cuda")
        d_c = torch.zeros(nb, dtype=torch.int64, device="cuda")
        M.h2_profile_batch(d_sh, nb, d_c)
        raw[b0:b0 + nb] = d_c.cpu().numpy()
    flips = int(np.sum(raw != want))
    got, mp = M.h2_inertia(shifts)
    info = M.h2_info()
    assert np.array_equal(got, want)
    assert flips >= 1, "no raw flip next to the spectrum: the test shows nothing"
    assert info["guard_reruns"] >= flips
    assert info["guard_checked"] == len(shifts)
    M.close()


def test_shift_where_the_fp32_error_exceeds_delta(pkg):
    """At this shift of the n = 1024 workload (0.0086 above an eigenvalue of
    A~), the mixed factorization at mu + Delta is wrong by one while the one at
    mu - Delta is right, so the two agree on the wrong count: the FP32 error
    there exceeds Delta.  Its smaller mixed min |pivot| is 3.9e-4 ||A||_inf,
    under the default pivot_guard of 1e-3, so the shift goes to FP64 (with the
    guard at 1e-4 it was certified wrong)."""
    X = W.uniform_cube(1024, 2, 1)
    mu = 1184.4096755702722
    F = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=4)
    want, _ = F.h2_inertia(np.array([mu]))
    F.close()
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=4, precision=pkg.H2_PREC_MIXED)
    got, _ = M.h2_inertia(np.array([mu]))
    assert M.h2_info()["guard_reruns"] == 1
    M.close()
    assert got[0] == want[0]


def test_device_entry_point_is_certified(pkg, c1):
    import torch
    X, shifts, want = c1
    for lanes in (64, 1):
        M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=lanes, precision=pkg.H2_PREC_MIXED)
        got = np.zeros(len(shifts), dtype=np.int64)
        for b0 in range(0, len(shifts), lanes):
            nb = min(lanes, len(shifts) - b0)
            d_sh = torch.tensor(shifts[b0:b0 + nb], dtype=torch.float64, device="cuda")
            d_c = torch.full((nb,), -1, dtype=torch.int64, device="cuda")
            d_mp = torch.zeros(nb, dtype=torch.float64, device="cuda")
            M.h2_inertia_device(d_sh, nb, d_c, d_mp)
            torch.cuda.synchronize()
            got[b0:b0 + nb] = d_c.cpu().numpy()
        assert np.array_equal(got, want), lanes
        M.close()


def test_group_batches_are_certified(pkg, c1):
    """Two mixed handles (the n = 1024 matrix and a smaller one) in one group:
    every count equals the FP64 count of its own matrix."""
    import torch
    X, shifts, want = c1
    X2 = W.uniform_cube(300, 2, 61)
    F2 = pkg.H2Matrix(X2, W.LAPLACE_EPS, KP, leaf=40, rank=16, max_lanes=32)
    ev2 = dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, KP, X2))
    sh2 = np.sort(np.concatenate([ev2[::10] - 1e-8, ev2[::10] + 1e-8]))[:32]
    want2, _ = F2.h2_inertia(sh2)
    F2.close()
    st = torch.cuda.Stream()
    Ms = [pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=32, precision=pkg.H2_PREC_MIXED,
                       stream=st.cuda_stream),
          pkg.H2Matrix(X2, W.LAPLACE_EPS, KP, leaf=40, rank=16, max_lanes=32, precision=pkg.H2_PREC_MIXED,
                       stream=st.cuda_stream)]
    G = pkg.H2Group(Ms)
    got1 = np.zeros(len(shifts), dtype=np.int64)
    for b0 in range(0, len(shifts), 32):
        nb = min(32, len(shifts) - b0)
        d_sh = torch.zeros((2, 32), dtype=torch.float64, device="cuda")
        d_c = torch.full((2, 32), -1, dtype=torch.int64, device="cuda")
        d_sh[0, :nb] = torch.tensor(shifts[b0:b0 + nb], dtype=torch.float64)
        d_sh[1, :len(sh2)] = torch.tensor(sh2, dtype=torch.float64)
        n2 = len(sh2) if b0 == 0 else 0
        with torch.cuda.stream(st):
            G.h2_group_inertia_device(d_sh, [nb, n2], d_c)
        st.synchronize()
        got1[b0:b0 + nb] = d_c[0, :nb].cpu().numpy()
        if n2:
            assert np.array_equal(d_c[1, :n2].cpu().numpy(), want2)
    assert np.array_equal(got1, want)
    assert Ms[0].h2_info()["guard_reruns"] >= 1
    G.close()
    for M in Ms:
        M.close()


def test_kth_group_mixed_matches_fp64(pkg):
    """batching.kth_group over mixed handles: every k-th eigenvalue within tol
    of the handle's own FP64 h2_kth_eig, and of the dense oracle within tol +
    ||A - A~||_2."""
    import torch
    from paper_2311_08618_gb300 import batching
    st = torch.cuda.Stream()
    pts = [W.uniform_cube(512, 2, 71), W.uniform_cube(400, 3, 72)]
    ks = [200, 37]
    tol = 1e-8
    mats = [pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=24, max_lanes=16, precision=pkg.H2_PREC_MIXED,
                         stream=st.cuda_stream) for X in pts]
    lam, rounds, shifts = batching.kth_group(mats, ks, tol, st)
    for X, k, l in zip(pts, ks, lam):
        F = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=24, max_lanes=16)
        lf, _ = F.h2_kth_eig([k], tol)
        e, a = F.h2_compression_error(30)
        F.close()
        assert abs(l - lf[0]) <= tol
        ev = dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, KP, X))
        assert abs(l - ev[k - 1]) <= tol + 1.5 * e
    for M in mats:
        M.close()


def test_serving_mixed_matrices(pkg):
    """The serving layer over mixed handles: each result within tol of the
    same request on FP64 handles, and of the dense oracle within tol +
    ||A - A~||_2 (measured on the device)."""
    from paper_2311_08618_gb300 import serving
    mats = {"a": W.uniform_cube(512, 2, 81), "b": W.uniform_cube(300, 3, 82)}
    reqs = [("a", 1, 1e-8), ("a", 300, 1e-9), ("b", 150, 1e-8), ("b", 300, 1e-7)]
    out = {}
    errs = {}
    for prec in (pkg.H2_PREC_FP64, pkg.H2_PREC_MIXED):
        s = serving.Server()
        for nm, X in mats.items():
            s.add_matrix(nm, X, W.LAPLACE_EPS, KP, 64, 24, lanes=16, precision=prec)
            if prec == pkg.H2_PREC_FP64:
                errs[nm] = s.mats[nm].h2.h2_compression_error(30)[0]
        for m, k, tol in reqs:
            s.submit(m, k, tol)
        res = []
        while s.busy():
            s.step()
            res += s.poll()
        res += s.poll()
        out[prec] = {r.rid: r.result for r in res}
        s.close()
    for i, (m, k, tol) in enumerate(reqs):
        assert abs(out[pkg.H2_PREC_MIXED][i] - out[pkg.H2_PREC_FP64][i]) <= tol
        ev = dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, KP, mats[m]))
        assert abs(out[pkg.H2_PREC_MIXED][i] - ev[k - 1]) <= tol + 1.5 * errs[m]
