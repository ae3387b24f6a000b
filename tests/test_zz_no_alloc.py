"""h2_dense_inertia_noalloc, the entry point for callers that cannot allocate
device memory (a fixed device memory budget reserved up front, or no
device-wide synchronization allowed): called through the C ABI, its counts must equal those
of h2_inertia (the allocating path) on the same small dense matrix, on two
calls in a row that share the library's static scratch array.  Collected last
on purpose (file name) so a stop-at-first-failure run has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2311_08618_gb300 as pkg
    from paper_2311_08618_gb300 import build
    build.build()
    return torch, pkg


def _dense_on_device(torch, X, p0):
    """A_ij = 1/(|x_i - x_j| + p0) built with torch on the GPU (test input)."""
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda")
    diff = Xt[:, None, :] - Xt[None, :, :]
    r = torch.sqrt((diff * diff).sum(dim=2))
    return (1.0 / (r + p0)).contiguous()


def test_noalloc_matches_allocating_path_two_calls(env):
    torch, pkg = env
    n = 48
    X = W.uniform_cube(n, 2, 31)
    p0 = 1e-3
    # n <= leaf: one cluster, so h2_inertia runs the dense Bunch-Kaufman LDL^T of A - sigma I
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, (p0, 0, 0, 0), leaf=64, rank=8, max_lanes=32)
    A = _dense_on_device(torch, X, p0)
    ev = np.linalg.eigvalsh(A.cpu().numpy())
    mids = 0.5 * (ev[1:] + ev[:-1])
    sets = [np.concatenate([mids[::3], [ev[0] - 1.0, ev[-1] + 1.0]]), mids[1::3]]
    L = pkg.lib()
    for shifts in sets:                                    # two calls in a row
        want, want_mp = M.h2_inertia(shifts)
        ns = len(shifts)
        d_sh = torch.tensor(shifts, dtype=torch.float64, device="cuda")
        d_cnt = torch.full((ns,), -1, dtype=torch.int64, device="cuda")
        d_mp = torch.full((ns,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.h2_dense_inertia_noalloc(C.c_void_p(A.data_ptr()), n, n, C.c_void_p(d_sh.data_ptr()), ns,
                                        C.c_void_p(d_cnt.data_ptr()), C.c_void_p(d_mp.data_ptr()), None)
        assert rc == 0, L.h2_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(d_cnt.cpu().numpy(), want)
        assert np.allclose(d_mp.cpu().numpy(), want_mp, rtol=1e-9, atol=1e-12 * np.abs(ev).max())
        assert np.array_equal(want, [np.sum(ev < s) for s in shifts])
    M.close()


def test_noalloc_rejects_oversize_without_launch(env):
    torch, pkg = env
    L = pkg.lib()
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    c = torch.zeros(4, dtype=torch.int64, device="cuda")
    p = C.c_void_p(d.data_ptr())
    # 2 * 1024 * 1024 doubles > the static maximum; n above the limit; lda < n
    assert L.h2_dense_inertia_noalloc(p, 1024, 1024, p, 2, C.c_void_p(c.data_ptr()), None, None) == -1
    assert b"static scratch" in L.h2_last_error()
    assert L.h2_dense_inertia_noalloc(p, 2000, 2000, p, 1, C.c_void_p(c.data_ptr()), None, None) == -1
    assert L.h2_dense_inertia_noalloc(p, 8, 4, p, 1, C.c_void_p(c.data_ptr()), None, None) == -1
