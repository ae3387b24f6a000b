"""GPU checks of the boundary's memory rules: admission by HBM footprint
(h2_options.hbm_budget) and an out-of-memory build that fails with
H2_ERR_OOM, leaves no device memory behind, and does not disturb the next
build."""
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


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_oom_build_leaks_nothing(pkg):
    X = W.uniform_cube(1024, 2, 1)
    free0 = _free()
    # 65535 lanes of the n = 1024 workload need about 640 GB
    with pytest.raises(pkg.H2Error) as e:
        pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=65535)
    assert e.value.code == -2 and "bytes" in str(e.value)
    assert abs(_free() - free0) <= 64 << 20
    # a budget below one lane's workspace
    with pytest.raises(pkg.H2Error) as e:
        pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=0, hbm_budget=1)
    assert e.value.code == -2 and "hbm_budget" in str(e.value)
    assert abs(_free() - free0) <= 64 << 20
    # the next build works and counts as before
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=16)
    A = dense.kernel_matrix(W.LAPLACE_EPS, KP, X)
    ev = np.linalg.eigvalsh(A)
    s = np.array([ev[0] - 1.0, 0.5 * (ev[300] + ev[301]), ev[-1] + 1.0])
    got, _ = M.h2_inertia(s)
    assert list(got) == [0, 301, 1024]
    M.close()
    assert abs(_free() - free0) <= 64 << 20


def test_hbm_budget_sets_the_lanes(pkg):
    X = W.uniform_cube(1024, 2, 1)
    one = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=1)
    per_lane = one.h2_info()["workspace_bytes"]
    one.close()
    budget = int(10.5 * per_lane)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=0, hbm_budget=budget)
    info = M.h2_info()
    assert info["lanes"] == 10
    assert info["workspace_bytes"] <= budget
    # max_lanes bounds the budget's choice
    M2 = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=16, max_lanes=4, hbm_budget=budget)
    assert M2.h2_info()["lanes"] == 4
    c1, _ = M.h2_inertia(np.linspace(900.0, 1100.0, 25))
    c2, _ = M2.h2_inertia(np.linspace(900.0, 1100.0, 25))
    assert np.array_equal(c1, c2)
    M.close()
    M2.close()
