"""The paper's own geometry (Sec. 5.1): A_ij = 1/(|x_i - x_j| + 1e-3) on points
uniformly distributed on the unit circle, under strong (box) admissibility,
with the settings of the scaling experiment (leaf 64, rank cap 32, eps_H2 =
1e-7 relative to ||A||_inf, k = n/2, eps_ev = 1e-5, start interval [0, 2048]).

GPU counts equal the H^2 oracle's (bit-exact bar); lambda_{n/2} from the
constant start interval and from the Gershgorin interval agrees with the
dense eigenvalue within eps_ev/2 + ||A - A~||_2 (Eq. error-bound plus Weyl).
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


def test_circle_strong_admissibility(pkg):
    import torch
    from paper_2311_08618_gb300 import batching
    n = 2048
    X = W.unit_circle(n, 5)
    st = torch.cuda.Stream()
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, KP, leaf=64, rank=32, eta=1.0, eps_h2=1e-7, max_lanes=16,
                     stream=st.cuda_stream)
    ref = oh2.construct(X, W.LAPLACE_EPS, KP, 64, 32, 1.0, eps_h2=1e-7)
    info = M.h2_info()
    assert info["near_pairs"] < info["leaves"] ** 2 // 4      # a 1D manifold: mostly far field
    assert info["max_rank"] == max(max(r) for r in ref.ranks)
    ev = dense.eigenvalues(dense.kernel_matrix(W.LAPLACE_EPS, KP, X))
    err, _ = M.h2_compression_error(40)
    # counts against the oracle
    s = np.concatenate([0.5 * (ev[1:] + ev[:-1])[::97], [0.0, 2048.0]])
    got, mp = M.h2_inertia(s)
    thr = 1e-10 * ref.scale
    for x, c, p in zip(s, got, mp):
        want, wmp, _ = oh2.h2_inertia(ref, x)
        if min(p, wmp) > thr:
            assert c == want, (x, c, want)
    k = n // 2
    assert got[-2] < k <= got[-1]              # nu(0) < k <= nu(2048)
    # k = n/2 from [0, 2048] (the paper's start) and from the Gershgorin interval
    G = pkg.H2Group([M])
    lam, rounds, shifts = batching.kth_group([M], [k], 1e-5, st, G, start=([0.0], [2048.0]))
    lam2, eb = M.h2_kth_eig([k], 1e-5)
    assert abs(lam[0] - ev[k - 1]) <= 0.5e-5 + 1.5 * err
    assert abs(lam2[0] - ev[k - 1]) <= 0.5e-5 + 1.5 * err
    assert abs(lam[0] - lam2[0]) <= 1e-5
    G.close()
    M.close()
