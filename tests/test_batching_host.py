"""Host logic of the many-matrix k-th eigenvalue rounds
(paper_2311_08618_gb300.batching.bracket_rounds), driven by exact counts
#{lambda < mu} of small symmetric matrices (numpy eigvalsh) instead of the
GPU group batch."""
import numpy as np

import workloads as W
from paper_2311_08618_gb300.batching import bracket_rounds


def _spectra():
    out = []
    for i, n in enumerate((5, 17, 40, 64)):
        A = W.gaussian(70 + i, n * n).reshape(n, n)
        A = A + A.T
        out.append(np.linalg.eigvalsh(A))
    return out


def test_rounds_reach_every_k_within_tol():
    ev = _spectra()
    ks = [1, 9, 40, 33]
    a = [e.min() - 1.0 for e in ev]
    b = [e.max() + 1.0 for e in ev]
    calls = []

    def evaluate(mu, ns):
        calls.append(ns.copy())
        nu = np.zeros(mu.shape, dtype=np.int64)
        for i, e in enumerate(ev):
            nu[i, :ns[i]] = np.searchsorted(e, mu[i, :ns[i]], side="left")   # #{lambda < mu}
        return nu

    tol, lanes = 1e-9, 4
    mid, rounds, shifts = bracket_rounds(a, b, ks, tol, lanes, evaluate)
    for i, k in enumerate(ks):
        assert abs(mid[i] - ev[i][k - 1]) < tol / 2
    # (lanes + 1)-section: the widest start interval shrinks by 5 per round
    width = max(bb - aa for aa, bb in zip(a, b))
    assert rounds <= int(np.ceil(np.log(width / tol) / np.log(lanes + 1))) + 1
    # a finished matrix asks for no shifts; the count of shifts is the sum of ns
    assert shifts == int(sum(c.sum() for c in calls))
    assert all(((c == 0) | (c == lanes)).all() for c in calls)


def test_single_lane_is_bisection():
    # spectrum {-1, 0.25, 3}: counts #{lambda < mu} for mu < 3
    mid, rounds, _ = bracket_rounds([-2.0], [4.0], [2], 1e-6, 1,
                                    lambda mu, ns: (mu < 0.25).astype(np.int64) + (mu >= 0.25) * 2
                                    - (mu < -1.0))
    assert abs(mid[0] - 0.25) < 5e-7
    assert rounds == int(np.ceil(np.log2(6.0 / 1e-6)))


def test_package_modules_import_without_a_gpu():
    """Every module of the package imports on a CPU-only host (the library
    itself is loaded only when a call needs it)."""
    import importlib
    for m in ("binding", "batching", "serving", "sharding", "build"):
        importlib.import_module("paper_2311_08618_gb300." + m)
