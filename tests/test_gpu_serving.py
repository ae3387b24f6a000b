"""Continuous-batching server: every result equals its stand-alone result
within tol (both bracket the same lambda_k of A~ to width < tol) and the
dense oracle within tol + ||A - A~|| + 1e-8 ||A||; admission never puts more
requests in flight on a matrix than it has lanes."""
import numpy as np
import pytest

import workloads as W
from oracle import dense

pytestmark = pytest.mark.gpu

MATS = {
    "lap2d": (lambda: W.uniform_cube(512, 2, 51), W.LAPLACE_EPS, (1e-3, 0, 0, 0), 64, 16),
    "yuk3d": (lambda: W.uniform_cube(400, 3, 52), W.YUKAWA_EPS, (1e-3, 0, 0, 0), 50, 24),
    "cyl": (lambda: W.cylinder_lattice(600, 53), W.GAUSS_PLUS_INV, (1e-2, 0.1, 0, 0), 40, 16),
}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_08618_gb300 import build, serving
    build.build()
    return serving


def _server(serving, names, lanes=16):
    s = serving.Server()
    for nm in names:
        pts, kind, kp, leaf, rank = MATS[nm]
        s.add_matrix(nm, pts(), kind, kp, leaf, rank, lanes=lanes)
    return s


def _drain(s):
    out = []
    while s.busy():
        s.step()
        out += s.poll()
    return out + s.poll()


REQS = [("lap2d", 1, 1e-8), ("lap2d", 256, 1e-10), ("lap2d", 257, 1e-6), ("lap2d", 512, 1e-9),
        ("yuk3d", 200, 1e-8), ("yuk3d", 1, 1e-7), ("yuk3d", 399, 1e-10),
        ("cyl", 300, 1e-8), ("cyl", 301, 1e-8), ("cyl", 600, 1e-6)]


def test_results_alone_equal_results_in_mix(env):
    serving = env
    alone = {}
    for i, (m, k, tol) in enumerate(REQS):
        s = _server(serving, [m])
        s.submit(m, k, tol)
        r = _drain(s)
        assert len(r) == 1
        alone[i] = r[0].result
        s.close()
    s = _server(serving, list(MATS))
    ids = {}
    for i, (m, k, tol) in enumerate(REQS[:5]):
        ids[s.submit(m, k, tol)] = i
    s.step()
    s.step()                                   # the rest arrive while work is in flight
    for i, (m, k, tol) in enumerate(REQS[5:], start=5):
        ids[s.submit(m, k, tol)] = i
    res = _drain(s)
    assert len(res) == len(REQS)
    for r in res:
        i = ids[r.rid]
        m, k, tol = REQS[i]
        assert abs(r.result - alone[i]) <= tol, (REQS[i], r.result, alone[i])
        pts, kind, kp, leaf, rank = MATS[m]
        A = dense.kernel_matrix(kind, kp, pts())
        ev = dense.eigenvalues(A)
        assert abs(r.result - ev[k - 1]) <= tol + 1e-7 * np.abs(ev).max(), (REQS[i], r.result, ev[k - 1])
    s.close()


def test_admission_respects_lanes(env):
    serving = env
    s = _server(serving, ["lap2d"], lanes=2)
    for k in (10, 100, 200, 300, 400):
        s.submit("lap2d", k, 1e-6)
    peak = 0
    out = []
    while s.busy():
        s.step()
        peak = max(peak, len(s.mats["lap2d"].active))
        out += s.poll()
    out += s.poll()
    assert peak <= 2 and len(out) == 5
    s.close()


def test_table_reuse_shortens_later_requests(env):
    serving = env
    s = _server(serving, ["lap2d"])
    s.submit("lap2d", 256, 1e-8)
    first = _drain(s)[0]
    s.submit("lap2d", 256, 1e-8)              # same k again: starts from the table
    again = _drain(s)[0]
    assert again.rounds < first.rounds
    assert abs(again.result - first.result) <= 1e-8
    s.close()


def test_group_and_separate_batches_agree(env):
    """The same requests on a server whose matrices share lanes (one group
    batch per tick) and on one whose lanes differ (per-matrix batches back to
    back): equal results within tol, and the first server uses a group."""
    serving = env
    s1 = _server(serving, ["lap2d", "yuk3d", "cyl"], lanes=8)
    s2 = serving.Server()
    for nm, ln in (("lap2d", 8), ("yuk3d", 16), ("cyl", 8)):
        pts, kind, kp, leaf, rank = MATS[nm]
        s2.add_matrix(nm, pts(), kind, kp, leaf, rank, lanes=ln)
    for s in (s1, s2):
        for m, k, tol in REQS:
            s.submit(m, k, tol)
    r1 = sorted(_drain(s1), key=lambda r: r.rid)
    r2 = sorted(_drain(s2), key=lambda r: r.rid)
    assert s1.group is not None and s2.group is None
    assert len(r1) == len(r2) == len(REQS)
    for a, b in zip(r1, r2):
        assert abs(a.result - b.result) <= a.tol
    s1.close()
    s2.close()
