"""GPU compression error and the exported representation (Sec. 3.1).

Accuracy requirement of the compression: ||A - A~||_2 / ||A||_2 <= 1e-8 for the GPU's own A~.
The GPU representation is exported (h2_export) and written out densely here;
its error is measured three ways: from that dense A~ on the host, by the
library's device power iteration (h2_compression_error), and against the
oracle's A~ of the same construction.  The oracle's generalized LDL^T then
runs on the GPU's exported A~ and must count exactly as the GPU does.
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


def exported_levels(M):
    return [M.h2_export(l) for l in range(M.h2_info()["levels"])]


def expanded_bases(ex):
    """E[l][c] (points x r_c): the leaf U^S, then the nested products with the
    transfer matrices (Eq. transfer-matrices)."""
    L = len(ex) - 1
    E = [None] * (L + 1)
    lv = ex[L]
    E[L] = []
    for c in range(len(lv["ranks"])):
        m = lv["offsets"][c + 1] - lv["offsets"][c]
        E[L].append(lv["Q"][c, :m, :lv["ranks"][c]])
    for l in range(L - 1, -1, -1):
        lv = ex[l]
        E[l] = []
        for P in range(len(lv["ranks"])):
            E1, E2 = E[l + 1][2 * P], E[l + 1][2 * P + 1]
            r1, r2 = E1.shape[1], E2.shape[1]
            blk = np.zeros((E1.shape[0] + E2.shape[0], r1 + r2))
            blk[:E1.shape[0], :r1] = E1
            blk[E1.shape[0]:, r1:] = E2
            E[l].append(blk @ lv["Q"][P, :r1 + r2, :lv["ranks"][P]])
    return E


def dense_from_export(ex):
    """A~ (tree order) from the exported near blocks and couplings."""
    L = len(ex) - 1
    off = ex[L]["offsets"]
    n = int(off[-1])
    E = expanded_bases(ex)
    out = np.zeros((n, n))
    lv = ex[L]
    for (c, d), B in zip(lv["near_pairs"], lv["B"]):
        mc, md = off[c + 1] - off[c], off[d + 1] - off[d]
        Qc, Qd = lv["Q"][c, :mc, :mc], lv["Q"][d, :md, :md]
        blk = Qc @ B[:mc, :md] @ Qd.T
        out[off[c]:off[c + 1], off[d]:off[d + 1]] = blk
        out[off[d]:off[d + 1], off[c]:off[c + 1]] = blk.T
    for l in range(L + 1):
        o = ex[l]["offsets"]
        for (c, d), C in zip(ex[l]["far_pairs"], ex[l]["C"]):
            rc, rd = ex[l]["ranks"][c], ex[l]["ranks"][d]
            blk = E[l][c] @ C[:rc, :rd] @ E[l][d].T
            out[o[c]:o[c + 1], o[d]:o[d + 1]] = blk
            out[o[d]:o[d + 1], o[c]:o[c + 1]] = blk.T
    return out


def oracle_on_export(ref, ex):
    """The oracle's H2Matrix with the GPU's bases, couplings and near blocks
    (same tree, block structure and tolerances as `ref`)."""
    L = len(ex) - 1
    E = expanded_bases(ex)
    Q = []
    for l in range(L + 1):
        lv = ex[l]
        Ql = []
        for c in range(len(lv["ranks"])):
            if l == L:
                m = lv["offsets"][c + 1] - lv["offsets"][c]
            else:
                m = ex[l + 1]["ranks"][2 * c] + ex[l + 1]["ranks"][2 * c + 1]
            Ql.append(lv["Q"][c, :m, :m].copy())
        Q.append(Ql)
    coupling = [dict() for _ in range(L + 1)]
    for l in range(L + 1):
        for (c, d), C in zip(ex[l]["far_pairs"], ex[l]["C"]):
            rc, rd = ex[l]["ranks"][c], ex[l]["ranks"][d]
            coupling[l][(int(c), int(d))] = C[:rc, :rd].copy()
            coupling[l][(int(d), int(c))] = C[:rc, :rd].T.copy()
    off = ex[L]["offsets"]
    near = {}
    for (c, d), B in zip(ex[L]["near_pairs"], ex[L]["B"]):
        mc, md = off[c + 1] - off[c], off[d + 1] - off[d]
        near[(int(c), int(d))] = B[:mc, :md].copy()
    ranks = [list(int(r) for r in ex[l]["ranks"]) for l in range(L + 1)]
    return oh2.H2Matrix(ref.st, ref.kind, ref.kparams, ref.X, ref.scale, ref.tol, ref.fill_cap, ranks, Q, E,
                        coupling, near, ref.gershgorin)


C1_KP = (1e-3, 0.0, 0.0, 0.0)


@pytest.mark.parametrize("rank", [16, 17])
def test_bench_configuration_compression(pkg, rank):
    """n = 1024 unit-square Laplace, leaf 64, eta 1, eps_H2 = 1e-10.  At the
    configured rank cap 16 the cap binds (h2_info flags it) and the error is
    1.07e-8 ||A||_2, just above the 1e-8 criterion; at cap 17 it meets it.
    Both measured on the GPU's own A~."""
    X = W.uniform_cube(1024, 2, 1)
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, C1_KP, leaf=64, rank=rank, eta=1.0, max_lanes=8)
    ref = oh2.construct(X, W.LAPLACE_EPS, C1_KP, 64, rank, 1.0)
    A = dense.kernel_matrix(W.LAPLACE_EPS, C1_KP, ref.X)
    n2 = np.linalg.norm(A, 2)
    ex = exported_levels(M)
    assert np.array_equal(ex[-1]["offsets"], np.array(ref.st.offsets[-1]))
    for l in range(len(ex)):
        assert list(ex[l]["ranks"]) == list(ref.ranks[l])
        assert list(ex[l]["colours"]) == list(ref.st.colors[l])
    At_gpu = dense_from_export(ex)
    At_ref = oh2.dense_approximation(ref)
    err_gpu = np.linalg.norm(A - At_gpu, 2)
    err_ref = np.linalg.norm(A - At_ref, 2)
    # the GPU's and the oracle's A~ come from the same sketch and pivoted QR:
    # they differ by far less than either's compression error
    assert np.linalg.norm(At_gpu - At_ref, 2) <= 0.05 * err_ref
    assert abs(err_gpu - err_ref) <= 0.05 * err_ref
    # skeleton columns of the leaf bases agree entry by entry with the oracle's.
    # Column j comes from the sketch remainder after j reflections (relative
    # size down to 1e-8 at j = 15 here), so rounding differences of the two
    # sketches move the late columns more: a 1e-16 relative perturbation moved
    # them by up to 4e-9 in the oracle itself.
    lv = ex[-1]
    for c in range(len(lv["ranks"])):
        m = lv["offsets"][c + 1] - lv["offsets"][c]
        r = lv["ranks"][c]
        Qr = ref.Q[-1][c]
        if r >= 2:
            assert np.abs(lv["Q"][c, :m, :r // 2] - Qr[:, :r // 2]).max() <= 1e-10
        if r >= 1:
            assert np.abs(lv["Q"][c, :m, :r] - Qr[:, :r]).max() <= 1e-6
        # the full square basis stays orthogonal
        assert np.abs(lv["Q"][c, :m, :m].T @ lv["Q"][c, :m, :m] - np.eye(m)).max() <= 1e-13
    # the device's power iteration measures the same error and norm
    e_dev, a_dev = M.h2_compression_error(40)
    assert a_dev == pytest.approx(n2, rel=1e-6)
    assert 0.95 * err_gpu <= e_dev <= 1.0001 * err_gpu
    info = M.h2_info()
    rel = err_gpu / n2
    if rank == 16:
        assert 1.0e-8 < rel < 1.1e-8
        assert info["cap_bound"] > 0 and info["max_residual"] > info["trunc_tol"]
    else:
        assert rel <= 1e-8
    M.close()


def test_nested_transfers_compression(pkg):
    """Points on the unit circle (the paper's Sec. 5.1 geometry), where the
    upper levels carry far field through the transfer matrices: the device
    H^2 product (upward and downward passes) gives the error of the exported
    A~, which matches the oracle's construction."""
    X = W.unit_circle(2048, 5)
    kp = C1_KP
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=64, rank=24, eta=1.0, eps_h2=1e-9, max_lanes=8)
    ref = oh2.construct(X, W.LAPLACE_EPS, kp, 64, 24, 1.0, eps_h2=1e-9)
    ex = exported_levels(M)
    assert sum(int(np.sum(ex[l]["ranks"])) for l in range(len(ex) - 1)) > 0   # transfers in use
    assert sum(len(ex[l]["far_pairs"]) for l in range(len(ex) - 1)) > 0
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, ref.X)
    At_gpu = dense_from_export(ex)
    At_ref = oh2.dense_approximation(ref)
    err_gpu = np.linalg.norm(A - At_gpu, 2)
    err_ref = np.linalg.norm(A - At_ref, 2)
    assert abs(err_gpu - err_ref) <= 0.05 * err_ref + 1e-12 * np.linalg.norm(A, 2)
    e_dev, a_dev = M.h2_compression_error(60)
    assert a_dev == pytest.approx(np.linalg.norm(A, 2), rel=1e-6)
    assert 0.9 * err_gpu <= e_dev <= 1.0001 * err_gpu + 1e-13 * a_dev
    assert err_gpu / a_dev <= 1e-8
    M.close()


def test_oracle_ldl_on_the_gpu_representation(pkg):
    """The oracle's generalized LDL^T (Sec. 3.2-3.4) on the GPU's exported A~
    counts exactly as the GPU does wherever min |pivot| > 1e-10 ||A||."""
    X = W.uniform_cube(512, 2, 23)
    kp = C1_KP
    M = pkg.H2Matrix(X, W.LAPLACE_EPS, kp, leaf=32, rank=16, eta=1.0, max_lanes=32)
    ref = oh2.construct(X, W.LAPLACE_EPS, kp, 32, 16, 1.0)
    hx = oracle_on_export(ref, exported_levels(M))
    At = oh2.dense_approximation(hx)
    ev = np.linalg.eigvalsh(At)
    s = np.concatenate([0.5 * (ev[1:] + ev[:-1])[::23], [ev[0] - 1.0, ev[-1] + 1.0]])
    got, mp = M.h2_inertia(s)
    thr = 1e-10 * ref.scale
    checked = 0
    for x, c, p in zip(s, got, mp):
        want, wmp, _ = oh2.h2_inertia(hx, x)
        assert want == np.sum(ev < x) or min(p, wmp) <= thr
        if min(p, wmp) > thr:
            assert c == want, (x, c, want)
            checked += 1
    assert checked >= len(s) - 2
    M.close()
