"""The library's host planner (tree, top-down block tree, fill-in closure,
distance-2 colouring; h2_plan_summary, no device needed) against the oracle's
independent implementation of the same readings: the same tree permutation,
the same near / fill / far pairs per level and the same colours."""
import numpy as np
import pytest

import workloads as W
from oracle import h2 as oh2


@pytest.fixture(scope="module")
def binding():
    from paper_2311_08618_gb300 import binding as b
    from paper_2311_08618_gb300 import build
    build.build()
    return b


CASES = [
    ("square300", lambda: W.uniform_cube(300, 2, 21), 32, oh2.ADM_BOX),
    ("square1024", lambda: W.uniform_cube(1024, 2, 1), 64, oh2.ADM_BOX),
    ("cube800", lambda: W.uniform_cube(800, 3, 22), 32, oh2.ADM_BOX),
    ("cube300_ragged", lambda: W.uniform_cube(300, 3, 22), 40, oh2.ADM_BOX),
    ("cylinder600", lambda: W.cylinder_lattice(600, 53), 40, oh2.ADM_BOX),
    ("line100", lambda: W.line_points(100), 16, oh2.ADM_BOX),
    ("square512_center", lambda: W.uniform_cube(512, 2, 5), 32, oh2.ADM_CENTER),
    ("circle1024_weak", lambda: W.unit_circle(1024, 5), 64, oh2.ADM_WEAK),
    # the 3D n = 65536 configuration (leaf 256): 191 colours at the leaf level
    ("cube65536_leaf256", lambda: W.uniform_cube(65536, 3, 2), 256, oh2.ADM_BOX),
]


@pytest.mark.parametrize("name,mk,leaf,rule", CASES, ids=[c[0] for c in CASES])
def test_planner_matches_oracle(binding, name, mk, leaf, rule):
    X = mk()
    perm, per, colours = binding.plan_summary(X, leaf, 1.0, rule)
    st = oh2.build_structure(X, leaf, 1.0, rule)
    assert np.array_equal(perm, st.perm)
    assert per.shape[0] == st.L + 1
    for l in range(st.L + 1):
        nc = len(st.offsets[l]) - 1
        assert per[l, 0] == nc
        assert per[l, 1] == int(st.near[l].sum()), ("near", l)
        assert per[l, 2] == int(st.fill[l].sum()), ("fill", l)
        assert per[l, 3] == int(st.far[l].sum()), ("far", l)
        assert np.array_equal(colours[l], np.asarray(st.colors[l])), ("colours", l)
        assert per[l, 4] == len(set(np.asarray(st.colors[l]).tolist()))


def test_planner_rejects_bad_arguments(binding):
    with pytest.raises(binding.H2Error):
        binding.plan_summary(W.uniform_cube(10, 2, 1), 1)          # leaf < 2
    with pytest.raises(binding.H2Error):
        binding.plan_summary(W.uniform_cube(10, 2, 1), 4, rule=7)  # unknown rule


@pytest.mark.parametrize("name,mk,leaf,rule", CASES[:8], ids=[c[0] for c in CASES[:8]])
def test_colour_writes_are_disjoint(binding, name, mk, leaf, rule):
    """What the concurrent launches of one colour and the lookahead schedule
    rely on, checked on the planner's colours: within a colour no two clusters
    share a stored block (near or fill), and no Schur target block (x, y),
    x, y in {p} + near(p), belongs to two clusters, so every block takes at
    most one Schur update per colour."""
    X = mk()
    _, _, colours = binding.plan_summary(X, leaf, 1.0, rule)
    st = oh2.build_structure(X, leaf, 1.0, rule)
    for l in range(st.L + 1):
        near = np.asarray(st.near[l]).astype(bool)
        fill = np.asarray(st.fill[l]).astype(bool)
        col = np.asarray(colours[l])
        nc = len(col)
        for c in range(col.max() + 1):
            members = np.nonzero(col == c)[0]
            written = {}
            rows = {}
            for p in members:
                tg = [p] + [x for x in range(nc) if x != p and near[p, x]]
                for i, a in enumerate(tg):
                    for b in tg[:i + 1]:
                        key = (max(a, b), min(a, b))
                        assert key not in written, (l, c, p, written.get(key), key)
                        written[key] = p
                rows[p] = {x for x in range(nc) if x != p and (near[p, x] or fill[p, x])}
            for p in members:
                for q in members:
                    if p != q:
                        assert q not in rows[p], (l, c, p, q)
