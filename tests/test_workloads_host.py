"""The seeded input generators (no arithmetic of the method): SplitMix64
against its published test vector, the derived uniforms and Gaussians, and
the shapes of the point sets the configurations describe."""
import math

import numpy as np

import workloads as W


def test_splitmix64_published_vector():
    # the first outputs of SplitMix64 from state 1234567, as listed with the
    # generator's reference implementation
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in W.splitmix64(1234567, 5)] == want


def test_uniform_and_gaussian():
    u = W.uniform(9, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))        # top 53 bits
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002
    assert np.array_equal(u, W.uniform(9, 200_000))                # seeded
    g = W.gaussian(9, 200_001)
    assert g.shape == (200_001,)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.01
    assert abs(np.mean(g ** 4) - 3.0) < 0.05


def test_point_sets():
    X = W.uniform_cube(1000, 3, 2)
    assert X.shape == (1000, 3) and X.min() >= 0.0 and X.max() < 1.0
    C = W.cylinder_lattice(1000, 4)
    per_ring = int(round(2.0 * math.pi * 5.0 / 0.14))
    assert per_ring == 224
    r = np.hypot(C[:, 0], C[:, 1])
    assert np.all(np.abs(r - 5.0) < 0.1)
    ring = np.arange(1000) // per_ring
    assert np.all(np.abs(C[:, 2] - 0.14 * ring) < 0.1)
    U = W.unit_circle(500, 5)
    assert np.allclose(np.hypot(U[:, 0], U[:, 1]), 1.0)
    assert np.array_equal(W.line_points(4).ravel(), [1.0, 2.0, 3.0, 4.0])


def test_batch_members_distribution():
    ms = W.batch_members()
    assert len(ms) == 512
    ns = np.array([m.points.shape[0] for m in ms])
    ds = np.array([m.points.shape[1] for m in ms])
    assert ns.min() >= 2048 and ns.max() < 32768
    assert 200 < np.sum(ds == 3) < 312                       # d = 3 with probability 1/2
    assert all((m.leaf, m.rank) == ((64, 16) if m.points.shape[1] == 2 else (256, 32)) for m in ms)
    assert all(1 <= m.ks[0] <= m.points.shape[0] for m in ms)
