"""The seeded input generators produce the statistics they claim."""
import numpy as np

from synth import corner_wells, five_spot_wells, gaussian_field, layered_field
from synth.configs import random_edges, workload


def test_gaussian_field_covariance():
    # exponential covariance sigma^2 exp(-r/lam): check variance and the lag-lam correlation
    sig, lam = 1.5, 6.0
    var, c_lag = [], []
    for seed in range(6):
        g = gaussian_field((192, 192), sig, lam, seed)
        g = g - g.mean()
        var.append(np.mean(g * g))
        L = int(lam)
        c_lag.append(0.5 * (np.mean(g[:, :-L] * g[:, L:]) + np.mean(g[:-L, :] * g[L:, :])))
    v = np.mean(var)
    assert abs(v / sig**2 - 1) < 0.15
    assert abs(np.mean(c_lag) / v - np.exp(-1.0)) < 0.08


def test_gaussian_field_seeded():
    a = gaussian_field((6, 10, 12), 2.0, 3.0, 7)
    b = gaussian_field((6, 10, 12), 2.0, 3.0, 7)
    c = gaussian_field((6, 10, 12), 2.0, 3.0, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_layered_field_ratios():
    K = layered_field((5, 20, 30), 3.0, (4, 20), (1e-3, 0.1), seed=0)
    r = K[2] / K[0]
    assert np.allclose(K[0], K[1])
    for k in range(5):
        assert np.allclose(r[k], r[k].flat[0])
        assert 1e-3 <= r[k].flat[0] <= 0.1


def test_wells_balance():
    for f in (corner_wells(7, 5, 3), five_spot_wells(9, 11, 4)):
        assert abs(f.sum()) < 1e-14
        assert (f != 0).sum() > 0


def test_random_edges_cover():
    rng = np.random.default_rng(0)
    e = random_edges(256, [8, 12, 16], rng)
    assert sum(e) == 256 and all(1 <= x <= 16 for x in e)


def test_named_workload_shapes():
    w = workload("c2")
    assert w.n_sub == 2244 and w.cells == 60 * 220 * 85
    w = workload("c5")
    assert w.n_sub == 32768
