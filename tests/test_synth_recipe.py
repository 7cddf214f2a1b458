"""The seeded input generator draws what its recipe states (CPU): catalogs of
the 100k-event recipe (fault patches, Laplace noise with outliers) and the
1M-event recipe (normal noise), scaled down, checked by brute force against
the stated pair radius, neighbour count, observing stations, perturbations,
noise laws, listing order and network initialisation."""
import math

import numpy as np
import pytest

from oracle import spider_oracle as O
from paper_2508_12117_gb300 import synth


@pytest.fixture(scope="module")
def cat3():
    return synth.make_catalog(synth.scaled_spec(3, 3000))


@pytest.fixture(scope="module")
def cat4():
    return synth.make_catalog(synth.scaled_spec(4, 3000))


def test_pairs_are_the_nearest_neighbours_within_the_radius(cat3):
    s = cat3.spec
    x = cat3.init_xyzt[:, :3]
    pairs = {}
    for a, b in zip(cat3.i.tolist(), cat3.j.tolist()):
        pairs.setdefault(a, set()).add(b)
    rng = np.random.default_rng(0)
    for m in rng.choice(cat3.M, 200, replace=False):
        d = np.linalg.norm(x - x[m], axis=1)
        d[m] = np.inf
        cand = np.flatnonzero(d <= synth.PAIR_RADIUS_KM)
        want = set(cand[np.argsort(d[cand], kind="stable")][: s.n_neighbours].tolist())
        assert pairs.get(int(m), set()) == want


def test_observing_stations_are_the_nearest_ones(cat3):
    s = cat3.spec
    x = cat3.init_xyzt[:, :3]
    for m in np.random.default_rng(1).choice(np.unique(cat3.i), 100, replace=False):
        ks = set(cat3.k[cat3.i == m].tolist())
        d = np.linalg.norm(cat3.stations - x[m], axis=1)
        assert ks == set(np.argsort(d, kind="stable")[: s.n_obs_stations].tolist())
    # every (i, j) pair is observed at the same stations, once each
    key = (cat3.i.astype(np.int64) * cat3.M + cat3.j) * cat3.S + cat3.k
    assert np.unique(key).size == key.size


def test_listing_order_events_morton_observations_ijk(cat3):
    assert np.array_equal(O.morton_perm(cat3.init_xyzt[:, :3]), np.arange(cat3.M))
    key = np.stack([cat3.i, cat3.j, cat3.k], 1)
    assert all(tuple(key[a]) < tuple(key[a + 1]) for a in range(0, key.shape[0] - 1, 97))
    assert np.all(np.lexsort((cat3.k, cat3.j, cat3.i)) == np.arange(cat3.N))


def test_initial_catalog_perturbation(cat4):
    d = cat4.init_xyzt - cat4.true_xyzt
    horiz = d[:, :2].ravel()
    assert abs(horiz.std() - 0.5) < 0.03 and abs(horiz.mean()) < 0.03
    assert abs(d[:, 3].std() - 0.1) < 0.008
    assert cat4.init_xyzt[:, 2].min() >= 0.2 and cat4.true_xyzt[:, 2].min() >= 0.5


def _noise(cat):
    s = cat.spec
    T = lambda ev: synth._true_tt(cat.true_xyzt[ev, :3], cat.stations[cat.k], s.medium)
    return cat.dt - ((T(cat.i) + cat.true_xyzt[cat.i, 3]) - (T(cat.j) + cat.true_xyzt[cat.j, 3]))


def test_laplace_noise_with_two_percent_outliers(cat3):
    e = _noise(cat3)
    out = np.abs(e) > 0.1
    # outliers are U(-0.5, 0.5) s on 2 % of the observations: 80 % of them
    # exceed 0.1 s; a Laplace(0, 5 ms) draw does so with probability e^-20
    assert abs(out.mean() - 0.02 * 0.8) < 0.003
    inl = e[~out]
    assert abs(np.median(np.abs(inl)) - 0.005 * math.log(2.0)) < 0.0002   # Laplace median |e| = b ln 2
    assert abs(np.abs(inl).mean() - 0.005) < 0.0003                       # and mean |e| = b


def test_normal_noise_of_the_1m_event_recipe(cat4):
    e = _noise(cat4)
    assert abs(e.std() - 0.005) < 0.0002 and abs(e.mean()) < 0.0002
    assert np.abs(e).max() < 0.005 * 7


def test_network_initialisation():
    net = synth.mlp_weights(256, 12345)
    dims = [6, 256, 256, 256, 256, 1]
    for l in range(5):
        bound = math.sqrt(6.0 / (dims[l] + dims[l + 1])) * 0.1
        W = net["W"][l].astype(np.float64)
        assert W.shape == (dims[l + 1], dims[l]) and np.abs(W).max() <= bound
        if W.size > 1000:
            assert abs(W.std() - bound / math.sqrt(3.0)) < 0.05 * bound    # uniform on [-b, b]
    assert all(not np.any(net["b"][l]) for l in range(4))
    assert net["b"][4][0] == np.float32(1.0 / 5.5)
