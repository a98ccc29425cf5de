"""Pins of the oracle's paper-faithful map mode (Sec. 3.2, the algorithm for
building a map by random marking).

* every map holds max(1, floor(N/10)) pairs whose sites are distinct and
  never inside another pair's covering (its sites and their neighbours) --
  the defining property of a map, checked by brute force;
* adjacency is allowed: on 4 x 4 the partner is a neighbour of a in about
  4/15 of the maps;
* the first pair of a map is a uniformly random ordered pair of distinct sites
  (chi-square over the 240 ordered pairs of 4 x 4);
* on 4 x 4 a map is one random pair -- the paper's serial algorithm -- so the
  map chain must reproduce exact enumeration, low-temperature peak included;
* on 8 x 8 the map chain and the colour-schedule chain sample the same
  ensemble.
"""
import numpy as np
import pytest

import oracle

from .mcstats import batch_heat, batch_mean, energy
from .test_oracle_physics import exact_averages


def _neighbours(Lx, Ly, s):
    x, y = s % Lx, s // Lx
    return {y * Lx + (x + 1) % Lx, y * Lx + (x - 1) % Lx, ((y + 1) % Ly) * Lx + x,
            ((y - 1) % Ly) * Lx + x}


@pytest.mark.parametrize("Lx,Ly", [(4, 4), (8, 8), (12, 8), (20, 16), (64, 32)])
def test_map_pairs_are_non_interacting(Lx, Ly):
    N = Lx * Ly
    for m in range(6):
        pairs = oracle.map_build(Lx, Ly, 11, m)
        assert pairs.shape == (max(1, N // 10), 2)
        sites = pairs.reshape(-1)
        assert len(set(sites.tolist())) == len(sites)
        assert sites.min() >= 0 and sites.max() < N
        cover = [{int(a), int(b)} | _neighbours(Lx, Ly, a) | _neighbours(Lx, Ly, b)
                 for a, b in pairs]
        for k, (a, b) in enumerate(pairs):
            for l in range(len(pairs)):
                if l != k:
                    assert int(a) not in cover[l] and int(b) not in cover[l]
        assert np.array_equal(pairs, oracle.map_build(Lx, Ly, 11, m))
    assert not np.array_equal(oracle.map_build(Lx, Ly, 11, 0), oracle.map_build(Lx, Ly, 11, 1))


def test_first_pair_is_a_uniform_ordered_pair_and_may_be_adjacent():
    Lx = Ly = 4
    N = 16
    nmaps = 24000
    counts = np.zeros((N, N), dtype=np.int64)
    adjacent = 0
    for m in range(nmaps):
        a, b = oracle.map_build(Lx, Ly, 5, m)[0]
        counts[a, b] += 1
        adjacent += int(b) in _neighbours(Lx, Ly, int(a))
    assert np.all(np.diag(counts) == 0)
    obs = counts[~np.eye(N, dtype=bool)]
    exp = nmaps / (N * (N - 1))
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    dof = N * (N - 1) - 1
    assert abs(chi2 - dof) < 5 * np.sqrt(2 * dof), chi2
    # a partner among a's 4 neighbours: probability 4/15
    p = 4 / 15
    assert abs(adjacent / nmaps - p) < 5 * np.sqrt(p * (1 - p) / nmaps)


def _map_chain(Lx, Ly, Q, T, Delta, V, J, nmaps, seed, burn=2000):
    N = Lx * Ly
    n_plus = max(Q, 0) + (N - abs(Q)) // 4
    st = oracle.init_counts(Lx, Ly, seed, n_plus, n_plus - Q)
    rec = oracle.map_sweeps(st, seed, 0, nmaps, 1.0 / T, Delta, V, J, obs_every=1)
    assert np.all(rec[:, 6] == Q)
    return rec[burn:]


@pytest.mark.parametrize("Q,params", [(2, (0.25, -0.5, 1.0, 1.0)), (2, (1.0, 0.5, 1.0, 1.0)),
                                      (0, (0.6, 0.0, 1.0, 1.0))])
def test_map_chain_matches_exact_enumeration_4x4(Q, params):
    T, Delta, V, J = params
    # one pair per map; 8 maps make one sweep's worth of pair moves
    rec = _map_chain(4, 4, Q, T, Delta, V, J, 1600000, seed=29)[::8]
    ex = exact_averages(4, 4, Q, T, Delta, V, J)
    E = energy(rec, Delta, V, J)
    for key, (m, s) in (("E", batch_mean(E / 16)), ("C", batch_heat(E, 16, T)),
                        ("Nc", batch_mean(rec[:, 1]))):
        assert abs(m - ex[key]) <= 4 * max(s, 1e-12), (key, m, ex[key], s)


def test_map_chain_agrees_with_colour_schedule_8x8():
    L, Q, T, Delta, V, J = 8, 4, 0.8, 0.3, 1.0, 1.0
    N = L * L
    n_plus = max(Q, 0) + (N - Q) // 4
    st = oracle.init_counts(L, L, 41, n_plus, n_plus - Q)
    a = oracle.sweeps(st, 41, 0, 120000, 1.0 / T, Delta, V, J, obs_every=1)[2000:]
    # 6 pairs a map: 16 maps are 96 pair moves, three sweeps' worth
    b = _map_chain(L, L, Q, T, Delta, V, J, 640000, seed=43, burn=16000)[::16]
    for col in (1, 2, 3):
        ma, sa = batch_mean(a[:, col])
        mb, sb = batch_mean(b[:, col])
        assert abs(ma - mb) <= 4 * np.hypot(sa, sb), (col, ma, mb)
