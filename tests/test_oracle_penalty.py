"""Exact pins of the penalty-function baseline (Sec. 2.2).

The baseline holds the charge with a chemical-potential term -mu sum S instead
of coupled pairs: single-site Metropolis moves under E - mu sum S (E of
Eq. 3).  Two things about it have exact references:

* its single-site energy change: for every site and every new state it must
  equal the difference of two full recounts of Eq. 3 (every torus from 2 x 2
  up, where a 2-wide torus has two bonds between the same sites);
* with mu held fixed (kappa = 0) the chain samples the grand-canonical
  ensemble exp(-beta (E - mu sum S)); on 3 x 3 and 4 x 2 its averages of E,
  the heat capacity, sum S and Nc must agree with exact enumeration summed
  over every charge sector Q with weight exp(beta mu Q), within 4 standard
  errors.

A J-for-J/4 slip, a dropped V term, a wrong sign of the mu term or a
neighbour counted once on a 2-wide torus each fails one of them.
"""
import numpy as np
import pytest

import oracle

from .mcstats import batch_heat, batch_mean, energy

SHAPES = [(2, 2), (2, 3), (3, 2), (3, 3), (4, 2), (2, 4), (4, 4), (5, 3), (8, 4), (4, 8)]


@pytest.mark.parametrize("Lx,Ly", SHAPES)
def test_site_delta_equals_recount_difference(Lx, Ly):
    rng = np.random.default_rng(100 * Lx + Ly)
    for _ in range(3):
        st = rng.integers(0, 4, size=(Ly, Lx), dtype=np.uint8)
        base = oracle.recount(st)
        for a in range(Lx * Ly):
            y, x = divmod(a, Lx)
            old = int(st[y, x])
            for nc in range(4):
                d = oracle.site_delta(st, a, nc)
                st[y, x] = nc
                after = oracle.recount(st)
                st[y, x] = old
                assert d == tuple(int(v) for v in (after - base)[:3]), (Lx, Ly, a, old, nc)


_DOS = {}


def grand_canonical(Lx, Ly, T, Delta, V, J, mu):
    """Exact averages of exp(-(E - mu Q) / T) over every state of the torus:
    the constrained histograms of all charge sectors Q = -N .. N, each weighted
    by exp(mu Q / T)."""
    N = Lx * Ly
    nc = np.arange(N + 1)[:, None, None]
    bv = (np.arange(4 * N + 1) - 2 * N)[None, :, None]
    bj = (np.arange(4 * N + 1) - 2 * N)[None, None, :]
    E = Delta * nc + V * bv + 0.25 * J * bj
    terms = []
    total = 0
    for Q in range(-N, N + 1):
        if (Lx, Ly, Q) not in _DOS:
            _DOS[(Lx, Ly, Q)] = oracle.enumerate_dos(Lx, Ly, Q)
        n, count = _DOS[(Lx, Ly, Q)][:2]
        total += n
        mask = count > 0
        if mask.any():
            terms.append((Q, count, mask))
    assert total == 4 ** N  # every state of the torus in exactly one sector
    # exponents relative to their minimum, for range
    emin = min(float((E - mu * Q)[m].min()) for Q, _, m in terms)
    Z = e1 = e2 = q1 = n1 = 0.0
    for Q, count, mask in terms:
        w = np.where(mask, np.exp(-((E - mu * Q) - emin) / T), 0.0) * count
        Z += w.sum()
        e1 += (w * E).sum()
        e2 += (w * E * E).sum()
        q1 += w.sum() * Q
        n1 += (w * nc).sum()
    e1, e2, q1, n1 = e1 / Z, e2 / Z, q1 / Z, n1 / Z
    return {"E": e1 / N, "C": (e2 - e1 * e1) / (N * T * T), "S": q1, "Nc": n1}


CASES = [
    # (Lx, Ly, T, Delta, V, J, mu, seed)
    (3, 3, 1.0, 0.3, 1.0, 1.0, 0.4, 11),
    (3, 3, 0.8, -0.5, 0.5, 2.0, -0.6, 12),
    (4, 2, 1.2, 0.5, -0.7, 1.5, 0.9, 13),
    (4, 2, 0.7, 0.0, 1.0, -1.0, -0.3, 14),
]


@pytest.mark.parametrize("Lx,Ly,T,Delta,V,J,mu,seed", CASES)
def test_fixed_mu_chain_matches_exact_grand_canonical_averages(Lx, Ly, T, Delta, V, J, mu, seed):
    N = Lx * Ly
    ex = grand_canonical(Lx, Ly, T, Delta, V, J, mu)
    st = oracle.init_counts(Lx, Ly, seed, 1, 1)
    rec, trace = oracle.penalty_sweeps(st, seed, 0, 120000, 1.0 / T, Delta, V, J, 0.0, mu, 0.0)
    assert np.all(trace == mu)  # kappa = 0 holds mu fixed
    rec = rec[2000:]
    E = energy(rec, Delta, V, J)
    got = {
        "E": batch_mean(E / N),
        "C": batch_heat(E, N, T),
        "S": batch_mean(rec[:, 6].astype(np.float64)),
        "Nc": batch_mean(rec[:, 1].astype(np.float64)),
    }
    for k, (m, s) in got.items():
        assert abs(m - ex[k]) <= 4.0 * max(s, 1e-12), (k, m, s, ex[k])
    # the charge is not held: it fluctuates across sectors
    assert rec[:, 6].std() > 0.2
