"""Statistical and exact pins of the oracle's Markov chain.

The chain must sample the constrained canonical ensemble of Eq. (3) under
Eq. (2).  Checked against:

* exact enumeration (the paper's own test, Sec. 3.3): 3 x 3 and 4 x 2 in the
  sequential random-pair mode, 4 x 4 under the colour schedule;
* infinite temperature: closed-form uniform averages;
* Delta -> +inf: charge creation is never accepted, so Nc falls to |Q| and
  stays; Delta -> -inf: every site ends up charged, Nc = N, BJ = 0;
* the Ising limit: transfer matrix on 4 x 4 and 8 x 8;
* colour schedule vs sequential random pairs on 8 x 8;
* a negative control: nearest-neighbour partners only (the paper's abandoned
  first version, Sec. 3.2) miss the low-temperature heat-capacity peak of
  4 x 4 that the colour schedule reproduces;
* the penalty-function baseline (Sec. 2.2): a chemical-potential term holds
  the charge only on average, and its heat capacity diverges as T -> 0.

Means are compared within 4 standard errors from batch means.
"""
import numpy as np
import pytest

import oracle
from oracle.closed_forms import beta0_averages, count_states
from oracle.ising_tm import ising_energy_and_heat, onsager_tc

from .mcstats import batch_heat, batch_mean, energy

_ENUM = {}


def exact_dos(Lx, Ly, Q):
    if (Lx, Ly, Q) not in _ENUM:
        _ENUM[(Lx, Ly, Q)] = oracle.enumerate_dos(Lx, Ly, Q)
    return _ENUM[(Lx, Ly, Q)]


def exact_averages(Lx, Ly, Q, T, Delta, V, J):
    n, count, m2, mabs, ms2 = exact_dos(Lx, Ly, Q)
    N = Lx * Ly
    nc = np.arange(N + 1)[:, None, None]
    bv = (np.arange(4 * N + 1) - 2 * N)[None, :, None]
    bj = (np.arange(4 * N + 1) - 2 * N)[None, None, :]
    E = Delta * nc + V * bv + 0.25 * J * bj
    mask = count > 0
    Emin = E[mask].min()
    w = np.where(mask, np.exp(-(E - Emin) / T), 0.0)
    Z = np.sum(w * count)
    e1 = np.sum(w * count * E) / Z
    e2 = np.sum(w * count * E * E) / Z
    return {
        "E": e1 / N,
        "C": (e2 - e1 * e1) / (N * T * T),
        "Nc": np.sum(w * count * nc) / Z,
        "M2": np.sum(w * m2) / Z,
        "Ms2": np.sum(w * ms2) / Z,
    }


def run_chain(Lx, Ly, Q, T, Delta, V, J, nsweeps, seed, sequential=False, burn=2000,
              n_plus=None):
    N = Lx * Ly
    if n_plus is None:
        n_plus = max(Q, 0) + (N - abs(Q)) // 4
    st = oracle.init_counts(Lx, Ly, seed, n_plus, n_plus - Q)
    rec = oracle.sweeps(st, seed, 0, nsweeps, 1.0 / T, Delta, V, J, obs_every=1,
                        sequential=sequential)
    assert np.all(rec[:, 6] == Q)  # the charge constraint holds after every sweep
    return rec[burn:]


def compare(rec, ex, N, T, Delta, V, J, tol=4.0):
    E = energy(rec, Delta, V, J)
    checks = {
        "E": batch_mean(E / N),
        "C": batch_heat(E, N, T),
        "Nc": batch_mean(rec[:, 1]),
        "M2": batch_mean(rec[:, 4].astype(np.float64) ** 2),
        "Ms2": batch_mean(rec[:, 5].astype(np.float64) ** 2),
    }
    for k, (m, s) in checks.items():
        s = max(s, 1e-12)
        assert abs(m - ex[k]) <= tol * s, (k, m, ex[k], s)


@pytest.mark.parametrize("Lx,Ly,Q", [(3, 3, 0), (3, 3, 1), (3, 3, -2), (4, 2, 0), (4, 2, 3),
                                     (4, 4, 2)])
def test_enumeration_counts_every_constrained_state(Lx, Ly, Q):
    n = exact_dos(Lx, Ly, Q)[0]
    assert n == count_states(Lx * Ly, Q)


@pytest.mark.parametrize("shape,Q,params", [
    ((3, 3), 1, (0.5, 0.5, 1.0, 1.0)),
    ((3, 3), 0, (2.0, -0.5, 1.0, 1.0)),
    ((4, 2), 0, (0.7, 0.2, 1.0, 1.0)),
    ((4, 2), 2, (1.5, 0.5, 0.3, 2.0)),
])
def test_sequential_chain_matches_exact_enumeration(shape, Q, params):
    Lx, Ly = shape
    T, Delta, V, J = params
    rec = run_chain(Lx, Ly, Q, T, Delta, V, J, 300000, seed=17, sequential=True)
    compare(rec, exact_averages(Lx, Ly, Q, T, Delta, V, J), Lx * Ly, T, Delta, V, J)


@pytest.mark.parametrize("Q,params", [
    (2, (1.0, 0.5, 1.0, 1.0)),
    (2, (0.4, 0.0, 0.5, 1.0)),
    (4, (0.3, 0.2, 0.1, 2.0)),
    (0, (3.0, -0.5, 1.0, 1.0)),
])
def test_colour_chain_matches_exact_enumeration_4x4(Q, params):
    T, Delta, V, J = params
    rec = run_chain(4, 4, Q, T, Delta, V, J, 400000, seed=23)
    compare(rec, exact_averages(4, 4, Q, T, Delta, V, J), 16, T, Delta, V, J)


@pytest.mark.parametrize("Lx,Ly,Q,seq", [(8, 8, 6, False), (4, 4, -2, False), (3, 3, 1, True)])
def test_infinite_temperature_closed_forms(Lx, Ly, Q, seq):
    N = Lx * Ly
    st = oracle.init_constrained(Lx, Ly, 31, Q / N, 0.3)
    rec = oracle.sweeps(st, 31, 0, 60000, 0.0, 1.0, 1.0, 1.0, obs_every=1, sequential=seq)[200:]
    ex = beta0_averages(N, Q)
    for k, col in (("Nc", 1), ("BV", 2), ("BJ", 3)):
        m, s = batch_mean(rec[:, col])
        assert abs(m - float(ex[k])) <= 4 * s, (k, m, float(ex[k]), s)
    m, s = batch_mean(rec[:, 4].astype(np.float64) ** 2)
    assert abs(m - float(ex["M2"])) <= 4 * s


def test_large_positive_delta_freezes_charge_count_at_minimum():
    Lx = Ly = 16
    Q = 8
    st = oracle.init_counts(Lx, Ly, 3, 20, 12)
    rec = oracle.sweeps(st, 3, 0, 400, 1.0, 1e9, 1.0, 1.0, obs_every=1)
    nc = rec[:, 1]
    assert np.all(np.diff(nc) <= 0) and nc[0] <= 32
    assert np.all(nc >= abs(Q)) and nc[-1] == abs(Q)
    assert np.all(rec[:, 6] == Q)


def test_large_negative_delta_charges_every_site():
    # the last magnetic sites must meet in one pair to turn into a +1/-1 pair,
    # which takes many sweeps once only a few are left
    Lx = Ly = 8
    Q = 8
    st = oracle.init_counts(Lx, Ly, 4, 14, 6)
    rec = oracle.sweeps(st, 4, 0, 20000, 1.0, -1e9, 1.0, 1.0, obs_every=1)
    nc = rec[:, 1]
    assert np.all(np.diff(nc) >= 0)
    assert nc[-1] == Lx * Ly and rec[-1, 3] == 0 and rec[-1, 6] == Q


@pytest.mark.parametrize("L,T", [(4, 0.4), (4, 1.0), (8, 0.5), (8, 0.567), (8, 1.2)])
def test_ising_limit_matches_transfer_matrix(L, T):
    J = 1.0
    st = oracle.init_counts(L, L, 5, 0, 0)  # all magnetic, Q = 0
    rec = oracle.sweeps(st, 5, 0, 200000, 1.0 / T, 1e9, 1.0, J, obs_every=1)[2000:]
    assert np.all(rec[:, 1] == 0)
    E = energy(rec, 1e9, 1.0, J)
    e_ex, c_ex = ising_energy_and_heat(L, T, J)
    m, s = batch_mean(E / (L * L))
    assert abs(m - e_ex) <= 4 * s, (m, e_ex, s)
    c, sc = batch_heat(E, L * L, T)
    assert abs(c - c_ex) <= 4 * sc, (c, c_ex, sc)


def test_onsager_temperature_in_units_of_J():
    assert abs(onsager_tc(1.0) - 0.5673) < 1e-3


def test_colour_schedule_agrees_with_sequential_random_pairs():
    L, Q, T, Delta, V, J = 8, 4, 0.8, 0.3, 1.0, 1.0
    a = run_chain(L, L, Q, T, Delta, V, J, 150000, seed=41)
    b = run_chain(L, L, Q, T, Delta, V, J, 150000, seed=43, sequential=True)
    for col in (1, 2, 3):
        ma, sa = batch_mean(a[:, col])
        mb, sb = batch_mean(b[:, col])
        assert abs(ma - mb) <= 4 * np.hypot(sa, sb), (col, ma, mb)


@pytest.mark.parametrize("L", [3, 4])
def test_transfer_matrix_matches_brute_force(L):
    N = L * L
    T, J = 0.7, 1.0
    bits = np.arange(1 << N)
    s = (1 - 2 * ((bits[:, None] >> np.arange(N)[None, :]) & 1)).reshape(-1, L, L)
    E = 0.25 * J * (np.sum(s * np.roll(s, -1, 2), axis=(1, 2))
                    + np.sum(s * np.roll(s, -1, 1), axis=(1, 2)))
    w = np.exp(-(E - E.min()) / T)
    e1 = np.sum(w * E) / np.sum(w)
    e2 = np.sum(w * E * E) / np.sum(w)
    e_tm, c_tm = ising_energy_and_heat(L, T, J)
    assert abs(e_tm - e1 / N) < 1e-10
    assert abs(c_tm - (e2 - e1 * e1) / (N * T * T)) < 1e-9


def test_short_range_pairs_miss_the_low_temperature_peak():
    """Negative control (Sec. 3.2): the paper's first version took the partner
    among a's nearest neighbours and, on 4 x 4, lost the heat capacity's
    low-temperature peak.  With Q = 2, Delta = -0.5, V = J = 1 the exact C(T)
    of 4 x 4 has a low-temperature peak at T = 0.25 besides the main one; the
    colour-schedule chain reproduces it, the short-range chain freezes in a
    metastable state (some states are out of its reach at that temperature)
    and misses it."""
    Q, Delta, V, J = 2, -0.5, 1.0, 1.0
    # the exact curve: a local maximum at T = 0.25, well below the main peak
    C = {T: exact_averages(4, 4, Q, T, Delta, V, J)["C"] for T in (0.15, 0.25, 0.4, 1.6)}
    assert C[0.25] > 1.5 * C[0.15] and C[0.25] > 1.5 * C[0.4]
    assert C[1.6] > 5 * C[0.25]
    T = 0.25
    ex = exact_averages(4, 4, Q, T, Delta, V, J)
    n_plus = max(Q, 0) + 14 // 4
    st = oracle.init_counts(4, 4, 5, n_plus, n_plus - Q)
    rec = oracle.sweeps(st, 5, 0, 200000, 1.0 / T, Delta, V, J, obs_every=1)[2000:]
    E = energy(rec, Delta, V, J)
    c_all, s_all = batch_heat(E, 16, T)
    e_all, se_all = batch_mean(E / 16)
    assert abs(c_all - ex["C"]) <= 4 * s_all
    assert abs(e_all - ex["E"]) <= 4 * max(se_all, 1e-12)
    st = oracle.init_counts(4, 4, 5, n_plus, n_plus - Q)
    rec = oracle.sweeps(st, 5, 0, 200000, 1.0 / T, Delta, V, J, obs_every=1,
                        neighbour=True)[2000:]
    assert np.all(rec[:, 6] == Q)
    E = energy(rec, Delta, V, J)
    c_nn, _ = batch_heat(E, 16, T)
    e_nn, _ = batch_mean(E / 16)
    assert c_nn < 0.25 * ex["C"]                       # the peak is missing
    assert e_nn - ex["E"] > 0.02 and e_nn - ex["E"] > 20 * se_all  # stuck above


def test_short_range_pairs_agree_at_high_temperature():
    """The short-range chain is a valid Metropolis chain (symmetric proposals,
    charge conserved): away from the low-temperature region it reproduces the
    exact averages, so the failure above is specific to low temperature."""
    Q, Delta, V, J, T = 2, -0.5, 1.0, 1.0, 1.6
    n_plus = max(Q, 0) + 14 // 4
    st = oracle.init_counts(4, 4, 9, n_plus, n_plus - Q)
    rec = oracle.sweeps(st, 9, 0, 200000, 1.0 / T, Delta, V, J, obs_every=1,
                        neighbour=True)[2000:]
    compare(rec, exact_averages(4, 4, Q, T, Delta, V, J), 16, T, Delta, V, J)


def test_penalty_function_heat_capacity_diverges_as_t_goes_to_zero():
    """Baseline of Sec. 2.2: holding the charge with a chemical-potential term
    -mu sum S (mu adjusted after every sweep) instead of coupled pairs.  The
    charge sum averages nN but keeps fluctuating, so the energy variance stays
    finite as T -> 0 and C = var(E) / (N T^2) grows like 1/T^2 -- the failure
    that led the paper to coupled pairs -- while the coupled-pair chain holds
    sum S = nN exactly and follows the exact C(T) to zero."""
    Q, Delta, V, J = 2, -0.5, 1.0, 1.0
    C = {}
    for T in (0.1, 0.25):
        st = oracle.init_counts(4, 4, 5, 5, 3)
        rec, mu = oracle.penalty_sweeps(st, 5, 0, 60000, 1.0 / T, Delta, V, J, Q / 16, 0.0, 0.5)
        rec = rec[5000:]
        S = rec[:, 6]
        assert abs(S.mean() - Q) < 0.1 and S.std() > 1.0  # held on average only
        C[T], _ = batch_heat(energy(rec, Delta, V, J), 16, T)
        assert C[T] * T * T > 1.0  # the energy variance per site does not vanish
        ex = exact_averages(4, 4, Q, T, Delta, V, J)["C"]
        assert C[T] > 100 * ex
    assert C[0.1] > 4 * C[0.25]
    # the coupled-pair chain at the same point: charge fixed, C tiny and exact
    st = oracle.init_counts(4, 4, 5, 5, 3)
    rec = oracle.sweeps(st, 5, 0, 60000, 10.0, Delta, V, J, obs_every=1)[2000:]
    assert np.all(rec[:, 6] == Q)
    c, _ = batch_heat(energy(rec, Delta, V, J), 16, 0.1)
    assert exact_averages(4, 4, Q, 0.1, Delta, V, J)["C"] < 0.01 and c < 0.01
