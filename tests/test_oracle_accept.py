"""Acceptance frequency of the oracle's pair move against its threshold.

The Metropolis test of Sec. 3.1 accepts an uphill move with probability
exp(-beta dE); the oracle takes it as u < thr with u a uniform 32-bit word and
thr = floor(2^32 exp(-beta dE)) (thresholds pinned against 50-digit exp
elsewhere).  u is split: its top half is the pair's random word R >> 16, its
low half the low 16 bits of the pair's SLOW Philox word.  Two binomial tests
pin that split: over uniform top halves the acceptance rate is thr / 2^32, and
with the top half equal to thr's (a tie) it is (thr mod 2^16) / 2^16, which
only the low half decides.
"""
import numpy as np

import oracle

A, B = 0, 5  # (0, 0) and (1, 1) of a 4x4 torus: diagonal, no shared bond
BETA, DELTA, V, J = 0.7, 0.0, 1.0, 1.0


def _setup():
    st = np.zeros((4, 4), dtype=np.uint8)  # sigma = +1 everywhere
    st.flat[A] = 2  # S = +1
    for i in (1, 4, 6):  # three neighbours of B, two of them shared with A
        st.flat[i] = 2
    st.flat[9] = 1  # the fourth: sigma = -1
    table = oracle.threshold_table(BETA, DELTA, V, J)
    key = oracle.seed_key(11)
    # choice class 2 of the q = +1 set moves the charge from A to B
    y = st.copy()
    assert oracle.pair_move(y, A, B, 2, key, np.zeros(4, np.uint32), np.full_like(table, ~np.uint32(0)))
    assert y.flat[A] == 0 and y.flat[B] == 2
    d = oracle.pair_delta(st, A, B, 0, 2)
    # dBV = -2 + 3, dBJ = 2 + 1 (unequal, so that swapped roles would show):
    # dE = V + (J / 4) 3 = 1.75
    assert d == (0, 1, 3)
    thr = int(table.reshape(-1)[oracle.lib().oracle_table_index(*d)])
    return st, table, key, thr


def _rate(st, table, key, top_halves):
    k = 0
    for i, uh in enumerate(top_halves):
        x = st.copy()
        k += oracle.pair_move(x, A, B, 2 | (int(uh) << 16), key,
                              np.array([i, 0x5A5A, 3, 0x51], np.uint32), table)
    return k


def _binomial_ok(k, n, p):
    return abs(k - n * p) <= 5.0 * np.sqrt(n * p * (1.0 - p))


def test_acceptance_rate_is_threshold_over_two_to_the_32():
    st, table, key, thr = _setup()
    p = thr / 2.0 ** 32
    assert abs(p - np.exp(-BETA * 1.75)) < 2.0 ** -31
    n = 60000
    top = np.random.default_rng(5).integers(0, 1 << 16, size=n)
    k = _rate(st, table, key, top)
    assert _binomial_ok(k, n, p), (k, n * p)


def test_ties_of_the_top_half_are_decided_by_the_low_half():
    st, table, key, thr = _setup()
    p = (thr & 0xFFFF) / 65536.0
    assert 0.05 < p < 0.95  # an informative tie for these parameters
    n = 20000
    k = _rate(st, table, key, np.full(n, thr >> 16))
    assert _binomial_ok(k, n, p), (k, n * p)
