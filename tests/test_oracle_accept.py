"""Acceptance frequency of the oracle's pair move against its threshold.

The Metropolis test of Sec. 3.1 accepts an uphill move with probability
exp(-beta dE); the oracle takes it as a uniform draw below thr / 2^32 with
thr = floor(2^32 exp(-beta dE)) (thresholds pinned against 50-digit exp
elsewhere).  The pair's 16-bit field v carries both the choice and the top
part of the acceptance draw: below 65532 = 12 x 5461 the choice is v mod 12
(mod the q-set's size) and w = floor(v / 12), uniform on [0, 5461), is the
draw's top part, the pair's SLOW word 0 its low part: accept iff
w 2^32 + s0 < 5461 thr.  From 65532 up the choice comes from SLOW word 1 and
the draw is SLOW word 0 alone.  Binomial tests pin each region:

* over uniform w the rate is thr / 2^32;
* w below T = floor(5461 thr / 2^32) always accepts, above it never does;
* at w = T (a tie) the rate is the fraction (5461 thr mod 2^32) / 2^32 that
  only the SLOW word decides;
* for v >= 65532 the rate is again thr / 2^32, drawn from SLOW word 0.
"""
import numpy as np

import oracle

A, B = 0, 5  # (0, 0) and (1, 1) of a 4x4 torus: diagonal, no shared bond
BETA, DELTA, V, J = 0.7, 0.0, 1.0, 1.0
CHOICE = 2  # choice class 2 of the q = +1 set moves the charge from A to B


def _setup():
    st = np.zeros((4, 4), dtype=np.uint8)  # sigma = +1 everywhere
    st.flat[A] = 2  # S = +1
    for i in (1, 4, 6):  # three neighbours of B, two of them shared with A
        st.flat[i] = 2
    st.flat[9] = 1  # the fourth: sigma = -1
    table = oracle.threshold_table(BETA, DELTA, V, J)
    key = oracle.seed_key(11)
    y = st.copy()
    assert oracle.pair_move(y, A, B, CHOICE, key, np.zeros(4, np.uint32),
                            np.full_like(table, ~np.uint32(0)))
    assert y.flat[A] == 0 and y.flat[B] == 2
    d = oracle.pair_delta(st, A, B, 0, 2)
    # dBV = -2 + 3, dBJ = 2 + 1 (unequal, so that swapped roles would show):
    # dE = V + (J / 4) 3 = 1.75
    assert d == (0, 1, 3)
    thr = int(table.reshape(-1)[oracle.lib().oracle_table_index(*d)])
    return st, table, key, thr


def _slow_ctr(i):
    return np.array([i, 0x5A5A, 3, oracle.TAG_SLOW], np.uint32)


def _rate(st, table, key, fields):
    k = 0
    for i, v in enumerate(fields):
        x = st.copy()
        k += oracle.pair_move(x, A, B, int(v), key, _slow_ctr(i), table)
    return k


def _binomial_ok(k, n, p):
    return abs(k - n * p) <= 5.0 * np.sqrt(n * p * (1.0 - p))


def test_acceptance_rate_is_threshold_over_two_to_the_32():
    st, table, key, thr = _setup()
    p = thr / 2.0 ** 32
    assert abs(p - np.exp(-BETA * 1.75)) < 2.0 ** -31
    n = 60000
    w = np.random.default_rng(5).integers(0, 5461, size=n)
    k = _rate(st, table, key, 12 * w + CHOICE)
    assert _binomial_ok(k, n, p), (k, n * p)


def test_draws_below_and_above_the_tie_are_decided_by_the_field_alone():
    st, table, key, thr = _setup()
    T = (5461 * thr) >> 32
    assert 10 < T < 5450
    below = [T - 1, T - 2, T // 2, 0]
    above = [T + 1, T + 2, (T + 5461) // 2, 5460]
    for w in below:
        assert _rate(st, table, key, [12 * w + CHOICE] * 200) == 200, w
    for w in above:
        assert _rate(st, table, key, [12 * w + CHOICE] * 200) == 0, w


def test_ties_are_decided_by_the_slow_word():
    st, table, key, thr = _setup()
    T = (5461 * thr) >> 32
    p = ((5461 * thr) - (T << 32)) / 2.0 ** 32
    assert 0.05 < p < 0.95  # an informative tie for these parameters
    n = 20000
    k = _rate(st, table, key, [12 * T + CHOICE] * n)
    assert _binomial_ok(k, n, p), (k, n * p)


def test_fields_from_65532_up_draw_choice_and_acceptance_from_the_slow_words():
    st, table, key, thr = _setup()
    p = thr / 2.0 ** 32
    n, k = 0, 0
    for i in range(40000):
        s = oracle.philox(_slow_ctr(i), key)
        x = st.copy()
        moved = oracle.pair_move(x, A, B, 65532 + i % 4, key, _slow_ctr(i), table)
        if int(s[1]) < 4294967292 and int(s[1]) % 4 == CHOICE:
            n += 1
            k += moved
        else:
            # another choice class: the charge stays, or goes with the other sign
            assert not (x.flat[A] == 0 and x.flat[B] == 2)
    assert 9000 < n < 11000  # choice class CHOICE drawn from word 1 a quarter of the time
    assert _binomial_ok(k, n, p), (k, n * p)
