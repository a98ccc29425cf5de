"""Detailed balance of the oracle's coupled-pair move on the 4x4 torus.

Sec. 3.1 makes each move a Metropolis step between the configurations of one
pair that keep its charge q = S_a + S_b: the proposal is uniform over the
q-set (the current configuration included) and the acceptance is
min(1, exp(-beta dE)) with dE from Eq. (3).  For a fixed pair (a, b) that move
is reversible with respect to the Boltzmann weight pi(x) = exp(-beta E(x))
restricted to sum S = Q, and a colour phase -- a product of such moves on
disjoint neighbourhoods -- therefore leaves that distribution stationary.

This pins the oracle to that property on every constrained state of the 4x4
torus at Q = +-13 (4960 states each), for four pairs (two bonded, a diagonal
and a distant one): with the move's 16-bit choice field v taken through all
twelve classes v mod 12 (each equally likely, as 65532 = 12 x 5461),
  * the proposal is uniform over the pair's q-set (the current configuration
    included) and frozen for |q| = 2,
  * every proposal x -> y is matched by y -> x with the same multiplicity, and
  * pi(x) A(x -> y) and pi(y) A(y -> x) agree to within 2^-32 max(pi(x), pi(y)),
    the rounding of the acceptance table (thresholds floored to 2^-32).
Proposals are read from the oracle's own move (every move accepted through a
table of 0xFFFFFFFF), acceptances from its threshold table at the index of its
pair_delta, and E from its full recount -- so a wrong q-set entry, a sign or
operand slip in dE, or a misplaced table index breaks one of the two checks.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

L = 4
BETA, DELTA, V, J = 1 / 1.3, 0.3, 1.0, 0.8
# (a, b) as site indices y * L + x: right and down bonds, a diagonal, (2, 1) away
PAIRS = [(0, 1), (0, 4), (0, 5), (5, 11)]


def _states(Q: int):
    """Every 4x4 configuration with sum S = Q (codes 0, 1: magnetic; 2: +1; 3: -1)."""
    N = L * L
    out = []
    for n_minus in range(N + 1):
        n_plus = Q + n_minus
        n0 = N - n_plus - n_minus
        if n_plus < 0 or n0 < 0:
            continue
        for plus in itertools.combinations(range(N), n_plus):
            rest = [i for i in range(N) if i not in plus]
            for minus in itertools.combinations(rest, n_minus):
                mag = [i for i in rest if i not in minus]
                for signs in range(1 << n0):
                    st = np.zeros(N, dtype=np.uint8)
                    st[list(plus)] = 2
                    st[list(minus)] = 3
                    for k, i in enumerate(mag):
                        st[i] = (signs >> k) & 1
                    out.append(st.reshape(L, L))
    return out


def _energy(st) -> float:
    c = oracle.recount(st)
    return DELTA * c[0] + V * c[1] + 0.25 * J * c[2]


@pytest.mark.parametrize("Q", [13, -13])
def test_pair_move_is_reversible_on_every_constrained_4x4_state(Q):
    states = _states(Q)
    # sum over n- of C(N, n+) C(N - n+, n-) 2^n0 with n+ = Q + n-
    N = L * L
    count = sum(math.comb(N, Q + m) * math.comb(N - Q - m, m) * 2 ** (N - Q - 2 * m)
                for m in range(N + 1) if 0 <= Q + m and Q + 2 * m <= N)
    assert len(states) == count == 4960
    table = oracle.threshold_table(BETA, DELTA, V, J)
    accept_all = np.full_like(table, 0xFFFFFFFF)
    key = oracle.seed_key(1)
    ctr = np.zeros(4, dtype=np.uint32)
    E = {s.tobytes(): _energy(s) for s in states}
    E0 = min(E.values())
    pi = {k: np.exp(-BETA * (e - E0)) for k, e in E.items()}
    lib = oracle.lib()
    for a, b in PAIRS:
        mult = {}  # (x, y) -> number of choice classes proposing y from x
        acc = {}   # (x, y) -> acceptance probability of the move
        for x in states:
            kx = x.tobytes()
            q = int(x.flat[a] >= 2) * (5 - 2 * int(x.flat[a])) + \
                int(x.flat[b] >= 2) * (5 - 2 * int(x.flat[b]))  # S_a + S_b
            per_y = {}
            for v in range(12):
                y = x.copy()
                moved = oracle.pair_move(y, a, b, v, key, ctr, accept_all)
                per_y[y.tobytes()] = per_y.get(y.tobytes(), 0) + 1
                if not moved:
                    continue  # frozen pair or the current configuration drawn
                ky = y.tobytes()
                assert ky in E, "a move left the constrained set"
                mult[kx, ky] = mult.get((kx, ky), 0) + 1
                d = oracle.pair_delta(x, a, b, int(y.flat[a]), int(y.flat[b]))
                thr = int(table.reshape(-1)[lib.oracle_table_index(*d)])
                acc[kx, ky] = 1.0 if thr == 0xFFFFFFFF else thr / 2.0 ** 32
            # the proposal is uniform over the pair's q-set, the current
            # configuration included: 4 (|q| = 1) or 6 (q = 0) outcomes, each
            # from 12 / |set| of the choice classes; |q| = 2 cannot move
            nset = {2: 1, 1: 4, 0: 6}[abs(q)]
            assert sorted(per_y.values()) == [12 // nset] * nset, (a, b, q, per_y.values())
        assert mult, (a, b)
        for (kx, ky), m in mult.items():
            assert mult.get((ky, kx)) == m, ("proposals not symmetric", a, b)
            lhs, rhs = pi[kx] * acc[kx, ky], pi[ky] * acc[ky, kx]
            tol = 2.0 ** -32 * max(pi[kx], pi[ky]) + 1e-15 * max(lhs, rhs)
            assert abs(lhs - rhs) <= tol, (a, b, lhs, rhs)
