"""Pins of the oracle's model arithmetic: pair sets, energy terms, dE,
acceptance thresholds, charge counts and the initial state.

Each check compares the oracle with something other than itself: the paper's
printed configuration lists (tests/golden/pair_sets.txt), energies of lattices
whose value follows by hand from Eq. (3), a full recount before and after every
possible move, the paper's own dE formulas where they hold, and exp evaluated
to 50 digits.
"""
import os
import re

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CODE = {"+1/2": 0, "-1/2": 1, "+1": 2, "-1": 3}
S = np.array([0, 0, 1, -1])
SIG = np.array([1, -1, 0, 0])


def golden_pair_sets():
    sets = {}
    with open(os.path.join(HERE, "golden", "pair_sets.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            q, rest = line.split(":")
            pairs = re.findall(r"\(([^,]+),([^)]+)\)", rest)
            sets[int(q[2:])] = [(CODE[a.strip()], CODE[b.strip()]) for a, b in pairs]
    return sets


def all_pass_table():
    return oracle.threshold_table(0.0, 0.0, 0.0, 0.0)


def test_pair_sets_match_paper_order():
    sets = golden_pair_sets()
    assert [len(sets[q]) for q in (2, 1, 0, -1, -2)] == [1, 4, 6, 4, 1]
    table = all_pass_table()
    key = oracle.seed_key(9)
    a, b = 0, 10  # distant sites of a 4x4 lattice
    for q in (1, -1, 0):
        for idx, expect in enumerate(sets[q]):
            st = np.zeros((4, 4), dtype=np.uint8)
            ca, cb = sets[q][(idx + 1) % len(sets[q])]
            st.flat[a], st.flat[b] = ca, cb
            oracle.pair_move(st, a, b, idx, key, [0, 0, 0, oracle.TAG_SLOW], table)
            assert (st.flat[a], st.flat[b]) == expect, (q, idx)
    for q in (2, -2):
        st = np.zeros((4, 4), dtype=np.uint8)
        st.flat[a], st.flat[b] = sets[q][0]
        for R in (0, 1, 5, 0xFFFFFFFF):
            assert oracle.pair_move(st, a, b, R, key, [0, 0, 0, 3], table) == 0
            assert (st.flat[a], st.flat[b]) == sets[q][0]


def test_q0_choice_fallback_uses_slow_word():
    # a choice field >= 65532 falls back to SLOW word 1 (mod 6 when below 6 * 715827882)
    sets = golden_pair_sets()
    table = all_pass_table()
    key = oracle.seed_key(77)
    for k in range(40):
        ctr = [k, 5, 0, oracle.TAG_SLOW]
        w1 = int(oracle.philox(ctr, key)[1])
        st = np.zeros((4, 4), dtype=np.uint8)
        st.flat[0], st.flat[10] = 0, 0
        oracle.pair_move(st, 0, 10, 0xFFFF, key, ctr, table)
        expect = sets[0][w1 % 6] if w1 < 6 * 715827882 else (0, 0)
        assert (st.flat[0], st.flat[10]) == expect


def test_recount_on_lattices_with_known_energy():
    for Lx, Ly in [(2, 2), (4, 4), (6, 4), (8, 8)]:
        N = Lx * Ly
        x, y = np.meshgrid(np.arange(Lx), np.arange(Ly))
        par = (x + y) % 2
        st = np.full((Ly, Lx), 2, np.uint8)  # every site S=+1
        assert list(oracle.recount(st)) == [N, 2 * N, 0, 0, 0, N, 0]
        st = np.zeros((Ly, Lx), np.uint8)  # ferromagnet
        assert list(oracle.recount(st)) == [0, 0, 2 * N, N, 0, 0, 0]
        st = par.astype(np.uint8)  # Neel state: sigma = +1 on even sites
        assert list(oracle.recount(st)) == [0, 0, -2 * N, 0, N, 0, 0]
        st = (2 + par).astype(np.uint8)  # charge checkerboard +1/-1
        assert list(oracle.recount(st)) == [N, -2 * N, 0, 0, 0, 0, N]
        st = np.zeros((Ly, Lx), np.uint8)
        st[0, 0] = 2  # one charge in a ferromagnet loses its 4 spin bonds
        if Lx > 2 and Ly > 2:
            assert list(oracle.recount(st)) == [1, 0, 2 * N - 4, N - 1, -1, 1, 1]


def _all_moves(st):
    Ly, Lx = st.shape
    N = Lx * Ly
    sets = golden_pair_sets()
    for a in range(N):
        for b in range(N):
            if a == b:
                continue
            q = S[st.flat[a]] + S[st.flat[b]]
            for na, nb in sets[q]:
                yield a, b, na, nb


@pytest.mark.parametrize("shape", [(2, 2), (4, 2), (2, 4), (3, 3), (4, 4), (5, 3), (8, 4)])
def test_pair_delta_equals_recount_difference(shape):
    Lx, Ly = shape
    rng = np.random.default_rng(Lx * 100 + Ly)
    for trial in range(3):
        st = rng.integers(0, 4, size=(Ly, Lx)).astype(np.uint8)
        before = oracle.recount(st)
        for a, b, na, nb in _all_moves(st):
            d = oracle.pair_delta(st, a, b, na, nb)
            s2 = st.copy()
            s2.flat[a], s2.flat[b] = na, nb
            after = oracle.recount(s2)
            assert d == tuple(after[:3] - before[:3]), (shape, a, b, na, nb)
            assert after[5] == before[5]  # the pair keeps its charge (Eq. 2)


def _nbr_sums(st, site):
    Ly, Lx = st.shape
    x, y = site % Lx, site // Lx
    nbrs = [y * Lx + (x - 1) % Lx, y * Lx + (x + 1) % Lx, ((y - 1) % Ly) * Lx + x,
            ((y + 1) % Ly) * Lx + x]
    return (sum(S[st.flat[n]] for n in nbrs), sum(SIG[st.flat[n]] for n in nbrs), nbrs)


def test_paper_delta_formulas_where_they_hold():
    """Sec. 3.1 prints E_V and E_J for distant and for neighbouring pairs.

    E_V holds for every move; the printed E_J assumes sigma_b changes by minus
    the change of sigma_a.  Where that holds the oracle must equal the printed
    forms; where it does not, the oracle must follow the recount instead.
    """
    rng = np.random.default_rng(5)
    seen_distant = seen_near = seen_other = 0
    for trial in range(4):
        st = rng.integers(0, 4, size=(6, 6)).astype(np.uint8)
        for a, b, na, nb in _all_moves(st):
            ca, cb = int(st.flat[a]), int(st.flat[b])
            dSa = S[na] - S[ca]
            dGa, dGb = SIG[na] - SIG[ca], SIG[nb] - SIG[cb]
            sSa, sGa, nbrs_a = _nbr_sums(st, a)
            sSb, sGb, _ = _nbr_sums(st, b)
            dQ, dBV, dBJ = oracle.pair_delta(st, a, b, na, nb)
            assert dQ == S[na] ** 2 + S[nb] ** 2 - S[ca] ** 2 - S[cb] ** 2
            near = b in nbrs_a
            if not near:
                assert dBV == dSa * (sSa - sSb)
            else:
                assert dBV == dSa * (sSa - sSb) - dSa ** 2
            if dGb == -dGa:
                if not near:
                    assert dBJ == dGa * (sGa - sGb)
                    seen_distant += 1
                else:
                    assert dBJ == dGa * (sGa - sGb) + dGa * dGb
                    seen_near += 1
            elif not near and dGa * (sGa - sGb) != dBJ:
                seen_other += 1
    assert seen_distant > 1000 and seen_near > 100 and seen_other > 100


@pytest.mark.parametrize("params", [(1.0, 0.5, 1.0, 1.0), (1 / 0.6, 0.2, 1.0, 0.5),
                                    (5.0, 0.0, 0.5, 1.0), (0.37, -0.5, 1.0, 1.0),
                                    (10.0, 1.0, 2.0, 1.0)])
def test_threshold_table_against_50_digit_exp(params):
    mpmath = pytest.importorskip("mpmath")
    beta, Delta, V, J = params
    t = oracle.threshold_table(beta, Delta, V, J)
    mpmath.mp.dps = 50
    two32 = mpmath.mpf(2) ** 32
    for dQ in range(-2, 3):
        for dBV in range(-oracle.DB, oracle.DB + 1):
            for dBJ in range(-oracle.DB, oracle.DB + 1, 3):
                dE = (mpmath.mpf(Delta) * dQ + mpmath.mpf(V) * dBV
                      + mpmath.mpf(J) / 4 * dBJ)
                got = int(t[dQ + 2, dBV + oracle.DB, dBJ + oracle.DB])
                if dE <= 0:
                    assert got == 0xFFFFFFFF
                    continue
                exact = mpmath.floor(two32 * mpmath.exp(-mpmath.mpf(beta) * dE))
                assert got != 0xFFFFFFFF
                assert abs(got - int(min(exact, 0xFFFFFFFE))) <= 1, (dQ, dBV, dBJ)


def test_threshold_table_limits():
    assert np.all(oracle.threshold_table(0.0, 1.0, 1.0, 1.0) == 0xFFFFFFFF)
    t = oracle.threshold_table(float("inf"), 1.0, 1.0, 1.0)
    assert t[2, oracle.DB, oracle.DB] == 0xFFFFFFFF  # dE = 0 is always accepted
    assert t[3, oracle.DB, oracle.DB] == 0  # dE > 0 is never accepted at T = 0
    assert t[1, oracle.DB, oracle.DB] == 0xFFFFFFFF


def test_charge_counts_reading():
    N2 = 4096 * 4096
    assert oracle.charge_counts(N2, 0.1, 0.3) == (1677722, 3355444, 1677722)
    N5 = 16384 * 16384
    assert oracle.charge_counts(N5, 0.05, 0.3) == (13421773, 46976205, 33554432)
    assert oracle.charge_counts(256, 0.125, 0.25) == (32, 48, 16)  # the 48 / 16 split
    assert oracle.charge_counts(256, -0.125, 0.0) == (-32, 0, 32)
    Q, npl, nmi = oracle.charge_counts(1024, 0.1, 0.3)  # C = 307 -> 308 for parity
    assert (Q, npl, nmi) == (102, 205, 103)
    assert oracle.charge_counts(16, 1.0, 1.5) is None


@pytest.mark.parametrize("N", [16, 48, 256, 1024, 4096, 16 * 20])
def test_feistel_rank_is_a_permutation(N):
    ranks = [oracle.feistel_rank(3, N, i) for i in range(N)]
    assert sorted(ranks) == list(range(N))


def test_initial_state_counts_and_uniformity():
    st = oracle.init_counts(16, 16, 1, 48, 16)
    assert list(np.bincount(st.ravel(), minlength=4)[2:]) == [48, 16]
    assert oracle.recount(st)[5] == 32
    st = oracle.init_constrained(64, 32, 11, 0.1, 0.3)
    Q, npl, nmi = oracle.charge_counts(64 * 32, 0.1, 0.3)
    assert list(np.bincount(st.ravel(), minlength=4)[2:]) == [npl, nmi]
    # over many seeds, every site is S=+1 with probability N+/N and the spins
    # of magnetic sites are balanced (chi-square, 15 degrees of freedom)
    nseed, Np = 3000, 3
    hits = np.zeros(16)
    up = down = 0
    for seed in range(nseed):
        s = oracle.init_counts(4, 4, seed, Np, 1).ravel()
        hits += s == 2
        up += np.sum(s == 0)
        down += np.sum(s == 1)
    expect = nseed * Np / 16
    chi2 = float(np.sum((hits - expect) ** 2 / expect))
    assert chi2 < 45.0  # p ~ 1e-4 for 15 dof
    assert abs(up - down) < 5 * np.sqrt(up + down)
