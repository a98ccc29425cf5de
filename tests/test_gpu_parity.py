"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Every comparison is bit-exact: lattice states, integer energy terms, the
charge sum (which must equal n N after every sweep), schedules and random
words.  Shapes cover several tiles of 16 sites, ragged row tails (Lx/4 not a
multiple of 16 or of 4), rows shorter than one word, and the full sizes of the
4096^2 and 16384^2 workloads (their first 20 and 5 sweeps).
"""
import numpy as np
import pytest

import oracle

from .gpu_util import first_difference, oracle_run

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4), (8, 8), (12, 20), (16, 16), (20, 12), (36, 44), (64, 64), (68, 20), (80, 72),
          (128, 128), (132, 8), (260, 36)]
PARAMS = [(1.0, 0.5, 1.0, 1.0), (1 / 0.6, 0.2, 1.0, 0.5), (5.0, 0.0, 0.5, 1.0),
          (0.5, -0.5, 1.0, 1.0), (1 / 3.0, -1.0, 2.0, 1.0)]


@pytest.fixture(scope="module")
def cc():
    import paper_2301_11735_gb300 as cc

    return cc


@pytest.mark.parametrize("ctr,key", [((0xFF800000, 7, 9, 2), (0xDEADBEEF, 0x12345678)),
                                     ((0, 0xFFFFFFFF, 1, 0x4D4F5645), (5, 0))])
def test_device_philox_matches_oracle_on_2_to_the_24_counters(cc, ctr, key):
    """Every output of 2^24 consecutive counters (the first set wraps word 0
    through 2^32), bit for bit."""
    n = 1 << 24
    dev = cc.philox_device(ctr, key, n)
    ref = oracle.philox_block(ctr, key, n)
    assert np.array_equal(dev, ref), first_difference(dev, ref)


def test_device_philox_matches_oracle(cc):
    for ctr, key in [((0, 0, 0, 0), (0, 0)), ((0xFFFFFF00, 7, 9, 2), (0xDEADBEEF, 0x12345678)),
                     ((123, 0xFFFFFFFF, 0, 5), (1, 0))]:
        dev = cc.philox_device(ctr, key, 300)
        for i in range(0, 300, 7):
            c = [(ctr[0] + i) & 0xFFFFFFFF, ctr[1], ctr[2], ctr[3]]
            assert np.array_equal(dev[i], oracle.philox(c, key)), (ctr, key, i)


@pytest.mark.parametrize("shape", SHAPES)
def test_initial_state_matches_oracle(cc, shape):
    Lx, Ly = shape
    N = Lx * Ly
    with cc.Lattice(Lx, Ly) as lat:
        for seed, (npl, nmi) in [(1, (N // 5, N // 10)), (2 ** 40 + 3, (0, 0)), (99, (N, 0)),
                                 (7, (N // 3, N // 3))]:
            lat.init_counts(seed, npl, nmi)
            got = lat.get_state()
            exp = oracle.init_counts(Lx, Ly, seed, npl, nmi)
            assert np.array_equal(got, exp), (shape, seed, first_difference(got, exp))
        lat.init_constrained(11, 0.1, 0.3)
        assert np.array_equal(lat.get_state(), oracle.init_constrained(Lx, Ly, 11, 0.1, 0.3))


@pytest.mark.parametrize("shape", [(4, 4), (20, 12), (68, 20), (128, 128)])
def test_state_roundtrip_and_bad_codes(cc, shape):
    Lx, Ly = shape
    rng = np.random.default_rng(3)
    st = rng.integers(0, 4, size=(Ly, Lx)).astype(np.uint8)
    with cc.Lattice(Lx, Ly) as lat:
        lat.set_state(st, 5, 0)
        assert np.array_equal(lat.get_state(), st)
        obs = lat.observables()
        assert [obs[k] for k in ("Nc", "BV", "BJ", "M", "M_stag", "S_sum", "S_stag")] == \
            list(oracle.recount(st))
        bad = st.copy()
        bad[0, 0] = 4
        with pytest.raises(cc.CcmcError):
            lat.set_state(bad, 5, 0)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("params", PARAMS[:3])
def test_sweeps_bit_exact_every_sweep(cc, shape, params):
    Lx, Ly = shape
    beta, Delta, V, J = params
    seed = 1000 + Lx * 7 + Ly
    st0 = oracle.init_constrained(Lx, Ly, seed, 0.1, 0.3)
    Q = int(oracle.recount(st0)[5])
    with cc.Lattice(Lx, Ly) as lat:
        lat.init_constrained(seed, 0.1, 0.3)
        st = st0.copy()
        for s in range(6):
            lat.sweep(1, beta, Delta, V, J, obs_every=1)
            st, rec = oracle_run(st, seed, s, 1, beta, Delta, V, J)
            got = lat.get_state()
            assert np.array_equal(got, st), (shape, s, first_difference(got, st))
            assert oracle.recount(got)[5] == Q
        recs = lat.obs_series()
        assert len(recs) == 6 and np.all(recs[:, 6] == Q)
        assert np.array_equal(recs[-1], rec[-1])


@pytest.mark.parametrize("params", PARAMS)
def test_multi_sweep_calls_graph_and_direct_paths(cc, params):
    """Long calls run through captured CUDA graphs, short or misaligned ones
    launch directly; both must give the oracle's records at every obs point."""
    beta, Delta, V, J = params
    Lx, Ly, seed = 36, 44, 77
    st = oracle.init_constrained(Lx, Ly, seed, -0.05, 0.4)
    with cc.Lattice(Lx, Ly, obs_capacity=512) as lat:
        lat.init_constrained(seed, -0.05, 0.4)
        done = 0
        all_rec = []
        for n, every in [(37, 1), (5, 3), (40, 3), (33, 0), (50, 7), (41, 20)]:
            lat.sweep(n, beta, Delta, V, J, obs_every=every)
            st, rec = oracle_run(st, seed, done, n, beta, Delta, V, J, obs_every=every)
            all_rec.append(rec)
            done += n
            got = lat.get_state()
            assert np.array_equal(got, st), (n, every, first_difference(got, st))
        exp = np.concatenate([r for r in all_rec if len(r)])
        assert np.array_equal(lat.obs_series(), exp)


def test_workload_16x16_full_length(cc):
    """L = 16, Delta = 0.5, V = J = 1, T = 1, 48 charges +1 and 16 charges -1,
    2000 sweeps with observables after every sweep: identical records."""
    seed = 1
    st = oracle.init_counts(16, 16, seed, 48, 16)
    _, rec = oracle_run(st, seed, 0, 2000, 1.0, 0.5, 1.0, 1.0, obs_every=1)
    with cc.Lattice(16, 16) as lat:
        lat.init_counts(seed, 48, 16)
        lat.sweep(2000, 1.0, 0.5, 1.0, 1.0, obs_every=1)
        got = lat.obs_series()
    assert np.all(got[:, 6] == 32)
    assert np.array_equal(got, rec)


@pytest.mark.parametrize("params", [(0.0, 1.0, 1.0, 1.0), (float("inf"), 0.5, 1.0, 1.0),
                                    (1.0, 1e9, 1.0, 1.0), (1.0, -1e9, 1.0, 1.0)])
@pytest.mark.parametrize("shape", [(16, 16), (20, 12)])
def test_degenerate_parameters(cc, params, shape):
    Lx, Ly = shape
    beta, Delta, V, J = params
    st = oracle.init_counts(Lx, Ly, 5, Lx * Ly // 8 + 4, Lx * Ly // 8)
    with cc.Lattice(Lx, Ly) as lat:
        lat.init_counts(5, Lx * Ly // 8 + 4, Lx * Ly // 8)
        lat.sweep(30, beta, Delta, V, J, obs_every=1)
        st, rec = oracle_run(st, 5, 0, 30, beta, Delta, V, J)
        assert np.array_equal(lat.get_state(), st)
        assert np.array_equal(lat.obs_series(), rec)


def test_checkpoint_resume_is_bit_exact(cc):
    Lx = Ly = 64
    with cc.Lattice(Lx, Ly) as a, cc.Lattice(Lx, Ly) as b:
        a.init_constrained(9, 0.1, 0.3)
        a.sweep(100, 1.2, 0.2, 1.0, 0.5, obs_every=10)
        b.init_constrained(9, 0.1, 0.3)
        b.sweep(50, 1.2, 0.2, 1.0, 0.5, obs_every=10)
        snap = b.get_state()
        b.init_counts(123, 1, 1)  # scramble, then restore
        b.set_state(snap, 9, 50)
        b.sweep(50, 1.2, 0.2, 1.0, 0.5, obs_every=10)
        assert np.array_equal(a.get_state(), b.get_state())
        assert np.array_equal(a.obs_series()[-5:], b.obs_series()[-5:])


def test_histograms_follow_the_records(cc):
    Lx = Ly = 32
    N = Lx * Ly
    nb = 64
    with cc.Lattice(Lx, Ly) as lat:
        lat.hist_enable(nb)
        lat.init_constrained(4, 0.05, 0.3)
        lat.sweep(200, 1 / 0.6, 0.2, 1.0, 0.5, obs_every=1)
        rec = lat.obs_series()
        h = lat.hist()
    for row, col in enumerate((4, 5, 7)):
        bins = (rec[:, col] + N) * nb // (2 * N + 1)
        assert np.array_equal(h[row], np.bincount(bins, minlength=nb))


@pytest.mark.parametrize("T", [0.5, 2.0])
def test_full_size_4096_first_sweeps(cc, T):
    """The 4096^2 workload (Delta = 0, V = 0.5, J = 1, n = 0.1, charged
    fraction 0.3): identical initial state, and identical lattice after each of
    the first 20 sweeps and records of every sweep."""
    L, seed = 4096, 20
    st = oracle.init_constrained(L, L, seed, 0.1, 0.3)
    with cc.Lattice(L, L) as lat:
        lat.init_constrained(seed, 0.1, 0.3)
        assert np.array_equal(lat.get_state(), st)
        recs = []
        for s in range(20):
            lat.sweep(1, 1.0 / T, 0.0, 0.5, 1.0, obs_every=1)
            st, rec = oracle_run(st, seed, s, 1, 1.0 / T, 0.0, 0.5, 1.0)
            recs.append(rec[-1])
            got = lat.get_state()
            assert np.array_equal(got, st), (s, first_difference(got, st))
        assert np.array_equal(lat.obs_series(), np.array(recs))
        assert all(r[6] == 1677722 for r in recs)


def test_full_size_16384_first_sweeps(cc):
    """The 16384^2 workload (Delta = 0.2, V = 1, J = 0.5, n = 0.05, T = 0.6):
    the oracle's own initial state (every site) and the lattice and records
    after each of the first five sweeps."""
    L, seed = 16384, 5
    params = (1 / 0.6, 0.2, 1.0, 0.5)
    Q, npl, nmi = oracle.charge_counts(L * L, 0.05, 0.3)
    st = oracle.init_constrained(L, L, seed, 0.05, 0.3)
    counts = np.bincount(st.ravel(), minlength=4)
    assert counts[2] == npl and counts[3] == nmi
    with cc.Lattice(L, L) as lat:
        lat.init_constrained(seed, 0.05, 0.3)
        assert np.array_equal(lat.get_state(), st)
        for s in range(5):
            lat.sweep(1, *params, obs_every=1)
            st, rec = oracle_run(st, seed, s, 1, *params)
            got = lat.get_state()
            assert np.array_equal(got, st), (s, first_difference(got, st))
            assert np.array_equal(lat.obs_series()[-1], rec[-1]), s
            assert rec[-1][6] == Q


@pytest.mark.parametrize("path", ["plain", "batch"])
@pytest.mark.parametrize("shape", [(64, 48), (256, 256), (36, 44)])
def test_resume_across_the_phase_counter_high_word(cc, shape, path):
    """A state resumed at sweep 2^29 - 1: its eight phases end at global phase
    2^32 - 1 and the next sweep's start at 2^32, so the schedule and move
    streams take the counter's high word (Philox counter word 2) from 0 to 1.
    The state is drawn by the seeded test generator, not by either side."""
    Lx, Ly = shape
    seed, sweep0 = 31 + Lx, (1 << 29) - 1
    params = (1 / 0.8, 0.1, 1.0, 0.5)
    rng = np.random.default_rng(Lx * Ly)
    st = rng.integers(0, 4, size=(Ly, Lx)).astype(np.uint8)
    exp, erec = oracle_run(st, seed, sweep0, 3, *params)
    assert erec[-1][0] == sweep0 + 3
    with cc.Lattice(Lx, Ly) as lat:
        lat.set_state(st, seed, sweep0)
        if path == "plain":
            lat.sweep(3, *params, obs_every=1)
        else:
            with cc.Batch([lat]) as b:
                b.sweep(3, *([p] for p in params), obs_every=1)
                b.sync()
        got = lat.get_state()
        assert np.array_equal(got, exp), first_difference(got, exp)
        assert np.array_equal(lat.obs_series(), erec)


def test_phase_steps_mixed_with_sweeps(cc):
    """ccmc_phases runs single colour phases (the paper's "steps"); mixed with
    ccmc_sweep the phase counter continues, matching the oracle phase by phase."""
    Lx, Ly, seed = 20, 12, 61
    beta, Delta, V, J = 1.3, 0.1, 1.0, 1.0
    st = oracle.init_constrained(Lx, Ly, seed, 0.2, 0.4)
    table = oracle.threshold_table(beta, Delta, V, J)
    P = 0
    with cc.Lattice(Lx, Ly) as lat:
        lat.init_constrained(seed, 0.2, 0.4)
        for nph in (3, 1, 4, 13):
            lat.phases(nph, beta, Delta, V, J)
            for _ in range(nph):
                oracle.phase(st, seed, P, table)
                P += 1
            assert np.array_equal(lat.get_state(), st), P
        lat.sweep(3, beta, Delta, V, J, obs_every=1)  # finishes the open sweep first
        while P % 8:
            oracle.phase(st, seed, P, table)
            P += 1
        st, rec = oracle_run(st, seed, P // 8, 2, beta, Delta, V, J)
        assert np.array_equal(lat.get_state(), st)
        got = lat.obs_series()
        assert np.array_equal(got[-2:], rec)
        assert got[0, 0] == 3  # the record of the sweep the phases left open


TILE_SHAPES = [(256, 256), (512, 128), (1024, 64), (2048, 32), (256, 4096), (512, 512),
               (1024, 256)]


def _lattice(cc, Lx, Ly, path: str):
    """A lattice on one phase path, chosen by environment variables read at
    creation: "tile" (the default: the single-tile kernel for phases that fit
    one wave of it, else the pipelined one), "pipelined" (the pipelined tile
    kernel on at most three CTAs, so that each takes several tiles and later
    phases stage their first tile early) or "direct" (no staging)."""
    import os

    env = {"tile": {}, "pipelined": {"CCMC_TILE_GRID": "3"}, "direct": {"CCMC_NO_TILE": "1"}}[path]
    for k in ("CCMC_NO_TILE", "CCMC_TILE_GRID"):
        os.environ.pop(k, None)
    os.environ.update(env)
    try:
        return cc.Lattice(Lx, Ly)
    finally:
        for k in env:
            os.environ.pop(k, None)


@pytest.mark.parametrize("shape", TILE_SHAPES)
@pytest.mark.parametrize("path", ["tile", "pipelined", "direct"])
def test_tile_and_direct_paths_match_oracle(cc, shape, path):
    Lx, Ly = shape
    seed = 300 + Lx + Ly
    params = (1 / 0.8, 0.1, 1.0, 1.0)
    st = oracle.init_constrained(Lx, Ly, seed, 0.05, 0.3)
    with _lattice(cc, Lx, Ly, path) as lat:
        lat.init_constrained(seed, 0.05, 0.3)
        for s in range(4):
            lat.sweep(1, *params, obs_every=1)
            st, rec = oracle_run(st, seed, s, 1, *params)
            got = lat.get_state()
            assert np.array_equal(got, st), (shape, path, s, first_difference(got, st))
        assert np.array_equal(lat.obs_series()[-1], rec[-1])
        # a multi-sweep call replays the captured graph of phases (the early
        # staging runs in graphs too)
        lat.sweep(16, *params, obs_every=0)
        st, _ = oracle_run(st, seed, 4, 16, *params)
        got = lat.get_state()
        assert np.array_equal(got, st), (shape, path, "graph", first_difference(got, st))


def _near_seed(Lx, Ly, want, max_phase=320):
    for seed in range(1, 20000):
        for P in range(max_phase):
            r = oracle.schedule(Lx, Ly, seed, P)[2:]
            if r == want:
                return seed, P
    raise AssertionError("no seed found")


@pytest.mark.parametrize("want", [(1, 0), (1023, 0), (0, 1), (0, 63)])
def test_tile_path_nearest_neighbour_phases(cc, want):
    """Phases whose offset is an exact nearest neighbour (the partner shares a
    bond, and b's class is one of a's neighbour classes) on the tile path."""
    Lx, Ly = 1024, 64
    seed, P = _near_seed(Lx, Ly, want)
    nsw = P // 8 + 1
    params = (1.3, -0.2, 1.0, 0.7)
    st = oracle.init_constrained(Lx, Ly, seed, 0.1, 0.4)
    with _lattice(cc, Lx, Ly, "tile") as lat:
        lat.init_constrained(seed, 0.1, 0.4)
        lat.sweep(nsw, *params, obs_every=1)
        st, rec = oracle_run(st, seed, 0, nsw, *params)
        assert np.array_equal(lat.get_state(), st), (want, seed, P)
        assert np.array_equal(lat.obs_series(), rec)


def _pack_rowmajor(st):
    """The compact form by its definition: site i at bits 2 (i mod 4) of byte i / 4."""
    c = st.reshape(-1, 4).astype(np.uint8)
    return (c[:, 0] | (c[:, 1] << 2) | (c[:, 2] << 4) | (c[:, 3] << 6)).astype(np.uint8)


@pytest.mark.parametrize("shape", [(4, 4), (12, 20), (64, 64), (68, 20), (260, 36), (256, 128),
                                   (1024, 64)])
def test_packed_state_roundtrip_and_resume(cc, shape):
    Lx, Ly = shape
    rng = np.random.default_rng(Lx + Ly)
    st = rng.integers(0, 4, size=(Ly, Lx)).astype(np.uint8)
    packed = _pack_rowmajor(st)
    seed, params = 17 + Lx, (1.2, 0.2, 1.0, 0.5)
    with cc.Lattice(Lx, Ly) as lat:
        lat.set_state_packed(packed, seed, 3)
        lat.sync()
        assert np.array_equal(lat.get_state(), st)
        assert np.array_equal(lat.get_state_packed(), packed)
        lat.sweep(2, *params, obs_every=1)
        got = lat.get_state()
        rec = lat.obs_series()
    exp, erec = oracle_run(st, seed, 3, 2, *params)
    assert np.array_equal(got, exp), first_difference(got, exp)
    assert np.array_equal(rec, erec)
