"""Batched replicas: many lattices of uneven size in one persistent launch.

Each lattice of a batch must end bit-identical to the same lattice advanced on
its own with ccmc_sweep (and, for small ones, to the oracle), with identical
observable records, whatever the launch shape the autotuner picks.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

MIX = [(4, 4), (16, 16), (20, 12), (32, 32), (36, 44), (64, 64), (68, 20), (128, 128),
       (256, 256), (132, 8)]


@pytest.fixture(scope="module")
def cc():
    import paper_2301_11735_gb300 as cc

    return cc


def _params(i):
    T = 0.3 + 0.17 * i
    return (1.0 / T, [-0.5, 0.0, 0.5][i % 3], 1.0, [1.0, 0.5][i % 2])


def _make(cc, shapes, seed0=100):
    lats = []
    for i, (Lx, Ly) in enumerate(shapes):
        lat = cc.Lattice(Lx, Ly, obs_capacity=256)
        lat.init_constrained(seed0 + i, [0.0, 0.1, -0.2, 0.3][i % 4], 0.3)
        lats.append(lat)
    return lats


def _run_batch(cc, shapes, nsweeps, obs_every, cfg=None, calls=1):
    lats = _make(cc, shapes)
    with cc.Batch(lats) as b:
        if cfg:
            b.config(*cfg)
        P = [_params(i) for i in range(len(shapes))]
        for _ in range(calls):
            b.sweep(nsweeps, [p[0] for p in P], [p[1] for p in P], [p[2] for p in P],
                    [p[3] for p in P], obs_every=obs_every)
        b.sync()
    out = [(lat.get_state(), lat.obs_series()) for lat in lats]
    for lat in lats:
        lat.close()
    return out


def _run_single(cc, shapes, nsweeps, obs_every, calls=1):
    lats = _make(cc, shapes)
    out = []
    for i, lat in enumerate(lats):
        for _ in range(calls):
            lat.sweep(nsweeps[i], *_params(i), obs_every=obs_every)
        out.append((lat.get_state(), lat.obs_series()))
        lat.close()
    return out


def test_batch_equals_individual_sweeps_and_oracle(cc):
    nsw = [11 + 3 * i for i in range(len(MIX))]
    got = _run_batch(cc, MIX, nsw, obs_every=2)
    ref = _run_single(cc, MIX, nsw, obs_every=2)
    for i, ((s1, r1), (s2, r2)) in enumerate(zip(got, ref)):
        assert np.array_equal(s1, s2), MIX[i]
        assert np.array_equal(r1, r2), MIX[i]
    for i in (0, 1, 2, 4, 6):
        Lx, Ly = MIX[i]
        st = oracle.init_constrained(Lx, Ly, 100 + i, [0.0, 0.1, -0.2, 0.3][i % 4], 0.3)
        rec = oracle.sweeps(st, 100 + i, 0, nsw[i], *_params(i), obs_every=2)
        assert np.array_equal(got[i][0], st) and np.array_equal(got[i][1], rec), MIX[i]


# More lattices than CTAs resident at once (one CTA an SM): those whose words
# fit one warp's share of the CTA's shared memory run one a warp.
PACKED = [(4, 4), (8, 12), (16, 16), (20, 12), (32, 32), (36, 44), (64, 64), (68, 20),
          (128, 128), (12, 40)]


@pytest.mark.parametrize("cfg", [(256, 1 << 17, 1, 4), (512, 1 << 17, 1, 2), (64, 1 << 17, 1, 1)])
def test_many_small_lattices_run_one_a_warp_bit_exact(cc, cfg):
    shapes = [PACKED[i % len(PACKED)] for i in range(200)]
    nsw = [5 + i % 7 for i in range(200)]
    got = _run_batch(cc, shapes, nsw, obs_every=3, cfg=cfg)
    ref = _run_single(cc, shapes, nsw, obs_every=3)
    for i, ((s1, r1), (s2, r2)) in enumerate(zip(got, ref)):
        assert np.array_equal(s1, s2), (cfg, i, shapes[i])
        assert np.array_equal(r1, r2), (cfg, i, shapes[i])


@pytest.mark.parametrize("cfg", [(64, 1 << 17, 1, 4), (128, 1 << 17, 4, 4), (256, 1 << 17, 8, 4),
                                 (256, 4096, 2, 4), (256, 1 << 17, 2, 1), (256, 1 << 17, 2, 2),
                                 (512, 1 << 17, 1, 1), (512, 1 << 17, 1, 2),
                                 (512, 1 << 17, 1, 4), (128, 1 << 17, 2, 2)])
def test_batch_results_do_not_depend_on_launch_shape(cc, cfg):
    """Launch shapes the autotuner may pick, including a resident limit that
    sends the larger lattices down the per-phase path."""
    nsw = [7] * len(MIX)
    base = _run_batch(cc, MIX, nsw, obs_every=3)
    got = _run_batch(cc, MIX, nsw, obs_every=3, cfg=cfg)
    for i, ((s1, r1), (s2, r2)) in enumerate(zip(got, base)):
        assert np.array_equal(s1, s2) and np.array_equal(r1, r2), (cfg, MIX[i])


def test_batch_continues_across_calls(cc):
    nsw = [5] * len(MIX)
    two = _run_batch(cc, MIX, nsw, obs_every=1, calls=2)
    one = _run_single(cc, MIX, [10] * len(MIX), obs_every=1)
    for (s1, r1), (s2, r2) in zip(two, one):
        assert np.array_equal(s1, s2) and np.array_equal(r1, r2)


def test_replica_workload_sample(cc):
    """A sample of the 512-replica workload (L in {32, 64, 128, 256}, T grid,
    n and Delta drawn per replica): batched == one by one."""
    from workloads import replicas_512

    sims = replicas_512(nsweeps=40)[:48]
    lats = []
    for s in sims:
        lat = cc.Lattice(s.Lx, s.Ly)
        lat.init_constrained(s.seed, s.n, s.charged_frac)
        lats.append(lat)
    with cc.Batch(lats) as b:
        b.sweep([s.nsweeps for s in sims], [s.beta for s in sims], [s.Delta for s in sims],
                [s.V for s in sims], [s.J for s in sims], obs_every=10)
        b.sync()
    for s, lat in zip(sims, lats):
        with cc.Lattice(s.Lx, s.Ly) as one:
            one.init_constrained(s.seed, s.n, s.charged_frac)
            one.sweep(s.nsweeps, s.beta, s.Delta, s.V, s.J, obs_every=10)
            assert np.array_equal(one.get_state(), lat.get_state())
            assert np.array_equal(one.obs_series(), lat.obs_series())
        lat.close()


def test_batch_rejects_bad_use(cc):
    a = cc.Lattice(16, 16)
    b_ = cc.Lattice(16, 16)
    with pytest.raises(cc.CcmcError):
        with cc.Batch([a, b_]) as b:  # b_ never initialised
            a.init_constrained(1, 0.0)
            b.sweep(2, 1.0, 0.0, 1.0, 1.0)
    b_.init_constrained(2, 0.0)
    a.phases(3, 1.0, 0.0, 1.0, 1.0)  # a is now mid-sweep
    with cc.Batch([a, b_]) as b:
        with pytest.raises(cc.CcmcError):
            b.sweep(2, 1.0, 0.0, 1.0, 1.0)
        with pytest.raises(cc.CcmcError):
            b.config(100, 1 << 16, 2)
        with pytest.raises(cc.CcmcError):
            b.config(256, 1 << 16, 2, 3)  # threads a word: 1, 2 or 4
    a.close()
    b_.close()


def test_autotuner_picks_a_valid_shape_and_results_stay_exact(cc, tmp_path, monkeypatch):
    from paper_2301_11735_gb300 import autotune

    monkeypatch.setattr(autotune, "_CACHE", str(tmp_path / "tune.json"))
    shapes = MIX[:6]
    best = autotune.tune(shapes, probe_sweeps=3)
    assert best in autotune.CANDIDATES
    assert autotune.tune(shapes, probe_sweeps=3) == best  # cached
    nsw = [6] * len(shapes)
    got = _run_batch(cc, shapes, nsw, obs_every=2, cfg=best)
    ref = _run_single(cc, shapes, nsw, obs_every=2)
    for (s1, r1), (s2, r2) in zip(got, ref):
        assert np.array_equal(s1, s2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("shapes", [[(512, 512)] * 8 + [(256, 256)],
                                    [(516, 260)] * 8 + [(1024, 1024)],
                                    [(1024, 1024)] * 4 + [(512, 512)] * 2 + [(1024, 512)] * 2])
def test_large_lattices_in_lockstep_equal_individual_runs(cc, shapes):
    """Eight or more lattices at the same sweep advance with one phase launch
    for all of them (a lock-step group: the tile-staged kernel in the first and
    third cases, with uneven tile counts in the third; the direct kernel for the
    eight 516 x 260); each must still match its own run.  A small resident limit
    sends every lattice down the large path."""
    n = len(shapes)
    seeds = [20 + i for i in range(n)]
    Ts = [0.2 + 0.25 * i for i in range(n)]
    lats = []
    for (Lx, Ly), sd in zip(shapes, seeds):
        lat = cc.Lattice(Lx, Ly)
        lat.init_constrained(sd, 0.1, 0.3)
        lats.append(lat)
    with cc.Batch(lats) as b:
        b.config(256, 1024, 2)
        for _ in range(2):  # the second call replays the captured group graph
            b.sweep(17, [1 / T for T in Ts], 0.0, 0.5, 1.0, obs_every=1)
        b.sync()
    for (Lx, Ly), sd, T, lat in zip(shapes, seeds, Ts, lats):
        with cc.Lattice(Lx, Ly) as one:
            one.init_constrained(sd, 0.1, 0.3)
            one.sweep(34, 1 / T, 0.0, 0.5, 1.0, obs_every=1)
            assert np.array_equal(one.get_state(), lat.get_state()), (Lx, Ly, T)
            assert np.array_equal(one.obs_series(), lat.obs_series()), (Lx, Ly, T)
        lat.close()


def test_resident_records_wrap_the_ring_and_fill_histograms(cc):
    """Lattices in the resident launch with a ring of 8 records and 32-bin
    histograms: 2 calls x 7 sweeps with a record after every sweep wrap the
    ring, and the ring and histograms equal those of the plain path."""
    shapes = [(16, 16), (32, 32), (64, 32), (32, 8)]

    def run(batched):
        out = []
        lats = []
        for i, (Lx, Ly) in enumerate(shapes):
            lat = cc.Lattice(Lx, Ly, obs_capacity=8)
            lat.hist_enable(32)
            lat.init_constrained(700 + i, [0.0, 0.1, -0.2, 0.3][i], 0.3)
            lats.append(lat)
        P = [_params(i) for i in range(len(shapes))]
        for _ in range(2):
            if batched:
                with cc.Batch(lats) as b:
                    b.sweep(7, [p[0] for p in P], [p[1] for p in P], [p[2] for p in P],
                            [p[3] for p in P], obs_every=1)
                    b.sync()
            else:
                for lat, p in zip(lats, P):
                    lat.sweep(7, *p, obs_every=1)
        for lat in lats:
            out.append((lat.get_state(), lat.obs_series(), lat.hist()))
            lat.close()
        return out

    got, ref = run(True), run(False)
    for (s1, r1, h1), (s2, r2, h2), shape in zip(got, ref, shapes):
        assert len(r1) == 8 and r1[-1, 0] == 14, shape
        assert np.array_equal(s1, s2) and np.array_equal(r1, r2), shape
        assert np.array_equal(h1, h2) and h1.sum() == 3 * 14, shape
