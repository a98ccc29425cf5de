"""Serving: continuous batching of independent simulations.

Every request's final lattice, final observables and observable records must
be the same when it runs in a mix through the server as when it runs alone;
admission must respect the slot and memory limits; requests that arrive while
others run must start before those finish.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import paper_2301_11735_gb300 as cc

    return cc


def _alone(cc, r):
    with cc.Lattice(r["Lx"], r["Ly"], obs_capacity=1024) as lat:
        lat.init_constrained(r["seed"], r["n"], 0.3)
        lat.sweep(r["nsweeps"], r["beta"], r["Delta"], r["V"], r["J"], obs_every=r["obs_every"])
        return lat.get_state(), lat.observables(), lat.obs_series()


def _requests():
    rng = np.random.default_rng(11)
    shapes = [(16, 16), (32, 32), (20, 12), (64, 64), (36, 44), (128, 128), (256, 256),
              (68, 20), (512, 512), (4, 4), (132, 8), (1024, 1024)]
    out = []
    for i, (Lx, Ly) in enumerate(shapes):
        out.append(dict(Lx=Lx, Ly=Ly, seed=900 + i, n=float(rng.choice([0.0, 0.1, -0.2])),
                        nsweeps=int(rng.integers(20, 400)), beta=float(1 / rng.uniform(0.2, 3.0)),
                        Delta=float(rng.uniform(-1, 1)), V=float(rng.uniform(0, 2)), J=1.0,
                        obs_every=int(rng.choice([0, 5, 7]))))
    return out


def test_each_result_is_the_same_alone_and_in_the_mix(cc):
    reqs = _requests()
    with cc.Server(hbm_budget_bytes=1 << 30, max_active=6, slice_ms=2.0) as srv:
        tickets = []
        for k, r in enumerate(reqs):
            out = np.zeros(r["Lx"] * r["Ly"], dtype=np.uint8)
            t = srv.submit(r["Lx"], r["Ly"], r["seed"], r["n"], r["nsweeps"], r["beta"],
                           r["Delta"], r["V"], r["J"], obs_every=r["obs_every"], state_out=out)
            tickets.append((t, out))
            if k % 3 == 2:
                time.sleep(0.003)  # let some arrive while others are running
        results = [(srv.wait(t), out, srv.series(t)) for t, out in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["rejected"] == 0 and st["failed"] == 0
    assert st["slices"] > 1
    for r, (res, out, series) in zip(reqs, results):
        assert res["status"] == 0
        state, obs, rec = _alone(cc, r)
        assert np.array_equal(out.reshape(r["Ly"], r["Lx"]), state), r
        for k in ("Nc", "BV", "BJ", "M", "M_stag", "S_sum", "S_stag", "sweeps_done"):
            assert res["final_obs"][k] == obs[k], (r, k)
        assert np.array_equal(series, rec), r
        assert res["site_updates"] == r["Lx"] * r["Ly"] * r["nsweeps"]


def test_admission_by_budget_and_slots(cc):
    # each 128^2 request needs ~0.15 MB: a 0.4 MB budget admits two at a time
    with cc.Server(hbm_budget_bytes=400_000, max_active=8, slice_ms=1.0) as srv:
        ts = [srv.submit(128, 128, 50 + i, 0.1, 300, 1.0, 0.0, 1.0, 1.0) for i in range(6)]
        big = srv.submit(2048, 2048, 7, 0.0, 10, 1.0, 0.0, 1.0, 1.0)  # never fits
        peak = 0
        while any(srv.poll(t) is None for t in ts):
            peak = max(peak, srv.stats()["active"])
            time.sleep(0.0005)
        res = [srv.wait(t) for t in ts]
        rb = srv.wait(big)
    assert all(r["status"] == 0 for r in res)
    assert rb["status"] == cc.E_BUDGET
    assert peak <= 2
    starts = sorted(r["start_s"] for r in res)
    dones = sorted(r["done_s"] for r in res)
    assert starts[2] >= dones[0] - 1e-6  # the third started only after one finished


def test_late_arrivals_join_while_others_run(cc):
    with cc.Server(hbm_budget_bytes=1 << 30, max_active=16, slice_ms=2.0) as srv:
        long_t = srv.submit(256, 256, 1, 0.1, 4000, 1.0, 0.0, 1.0, 1.0)
        time.sleep(0.02)
        short_t = srv.submit(32, 32, 2, 0.1, 50, 1.0, 0.0, 1.0, 1.0)
        rs = srv.wait(short_t)
        rl = srv.wait(long_t)
    assert rs["done_s"] < rl["done_s"]
    assert rs["start_s"] > rl["start_s"]


def test_poll_release_and_bad_requests(cc):
    with cc.Server(hbm_budget_bytes=1 << 28, max_active=4) as srv:
        t = srv.submit(16, 16, 3, 0.125, 10, 1.0, 0.5, 1.0, 1.0)
        srv.wait(t)
        assert srv.poll(t)["status"] == 0
        srv.release(t)
        with pytest.raises(cc.CcmcError):
            srv.poll(t)
        with pytest.raises(cc.CcmcError):
            srv.submit(18, 16, 3, 0.0, 10, 1.0, 0.0, 1.0, 1.0)  # Lx not a multiple of 4
        with pytest.raises(cc.CcmcError):
            srv.submit(16, 16, 3, 0.0, 10, -1.0, 0.0, 1.0, 1.0)  # negative beta
