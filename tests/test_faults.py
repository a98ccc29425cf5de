"""Failure paths without faulting a GPU.

Host-side fault injection (the CCMC_FAULT environment variable, read at each
call): allocation failure at handle creation (checked on CPU: the library
returns before any CUDA call), launch failure of a sweep (the handle stays
usable and later sweeps are bit-exact), admission refusal by the server; and
the device-side bounded wait, whose self-test waits on a barrier nothing
completes, gives up, and leaves the context usable.
"""
import os

import numpy as np
import pytest

import oracle

from .gpu_util import oracle_run


@pytest.fixture
def fault(monkeypatch):
    def set_fault(v):
        if v:
            monkeypatch.setenv("CCMC_FAULT", v)
        else:
            monkeypatch.delenv("CCMC_FAULT", raising=False)
    yield set_fault
    monkeypatch.delenv("CCMC_FAULT", raising=False)


def test_injected_allocation_failure_needs_no_gpu(fault):
    import paper_2301_11735_gb300 as cc

    fault("launch,alloc")
    with pytest.raises(cc.CcmcError) as e:
        cc.Lattice(16, 16)
    assert e.value.code == cc.E_NOMEM
    # argument checks still come first
    fault("alloc")
    with pytest.raises(cc.CcmcError) as e:
        cc.Lattice(10, 16)
    assert e.value.code == cc.E_INVAL


@pytest.mark.gpu
def test_injected_launch_failure_leaves_the_lattice_usable(fault):
    import paper_2301_11735_gb300 as cc

    L, seed, params = 32, 7, (1.2, 0.1, 1.0, 1.0)
    st = oracle.init_constrained(L, L, seed, 0.1, 0.3)
    with cc.Lattice(L, L) as lat:
        lat.init_constrained(seed, 0.1, 0.3)
        lat.sweep(2, *params, obs_every=1)
        fault("launch")
        for call in (lambda: lat.sweep(3, *params), lambda: lat.phases(5, *params)):
            with pytest.raises(cc.CcmcError) as e:
                call()
            assert e.value.code == cc.E_CUDA
        fault(None)
        lat.sweep(3, *params, obs_every=1)
        st, rec = oracle_run(st, seed, 0, 5, *params)
        assert np.array_equal(lat.get_state(), st)
        assert np.array_equal(lat.obs_series(), rec)


@pytest.mark.gpu
def test_injected_admission_refusal(fault):
    import paper_2301_11735_gb300 as cc

    with cc.Server(hbm_budget_bytes=1 << 30) as srv:
        fault("admit")
        t = srv.submit(32, 32, 5, 0.1, 4, 1.0, 0.0, 1.0, 1.0)
        r = srv.wait(t, timeout_s=30.0)
        assert r["status"] == cc.E_BUDGET
        assert srv.stats()["rejected"] == 1
        fault(None)
        t = srv.submit(32, 32, 5, 0.1, 4, 1.0, 0.0, 1.0, 1.0)
        r = srv.wait(t, timeout_s=30.0)
        assert r["status"] == cc.OK and r["final_obs"]["sweeps_done"] == 4


@pytest.mark.gpu
def test_device_wait_gives_up_and_the_context_stays_usable():
    import paper_2301_11735_gb300 as cc

    assert cc.selftest_wait(1 << 16) == cc.E_TIMEOUT
    assert cc.selftest_wait(0) == cc.E_INVAL
    # the context still runs kernels correctly afterwards
    got = cc.philox_device([5, 6, 7, 8], [9, 10], 4)
    ref = np.array([oracle.philox([5 + i, 6, 7, 8], [9, 10]) for i in range(4)],
                   dtype=np.uint32).ravel()
    assert np.array_equal(got.ravel(), ref)
