"""The library's host map builder (ccmc_maps_build, no GPU needed) against the
oracle's: the same maps bit for bit, whatever the number of host threads, and
bad arguments rejected."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def cc():
    import paper_2301_11735_gb300 as cc

    return cc


@pytest.mark.parametrize("Lx,Ly,seed,map0", [(4, 4, 1, 0), (8, 8, 77, 5), (12, 8, 3, 2 ** 33),
                                             (20, 16, 2 ** 63 + 9, 7), (68, 20, 5, 0),
                                             (256, 256, 11, 1)])
def test_library_maps_equal_oracle_maps(cc, Lx, Ly, seed, map0):
    assert cc.map_size(Lx, Ly) == oracle.map_size(Lx, Ly) == max(1, Lx * Ly // 10)
    got = cc.maps_build(Lx, Ly, seed, map0, 5, nthreads=3)
    for k in range(5):
        assert np.array_equal(got[k], oracle.map_build(Lx, Ly, seed, map0 + k)), k


def test_maps_do_not_depend_on_thread_count(cc):
    a = cc.maps_build(64, 48, 9, 0, 13, nthreads=1)
    for t in (2, 5, 0):
        assert np.array_equal(a, cc.maps_build(64, 48, 9, 0, 13, nthreads=t))


def test_map_builder_rejects_bad_arguments(cc):
    lib = cc.lib()
    buf = np.zeros(64, dtype=np.int32)
    ptr = buf.ctypes.data_as(__import__("ctypes").POINTER(__import__("ctypes").c_int32))
    assert lib.ccmc_maps_build(1, 8, 0, 0, 1, ptr, 1) == cc.E_INVAL
    assert lib.ccmc_maps_build(8, 8, 0, -1, 1, ptr, 1) == cc.E_INVAL
    assert lib.ccmc_maps_build(8, 8, 0, 0, -1, ptr, 1) == cc.E_INVAL
    assert lib.ccmc_maps_build(8, 8, 0, 0, 1, None, 1) == cc.E_INVAL
    assert lib.ccmc_maps_build(8, 8, 0, 0, 0, None, 1) == cc.OK
    assert lib.ccmc_map_size(1, 8) == cc.E_INVAL
