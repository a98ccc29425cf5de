"""The C ABI library loads on a machine without a GPU and exports every entry
point that include/*.h declares; its host-only threshold table equals the
oracle's bit for bit (both built with -ffp-contract=off, both calling libm exp).
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ccmc_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libccmc():
    import paper_2301_11735_gb300 as cc

    return cc.lib()


def test_library_exports_every_declared_symbol(libccmc):
    names = _declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(libccmc, n)]
    assert not missing, missing


@pytest.mark.parametrize("params", [(1.0, 0.5, 1.0, 1.0), (1 / 0.6, 0.2, 1.0, 0.5), (0.0, 1.0, 1.0, 1.0),
                                    (5.0, 0.0, 0.5, 1.0), (float("inf"), 1.0, 1.0, 1.0),
                                    (0.37, -0.5, 1.0, 1.0), (1 / 0.2, 0.0, 0.5, 1.0),
                                    (1 / 3.0, -1.0, 2.0, 1.0)])
def test_library_threshold_table_equals_oracle(params):
    import paper_2301_11735_gb300 as cc

    lib_t = cc.threshold_table(*params)
    ora = oracle.threshold_table(*params)  # dQ in [-2, 2], dBV, dBJ in [-24, 24]
    d = oracle.DB
    assert np.array_equal(lib_t, ora[[0, 2, 4]][:, d - 20:d + 21, d - 20:d + 21])


def test_invalid_arguments_are_rejected_without_a_gpu(libccmc):
    import paper_2301_11735_gb300 as cc

    out = np.zeros(cc.TABLE_N, dtype=np.uint32)
    ptr = out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    assert libccmc.ccmc_threshold_table(-1.0, 0.0, 0.0, 0.0, ptr) == cc.E_INVAL
    assert libccmc.ccmc_threshold_table(float("nan"), 0.0, 0.0, 0.0, ptr) == cc.E_INVAL
    h = ctypes.c_void_p()
    for Lx, Ly in [(6, 8), (8, 2), (0, 8), (4, 3)]:
        assert libccmc.ccmc_lattice_create(Lx, Ly, None, 0, ctypes.byref(h)) == cc.E_INVAL
    assert libccmc.ccmc_strerror(cc.E_BUDGET) == b"memory budget exhausted"
