"""ccmc_recount_noalloc: observables of a caller-owned device lattice computed
without any allocation by the library (its scratch is a fixed static array).

Meant for callers that cannot let a library allocate device memory during a
call -- a server holding a pre-reserved memory budget, or a latency-critical
path that must not pay for cudaMalloc/cudaFree.  Checked through the C ABI
against ccmc_observables on the same states, exactly (integer counts), on two
calls in a row so that the reused scratch is exercised.  Collected last so that
a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

FIELDS = ("Nc", "BV", "BJ", "M", "M_stag", "S_sum", "S_stag")


def _fn(cc):
    f = cc.lib().ccmc_recount_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return f


@pytest.mark.parametrize("shape", [(16, 16), (68, 20), (4096, 4096)])
def test_noalloc_recount_matches_observables_twice(shape):
    torch = pytest.importorskip("torch")
    import paper_2301_11735_gb300 as cc

    Lx, Ly = shape
    fn = _fn(cc)
    out = torch.zeros(7, dtype=torch.int64, device="cuda")
    with cc.Lattice(Lx, Ly) as lat:
        for call, seed in enumerate((3, 4)):
            lat.init_constrained(seed, 0.1, 0.3)
            lat.sweep(2, 1.0, 0.3, 1.0, 1.0)
            ref = lat.observables()
            st = torch.from_numpy(lat.get_state()).cuda()
            rc = fn(st.data_ptr(), Lx, Ly, out.data_ptr(), None)
            assert rc == cc.OK, (call, rc)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert list(got) == [ref[k] for k in FIELDS], (call, shape)
            if Lx * Ly <= 4096:
                assert list(got) == list(oracle.recount(lat.get_state()))


@pytest.mark.parametrize("shape", [(2, 6), (5, 3), (7, 4), (2, 2), (3, 9)])
def test_noalloc_recount_of_shapes_the_sweep_does_not_take(shape):
    """Odd widths and 2-wide tori (which ccmc_lattice_create rejects) follow
    Eq. 3 by definition: the 2N right and down bonds, both bonds counted where
    a 2-wide torus joins the same two sites twice, the staggered sign (x + y)
    mod 2 wrapping across an odd seam.  Compared with the oracle's recount of
    uniformly random site codes, exactly, on two calls in a row."""
    torch = pytest.importorskip("torch")
    import paper_2301_11735_gb300 as cc

    Lx, Ly = shape
    fn = _fn(cc)
    out = torch.zeros(7, dtype=torch.int64, device="cuda")
    rng = np.random.default_rng(7 * Lx + Ly)
    for call in range(2):
        host = rng.integers(0, 4, size=(Ly, Lx), dtype=np.uint8)
        st = torch.from_numpy(host.reshape(-1).copy()).cuda()
        rc = fn(st.data_ptr(), Lx, Ly, out.data_ptr(), None)
        assert rc == cc.OK, (call, rc)
        torch.cuda.synchronize()
        assert list(out.cpu().numpy()) == list(oracle.recount(host)), (call, shape)


def test_noalloc_recount_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    import paper_2301_11735_gb300 as cc

    fn = _fn(cc)
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(7, dtype=torch.int64, device="cuda")
    assert fn(None, 8, 8, out.data_ptr(), None) == cc.E_INVAL
    assert fn(buf.data_ptr(), 8, 8, None, None) == cc.E_INVAL
    assert fn(buf.data_ptr(), 1, 8, out.data_ptr(), None) == cc.E_INVAL
    assert fn(buf.data_ptr(), 1 << 16, 1 << 15, out.data_ptr(), None) == cc.E_INVAL
