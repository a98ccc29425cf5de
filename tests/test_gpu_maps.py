"""GPU parity of the paper-faithful map mode (Sec. 3.2): host-built maps applied
by the device kernel, one thread per pair, against the oracle's map chain --
bit-exact lattices and observables.  Small lattices give many maps whose
partner is a nearest neighbour of a (the near move table); the ragged shapes
have row tails shorter than a packed word."""
import numpy as np
import pytest

import oracle

from .gpu_util import first_difference

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4), (8, 8), (12, 20), (64, 64), (68, 20), (260, 36), (1024, 1024)]
PARAMS = [(1.0, 0.5, 1.0, 1.0), (4.0, -0.5, 1.0, 1.0), (1 / 3.0, 0.2, 2.0, 0.5),
          (0.0, 0.0, 1.0, 1.0)]


@pytest.fixture(scope="module")
def cc():
    import paper_2301_11735_gb300 as cc

    return cc


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("params", PARAMS)
def test_map_apply_is_bit_exact(cc, shape, params):
    Lx, Ly = shape
    beta, Delta, V, J = params
    seed = 1000 + Lx + 7 * Ly
    nmaps = 40 if Lx * Ly <= 4096 else 4
    maps = cc.maps_build(Lx, Ly, seed, 3, nmaps)
    exp = oracle.init_constrained(Lx, Ly, seed, 0.1, 0.3)
    with cc.Lattice(Lx, Ly) as lat:
        lat.init_constrained(seed, 0.1, 0.3)
        half = nmaps // 2
        lat.map_apply(maps[:half], 3, beta, Delta, V, J)
        lat.map_apply(maps[half:], 3 + half, beta, Delta, V, J)
        got = lat.get_state()
        obs = lat.observables()
    oracle.map_sweeps(exp, seed, 3, nmaps, beta, Delta, V, J)
    assert np.array_equal(got, exp), (shape, params, first_difference(got, exp))
    r = oracle.recount(exp)
    assert [obs[k] for k in ("Nc", "BV", "BJ", "M", "M_stag", "S_sum", "S_stag")] == list(r)


def test_maps_and_colour_sweeps_interleave(cc):
    Lx, Ly, seed = 36, 44, 21
    beta, Delta, V, J = 1.5, 0.3, 1.0, 1.0
    maps = cc.maps_build(Lx, Ly, seed, 0, 6)
    exp = oracle.init_constrained(Lx, Ly, seed, 0.05, 0.3)
    with cc.Lattice(Lx, Ly) as lat:
        lat.init_constrained(seed, 0.05, 0.3)
        lat.sweep(2, beta, Delta, V, J)
        lat.map_apply(maps[:4], 0, beta, Delta, V, J)
        lat.sweep(3, beta, Delta, V, J)  # the colour phases continue at sweep 2
        lat.map_apply(maps[4:], 4, beta, Delta, V, J)
        got = lat.get_state()
    oracle.sweeps(exp, seed, 0, 2, beta, Delta, V, J)
    oracle.map_sweeps(exp, seed, 0, 4, beta, Delta, V, J)
    oracle.sweeps(exp, seed, 2, 3, beta, Delta, V, J)
    oracle.map_sweeps(exp, seed, 4, 2, beta, Delta, V, J)
    assert np.array_equal(got, exp), first_difference(got, exp)


def test_map_apply_rejects_bad_maps(cc):
    with cc.Lattice(16, 16) as lat:
        with pytest.raises(cc.CcmcError):
            lat.map_apply(np.zeros((1, 25, 2), dtype=np.int32), 0, 1.0, 0.0, 1.0, 1.0)  # not initialised
        lat.init_constrained(3, 0.1)
        before = lat.get_state()
        bad = cc.maps_build(16, 16, 3, 0, 2)
        bad[1, 5, 1] = 256  # outside the lattice
        with pytest.raises(cc.CcmcError):
            lat.map_apply(bad, 0, 1.0, 0.0, 1.0, 1.0)
        bad[1, 5, 1] = -1
        with pytest.raises(cc.CcmcError):
            lat.map_apply(bad, 0, 1.0, 0.0, 1.0, 1.0)
        with pytest.raises(cc.CcmcError):
            lat.map_apply(cc.maps_build(16, 16, 3, 0, 1), 0, -1.0, 0.0, 1.0, 1.0)
        assert np.array_equal(lat.get_state(), before)
