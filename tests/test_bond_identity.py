"""The bond-count identity the recount kernel completes BJ with.

Every site has two bonds (its right and its down neighbour) and so appears
in four bond ends; charged-charged bonds take two charged ends each and mixed
bonds one: 4 Nc = 2 nKK + n_mixed.  With 2N bonds in all, the magnetic-magnetic
bonds number nUU = 2N - 4 Nc + nKK on any periodic lattice -- 2-wide tori
included, where the two bonds between a pair of sites both count (the
multigraph convention of the oracle's recount).  The GPU recount counts nKK
and the sign-differing bonds and takes nUU from this identity; here it is
checked by brute force, and the resulting BJ against the oracle's recount
(Eq. 3), on random states.
"""
import numpy as np
import pytest

import oracle

SHAPES = [(2, 2), (2, 6), (5, 3), (4, 4), (7, 4), (8, 12), (64, 8), (16, 64)]


def _bonds(st):
    """(right, down) neighbour states of every site (periodic)."""
    return np.roll(st, -1, axis=1), np.roll(st, -1, axis=0)


@pytest.mark.parametrize("shape", SHAPES)
def test_magnetic_bond_count_from_charged_counts(shape):
    Lx, Ly = shape
    rng = np.random.default_rng(Lx * 100 + Ly)
    for _ in range(20):
        st = rng.integers(0, 4, size=(Ly, Lx), dtype=np.uint8)
        N = Lx * Ly
        charged = st >= 2  # codes 2, 3: S = +1, -1; codes 0, 1: magnetic
        Nc = int(charged.sum())
        nKK = nUU = nUUd = 0
        for nb in _bonds(st):
            nbc = nb >= 2
            nKK += int((charged & nbc).sum())
            mm = ~charged & ~nbc
            nUU += int(mm.sum())
            nUUd += int((mm & ((st & 1) != (nb & 1))).sum())  # sigma differs
        assert nUU == 2 * N - 4 * Nc + nKK
        # BJ = sum over magnetic-magnetic bonds of sigma sigma, from the identity
        bj = 2 * N - 4 * Nc + nKK - 2 * nUUd
        assert bj == int(oracle.recount(st)[2])
