"""Pins of the colour schedule (the "map" of Sec. 3.2, drawn per phase).

A phase is the set of pairs (a, a + r) over one residue class a = a0 (mod 4).
The paper's requirement for a map is that its pairs do not interact: no site
of one pair is, or neighbours, a site of another pair.  Brute force over every
class and every offset of small tori must find exactly the oracle's allowed
offset set.  The draws must be uniform, and on the 4 x 4 torus a phase must be
one uniformly random ordered pair -- the paper's serial algorithm.
"""
import numpy as np
import pytest

import oracle


def _phase_pairs(Lx, Ly, a0x, a0y, rx, ry):
    pairs = []
    for j in range(Ly // 4):
        for i in range(Lx // 4):
            ax, ay = 4 * i + a0x, 4 * j + a0y
            bx, by = (ax + rx) % Lx, (ay + ry) % Ly
            pairs.append((ay * Lx + ax, by * Lx + bx))
    return pairs


def _closed_nbhd(Lx, Ly, s):
    x, y = s % Lx, s // Lx
    return {s, y * Lx + (x - 1) % Lx, y * Lx + (x + 1) % Lx, ((y - 1) % Ly) * Lx + x,
            ((y + 1) % Ly) * Lx + x}


def _independent(Lx, Ly, pairs):
    owner = {}
    for p, (a, b) in enumerate(pairs):
        if a == b:
            return False
        for s in (a, b):
            if s in owner:
                return False
            owner[s] = p
    for p, (a, b) in enumerate(pairs):
        for s in _closed_nbhd(Lx, Ly, a) | _closed_nbhd(Lx, Ly, b):
            if owner.get(s, p) != p:
                return False
    return True


@pytest.mark.parametrize("shape", [(4, 4), (8, 8), (12, 12), (4, 8), (8, 12), (16, 4), (16, 16)])
def test_allowed_offsets_are_exactly_the_independent_ones(shape):
    Lx, Ly = shape
    classes = [(x, y) for y in range(4) for x in range(4)]
    if Lx * Ly > 144:
        classes = [(0, 0), (3, 1), (2, 3)]
    for ry in range(Ly):
        for rx in range(Lx):
            allowed = oracle.offset_allowed(Lx, Ly, rx, ry)
            for a0x, a0y in classes:
                ind = _independent(Lx, Ly, _phase_pairs(Lx, Ly, a0x, a0y, rx, ry))
                assert ind == allowed, (shape, rx, ry, a0x, a0y)


def test_schedule_draws_are_uniform():
    Lx = Ly = 8
    allowed = [(rx, ry) for ry in range(Ly) for rx in range(Lx)
               if oracle.offset_allowed(Lx, Ly, rx, ry)]
    index = {r: t for t, r in enumerate(allowed)}
    n = 30000
    cls = np.zeros(16)
    off = np.zeros(len(allowed))
    for P in range(n):
        a0x, a0y, rx, ry = oracle.schedule(Lx, Ly, 4242, P)
        cls[a0y * 4 + a0x] += 1
        off[index[(rx, ry)]] += 1
    for h in (cls, off):
        e = n / len(h)
        chi2 = float(np.sum((h - e) ** 2 / e))
        dof = len(h) - 1
        assert chi2 < dof + 6 * np.sqrt(2 * dof), chi2


def test_4x4_phase_is_one_uniform_random_pair():
    n = 48000
    hist = np.zeros((16, 16))
    for P in range(n):
        a0x, a0y, rx, ry = oracle.schedule(4, 4, 7, P)
        (a, b), = _phase_pairs(4, 4, a0x, a0y, rx, ry)
        hist[a, b] += 1
    assert np.all(np.diag(hist) == 0)
    h = hist[~np.eye(16, dtype=bool)]
    e = n / 240
    chi2 = float(np.sum((h - e) ** 2 / e))
    assert chi2 < 239 + 6 * np.sqrt(2 * 239), chi2


def test_schedule_depends_on_seed_and_phase():
    a = [oracle.schedule(64, 64, 1, P) for P in range(50)]
    b = [oracle.schedule(64, 64, 2, P) for P in range(50)]
    assert len(set(a)) > 45 and a != b
    assert all(oracle.offset_allowed(64, 64, r[2], r[3]) for r in a + b)
