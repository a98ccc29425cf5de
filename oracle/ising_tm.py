"""Row transfer matrix of the two-dimensional Ising model on an L x L torus.

TEST INFRASTRUCTURE (part of the oracle package; pins the chain, not the GPU).

With Delta -> +infinity, no charges and an all-magnetic start, the model of
Eq. (3) keeps every site magnetic and reduces to E = (J/4) sum_<ij> sigma_i
sigma_j, the nearest-neighbour Ising model with coupling J/4.  Its partition
function on an L x L torus is Z = Tr(T^L) with the symmetric row matrix

    T[s, s'] = exp(-beta * (e_h(s) + e_v(s, s')))

over the 2^L spin rows s, where e_h is the energy of the L horizontal bonds of
row s and e_v that of the L vertical bonds between rows s and s'.  Writing
D = e_h + e_v (elementwise over [s, s']),
    dZ/dbeta   = -L Tr(T^(L-1) (D o T)),
    d2Z/dbeta2 =  L Tr(T^(L-1) (D^2 o T)) + L sum_{k=0}^{L-2} Tr(T^k (D o T) T^(L-2-k) (D o T)),
so <E> = -Z'/Z and <E^2> = Z''/Z exactly (up to float64 rounding).
"""
from __future__ import annotations

import numpy as np


def ising_moments(L: int, beta: float, J: float):
    """(<E>, <E^2>) of the Ising limit of Eq. (3) on an L x L torus."""
    n = 1 << L
    states = np.arange(n)
    spins = 1 - 2 * ((states[:, None] >> np.arange(L)[None, :]) & 1)  # +1 / -1
    K = 0.25 * J
    e_h = K * np.sum(spins * np.roll(spins, -1, axis=1), axis=1)
    e_v = K * spins @ spins.T
    # every row energy is shifted by s so the largest weight is 1; the moments
    # of the shifted total E - L s are converted back at the end
    s = (e_h[:, None] + e_v).min()
    D = e_h[:, None] + e_v - s
    T = np.exp(-beta * D)
    Dt = D * T
    D2t = D * D * T
    powers = [np.eye(n)]
    for _ in range(L):
        powers.append(powers[-1] @ T)
    Z = np.trace(powers[L])
    dZ = -L * np.trace(powers[L - 1] @ Dt)
    d2Z = L * np.trace(powers[L - 1] @ D2t)
    for k in range(L - 1):
        d2Z += L * np.trace(powers[k] @ Dt @ powers[L - 2 - k] @ Dt)
    m1, m2 = -dZ / Z, d2Z / Z
    return m1 + L * s, m2 + 2 * L * s * m1 + (L * s) ** 2


def ising_energy_and_heat(L: int, T: float, J: float):
    """<E>/N and C = (<E^2> - <E>^2) / (N T^2) (Sec. 2.2, k = 1)."""
    e1, e2 = ising_moments(L, 1.0 / T, J)
    N = L * L
    return e1 / N, (e2 - e1 * e1) / (N * T * T)


def onsager_tc(J: float) -> float:
    """Critical temperature of the infinite lattice for coupling |J|/4."""
    return 2.0 * (abs(J) / 4.0) / np.log(1.0 + np.sqrt(2.0))
