"""Closed-form averages of the constrained ensemble at infinite temperature.

TEST INFRASTRUCTURE (part of the oracle package; pins the chain, not the GPU).

At beta = 0 every state with sum_i S_i = Q (Eq. 2) has the same weight.  A state
with N+ charges +1, N- charges -1 and N0 = N - N+ - N- magnetic sites can be
placed in N! / (N+! N-! N0!) ways, each with 2^N0 spin choices, and
N+ - N- = Q.  Averages over that uniform measure:

* <Nc>   = sum over N- of (N+ + N-) * weight / total;
* <BV>   = 2N * (Q^2 - <Nc>) / (N (N - 1)): the measure is exchangeable, so for
  distinct sites E[S_i S_j] = (E[(sum S)^2] - E[sum S^2]) / (N (N - 1)), and the
  torus has 2N bonds, each between distinct sites when Lx, Ly >= 2;
* <BJ>   = 0 (flipping every spin maps the measure onto itself);
* <M^2>  = <N0> = N - <Nc> (independent +-1 spins on the magnetic sites).
Exact rationals are returned.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb


def _weights(N: int, Q: int):
    for n_minus in range(0, N + 1):
        n_plus = Q + n_minus
        if n_plus < 0 or n_plus + n_minus > N:
            continue
        n0 = N - n_plus - n_minus
        w = comb(N, n_plus) * comb(N - n_plus, n_minus) * (2 ** n0)
        yield n_plus, n_minus, n0, w


def count_states(N: int, Q: int) -> int:
    """Number of lattice states with charge sum Q."""
    return sum(w for *_, w in _weights(N, Q))


def beta0_averages(N: int, Q: int) -> dict:
    total = count_states(N, Q)
    nc = Fraction(sum((p + m) * w for p, m, _, w in _weights(N, Q)), total)
    bv = Fraction(2 * N) * (Fraction(Q * Q) - nc) / Fraction(N * (N - 1))
    return {"Nc": nc, "BV": bv, "BJ": Fraction(0), "M2": Fraction(N) - nc, "states": total}
