"""Thermodynamics over a temperature grid: <E>, C(T) and susceptibilities with
error bars, from batched sweeps on the GPU.

The paper computes thermodynamic curves from the energy series of the chain
(the heat capacity from energy fluctuations, Sec. 2.2) and averages over
several copies of the lattice run in parallel (Sec. 3.2).  Here every
(temperature, replica) pair is one lattice of one ccmc batch: all lattices are
equilibrated together, then swept further with a record every `obs_every`
sweeps; each record holds the exact integer counts (Nc, BV, BJ, M, M_stag,
S_sum, S_stag).  Per temperature, with N sites and E = Delta Nc + V BV + (J/4) BJ:

    C       = (<E^2> - <E>^2) / (N T^2)
    chi     = (<M^2> - <|M|>^2) / (N T)             M = sum of sigma
    chi_s   = (<M_s^2> - <|M_s|>^2) / (N T)         M_s = staggered sum of sigma
    chi_c   = (<S_s^2> - <|S_s|>^2) / (N T)         S_s = staggered sum of S

The paper never defines its susceptibility; the forms above (fluctuations of
the order parameter's modulus, the usual choice on a finite lattice without a
field) are this library's reading.

Errors.  The records of one replica are correlated.  The Flyvbjerg-Petersen
blocking transformation (repeatedly averaging neighbouring pairs; J. Chem.
Phys. 91, 461 (1989)) gives the error of a mean and the block length past which
block means are independent.  Every estimate above is a function of pooled
means, so its error comes from a delete-one-block jackknife over the blocks of
all replicas, with blocks at least that long.  Only host arithmetic on the
record series happens here; the sweeps and the counts run in the library.
"""
from __future__ import annotations

import numpy as np

__all__ = ["blocking", "estimate", "thermodynamics"]


def blocking(x):
    """Flyvbjerg-Petersen blocking of a series: (mean, error of the mean,
    block length at which the error estimate reaches its plateau)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    if n < 2:
        return float(x.mean()) if n else float("nan"), float("nan"), 1
    mean = float(x.mean())
    levels = []
    y = x
    length = 1
    while len(y) >= 16:
        m = len(y)
        s2 = float(np.var(y)) / (m - 1)
        levels.append((np.sqrt(s2), np.sqrt(s2) / np.sqrt(2.0 * (m - 1)), length))
        y = 0.5 * (y[: m // 2 * 2 : 2] + y[1: m // 2 * 2 : 2])
        length *= 2
    if not levels:
        return mean, float(np.std(x, ddof=1) / np.sqrt(n)), 1
    # the first level whose successor does not exceed it by more than its own
    # statistical uncertainty: the estimate no longer grows with the block size
    for k in range(len(levels) - 1):
        sk, ek, lk = levels[k]
        if levels[k + 1][0] <= sk + ek:
            return mean, float(sk), int(lk)
    sk, _, lk = levels[-1]
    return mean, float(sk), int(lk)


def _columns(rec, N, T, Delta, V, J):
    rec = np.asarray(rec, dtype=np.float64)
    E = Delta * rec[:, 1] + V * rec[:, 2] + 0.25 * J * rec[:, 3]
    M, Ms, Ss = rec[:, 4], rec[:, 5], rec[:, 7]
    return np.stack([E, E * E, M * M, np.abs(M), Ms * Ms, np.abs(Ms), Ss * Ss, np.abs(Ss),
                     rec[:, 1]], axis=1)


def _derived(mu, N, T):
    E, E2, M2, Ma, Ms2, Msa, Ss2, Ssa, Nc = mu
    return np.array([E / N, (E2 - E * E) / (N * T * T), (M2 - Ma * Ma) / (N * T),
                     (Ms2 - Msa * Msa) / (N * T), (Ss2 - Ssa * Ssa) / (N * T), Nc / N])


_NAMES = ("E", "C", "chi", "chi_stag", "chi_charge", "Nc")


def estimate(records, N, T, Delta, V, J, min_blocks=8):
    """Estimates and errors at one temperature from the record series of one or
    more independent replicas (each an int64 array of rows (sweeps_done, Nc,
    BV, BJ, M, M_stag, S_sum, S_stag)).  Returns {name: (value, error)} for E
    (per site), C, chi, chi_stag, chi_charge and Nc (per site)."""
    cols = [_columns(r, N, T, Delta, V, J) for r in records if len(r)]
    if not cols:
        raise ValueError("no records")
    nmin = min(len(c) for c in cols)
    # block length: the longest plateau length of E and of the order
    # parameters over the replicas, capped so each replica keeps min_blocks
    blen = 1
    for c in cols:
        for j in (0, 2, 4, 6):
            blen = max(blen, blocking(c[:, j])[2])
    blen = max(1, min(blen, nmin // min_blocks))
    blocks = []
    for c in cols:
        nb = len(c) // blen
        blocks.append(c[: nb * blen].reshape(nb, blen, -1).mean(axis=1))
    B = np.concatenate(blocks, axis=0)  # equal-length blocks of every replica
    nb = len(B)
    total = B.sum(axis=0)
    full = _derived(total / nb, N, T)
    if nb < 2:
        return {k: (float(v), float("nan")) for k, v in zip(_NAMES, full)}
    jack = np.array([_derived((total - B[i]) / (nb - 1), N, T) for i in range(nb)])
    err = np.sqrt((nb - 1) / nb * np.sum((jack - jack.mean(axis=0)) ** 2, axis=0))
    return {k: (float(v), float(e)) for k, v, e in zip(_NAMES, full, err)}


def thermodynamics(L, temperatures, replicas=4, *, Delta, V, J, n=0.0, charged_frac=0.3,
                   counts=None, seed=1, equil_sweeps=2000, meas_sweeps=20000, obs_every=1,
                   Ly=None, batch_config=None):
    """Sweep an L x Ly lattice (Ly = L by default) at every temperature of the
    grid with `replicas` independent copies each, all in one ccmc batch, and
    return a dict of arrays over the grid: T and, for each estimate of
    `estimate`, its value and its error (key + "_err").

    The initial states are ccmc_init_constrained(seed_i, n, charged_frac), or
    ccmc_init_counts(seed_i, *counts) when counts = (n_plus, n_minus) is given;
    seed_i = seed + i over the lattices."""
    from . import Batch, Lattice

    Ly = L if Ly is None else Ly
    temps = [float(t) for t in temperatures]
    N = L * Ly
    nrec = meas_sweeps // obs_every
    lats = []
    try:
        for i in range(len(temps) * replicas):
            lat = Lattice(L, Ly, obs_capacity=max(nrec, 1) + 1)
            if counts is not None:
                lat.init_counts(seed + i, counts[0], counts[1])
            else:
                lat.init_constrained(seed + i, n, charged_frac)
            lats.append(lat)
        betas = [1.0 / t for t in temps for _ in range(replicas)]
        k = len(lats)
        with Batch(lats) as b:
            if batch_config is not None:
                b.config(*batch_config)
            b.sweep(equil_sweeps, betas, [Delta] * k, [V] * k, [J] * k, obs_every=0)
            b.sweep(meas_sweeps, betas, [Delta] * k, [V] * k, [J] * k, obs_every=obs_every)
            b.sync()
        series = [lat.obs_series(cap=nrec + 1) for lat in lats]
    finally:
        for lat in lats:
            lat.close()
    out = {"T": np.array(temps)}
    for name in _NAMES:
        out[name] = np.zeros(len(temps))
        out[name + "_err"] = np.zeros(len(temps))
    for ti, T in enumerate(temps):
        recs = series[ti * replicas:(ti + 1) * replicas]
        est = estimate(recs, N, T, Delta, V, J)
        for name, (v, e) in est.items():
            out[name][ti] = v
            out[name + "_err"][ti] = e
    return out
