"""Seeded synthetic workloads shaped like the paper's runs.

Shared by the tests, the benchmark and the serving examples.  This module holds
no arithmetic of the method: it only fixes lattice sizes, parameters, seeds
and request streams (numpy's seeded generator), and its output feeds both the
CUDA path and the oracle.

The paper measures on no public dataset; its runs span 4 x 4 to 256 x 256
lattices, 64 x 64 "drop" snapshots and several lattice copies (Sec. 3.3, 4, 5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Sim:
    """One independent simulation: lattice, parameters, seed and length."""
    Lx: int
    Ly: int
    seed: int
    n: float
    charged_frac: float
    T: float
    Delta: float
    V: float
    J: float
    nsweeps: int
    obs_every: int = 10

    @property
    def beta(self) -> float:
        return 1.0 / self.T

    @property
    def sites(self) -> int:
        return self.Lx * self.Ly


# 16 x 16, Delta = 0.5, V = J = 1, T = 1, 48 charges +1 / 16 charges -1 (n = 0.125)
SMALL_16 = dict(L=16, Delta=0.5, V=1.0, J=1.0, T=1.0, n_plus=48, n_minus=16, seed=1,
                nsweeps=2000, obs_every=1)


def temperature_sweep_4096(nsweeps: int = 10_000, obs_every: int = 10):
    """4096^2, Delta = 0, V = 0.5, J = 1, n = 0.1, charged fraction 0.3,
    T in {0.2, 0.5, 1.0, 2.0} with seeds 20..23."""
    return [Sim(4096, 4096, 20 + k, 0.1, 0.3, T, 0.0, 0.5, 1.0, nsweeps, obs_every)
            for k, T in enumerate((0.2, 0.5, 1.0, 2.0))]


def large_16384(nsweeps: int = 20_000, obs_every: int = 1):
    """16384^2 near the charge-ordering crossover: Delta = 0.2, V = 1, J = 0.5,
    n = 0.05, T = 0.6, seed 5."""
    return Sim(16384, 16384, 5, 0.05, 0.3, 0.6, 0.2, 1.0, 0.5, nsweeps, obs_every)


def replicas_512(seed: int = 3, nsweeps: int = 5000, count: int = 512):
    """512 independent lattices: L uniform in {32, 64, 128, 256}, T on a
    64-point grid of [0.1, 3.0], n in {0, 0.1, 0.2, 0.3}, Delta in
    {-0.5, 0, 0.5}, V = J = 1, seed 1000 + i."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice([32, 64, 128, 256], size=count)
    ns = rng.choice([0.0, 0.1, 0.2, 0.3], size=count)
    Ds = rng.choice([-0.5, 0.0, 0.5], size=count)
    Ts = np.linspace(0.1, 3.0, 64)
    return [Sim(int(Ls[i]), int(Ls[i]), 1000 + i, float(ns[i]), 0.3, float(Ts[i % 64]),
                float(Ds[i]), 1.0, 1.0, nsweeps, 0) for i in range(count)]


def request_stream(seed: int = 4, count: int = 2000, rate: float = 200.0,
                   L_range=(32, 2048), sweep_range=(1_000, 100_000)):
    """Poisson arrivals (mean `rate` per second) of simulations with L
    log-uniform in L_range (rounded to a multiple of 4), sweeps log-uniform in
    sweep_range, T ~ U[0.1, 3], n ~ U[0, 0.4], Delta ~ U[-1, 1], V ~ U[0, 2],
    J = 1.  Returns (arrival_times_s, sims)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sims = []
    for i in range(count):
        L = int(round(np.exp(rng.uniform(np.log(L_range[0]), np.log(L_range[1]))) / 4.0)) * 4
        L = max(L, 4)
        sw = int(round(np.exp(rng.uniform(np.log(sweep_range[0]), np.log(sweep_range[1])))))
        sims.append(Sim(L, L, 5000 + i, float(rng.uniform(0.0, 0.4)), 0.3,
                        float(rng.uniform(0.1, 3.0)), float(rng.uniform(-1.0, 1.0)),
                        float(rng.uniform(0.0, 2.0)), 1.0, sw, 0))
    return t, sims
