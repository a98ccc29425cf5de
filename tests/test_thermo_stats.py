"""Pins of the thermodynamics estimators (paper_2301_11735_gb300.thermo), which
need no GPU: the blocking error against series with known errors, and the
estimates of E, C, chi and Nc from oracle-chain records against exact 4 x 4
enumeration (the paper's own test, Sec. 3.3)."""
import numpy as np
import pytest

import oracle
from paper_2301_11735_gb300.thermo import blocking, estimate

from .test_oracle_physics import exact_dos


def test_blocking_of_independent_samples():
    rng = np.random.default_rng(1)
    for n in (1 << 12, 1 << 16):
        x = rng.normal(3.0, 2.0, size=n)
        mean, err, blen = blocking(x)
        assert abs(err - 2.0 / np.sqrt(n)) < 0.15 * 2.0 / np.sqrt(n)
        assert blen <= 4
        assert abs(mean - 3.0) < 5 * err


@pytest.mark.parametrize("phi", [0.5, 0.9, 0.97])
def test_blocking_of_an_autoregressive_series(phi):
    # x_t = phi x_{t-1} + e_t: var x = 1/(1 - phi^2), and the error of the
    # mean of n samples is sqrt(var x (1 + phi) / (1 - phi) / n)
    rng = np.random.default_rng(int(phi * 100))
    n = 1 << 18
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    true = np.sqrt((1 + phi) / (1 - phi) / (1 - phi * phi) / n)
    _, err, blen = blocking(x)
    assert abs(err - true) < 0.2 * true, (err, true)
    assert blen >= (1 + phi) / (1 - phi)  # blocks longer than the correlation time


def _exact(Q, T, Delta, V, J):
    _, count, m2, mabs, _ = exact_dos(4, 4, Q)
    N = 16
    nc = np.arange(N + 1)[:, None, None]
    bv = (np.arange(4 * N + 1) - 2 * N)[None, :, None]
    bj = (np.arange(4 * N + 1) - 2 * N)[None, None, :]
    E = Delta * nc + V * bv + 0.25 * J * bj
    mask = count > 0
    w = np.where(mask, np.exp(-(E - E[mask].min()) / T), 0.0)
    Z = np.sum(w * count)
    e1, e2 = np.sum(w * count * E) / Z, np.sum(w * count * E * E) / Z
    M2, Ma = np.sum(w * m2) / Z, np.sum(w * mabs) / Z
    return {"E": e1 / N, "C": (e2 - e1 * e1) / (N * T * T), "chi": (M2 - Ma * Ma) / (N * T),
            "Nc": np.sum(w * count * nc) / Z / N}


@pytest.mark.parametrize("T", [0.25, 0.6, 1.6])
def test_estimates_from_oracle_records_match_exact_4x4(T):
    Q, Delta, V, J = 2, -0.5, 1.0, 1.0
    recs = []
    for r in range(4):
        st = oracle.init_counts(4, 4, 100 + r, 5, 3)
        recs.append(oracle.sweeps(st, 100 + r, 0, 60000, 1.0 / T, Delta, V, J,
                                  obs_every=1)[2000:])
    est = estimate(recs, 16, T, Delta, V, J)
    ex = _exact(Q, T, Delta, V, J)
    for k in ("E", "C", "chi", "Nc"):
        v, e = est[k]
        assert e > 0
        assert abs(v - ex[k]) <= 4 * e + 1e-9, (k, v, ex[k], e)
