"""Error bars for Monte Carlo time series (batch means).

A series is cut into B equal consecutive batches; the batch means are close to
independent when a batch is much longer than the autocorrelation time, so the
standard error of the overall mean is std(batch means) / sqrt(B).  For the heat
capacity each batch gives its own fluctuation estimate
C_b = (<E^2>_b - <E>_b^2) / (N T^2) (Sec. 2.2) and the same rule applies.
"""
import numpy as np


def batch_mean(x, nbatch=40):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbatch * nbatch
    b = x[:n].reshape(nbatch, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbatch))


def batch_heat(E, N, T, nbatch=40):
    E = np.asarray(E, dtype=np.float64)
    n = len(E) // nbatch * nbatch
    b = E[:n].reshape(nbatch, -1)
    c = b.var(axis=1) / (N * T * T)
    return float(c.mean()), float(c.std(ddof=1) / np.sqrt(nbatch))


def energy(rec, Delta, V, J):
    """E = Delta Nc + V BV + (J/4) BJ from integer record columns (Eq. 3)."""
    rec = np.asarray(rec)
    return Delta * rec[:, 1] + V * rec[:, 2] + 0.25 * J * rec[:, 3]
