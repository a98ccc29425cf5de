"""Helpers shared by the GPU parity tests."""
import numpy as np

import oracle


def oracle_run(st, seed, sweep0, nsweeps, beta, Delta, V, J, obs_every=1):
    st = st.copy()
    rec = oracle.sweeps(st, seed, sweep0, nsweeps, beta, Delta, V, J, obs_every=obs_every)
    return st, rec


def first_difference(a, b):
    d = np.argwhere(a != b)
    return None if len(d) == 0 else (tuple(d[0]), int(a[tuple(d[0])]), int(b[tuple(d[0])]),
                                     len(d))
