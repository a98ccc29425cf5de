"""CPU oracle for the charge-conserving coupled-pair Metropolis method.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library (``paper_2301_11735_gb300``) never imports it and
shares no code with it; the two must agree bit for bit.

The heavy lifting is plain single-threaded C (``ccmc_oracle.c``); this module
only marshals numpy arrays.  Exact references used to pin the oracle live beside
it: ``exact_enum.c`` (enumeration on tiny lattices), ``closed_forms.py``
(infinite-temperature averages) and ``ising_tm.py`` (transfer matrix of the
Ising limit).

Lattices are ``uint8`` arrays of shape (Ly, Lx), codes 0: s=+1/2, 1: s=-1/2,
2: S=+1, 3: S=-1.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_uint32, c_uint64

import numpy as np

from . import build as _build

TAG_SCHED, TAG_MOVE, TAG_SLOW, TAG_FEISTEL, TAG_SIGN, TAG_SEQ, TAG_SEQSLOW = 1, 2, 3, 4, 5, 6, 7
DB = 24
NB = 2 * DB + 1
TABLE_SIZE = 5 * NB * NB
REC = 8
REC_FIELDS = ("sweeps_done", "Nc", "BV", "BJ", "M", "M_stag", "S_sum", "S_stag")

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p, u8p, i64p = POINTER(c_uint32), POINTER(ctypes.c_uint8), POINTER(c_int64)
        ip, i32p = POINTER(c_int), POINTER(c_int32)
        sig = {
            "oracle_philox4x32_10": (None, [u32p, u32p, u32p]),
            "oracle_philox_block": (None, [u32p, u32p, c_int64, u32p]),
            "oracle_charge_counts": (c_int, [c_int64, c_double, c_double, i64p, i64p, i64p]),
            "oracle_feistel_rank": (c_int64, [c_uint64, c_int64, c_int64]),
            "oracle_init_counts": (c_int, [c_int, c_int, c_uint64, c_int64, c_int64, u8p]),
            "oracle_threshold_table": (None, [c_double, c_double, c_double, c_double, u32p]),
            "oracle_table_index": (c_int, [c_int, c_int, c_int]),
            "oracle_offset_allowed": (c_int, [c_int, c_int, c_int, c_int]),
            "oracle_schedule": (None, [c_int, c_int, c_uint64, c_uint64, ip, ip, ip, ip]),
            "oracle_pair_delta": (None, [u8p, c_int, c_int, c_int, c_int, c_int, c_int, ip]),
            "oracle_site_delta": (None, [u8p, c_int, c_int, c_int, c_int, ip]),
            "oracle_pair_move": (c_int, [u8p, c_int, c_int, c_int, c_int, c_uint32, u32p, u32p,
                                         u32p]),
            "oracle_recount": (None, [u8p, c_int, c_int, i64p]),
            "oracle_phase": (None, [u8p, c_int, c_int, c_uint64, c_uint64, u32p]),
            "oracle_sweeps": (c_int64, [u8p, c_int, c_int, c_uint64, c_int64, c_int64, c_double,
                                        c_double, c_double, c_double, c_int, i64p]),
            "oracle_sequential_sweeps": (c_int64, [u8p, c_int, c_int, c_uint64, c_int64, c_int64,
                                                   c_double, c_double, c_double, c_double, c_int,
                                                   i64p]),
            "oracle_neighbour_sweeps": (c_int64, [u8p, c_int, c_int, c_uint64, c_int64, c_int64,
                                                  c_double, c_double, c_double, c_double, c_int,
                                                  i64p]),
            "oracle_map_size": (c_int64, [c_int, c_int]),
            "oracle_map_build": (c_int, [c_int, c_int, c_uint64, c_int64, i32p]),
            "oracle_map_sweeps": (c_int64, [u8p, c_int, c_int, c_uint64, c_int64, c_int64,
                                            c_double, c_double, c_double, c_double, c_int, i64p]),
            "oracle_penalty_sweeps": (c_int64, [u8p, c_int, c_int, c_uint64, c_int64, c_int64,
                                                c_double, c_double, c_double, c_double, c_double,
                                                POINTER(c_double), c_double, c_int, i64p,
                                                POINTER(c_double)]),
            "oracle_enumerate": (c_int64, [c_int, c_int, c_int, i64p, i64p, i64p, i64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(POINTER(ct))


def _u8(st):
    assert st.dtype == np.uint8 and st.flags.c_contiguous
    return _p(st, ctypes.c_uint8)


def seed_key(seed: int):
    seed &= (1 << 64) - 1
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c, c_uint32), _p(k, c_uint32), _p(out, c_uint32))
    return out


def philox_block(ctr, key, count: int) -> np.ndarray:
    """(count, 4) outputs for counters (ctr[0] + i mod 2^32, ctr[1], ctr[2], ctr[3])."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4 * count, dtype=np.uint32)
    lib().oracle_philox_block(_p(c, c_uint32), _p(k, c_uint32), count, _p(out, c_uint32))
    return out.reshape(count, 4)


def charge_counts(N: int, n: float, c: float = 0.3):
    """(Q, N+, N-) from density n and charged fraction c; None if infeasible."""
    Q, npl, nmi = c_int64(), c_int64(), c_int64()
    r = lib().oracle_charge_counts(N, n, c, ctypes.byref(Q), ctypes.byref(npl), ctypes.byref(nmi))
    return None if r != 0 else (Q.value, npl.value, nmi.value)


def feistel_rank(seed: int, N: int, i: int) -> int:
    return lib().oracle_feistel_rank(seed & ((1 << 64) - 1), N, i)


def init_counts(Lx: int, Ly: int, seed: int, n_plus: int, n_minus: int) -> np.ndarray:
    st = np.zeros((Ly, Lx), dtype=np.uint8)
    r = lib().oracle_init_counts(Lx, Ly, seed & ((1 << 64) - 1), n_plus, n_minus, _u8(st))
    if r != 0:
        raise ValueError("infeasible charge counts")
    return st


def init_constrained(Lx: int, Ly: int, seed: int, n: float, c: float = 0.3) -> np.ndarray:
    cc = charge_counts(Lx * Ly, n, c)
    if cc is None:
        raise ValueError("infeasible (n, c)")
    return init_counts(Lx, Ly, seed, cc[1], cc[2])


def threshold_table(beta: float, Delta: float, V: float, J: float) -> np.ndarray:
    """uint32 table of shape (5, NB, NB) indexed [dQ + 2, dBV + DB, dBJ + DB]."""
    t = np.zeros(TABLE_SIZE, dtype=np.uint32)
    lib().oracle_threshold_table(beta, Delta, V, J, _p(t, c_uint32))
    return t.reshape(5, NB, NB)


def offset_allowed(Lx: int, Ly: int, rx: int, ry: int) -> bool:
    return bool(lib().oracle_offset_allowed(Lx, Ly, rx, ry))


def schedule(Lx: int, Ly: int, seed: int, P: int):
    """(a0x, a0y, rx, ry) of global phase P."""
    v = [c_int() for _ in range(4)]
    lib().oracle_schedule(Lx, Ly, seed & ((1 << 64) - 1), P, *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def pair_delta(st: np.ndarray, a: int, b: int, na: int, nb: int):
    Ly, Lx = st.shape
    out = (c_int * 3)()
    lib().oracle_pair_delta(_u8(st), Lx, Ly, a, b, na, nb, out)
    return tuple(out)


def site_delta(st: np.ndarray, a: int, nc: int):
    """(dNc, dBV, dBJ) of Eq. 3 when site a alone takes code nc."""
    Ly, Lx = st.shape
    out = (c_int * 3)()
    lib().oracle_site_delta(_u8(st), Lx, Ly, a, nc, out)
    return tuple(out)


def pair_move(st: np.ndarray, a: int, b: int, R: int, key, slow_ctr, table) -> int:
    """One move; R = 16-bit choice | top half of the acceptance word << 16."""
    Ly, Lx = st.shape
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    c = np.ascontiguousarray(np.asarray(slow_ctr, dtype=np.uint32))
    t = np.ascontiguousarray(table.reshape(-1), dtype=np.uint32)
    return lib().oracle_pair_move(_u8(st), Lx, Ly, a, b, R & 0xFFFFFFFF, _p(k, c_uint32),
                                  _p(c, c_uint32), _p(t, c_uint32))


def recount(st: np.ndarray) -> np.ndarray:
    """int64[7]: Nc, BV, BJ, M, M_stag, S_sum, S_stag."""
    Ly, Lx = st.shape
    out = np.zeros(7, dtype=np.int64)
    lib().oracle_recount(_u8(st), Lx, Ly, _p(out, c_int64))
    return out


def phase(st: np.ndarray, seed: int, P: int, table) -> None:
    Ly, Lx = st.shape
    t = np.ascontiguousarray(table.reshape(-1), dtype=np.uint32)
    lib().oracle_phase(_u8(st), Lx, Ly, seed & ((1 << 64) - 1), P, _p(t, c_uint32))


def sweeps(st: np.ndarray, seed: int, sweep0: int, nsweeps: int, beta: float, Delta: float,
           V: float, J: float, obs_every: int = 0, sequential: bool = False,
           neighbour: bool = False) -> np.ndarray:
    """Advance ``st`` in place; returns the int64 records (rows of REC_FIELDS).

    Default: the colour-phase chain.  ``sequential``: one uniformly random
    ordered pair per move.  ``neighbour``: the short-range negative control
    (partner among a's four nearest neighbours)."""
    Ly, Lx = st.shape
    nrec_max = nsweeps // obs_every + 1 if obs_every > 0 else 0
    rec = np.zeros((max(nrec_max, 1), REC), dtype=np.int64)
    if neighbour:
        fn = lib().oracle_neighbour_sweeps
    else:
        fn = lib().oracle_sequential_sweeps if sequential else lib().oracle_sweeps
    n = fn(_u8(st), Lx, Ly, seed & ((1 << 64) - 1), sweep0, nsweeps, beta, Delta, V, J,
           obs_every, _p(rec, c_int64))
    if n < 0:
        raise MemoryError("oracle allocation failed")
    return rec[:n]


def map_size(Lx: int, Ly: int) -> int:
    """Pairs per paper map: max(1, floor(N / 10))."""
    return int(lib().oracle_map_size(Lx, Ly))


def map_build(Lx: int, Ly: int, seed: int, m: int) -> np.ndarray:
    """Map m of the paper's random-marking algorithm: (P, 2) site indices."""
    P = map_size(Lx, Ly)
    out = np.zeros((P, 2), dtype=np.int32)
    if lib().oracle_map_build(Lx, Ly, seed & ((1 << 64) - 1), m, _p(out, c_int32)) != 0:
        raise MemoryError("oracle allocation failed")
    return out


def map_sweeps(st: np.ndarray, seed: int, map0: int, nmaps: int, beta: float, Delta: float,
               V: float, J: float, obs_every: int = 0) -> np.ndarray:
    """Apply paper maps map0 .. map0 + nmaps - 1 to ``st`` in place; records
    after every obs_every-th map (sweeps_done = maps done)."""
    Ly, Lx = st.shape
    nrec_max = nmaps // obs_every + 1 if obs_every > 0 else 0
    rec = np.zeros((max(nrec_max, 1), REC), dtype=np.int64)
    n = lib().oracle_map_sweeps(_u8(st), Lx, Ly, seed & ((1 << 64) - 1), map0, nmaps, beta,
                                Delta, V, J, obs_every, _p(rec, c_int64))
    if n < 0:
        raise MemoryError("oracle allocation failed")
    return rec[:n]


def penalty_sweeps(st: np.ndarray, seed: int, sweep0: int, nsweeps: int, beta: float,
                   Delta: float, V: float, J: float, n: float, mu: float, kappa: float,
                   obs_every: int = 1):
    """Penalty-function baseline (Sec. 2.2) on ``st`` in place: single-site
    Metropolis with -mu sum S, mu adjusted after every sweep.  Returns
    (records, mu after every sweep)."""
    Ly, Lx = st.shape
    nrec_max = nsweeps // obs_every + 1 if obs_every > 0 else 0
    rec = np.zeros((max(nrec_max, 1), REC), dtype=np.int64)
    trace = np.zeros(max(nsweeps, 1), dtype=np.float64)
    m = c_double(mu)
    k = lib().oracle_penalty_sweeps(_u8(st), Lx, Ly, seed & ((1 << 64) - 1), sweep0, nsweeps,
                                    beta, Delta, V, J, n, ctypes.byref(m), kappa, obs_every,
                                    _p(rec, c_int64), _p(trace, c_double))
    return rec[:k], trace[:nsweeps]


def enumerate_dos(Lx: int, Ly: int, Q: int):
    """Exact histogram over (Nc, BV, BJ) of all states with charge sum Q."""
    N = Lx * Ly
    shape = (N + 1, 4 * N + 1, 4 * N + 1)
    arrs = [np.zeros(shape, dtype=np.int64) for _ in range(4)]
    n = lib().oracle_enumerate(Lx, Ly, Q, *[_p(a, c_int64) for a in arrs])
    if n < 0:
        raise ValueError("unsupported shape for enumeration")
    return n, arrs[0], arrs[1], arrs[2], arrs[3]
