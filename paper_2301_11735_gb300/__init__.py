"""Python binding of libccmc: the charge-conserving coupled-pair Metropolis
sweep (Budrin et al.) on one GB300.

Argument marshalling only: every step of the method runs in the CUDA kernels of
``libccmc.so`` behind the C ABI of ``include/ccmc.h``.  The library must have
been built (``__graft_entry__.build()`` or ``python -m
paper_2301_11735_gb300.build``); the first call into the package raises
ImportError when it is missing -- there is no CPU fallback.

Site codes of every host array: 0: s=+1/2, 1: s=-1/2, 2: S=+1, 3: S=-1, as a
``uint8`` array of shape (Ly, Lx).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int64, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libccmc.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_BUDGET, E_STATE, E_NOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
PENDING = 1
TABLE_N = 3 * 41 * 41
OBS_FIELDS = ("sweeps_done", "Nc", "BV", "BJ", "M", "M_stag", "S_sum", "S_stag", "E")


class CcmcError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {lib().ccmc_strerror(code).decode()} ({code})")
        self.code = code


class Obs(ctypes.Structure):
    _fields_ = [(n, c_int64) for n in OBS_FIELDS[:-1]] + [("E", c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n in OBS_FIELDS}


class Request(ctypes.Structure):
    _fields_ = [("Lx", c_int), ("Ly", c_int), ("seed", c_uint64), ("n", c_double),
                ("charged_frac", c_double), ("nsweeps", c_int64), ("beta", c_double),
                ("Delta", c_double), ("V", c_double), ("J", c_double), ("obs_every", c_int),
                ("state_out", c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", c_int), ("final_obs", Obs), ("site_updates", c_int64),
                ("submit_s", c_double), ("start_s", c_double), ("done_s", c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k in ("status", "site_updates", "submit_s", "start_s",
                                            "done_s")}
        d["final_obs"] = self.final_obs.as_dict()
        return d


class ServerStats(ctypes.Structure):
    _fields_ = [(k, c_int64) for k in ("submitted", "queued", "active", "completed", "rejected",
                                       "failed", "slices", "site_updates", "bytes_in_use")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
            "(the package has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64p, u32p, u8p = c_void_p, POINTER(c_int64), POINTER(c_uint32), POINTER(ctypes.c_uint8)
    sigs = {
        "ccmc_strerror": (ctypes.c_char_p, [c_int]),
        "ccmc_threshold_table": (c_int, [c_double, c_double, c_double, c_double, u32p]),
        "ccmc_lattice_create": (c_int, [c_int, c_int, vp, c_int64, POINTER(vp)]),
        "ccmc_lattice_destroy": (c_int, [vp]),
        "ccmc_init_constrained": (c_int, [vp, c_uint64, c_double, c_double]),
        "ccmc_init_counts": (c_int, [vp, c_uint64, c_int64, c_int64]),
        "ccmc_sweep": (c_int, [vp, c_int64, c_double, c_double, c_double, c_double, c_int]),
        "ccmc_phases": (c_int, [vp, c_int64, c_double, c_double, c_double, c_double]),
        "ccmc_observables": (c_int, [vp, POINTER(Obs)]),
        "ccmc_obs_series": (c_int, [vp, POINTER(Obs), c_int64, i64p]),
        "ccmc_hist_enable": (c_int, [vp, c_int]),
        "ccmc_hist_get": (c_int, [vp, i64p]),
        "ccmc_get_state": (c_int, [vp, u8p]),
        "ccmc_set_state": (c_int, [vp, u8p, c_uint64, c_int64]),
        "ccmc_get_state_packed": (c_int, [vp, u8p]),
        "ccmc_set_state_packed": (c_int, [vp, u8p, c_uint64, c_int64]),
        "ccmc_sync": (c_int, [vp]),
        "ccmc_philox_device": (c_int, [c_uint32] * 6 + [c_int64, u32p]),
        "ccmc_selftest_wait": (c_int, [c_uint32]),
        "ccmc_peak_smem_read": (c_int, [POINTER(c_double)]),
        "ccmc_peak_l2_read": (c_int, [c_int64, POINTER(c_double)]),
        "ccmc_batch_create": (c_int, [c_int, POINTER(vp), vp, POINTER(vp)]),
        "ccmc_batch_destroy": (c_int, [vp]),
        "ccmc_batch_config": (c_int, [vp, c_int, c_int64, c_int, c_int]),
        "ccmc_batch_sweep": (c_int, [vp, i64p, POINTER(c_double), POINTER(c_double),
                                     POINTER(c_double), POINTER(c_double), c_int]),
        "ccmc_batch_sync": (c_int, [vp]),
        "ccmc_server_start": (c_int, [ctypes.c_size_t, c_int, c_double, POINTER(vp)]),
        "ccmc_server_submit": (c_int, [vp, POINTER(Request), POINTER(c_uint64)]),
        "ccmc_server_poll": (c_int, [vp, c_uint64, POINTER(Result)]),
        "ccmc_server_wait": (c_int, [vp, c_uint64, POINTER(Result), c_double]),
        "ccmc_server_series": (c_int, [vp, c_uint64, POINTER(Obs), c_int64, i64p]),
        "ccmc_server_release": (c_int, [vp, c_uint64]),
        "ccmc_server_stats_get": (c_int, [vp, POINTER(ServerStats)]),
        "ccmc_server_stop": (c_int, [vp]),
        "ccmc_map_size": (c_int64, [c_int, c_int]),
        "ccmc_maps_build": (c_int, [c_int, c_int, c_uint64, c_int64, c_int64,
                                    POINTER(ctypes.c_int32), c_int]),
        "ccmc_map_apply": (c_int, [vp, POINTER(ctypes.c_int32), c_int64, c_int64, c_double,
                                   c_double, c_double, c_double]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    """The loaded libccmc (loaded on first use; ImportError if it was not built)."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def _check(code: int, what: str):
    if code != OK:
        raise CcmcError(code, what)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return c_void_p(stream.cuda_stream)
    return c_void_p(int(stream))


def threshold_table(beta: float, Delta: float, V: float, J: float) -> np.ndarray:
    """The library's acceptance thresholds, shape (3, 41, 41) = [dQ/2 + 1, dBV + 20, dBJ + 20]."""
    out = np.zeros(TABLE_N, dtype=np.uint32)
    _check(lib().ccmc_threshold_table(beta, Delta, V, J, out.ctypes.data_as(POINTER(c_uint32))),
           "ccmc_threshold_table")
    return out.reshape(3, 41, 41)


def philox_device(ctr, key, count: int) -> np.ndarray:
    """Device Philox4x32-10 of counters (ctr[0] + i, ctr[1], ctr[2], ctr[3])."""
    out = np.zeros(4 * count, dtype=np.uint32)
    _check(lib().ccmc_philox_device(*[int(c) & 0xFFFFFFFF for c in ctr],
                                   *[int(k) & 0xFFFFFFFF for k in key], count,
                                   out.ctypes.data_as(POINTER(c_uint32))), "ccmc_philox_device")
    return out.reshape(count, 4)


def selftest_wait(polls: int = 1 << 16) -> int:
    """The bounded-wait self-test: a device wait on a barrier nothing completes
    gives up after `polls` polls; returns the call's code (E_TIMEOUT expected)."""
    return lib().ccmc_selftest_wait(polls)


def peak_smem_read() -> float:
    """Measured shared-memory read bandwidth of the current device (bytes/s)."""
    x = c_double()
    _check(lib().ccmc_peak_smem_read(ctypes.byref(x)), "ccmc_peak_smem_read")
    return x.value


def peak_l2_read(buffer_bytes: int = 64 << 20) -> float:
    """Measured L2 read bandwidth over an L2-resident buffer (bytes/s)."""
    x = c_double()
    _check(lib().ccmc_peak_l2_read(buffer_bytes, ctypes.byref(x)), "ccmc_peak_l2_read")
    return x.value


def map_size(Lx: int, Ly: int) -> int:
    """Pairs per paper map (Sec. 3.2): max(1, floor(Lx Ly / 10))."""
    n = int(lib().ccmc_map_size(Lx, Ly))
    if n < 0:
        raise CcmcError(n, "ccmc_map_size")
    return n


def maps_build(Lx: int, Ly: int, seed: int, map0: int, nmaps: int, nthreads: int = 0,
               out: np.ndarray = None) -> np.ndarray:
    """Host-built paper maps map0 .. map0 + nmaps - 1: int32 array (nmaps, P, 2)
    of site indices y * Lx + x (a, b) -- the random-marking algorithm of Sec. 3.2."""
    P = map_size(Lx, Ly)
    if out is None:
        out = np.empty((nmaps, P, 2), dtype=np.int32)
    if out.dtype != np.int32 or not out.flags.c_contiguous or out.size < 2 * P * nmaps:
        raise ValueError("out must be a C-contiguous int32 array of nmaps * P * 2 entries")
    _check(lib().ccmc_maps_build(Lx, Ly, seed & (2 ** 64 - 1), map0, nmaps,
                                 out.ctypes.data_as(POINTER(ctypes.c_int32)), nthreads),
           "ccmc_maps_build")
    return out


class Lattice:
    """An Lx x Ly lattice resident on the current CUDA device."""

    def __init__(self, Lx: int, Ly: int, stream=None, obs_capacity: int = 4096):
        self.Lx, self.Ly = int(Lx), int(Ly)
        h = c_void_p()
        _check(lib().ccmc_lattice_create(self.Lx, self.Ly, _stream_handle(stream), obs_capacity,
                                        ctypes.byref(h)), "ccmc_lattice_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().ccmc_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_constrained(self, seed: int, n: float, charged_frac: float = 0.3):
        _check(lib().ccmc_init_constrained(self._h, seed & (2 ** 64 - 1), n, charged_frac),
               "ccmc_init_constrained")

    def init_counts(self, seed: int, n_plus: int, n_minus: int):
        _check(lib().ccmc_init_counts(self._h, seed & (2 ** 64 - 1), n_plus, n_minus),
               "ccmc_init_counts")

    def sweep(self, nsweeps: int, beta: float, Delta: float, V: float, J: float,
              obs_every: int = 0):
        _check(lib().ccmc_sweep(self._h, nsweeps, beta, Delta, V, J, obs_every), "ccmc_sweep")

    def phases(self, nphases: int, beta: float, Delta: float, V: float, J: float):
        """Run nphases colour phases (the paper's "steps", one map each)."""
        _check(lib().ccmc_phases(self._h, nphases, beta, Delta, V, J), "ccmc_phases")

    def map_apply(self, pairs: np.ndarray, map0: int, beta: float, Delta: float, V: float,
                  J: float):
        """Apply host-built paper maps (maps_build's layout, nmaps = len(pairs))
        with one kernel per map; returns once the maps have been copied."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        if pairs.ndim != 3 or pairs.shape[2] != 2:
            raise ValueError("pairs must have shape (nmaps, P, 2)")
        _check(lib().ccmc_map_apply(self._h, pairs.ctypes.data_as(POINTER(ctypes.c_int32)),
                                    map0, pairs.shape[0], beta, Delta, V, J), "ccmc_map_apply")

    def sync(self):
        _check(lib().ccmc_sync(self._h), "ccmc_sync")

    def observables(self) -> dict:
        o = Obs()
        _check(lib().ccmc_observables(self._h, ctypes.byref(o)), "ccmc_observables")
        return o.as_dict()

    def obs_series(self, cap: int = 1 << 20) -> np.ndarray:
        """int64 records (sweeps_done, Nc, BV, BJ, M, M_stag, S_sum, S_stag), oldest first."""
        buf = (Obs * cap)()
        n = c_int64()
        _check(lib().ccmc_obs_series(self._h, buf, cap, ctypes.byref(n)), "ccmc_obs_series")
        raw = np.frombuffer(buf, dtype=np.int64).reshape(cap, 9)  # 8 int64 + the double E
        return raw[:n.value, :8].copy()

    def hist_enable(self, nbins: int):
        _check(lib().ccmc_hist_enable(self._h, nbins), "ccmc_hist_enable")
        self._nbins = nbins

    def hist(self) -> np.ndarray:
        out = np.zeros(3 * self._nbins, dtype=np.int64)
        _check(lib().ccmc_hist_get(self._h, out.ctypes.data_as(POINTER(c_int64))), "ccmc_hist_get")
        return out.reshape(3, self._nbins)

    def get_state(self) -> np.ndarray:
        out = np.zeros((self.Ly, self.Lx), dtype=np.uint8)
        _check(lib().ccmc_get_state(self._h, out.ctypes.data_as(POINTER(ctypes.c_uint8))),
               "ccmc_get_state")
        return out

    def set_state_ptr(self, host_ptr: int, seed: int, sweeps_done: int = 0):
        """set_state from a raw host pointer to Lx * Ly site codes (e.g. pinned)."""
        _check(lib().ccmc_set_state(self._h, ctypes.cast(host_ptr, POINTER(ctypes.c_uint8)),
                                   seed & (2 ** 64 - 1), sweeps_done), "ccmc_set_state")

    def get_state_packed(self) -> np.ndarray:
        """The state in the compact form: Lx * Ly / 4 bytes, site y * Lx + x at
        bits 2 ((y * Lx + x) mod 4) of byte (y * Lx + x) / 4."""
        out = np.empty(self.Lx * self.Ly // 4, dtype=np.uint8)
        _check(lib().ccmc_get_state_packed(self._h, out.ctypes.data_as(POINTER(ctypes.c_uint8))),
               "ccmc_get_state_packed")
        return out

    def set_state_packed_ptr(self, host_ptr: int, seed: int, sweeps_done: int = 0):
        """Queue a compact-state upload from a raw host pointer (e.g. pinned);
        the buffer must stay valid until the next synchronising call."""
        _check(lib().ccmc_set_state_packed(self._h, ctypes.cast(host_ptr,
                                                                POINTER(ctypes.c_uint8)),
                                           seed & (2 ** 64 - 1), sweeps_done),
               "ccmc_set_state_packed")

    def set_state_packed(self, packed: np.ndarray, seed: int, sweeps_done: int = 0):
        """Queue a compact-state upload; the array is kept alive until sync()."""
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        if packed.size != self.Lx * self.Ly // 4:
            raise ValueError("packed state must hold Lx * Ly / 4 bytes")
        self._pending = packed
        self.set_state_packed_ptr(packed.ctypes.data, seed, sweeps_done)

    def set_state(self, st: np.ndarray, seed: int, sweeps_done: int = 0):
        st = np.ascontiguousarray(st, dtype=np.uint8)
        assert st.shape == (self.Ly, self.Lx)
        _check(lib().ccmc_set_state(self._h, st.ctypes.data_as(POINTER(ctypes.c_uint8)),
                                   seed & (2 ** 64 - 1), sweeps_done), "ccmc_set_state")


class Batch:
    """Several lattices swept together (ccmc_batch_*): small ones share one
    persistent shared-memory-resident launch, large ones run alongside."""

    def __init__(self, lattices, stream=None):
        self.lattices = list(lattices)
        arr = (c_void_p * len(self.lattices))(*[lat.handle.value for lat in self.lattices])
        h = c_void_p()
        _check(lib().ccmc_batch_create(len(self.lattices), arr, _stream_handle(stream),
                                       ctypes.byref(h)), "ccmc_batch_create")
        self._h = h

    def config(self, threads: int = 256, resident_max_sites: int = 1 << 17, ctas_per_sm: int = 2,
               max_threads_per_word: int = 4):
        _check(lib().ccmc_batch_config(self._h, threads, resident_max_sites, ctas_per_sm,
                                       max_threads_per_word), "ccmc_batch_config")

    def autotune(self, probe_sweeps: int = 20):
        """Time the candidate launch shapes on a probe batch of the same shapes
        (cached per GPU and shape mix) and apply the fastest."""
        from . import autotune

        best = autotune.tune([(lat.Lx, lat.Ly) for lat in self.lattices], probe_sweeps)
        self.config(*best)
        return best

    def sweep(self, nsweeps, beta, Delta, V, J, obs_every: int = 0):
        n = len(self.lattices)

        def arr(x, dt):
            a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=dt), (n,)))
            return a

        ns, b, d, v, j = (arr(nsweeps, np.int64), arr(beta, np.float64), arr(Delta, np.float64),
                          arr(V, np.float64), arr(J, np.float64))
        dp = POINTER(c_double)
        _check(lib().ccmc_batch_sweep(self._h, ns.ctypes.data_as(POINTER(c_int64)),
                                      b.ctypes.data_as(dp), d.ctypes.data_as(dp),
                                      v.ctypes.data_as(dp), j.ctypes.data_as(dp), obs_every),
               "ccmc_batch_sweep")

    def sync(self):
        _check(lib().ccmc_batch_sync(self._h), "ccmc_batch_sync")

    def close(self):
        if getattr(self, "_h", None):
            lib().ccmc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request loop (ccmc_server_*): independent simulations
    admitted by a device-memory budget, advanced together in slices."""

    def __init__(self, hbm_budget_bytes: int = 120 << 30, max_active: int = 1024,
                 slice_ms: float = 20.0):
        h = c_void_p()
        _check(lib().ccmc_server_start(hbm_budget_bytes, max_active, slice_ms, ctypes.byref(h)),
               "ccmc_server_start")
        self._h = h
        self._outs = {}

    def submit(self, Lx, Ly, seed, n, nsweeps, beta, Delta, V, J, charged_frac=0.3,
               obs_every=0, state_out: np.ndarray | None = None) -> int:
        req = Request(Lx, Ly, seed & (2 ** 64 - 1), n, charged_frac, nsweeps, beta, Delta, V, J,
                      obs_every, None)
        if state_out is not None:
            assert state_out.dtype == np.uint8 and state_out.size == Lx * Ly
            assert state_out.flags.c_contiguous
            req.state_out = state_out.ctypes.data
        t = c_uint64()
        _check(lib().ccmc_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)),
               "ccmc_server_submit")
        if state_out is not None:
            self._outs[t.value] = state_out  # keep the buffer alive until the request is done
        return t.value

    def poll(self, ticket: int):
        """Result dict once finished, None while pending."""
        r = Result()
        code = lib().ccmc_server_poll(self._h, ticket, ctypes.byref(r))
        if code == PENDING:
            return None
        _check(code, "ccmc_server_poll")
        self._outs.pop(ticket, None)
        return r.as_dict()

    def wait(self, ticket: int, timeout_s: float = 600.0):
        r = Result()
        _check(lib().ccmc_server_wait(self._h, ticket, ctypes.byref(r), timeout_s),
               "ccmc_server_wait")
        self._outs.pop(ticket, None)
        return r.as_dict()

    def series(self, ticket: int, cap: int = 1 << 16) -> np.ndarray:
        buf = (Obs * cap)()
        n = c_int64()
        _check(lib().ccmc_server_series(self._h, ticket, buf, cap, ctypes.byref(n)),
               "ccmc_server_series")
        return np.frombuffer(buf, dtype=np.int64).reshape(cap, 9)[:n.value, :8].copy()

    def release(self, ticket: int):
        _check(lib().ccmc_server_release(self._h, ticket), "ccmc_server_release")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().ccmc_server_stats_get(self._h, ctypes.byref(st)), "ccmc_server_stats_get")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def stop(self):
        if getattr(self, "_h", None):
            lib().ccmc_server_stop(self._h)
            self._h = None
            self._outs.clear()

    def __del__(self):
        self.stop()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()
