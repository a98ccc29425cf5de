"""Benchmark of the coupled-pair Metropolis sweep on GB300.

Workload (default, `large16384`): one 16384 x 16384 lattice near the
charge-ordering crossover (Delta = 0.2, V = 1, J = 0.5, n = 0.05, charged
fraction 0.3, T = 0.6, seed 5).  One step = 50 sweeps (one ccmc_batch_sweep
call), with an exact recount of the observables and the histograms of M,
M_stag and S_stag after every sweep.  `--workload temperature4096`: four
4096 x 4096 lattices (Delta = 0, V = 0.5, J = 1, n = 0.1, T = 0.2, 0.5, 1, 2,
seeds 20..23), one step = 200 sweeps of each (the four concurrently on their
own streams), records every 10 sweeps.  The metric is site-updates per second
(one sweep = N site-updates).

Timing: W warm-up steps, then K timed steps, each bracketed by CUDA events on
the issuing stream; L2 is flushed (a 256 MB write) between timed steps,
outside the events.  nvidia-smi samples clocks during the timed region.
`roofline` is the colour phase of the first lattice: 1.5 algorithmic bytes a
site-update over its launch time, measured with CUDA events on the lattice's
own stream around graphs of 128 phase launches, right after the timed steps
(same lattice, stream and launch configuration); `roofline.aggregate` puts
the same bytes over the whole timed run.  `e2e` repeats the steps through the
C ABI with host buffers: every step uploads the lattices from pinned host
memory in the compact form, 2 bits a site (ccmc_set_state_packed,
stream-ordered), and reads the observable records back (ccmc_obs_series).

Beside the headline the same JSON line carries side measurements:
`temperature4096` (the four 4096^2 lattices above, with their own roofline),
`paper_maps` (the paper's own host-built maps against the colour schedule),
`batched` (512 replicas of uneven L in one persistent launch, against the same
lattices swept one at a time), `served` (a Poisson request stream through the
continuous-batching server: p50/p99 latency, achieved vs offered
site-updates/s, against the same requests run one at a time) and `small16`
(the 16x16 lattice's microseconds a sweep, plain and as a batch of one).

`--impl reference` times the CPU oracle (single-threaded C) on a bounded sample
of the same workload.  Under torchrun each rank runs its own lattices (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Sweeps of every lattice per timed step (long enough for the nvidia-smi clock
# samples, taken every 50 ms, to fall inside the timed region).
STEP_SWEEPS = {"temperature4096": 200, "large16384": 50}
OBS_EVERY = {"temperature4096": 10, "large16384": 1}

# Counters of one phase launch of the bench's dominant kernel, from the ncu
# captures of that kernel on each workload:
# dram__bytes_read.sum + dram__bytes_write.sum and smsp__inst_executed.sum.
# They hold only for the kernel sources they were taken with (kernel_digest);
# after any change to those sources the bench reports them as null.
PHASE_COUNTERS = {
    "large16384": {"digest": "e6ddb005f8d5ceedad68da55ac243d2d058a839479b6933f3ebea067275a9715",
                   "traffic": 33_638_144 + 118_528, "warp_inst": 26_336_685},
    "temperature4096": {"digest": "e6ddb005f8d5ceedad68da55ac243d2d058a839479b6933f3ebea067275a9715",
                        "traffic": 2_152_960, "warp_inst": 1_906_504},
}
# What bounds the dominant kernel, from the same captures: the HBM roofline is
# the algorithm's bound, these are the kernel's.
PHASE_LIMITER = {
    "large16384": "integer instruction issue, then the shared-memory pipe (issue active 61 %, "
                  "ALU pipe 59 %, shared-memory wavefronts 44 % of peak, half of them bank "
                  "conflicts of the table lookups; DRAM 11 %)",
    "temperature4096": "latency: one lattice's phase fills a fifth of the warp slots (warps "
                       "active 21 %, issue 27 %); the four lattices overlap on their streams",
}
# (file, first line, end line): the sources that define the tile phase kernel
# and its launch -- ccmc_phase.cu from the per-word code through the tile
# kernel, and its launchers; the headers whole.
KERNEL_SOURCES = (
    ("ccmc_phase.cu", "// One colour phase", "// Lock-step phase of several lattices"),
    ("ccmc_phase.cu", "// Launchers.", None),
    ("ccmc_device.cuh", None, None),
    ("ccmc_launch.cuh", None, None),
    ("ccmc_internal.h", None, None),
)


def kernel_digest() -> str:
    """sha256 over the tile phase kernel's sources (KERNEL_SOURCES, in order)."""
    h = hashlib.sha256()
    for name, first, end in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2301_11735_gb300", "csrc", name)) as f:
            text = f.read()
        a = text.index(first) if first else 0
        b = text.index(end, a) if end else len(text)
        h.update(text[a:b].encode())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle samples every 50 ms.  Started before the
    warm-up (nvidia-smi takes a moment to start); mark() brackets the timed
    region and summary() keeps the samples whose timestamps fall inside it."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.window = [None, None]
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # wait (at most 5 s) for the first sample
        t0 = time.time()
        while self.proc and time.time() - t0 < 5.0 and os.path.getsize(self.file.name) == 0:
            time.sleep(0.02)
        return self

    def mark(self, k: int):
        self.window[k] = time.time()

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        import datetime

        self.file.flush()
        self.file.seek(0)
        rows = [r.split(", ") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        lo, hi = self.window
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if lo is not None and hi is not None and not lo <= ts <= hi:
                    continue
                sm.append(float(r[2]))
                smax = max(smax, float(r[3]))
                for name, v in zip(names, r[6:10]):
                    if v.strip() == "Active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": smax or None, "reasons": sorted(reasons), "samples": len(sm),
                "interval_ms": 50}


def launches_per_call(nsweeps: int, obs_every: int, done: int) -> int:
    """Kernel launches of one ccmc_sweep call, following the library's rule:
    16-sweep (or obs_every-aligned) captured chunks when they fit, single
    sweeps otherwise; a sweep is 8 phase kernels, each recount one kernel, each
    chunk or single sweep ends with one counter-advance kernel."""
    n, s = 0, 0
    while s < nsweeps:
        a = done + s
        rem = nsweeps - s
        if 0 < obs_every <= 16:
            g = obs_every * (16 // obs_every)
            if a % obs_every == 0 and rem >= g:
                n += 8 * g + g // obs_every + 1
                s += g
                continue
        else:
            dist = obs_every - a % obs_every if obs_every > 0 else 1 << 60
            if rem >= 16 and dist > 16:
                n += 8 * 16 + 1
                s += 16
                continue
        n += 8 + (1 if obs_every > 0 and (a + 1) % obs_every == 0 else 0) + 1
        s += 1
    return n


def tile_ok(s) -> bool:
    """Whether the lattice takes the tile-staged phase kernel (rows of W words
    with W a multiple of 4 dividing 256, and Ly/4 a multiple of 256/W)."""
    W = (s.Lx // 4 + 15) // 16
    return (s.Lx // 4) % 16 == 0 and W % 4 == 0 and 256 % W == 0 and (s.Ly // 4) % (256 // W) == 0


def tile_kernel_name(s) -> str:
    """The tile-staged phase kernel a lattice takes: the single-tile compact
    instantiation when its phase fits one wave of it (five CTAs per SM on the
    152 SMs of a GB300), the pipelined one otherwise."""
    W = (s.Lx // 4 + 15) // 16
    tiles = (s.Ly // 4) // (256 // W)
    return ("phase_tile_kernel<5, true, 1> (one tile per CTA)" if tiles <= 5 * 152
            else "phase_tile_kernel<4, false, 1> (pipelined tiles)")


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_sims(sims, rank: int):
    """This rank's lattices under torchrun: the workload's, with seeds moved by
    len(sims) * rank, so every rank sweeps its own, distinct lattices (weak
    scaling; nothing on the data path crosses ranks)."""
    return [dataclasses.replace(s, seed=s.seed + len(sims) * rank) for s in sims]


def max_over_ranks(x: float, dist, device) -> float:
    """x maximised over the ranks of the process group (dist None: one rank);
    the job's time is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name: str, step_sweeps: int = 0):
    """(sims, description) of a named bench workload; step_sweeps: sweeps of
    every lattice per step (0: the workload's default)."""
    from workloads import large_16384, temperature_sweep_4096

    if name == "large16384":
        return [large_16384(obs_every=OBS_EVERY[name])], (
            f"16384x16384 near the charge-ordering crossover (Delta=0.2, V=1, J=0.5, n=0.05, "
            f"T=0.6), {step_sweeps or STEP_SWEEPS[name]} sweeps per step, observables and "
            f"histograms of M, M_stag, S_stag every sweep")
    name = "temperature4096"
    return temperature_sweep_4096(obs_every=OBS_EVERY[name]), (
        f"4096x4096 temperature sweep: 4 lattices (T=0.2,0.5,1,2; Delta=0, V=0.5, J=1, n=0.1, "
        f"c=0.3), {step_sweeps or STEP_SWEEPS[name]} sweeps each per step, observables every "
        f"{OBS_EVERY[name]} sweeps")


def run_reference(args):
    """The CPU oracle on a bounded sample of the workload (rank 0 only)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    sims, desc = workload(args.workload)
    # bounded sample: the first sweeps of one lattice per step (recounts at the
    # workload's observable interval included), the lattices visited in turn
    sample_sweeps = 1 if sims[0].sites > (1 << 26) else 2
    states = {}
    for s in sims:
        states[s.seed] = oracle.init_constrained(s.Lx, s.Ly, s.seed, s.n, s.charged_frac)
    times = []
    done = {s.seed: 0 for s in sims}
    for k in range(args.warmup + args.steps):
        s = sims[k % len(sims)]
        t0 = time.perf_counter()
        oracle.sweeps(states[s.seed], s.seed, done[s.seed], sample_sweeps, s.beta, s.Delta, s.V,
                      s.J, obs_every=s.obs_every)
        dt = time.perf_counter() - t0
        done[s.seed] += sample_sweeps
        if k >= args.warmup:
            times.append(dt)
    N = sims[0].sites
    value = N * sample_sweeps * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": desc, "sample_per_step": f"{sample_sweeps} sweeps of one "
                                                        f"{s.Lx}^2 lattice"},
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample_sweeps} sweeps of one {s.Lx}^2 lattice per step, "
                                   f"{args.steps} steps"},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(sims, target_s: float = 12.0):
    """Time the oracle (single-threaded C, as it stands) on whole sweeps of one
    lattice of the workload (the second if there are several), with the
    workload's observable interval, until about target_s seconds pass."""
    import oracle

    s = sims[1 if len(sims) > 1 else 0]
    st = oracle.init_constrained(s.Lx, s.Ly, s.seed, s.n, s.charged_frac)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < target_s:
        oracle.sweeps(st, s.seed, n, 1, s.beta, s.Delta, s.V, s.J,
                      obs_every=1 if s.obs_every == 1 else 0)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": s.sites * n / dt, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} sweeps of one {s.Lx}^2 lattice of the workload at T={s.T} "
                      f"({dt:.1f} s, 1 thread)"}


def measure_batched(cc, nsweeps=5000, plain_per_size=4):
    """512 independent replicas (L in {32..256}, 5000 sweeps) in one batched
    call, against the same lattices swept one at a time: a stated subset
    (the first `plain_per_size` lattices of every size), each for the full
    5000 sweeps from the same state, whose final states must equal the
    batch's bit for bit."""
    import numpy as np
    import torch

    from workloads import replicas_512

    sims = replicas_512(nsweeps=nsweeps)
    cols = ([s.beta for s in sims], [s.Delta for s in sims], [s.V for s in sims],
            [s.J for s in sims])
    lats = []
    for s in sims:
        lat = cc.Lattice(s.Lx, s.Ly)
        lat.init_constrained(s.seed, s.n, s.charged_frac)
        lats.append(lat)
    with cc.Batch(lats) as b:
        cfg = b.autotune(probe_sweeps=200)
        b.sweep(3, *cols)
        b.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.sweep(nsweeps, *cols)
        b.sync()
        dt = time.perf_counter() - t0
    work = sum(s.sites for s in sims) * nsweeps
    picked, seen = [], {}
    for i, s in enumerate(sims):
        if seen.get(s.Lx, 0) < plain_per_size:
            seen[s.Lx] = seen.get(s.Lx, 0) + 1
            picked.append(i)
    t_plain, identical = 0.0, True
    for i in picked:
        s = sims[i]
        with cc.Lattice(s.Lx, s.Ly) as one:
            one.init_constrained(s.seed, s.n, s.charged_frac)
            one.sweep(3, s.beta, s.Delta, s.V, s.J)
            one.sync()
            t0 = time.perf_counter()
            one.sweep(nsweeps, s.beta, s.Delta, s.V, s.J)
            one.sync()
            t_plain += time.perf_counter() - t0
            identical &= bool(np.array_equal(one.get_state(), lats[i].get_state()))
    plain = sum(sims[i].sites for i in picked) * nsweeps / t_plain
    for lat in lats:
        lat.close()
    return {"workload": "512 replicas, L~U{32,64,128,256}, T grid [0.1,3], n~U{0,.1,.2,.3}, "
                        "Delta~U{-.5,0,.5}, V=J=1, 5000 sweeps",
            "value": work / dt, "unit": "site-updates/s", "seconds": dt,
            "config": {"threads": cfg[0], "resident_max_sites": cfg[1], "ctas_per_sm": cfg[2],
                       "max_threads_per_word": cfg[3]},
            "plain_back_to_back": {"value": plain, "unit": "site-updates/s",
                                   "sample": f"{len(picked)} of the lattices ({plain_per_size} of "
                                             f"each size), the full {nsweeps} sweeps each, one "
                                             "ccmc_sweep call at a time",
                                   "identical_final_states": identical},
            "speedup_vs_plain": (work / dt) / plain}


def measure_small(cc, reps=3):
    """The 16x16 lattice of 48 + 16 charges (Delta = 0.5, V = J = 1, T = 1):
    2000 sweeps with observables after every sweep, as microseconds a sweep on
    the plain single-lattice path (eight phase launches and a recount a sweep,
    replayed as graphs) and as a batch of one (one resident launch with the
    lattice in shared memory, autotuned launch shape); best of reps, host clock
    around a synchronised call."""
    from workloads import SMALL_16 as c

    beta, nsw = 1.0 / c["T"], c["nsweeps"]
    out = {"workload": f"{c['L']}x{c['L']}, {c['n_plus']} + {c['n_minus']} charges, "
                       f"Delta={c['Delta']}, V={c['V']}, J={c['J']}, T={c['T']}: {nsw} sweeps, "
                       f"observables every sweep"}
    with cc.Lattice(c["L"], c["L"]) as lat:
        lat.init_counts(c["seed"], c["n_plus"], c["n_minus"])
        lat.sweep(20, beta, c["Delta"], c["V"], c["J"], obs_every=1)
        lat.sync()
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            lat.sweep(nsw, beta, c["Delta"], c["V"], c["J"], obs_every=1)
            lat.sync()
            best = min(best, time.perf_counter() - t0)
        out["plain_us_per_sweep"] = 1e6 * best / nsw
        with cc.Batch([lat]) as b:
            out["batched_config"] = list(b.autotune(probe_sweeps=200))
            cols = ([beta], [c["Delta"]], [c["V"]], [c["J"]])
            b.sweep(20, *cols, obs_every=1)
            b.sync()
            best = float("inf")
            for _ in range(reps):
                t0 = time.perf_counter()
                b.sweep(nsw, *cols, obs_every=1)
                b.sync()
                best = min(best, time.perf_counter() - t0)
        out["batched_us_per_sweep"] = 1e6 * best / nsw
    return out


def measure_paper_maps(cc, L=4096, nmaps=40, batch=8):
    """The paper's own parallel scheme (Sec. 3.2) on one lattice of the
    workload: maps of N/10 pairs built on the host by random marking (all host
    cores), copied to the GPU and applied one kernel per map.  Reports the host
    generation rate, the device rate with maps already built, the pipelined
    rate (the host builds the next batch while the GPU applies the current
    one) and the colour schedule's rate on the same lattice."""
    import torch

    from workloads import temperature_sweep_4096

    s = temperature_sweep_4096()[1]
    P = cc.map_size(L, L)
    updates_per_map = 2 * P
    stream = torch.cuda.Stream()
    with cc.Lattice(L, L, stream=stream) as lat:
        lat.init_constrained(s.seed, s.n, s.charged_frac)
        t0 = time.perf_counter()
        maps = cc.maps_build(L, L, s.seed, 0, nmaps)
        t_gen = time.perf_counter() - t0
        lat.map_apply(maps[:2], 0, s.beta, s.Delta, s.V, s.J)  # warm-up
        lat.sync()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.map_apply(maps, 0, s.beta, s.Delta, s.V, s.J)
        b.record(stream)
        lat.sync()
        t_dev = a.elapsed_time(b) / 1e3  # copy of all maps + one kernel per map
        t0 = time.perf_counter()
        for k in range(0, nmaps, batch):
            m = cc.maps_build(L, L, s.seed, nmaps + k, batch)
            lat.map_apply(m, nmaps + k, s.beta, s.Delta, s.V, s.J)
        lat.sync()
        t_pipe = time.perf_counter() - t0
        lat.sweep(2, s.beta, s.Delta, s.V, s.J)
        lat.sync()
        a.record(stream)
        lat.sweep(16, s.beta, s.Delta, s.V, s.J)
        b.record(stream)
        lat.sync()
        t_col = a.elapsed_time(b) / 1e3
    return {
        "workload": f"{L}x{L} at T={s.T} (Delta={s.Delta}, V={s.V}, J={s.J}): {nmaps} maps of "
                    f"{P} pairs (N/10)",
        "host_threads": os.cpu_count(),
        "host_generation": {"value": nmaps * updates_per_map / t_gen, "unit": "site-updates/s",
                            "ms_per_map": 1e3 * t_gen / nmaps},
        "device_only": {"value": nmaps * updates_per_map / t_dev, "unit": "site-updates/s",
                        "ms_per_map": 1e3 * t_dev / nmaps,
                        "h2d_bytes_per_map": 8 * P},
        "pipelined": {"value": nmaps * updates_per_map / t_pipe, "unit": "site-updates/s"},
        "colour_schedule": {"value": 16 * L * L / t_col, "unit": "site-updates/s"},
    }


def measure_served(cc, count=2000, plain_every=125):
    """Poisson request stream (200 req/s; L log-uniform in [32, 2048]; sweeps
    log-uniform in [1e3, 1e5]) through the continuous-batching server under a
    120 GB budget; p50/p99 latency from submission to completion.  Beside it,
    a stated subset of the same requests (every plain_every-th) runs one at a
    time, uncapped, through the plain single-lattice path; their final
    observables must equal the served ones."""
    import numpy as np

    from workloads import request_stream

    arrivals, sims = request_stream(count=count)
    srv = cc.Server(hbm_budget_bytes=120 << 30, max_active=1024, slice_ms=20.0)
    t0 = time.perf_counter()
    tickets = []
    for a, s in zip(arrivals, sims):
        delay = a - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(s.Lx, s.Ly, s.seed, s.n, s.nsweeps, s.beta, s.Delta, s.V, s.J))
    res = [srv.wait(t, timeout_s=3600.0) for t in tickets]
    stats = srv.stats()
    srv.stop()
    ok = [r for r in res if r["status"] == 0]
    lat = np.array([r["done_s"] - r["submit_s"] for r in ok])
    work = sum(r["site_updates"] for r in ok)
    span = max(r["done_s"] for r in ok) - min(r["submit_s"] for r in res)
    offered = sum(s.sites * s.nsweeps for s in sims) / max(arrivals[-1], 1e-9)
    picked = list(range(0, count, plain_every))
    t_plain, identical = 0.0, True
    keys = ("Nc", "BV", "BJ", "M", "M_stag", "S_sum", "S_stag", "sweeps_done")
    for i in picked:
        s = sims[i]
        tp = time.perf_counter()
        with cc.Lattice(s.Lx, s.Ly) as one:
            one.init_constrained(s.seed, s.n, s.charged_frac)
            one.sweep(s.nsweeps, s.beta, s.Delta, s.V, s.J)
            obs = one.observables()
        t_plain += time.perf_counter() - tp
        identical &= all(obs[k] == res[i]["final_obs"][k] for k in keys)
    plain = sum(sims[i].sites * sims[i].nsweeps for i in picked) / t_plain
    return {"workload": f"{count} Poisson requests at 200/s (L log-U[32,2048], sweeps "
                        "log-U[1e3,1e5], T~U[0.1,3], n~U[0,.4], Delta~U[-1,1], V~U[0,2], J=1), "
                        "120 GB budget, at most 1024 running, 20 ms slices",
            "value": work / span, "unit": "site-updates/s", "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "offered": offered,
            "completed": stats["completed"], "failed": stats["failed"],
            "rejected": stats["rejected"], "slices": stats["slices"], "span_s": span,
            "plain_back_to_back": {"value": plain, "unit": "site-updates/s",
                                   "sample": f"{len(picked)} of the requests (every "
                                             f"{plain_every}th), uncapped, one at a time "
                                             "(init, ccmc_sweep, observables)",
                                   "identical_final_observables": identical},
            "speedup_vs_plain": (work / span) / plain}


def time_workload(cc, sims, step_sweeps, steps, warmup, dist, sampler=None, hist=False):
    """Sweep `sims` (one lattice each, on their own streams, one ccmc_batch
    call a step) for `warmup` untimed and `steps` timed steps of `step_sweeps`
    sweeps, L2 flushed between timed steps; then time the colour phase of the
    first lattice alone on its own stream, and repeat the steps end to end
    from pinned host memory.  Returns the measured numbers."""
    import torch

    main = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in sims]
    lats = [cc.Lattice(s.Lx, s.Ly, stream=st) for s, st in zip(sims, streams)]
    for lat, s in zip(lats, sims):
        lat.init_constrained(s.seed, s.n, s.charged_frac)
        if hist:
            lat.hist_enable(1024)
    batch = cc.Batch(lats, stream=main)
    cols = ([s.beta for s in sims], [s.Delta for s in sims], [s.V for s in sims],
            [s.J for s in sims])
    obs_every = sims[0].obs_every
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step():
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(main)
        for st in streams:
            st.wait_event(ev0)
        batch.sweep(step_sweeps, *cols, obs_every=obs_every)
        for st in streams:
            e = torch.cuda.Event()
            e.record(st)
            main.wait_event(e)
        ev1.record(main)
        return ev0, ev1

    evs = []
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(0)
    t_wall = time.perf_counter()
    for _ in range(steps):
        with torch.cuda.stream(main):
            flush.zero_()
        evs.append(step())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if sampler:
        sampler.mark(1)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, "cuda")
    updates_per_step = sum(s.sites for s in sims) * step_sweeps
    world = dist.get_world_size() if dist else 1
    value = updates_per_step * steps * world / total_s

    # the dominant kernel: the colour phase of the first lattice, in the launch
    # configuration of the timed steps (same lattice, stream and graphs).  A
    # chunk of 16 sweeps is 128 phase launches (plus a one-thread counter
    # advance), replayed as one graph; events on the lattice's stream around it
    # give the average phase-launch time (slightly over, by the advance).
    lat0, s0, st0 = lats[0], sims[0], streams[0]
    cal = []
    for _ in range(6):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st0)
        lat0.sweep(16, s0.beta, s0.Delta, s0.V, s0.J, obs_every=0)
        b.record(st0)
        cal.append((a, b))
    torch.cuda.synchronize()
    phase_ms = statistics.mean(x.elapsed_time(y) for x, y in cal[2:]) / 128

    # end to end through the C ABI with host buffers: every step uploads each
    # lattice's state in the compact form (2 bits a site) from pinned host
    # memory, stream-ordered so that one lattice's upload overlaps the others'
    # sweeps, and reads the records back
    recs_per_step = step_sweeps // obs_every if obs_every > 0 else 0
    host_states = [torch.from_numpy(lat.get_state_packed()).pin_memory() for lat in lats]
    rec_bytes = 0
    e2e_times = []
    for k in range(max(2, steps // 2) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for lat, s, h in zip(lats, sims, host_states):
            lat.set_state_packed_ptr(h.data_ptr(), s.seed, 0)
        batch.sweep(step_sweeps, *cols, obs_every=obs_every)
        recs = [lat.obs_series(cap=max(recs_per_step, 1)) for lat in lats]
        dt = time.perf_counter() - t0
        rec_bytes = sum(r.nbytes for r in recs)
        if k > 0:
            e2e_times.append(dt)
    e2e_value = updates_per_step * len(e2e_times) * world / max_over_ranks(sum(e2e_times), dist,
                                                                           "cuda")
    batch.close()
    for lat in lats:
        lat.close()
    del flush
    return {"value": value, "total_s": total_s, "step_ms": step_ms, "t_wall": t_wall,
            "phase_ms": phase_ms, "e2e_value": e2e_value,
            "h2d": int(sum(h.numel() for h in host_states)), "d2h": int(rec_bytes)}


def roofline(name, s0, m, value, peak, peak_kind, clocks, local):
    """The roofline object of the colour phase of lattice s0: algorithmic bytes
    (1.5 B a site-update, N/8 updates a phase launch) over the measured launch
    time; `aggregate` carries the same bytes over the whole timed run."""
    import torch

    alg_bytes = 1.5 * s0.sites / 8
    achieved = alg_bytes / (m["phase_ms"] * 1e-3) / 1e9
    counters = PHASE_COUNTERS.get(name)
    if counters and counters["digest"] != kernel_digest():
        counters = None  # the kernel changed since the capture
    issue = None
    if counters:
        # warp-instructions per second against one per scheduler per cycle
        # (4 schedulers per SM) at the maximum SM clock
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak_issue = 4 * sms * float((clocks or {}).get("sm_max_mhz") or 2070.0) * 1e6
        rate = counters["warp_inst"] / (m["phase_ms"] * 1e-3)
        issue = {"warp_inst_per_launch": counters["warp_inst"], "achieved": rate,
                 "peak": peak_issue, "unit": "warp-inst/s", "frac": rate / peak_issue}
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": counters["traffic"] if counters else None,
            "issue": issue,
            "limiter": PHASE_LIMITER.get(name) if counters else None,
            "kernel": f"colour phase of one {s0.Lx}^2 lattice "
                      f"({tile_kernel_name(s0) if tile_ok(s0) else 'phase_kernel'})",
            "peak_source": peak_kind, "launch_ms": m["phase_ms"],
            # the same algorithmic bytes over the whole timed run (every lattice's
            # phases, recounts and histograms included)
            "aggregate": {"achieved": 1.5 * value / 1e9, "frac": 1.5 * value / 1e9 / peak,
                          "unit": "GB/s"}}


def run_ours(args):
    import torch

    import paper_2301_11735_gb300 as cc

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sims, workload_desc = workload(args.workload, args.sweeps_per_step)
    sims = rank_sims(sims, rank)
    step_sweeps = args.sweeps_per_step or STEP_SWEEPS[args.workload]
    if step_sweeps % sims[0].obs_every:
        raise SystemExit(f"--sweeps-per-step must be a multiple of {sims[0].obs_every}")
    sampler = ClockSampler(local)
    with sampler:
        m = time_workload(cc, sims, step_sweeps, args.steps, args.warmup, dist, sampler,
                          hist=args.workload == "large16384")
    clocks = sampler.summary()
    value = m["value"]
    peak, peak_kind = _peaks()

    if rank == 0:
        s0 = sims[0]
        line = {
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * m["total_s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload_desc,
                       "lattices_per_gpu": len(sims), "sweeps_per_step": step_sweeps,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas{world}"},
            "clocks": clocks, "wall_s": m["t_wall"],
            # per step and lattice: 8 phase launches a sweep, the recounts, counter advances
            "gpu_launches": args.steps * len(sims) * launches_per_call(
                step_sweeps, s0.obs_every, step_sweeps),
            "roofline": roofline(args.workload, s0, m, value, peak, peak_kind, clocks, local),
            "e2e": {"value": m["e2e_value"], "unit": "site-updates/s",
                    "h2d_bytes_per_step": m["h2d"], "d2h_bytes_per_step": m["d2h"]},
        }
        # share of the timed steps spent in phase launches (the rest: recounts,
        # histograms, counter advances)
        line["roofline"]["phase_share"] = (8 * step_sweeps * len(sims) * m["phase_ms"]
                                           / (1e3 * m["total_s"] / args.steps))
        if not args.no_side:
            peaks = measure_peaks(cc)
            line["peaks"] = peaks
            if args.workload == "large16384":
                t = measure_temperature(cc, args, peak, peak_kind, local)
                t["l2_roofline"] = onchip_roofline("l2", 1.5 * t["value"] / 1e9, peaks)
                line["temperature4096"] = t
            b = measure_batched(cc)
            b["roofline"] = onchip_roofline("smem", 1.5 * b["value"] / 1e9, peaks)
            line["batched"] = b
            line["served"] = measure_served(cc, count=args.served_requests)
            line["paper_maps"] = measure_paper_maps(cc)
            sm = measure_small(cc)
            sm["roofline"] = onchip_roofline("smem", 1.5 * 256 / (sm["batched_us_per_sweep"] * 1e-6)
                                             / 1e9, peaks)
            line["small16"] = sm
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_sample(sims)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measure_peaks(cc):
    """The device's measured on-chip read bandwidths (the shared-memory and L2
    paths' roofline denominators): every SM streaming conflict-free 16-byte
    shared-memory reads, and 16-byte L1-bypassing reads of a 64 MB buffer that
    L2 holds."""
    return {"smem_gbs": cc.peak_smem_read() / 1e9, "l2_gbs": cc.peak_l2_read(64 << 20) / 1e9,
            "how": "ccmc_peak_smem_read / ccmc_peak_l2_read(64 MB): one timed launch after a "
                   "warm-up, CUDA events"}


def onchip_roofline(bound, achieved_gbs, peaks):
    """Roofline object of a path bound by on-chip memory: 1.5 algorithmic bytes
    a site-update over the measured shared-memory (smem) or L2 read peak."""
    p = peaks["smem_gbs" if bound == "smem" else "l2_gbs"]
    return {"bound": bound, "achieved": achieved_gbs, "peak": p, "unit": "GB/s",
            "frac": achieved_gbs / p, "traffic": None, "peak_source": "measured on this device"}


def measure_temperature(cc, args, peak, peak_kind, local):
    """Side measurement: the 4096^2 temperature sweep (four lattices on their
    own streams, 200 sweeps each a step, records every 10 sweeps), 10 timed
    steps after 3 warm-up steps, with its own roofline object."""
    sims, desc = workload("temperature4096")
    step_sweeps = STEP_SWEEPS["temperature4096"]
    m = time_workload(cc, sims, step_sweeps, 10, 3, None)
    out = {"workload": desc, "value": m["value"], "unit": "site-updates/s",
           "ms_per_step": 1e3 * m["total_s"] / 10, "steps": 10, "warmup": 3,
           "e2e": {"value": m["e2e_value"], "unit": "site-updates/s",
                   "h2d_bytes_per_step": m["h2d"], "d2h_bytes_per_step": m["d2h"]},
           "roofline": roofline("temperature4096", sims[0], m, m["value"], peak, peak_kind,
                                None, local)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the batched-replica and served-stream measurements")
    ap.add_argument("--sweeps-per-step", type=int, default=0,
                    help="sweeps of every lattice per step (default: the workload's)")
    ap.add_argument("--workload", default="large16384",
                    choices=["temperature4096", "large16384"],
                    help="large16384 (default): one 16384^2 lattice with observables and "
                         "histograms every sweep; temperature4096: four 4096^2 lattices")
    ap.add_argument("--served-requests", type=int, default=2000,
                    help="requests of the served Poisson stream (side measurement)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
