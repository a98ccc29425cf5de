"""Host-side pieces of bench.py (no GPU): the launch-count rule that the JSON
line's gpu_launches claim follows, the kernel-source digest that gates the
capture counters, and the workload table."""
import re

import bench


def test_launch_count_rule():
    # 10 sweeps recorded every 10: one 10-sweep graph = 80 phases + 1 recount + 1 advance
    assert bench.launches_per_call(10, 10, 10) == 82
    # recorded every sweep: 10 single sweeps of 8 phases + recount + advance
    assert bench.launches_per_call(10, 1, 10) == 100
    # no records: one 16-sweep graph and 4 single sweeps
    assert bench.launches_per_call(20, 0, 0) == 8 * 16 + 1 + 4 * 9


def test_kernel_digest_and_counters():
    d = bench.kernel_digest()
    assert re.fullmatch(r"[0-9a-f]{64}", d)
    for c in bench.PHASE_COUNTERS.values():
        assert c["traffic"] > 0 and c["warp_inst"] > 0 and re.fullmatch(r"[0-9a-f]{64}", c["digest"])


def test_workloads():
    sims, desc = bench.workload("temperature4096")
    assert len(sims) == 4 and all(s.Lx == 4096 for s in sims) and "4096" in desc
    sims, desc = bench.workload("large16384")
    assert len(sims) == 1 and sims[0].Lx == 16384 and sims[0].obs_every == 1


def test_step_lengths():
    # every timed step ends on an observable record, and is long enough for
    # several 50 ms clock samples (about 15 ms a step on a GB300)
    for name, sweeps in bench.STEP_SWEEPS.items():
        assert sweeps % bench.OBS_EVERY[name] == 0
        sims, _ = bench.workload(name)
        assert sum(s.sites for s in sims) * sweeps >= 10 ** 10
