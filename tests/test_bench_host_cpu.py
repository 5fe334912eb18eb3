"""The benchmark's host logic on CPU: the multi-rank timing (two gloo ranks)
and the energy accounting (against a fake NVML).

The method has no exchange step between GPUs (each rank advances its own
replica of the grid), so the only cross-rank operations are the barrier and
the max-over-ranks of the timed durations.  These run here as two processes
on the gloo backend; the reference arm's rule that only rank 0 runs and
prints is checked in-process."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_BODY = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rank, world = dist.get_rank(), dist.get_world_size()
local_seconds = 1.5 + rank            # rank 1 is the slow one
dist.barrier()
slowest = bench.max_over_ranks(local_seconds, dist, "cpu")
assert slowest == 1.5 + (world - 1), slowest
rate = bench.job_rate(1000.0, world, slowest)
assert abs(rate - 1000.0 * world / slowest) < 1e-9
print("rank", rank, "ok", slowest, rate, flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_job_rate_gloo_world2():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_BODY.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            out, err = p.communicate()
        outs.append((p.returncode, out, err))
    for rank, (rc, out, err) in enumerate(outs):
        assert rc == 0, (rank, out, err[-2000:])
        assert f"rank {rank} ok 2.5" in out


def test_single_process_values_pass_through():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    """Under torchrun every rank but 0 exits at once, without work or output."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup = 1, 3

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


class _FakeNVML:
    """Stands in for libnvidia-ml: an energy counter that grows by 10 mJ per run."""

    def __init__(self):
        self.mj = 5_000
        self.bus = None

    def nvmlInit_v2(self):
        return 0

    def nvmlDeviceGetHandleByPciBusId_v2(self, bus, ref):
        self.bus = bus
        return 0

    def nvmlDeviceGetHandleByIndex_v2(self, idx, ref):
        return 0

    def nvmlDeviceGetTotalEnergyConsumption(self, h, ref):
        ref._obj.value = self.mj
        return 0


def test_energy_per_update_with_fake_nvml():
    """Energy accounting of the schedule comparison: (counter delta) / (runs x
    updates), here 10 mJ per run of 1e6 updates = 10 nJ per update."""
    import time
    import bench
    fake = _FakeNVML()
    meter = bench.EnergyMeter(0, "00000000:1B:00.0", lib=fake)
    assert meter.ok and fake.bus == b"00000000:1B:00.0"

    def run():
        time.sleep(0.002)
        fake.mj += 10

    en = bench.energy_per_update_nj(meter, run, lambda: None, 1e6, min_seconds=0.02)
    assert abs(en["nJ_per_update"] - 10.0) < 1e-9
    assert en["runs"] >= 2 and en["avg_W"] > 0


def test_energy_meter_absent_library_is_reported_not_raised():
    import bench

    class Broken:
        def nvmlInit_v2(self):
            return 9   # NVML_ERROR_DRIVER_NOT_LOADED-like failure

    assert not bench.EnergyMeter(0, None, lib=Broken()).ok
    assert bench.energy_per_update_nj(None, lambda: None, lambda: None, 1.0) is None


def test_fp64_configuration_names_real_schedules_and_the_dp_roof():
    """The FP64 exact comparison in the default run names schedules the
    library has, heads with the non-redundant skewed tiles, and states its
    DP-pipe roof from the unit counts: 152 SMs x 2 DP instructions per clock
    x 2.07 GHz over the 9 DP instructions (5 multiplies, 4 adds) of one
    exact-mode update."""
    sys.path.insert(0, ROOT)
    import bench
    pcot = pytest.importorskip("paper_1802_00166_gb300")
    names = [r[0] for r in bench.F64_RUNS]
    assert names[0] == "sweep" and bench.F64_HEAD in names
    assert dict((r[0], r[1]) for r in bench.F64_RUNS)[bench.F64_HEAD] == "skew"
    for _, sched, prm in bench.F64_RUNS:
        assert sched in pcot.SCHEDULES
        if prm is not None:
            pcot.tile_params(**prm)
    assert bench.F64_EXACT_INSTR_PER_UPDATE == 9
    assert abs(bench.DP_INSTR_PER_S / bench.F64_EXACT_INSTR_PER_UPDATE / 1e9 - 69.92) < 0.01
