"""Benchmark: Heat-2D 5-point Jacobi, 8192 x 8192 interior, T = 512 steps.

One step = one call of the library's run entry point advancing the whole grid
by T = 512 time steps in FP32 under the fastest schedule found by the
autotuner (BEST below): the recursive-order persistent executor over the
skewed (time block, tile) lattice, whose leaves are trapezoid tiles of depth k
streamed through registers and fed by TMA.  With --schedules the plain sweep,
the single-level schedule and a fine-grained recursive order (L2-sized leaves)
are timed beside it.  Inputs are
seeded synthetic U[0,1) values with a zero Dirichlet ring (resident in HBM
before timing; the two 256 MiB buffers exceed the 129 MB L2, so no flush is
needed between steps).

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle (the
plain FP64 naive sweep) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 8192
T_STEPS = 512
HEAT2D = [0.5, 0.125, 0.125, 0.125, 0.125]
METRIC = "GUpdates/s & DRAM bytes/update vs plain sweep; % HBM roofline at stated error"
UNIT = "GUpdates/s"
# Tile parameters of the timed schedule (from the autotuner's sweep on GB300).
BEST = {"schedule": "cot", "tile": (80, 112), "time_depth": 8, "cot_threshold": (2, 256, 256)}
BEST_SLT = {"schedule": "slt", "tile": (40, 112), "time_depth": 4, "cot_threshold": (2, 256, 256)}
# Depths (with their best tile heights) scanned beside the headline.
DEPTH_SCAN = [(2, (80, 112)), (4, (80, 112)), (6, (96, 112)), (8, (80, 112))]
WORKLOAD = "heat2d-5pt 8192x8192 T=512 fp32 zero-Dirichlet"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:   # sampler running before timing starts
                time.sleep(0.02)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def _traffic_from_profile(kernel_tag, blocks_per_launch):
    """DRAM bytes per launch of the timed kernel from the committed ncu
    summary (bytes per time block x blocks per launch), or None when the
    kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "heat2d_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for fn in rec.get("sources", []):
            with open(os.path.join(ROOT, fn), "rb") as f:
                h.update(f.read())
    except Exception:
        return None
    per_block = rec.get("bytes_per_block", {}).get(kernel_tag)
    if h.hexdigest() != rec.get("sources_sha256") or per_block is None:
        return None
    return per_block * blocks_per_launch


def _cpu_oracle_sample(seconds=12.0, threads=None):
    """The oracle (naive FP64 sweep, OpenMP over rows) on the full 8192^2 grid
    for as many steps as fit in about `seconds`; returns (GU/s, steps, cores)."""
    import numpy as np
    import oracle
    import seeded_inputs as si
    oracle.build()
    cores = threads or os.cpu_count() or 1
    sizes = (N_SIDE, N_SIDE)
    g = si.uniform_grid(sizes, 2, dtype=np.float32).astype(np.float64)
    t0 = time.perf_counter()
    oracle.sweep(g, sizes, HEAT2D, 1, threads=cores)
    one = time.perf_counter() - t0
    steps = max(1, min(64, int(seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.sweep(g, sizes, HEAT2D, steps, threads=cores)
    dt = time.perf_counter() - t0
    return N_SIDE * N_SIDE * steps / dt / 1e9, steps, cores


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class EnergyMeter:
    """The GPU's total-energy counter (NVML, millijoules since driver load),
    read through the driver's own libnvidia-ml with ctypes.  Reads only; no
    setting of the GPU is touched.  `ok` is False where NVML is missing."""

    def __init__(self, index=0, pci_bus_id=None, lib=None):
        import ctypes
        self.ct = ctypes
        self.ok = False
        try:
            self.nvml = lib if lib is not None else ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            rc = 1
            if pci_bus_id:
                rc = self.nvml.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(h))
            if rc != 0:
                rc = self.nvml.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h))
            if rc != 0:
                return
            self.h = h
            self.ok = self.read_mj() is not None
        except Exception:
            self.ok = False

    def read_mj(self):
        e = self.ct.c_ulonglong(0)
        try:
            if self.nvml.nvmlDeviceGetTotalEnergyConsumption(self.h, self.ct.byref(e)) != 0:
                return None
        except Exception:
            return None
        return int(e.value)


def energy_per_update_nj(meter, run, sync, updates_per_run, min_seconds=1.5):
    """Joules the GPU drew over repeated runs, per point update, in nJ (None
    without a meter).  Runs for at least `min_seconds` so the counter's update
    period is small against the interval."""
    if meter is None or not meter.ok:
        return None
    run()
    sync()
    t0 = time.perf_counter()
    run()
    sync()
    n = max(2, int(min_seconds / max(time.perf_counter() - t0, 1e-4)) + 1)
    e0 = meter.read_mj()
    t0 = time.perf_counter()
    for _ in range(n):
        run()
    sync()
    dt = time.perf_counter() - t0
    e1 = meter.read_mj()
    if e0 is None or e1 is None or e1 <= e0:
        return None
    return {"nJ_per_update": (e1 - e0) * 1e-3 / (updates_per_run * n) * 1e9, "avg_W": (e1 - e0) * 1e-3 / dt,
            "runs": n, "seconds": dt}


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest value over all ranks (a job takes as long as its slowest
    rank); the value itself on a single process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of replicated work: the units every rank
    processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import seeded_inputs as si
    oracle.build()
    cores = os.cpu_count() or 1
    sizes = (N_SIDE, N_SIDE)
    g = si.uniform_grid(sizes, 2, dtype=np.float32).astype(np.float64)
    t0 = time.perf_counter()
    oracle.sweep(g, sizes, HEAT2D, 1, threads=cores)
    one = time.perf_counter() - t0
    # Each step: a bounded sample (whole grid, a few time steps) sized so the
    # whole run stays within a couple of minutes.
    budget = 120.0 / max(1, args.steps + args.warmup)
    sample_steps = max(1, min(T_STEPS, int(budget / max(one, 1e-3))))
    for _ in range(args.warmup):
        oracle.sweep(g, sizes, HEAT2D, sample_steps, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sweep(g, sizes, HEAT2D, sample_steps, threads=cores)
    dt = time.perf_counter() - t0
    v = N_SIDE * N_SIDE * sample_steps * args.steps / dt / 1e9
    sample = f"full 8192^2 grid, {sample_steps} of the {T_STEPS} steps per bench step (FP64 naive sweep)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    import paper_1802_00166_gb300 as pcot
    import seeded_inputs as si
    from paper_1802_00166_gb300 import build as pbuild

    ws, rank, local = _dist()
    pbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    sched = pcot.SCHEDULES[args.schedule or BEST["schedule"]]
    params = pcot.tile_params(tile=BEST["tile"], time_depth=BEST["time_depth"],
                              cot_threshold=BEST["cot_threshold"])
    sizes = (N_SIDE, N_SIDE)
    shape = (N_SIDE + 2, N_SIDE + 2)
    pitch = ((N_SIDE + 2 + 31) // 32) * 32           # 128-byte rows for 16-byte vector access
    strides = (pitch, 1)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    g0 = si.uniform_grid(sizes, 2, dtype=np.float32)
    base = torch.zeros(shape[0] * pitch, dtype=torch.float32, device="cuda")
    view = torch.as_strided(base, shape, strides)
    view.copy_(torch.from_numpy(g0).cuda())
    nb = pcot.pcot_workspace_bytes(h, sizes, strides, T_STEPS, pcot.PCOT_F32, sched, params)
    wsbuf = torch.empty(nb, dtype=torch.uint8, device="cuda")

    def step():
        pcot.pcot_run(h, base.data_ptr(), wsbuf.data_ptr(), nb, sizes, strides, T_STEPS, pcot.PCOT_F32, sched,
                      params, stream)

    for _ in range(args.warmup):
        step()
    st = pcot.pcot_check(h, stream)
    if st != pcot.PCOT_OK:
        raise pcot.PcotError(st, "warm-up")
    n0 = pcot.pcot_launch_count(h)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = pcot.pcot_launch_count(h) - n0
    st = pcot.pcot_check(h, stream)
    if st != pcot.PCOT_OK:
        raise pcot.PcotError(st, "timed region")
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    updates = float(N_SIDE * N_SIDE * T_STEPS)
    value = job_rate(updates * args.steps, ws, ms / 1e3) / 1e9

    # End to end through the host-buffer entry point (pinned host grid, the
    # H2D copy, the run and the D2H copy inside each timed step).
    host = torch.empty(shape[0] * pitch, dtype=torch.float32).pin_memory()
    host.copy_(base.cpu())
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pcot.pcot_run_host(h, host.data_ptr(), base.data_ptr(), wsbuf.data_ptr(), nb, sizes, strides, T_STEPS,
                           pcot.PCOT_F32, sched, params, stream)
    e2e_dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    span = (shape[0] - 1) * pitch + shape[1]
    e2e = {"value": job_rate(updates * e2e_steps, ws, e2e_dt) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": span * 4, "d2h_bytes_per_step": span * 4}

    # Roofline of the dominant kernel.  The temporal-blocking model charges one
    # read and one write of the grid per time block of depth k; the single-level
    # schedule launches one kernel per block, the recursive one a single
    # persistent kernel for all blocks.  Durations are the step's CUDA events
    # divided over its launches (the ring copy is a few microseconds).
    q = pcot.pcot_plan_query(h, sizes, T_STEPS, pcot.PCOT_F32, params, with_queue=False)
    k = q["depth"]
    grid_bytes = 2.0 * N_SIDE * N_SIDE * 4
    if sched == pcot.PCOT_COT:
        # One persistent launch covers the lattice's (even) block count; the
        # last T mod (2k) steps run as single-level launches.  Time that
        # launch alone: a run of exactly its blocks is one launch and nothing else.
        blocks = q["lattice"][0]
        per_launch_bytes, kname, units = blocks * grid_bytes, "cot_kernel", blocks
        T_dom = blocks * k
        for _ in range(2):
            pcot.pcot_run(h, base.data_ptr(), wsbuf.data_ptr(), nb, sizes, strides, T_dom, pcot.PCOT_F32, sched,
                          params, stream)
        n1 = pcot.pcot_launch_count(h)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            pcot.pcot_run(h, base.data_ptr(), wsbuf.data_ptr(), nb, sizes, strides, T_dom, pcot.PCOT_F32, sched,
                          params, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        n_dom = (pcot.pcot_launch_count(h) - n1) // args.steps   # the ring copy + the persistent kernel
        launch_s = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / 1e3 / args.steps
    else:
        blocks = math.ceil(T_STEPS / k) if sched != pcot.PCOT_SWEEP else T_STEPS
        per_launch_bytes, units = grid_bytes, 1
        kname = "slt_kernel" if sched == pcot.PCOT_SLT else "sweep2d_vec_kernel"
        n_dom = blocks
        launch_s = ms / 1e3 / args.steps / blocks
    peak, peak_kind = _peaks()
    achieved = per_launch_bytes / launch_s / 1e9
    kernel_tag = f"{kname} f32 k={k} tile={q['tile_ext'][:2]}"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": _traffic_from_profile(kernel_tag, units),
            "peak_kind": peak_kind,
            "kernel": kernel_tag, "alg_bytes_per_launch": per_launch_bytes, "blocks_per_launch": units,
            "launch_ms": launch_s * 1e3, "launches_timed_per_step": n_dom,
            "model": "per time block of depth k: one read + one write of the 8192^2 fp32 grid"}

    # The temporal-blocking roof rises with the block depth k (one HBM pass per
    # k steps), so a deeper block can be faster yet reach a smaller fraction of
    # its own roof.  Scan the recursive schedule's depths on the same grid and
    # report, per depth, the throughput and the fraction of that depth's roof.
    if rank == 0 and sched == pcot.PCOT_COT and not args.schedule:
        scan = []
        for kd, tl in DEPTH_SCAN:
            prm = pcot.tile_params(tile=tl, time_depth=kd, cot_threshold=BEST["cot_threshold"])
            nbk = pcot.pcot_workspace_bytes(h, sizes, strides, T_STEPS, pcot.PCOT_F32, sched, prm)
            wsk = torch.empty(nbk, dtype=torch.uint8, device="cuda")
            runk = lambda: pcot.pcot_run(h, base.data_ptr(), wsk.data_ptr(), nbk, sizes, strides, T_STEPS,
                                         pcot.PCOT_F32, sched, prm, stream)
            runk()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(3):
                runk()
            e1.record(stream)
            torch.cuda.synchronize()
            msk = e0.elapsed_time(e1) / 3
            t_roof = math.ceil(T_STEPS / kd) * grid_bytes / (peak * 1e9) * 1e3
            scan.append({"time_depth": kd, "tile": list(tl), "ms": msk,
                         "GUpdates/s": N_SIDE * N_SIDE * T_STEPS / msk / 1e6, "roofline_frac": t_roof / msk})
            del wsk
        roof["by_depth"] = scan

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "schedule": args.schedule or BEST["schedule"],
                       "tile": list(q["tile_ext"][:2]), "time_depth": k,
                       "cot_threshold": list(BEST["cot_threshold"]), "l2": "inputs larger than L2 (2 x 256 MiB)",
                       "parallelism": "replicas" if ws > 1 else "single-gpu"},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks

    # Everything below runs after the timed region and leaves `value` alone.
    extra = rank == 0 and not args.schedule
    final = None
    if extra:
        # The headline configuration once more from the seeded initial grid,
        # for the error against the FP64 oracle (computed in the CPU leg).
        view.copy_(torch.from_numpy(g0).cuda())
        step()
        torch.cuda.synchronize()
        final = view.cpu().numpy()
        line["vs_sweep"] = compare_schedules(pcot, h, base, sizes, strides, stream)
    configs = {}
    if extra:
        del wsbuf, host
        base = view = None
        torch.cuda.empty_cache()
        j1, j1_out = run_jacobi1d(pcot, stream, args.steps)
        j3, j3_out = run_jacobi3d(pcot, stream, args.steps, peak)
        f64, f64_out = run_heat2d_f64(pcot, stream, args.steps, g0)
        configs = {"jacobi1d": j1, "jacobi3d": j3, "batched": run_batched(pcot, stream, args.steps, peak),
                   "heat2d_f64": f64}
    if rank == 0 and not args.no_cpu_baseline:
        cpu, ref = _cpu_oracle_heat2d(g0, full=extra)
        line["cpu_baseline"] = cpu
        if final is not None and ref is not None:
            import oracle
            err = oracle.errors(oracle.interior(final, sizes), oracle.interior(ref, sizes))
            line["error"] = dict(err, vs="FP64 oracle run on the widened FP32 inputs", T=T_STEPS,
                                 bound=1e-5)
        if extra:
            _cpu_leg_configs(configs, j1_out, j3_out)
            if ref is not None:
                import numpy as np
                configs["heat2d_f64"]["bitwise_equal_to_oracle"] = {
                    k: bool(np.array_equal(v, ref)) for k, v in f64_out.items()}
            del f64_out
    if configs:
        line["configs"] = configs
    if (args.gs2d or args.fdtd2d or args.la) and rank == 0:
        torch.cuda.empty_cache()
    if args.gs2d and rank == 0:
        line["gs2d"] = run_gs2d(pcot, h, stream, args.steps)
    if args.fdtd2d and rank == 0:
        line["fdtd2d"] = run_fdtd2d(pcot, h, stream, args.steps)
    if args.la and rank == 0:
        line["la"] = run_la(pcot, h, stream, args.steps)
    pcot.pcot_destroy(h)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


# Jacobi-1D 3-point, FP64 exact, n = 4096, T = 1024, weights 1/3, seeded ring.
J1D_RUNS = [("sweep", None), ("slt", dict(tile=(32,), time_depth=16)),
            ("cot", dict(tile=(64,), time_depth=16, cot_threshold=(4, 4)))]
# Jacobi-3D 7-point, 512^3 periodic FP32, T = 128, Fourier-mode input.
J3D_RUNS = [("sweep", None, 1), ("slt_k2", dict(tile=(64, 56, 0), time_depth=2), 2),
            ("slt_k3", dict(tile=(64, 56, 0), time_depth=3), 3),
            ("slt_k4", dict(tile=(64, 56, 0), time_depth=4), 4)]
J3D_HEAD = "slt_k4"


def _time_runs(run, reps, stream):
    import torch
    run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_jacobi1d(pcot, stream, steps):
    """Jacobi-1D at the configuration's size on every schedule, FP64 exact
    mode; results kept for the bitwise check against the oracle."""
    import numpy as np
    import torch

    import seeded_inputs as si
    n, T = 4096, 1024
    h = pcot.pcot_create(1, 1, [1.0 / 3.0] * 3, pcot.PCOT_DIRICHLET)
    g = si.uniform_grid((n,), 1, ring="random")
    dev = torch.from_numpy(g.copy()).cuda()
    out, results = {"workload": "jacobi1d-3pt n=4096 T=1024 fp64-exact Dirichlet (seeded ring)"}, {}
    for name, prm in J1D_RUNS:
        sched = pcot.SCHEDULES[name]
        p = pcot.tile_params(**prm) if prm else None
        nb = pcot.pcot_workspace_bytes(h, (n,), None, T, pcot.PCOT_F64_EXACT, sched, p)
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device="cuda")
        run = lambda: pcot.pcot_run(h, dev.data_ptr(), ws.data_ptr(), nb, (n,), None, T, pcot.PCOT_F64_EXACT,
                                    sched, p, stream)
        ms = _time_runs(run, max(5, min(steps, 20)), stream)
        dev.copy_(torch.from_numpy(g))
        run()
        st = pcot.pcot_check(h, stream)
        if st != pcot.PCOT_OK:
            raise pcot.PcotError(st, "jacobi1d " + name)
        results[name] = dev.cpu().numpy()
        out[name] = {"ms": ms, "GUpdates/s": n * T / ms / 1e6, "params": prm}
        dev.copy_(torch.from_numpy(g))
    pcot.pcot_destroy(h)
    return out, (g, results)


def run_jacobi3d(pcot, stream, steps, peak):
    """Jacobi-3D 512^3 periodic FP32 (T = 128, 8 seeded Fourier modes): the
    sweep and the single-level schedule at depths 2-4, each with the fraction
    of its temporal-blocking HBM roof; the depth-4 result is kept for the
    error against the FP64 oracle."""
    import numpy as np
    import torch

    import seeded_inputs as si
    n, T = 512, 128
    sizes = (n, n, n)
    h = pcot.pcot_create(3, 1, [0.4] + [0.1] * 6, pcot.PCOT_PERIODIC)
    g64, _ = si.fourier_grid(sizes, 3)
    g32 = g64.astype(np.float32)
    del g64
    dev = torch.from_numpy(g32).cuda()
    grid_bytes = 2.0 * n ** 3 * 4
    out = {"workload": "jacobi3d-7pt 512^3 T=128 fp32 periodic (8 Fourier modes)", "head": J3D_HEAD}
    result = None
    for name, prm, k in J3D_RUNS:
        sched = pcot.PCOT_SWEEP if prm is None else pcot.PCOT_SLT
        p = pcot.tile_params(**prm) if prm else None
        nb = pcot.pcot_workspace_bytes(h, sizes, None, T, pcot.PCOT_F32, sched, p)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        run = lambda: pcot.pcot_run(h, dev.data_ptr(), ws.data_ptr(), nb, sizes, None, T, pcot.PCOT_F32, sched, p,
                                    stream)
        ms = _time_runs(run, max(3, min(steps, 10)), stream)
        t_roof = math.ceil(T / k) * grid_bytes / (peak * 1e9) * 1e3
        out[name] = {"ms": ms, "GUpdates/s": n ** 3 * T / ms / 1e6, "time_depth": k,
                     "roofline_frac": t_roof / ms, "params": prm}
        if name == J3D_HEAD:
            dev.copy_(torch.from_numpy(g32))
            run()
            torch.cuda.synchronize()
            result = dev.cpu().numpy()
            dev.copy_(torch.from_numpy(g32))
        st = pcot.pcot_check(h, stream)
        if st != pcot.PCOT_OK:
            raise pcot.PcotError(st, "jacobi3d " + name)
        del ws
    pcot.pcot_destroy(h)
    del dev
    torch.cuda.empty_cache()
    return out, (g32, result)


# Heat-2D 8192^2 FP64 exact mode (bitwise the loop nest), T = 512: the sweep,
# the best overlapped tiles (single-level, depth 1) and the non-redundant
# parallelogram tiles of the skewed space.  The DP pipe bounds all three.
F64_RUNS = [("sweep", "sweep", None), ("slt_k1", "slt", dict(tile=(64, 0), time_depth=1)),
            ("skew", "skew", dict(tile=(32, 64), time_depth=4))]
F64_HEAD = "skew"
# Nominal FP64 rate of GB300, 1.25 TFLOP/s, counting an FMA as two flops:
# 152 SMs x 2 DP instructions per clock x 2.07 GHz.  FP64 exact mode issues
# 9 DP instructions per update (5 multiplies, 4 adds).
DP_INSTR_PER_S = 152 * 2 * 2.07e9
F64_EXACT_INSTR_PER_UPDATE = 9


def run_heat2d_f64(pcot, stream, steps, g0):
    """Heat-2D on the benchmark's grid (its FP32 seeded values widened) in
    FP64 exact mode on the schedules of F64_RUNS, each with its fraction of
    the DP-pipe roof; results kept for the bitwise check against the oracle's
    512 steps on the same widened inputs (computed in the CPU leg)."""
    import numpy as np
    import torch
    n, T = N_SIDE, T_STEPS
    sizes = (n, n)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    pitch = ((n + 2) * 8 + 127) // 128 * 128 // 8
    strides = (pitch, 1)
    base = torch.zeros((n + 2) * pitch, dtype=torch.float64, device="cuda")
    view = torch.as_strided(base, (n + 2, n + 2), strides)
    src = torch.from_numpy(g0.astype(np.float64)).cuda()
    roof_gu = DP_INSTR_PER_S / F64_EXACT_INSTR_PER_UPDATE / 1e9
    out = {"workload": f"heat2d-5pt {n}^2 T={T} fp64-exact Dirichlet (the benchmark's grid, widened)",
           "head": F64_HEAD, "bound": "alu",
           "peak": {"GUpdates/s": roof_gu, "basis": "nominal 1.25 TFLOP/s FP64 = 152 SMs x 2 DP instr/clk x 2.07 GHz, "
                                                  "9 DP instructions per update"}}
    results = {}
    for name, sname, prm in F64_RUNS:
        sched = pcot.SCHEDULES[sname]
        p = pcot.tile_params(**prm) if prm else None
        nb = pcot.pcot_workspace_bytes(h, sizes, strides, T, pcot.PCOT_F64_EXACT, sched, p)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        run = lambda: pcot.pcot_run(h, view.data_ptr(), ws.data_ptr(), nb, sizes, strides, T,
                                    pcot.PCOT_F64_EXACT, sched, p, stream)
        ms = _time_runs(run, max(3, min(steps, 5)), stream)
        gu = n * n * T / ms / 1e6
        out[name] = {"ms": ms, "GUpdates/s": gu, "alu_frac": gu / roof_gu, "params": prm}
        view.copy_(src)
        run()
        torch.cuda.synchronize()
        st = pcot.pcot_check(h, stream)
        if st != pcot.PCOT_OK:
            raise pcot.PcotError(st, "heat2d fp64 " + name)
        results[name] = view.cpu().numpy()
        del ws
    out["speedup_vs_sweep"] = out["sweep"]["ms"] / out[F64_HEAD]["ms"]
    pcot.pcot_destroy(h)
    del base, view, src
    torch.cuda.empty_cache()
    return out, results


def _cpu_oracle_heat2d(g0, full=True, seconds=12.0):
    """CPU leg: the oracle (naive FP64 sweep, OpenMP over rows, all host
    cores) on the benchmark grid.  With `full`, all 512 steps when they fit
    about a minute, and the result is returned for the error of the GPU run;
    otherwise a bounded number of steps.  Returns (cpu_baseline, result)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    sizes = (N_SIDE, N_SIDE)
    g = g0.astype("float64")
    oracle.sweep(g, sizes, HEAT2D, 1, threads=cores)      # warm-up: threads, first-touch pages
    t0 = time.perf_counter()
    oracle.sweep(g, sizes, HEAT2D, 2, threads=cores)
    one = (time.perf_counter() - t0) / 2
    if full and one * T_STEPS <= 90.0:
        t0 = time.perf_counter()
        ref = oracle.sweep(g, sizes, HEAT2D, T_STEPS, threads=cores)
        dt = time.perf_counter() - t0
        return ({"value": N_SIDE * N_SIDE * T_STEPS / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                 "sample": f"full 8192^2 grid, all {T_STEPS} steps of the FP64 naive sweep"}, ref)
    steps = max(1, min(64, int(seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.sweep(g, sizes, HEAT2D, steps, threads=cores)
    dt = time.perf_counter() - t0
    return ({"value": N_SIDE * N_SIDE * steps / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"full 8192^2 grid, {steps} steps of the FP64 naive sweep"}, None)


def _cpu_leg_configs(configs, j1_out, j3_out):
    """CPU leg for the other configurations: the oracle timed on each, its
    results compared with the GPU's (Jacobi-1D bitwise, Jacobi-3D error)."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    g, results = j1_out
    t0 = time.perf_counter()
    ref = oracle.sweep(g, (4096,), [1.0 / 3.0] * 3, 1024, threads=1)
    dt = time.perf_counter() - t0
    c1 = configs["jacobi1d"]
    c1["cpu_baseline"] = {"value": 4096 * 1024 / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                          "sample": "the whole configuration on one core"}
    c1["bitwise_equal_to_oracle"] = {k: bool(np.array_equal(v, ref)) for k, v in results.items()}
    g32, res = j3_out
    n, T = 512, 128
    t0 = time.perf_counter()
    ref = oracle.sweep(g32, (n, n, n), [0.4] + [0.1] * 6, T, periodic=True, threads=cores)
    dt = time.perf_counter() - t0
    c3 = configs["jacobi3d"]
    c3["cpu_baseline"] = {"value": n ** 3 * T / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                          "sample": "the whole configuration (FP64 naive sweep)"}
    if res is not None:
        c3["error"] = dict(oracle.errors(res, ref), vs="FP64 oracle run on the widened FP32 inputs",
                           schedule=J3D_HEAD, bound=1e-5)


GS2D = {"n": 2000, "T": 500, "slt": {"tile": (32, 128), "time_depth": 8},
        "slt_f64": {"tile": (16, 128), "time_depth": 8},
        "cot": {"tile": (32, 128), "time_depth": 8, "cot_threshold": (32, 32, 32)},
        "cot_f64": {"tile": (16, 128), "time_depth": 8, "cot_threshold": (32, 32, 32)}}


def run_gs2d(pcot, h, stream, steps):
    """Gauss-Seidel 2-D at the paper's size (2000^2 interior, T = 500; Table 2):
    in place on the device, sweep / single-level (wavefront) / recursive tile
    orders, FP64 (bitwise the loop nest) and FP32; CUDA events, inputs resident."""
    import torch
    n, T = GS2D["n"], GS2D["T"]
    out = {"workload": f"gs2d-9pt {n}x{n} T={T} in place", "unit": "GUpdates/s"}
    for dtype, dn in ((pcot.PCOT_F64, "f64"), (pcot.PCOT_F32, "f32")):
        tdt = torch.float32 if dtype == pcot.PCOT_F32 else torch.float64
        base = torch.rand((n + 2) * (n + 2), dtype=tdt, device="cuda")
        for name, sched, prm in (("sweep", pcot.PCOT_SWEEP, None),
                                 ("slt", pcot.PCOT_SLT, GS2D["slt_f64" if dn == "f64" else "slt"]),
                                 ("cot", pcot.PCOT_COT, GS2D["cot_f64" if dn == "f64" else "cot"])):
            p = pcot.tile_params(**prm) if prm else None
            nb = pcot.pcot_gs2d_workspace_bytes((n, n), T, sched, p)
            ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            run = lambda: pcot.pcot_gs2d_run(h, base.data_ptr(), ws.data_ptr(), nb, (n, n), None, T, dtype, sched,
                                             p, stream)
            for _ in range(2):
                run()
            torch.cuda.synchronize()
            reps = max(1, min(steps, 3))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            st = pcot.pcot_check(h, stream)
            if st != pcot.PCOT_OK:
                raise pcot.PcotError(st, "gs2d " + name)
            ms = e0.elapsed_time(e1) / reps
            gups = n * n * T / ms / 1e6
            # ALU roof: 9 flops per update (8 adds, 1 division); FP64 against the
            # nominal 1.25 TFLOP/s of the part, FP32 against 152 SMs x 128 lanes x
            # 2 flops x 2.07 GHz = 80.5 TFLOP/s (no measured FP64/FP32 peaks exist).
            peak = 1250.0 if dn == "f64" else 80540.0
            out[f"{name}_{dn}"] = {"ms": ms, "GUpdates/s": gups,
                                   "roofline": {"bound": "alu", "achieved": 9 * gups, "peak": peak,
                                                "unit": "GFLOP/s", "frac": 9 * gups / peak, "peak_kind": "nominal"},
                                   "params": {k: list(v) if isinstance(v, tuple) else v for k, v in (prm or {}).items()}}
        del base
    return out


FDTD2D = {"n": 2000, "T": 500, "slt_f64": {"tile": (32, 64), "time_depth": 4},
          "slt_f32": {"tile": (32, 64), "time_depth": 4},
          "cot_f64": {"tile": (32, 32), "time_depth": 4, "cot_threshold": (2, 256, 256)},
          "cot_f32": {"tile": (48, 64), "time_depth": 8, "cot_threshold": (2, 256, 256)}}


def run_fdtd2d(pcot, h, stream, steps):
    """FDTD-2D at the paper's size (2000^2, T = 500; Table 2): the three fields
    advanced on the device under the sweep, single-level and recursive
    schedules, FP64 (bitwise the loop nest) and FP32; CUDA events, inputs
    resident.  Roofline: FP64 against the DP pipe (11 flops per update); FP32
    against HBM with one read and one write of the three fields per pass (a
    pass is one step for the sweep, k steps for the tiles)."""
    import torch
    n, T = FDTD2D["n"], FDTD2D["T"]
    peak_bw, _ = _peaks()
    out = {"workload": f"fdtd2d {n}x{n} T={T}", "unit": "GUpdates/s"}
    for dtype, dn in ((pcot.PCOT_F64, "f64"), (pcot.PCOT_F32, "f32")):
        tdt = torch.float32 if dtype == pcot.PCOT_F32 else torch.float64
        esz = 4 if dtype == pcot.PCOT_F32 else 8
        f = [torch.rand(n * n, dtype=tdt, device="cuda") for _ in range(3)]
        fict = torch.rand(T, dtype=tdt, device="cuda")
        for name, sched, prm in (("sweep", pcot.PCOT_SWEEP, None), ("slt", pcot.PCOT_SLT, FDTD2D["slt_" + dn]),
                                 ("cot", pcot.PCOT_COT, FDTD2D["cot_" + dn])):
            p = pcot.tile_params(**prm) if prm else None
            nb = pcot.pcot_fdtd2d_workspace_bytes((n, n), None, T, dtype, sched, p)
            ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            run = lambda: pcot.pcot_fdtd2d_run(h, f[0].data_ptr(), f[1].data_ptr(), f[2].data_ptr(), fict.data_ptr(),
                                               ws.data_ptr(), nb, (n, n), None, T, dtype, sched, p, stream)
            for _ in range(2):
                run()
            torch.cuda.synchronize()
            reps = max(1, min(steps, 3))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            st = pcot.pcot_check(h, stream)
            if st != pcot.PCOT_OK:
                raise pcot.PcotError(st, "fdtd2d " + name)
            ms = e0.elapsed_time(e1) / reps
            k = 1 if prm is None else prm["time_depth"]
            gups = n * n * T / ms / 1e6
            if dn == "f64":
                # FP64 is bound by the DP pipe: 11 flops per update (3 + 3 + 5)
                # against the part's nominal 1.25 TFLOP/s
                roof = {"bound": "alu", "achieved": 11 * gups, "peak": 1250.0, "unit": "GFLOP/s",
                        "frac": 11 * gups / 1250.0, "peak_kind": "nominal"}
            else:
                alg = math.ceil(T / k) * 2.0 * 3 * n * n * esz
                roof = {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak_bw, "unit": "GB/s",
                        "frac": alg / (ms / 1e3) / 1e9 / peak_bw}
            out[f"{name}_{dn}"] = {"ms": ms, "GUpdates/s": gups, "roofline": roof,
                                   "params": {a: list(v) if isinstance(v, tuple) else v for a, v in (prm or {}).items()}}
        del f, fict
    return out


LA = {"lu": {"n": 3000, "slt": {"tile": (32, 0, 0)}, "cot": {"tile": (32, 0, 0), "cot_threshold": (2, 32, 32)}},
      "cholesky": {"n": 4000, "slt": {"tile": (32, 0, 0)},
                   "cot": {"tile": (32, 0, 0), "cot_threshold": (2, 32, 32)}}}
LA_CPU_SAMPLE_N = 1000


def run_la(pcot, h, stream, steps):
    """LU (no pivoting) and Cholesky at the paper's sizes (Table 2: LUD 3000^2,
    Cholesky 4000^2), FP64, seeded diagonally dominant matrices resident on
    the device, factored in place under the sweep, level-synchronous and
    recursive-order schedules, fused (PCOT_F64) and unfused (PCOT_F64_EXACT)
    updates, each bitwise the oracle's loops.  CUDA events around each
    factorization (the copy that restores the input is outside them).  Roof:
    the DP pipe, against the part's nominal 1.25 TFLOP/s (LU 2n^3/3 flops,
    Cholesky n^3/3); the unfused mode issues two DP instructions per update,
    so it tops out at half that rate."""
    import numpy as np
    import torch

    import oracle
    import seeded_inputs as si
    out = {"unit": "GFLOP/s", "flops": "LU 2n^3/3, Cholesky n^3/3",
           "inputs": "seeded, off-diagonal U[0,1), diagonal n + U[0,1) (Cholesky: symmetric)"}
    for kind in ("lu", "cholesky"):
        n = LA[kind]["n"]
        K = pcot.LA_KINDS[kind]
        A0 = torch.from_numpy(si.dominant_matrix(n, 7, symmetric=(kind == "cholesky"))).cuda()
        A = torch.empty_like(A0)
        flops = 2.0 * n ** 3 / 3 if kind == "lu" else n ** 3 / 3.0
        res = {"workload": f"{kind} {n}x{n} fp64 in place"}
        for dtype, dn in ((pcot.PCOT_F64, "f64"), (pcot.PCOT_F64_EXACT, "f64_exact")):
            for name, sched, prm in (("sweep", pcot.PCOT_SWEEP, None), ("slt", pcot.PCOT_SLT, LA[kind]["slt"]),
                                     ("cot", pcot.PCOT_COT, LA[kind]["cot"])):
                p = pcot.tile_params(**prm) if prm else None
                nb = pcot.pcot_la_workspace_bytes(K, n, sched, p)
                ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
                reps = max(2, min(steps, 4))
                total = 0.0
                for r in range(reps + 1):
                    A.copy_(A0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    pcot.pcot_la_run(h, K, A.data_ptr(), ws.data_ptr(), nb, n, n, dtype, sched, p, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if r > 0:  # the first run is the warm-up
                        total += e0.elapsed_time(e1)
                st = pcot.pcot_check(h, stream)
                if st != pcot.PCOT_OK:
                    raise pcot.PcotError(st, f"{kind} {name}")
                ms = total / reps
                gf = flops / ms / 1e6
                res[f"{name}_{dn}"] = {"ms": ms, "GFLOP/s": gf,
                                       "roofline": {"bound": "alu", "achieved": gf, "peak": 1250.0,
                                                    "unit": "GFLOP/s", "frac": gf / 1250.0, "peak_kind": "nominal"},
                                       "params": {a: list(v) if isinstance(v, tuple) else v
                                                  for a, v in (prm or {}).items()}}
        # the oracle (one core) on a bounded sample of the same kind of matrix
        m = LA_CPU_SAMPLE_N
        As = si.dominant_matrix(m, 7, symmetric=(kind == "cholesky"))
        t0 = time.perf_counter()
        getattr(oracle, kind)(As, fused=False)
        dt = time.perf_counter() - t0
        fs = 2.0 * m ** 3 / 3 if kind == "lu" else m ** 3 / 3.0
        res["cpu_baseline"] = {"value": fs / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                               "sample": f"{kind} of a {m}x{m} matrix (plain loops, unfused)"}
        out[kind] = res
        del A, A0
        torch.cuda.empty_cache()
    return out


def run_batched(pcot, stream, steps, peak):
    """256 independent Heat-2D grids (sides log-uniform in [256, 2048], T in
    [64, 1024], seeded) advanced by one persistent launch replayed from a CUDA
    graph: throughput and per-grid completion latency (p50 / p99).  The tile
    shape is the autotuner's pick, timed on this batch (`tuner.tune_batched`)."""
    import numpy as np
    import torch

    import seeded_inputs as si
    from paper_1802_00166_gb300 import tuner
    probs = si.batched_problem_set(seed=4, count=256)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    grids, sizes, strides, Ts = [], [], [], []
    updates = 0.0
    for side, T, seed in probs:
        shape = (side + 2, side + 2)
        pitch = ((shape[1] + 31) // 32) * 32
        base = torch.empty(pitch * shape[0], dtype=torch.float32, device="cuda")
        torch.as_strided(base, shape, (pitch, 1)).copy_(
            torch.from_numpy(si.uniform_grid((side, side), seed, dtype=np.float32)).cuda())
        grids.append(base)
        sizes += [side, side]
        strides += [pitch, 1]
        Ts.append(T)
        updates += float(side) * side * T
    best, tried = tuner.tune_batched(h, grids, sizes, strides, Ts, pcot.PCOT_F32, stream)
    params = [pcot.tile_params(**best)] * len(probs)
    nb = pcot.pcot_batch_workspace_bytes(h, sizes, strides, Ts, pcot.PCOT_F32, params)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    done = torch.zeros(len(probs) + 1, dtype=torch.int64, device="cuda")
    b = pcot.pcot_batch_create(h, grids, sizes, strides, Ts, pcot.PCOT_F32, params, ws, nb, done, stream)
    pcot.pcot_batch_launch(b, stream)
    torch.cuda.synchronize()
    reps = max(1, min(steps, 5))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        pcot.pcot_batch_launch(b, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    st = pcot.pcot_check(h, stream)
    pcot.pcot_batch_destroy(b)
    pcot.pcot_destroy(h)
    if st != pcot.PCOT_OK:
        raise pcot.PcotError(st, "batched")
    ms = e0.elapsed_time(e1) / reps
    d = done.cpu().numpy().astype(np.float64)
    lat = (d[1:] - d[0]) / 1e6
    # HBM roof at the picked depth k: every time block reads and writes each
    # grid's interior once (the headline's model, summed over the grids)
    k = int(best["time_depth"])
    alg_bytes = sum(math.ceil(T / k) * 2.0 * side * side * 4 for side, T, _ in probs)
    return {"grids": len(probs), "updates": updates, "ms": ms, "GUpdates/s": updates / ms / 1e6,
            "roofline": {"bound": "hbm", "alg_bytes": alg_bytes, "achieved_gbs": alg_bytes / ms / 1e6,
                         "peak_gbs": peak, "frac": alg_bytes / ms / 1e6 / peak},
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "latency_ms_max": float(lat.max()), "launch": "one persistent kernel, CUDA graph",
            "params": {a: list(v) if isinstance(v, tuple) else v for a, v in best.items()},
            "tuned": [{"tile": list(c["tile"]), "time_depth": c["time_depth"], "ms": round(ms, 3)} for c, ms in tried]}


def compare_schedules(pcot, h, base, sizes, strides, stream):
    """Context numbers: the plain sweep, SLT and COT in FP32 (own workspaces),
    with the energy the GPU drew per update where NVML is available (the
    paper's closing conjecture, Sec. 7: fewer off-chip accesses may save energy)."""
    import torch
    out = {}
    dev = torch.cuda.current_device()
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
        pci = "%08X:%02X:%02X.0" % (torch.cuda.get_device_properties(dev).pci_domain_id, bus,
                                     torch.cuda.get_device_properties(dev).pci_device_id)
    except Exception:
        pci = None
    meter = EnergyMeter(dev, pci)
    slt_prm = pcot.tile_params(tile=BEST_SLT["tile"], time_depth=BEST_SLT["time_depth"],
                               cot_threshold=BEST_SLT["cot_threshold"])
    cot_prm = pcot.tile_params(tile=BEST["tile"], time_depth=BEST["time_depth"], cot_threshold=BEST["cot_threshold"])
    cot_fine = pcot.tile_params(tile=(32, 112), time_depth=8, cot_threshold=(8, 8, 8))
    cases = [("sweep_f32", pcot.PCOT_SWEEP, None), ("slt_f32", pcot.PCOT_SLT, slt_prm),
             ("cot_f32", pcot.PCOT_COT, cot_prm), ("cot_f32_l2_leaves", pcot.PCOT_COT, cot_fine)]
    for name, sched, p in cases:
        nb = pcot.pcot_workspace_bytes(h, sizes, strides, T_STEPS, pcot.PCOT_F32, sched, p)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        run = lambda: pcot.pcot_run(h, base.data_ptr(), ws.data_ptr(), nb, sizes, strides, T_STEPS,
                                    pcot.PCOT_F32, sched, p, stream)
        run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        st = pcot.pcot_check(h, stream)
        if st != pcot.PCOT_OK:
            raise pcot.PcotError(st, name)
        ms = e0.elapsed_time(e1) / 3
        out[name] = {"ms": ms, "GUpdates/s": N_SIDE * N_SIDE * T_STEPS / ms / 1e6}
        en = energy_per_update_nj(meter, run, torch.cuda.synchronize, N_SIDE * N_SIDE * T_STEPS)
        if en is not None:
            out[name]["energy"] = en
        if p is not None:
            out[name]["params"] = {"tile": list(p.tile)[:2], "time_depth": p.time_depth,
                                   "cot_threshold": list(p.cot_threshold)[:3]}
        # DRAM bytes per update from the committed ncu capture of this kernel
        # (null once the kernel sources changed since it was taken).
        q = pcot.pcot_plan_query(h, sizes, T_STEPS, pcot.PCOT_F32, p, with_queue=False) if p else None
        if sched == pcot.PCOT_SWEEP:
            tag, per_update_blocks = "sweep2d_vec_kernel f32 k=1 tile=[0, 0]", T_STEPS
        else:
            kk = q["depth"]
            kern = "slt_kernel" if sched == pcot.PCOT_SLT else "cot_kernel"
            tag, per_update_blocks = f"{kern} f32 k={kk} tile={q['tile_ext'][:2]}", T_STEPS // kk
        traffic = _traffic_from_profile(tag, per_update_blocks)
        out[name]["dram_bytes_per_update"] = traffic / (N_SIDE * N_SIDE * T_STEPS) if traffic else None
    sw = out["sweep_f32"]
    for name in out:
        if name != "sweep_f32":
            out[name]["speedup_vs_sweep"] = sw["ms"] / out[name]["ms"]
            a, b = out[name].get("dram_bytes_per_update"), sw.get("dram_bytes_per_update")
            out[name]["dram_bytes_vs_sweep"] = a / b if a and b else None
    return out


def run_profile_case(args):
    """One configuration run `--case-runs` times without timing (the command
    the committed ncu summaries were captured with)."""
    import torch

    import paper_1802_00166_gb300 as pcot
    from paper_1802_00166_gb300 import build as pbuild
    pbuild.build()
    n, T = args.case_n, args.case_T
    th = tuple(int(v) for v in args.case_theta.split(","))
    sched = pcot.SCHEDULES[args.profile_case]
    if args.case_la:
        # LU / Cholesky of a seeded n x n FP64 matrix (tile side from --case-tile)
        import seeded_inputs as si
        kind = pcot.LA_KINDS[args.case_la]
        b = int(args.case_tile.split(",")[0])
        h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
        A0 = torch.from_numpy(si.dominant_matrix(n, 7, symmetric=(args.case_la == "cholesky"))).cuda()
        A = torch.empty_like(A0)
        p = pcot.tile_params(tile=(b, 0, 0), cot_threshold=th)
        nb = pcot.pcot_la_workspace_bytes(kind, n, sched, p)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        for _ in range(args.case_runs):
            A.copy_(A0)
            pcot.pcot_la_run(h, kind, A.data_ptr(), ws.data_ptr(), nb, n, n, pcot.PCOT_F64, sched, p)
        st = pcot.pcot_check(h)
        pcot.pcot_destroy(h)
        if st != pcot.PCOT_OK:
            raise pcot.PcotError(st, "profile case")
        print(f"ok {args.case_la} {args.profile_case} n={n} b={b} theta={th}")
        return 0
    if args.case_dims == 3:
        # Jacobi-3D 7-point, periodic n^3 grid (the 3-D workload's stencil)
        tile = tuple(int(v) for v in args.case_tile.split(","))
        h = pcot.pcot_create(3, 1, [0.4] + [0.1] * 6, pcot.PCOT_PERIODIC)
        base = torch.rand(n ** 3, device="cuda")
        p = pcot.tile_params(tile=tile, time_depth=args.case_k)
        nb = pcot.pcot_workspace_bytes(h, (n, n, n), None, T, pcot.PCOT_F32, sched, p)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        for _ in range(args.case_runs):
            pcot.pcot_run(h, base.data_ptr(), ws.data_ptr(), nb, (n, n, n), None, T, pcot.PCOT_F32, sched, p)
        st = pcot.pcot_check(h)
        pcot.pcot_destroy(h)
        if st != pcot.PCOT_OK:
            raise pcot.PcotError(st, "profile case")
        print(f"ok 3-D {args.profile_case} n={n} T={T} k={args.case_k} tile={tile}")
        return 0
    H, W = (int(v) for v in args.case_tile.split(","))
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    dt = pcot.DTYPES[args.case_dtype]
    elem = 4 if dt == pcot.PCOT_F32 else 8
    pitch = ((n + 2) * elem + 127) // 128 * 128 // elem          # rows padded to 128 bytes
    base = torch.rand((n + 2) * pitch, device="cuda", dtype=torch.float32 if elem == 4 else torch.float64)
    p = pcot.tile_params(tile=(H, W), time_depth=args.case_k, cot_threshold=th)
    nb = pcot.pcot_workspace_bytes(h, (n, n), (pitch, 1), T, dt, sched, p)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    for _ in range(args.case_runs):
        pcot.pcot_run(h, base.data_ptr(), ws.data_ptr(), nb, (n, n), (pitch, 1), T, dt, sched, p)
    st = pcot.pcot_check(h)
    pcot.pcot_destroy(h)
    if st != pcot.PCOT_OK:
        raise pcot.PcotError(st, "profile case")
    print(f"ok {args.profile_case} {args.case_dtype} n={n} T={T} k={args.case_k} tile={H},{W} theta={th}")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--schedule", default=None, choices=[None, "sweep", "slt", "cot"])
    ap.add_argument("--schedules", action="store_true", help="(default) sweep / SLT / COT side by side")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", action="store_true", help="(default) the 256-grid batched persistent launch")
    ap.add_argument("--gs2d", action="store_true", help="also time Gauss-Seidel 2-D at the paper's size")
    ap.add_argument("--fdtd2d", action="store_true", help="also time FDTD-2D at the paper's size")
    ap.add_argument("--la", action="store_true", help="also time LU and Cholesky at the paper's sizes")
    ap.add_argument("--profile-case", default=None, choices=[None, "sweep", "slt", "cot", "skew"],
                    help="run one Heat-2D configuration (no timing) for a profiler")
    ap.add_argument("--case-dims", type=int, default=2, choices=[2, 3])
    ap.add_argument("--case-la", default=None, choices=[None, "lu", "cholesky"],
                    help="profile case: an LU or Cholesky factorization instead of a stencil")
    ap.add_argument("--case-n", type=int, default=8192)
    ap.add_argument("--case-T", type=int, default=64)
    ap.add_argument("--case-k", type=int, default=8)
    ap.add_argument("--case-tile", default="96,112")
    ap.add_argument("--case-theta", default="2,256,256")
    ap.add_argument("--case-runs", type=int, default=2)
    ap.add_argument("--case-dtype", default="f32", choices=["f32", "f64", "f64_exact"],
                    help="profile case: arithmetic of a 2-D stencil case")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
