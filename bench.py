"""Benchmark: rD3Q53 MRT-LB collide-stream throughput on one GB300 (or N replicas).

Workload: the rD3Q53 compressible isothermal Taylor-Green vortex on 256 x 256 x 192 cells
(dz/dx = 4/3), Ma = 0.3, Re = 1600, FP32 populations and arithmetic. One benchmark step is one
lattice-Boltzmann time step of the whole grid: one launch of the fused pull-gather / collide /
store kernel (streaming, fields, equilibrium, sources, collision). The two population arrays
(2 x 2.67 GB) are far larger than the 129 MB L2, so no flush is needed between steps.

Printed (rank 0, one JSON line): MLUPS over all ranks, the roofline of the collide-stream kernel
against the measured HBM copy bandwidth (algorithmic bytes 2 Q 4 B per cell update), SM clocks
sampled during the timed region, an end-to-end number through the C ABI with pinned host
buffers, and the FP64 oracle timed on the host cores on a bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rD3Q53 MLUPS"
UNIT = "MLUPS"
GRID = (256, 256, 192)
Q = 53
# DRAM traffic of the benchmark kernel per cell update, from an ncu capture of the same workload on
# 256 x 256 x 96 cells (half the grid: 2.7 GB on the device), scaled to the benchmark grid by cells
PROFILE = os.path.join(ROOT, "profiles", "k_step_rd3q53_f32_tgv3d_256x256x96.md")
# the sources the benchmark kernel is compiled from (the traffic figure is void once their code,
# comments aside, changes)
KERNEL_SOURCES = ("include/lbm_mrt.h", "paper_2512_16230_gb300/csrc/lattices.cuh",
                  "paper_2512_16230_gb300/csrc/lbm_internal.cuh", "paper_2512_16230_gb300/csrc/mrt_kernels.cuh",
                  "paper_2512_16230_gb300/csrc/tc_kernels.cuh", "paper_2512_16230_gb300/csrc/tcgen05.cuh",
                  "paper_2512_16230_gb300/csrc/k_rd3q53.cu")
CPU_SAMPLE_GRID = (256, 256, 16)    # cpu_baseline: ~10-30 s of oracle work on the GPU machine
CPU_SAMPLE_STEPS = 8
REF_BUDGET_S = 150.0                  # --impl reference: wall-clock budget for W + K sample steps
HIGH_RATES = {4: 0.8, 5: 1.35, 6: 1.6, 7: 0.9, 8: 1.25}   # variant: one rate per order >= 4
VARIANT_STEPS = 100


STORE_DTYPE = {"f32": ("f32", 4, "FP32"), "f16_dev": ("f16", 2, "FP16 deviation storage"),
               "bf16_dev": ("bf16", 2, "BF16 deviation storage")}


def _workload(grid=GRID, store="f32"):
    from paper_2512_16230_gb300 import workloads as W
    return W.taylor_green_3d(n=tuple(grid), steps=1000, store=store)


def _config(extra=None, grid=GRID, store="f32"):
    cfg = {
        "workload": f"rD3Q53 Taylor-Green 3D, {grid[0]}x{grid[1]}x{grid[2]} cells (dz/dx=4/3), Ma 0.3, Re 1600, "
                    f"{STORE_DTYPE[store][2]}",
        "lattice": "rD3Q53", "cells": int(math.prod(grid)), "grid": list(grid), "Q": Q,
        "store": store, "compute": "f32",
        "l2": ("inputs larger than L2 (2 x {:.3g} GB population arrays vs 129 MB L2), no flush"
               if Q * math.prod(grid) * STORE_DTYPE[store][1] > 129e6 else
               "population arrays of 2 x {:.3g} GB fit in the 129 MB L2: not an HBM measurement").format(
            Q * math.prod(grid) * STORE_DTYPE[store][1] / 1e9),
        "parallelism": "replicas",
    }
    if extra:
        cfg.update(extra)
    return cfg


def _code_only(text):
    """C/C++ source without its comments and with every run of whitespace as one space, so that
    an edit of the documentation alone leaves the hash of the compiled code unchanged."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _source_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(f.encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def _profile_traffic(cells):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None, None
    m = re.search(r"dram_bytes_per_cell_update:\s*([0-9.eE+-]+)", text)
    s = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != _source_sha():
        return None, s.group(1) if s else None
    return float(m.group(1)) * cells, s.group(1)


def _kernel_name(args, grid):
    """The collide-stream kernel the library runs for this storage and grid."""
    rows = args.store != "f32" and grid[0] % 8 == 0 and grid[0] <= 256
    if args.store == "f32":
        return "k_step<rD3Q53, f32, NSE>"
    base = ("k_step_rows_tc" if args.tensor_cores else "k_step_rows") if rows else \
        ("k_step_tc" if args.tensor_cores else "k_step")
    return f"{base}<rD3Q53, {args.store}, NSE>"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self, busy_fraction=0.5):
        rows = []
        for rec in csv.reader(io.StringIO(self.out)):
            rec = [r.strip() for r in rec]
            if len(rec) < 9:
                continue
            try:
                rows.append(dict(sm=float(rec[1]), smax=float(rec[2]), power=float(rec[3]), hw=rec[5], hwt=rec[6],
                                 swt=rec[7], swp=rec[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        load = [r for r in rows if r["power"] >= busy_fraction * max(x["power"] for x in rows)] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(load),
                "power_w_max": max(r["power"] for r in rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, ws, device=None):
    """Max of a float over the ranks of the default process group (identity for one rank)."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank, steps, ws, seconds_max):
    """Whole-job MLUPS: every rank advances its own replica, timed by the slowest rank."""
    return cells_per_rank * steps * ws / seconds_max / 1e6


def cpu_baseline_worker(nx, ny, nz, steps):
    """Time the FP64 oracle, as it stands, on a slab of the benchmark grid (run in a fresh
    process; prints one JSON object)."""
    import numpy as np  # noqa: F401
    from oracle import lattice as OL
    from oracle import mrt as OM
    from paper_2512_16230_gb300 import workloads as W
    wl = W.taylor_green_3d(n=GRID, steps=1)
    spec = wl.lattice
    lat = OL.build(spec.kind, spec.c, spec.cs2, spec.free_w)
    n = (nx, ny, nz)
    m = OM.Model(lat, "nse", n, wl.s, wl.s_high)
    from paper_2512_16230_gb300 import inputs as I
    rho, u = I.taylor_green_3d(n, spec.c, wl.init["u0"], 1.0, spec.cs2[0])
    m.init_fields(rho, u)
    t0 = time.perf_counter()
    m.step(steps)
    dt = time.perf_counter() - t0
    print(json.dumps({"mlups": nx * ny * nz * steps / dt / 1e6, "seconds": dt}))


ORACLE_CONFIG_STEPS = {"taylor_green_rD2Q25_64x48_f64": 200, "ncde_hill_rD2Q13_1024x768": 10}


def oracle_config_worker(name, steps):
    """Time the FP64 oracle, as it stands, on one of the smaller configurations at full size (run in
    a fresh process; prints one JSON object)."""
    from oracle import lattice as OL
    from oracle import mrt as OM
    from paper_2512_16230_gb300 import workloads as W
    wl = W.taylor_green_2d() if name.startswith("taylor_green") else W.ncde_hill(store="f64")
    spec = wl.lattice
    lat = OL.build(spec.kind, spec.c, spec.cs2, spec.free_w)
    m = OM.Model(lat, wl.eq, wl.n, wl.s, wl.s_high, force=wl.force, u_const=wl.u_const, nonlin=wl.nonlin)
    rho, u = wl.fields()
    m.init_fields(rho, u)
    t0 = time.perf_counter()
    m.step(steps)
    dt = time.perf_counter() - t0
    print(json.dumps({"mlups": wl.ncells * steps / dt / 1e6, "seconds": dt}))


def run_oracle_configs(threads=None):
    """The oracle on the smaller configurations at full size: config 1 for all its 200 steps,
    config 2 (FP64) for a 10-step sample of its 5000."""
    threads = threads or os.cpu_count() or 1
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = str(threads)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    out = {}
    for name, steps in ORACLE_CONFIG_STEPS.items():
        code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
                f"bench.oracle_config_worker({name!r}, {steps})")
        res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
        if res.returncode != 0:
            out[name] = {"error": res.stderr[-300:]}
            continue
        r = json.loads(res.stdout.strip().splitlines()[-1])
        out[name] = {"kind": "oracle", "mlups": r["mlups"], "steps": steps, "seconds": r["seconds"],
                     "cores": threads}
    return out


def _oracle_timing(threads, grid, steps):
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = str(threads)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"bench.cpu_baseline_worker({grid[0]}, {grid[1]}, {grid[2]}, {steps})")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if res.returncode != 0:
        return None, res.stderr[-500:]
    return json.loads(res.stdout.strip().splitlines()[-1]), None


def run_cpu_baseline(threads=None):
    """The oracle on all host cores (the reported baseline) and, on a sixteenth of the slab, on one
    core (BLAS threads = 1)."""
    threads = threads or os.cpu_count() or 1
    out, err = _oracle_timing(threads, CPU_SAMPLE_GRID, CPU_SAMPLE_STEPS)
    if out is None:
        return {"value": None, "unit": UNIT, "cores": threads, "kind": "oracle", "error": err}
    one_grid = (CPU_SAMPLE_GRID[0] // 4, CPU_SAMPLE_GRID[1] // 4, CPU_SAMPLE_GRID[2])
    one, _ = _oracle_timing(1, one_grid, CPU_SAMPLE_STEPS)
    return {"value": out["mlups"], "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"FP64 numpy oracle, {CPU_SAMPLE_STEPS} steps of the same rD3Q53 Taylor-Green workload on a "
                       f"{CPU_SAMPLE_GRID[0]}x{CPU_SAMPLE_GRID[1]}x{CPU_SAMPLE_GRID[2]} periodic slab of the benchmark "
                       f"grid ({out['seconds']:.1f} s; BLAS threads = cores)"),
            "single_core": None if one is None else {
                "value": one["mlups"], "unit": UNIT, "cores": 1,
                "sample": f"{CPU_SAMPLE_STEPS} steps on {one_grid[0]}x{one_grid[1]}x{one_grid[2]} ({one['seconds']:.1f} s)"}}


def reference_worker(steps, warmup, budget_s):
    """The reference arm: the FP64 oracle, as it stands, advancing a slab of the benchmark grid by
    one time step per benchmark step. The slab is sized from a one-step calibration so that the
    W + K steps fit the budget. Prints one JSON object."""
    from oracle import lattice as OL
    from oracle import mrt as OM
    from paper_2512_16230_gb300 import inputs as I
    from paper_2512_16230_gb300 import workloads as W
    wl = W.taylor_green_3d(n=GRID, steps=1)
    spec = wl.lattice
    lat = OL.build(spec.kind, spec.c, spec.cs2, spec.free_w)

    def slab(nz):
        n = (GRID[0], GRID[1], nz)
        m = OM.Model(lat, "nse", n, wl.s, wl.s_high)
        rho, u = I.taylor_green_3d(n, spec.c, wl.init["u0"], 1.0, spec.cs2[0])
        m.init_fields(rho, u)
        return n, m

    n, m = slab(2)
    t0 = time.perf_counter()
    m.step(1)
    per_cell = (time.perf_counter() - t0) / math.prod(n)
    cells = max(2 * 2 * 2, int(budget_s / max(steps + warmup, 1) / per_cell))
    nz, ny = 2, GRID[1]
    while GRID[0] * ny * nz * 2 <= cells and nz < GRID[2]:
        nz *= 2
    while GRID[0] * ny * nz > cells and ny > 2:
        ny //= 2
    n = (GRID[0], ny, nz)
    m = OM.Model(lat, "nse", n, wl.s, wl.s_high)
    rho, u = I.taylor_green_3d(n, spec.c, wl.init["u0"], 1.0, spec.cs2[0])
    m.init_fields(rho, u)
    m.step(warmup)
    t0 = time.perf_counter()
    m.step(steps)
    dt = time.perf_counter() - t0
    print(json.dumps({"mlups": math.prod(n) * steps / dt / 1e6, "seconds": dt, "n": list(n)}))


def bench_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = str(threads)
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"bench.reference_worker({args.steps}, {args.warmup}, {REF_BUDGET_S})")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if res.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + res.stderr[-300:]}))
        return
    out = json.loads(res.stdout.strip().splitlines()[-1])
    n = out["n"]
    sample = (f"FP64 numpy oracle, {args.warmup} + {args.steps} time steps of the rD3Q53 Taylor-Green workload "
              f"on a {n[0]}x{n[1]}x{n[2]} periodic block of the benchmark grid per benchmark step "
              f"({out['seconds']:.1f} s timed, BLAS threads = {threads})")
    base = {"value": out["mlups"], "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
    line = {"impl": "reference", "metric": METRIC, "value": out["mlups"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * out["seconds"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (analytic Taylor-Green initial field)",
            "config": _config({"reference": "FP64 numpy oracle on the host cores (the paper has no code)"}),
            "cpu_baseline": base, "e2e": {"value": out["mlups"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2512_16230_gb300 import build as B
    from paper_2512_16230_gb300 import lbm

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    lbm.load()
    grid = tuple(args.grid)
    wl = _workload(grid, args.store)
    spec = wl.lattice
    cells = wl.ncells
    lat = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
    stream = torch.cuda.current_stream(dev)
    model = lbm.Model(lat, "nse", wl.n, store=args.store, stream=stream.cuda_stream)
    model.set_relaxation(wl.s, wl.s_high)
    if args.tensor_cores:
        model.set_tensor_cores(1)
    rho, u = wl.fields()
    rho_d = torch.from_numpy(rho).to(dev)
    u_d = torch.from_numpy(np.ascontiguousarray(u)).to(dev)
    model.init_fields(rho_d, u_d)
    model.step(args.warmup)
    model.synchronize()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = str(local)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid) as clocks:
        barrier()
        _, launches0 = model.counters()
        start.record(stream)
        model.step(args.steps)
        end.record(stream)
        barrier()
    _, launches1 = model.counters()
    ms = start.elapsed_time(end)
    sums = model.conserved_sums()
    ms_max = reduce_max(ms, ws, dev)
    value = job_throughput(cells, args.steps, ws, ms_max / 1e3)
    launch_ms = ms / args.steps

    # end to end through the public API: pinned host fields in, K steps, pinned host fields out
    rho_h = torch.from_numpy(rho).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    barrier()
    t0 = time.perf_counter()
    model.init_fields(rho_h.numpy(), u_h.numpy())
    model.step(args.steps)
    model.read_fields(rho_o.numpy(), u_o.numpy())
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value = job_throughput(cells, args.steps, ws, reduce_max(e2e_s, ws, dev))
    io_bytes = (rho_h.numel() + u_h.numel()) * 8

    # the full Q x Q collision with one rate per order >= 4 on the same solve: the CUDA-core
    # kernel with explicit higher rows (k_step_high), then the higher rows on tcgen05
    model.set_high_rates([HIGH_RATES[k] for k in sorted(HIGH_RATES)])
    vsteps = min(args.steps, VARIANT_STEPS)
    v0 = torch.cuda.Event(enable_timing=True)
    v1 = torch.cuda.Event(enable_timing=True)

    def time_steps(mdl):
        mdl.step(3)
        barrier()
        v0.record(stream)
        mdl.step(vsteps)
        v1.record(stream)
        barrier()
        return v0.elapsed_time(v1) / vsteps

    model.set_tensor_cores(0)
    high_ms = time_steps(model)
    high_tc_ms = None
    if args.store != "f64":
        model.set_tensor_cores(1)
        high_tc_ms = time_steps(model)

    if rank == 0:
        peak, peak_src = _peaks()
        algo_bytes = 2 * Q * STORE_DTYPE[args.store][1] * cells
        achieved = algo_bytes / (launch_ms / 1e3) / 1e9
        traffic, sha = _profile_traffic(cells)
        if args.store != "f32" or args.tensor_cores:
            traffic = None
        cpu = run_cpu_baseline() if (ws == 1 and not args.no_cpu_baseline) else None
        if grid != GRID:
            traffic = None
        csum = clocks.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": STORE_DTYPE[args.store][0], "data": "synthetic (analytic Taylor-Green initial field)",
            "config": _config(grid=grid, store=args.store),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                         "kernel": _kernel_name(args, grid) + " (fused pull-gather, collide, store)",
                         "algorithmic_bytes_per_launch": algo_bytes, "launch_ms": launch_ms},
            "clocks": {k: csum[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes / args.steps,
                    "d2h_bytes_per_step": io_bytes / args.steps,
                    "definition": "one solve through the C ABI: pinned host fields in, K steps, pinned host fields out"},
            "gpu_launches": int(launches1 - launches0),
            "mass_sum": float(sums[0]),
            "variants": {
                "high_order_rates": {
                    "kernel": "k_step_high<rD3Q53, f32, NSE> (explicit rows of order >= 4, one rate per order)",
                    "rates": {str(k): v for k, v in HIGH_RATES.items()}, "steps": vsteps,
                    "ms_per_step": high_ms, "mlups": cells / high_ms / 1e3,
                    "hbm_frac": algo_bytes / (high_ms / 1e3) / 1e9 / peak},
                "high_order_rates_tensor_cores": None if high_tc_ms is None else {
                    "kernel": "k_step_tc32_high<rD3Q53, NSE> (CUDA-core reduced form + higher rows on tcgen05, "
                              "FP16 high/low splits)",
                    "rates": {str(k): v for k, v in HIGH_RATES.items()}, "steps": vsteps,
                    "ms_per_step": high_tc_ms, "mlups": cells / high_tc_ms / 1e3,
                    "hbm_frac": algo_bytes / (high_tc_ms / 1e3) / 1e9 / peak},
            },
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
    model.close()
    del model
    torch.cuda.empty_cache()
    # the same variant with FP16-deviation storage, where its dense higher rows run on tcgen05
    m16 = lbm.Model(lat, "nse", wl.n, store="f16_dev", stream=stream.cuda_stream)
    m16.set_relaxation(wl.s, wl.s_high)
    m16.set_high_rates([HIGH_RATES[k] for k in sorted(HIGH_RATES)])
    m16.init_fields(rho_d, u_d)
    high16_ms = time_steps(m16)
    m16.close()
    del m16
    torch.cuda.empty_cache()
    if rank == 0:
        line["variants"]["high_order_rates_f16_tensor_cores"] = {
            "kernel": "k_step_rows_tc<rD3Q53, f16_dev, NSE, higher rows> (row-staged, tcgen05 products with the "
                      "dense higher rows)",
            "rates": {str(k): v for k, v in HIGH_RATES.items()}, "steps": vsteps,
            "ms_per_step": high16_ms, "mlups": cells / high16_ms / 1e3,
            "hbm_frac": 2 * Q * 2 * cells / (high16_ms / 1e3) / 1e9 / peak}
    # the same workload with 16-bit deviation storage (the reduced-precision configuration): FP16
    # and BF16 on the CUDA cores, FP16 with the contractions on tcgen05
    for key, store, tc, gather, kern in (
            ("f16_deviations", "f16_dev", 0, "auto",
             "k_step_rows<rD3Q53, f16_dev, NSE> (source x-rows staged in shared memory by cp.async)"),
            ("bf16_deviations", "bf16_dev", 0, "auto", "k_step_rows<rD3Q53, bf16_dev, NSE>"),
            ("f16_deviations_thread_gather", "f16_dev", 0, "threads",
             "k_step<rD3Q53, f16_dev, NSE> (per-thread gather from global memory)"),
            ("f16_deviations_tensor_cores", "f16_dev", 1, "auto",
             "k_step_rows_tc<rD3Q53, f16_dev, NSE> (row-staged, contractions on tcgen05)"),
            ("f16_deviations_tensor_cores_thread_gather", "f16_dev", 1, "threads",
             "k_step_tc<rD3Q53, f16_dev, NSE> (per-thread gather, contractions on tcgen05)")):
        mr = lbm.Model(lat, "nse", wl.n, store=store, stream=stream.cuda_stream)
        mr.set_relaxation(wl.s, wl.s_high)
        mr.set_tensor_cores(tc)
        mr.set_gather(gather)
        mr.init_fields(rho_d, u_d)
        r_ms = time_steps(mr)
        mr.close()
        del mr
        torch.cuda.empty_cache()
        if rank == 0:
            line["variants"][key] = {"kernel": kern, "steps": vsteps, "ms_per_step": r_ms,
                                     "mlups": cells / r_ms / 1e3,
                                     "hbm_frac": 2 * Q * 2 * cells / (r_ms / 1e3) / 1e9 / peak}
    ext = run_extensions(lbm, args, stream, time_steps)
    if rank == 0:
        line["extensions"] = ext
    if not args.no_other_configs:
        other = run_other_configs(lbm, W_stream=stream, barrier=barrier)
        if rank == 0:
            if ws == 1 and not args.no_cpu_baseline:
                oc = run_oracle_configs()
                other["taylor_green_rD2Q25_64x48_f64"]["oracle"] = oc["taylor_green_rD2Q25_64x48_f64"]
                other["ncde_hill_rD2Q13_1024x768_f64"]["oracle"] = oc["ncde_hill_rD2Q13_1024x768"]
            line["other_configs"] = other
    if args.serving_requests > 0 and ws == 1:   # the serving leg (config 5) runs at N = 1 only
        line["serving"] = run_serving(args.serving_requests)
    if rank == 0:
        for key in ("extensions", "other_configs", "variants", "serving"):   # the long extras last
            if key in line:
                line[key] = line.pop(key)
        line["summary"] = _summary(line)   # a compact digest of the extras, at the very end
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_extensions(lbm, args, stream, time_steps):
    """The cost of the model extensions on grids larger than L2, timed like the variants: the bulk
    block of Eq. (4-27) on the benchmark workload; the single-speed rD3Q27 Taylor-Green flow on
    the same grid with the delta4 term of M2G (a density read at the 2d neighbours and one written
    per cell); the config-2 lattice (rD2Q13 NCDE) on a 4096 x 3072 grid, moment variant and the
    per-cell-rate variant with the mixed-derivative and cross-diffusion terms (phi and psi
    fields)."""
    import numpy as np
    import torch
    from paper_2512_16230_gb300 import inputs as I
    from paper_2512_16230_gb300 import workloads as W
    peak, _ = _peaks()
    out = {}

    def run(key, wl, setup, bytes_per_cell, note):
        spec = wl.lattice
        lat = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
        m = lbm.Model(lat, wl.eq, wl.n, store=wl.store, stream=stream.cuda_stream)
        m.set_relaxation(wl.s, wl.s_high)
        if wl.force is not None:
            m.set_force(*wl.force)
        if wl.u_const is not None:
            m.set_ncde(wl.u_const, wl.nonlin)
        rho, u = wl.fields()
        m.init_fields(rho, None if u is None else np.ascontiguousarray(u))
        setup(m)
        ms = time_steps(m)
        m.close()
        torch.cuda.empty_cache()
        out[key] = {"workload": note, "ms_per_step": ms, "mlups": wl.ncells / ms / 1e3,
                    "algorithmic_bytes_per_cell": bytes_per_cell,
                    "hbm_frac": bytes_per_cell * wl.ncells / (ms / 1e3) / 1e9 / peak}

    grid = tuple(args.grid)
    wl = W.taylor_green_3d(n=grid)
    run("bulk_viscosity", wl, lambda m: m.set_bulk(0.9), 2 * 53 * 4,
        f"rD3Q53 Taylor-Green {grid[0]}x{grid[1]}x{grid[2]} FP32, s_b = 0.9")
    wl = W.taylor_green_3d(n=grid, lattice="rD3Q27", re=100.0, ma=0.1)
    run("single_speed_m2g_delta4", wl, lambda m: m.set_m2g_anisotropy(1), 2 * 27 * 4 + 8,
        f"rD3Q27 Taylor-Green {grid[0]}x{grid[1]}x{grid[2]} FP32 with the delta4 term of M2G")
    nc = (4096, 3072)
    wl = W.ncde_hill(n=nc, sigma=80.0)
    run("ncde_moment", wl, lambda m: None, 2 * 13 * 4 + 8,
        f"rD2Q13 nonlinear CDE {nc[0]}x{nc[1]} FP32, moment variant")
    psi = I.random_scalar(nc, seed=1)

    def rate_cross(m):
        m.set_ncde_variant("rate", -0.2)
        m.set_ncde_cross_diffusion(0.02, psi)
    run("ncde_rate_mixed_cross", wl, rate_cross, 2 * 13 * 4 + 8 + 4,
        f"rD2Q13 nonlinear CDE {nc[0]}x{nc[1]} FP32, per-cell rates, a1 = -0.2, cross diffusion a2 = 0.02")
    return out


def run_other_configs(lbm, W_stream, barrier):
    """The smaller configurations at full size, timed the same way (CUDA events over a run of
    steps): the rD2Q13 nonlinear CDE hill (1024 x 768, FP32 and FP64, the full 5000 steps; 104 or
    208 B of populations plus 8 or 16 B of phi history per cell update) and the rD2Q25
    Taylor-Green vortex (64 x 48, FP64, 200 steps). The FP32 hill (82 MB of state) and the vortex
    (1.2 MB) stay resident in L2, so their hbm_frac is not an HBM measurement (l2_resident marks
    them); the FP64 hill (164 MB) is bound by the FP64 pipe, not by HBM."""
    import numpy as np
    import torch
    from paper_2512_16230_gb300 import workloads as W
    peak, _ = _peaks()
    l2_bytes = getattr(torch.cuda.get_device_properties(torch.cuda.current_device()), "L2_cache_size", 126 << 20)
    out = {}
    cases = [("ncde_hill_rD2Q13_1024x768_f32", W.ncde_hill(store="f32"), 4),
             ("ncde_hill_rD2Q13_1024x768_f64", W.ncde_hill(store="f64"), 8),
             ("taylor_green_rD2Q25_64x48_f64", W.taylor_green_2d(), 8)]
    for name, wl, nbytes in cases:
        spec = wl.lattice
        lat = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
        m = lbm.Model(lat, wl.eq, wl.n, store=wl.store, stream=W_stream.cuda_stream)
        m.set_relaxation(wl.s, wl.s_high)
        if wl.u_const is not None:
            m.set_ncde(wl.u_const, wl.nonlin)
        rho, u = wl.fields()
        m.init_fields(rho, None if u is None else np.ascontiguousarray(u))
        m.step(10)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a.record(W_stream)
        m.step(wl.steps)
        b.record(W_stream)
        barrier()
        ms = a.elapsed_time(b) / wl.steps
        per_cell = 2 * lat.Q * nbytes + (2 * nbytes if wl.eq == "ncde" else 0)
        state = (2 * lat.Q + (1 if wl.eq == "ncde" else 0)) * nbytes * wl.ncells
        out[name] = {"steps": wl.steps, "ms_per_step": ms, "mlups": wl.ncells / ms / 1e3,
                     "algorithmic_bytes_per_cell": per_cell, "state_bytes": state,
                     "l2_resident": bool(state < l2_bytes),
                     "hbm_frac": per_cell * wl.ncells / (ms / 1e3) / 1e9 / peak}
        m.close()
    return out


SERVING_PRECISION_GRID = {"tgv2d": (256, 192), "ncde": (256, 192), "kolmogorov": (64, 64, 64)}
SERVING_PRECISION_STEPS = 1000


def serving_precision(lbm, S):
    """Per served class, the relative L2 error of u (or phi) after 1000 steps in FP32 and in FP16
    deviation storage against the library's FP64 path (pinned to the FP64 oracle at 1e-12 by the
    parity tests), on a mid-size grid of the class, with the class's FP16 threshold."""
    import numpy as np
    import torch
    from paper_2512_16230_gb300 import workloads as W
    out = {}
    for flow, lat in S.SERVING_CLASSES:
        req = dict(rid=0, flow=flow, lattice=lat, grid=SERVING_PRECISION_GRID[flow], steps=SERVING_PRECISION_STEPS,
                   seed=7, store="16bit")
        fields = {}
        for store in ("f64", "f32", "f16_dev"):
            wl = W.serving_workload(req, store)
            spec = wl.lattice
            m = lbm.Model(lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w), wl.eq, wl.n, store=store)
            m.set_relaxation(wl.s, wl.s_high)
            if wl.force is not None:
                m.set_force(*wl.force)
            if wl.u_const is not None:
                m.set_ncde(wl.u_const, wl.nonlin)
            rho, u = wl.fields()
            m.init_fields(rho, None if u is None else np.ascontiguousarray(u))
            m.step(wl.steps)
            r, v = m.read_fields()
            fields[store] = v if wl.eq == "nse" else r
            m.close()
        torch.cuda.empty_cache()
        ref = fields["f64"]

        def err(a):
            return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
        out[f"{flow}|{lat}"] = {"grid": list(req["grid"]), "steps": SERVING_PRECISION_STEPS,
                                "quantity": "u" if flow != "ncde" else "phi",
                                "f32": err(fields["f32"]), "f16_dev": err(fields["f16_dev"]),
                                "f16_max_steps": S.F16_MAX_STEPS[flow, lat]}
    return out


SERVING_LARGE_STEP_BYTES = 5e8   # serve_batched: requests moving this much per step run one at a time


def run_serving(n_requests, rate_per_s=20.0, seed=0, sustained_requests=300, large_step_bytes=SERVING_LARGE_STEP_BYTES):
    """Config 5: the seeded request stream at its stated size, served by continuous batching
    (policy "f16_dev": FP16 deviations only where the class and run length keep the error within
    1e-3, FP32 otherwise; launch shapes from the autotuner; large requests one at a time with the
    small ones admitted beside them) and by the plain FP32 one-solve-at-a-time path,
    same requests and arrival times (20 arrivals/s, more than either path serves: solves/s is the
    capacity). Then both paths on a shorter stream arriving at 0.8 x the smaller capacity, where
    p50/p99 measure service rather than queueing. Also the per-class errors."""
    from paper_2512_16230_gb300 import autotune
    from paper_2512_16230_gb300 import inputs as I
    from paper_2512_16230_gb300 import lbm
    from paper_2512_16230_gb300 import serve as S

    def both(reqs, tuning):
        eng = S.GpuEngine(tuning=tuning)
        rec_b, t_b = S.serve_batched(reqs, eng, budget_bytes=150e9, max_resident=512, tick=64,
                                     store_policy="f16_dev", large_step_bytes=large_step_bytes)
        launches = eng.batch.counters()["launches"]
        eng.close()
        b = dict(S.summarize(rec_b, t_b), batched_launches=launches, hbm_budget_gb=150,
                 peak_resident_gb=S.serve_batched.peak_bytes / 1e9,
                 f16_requests=sum(r.store == "f16_dev" for r in rec_b))
        seq = S.GpuEngine()
        rec_s, t_s = S.serve_sequential(reqs, seq, store="f32")
        seq.close()
        return b, S.summarize(rec_s, t_s)

    reqs = I.serving_requests(n_requests, seed=seed, rate_per_s=rate_per_s)
    tuning = autotune.autotune()
    b, q = both(reqs, tuning)
    rate2 = 0.8 * min(b["solves_per_s"], q["solves_per_s"])
    reqs2 = I.serving_requests(sustained_requests, seed=seed + 1, rate_per_s=rate2)
    b2, q2 = both(reqs2, tuning)
    groups = {}
    for key, ms in tuning["ms_per_step"].items():
        if "|tile=" in key:
            g = key.split("|tile=")[0]
            lo, hi = groups.get(g, (ms, ms))
            groups[g] = (min(lo, ms), max(hi, ms))
    return {
        "requests": n_requests, "arrival_rate_per_s": rate_per_s, "seed": seed,
        "mix": "2D rD2Q17/21/25 Taylor-Green + NCDE (32..1024 x 32..768), 3D rD3Q33/45/53 Kolmogorov "
               "(32^3..160^3), 200..5000 steps, Poisson arrivals",
        "batched": dict(b, storage="policy f16_dev: FP16 deviations where the class and run length keep the "
                                   "u (phi) error <= 1e-3, FP32 otherwise",
                  admission="arrival order; requests moving >= large_step_bytes per step one at a time, smaller "
                            "ones admitted past a waiting large one", large_step_bytes=large_step_bytes,
                  engine="one persistent work-list launch per (lattice, storage, equation) group and step, each "
                         "group on its own stream; solves of >= solo_cells cells on the single-solve kernels on "
                         "another stream; all forked from and joined back into the batch stream per call; "
                         "8-step chunks replayed from a CUDA graph"),
        "sequential_fp32": q,
        "speedup_solves_per_s": b["solves_per_s"] / q["solves_per_s"],
        "sustained": {"requests": sustained_requests, "seed": seed + 1, "arrival_rate_per_s": rate2,
                      "batched": b2, "sequential_fp32": q2},
        "errors_vs_fp64": serving_precision(lbm, S),
        "tuning": dict(autotune.summary(tuning),
                       group_ms_best_worst={g: [round(v[0], 4), round(v[1], 4)] for g, v in groups.items()},
                       solo_ms={k: round(v, 4) for k, v in tuning["ms_per_step"].items() if k.startswith("solo_cells=")}),
    }


def _summary(line):
    """The figures of the long extras that matter most, rounded: the per-step time and HBM
    fraction (algorithmic bytes over the measured copy bandwidth) of each kernel variant on the
    benchmark solve, and the serving comparison (config 5)."""
    var = {k: v for k, v in line.get("variants", {}).items() if isinstance(v, dict) and "ms_per_step" in v}
    out = {"variants_ms_per_step": {k: round(v["ms_per_step"], 4) for k, v in var.items()},
           "variants_hbm_frac": {k: round(v["hbm_frac"], 3) for k, v in var.items() if "hbm_frac" in v}}
    sv = line.get("serving")
    if sv and "batched" in sv:
        b, q = sv["batched"], sv["sequential_fp32"]
        out["serving"] = {
            "requests": sv["requests"],
            "solves_per_s": [round(b["solves_per_s"], 3), round(q["solves_per_s"], 3)],
            "p50_s": [round(b["latency_p50_s"], 3), round(q["latency_p50_s"], 3)],
            "p99_s": [round(b["latency_p99_s"], 3), round(q["latency_p99_s"], 3)],
            "order": "batched (size-aware admission, f16_dev policy), plain FP32 one at a time",
        }
        st = sv.get("sustained")
        if st:
            out["serving"]["sustained"] = {
                "arrival_rate_per_s": round(st["arrival_rate_per_s"], 3),
                "p50_s": [round(st["batched"]["latency_p50_s"], 3), round(st["sequential_fp32"]["latency_p50_s"], 3)],
                "p99_s": [round(st["batched"]["latency_p99_s"], 3), round(st["sequential_fp32"]["latency_p99_s"], 3)],
            }
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests of the seeded serving mix (config 5) served after the step benchmark; 0 skips")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the full-size runs of the smaller configurations (profiling commands)")
    ap.add_argument("--store", choices=sorted(STORE_DTYPE), default="f32",
                    help="population storage (the benchmark is FP32; 16-bit deviations for the reduced-precision path)")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="16-bit storage only: the collision's contractions on tcgen05 (k_step_tc)")
    ap.add_argument("--grid", type=int, nargs=3, default=list(GRID),
                    help="grid for a smaller profiling case (the benchmark workload is 256 256 192)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
