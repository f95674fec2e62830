#!/usr/bin/env python3
"""Throughput benchmark of the fused thermal lattice Boltzmann step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A "step" is one time step of the whole hot path (pull streaming with the wall
rules, macros, flow MRT with Guo forcing, thermal MRT, store) over the whole
cell.  Headline workload: 2D Rayleigh-Benard, D2Q9 + D2Q5, 8193 x 8193 nodes,
FP32 storage, Ra = 1e8, Pr = 0.71, Ma = 0.1, seeded conductive start with
noise 1e-3.  Further lines of the same run (FP16/BF16-offset storage, the 385^3
D3Q19 + D3Q7 cube, FP64) are reported under "variants".

GLUPS = nodes x steps / seconds / 1e9 (real nodes only).  Device time comes from
CUDA events on the library's stream around the timed steps; the population
buffers (>= 7 GB) are far larger than L2, so every step streams from HBM.
With N > 1 (torchrun) every rank runs an independent replica of the workload
(replicas only: the method's multi-GPU domain decomposition is not part of this
build) and `value` is the sum over ranks divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle (oracle/) on the host cores on a
bounded sample of the same workload; it is the only other place this script
runs the oracle besides the cpu_baseline leg.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("GLUPS & % HBM roofline, 8193² D2Q9+D2Q5 / 385³ D3Q19+D3Q7, "
          "FP16-store vs FP32")
# algorithmic bytes per lattice update: every population read once, written once
BYTES_PER_LU = {(2, "fp64"): 224, (2, "fp32"): 112, (2, "fp16"): 56, (2, "bf16"): 56,
                (3, "fp64"): 416, (3, "fp32"): 208, (3, "fp16"): 104, (3, "bf16"): 104}
# FP64 operations the FP64 storage step executes per lattice update (ncu:
# smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on per node on
# 1025^2 / 129^3; FLOP counts a DFMA as 2).  The FP64 build is compiled without
# FMA contraction (oracle parity to 1e-12), so nearly every operation is its own
# FP64 instruction: the roof of that mix is the FP64 pipe's instruction rate.
FP64_OPS_PER_LU = {2: {"dadd": 121.5, "dmul": 90.8, "dfma": 5.3}, 3: {"dadd": 288.2, "dmul": 193.5, "dfma": 6.2}}
KERNEL_SOURCES = ["paper_2211_03160_gb300/csrc/kernels.cuh", "paper_2211_03160_gb300/csrc/lattice.cuh",
                  "paper_2211_03160_gb300/csrc/dispatch.h", "paper_2211_03160_gb300/csrc/step_2d_f32.cu",
                  "paper_2211_03160_gb300/csrc/step_2d_f16.cu", "paper_2211_03160_gb300/csrc/step_3d_f32.cu",
                  "paper_2211_03160_gb300/csrc/step_3d_f16.cu", "paper_2211_03160_gb300/csrc/step_fp64.cu",
                  "paper_2211_03160_gb300/csrc/staged.cuh", "paper_2211_03160_gb300/csrc/step_staged.cu"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def ncu_traffic(name: str):
    """DRAM bytes per launch from the committed ncu summary for this kernel and
    workload, or None if absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", f"{name}.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as fh:
        for ln in fh:
            if ":" in ln:
                k, v = ln.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != kernel_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ distributed

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist

    backend = "nccl" if os.environ.get("TLBM_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), int(os.environ.get("LOCAL_RANK", "0"))


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v: float, ws: int, device=None) -> float:
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ workloads

def workload(name: str):
    """(dim, nx, ny, nz, Ra, precision name, seed) of a named workload; a name
    ending in "_inplace" is the same workload with in-place streaming, one
    ending in "_side" the paper's side-heated cavity instead of the
    Rayleigh-Benard cell."""
    name = name.removesuffix("_inplace").removesuffix("_side")
    table = {
        "2d_8193_fp32": (2, 8193, 8193, 1, 1e8, "fp32", 2),
        "2d_8193_fp16": (2, 8193, 8193, 1, 1e8, "fp16", 2),
        "2d_8193_bf16": (2, 8193, 8193, 1, 1e8, "bf16", 2),
        "2d_8193_fp64": (2, 8193, 8193, 1, 1e8, "fp64", 2),
        "3d_385_fp64": (3, 385, 385, 385, 1e7, "fp64", 3),
        "3d_385_fp32": (3, 385, 385, 385, 1e7, "fp32", 3),
        "3d_385_fp16": (3, 385, 385, 385, 1e7, "fp16", 3),
        "3d_385_bf16": (3, 385, 385, 385, 1e7, "bf16", 3),
        # smaller cases of the same physics for profiler captures (still > L2)
        "2d_4097_fp32": (2, 4097, 4097, 1, 1e8, "fp32", 2),
        "2d_4097_fp16": (2, 4097, 4097, 1, 1e8, "fp16", 2),
        "3d_257_fp32": (3, 257, 257, 257, 1e7, "fp32", 3),
        "3d_257_fp16": (3, 257, 257, 257, 1e7, "fp16", 3),
    }
    return table[name]


def inplace(name: str) -> bool:
    return name.endswith("_inplace")


def side_heated(name: str) -> bool:
    return name.endswith("_side")


def describe(name: str) -> str:
    dim, nx, ny, nz, Ra, prec, seed = workload(name)
    how = ", in-place (AA) streaming in one buffer" if inplace(name) else ""
    if side_heated(name):
        return (f"2D side-heated cavity D2Q9+D2Q5 {nx}x{ny}, {prec.upper()} storage, Ra={Ra:g}, Pr=0.71, Ma=0.1, "
                f"seed {seed}, noise 1e-3")
    if dim == 2:
        return (f"2D Rayleigh-Benard D2Q9+D2Q5 {nx}x{ny}, {prec.upper()} storage, Ra={Ra:g}, Pr=0.71, Ma=0.1, "
                f"seed {seed}, noise 1e-3{how}")
    return (f"3D Rayleigh-Benard cube D3Q19+D3Q7 {nx}x{ny}x{nz}, {prec.upper()} storage, Ra={Ra:g}, Pr=0.71, "
            f"Ma=0.1, seed {seed}, noise 1e-3{how}")


def run_gpu(name: str, steps: int, warmup: int, ws: int, device_index: int, e2e: bool):
    import numpy as np
    import torch

    from paper_2211_03160_gb300 import tlbm

    dim, nx, ny, nz, Ra, prec, seed = workload(name)
    lattice = tlbm.TLBM_D2Q9_D2Q5 if dim == 2 else tlbm.TLBM_D3Q19_D3Q7
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = tlbm.Sim(nx, ny, nz, lattice=lattice, Ra=Ra, Pr=0.71, Ma=0.1, precision=tlbm.PRECISIONS[prec],
                       stream=stream,
                       streaming=tlbm.TLBM_STREAM_INPLACE if inplace(name) else tlbm.TLBM_STREAM_PULL,
                       walls=tlbm.TLBM_SIDE_HEATED if side_heated(name) else tlbm.TLBM_RB)
        sim.init(seed, 1e-3)
        _, mass0 = sim.energy()
        sim.step(warmup)
        stream.synchronize()
        nodes = nx * ny * nz
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize()
        launches0 = sim.launches
        with ClockSampler(device_index) as clk:
            ev0.record(stream)
            sim.step(steps)
            ev1.record(stream)
            ev1.synchronize()
        launches = sim.launches - launches0
        torch.cuda.synchronize()
        barrier(ws)
        sec = ev0.elapsed_time(ev1) / 1e3
        sec_max = max_over_ranks(sec, ws, device=torch.device("cuda", device_index) if ws > 1 else None)
        out = {
            "name": name, "nodes": nodes, "dim": dim, "prec": prec, "sec": sec, "sec_max": sec_max,
            "glups_rank": nodes * steps / sec / 1e9, "launches": launches, "clocks": clk.summary(),
            "device_bytes": sim.nbytes,
        }
        div, _ = sim.status()
        out["diverged"] = bool(div)
        out["nusselt"] = sim.nusselt()
        ekin, mass = sim.energy()
        out["ekin_per_node"] = ekin / nodes
        out["mass_drift"] = (mass - mass0) / mass0
        if e2e:
            # end to end through the public API from pinned host memory:
            # H2D of the state, `steps` steps, D2H of the reduction result
            f = torch.empty((sim.qf,) + sim.shape, dtype=torch.float64, pin_memory=True)
            g = torch.empty((sim.qg,) + sim.shape, dtype=torch.float64, pin_memory=True)
            sim.init(seed, 1e-3)
            sim.get_populations_into(f.numpy(), g.numpy())
            barrier(ws)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.set_populations(f.numpy(), g.numpy())
            sim.step(steps)
            nu = sim.nusselt()
            t1 = time.perf_counter()
            e_sec = max_over_ranks(t1 - t0, ws, device=torch.device("cuda", device_index) if ws > 1 else None)
            out["e2e"] = {"sec": e_sec, "h2d_bytes": (f.numel() + g.numel()) * 8, "d2h_bytes": 6 * 8, "nu": nu}
            del f, g
        sim.close()
        del sim
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def ensemble_draws(n: int = 64, master_seed: int = 4):
    """64-instance ensemble: square cells with N uniform in {129, 257, 513, 1025},
    log10 Ra uniform in [5, 8], Pr in {0.71, 7.0}, seeds 1000 + i."""
    import numpy as np

    r = np.random.default_rng(master_seed)
    out = []
    for i in range(n):
        N = int(r.choice([129, 257, 513, 1025]))
        Ra = float(10.0 ** r.uniform(5.0, 8.0))
        Pr = float(r.choice([0.71, 7.0]))
        out.append((N, N, 1, Ra, Pr, 0.1, 1000 + i))
    return out


def run_batch(prec: str, steps: int, warmup: int, ws: int, device_index: int) -> dict:
    """The ensemble stepped by one flattened launch per step (CUDA-graph step
    blocks) and by the persistent kernel (many steps per launch, grid barrier
    between steps) against the same 64 cells stepped by 64 separate launches per
    step."""
    import torch

    from paper_2211_03160_gb300 import tlbm

    inst = ensemble_draws()
    nodes = sum(nx * ny for nx, ny, *_ in inst)
    stream = torch.cuda.Stream()
    out = {"instances": len(inst), "nodes": nodes, "prec": prec}
    with torch.cuda.stream(stream):
        b = tlbm.Batch(inst, lattice=tlbm.TLBM_D2Q9_D2Q5, precision=tlbm.PRECISIONS[prec], stream=stream)
        b.init(1e-3)
        b.autotune(3)
        b.step(warmup)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize()
        l0 = b.launches
        ev0.record(stream)
        b.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        out["batched"] = {"sec": max_over_ranks(sec, ws, torch.device("cuda", device_index) if ws > 1 else None),
                          "launches": b.launches - l0, "variant": list(b.variant), "staged": b.staged[0],
                          "diverged": sum(b.status())}
        # the persistent form: 64 steps per cooperative launch, grid barrier between steps
        b.set_persistent(64)
        b.step(warmup)
        barrier(ws)
        torch.cuda.synchronize()
        l0 = b.launches
        ev0.record(stream)
        b.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        out["persistent"] = {"sec": max_over_ranks(sec, ws, torch.device("cuda", device_index) if ws > 1 else None),
                             "launches": b.launches - l0, "diverged": sum(b.status())}
        b.close()
        sims = [tlbm.Sim(nx, ny, nz, lattice=tlbm.TLBM_D2Q9_D2Q5, Ra=Ra, Pr=Pr, Ma=Ma,
                         precision=tlbm.PRECISIONS[prec], stream=stream) for nx, ny, nz, Ra, Pr, Ma, _ in inst]
        for s, (*_, seed) in zip(sims, inst):
            s.init(seed, 1e-3)
        for _ in range(warmup):
            for s in sims:
                s.step(1)
        barrier(ws)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            for s in sims:
                s.step(1)
        ev1.record(stream)
        ev1.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        out["separate"] = {"sec": max_over_ranks(sec, ws, torch.device("cuda", device_index) if ws > 1 else None),
                           "launches": steps * len(sims)}
        for s in sims:
            s.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def warm_start_record():
    """The learned warm start's measured gain on the 513^2 workload (16 held-out
    draws, Ra 1e6-1e8): median ratio of steps to reach the conductive run's
    steady Nusselt level, conductive / learned start, from the committed result
    of `python -m paper_2211_03160_gb300.surrogate` (a run of several minutes,
    not repeated here)."""
    p = os.path.join(ROOT, "results", "warm_start_513.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        r = json.load(fh)
    sm = r["summary"]
    rec = {"unit": "x fewer steps to steady Nu", "source": "results/warm_start_513.json (not re-run by bench.py)"}
    for k in ("coarse", "coords"):
        if k in sm and sm[k]["reach"]["median_speedup"]:
            rec[k] = round(sm[k]["reach"]["median_speedup"], 3)
            rec[k + "_faster"] = f'{sm[k]["reach"]["faster"]}/{sm[k]["reach"]["compared"]}'
    rec["value"] = rec.get("coarse", rec.get("coords"))
    return rec


_FP64_PEAK = None


def fp64_peak() -> float:
    """Measured FP64 FMA rate of this GPU (FLOP/s), taken once per run."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        from paper_2211_03160_gb300 import tlbm

        _FP64_PEAK = tlbm.tlbm_fp64_fma_rate()
    return _FP64_PEAK


def cpu_baseline(target_seconds: float = 12.0) -> dict:
    """The FP64 oracle as it stands on the host cores (OpenMP over all cores),
    on a bounded sample of the headline workload: the same physics (Ra = 1e8,
    Pr = 0.71, Ma = 0.1, RB walls, seed 2) on a 2049 x 2049 cell, stepped until
    about target_seconds have passed."""
    from oracle import oracle

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = 2049
    s = oracle.Sim(n, n, Ra=1e8, Pr=0.71, Ma=0.1)
    s.init(2, 1e-3)
    s.step(1)
    steps, t0 = 0, time.perf_counter()
    while True:
        s.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > target_seconds or steps >= 200:
            break
    s.close()
    return {"value": n * n * steps / el / 1e9, "unit": "GLUPS", "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {n}x{n} cell of the same physics, {steps} steps ({el:.1f} s), "
                      f"{oracle.get_threads()} OpenMP threads"}


def _host_available_bytes() -> int:
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def cpu_extended() -> dict:
    """The oracle's own speed at the measurement cases: one thread on the
    129^2 FP64 case (2000 steps), and all host cores on 10 steps of the 8193^2
    and 385^3 workloads (FP64, two population buffers).  A full-size case runs
    only when the host has three times its memory available."""
    from oracle import oracle

    cores = os.cpu_count() or 1
    out = {"cores": cores}
    oracle.set_threads(1)
    s = oracle.Sim(129, 129, Ra=1e5, Pr=0.71, Ma=0.1)
    s.init(1, 1e-3)
    t0 = time.perf_counter()
    s.step(2000)
    el = time.perf_counter() - t0
    s.close()
    out["129sq_fp64_1_thread_mlups"] = 129 * 129 * 2000 / el / 1e6
    oracle.set_threads(cores)
    for name, (nx, ny, nz, lattice, Ra, q) in {"8193sq": (8193, 8193, 1, oracle.D2Q9_D2Q5, 1e8, 14),
                                             "385cube": (385, 385, 385, oracle.D3Q19_D3Q7, 1e7, 26)}.items():
        need = 2 * q * 8 * nx * ny * nz
        if _host_available_bytes() < 3 * need:
            out[f"{name}_fp64_all_cores_mlups"] = None
            continue
        s = oracle.Sim(nx, ny, nz, lattice=lattice, Ra=Ra, Pr=0.71, Ma=0.1)
        s.init(2 if nz == 1 else 3, 1e-3)
        t0 = time.perf_counter()
        s.step(10)
        el = time.perf_counter() - t0
        s.close()
        out[f"{name}_fp64_all_cores_mlups"] = nx * ny * nz * 10 / el / 1e6
    return out


def run_reference(args):
    """The oracle timed as the reference arm: each step is one oracle time step
    on a 513 x 513 sample of the headline workload's physics."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = 513
    s = oracle.Sim(n, n, Ra=1e8, Pr=0.71, Ma=0.1)
    s.init(2, 1e-3)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    sec = time.perf_counter() - t0
    s.close()
    v = n * n * args.steps / sec / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe("2d_8193_fp32"), "sample": f"{n}x{n} cell of the same physics",
                   "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"FP64 oracle, {n}x{n} cell, {args.steps} timed steps after {args.warmup}"},
        "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d_8193_fp32")
    ap.add_argument("--variants", default="2d_8193_fp16,2d_8193_bf16,3d_385_fp32,3d_385_fp16,3d_385_bf16,"
                                          "2d_8193_fp64,3d_385_fp64,2d_8193_fp32_inplace,3d_385_fp16_inplace,"
                                          "2d_8193_fp32_side,batch64_fp32,batch64_fp16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time the oracle single-threaded at 129^2 and on all cores at full size")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    rank, ws, local = dist_setup()
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    peaks = measured_peaks()

    main_run = run_gpu(args.workload, args.steps, args.warmup, ws, local, e2e=not args.no_e2e)
    variants = {}
    for v in [x for x in args.variants.split(",") if x]:
        if v.startswith("batch64_"):
            st = max(10, args.steps // 4)
            r = run_batch(v.split("_")[1], st, min(args.warmup, 20), ws, local)
            bt, sp = r["batched"], r["separate"]
            bpl = BYTES_PER_LU[(2, r["prec"])]
            val = r["nodes"] * ws * st / bt["sec"] / 1e9
            variants[v] = {
                "value": round(val, 3), "frac": round(val * bpl / peaks["hbm_gbs"], 4),
                "persistent": round(r["nodes"] * ws * st / r["persistent"]["sec"] / 1e9, 3),
                "separate": round(r["nodes"] * ws * st / sp["sec"] / 1e9, 3),
                "speedup": round(sp["sec"] / bt["sec"], 3), "diverged": bt["diverged"],
                "form": f"staged{bt['staged']}" if bt["staged"] else f"vec{bt['variant'][0]}",
            }
            continue
        st = args.steps if not v.endswith("fp64") else max(10, args.steps // 10)
        if v.startswith("3d"):
            st = max(10, st // 2) if not v.endswith("fp64") else max(5, args.steps // 20)
        r = run_gpu(v, st, args.warmup if not v.endswith("fp64") else 3, ws, local, e2e=False)
        bpl = BYTES_PER_LU[(r["dim"], r["prec"])]
        glups = r["nodes"] * ws * st / r["sec_max"] / 1e9
        gbs = bpl * r["nodes"] * st / r["sec"] / 1e9
        rec = {"value": round(glups, 3), "ms": round(r["sec_max"] / st * 1e3, 4),
               "frac": round(gbs / peaks["hbm_gbs"], 4)}
        if r["prec"] == "fp64":
            # FP64 roof: the measured FMA rate (FLOP/s, 2 per DFMA) and, for the
            # kernel's uncontracted mix, the FP64 instruction rate (half of it)
            ops = FP64_OPS_PER_LU[r["dim"]]
            flop = ops["dadd"] + ops["dmul"] + 2 * ops["dfma"]
            inst = ops["dadd"] + ops["dmul"] + ops["dfma"]
            rate = r["nodes"] * st / r["sec"]
            peak = fp64_peak()
            rec["roofline"] = {"bound": "fp64", "achieved": round(flop * rate / 1e12, 4),
                               "peak": round(peak / 1e12, 4), "unit": "TFLOP/s",
                               "frac": round(flop * rate / peak, 4),
                               "pipe_frac": round(inst * rate / (peak / 2), 4)}
        if r["diverged"]:
            rec["diverged"] = True
        variants[v] = rec

    ws_rec = warm_start_record()
    if ws_rec:
        variants["warm_start_513"] = ws_rec

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
        if args.cpu_full:
            cpu["extended"] = cpu_extended()

    if rank != 0:
        return 0
    r = main_run
    steps = args.steps
    bpl = BYTES_PER_LU[(r["dim"], r["prec"])]
    achieved = bpl * r["nodes"] * steps / r["sec"] / 1e9
    traffic = ncu_traffic(f"step_{r['dim']}d_{r['prec']}_{workload(args.workload)[1]}")
    line = {
        "metric": METRIC,
        "value": r["nodes"] * ws * steps / r["sec_max"] / 1e9,
        "unit": "GLUPS",
        "n_gpus": ws,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": r["sec_max"] / steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16-offset storage, f32 compute", "bf16": "bf16-offset storage, f32 compute",
                  "fp64": "f64"}[r["prec"]],
        "data": "synthetic",
        "config": {"workload": describe(args.workload), "nodes": r["nodes"],
                   "l2": "inputs larger than L2 (population buffers >= 7 GB per replica)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"],
                     "bytes_per_lu": bpl,
                     "traffic": traffic},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "nusselt": r["nusselt"],
        "ekin_per_node": r["ekin_per_node"],
        "mass_drift": r["mass_drift"],
        "diverged": r["diverged"],
        "variants": variants,
        "variant_keys": "value GLUPS; ms per step; frac = algorithmic bytes / time / measured HBM copy peak; "
                        "batch: persistent / separate = GLUPS of the persistent form / of 64 separate launches",
    }
    if "e2e" in r:
        e = r["e2e"]
        line["e2e"] = {"value": r["nodes"] * ws * steps / e["sec"] / 1e9, "unit": "GLUPS",
                       "h2d_bytes_per_step": e["h2d_bytes"] / steps, "d2h_bytes_per_step": e["d2h_bytes"] / steps}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
