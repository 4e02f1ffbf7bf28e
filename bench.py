"""Benchmark of the multi-phase SPH relaxation step (arXiv 1906.07925).

Metric: particle-updates/s (one particle advanced by one full relaxation step:
cell list, density + pressure + surface tension, time step, viscous force,
integration, projection). Default workload: the 3D unit cube minus a ball
r = 0.25, graded spacing s = 0.004 + 0.03 dist, 8,388,608 particles, 256
colours, FP32 with split-precision positions.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c1]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

One JSON line on stdout (rank 0). Multi-GPU runs (torchrun) are independent
replicas of the workload, one per GPU (weak scaling; no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "particle-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "c3": dict(desc="3D [0,1]^3 minus ball r=0.25, s=0.004+0.03*dist (graded), 8,388,608 particles, 256 colours, "
                    "FP32 split-precision, seed 2",
               dim=3, n=1 << 23, ncol=256, precision="fp32", seed=2,
               make=lambda n, c: W.graded_inclusion_3d(n, c, rho_scale=0.0)),
    "c2": dict(desc="2D [0,1]^2 minus disk r=0.2, s=0.002+0.02*dist (graded), 1,048,576 particles, 64 colours, "
                    "FP32 split-precision, seed 1",
               dim=2, n=1 << 20, ncol=64, precision="fp32", seed=1,
               make=lambda n, c: W.graded_hole_2d(n, c, rho_scale=0.0)),
    "c1": dict(desc="2D unit square, uniform, 4,096 particles (64x64 lattice + 0.3 jitter), 4 colours, FP64, seed 0",
               dim=2, n=4096, ncol=4, precision="fp64", seed=0,
               make=lambda n, c: W.uniform_square_2d(64, c)),
}

# algorithmic DRAM bytes per particle and launch (FP32 split precision)
ALG_BYTES = {"pass_a": 44, "pass_b": 72, "cells": 84}
ALG_BYTES_FP64 = {"pass_a": 72, "pass_b": 120, "cells": 100}
CELL_BYTES_PER_CELL = 12  # scan: read counts twice, write starts
KERNELS_PER_STEP = 8      # count, 3 scan, scatter, gather, pass A, pass B


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle --
def oracle_workload_sample(wl, target_n=None):
    """A bounded sample of the workload for the FP64 oracle: the particles of a
    sub-box of the same field at the workload's density (so the neighbour
    counts match the full run). Returns (problem, pos, col, description)."""
    n_full, dim = wl["n"], wl["dim"]
    p = wl["make"](n_full, wl["ncol"])
    if wl["n"] == 4096 and wl["dim"] == 2:
        pos, col, _ = W.lattice_jitter_2d(p, 64, 0.3, 0)
        return p, pos, col, f"full workload ({len(pos)} particles)"
    target_n = target_n or (60000 if dim == 2 else 30000)
    p.rho_scale = W.rho_scale_for(p, n_full, res=1024 if dim == 2 else 128)
    c0 = 0.5 + (0.2 if dim == 2 else 0.25) * 0.8  # just outside the inner boundary
    side = 0.3
    for _ in range(40):
        lo = [c0] * dim
        hi = [min(1.0, c0 + side)] * dim
        q = p.copy(lo=lo + [0.0] * (3 - dim), hi=hi + [0.0] * (3 - dim))
        n_est = p.rho_scale / W.rho_scale_for(q, 1, res=256 if dim == 2 else 48)
        if abs(n_est / target_n - 1) < 0.15:
            break
        side *= (target_n / n_est) ** (1.0 / dim)
    q.rho_scale = p.rho_scale
    pos, col, _ = W.sample_density(q, int(n_est), wl["seed"])
    desc = (f"sub-box [{c0:.3f}, {c0 + side:.3f}]^{dim} of the workload field at the workload's density "
            f"({len(pos)} particles)")
    return q, pos, col, desc


def oracle_time(q, pos, col, steps):
    """Seconds per oracle step (FP64, OpenMP over the host cores), list per step."""
    import oracle
    oracle.build()
    x = pos
    out = []
    for s in range(steps):
        t0 = time.perf_counter()
        x, _, _ = oracle.step(q, x, col, s, want=False)
        out.append(time.perf_counter() - t0)
    return out, oracle.num_threads()


# ---------------------------------------------------------------- GPU arm --
def run_gpu(args, wl, rank, world):
    import torch
    import torch.distributed as dist
    from paper_1906_07925_gb300 import Relaxation

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    p = wl["make"](wl["n"], wl["ncol"])
    n = wl["n"]
    t_setup = time.perf_counter()
    r = Relaxation(p, n, wl["ncol"], precision=wl["precision"], seed=wl["seed"] + 1000 * rank, use_graph=True,
                   skin=args.skin)
    torch.cuda.synchronize()
    log(f"[rank {rank}] create {time.perf_counter() - t_setup:.2f}s, grid {r.grid()['n_levels']} levels")
    stream = r.stream
    r.step(args.warmup)
    r.sync()

    def barrier():
        if world > 1:
            dist.barrier()

    clocks = ClockSampler(dev)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    st = r.stats()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = world * n * args.steps / (ms / 1e3)

    # per-kernel device time over a second timed run (direct launches, events
    # on the handle's stream around each phase)
    kprof = min(args.steps, 10)
    ph = r.step_profiled(kprof)
    phase_ms = {"cells": ph[0] / kprof, "pass_a": ph[1] / kprof, "pass_b": ph[2] / kprof}

    # end to end through the public API with host buffers: upload the state
    # from pinned memory, K steps, read positions and stats back
    d = wl["dim"]
    xh = torch.empty((n, d), dtype=torch.float64, pin_memory=True)
    ch = torch.empty((n,), dtype=torch.uint8, pin_memory=True)
    xh.numpy()[:] = r.positions()
    ch.numpy()[:] = r.colors()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r.set_state(xh.numpy(), ch.numpy())
    r.step(args.steps)
    lib = r.lib
    rc = lib.sph_get_positions(r.h, xh.data_ptr(), 0)
    st2 = r.stats()
    e2e_s = time.perf_counter() - t0
    assert rc == 0
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * n * args.steps / e2e_s, "unit": METRIC,
           "h2d_bytes_per_step": (n * d * 8 + n) / args.steps, "d2h_bytes_per_step": (n * d * 8 + 128) / args.steps}
    info = dict(grid=r.grid(), stats=st, stats_e2e=st2)
    r.close()
    return dict(ms=ms, ms_step=ms_step, value=value, clocks=ck, phase_ms=phase_ms, e2e=e2e, info=info)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skin", type=float, default=0.0, help="neighbour-list skin / (kappa h); 0: library default")
    ap.add_argument("--particles", type=int, default=0,
                    help="override the particle count (small cases for profiler captures)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.particles > 0:
        wl["n"] = args.particles
        wl["desc"] = wl["desc"].split(",")[0] + f", {args.particles} particles (reduced)"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    config = {"workload": wl["desc"], "particles": wl["n"], "dim": wl["dim"], "colors": wl["ncol"],
              "kernel": "Wendland C2", "tau": 2.0, "kappa": 1.0, "gamma": 2.0, "P0": 1.0, "sigma0": 3.0,
              "l2": "inputs larger than L2 (state ~100 B/particle)", "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        # the FP64 CPU oracle as it stands, on this host's cores; rank 0 only
        if rank != 0:
            return
        q, pos, col, desc = oracle_workload_sample(wl)
        times, cores = oracle_time(q, pos, col, args.warmup + args.steps)
        times = times[args.warmup:]
        value = len(pos) * len(times) / sum(times)
        desc += f", {len(times)} timed steps after {args.warmup} warm-up"
        out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-updates/s",
               "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64", "data": "synthetic", "config": config,
               "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": desc},
               "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    res = run_gpu(args, wl, rank, world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    hbm, hbm_src = peaks()
    n = wl["n"]
    ab = ALG_BYTES_FP64 if wl["precision"] == "fp64" else ALG_BYTES
    cells = res["info"]["grid"]["base"][-1]
    per_particle = dict(ab)
    per_particle["cells"] = ab["cells"] + CELL_BYTES_PER_CELL * cells / n
    dom = max(("pass_a", "pass_b"), key=lambda k: res["phase_ms"][k])
    ach = per_particle[dom] * n / (res["phase_ms"][dom] * 1e-3) / 1e9
    step_bytes = sum(per_particle.values()) * n
    roof = {"kernel": "k_pass_a" if dom == "pass_a" else "k_pass_b", "bound": "hbm", "achieved": ach,
            "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
            "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback",
            "alg_bytes_per_particle": per_particle[dom],
            "step_alg_bytes_per_particle": sum(per_particle.values()),
            "step_achieved_gbs": step_bytes / (res["ms_step"] * 1e-3) / 1e9,
            "phase_ms": res["phase_ms"]}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        q, pos, col, desc = oracle_workload_sample(wl)
        times, cores = oracle_time(q, pos, col, 3)
        v = len(pos) * 2 / sum(times[1:])
        cpu = {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
               "sample": desc + ", 2 timed steps after 1 warm-up"}
    st = res["info"]["stats"]
    out = {"metric": METRIC, "value": res["value"], "unit": "particle-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if wl["precision"] == "fp32" else "f64",
           "data": "synthetic", "config": config, "clocks": res["clocks"], "e2e": res["e2e"],
           "gpu_launches": KERNELS_PER_STEP * args.steps, "roofline": roof, "cpu_baseline": cpu,
           "step_stats": {"force_pairs_per_particle": 2 * st["force_pairs"] / n, "list_entries_per_particle": st["list_entries"] / n, "list_rebuilds": st["list_rebuilds"], "dt1": st["dt1"],
                          "err_l2_rms": math.sqrt(st["err_l2"] / n), "levels": res["info"]["grid"]["n_levels"],
                          "cells": cells}}
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
