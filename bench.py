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
    "c4": dict(desc="adjoint: 2D graded hole + 8-coefficient polynomial density (seed 3), 262,144 particles, "
                    "32 colours, FP32, K = 20 steps, checkpoint every 5",
               dim=2, n=1 << 18, ncol=32, precision="fp32", seed=3, make=None),
    "c5": dict(desc="512 independent instances (256 2D + 256 3D), particle counts log-uniform in [2k, 200k] "
                    "(seed 4), 2-64 colours, random sphere/box region, linear graded spacing, FP32",
               dim=0, n=0, ncol=0, precision="fp32", seed=4, make=None),
    "c1": dict(desc="2D unit square, uniform, 4,096 particles (64x64 lattice + 0.3 jitter), 4 colours, FP64, seed 0",
               dim=2, n=4096, ncol=4, precision="fp64", seed=0,
               make=lambda n, c: W.uniform_square_2d(64, c)),
}

# algorithmic DRAM bytes per particle and launch: the particle record read and
# the results written once, as a cell-list method with a per-step re-sort needs
# them (3D FP32: key + sort 20, record gather 17 R + 17 W, pass A 17 R + 16 W,
# pass B 29 R + 20 W; FP64 about 1.7x). The neighbour lists this library keeps
# are extra traffic by design and are not counted.
ALG_BYTES = {"cells": 54, "pass_a": 33, "pass_b": 49}
ALG_BYTES_FP64 = {"cells": 92, "pass_a": 56, "pass_b": 83}
# launches per step (gamma = 2): gate; rekey, count, 3 scan, scatter, gather,
# make_view, list_build (predicated: they exit at once unless the list is
# rebuilt); pass A; pass B; with the staged pass A one more predicated
# rebuild kernel (the blocks' neighbour sets)
KERNELS_PER_STEP = 12
# pair arithmetic (FP32 flop, counted from the equations as the kernels evaluate
# them): distance of a pair 10 (differences, squared norm, root), density term 8
# (Eq. density_sum), pressure + surface-tension term 30 (Eqs.
# sph_pressure_force_2, sph_st_force), viscous term 28 (Eq. sph_viscous_force)
FLOP_PER_PAIR = {"distance": 10, "density": 8, "force": 30, "visc": 28}
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# ncu DRAM traffic of the pair-pass kernel: a summary under profiles/ records the
# bytes per particle of one k_pass_a launch and the hash of the kernel sources
# it was captured from; the figure is reported only while the sources still
# have that hash (else the counters describe another kernel and traffic is null)
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_pass_a_traffic_c3_1m.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1906_07925_gb300", "csrc", f)
                  for f in ("sph_step_impl.cuh", "sph_device.cuh", "sph_internal.h")]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic_per_particle():
    """(bytes per particle of one k_pass_a launch, source hash) from the ncu
    summary, or (None, reason) when it is missing or was taken on other sources."""
    import re
    try:
        txt = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None, "no ncu summary"
    m = re.search(r"sources sha256/16: `?([0-9a-f]{16})", txt)
    b = re.search(r"dram bytes per particle: ([0-9.]+)", txt)
    if not m or not b:
        return None, "ncu summary without source hash or bytes per particle"
    if m.group(1) != kernel_source_hash():
        return None, f"ncu summary taken on sources {m.group(1)}, current {kernel_source_hash()}"
    return float(b.group(1)), m.group(1)


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
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is producing samples
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:
                time.sleep(0.01)
            self.lines.clear()
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
def max_over_ranks(x, world, device="cuda"):
    """The largest value of x over the ranks: the job's time is its slowest
    rank's (replicas run independently; this is the only collective)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, steps, seconds):
    """Whole-job throughput: the units every rank advanced, over the job time."""
    return world * units_per_rank * steps / seconds


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
                   skin=args.skin, cell_factor=args.cell_factor)
    if args.stage >= 0 and wl["precision"] == "fp32":
        r.set_tuning(stage_views=args.stage)
    staged = r.tuning()["stage_views"]
    torch.cuda.synchronize()
    log(f"[rank {rank}] create {time.perf_counter() - t_setup:.2f}s, grid {r.grid()['n_levels']} levels")
    stream = r.stream
    r.step(args.warmup)
    r.sync()
    # the state the timed steps start from, kept in pinned host memory: the
    # end-to-end run below replays exactly these steps from the host
    d = wl["dim"]
    xh = torch.empty((n, d), dtype=torch.float64, pin_memory=True)
    ch = torch.empty((n,), dtype=torch.uint8, pin_memory=True)
    xh.numpy()[:] = r.positions()
    ch.numpy()[:] = r.colors()

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
    ms = max_over_ranks(ms, world)
    ms_step = ms / args.steps
    value = job_rate(n, world, args.steps, ms / 1e3)

    # per-kernel device time over a second timed run (direct launches, events
    # on the handle's stream around each phase)
    kprof = min(args.steps, 10)
    ph = r.step_profiled(kprof)
    phase_ms = {"cells": ph[0] / kprof, "pass_a": ph[1] / kprof, "pass_b": ph[2] / kprof}

    # end to end through the public API with host buffers: upload the state the
    # timed steps started from (pinned memory), the same K steps, positions and
    # statistics back
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
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = {"value": job_rate(n, world, args.steps, e2e_s), "unit": METRIC,
           "h2d_bytes_per_step": (n * d * 8 + n) / args.steps, "d2h_bytes_per_step": (n * d * 8 + 128) / args.steps}
    info = dict(grid=r.grid(), stats=st, stats_e2e=st2, stage=dict(r.stage_info(), enabled=staged),
                kernels_per_step=KERNELS_PER_STEP + (1 if staged else 0))
    r.close()
    out = dict(ms=ms, ms_step=ms_step, value=value, clocks=ck, phase_ms=phase_ms, e2e=e2e, info=info)
    if not args.no_extras and wl["precision"] == "fp32":
        out["fp64"] = run_fp64(args, wl, p, rank)
        if wl["dim"] == 3 and wl["n"] == 1 << 23:
            out["adjoint"] = run_adjoint(rank)
            out["batch"] = batch_summary(run_batch(args, rank, world), args)
    return out


def batch_summary(res, args):
    """The batched form (512 instances) in a few numbers for the default line."""
    return {"workload": WORKLOADS["c5"]["desc"], "instances": 512, "particles": res["total"],
            "ms_per_step": res["ms"] / args.steps, "value": res["total"] * args.steps / (res["ms"] * 1e-3),
            "unit": METRIC, "per_instance_graphs_ms_per_step": res["ms_each"] / args.steps,
            "speedup_of_batched": res["ms_each"] / res["ms"], "autotuner": res["tune"], "clocks": res["clocks"]}


def run_fp64(args, wl, p, rank):
    """The same workload with the FP64 path: graph-timed steps."""
    import torch
    from paper_1906_07925_gb300 import Relaxation
    n = wl["n"]
    r = Relaxation(p, n, wl["ncol"], precision="fp64", seed=wl["seed"] + 1000 * rank, use_graph=True)
    r.step(3)
    r.sync()
    k = max(3, min(args.steps, 10))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(r.stream)
    r.step(k)
    e1.record(r.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / k
    r.close()
    return {"value": n / (ms * 1e-3), "unit": METRIC, "ms_per_step": ms, "steps": k, "warmup": 3, "dtype": "f64"}


def run_adjoint(rank, K=20, ckpt=5):
    """Adjoint cost ratio on the polynomial-field workload: 262,144 particles
    (2D graded hole), 32 colours, FP32, K = 20 steps, checkpoint every 5:
    wall time of sph_backward (its own forward run, the objective and the
    reverse sweep) over that of K forward steps, both synchronised."""
    import torch
    from paper_1906_07925_gb300 import Relaxation
    n = 1 << 18
    p = W.adjoint_poly_2d(n=n, n_colors=32, seed=3)
    r = Relaxation(p, n_particles=n, n_colors=32, precision="fp32", seed=3 + 1000 * rank, use_graph=True)
    x0, c0 = r.positions(), r.colors()
    gout = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    r.step(K)  # warm-up
    r.set_state(x0, c0)
    r.backward(K, lam=1.0, ckpt_every=ckpt, out=gout)  # warm-up (allocates the reverse buffers and graphs)
    fw, bw = [], []
    for _ in range(3):
        r.set_state(x0, c0)
        r.sync()
        t0 = time.perf_counter()
        r.step(K)
        r.sync()
        fw.append(time.perf_counter() - t0)
        r.set_state(x0, c0)
        r.sync()
        t0 = time.perf_counter()
        g = r.backward(K, lam=1.0, ckpt_every=ckpt, out=gout)  # gradient stays on the device
        bw.append(time.perf_counter() - t0)
    r.close()
    f, b = statistics.median(fw), statistics.median(bw)
    return {"workload": "2D graded hole + 8-coefficient polynomial density, 262,144 particles, 32 colours, FP32",
            "K": K, "ckpt_every": ckpt, "forward_ms": f * 1e3, "backward_ms": b * 1e3, "ratio": b / f,
            "L": g["L"]}


def batch_problems(n_inst=512, seed=4):
    inst = W.batch_instances(n_inst, seed=seed)
    probs, ns, cols = [], [], []
    for p, n in inst:
        p.rho_scale = 0.0  # normalised by the library to n particles
        probs.append(p)
        ns.append(n)
        cols.append(p.n_colors)
    return probs, ns, cols


def run_batch(args, rank, world):
    """Batched form: every instance advanced by one CUDA graph per step
    (branch count autotuned), against the same steps issued as a loop of
    per-instance graphs on the same stream."""
    import torch
    from paper_1906_07925_gb300 import Batch
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    probs, ns, cols = batch_problems()
    total = sum(ns)
    seeds = [1000 * rank + k for k in range(len(probs))]
    t0 = time.perf_counter()
    b = Batch(probs, ns, cols, precision="fp32", seeds=seeds)
    log(f"[rank {rank}] batch create {time.perf_counter() - t0:.1f}s, {len(probs)} instances, {total} particles")
    tune = b.tune(candidates=(1, 8, 16, 32, 64, 128, 256), steps_each=4)
    b.step(args.warmup)
    b.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev[0].record(b.stream)
    b.step(args.steps)
    ev[1].record(b.stream)
    ev[1].synchronize()
    ck = clocks.stop()
    ms = ev[0].elapsed_time(ev[1])
    # the same steps as per-instance graphs (reference mode), same stream
    b.step_each(1)
    b.sync()
    ev[2].record(b.stream)
    b.step_each(args.steps)
    ev[3].record(b.stream)
    ev[3].synchronize()
    ms_each = ev[2].elapsed_time(ev[3])
    # end to end: host state in, K batched steps, positions out
    xs = [b.positions(k) for k in range(len(probs))]
    cs = [b.colors(k) for k in range(len(probs))]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(len(probs)):
        b.set_state(k, xs[k], cs[k])
    b.step(args.steps)
    for k in range(len(probs)):
        xs[k] = b.positions(k)
    e2e_s = time.perf_counter() - t0
    b.close()
    ms, ms_each, e2e_s = (max_over_ranks(v, world) for v in (ms, ms_each, e2e_s))
    hb = sum(n * p.dim * 8 + n for p, n in zip(probs, ns))
    return dict(ms=ms, ms_each=ms_each, total=total, clocks=ck, tune=tune,
                e2e={"value": job_rate(total, world, args.steps, e2e_s), "unit": METRIC,
                     "h2d_bytes_per_step": hb / args.steps, "d2h_bytes_per_step": (hb - total) / args.steps})


def batch_oracle_sample(args):
    """The four smallest instances (two 2D, two 3D), 2 oracle steps each."""
    import oracle
    oracle.build()
    probs, ns, cols = batch_problems()
    pick = sorted([k for k in range(len(probs)) if probs[k].dim == 2], key=lambda k: ns[k])[:2] + \
        sorted([k for k in range(len(probs)) if probs[k].dim == 3], key=lambda k: ns[k])[:2]
    parts, secs = 0, 0.0
    for k in pick:
        p = probs[k]
        p.rho_scale = W.rho_scale_for(p, ns[k], res=512 if p.dim == 2 else 64)
        pos, col, _ = W.sample_density(p, ns[k], k)
        x = pos
        for s in range(3):
            t0 = time.perf_counter()
            x, _, _ = oracle.step(p, x, col, s, want=False)
            if s > 0:
                secs += time.perf_counter() - t0
                parts += len(pos)
    return parts / secs, oracle.num_threads(), (f"instances {pick} ({sum(ns[k] for k in pick)} particles), "
                                               "2 timed oracle steps each after 1 warm-up")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skin", type=float, default=0.0, help="neighbour-list skin / (kappa h); 0: library default")
    ap.add_argument("--cell-factor", type=float, default=0.0, help="finest cell edge / smallest support; 0: default")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"],
                    help="override the workload's precision (the FP64 path of the same workload)")
    ap.add_argument("--stage", type=int, default=-1, choices=[-1, 0, 1],
                    help="staged density/force pass: 1 on, 0 off, -1 library default")
    ap.add_argument("--particles", type=int, default=0,
                    help="override the particle count (small cases for profiler captures)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 and adjoint side measurements")
    args = ap.parse_args()
    if args.workload == "c5":
        return main_batch(args)
    if args.workload == "c4":
        return main_adjoint(args)
    wl = dict(WORKLOADS[args.workload])
    if args.particles > 0:
        wl["n"] = args.particles
        wl["desc"] = wl["desc"].split(",")[0] + f", {args.particles} particles (reduced)"
    if args.precision and args.precision != wl["precision"]:
        wl["precision"] = args.precision
        wl["desc"] = wl["desc"].replace("FP32 split-precision", "FP64").replace(", FP64, ", ", FP64, ")
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
    dom = max(("pass_a", "pass_b"), key=lambda k: res["phase_ms"][k])
    t_dom = res["phase_ms"][dom] * 1e-3
    st0 = res["info"]["stats"]
    fpp = 2 * st0["force_pairs"] / n  # ordered force pairs per particle
    dpp = fpp + 1.0                   # density pairs (the particle itself included)
    if dom == "pass_a":
        flop_pp = dpp * (FLOP_PER_PAIR["distance"] + FLOP_PER_PAIR["density"]) + fpp * FLOP_PER_PAIR["force"]
    else:
        flop_pp = fpp * (FLOP_PER_PAIR["distance"] + FLOP_PER_PAIR["visc"])
    tflops = flop_pp * n / t_dom / 1e12
    ach_gbs = per_particle[dom] * n / t_dom / 1e9
    step_bytes = sum(per_particle.values()) * n
    traffic, tsrc = None, "not captured for this workload"
    if (dom == "pass_a" and wl["dim"] == 3 and wl["precision"] == "fp32" and args.skin == 0.0
            and args.cell_factor == 0.0):
        bpp, tsrc = profiled_traffic_per_particle()
        if bpp is not None:
            traffic = bpp * n
            tsrc = f"ncu dram bytes per particle at 1,048,576 particles (sources {tsrc}), x particle count"
    # the pair passes are bound by instruction issue (ncu: issue active ~74 %,
    # half the lanes idle on screened list entries), not by DRAM: the bound is
    # the FP32 pipe, the achieved figure the pair arithmetic the equations need
    roof = {"kernel": "k_pass_a" if dom == "pass_a" else "k_pass_b", "bound": "alu",
            "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tflops / FP32_PEAK_TFLOPS,
            "traffic": traffic, "traffic_source": tsrc,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (FP32 CUDA-core peak)",
            "alg_flop_per_particle": flop_pp,
            "hbm": {"alg_bytes_per_particle": per_particle[dom], "achieved_gbs": ach_gbs, "peak_gbs": hbm,
                    "frac": ach_gbs / hbm, "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "dram_gbs_from_traffic": traffic / t_dom / 1e9 if traffic else None,
                    "step_alg_bytes_per_particle": sum(per_particle.values()),
                    "step_achieved_gbs": step_bytes / (res["ms_step"] * 1e-3) / 1e9},
            "phase_ms": res["phase_ms"]}
    flop = fpp * (FLOP_PER_PAIR["force"] + FLOP_PER_PAIR["visc"]) + dpp * FLOP_PER_PAIR["density"] + \
        (dpp + fpp) * FLOP_PER_PAIR["distance"]
    roof["fp32_pair_flop_per_particle_step"] = flop
    roof["fp32_tflops_step"] = flop * n / (res["ms_step"] * 1e-3) / 1e12
    roof["fp32_frac_of_nominal_peak_step"] = roof["fp32_tflops_step"] / FP32_PEAK_TFLOPS
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
           "gpu_launches": res["info"]["kernels_per_step"] * args.steps, "roofline": roof, "cpu_baseline": cpu,
           "fp64": res.get("fp64"), "adjoint": res.get("adjoint"), "batch": res.get("batch"),
           "step_stats": {"force_pairs_per_particle": 2 * st["force_pairs"] / n, "list_entries_per_particle": st["list_entries"] / n, "list_rebuilds": st["list_rebuilds"], "dt1": st["dt1"],
                          "err_l2_rms": math.sqrt(st["err_l2"] / n), "levels": res["info"]["grid"]["n_levels"],
                          "cells": cells},
           "staged_pass": res["info"]["stage"]}
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main_adjoint(args):
    """Adjoint cost: backward (sph_backward: its forward run, the objective,
    the checkpointed reverse sweep) over K forward steps, one GPU."""
    rank = int(os.environ.get("RANK", "0"))
    wl = WORKLOADS["c4"]
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps({"impl": "reference", "unavailable": "the adjoint cost ratio is a GPU-only measurement; "
                          "the oracle's reverse pass is a correctness reference (tests/test_oracle_adjoint.py)"}))
        return
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    adj = run_adjoint(rank)
    ck = clocks.stop()
    if rank == 0:
        print(json.dumps({"metric": "adjoint/forward cost ratio", "value": adj["ratio"], "unit": "x",
                          "n_gpus": 1, "steps": adj["K"], "warmup": 1, "ms_per_step": adj["backward_ms"] / adj["K"],
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic", "config": {"workload": wl["desc"]}, "clocks": ck, "adjoint": adj}),
              flush=True)


def main_batch(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    wl = WORKLOADS["c5"]
    config = {"workload": wl["desc"], "instances": 512, "kernel": "Wendland C2", "tau": 2.0, "kappa": 1.0,
              "gamma": 2.0, "l2": "inputs larger than L2 (about 22M particles)", "parallelism": f"replicas x{world}"}
    if args.impl == "reference":
        if rank != 0:
            return
        v, cores, desc = batch_oracle_sample(args)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": config,
                          "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                                           "sample": desc},
                          "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
              flush=True)
        return
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    res = run_batch(args, rank, world)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            v, cores, desc = batch_oracle_sample(args)
            cpu = {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": desc}
        ms_step = res["ms"] / args.steps
        out = {"metric": METRIC, "value": job_rate(res["total"], world, args.steps, res["ms"] * 1e-3), "unit": METRIC,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic", "config": config, "clocks": res["clocks"], "e2e": res["e2e"],
               "gpu_launches": (KERNELS_PER_STEP + (1 if res["tune"]["chosen"].get("stage_views") else 0))
               * 512 * args.steps,
               "per_instance_graphs": {"value": job_rate(res["total"], world, args.steps, res["ms_each"] * 1e-3),
                                       "ms_per_step": res["ms_each"] / args.steps,
                                       "speedup_of_batched": res["ms_each"] / res["ms"]},
               "autotuner": res["tune"], "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
