#!/usr/bin/env python
"""Benchmark of the time-tiled 3D acoustic wave forward path on GB300.

One "step" is one full forward modelling run of the 512^3, SO8, 1000-time-step
layered workload (seeded synthetic model, 15 Hz Ricker at 20 m depth, 10-cell
sponge, a line of 512 receivers at 20 m depth whose traces are the result).
The metric is point-steps per second (GPt/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU; the per-shot path does not
shard), launched by torch.distributed.run; rank 0 prints one JSON line.
--impl reference times the FP64 oracle (the plain C loop nest) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GPt/s (point-steps/s) tiled vs untiled; % HBM roofline; FWI gradient s/shot"
WORKLOAD = ("tiled forward 512x512x512, h=10 m, SO8, 1000 steps, 20-layer 1.5-4.5 km/s model + seeded 5% "
            "blurred perturbation (seed 1), 15 Hz Ricker at 20 m depth, 10-cell sponge, 512 receivers at 20 m")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=None,
                    help="grid edge (tiled512: n^3, default 512; so16: n x n x n/2, default 768, receivers scaled)")
    ap.add_argument("--nt", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-untiled", action="store_true")
    ap.add_argument("--no-gradient", action="store_true", help="leave out the FWI gradient record")
    ap.add_argument("--tiling", default="", help="force T,by,bz,xc[,unroll] instead of autotuning")
    ap.add_argument("--so", type=int, default=8, help="space order of the tiled512 workload (4, 8 or 16)")
    ap.add_argument("--workload", choices=["tiled512", "so16", "batched", "gradient"], default="tiled512",
                    help="tiled512: the headline 512^3 SO8 run; so16: 768x768x384 SO16 with 501x501 "
                         "surface receivers; batched: 24 uneven SO4/SO8 shots in one graph launch")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.samples = []
        self.proc = None
        self.thread = None
        self.gpu_id = gpu_id
        self.active = False  # False, or the name of the timed region being sampled

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    self.samples.append((self.active, parts))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, region=None):
        """Clocks of the samples taken while a region was active (any region,
        or only `region`)."""
        load = [p for a, p in self.samples if a and (region is None or a == region)]
        if not load:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[1]) for p in load if num(p[1]) is not None]
        smax = [num(p[2]) for p in load if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for p in load for k in range(4) if p[5 + k].lower().startswith("active")})
        pw = [num(p[3]) for p in load if num(p[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(load), "power_w_max": max(pw) if pw else None}


# source files of each pass kernel variant: overlapped halos (0-2), skewed
# wavefront (4), warp-specialised (5, 6); the kernel files include wave_pass.cuh
def kernel_sources(variant):
    extra = {4: ("wave_skew.cuh",), 5: ("wave_lean.cuh",), 6: ("wave_lean.cuh",), 7: ("wave_lean.cuh",)}.get(variant, ())
    return ("wave_pass.cuh",) + extra


def kernel_name(so, T, variant):
    base = {4: "skew_kernel", 5: "lean_kernel", 6: "lean_kernel", 7: "lean_kernel"}.get(variant, "pass_kernel")
    return "%s<%d,%d> (SO%d, T=%d, variant %d)" % (base, so // 2, T, so, T, variant)


def kernel_traffic(T, so=8, variant=2, key="dram_bytes_per_point"):
    """dram bytes (or, with key="smem_wavefronts_per_point", shared-memory
    wavefronts) per grid point per launch of the pass kernel (T, variant)
    from the committed ncu summary of this space order, only if it was taken
    on the current kernel sources."""
    sha = hashlib.sha256()
    for f in kernel_sources(variant):
        sha.update(open(os.path.join(ROOT, "paper_1707_02347_gb300", "csrc", f), "rb").read())
    h = sha.hexdigest()[:16]
    name = {4: "tiled_pass_so4_512.md", 8: "tiled_pass_so8_512.md", 16: "tiled_pass_so16_768.md"}.get(so)
    if name is None:
        return None, h
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None, h
    txt = open(path).read()
    m_h = re.search(r"kernel_source_sha256_16_v%d:\s*([0-9a-f]+)" % variant, txt)
    m_t = re.search(r"%s_T%d_v%d:\s*([0-9.eE+-]+)" % (key, T, variant), txt)
    if not m_h or not m_t or m_h.group(1) != h:
        return None, h
    return float(m_t.group(1)), h


def run_reference(args, rank):
    """Time the FP64 oracle on the host cores on a bounded sample: each step is
    2 time steps of the same 512^3 workload (full grid)."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1707_02347_gb300 import inputs

    oracle.build()
    n = args.grid or 512
    w = inputs.layered_forward((n, n, n), 8, max(args.nt, 2), seed=1, f=15.0, h=10.0, sponge_width=10,
                               nrec_line=512)
    nt_s = 2
    m64 = w.m.astype(np.float64)
    cores = os.cpu_count()

    def one():
        oracle.forward(w.shape, w.spacing, w.so, w.dt, nt_s, m64, src_xyz=w.src_xyz, wavelet=w.wavelet[:nt_s],
                       rec_xyz=w.rec_xyz, sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    pts = float(n) ** 3 * nt_s * args.steps
    val = pts / el / 1e9
    sample = "%d time steps of the %d^3 SO8 workload per step (full grid, sources and receivers)" % (nt_s, n)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GPt/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "grid": [n, n, n], "so": 8, "nt": args.nt,
                      "note": "oracle: plain FP64 C loop nest, OpenMP on the outer loop"},
           "cpu_baseline": {"value": val, "unit": "GPt/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": "GPt/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(w):
    """The oracle as it stands on a bounded sample of the same workload (~10-20 s)."""
    import numpy as np

    import oracle

    oracle.build()
    m64 = w.m.astype(np.float64)

    def run(k):
        t0 = time.perf_counter()
        oracle.forward(w.shape, w.spacing, w.so, w.dt, k, m64, src_xyz=w.src_xyz, wavelet=w.wavelet[:k],
                       rec_xyz=w.rec_xyz, sponge_width=w.sponge_width, sponge_faces=w.sponge_faces, vmax=w.vmax)
        return time.perf_counter() - t0

    t1 = run(1)
    k = int(max(1, min(20, 12.0 / max(t1, 1e-3))))
    tk = run(k)
    pts = float(np.prod(w.shape)) * k
    grid = "x".join(str(s) for s in w.shape)
    out = {"value": pts / tk / 1e9, "unit": "GPt/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "%d time steps of the full %s SO%d workload (FP64, OpenMP over x), %.1f s" %
                     (k, grid, w.so, tk)}
    # the same oracle on one core: one time step of the full grid
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(1)
        try:
            t1c = run(1)
        finally:
            gomp.omp_set_num_threads(os.cpu_count())
        out["single_core"] = {"value": float(np.prod(w.shape)) / t1c / 1e9, "unit": "GPt/s", "cores": 1,
                              "sample": "1 time step of the full %s SO%d workload on one thread, %.1f s" %
                                        (grid, w.so, t1c)}
    except OSError:
        out["single_core"] = None
    return out


def run_batched(args, W, inputs, dev, world, rank, dist, local):
    """24 shots, grids drawn seeded from [128,320] x [128,320] x [128,256],
    SO alternating 4 / 8, Ricker 8-15 Hz, each with its own autotuned tiling:
    observed data by one batched forward on the true models, then the FWI
    gradient of every shot on a start model 3 % slower (forward with
    checkpoints every 40 steps, adjoint sweep, imaging), all shots in one CUDA
    graph launch.  The value is gradient seconds per shot; the batched forward
    alone is reported in GPt/s beside it."""
    import numpy as np
    import torch

    from paper_1707_02347_gb300 import replicas

    rng = np.random.default_rng(5)
    nshots, nt = 24, min(args.nt, 600)
    mine = replicas.shard(nshots, rank, world)
    plans, pts, m_true = [], 0.0, []
    for s in range(nshots):
        shape = (int(rng.integers(128, 321)), int(rng.integers(128, 321)), int(rng.integers(128, 257)))
        so = 4 if s % 2 == 0 else 8
        f = float(rng.uniform(8.0, 15.0))
        if s not in mine:
            continue
        w = inputs.layered_forward(shape, so, nt, seed=500 + s, f=f, h=10.0, sponge_width=10, nrec_line=64)
        m = torch.from_numpy(w.m).to(dev)
        p = W.WavePlan(w.shape, w.spacing, so, w.dt, nt, m, sponge_width=w.sponge_width, vmax=w.vmax)
        p.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
        p.set_receivers(w.rec_xyz)
        plans.append(p)
        m_true.append(m)
        pts += float(np.prod(shape)) * nt
    batch = W.WaveBatch(plans)
    # every shot tuned over the tilings of the persistent batched kernel
    batch.autotune(passes=2)
    clk = ClockSampler(gpu_uuid_of(dev, local))
    clk.start()
    time.sleep(0.5)
    # batched forward on the true models: the observed data, and its timing
    recs = batch.forward()
    for _ in range(args.warmup):
        batch.forward(recs)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk.active = "forward"
    t0 = time.perf_counter()
    for _ in range(args.steps):
        batch.forward(recs)
    torch.cuda.synchronize()
    el_f = time.perf_counter() - t0
    clk.active = False
    el_f = replicas.max_over_ranks(el_f, dev)
    persistent, n_items, n_blocks = batch.mode()
    d_obs = [r.clone() for r in recs]
    for p, m in zip(plans, m_true):
        p.set_model(m * (1.03 ** 2))
    grads = [torch.empty(p.shape, dtype=torch.float32, device=dev) for p in plans]
    for _ in range(max(args.warmup, 1)):
        mis, _ = batch.gradient(d_obs, checkpoint_every=40, grads=grads)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk.active = "gradient"
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mis, _ = batch.gradient(d_obs, checkpoint_every=40, grads=grads)
    torch.cuda.synchronize()
    el_g = time.perf_counter() - t0
    clk.active = False
    clk.stop()
    el_g = replicas.max_over_ranks(el_g, dev)
    ok = all(np.isfinite(mis)) and all(bool(torch.isfinite(g).all()) for g in grads)
    if rank == 0:
        out = {"metric": "FWI gradient s/shot", "value": el_g / args.steps / (len(plans) * world),
               "unit": "s/shot", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * el_g / args.steps, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": "24 batched shots, grids U[128,320]x[128,320]x[128,256] (seed 5), SO 4/8, "
                                      "%d steps, Ricker 8-15 Hz, per-shot autotuned tiling; forward (one persistent "
                                      "kernel fed by a device work queue) + FWI gradient (checkpoints every 40 "
                                      "steps), each one graph launch for all shots" % nt,
                          "shots_per_rank": len(plans), "gradients_finite": ok,
                          "tilings": [p.get_tiling() for p in plans]},
               "forward": {"value": pts * world * args.steps / el_f / 1e9, "unit": "GPt/s",
                           "ms_per_step": 1e3 * el_f / args.steps, "clocks": clk.summary("forward"),
                           "persistent_kernel": persistent, "work_items": n_items, "thread_blocks": n_blocks},
               "gradient_point_steps_per_s": pts * world * args.steps / el_g,
               "clocks": clk.summary("gradient")}
        print(json.dumps(out), flush=True)
    batch.close()
    for p in plans:
        p.close()


def gpu_uuid_of(dev, local):
    import torch

    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]


def gradient_record(args, W, inputs, dev, world, dist, clk, steps=None, warmup=None):
    """FWI gradient of one shot: 256^3, SO8, 800 steps, 10 Hz Ricker, 256
    receivers on a line at 20 m; data from the seeded true model (seed 3),
    gradient on the true model blurred with sigma = 10 cells, checkpoints
    every 40 steps.  Seconds per shot (forward + checkpoints + recompute +
    adjoint + imaging condition), timed with the clocks sampled under the
    region name "gradient"."""
    import numpy as np
    import torch

    from paper_1707_02347_gb300 import replicas

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    n, nt = 256, min(args.nt, 800)
    w = inputs.layered_forward((n, n, n), 8, nt, seed=3, f=10.0, h=10.0, sponge_width=10, nrec_line=256)
    v_true = 1.0 / np.sqrt(w.m.astype(np.float64))
    v0 = inputs.gaussian_blur(v_true.astype(np.float32), 10.0) / inputs.gaussian_blur(np.ones(w.shape, np.float32), 10.0)
    m_true = torch.from_numpy(w.m).to(dev)
    m0 = torch.from_numpy(inputs.slowness2(v0)).to(dev)
    plan = W.WavePlan(w.shape, w.spacing, 8, w.dt, nt, m_true, sponge_width=w.sponge_width, vmax=w.vmax)
    plan.set_sources(w.src_xyz, torch.from_numpy(w.wavelet.astype(np.float32)).to(dev))
    plan.set_receivers(w.rec_xyz)
    plan.autotune(passes=2)
    d_obs, _ = plan.forward()
    d_obs = d_obs.clone()
    plan.set_model(m0)
    grad = torch.empty(w.shape, dtype=torch.float32, device=dev)
    for _ in range(max(warmup, 1)):
        J, g = plan.gradient(d_obs, checkpoint_every=40, grad_out=grad)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk.active = "gradient"
    t0 = time.perf_counter()
    for _ in range(steps):
        J, g = plan.gradient(d_obs, checkpoint_every=40, grad_out=grad)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clk.active = False
    el = replicas.max_over_ranks(el, dev)
    rec = {"metric": "FWI gradient s/shot", "value": el / steps, "unit": "s/shot", "higher_is_better": False,
           "steps": steps, "warmup": warmup,
           "workload": "FWI gradient 256x256x256, h=10 m, SO8, %d steps, 10 Hz Ricker, 256 receivers at 20 m, "
                       "true model seed 3, start = true blurred sigma 10, checkpoint every 40 steps" % nt,
           "tiling": list(plan.get_tiling()), "sweep_tiling": list(plan.get_sweep_tiling()), "misfit": J,
           "gradient_finite": bool(torch.isfinite(g).all()),
           "point_steps_per_s": float(n) ** 3 * nt / (el / steps), "clocks": clk.summary("gradient")}
    plan.close()
    return rec


def run_gradient(args, W, inputs, dev, world, rank, dist, local):
    """The FWI gradient workload on its own line (see gradient_record)."""
    clk = ClockSampler(gpu_uuid_of(dev, local))
    clk.start()
    time.sleep(0.5)
    try:
        g = gradient_record(args, W, inputs, dev, world, dist, clk)
    finally:
        clk.stop()
    if rank == 0:
        out = {"metric": g["metric"], "value": g["value"], "unit": "s/shot", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * g["value"], "higher_is_better": False,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": g["workload"], "tiling": g["tiling"], "sweep_tiling": g["sweep_tiling"],
                          "misfit": g["misfit"], "point_steps_per_s": g["point_steps_per_s"]},
               "clocks": g["clocks"]}
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch

    import paper_1707_02347_gb300 as W
    from paper_1707_02347_gb300 import inputs

    W.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.workload == "batched":
        run_batched(args, W, inputs, dev, world, rank, dist, local)
        return
    if args.workload == "gradient":
        run_gradient(args, W, inputs, dev, world, rank, dist, local)
        return
    n = args.grid or 512
    if args.workload == "so16":
        g = args.grid or 768
        side = 501 if g == 768 else max(64, g * 501 // 768)
        w = inputs.high_order_forward(nt=min(args.nt, 500), shape=(g, g, g // 2), n_side=side)
        workload_name = ("high-order forward %dx%dx%d, h=12.5 m, SO16, %d steps, layered + perturbed model "
                         "(seed 2), %dx%d surface receivers at 25 m (trilinear)" % (g, g, g // 2, w.nt, side, side))
        so = 16
    else:
        so = args.so
        w = inputs.layered_forward((n, n, n), so, args.nt, seed=1, f=15.0, h=10.0, sponge_width=10, nrec_line=512)
        workload_name = WORKLOAD if so == 8 and n == 512 else WORKLOAD.replace("SO8", "SO%d" % so).replace(
            "512x512x512", "%dx%dx%d" % (n, n, n))
    npts = float(np.prod(w.shape))
    stream = torch.cuda.Stream(device=dev)
    m = torch.from_numpy(w.m).to(dev)
    wav = torch.from_numpy(w.wavelet.astype(np.float32)).to(dev).contiguous()
    with torch.cuda.stream(stream):
        plan = W.WavePlan(w.shape, w.spacing, w.so, w.dt, w.nt, m, sponge_width=w.sponge_width,
                          sponge_faces=w.sponge_faces, vmax=w.vmax, stream=stream)
    plan.set_sources(w.src_xyz, wav)
    plan.set_receivers(w.rec_xyz)
    # autotune: the fastest tiling overall (the headline), the fastest one-step
    # (T = 1, untiled) tiling and the fastest time-tiled (T >= 2) tiling
    if args.tiling:
        best = tuple(int(x) for x in args.tiling.split(","))
        plan.set_tiling(best)
        best = plan.get_tiling()
        tuned = []
    else:
        tuned = plan.autotune(passes=3)
        best = plan.get_tiling()
    one = [t for t in tuned if t[0][0] == 1]
    multi = [t for t in tuned if t[0][0] >= 2]
    untiled_tiling = min(one, key=lambda c: c[1])[0] if one else None
    tiled_tiling = min(multi, key=lambda c: c[1])[0] if multi else None

    rec = torch.empty((w.nt, w.rec_xyz.shape[0]), dtype=torch.float32, device=dev)
    lib = W.load()

    def timed(tiling, K, Wm):
        """K forward runs in `tiling` after Wm untimed ones: (ms, pass launches,
        summed pass-kernel ms, point-steps of those passes, kernels launched)."""
        plan.set_tiling(tiling)
        for _ in range(Wm):
            plan.forward(rec_out=rec)
        lib.wave_profile_read(plan._h, 1, None, None, None, None)
        lib.wave_profile_enable(plan._h, 1)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            plan.forward(rec_out=rec)
        e1.record(stream)
        e1.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        nl, pms, pst, lau = ctypes.c_longlong(0), ctypes.c_double(0), ctypes.c_double(0), ctypes.c_longlong(0)
        lib.wave_profile_read(plan._h, 1, ctypes.byref(nl), ctypes.byref(pms), ctypes.byref(pst), ctypes.byref(lau))
        lib.wave_profile_enable(plan._h, 0)
        return ms, nl.value, pms.value, pst.value, lau.value

    hbm, smmax, peak_kind = peaks()
    clk = ClockSampler(gpu_uuid_of(dev, local))
    clk.start()
    time.sleep(0.5)
    runs = {}

    def measure(tiling):
        key = tuple(tiling)
        if key not in runs:
            clk.active = "forward"
            ms, nl, pms, pst, la = timed(tiling, args.steps, args.warmup)
            clk.active = False
            runs[key] = dict(ms=ms, launches=nl, pass_ms=pms, pass_pts=pst, kernels=la)
        return runs[key]

    def forward_record(tiling, r):
        """GPt/s of a forward run in `tiling`, with its pass kernel against the
        compulsory-traffic roofline: 16 B per grid point per pass (read
        u^{n-1}, u^n and m, write u^{n+T}; 16/T B per point-step), and the
        20 B the design moves (u, v, kappa in; u, v out) beside it."""
        T = tiling[0]
        launch_s = r["pass_ms"] / max(r["launches"], 1) * 1e-3
        v = world * args.steps * npts * w.nt / (r["ms"] * 1e-3) / 1e9
        return {"value": v, "unit": "GPt/s", "ms_per_step": r["ms"] / args.steps, "tiling": list(tiling),
                "kernel": kernel_name(so, T, tiling[4] if len(tiling) > 4 else 0),
                "pass_avg_launch_ms": launch_s * 1e3,
                "compulsory_bytes_per_point_step": 16.0 / T,
                "hbm_frac": 16.0 * npts / launch_s / 1e9 / hbm,
                "design_bytes_per_point_step": 20.0 / T,
                "hbm_frac_design_bytes": 20.0 * npts / launch_s / 1e9 / hbm}

    rb = measure(best)
    value = world * args.steps * npts * w.nt / (rb["ms"] * 1e-3) / 1e9
    ms_step = rb["ms"] / args.steps
    untiled = tiled = None
    if not args.no_untiled:
        if untiled_tiling is not None:
            untiled = forward_record(untiled_tiling, measure(untiled_tiling))
        if tiled_tiling is not None:
            tiled = forward_record(tiled_tiling, measure(tiled_tiling))
            if untiled is not None:
                tiled["speedup_over_untiled"] = tiled["value"] / untiled["value"]

    T = best[0]
    variant = best[4] if len(best) > 4 else 0
    avg_launch_s = (rb["pass_ms"] / max(rb["launches"], 1)) * 1e-3
    bytes_per_launch = 16.0 * npts  # compulsory: read u^{n-1}, u^n, m; write u^{n+T}
    achieved = bytes_per_launch / avg_launch_s / 1e9
    traffic_pp, src_hash = kernel_traffic(T, so, variant)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic_pp * npts if traffic_pp is not None else None,
            "kernel": kernel_name(so, T, variant), "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "algorithmic_bytes_note": "compulsory 16 B per grid point and pass (u^{n-1}, u^n, m in; u^{n+T} out)",
            "design_bytes_per_launch": 20.0 * npts,
            "frac_design_bytes": 20.0 * npts / avg_launch_s / 1e9 / hbm,
            "avg_launch_ms": avg_launch_s * 1e3, "launches_timed": rb["launches"],
            "kernel_source_sha256_16": src_hash}
    flops_pp = 9 * (so // 2) + 5  # per point-step: 3 axes x r pairs x (add + fma), centre, update
    fp32_peak = 152 * 128 * 2 * smmax * 1e6 / 1e12
    # shared memory: one 128-byte wavefront per SM and clock
    wf_pp, _ = kernel_traffic(T, so, variant, "smem_wavefronts_per_point")
    smem_peak = 152 * 128 * smmax * 1e6 / 1e9
    roof_smem = None
    if wf_pp is not None:
        smem_ach = wf_pp * npts * 128 / avg_launch_s / 1e9
        roof_smem = {"bound": "smem", "achieved": smem_ach, "peak": smem_peak, "unit": "GB/s",
                     "frac": smem_ach / smem_peak, "wavefronts_per_point": wf_pp,
                     "note": "shared-memory load/store wavefronts of one launch (ncu, 128 B each) over the "
                             "measured launch time, vs one wavefront per SM per clock at max clock"}
    pass_ms, pass_pts = rb["pass_ms"], rb["pass_pts"]
    roof_alu = {"bound": "alu", "achieved": flops_pp * pass_pts / (pass_ms * 1e-3) / 1e12, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": flops_pp * pass_pts / (pass_ms * 1e-3) / 1e12 / fp32_peak,
                "flops_per_point_step": flops_pp,
                "note": "algorithmic FP32 flops (no halo recompute) vs 152 SMs x 128 lanes x 2 x max clock"}

    e2e = None
    if not args.no_e2e:
        m_h = torch.from_numpy(w.m).pin_memory()
        w_h = torch.from_numpy(w.wavelet.astype(np.float32)).pin_memory()
        r_h = torch.empty((w.nt, w.rec_xyz.shape[0]), dtype=torch.float32).pin_memory()
        plan.set_tiling(best)
        for _ in range(max(1, args.warmup)):
            plan.forward_host(m_h, w_h, r_h)
        barrier()
        clk.active = "e2e"
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.forward_host(m_h, w_h, r_h)
        barrier()
        el = time.perf_counter() - t0
        clk.active = False
        if dist is not None:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * args.steps * npts * w.nt / el / 1e9, "unit": "GPt/s",
               "h2d_bytes_per_step": int(m_h.numel() * 4 + w_h.numel() * 4),
               "d2h_bytes_per_step": int(r_h.numel() * 4)}
        plan.set_tiling(best)
        plan.forward(rec_out=rec)
        ref_rec = rec.cpu()
        assert torch.equal(ref_rec, r_h), "host-buffer path differs from the device path"
    plan.close()

    # the metric's third quantity: FWI gradient seconds per shot (256^3, SO8, 800 steps)
    grad = None
    if args.workload == "tiled512" and not args.no_gradient:
        grad = gradient_record(args, W, inputs, dev, world, dist, clk)
    clk.stop()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GPt/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": workload_name, "grid": list(w.shape), "so": so, "nt": w.nt, "tiling": list(best),
                          "dt_ms": w.dt, "l2": "inputs larger than L2 (each field %.0f MB > 129 MB)" % (npts * 4 / 1e6),
                          "parallelism": "replicas" if world > 1 else "single GPU"},
               "value_note": "the autotuner's pick over every compiled one-step and time-tiled pass",
               "untiled": untiled, "tiled": tiled,
               "speedup_tiled_over_untiled": (tiled["value"] / untiled["value"]) if tiled and untiled else None,
               "roofline": roof, "roofline_alu": roof_alu, "roofline_smem": roof_smem,
               "gradient": grad,
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": rb["kernels"], "clocks": clk.summary("forward"),
               "clocks_e2e": clk.summary("e2e") if e2e else None,
               "autotune": [[list(t), ms_] for t, ms_ in sorted(tuned, key=lambda c: c[1])[:8]]}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
