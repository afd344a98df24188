"""Throughput benchmark of the PIC step (push + deposit + re-sort + Yee).

Default workload (N=1): the large single-run thermal plasma at full size,
2048x2048 cells, 4x4 thermal electrons per cell (67,108,864 particles,
u_th = 0.2) with a seeded sinusoidal Ex mode (k = 2 pi / L_x, amplitude 1e-3),
16x16-cell tiles, dt = 0.05, dx = dy = 0.1, random synthetic inputs.  A step
is one pass of the whole hot path over all particles.  ``value`` is particle
updates per second with the state resident in HBM; ``e2e`` is the same
metric through the C ABI from pinned host buffers (load, K steps, field
read-back and diagnostics inside the timed region).  The particle state
(1.6 GB) is larger than the 129 MB L2, so no L2 flush is needed between
steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle updates/s (push+deposit+sort)"
UNIT = "particle-updates/s"
PEAK_FALLBACK_GBS = 6800.0

WORKLOADS = {
    # name: (factory kwargs, tile)
    "weibel_512": dict(kind="weibel", kw=dict(nx=512, ny=512, k=8), tile=16),
    # smaller instance of the same physics (8.4M particles, 201 MB state > L2)
    # for profiler captures
    "weibel_256": dict(kind="weibel", kw=dict(nx=256, ny=256, k=8), tile=16),
    # L2-resident instance (2.1M particles, 50 MB state < L2): compute-bound reference
    "weibel_128": dict(kind="weibel", kw=dict(nx=128, ny=128, k=8), tile=16),
    "thermal_2048": dict(kind="thermal_seeded", kw=dict(nx=2048, ny=2048, k=4), tile=16),
    # the thesis's own Weibel shape: electrons and positrons, 10x10 ppc each,
    # 512^2 (26.2M per species; the thesis has 25M per species on 500^2)
    "weibel_pair_512": dict(kind="weibel_pair", kw=dict(nx=512, ny=512, k=10), tile=16),
    # smaller instance (16.8M particles, 403 MB state > L2) for profiler captures
    "thermal_1024": dict(kind="thermal_seeded", kw=dict(nx=1024, ny=1024, k=4), tile=16),
    "two_stream_64": dict(kind="two_stream", kw=dict(nx=64, ny=64, k=4), tile=16),
    # 64 independent two-stream simulations (grid side from {64,128,256,512},
    # ppc from {4,16,64}, drift U[0.1,0.5], u_th 0.05, per-simulation seeds)
    # stepped as one batch; tiles and threads autotuned per (grid, ppc)
    "batched_64": dict(kind="batch", kw=dict(members=64), tile=0),
    # laser pulse (a0 = 2, Gaussian, W0 = 3) entering a cold 4x4-ppc plasma that
    # fills the right half of a 2048x1024 moving window (16.8M particles at
    # the start, more as the window injects plasma)
    "laser_wakefield_2048": dict(kind="laser_wakefield",
                                 kw=dict(nx=2048, ny=1024, k=4, a0=2.0, W0=3.0, steps=500),
                                 tile=16),
    # learned current denoiser: 256x256 two-stream draws, 2,000 training pairs
    # (64 ppc vs its 1/16 subsample), the denoised 4-ppc run against 64 ppc
    "denoiser": dict(kind="denoiser", kw=dict(nx=256, ny=256, pairs_per_draw=200, draws=10,
                                              iters=4000, batch=16), tile=16),
    # the denoiser's forward pass alone on one 2048x2048 sample (the largest
    # grid the in-loop speedup is quoted on), parameters of the network's shapes
    "denoiser_fwd_2048": dict(kind="denoiser_fwd", kw=dict(nx=2048, ny=2048), tile=16),
    # the same at 1024x1024 (a smaller case of the same kernels, for profiling)
    "denoiser_fwd_1024": dict(kind="denoiser_fwd", kw=dict(nx=1024, ny=1024), tile=16),
    # one training step of the denoiser (forward, backward through every layer,
    # Adam) on a batch of synthetic currents: 16 samples of 256x256, the
    # training batch of the denoiser workload, and one sample of 2048x2048
    "denoiser_train_256": dict(kind="denoiser_train", kw=dict(nx=256, ny=256, batch=16), tile=16),
    "denoiser_train_2048": dict(kind="denoiser_train", kw=dict(nx=2048, ny=2048, batch=1),
                                tile=16),
}


def make_workload(name):
    from paper_2501_14795_gb300 import workloads as wl
    spec = WORKLOADS[name]
    w = getattr(wl, spec["kind"])(tile=spec["tile"], **spec["kw"])
    return w


def workload_config(name, w, threads):
    return {"workload": name, "grid": [w.nx, w.ny], "particles": w.n_particles,
            "ppc": w.meta.get("ppc"), "tile": w.tile, "threads_per_tile": threads,
            "dt": w.dt, "dx": w.dx, "steps_of_workload": w.steps,
            "timed_steps": "the K steps after W warm-up steps from the workload's initial state",
            "l2": "inputs larger than L2 (particle state {:.0f} MB > 129 MB)".format(
                w.n_particles * 24 / 1e6)}


# ------------------------------------------------------------ measurements

def max_over_ranks(*vals):
    """Each value's maximum over the ranks of the default process group (the
    slowest replica sets the time of the whole job); the values themselves
    without a group.  NCCL reduces on the GPU, gloo on the host."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return [float(v) for v in vals]
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank, world, steps, ms_max):
    """Units every replica processed in `steps` steps over the slowest
    replica's time in ms (weak scaling: each rank holds the same workload)."""
    return units_per_rank * world * steps / (ms_max * 1e-3)


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return PEAK_FALLBACK_GBS, "fallback"


def push_source_hash():
    h = hashlib.sha256()
    for f in ("kernels_push.cu", "device_util.cuh", "pic_internal.h"):
        with open(os.path.join(ROOT, "paper_2501_14795_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_value(name, workload):
    """A per-workload figure of the particle advance from a committed ncu
    summary under profiles/ (lines: workload value source-hash), valid only
    while the kernel sources hash the same as when it was captured."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    want = push_source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == workload and parts[2] == want:
            return float(parts[1])
    return None


def recorded_traffic(workload):
    """DRAM bytes per particle-advance launch (profiles/traffic.txt)."""
    return recorded_value("traffic.txt", workload)


def issue_roofline(workload, particles_per_s, sm_mhz):
    """The particle advance's own ceiling: it is bound by instruction issue
    (one warp-instruction per scheduler per clock, four schedulers per SM).
    Warp-instructions per 32 particles from profiles/issue.txt (ncu,
    smsp__inst_executed.sum at the same kernel source); achieved = that times
    the particles advanced per second."""
    per32 = recorded_value("issue.txt", workload)
    if per32 is None or not sm_mhz:
        return None
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    achieved = per32 / 32.0 * particles_per_s
    peak = 4.0 * sms * sm_mhz * 1e6
    return {"bound": "issue", "warp_instructions_per_32_particles": per32, "achieved": achieved,
            "peak": peak, "unit": "warp-instructions/s", "frac": achieved / peak,
            "peak_source": f"4 schedulers x {sms} SMs x the sampled median SM clock"}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# reduced instance of each workload's physics for the CPU oracle's timed
# samples (the full sizes take minutes per step on the host)
CPU_SAMPLES = {
    "thermal_seeded": ("thermal_seeded", dict(nx=256, ny=256, k=4)),
    "weibel": ("weibel", dict(nx=64, ny=64, k=8)),
    "weibel_pair": ("weibel_pair", dict(nx=64, ny=64, k=10)),
    "two_stream": ("two_stream", dict(nx=64, ny=64, k=4)),
}


def cpu_sample(name):
    """(workload, description) of the bounded CPU sample of workload `name`:
    the same physics on a smaller periodic grid (the Weibel sample for the
    kinds without a periodic single-grid form)."""
    from paper_2501_14795_gb300 import workloads as wl
    kind = WORKLOADS[name]["kind"] if name in WORKLOADS else name
    fac, kw = CPU_SAMPLES.get(kind, CPU_SAMPLES["weibel"])
    w = getattr(wl, fac)(tile=16, **kw)
    return w, (f"{fac} physics on a {w.nx}x{w.ny} periodic grid, {w.meta.get('ppc')} ppc "
               f"({w.n_particles} particles)")


def oracle_sim(w, threads):
    import oracle
    sps = [oracle.SpeciesState(s.q_over_m, s.qtilde, *s.arrays()) for s in w.species]
    return oracle.OracleSim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tile, sps,
                            background=w.background, E=w.E0, B=w.B0, threads=threads)


def time_oracle(w, threads, budget_s):
    """Oracle steps of `w` for about budget_s seconds after one warm-up step;
    returns (particle updates/s, steps)."""
    o = oracle_sim(w, threads)
    o.step(1)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        o.step(1)
        steps += 1
    return w.n_particles * steps / (time.perf_counter() - t0), steps


def cpu_baseline(name, budget_s=12.0):
    """The FP64 oracle as it stands on a bounded sample of the workload's
    physics: its threaded particle loop (the thesis's CPU scheme: blocks of
    tile-sorted particles over threads, private current arrays) on all host
    cores, and the plain single-threaded loop beside it."""
    w, what = cpu_sample(name)
    cores = os.cpu_count() or 1
    v, steps = time_oracle(w, cores, budget_s)
    v1, steps1 = time_oracle(w, 1, budget_s / 2)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}, {steps} steps after 1 warm-up, FP64 C oracle, particle loop "
                      f"over {cores} threads (private current arrays), serial re-sort and field "
                      f"advance",
            "single_thread": {"value": v1, "steps": steps1},
            "cpu_model": _cpu_model(), "host_cores": cores}


def _cpu_model():
    try:
        for l in open("/proc/cpuinfo"):
            if l.lower().startswith(("model name", "cpu part", "hardware")):
                return l.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------ arms

def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on bounded samples of the same workload."""
    if rank != 0:
        return
    kind = WORKLOADS[args.workload]["kind"]
    if kind == "denoiser_fwd":
        run_reference_denoiser_fwd(args, world)
        return
    if kind == "denoiser_train":
        run_reference_denoiser_train(args, world)
        return
    w, what = cpu_sample(args.workload)
    cores = os.cpu_count() or 1
    o = oracle_sim(w, cores)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = w.n_particles * args.steps / dt
    if kind in ("batch", "denoiser"):
        config = {"workload": args.workload}
    else:
        config = workload_config(args.workload, make_workload(args.workload), args.threads)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {what}, FP64 C oracle, particle loop over "
                                       f"{cores} threads (private current arrays)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_denoiser_fwd(args, world):
    """Reference arm of the forward-only denoiser workload: the FP64 numpy
    oracle's forward pass on a bounded 64x64 sample, in the same unit."""
    from oracle import denoiser as D
    from paper_2501_14795_gb300 import denoise as dn
    n = 64
    rng = np.random.Generator(np.random.PCG64(dn.SEED_DENOISER + 11))
    x = 0.03 * rng.standard_normal((1, n, n, 3))
    p = D.init_params(dn.SEED_DENOISER + 7)
    for _ in range(args.warmup):
        D.forward(p, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        D.forward(p, x)
    dt = time.perf_counter() - t0
    value = dn.forward_flops(n, n) * args.steps / dt / 1e12
    print(json.dumps({
        "impl": "reference", "metric": "denoiser forward throughput", "value": value,
        "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: the FP64 numpy oracle's forward pass of one "
                                   f"{n}x{n} sample"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


# kernels of one training step: 11 layers' forward, the loss, the input and
# weight gradients and ReLU backward of each layer (the pooling and upsampling
# adjoints fused into four of them), the weight packing and Adam (counted from
# an ncu launch list of the 256x256 x 16 step; the same layers run at every
# grid size)
TRAIN_LAUNCHES = 49


def oracle_train_rate(n, steps, warmup=0):
    """TFLOP/s of the FP64 numpy oracle's loss and gradients (the arithmetic
    of a training step) on one n x n sample of synthetic currents."""
    from oracle import denoiser as D
    from paper_2501_14795_gb300 import denoise as dn
    rng = np.random.Generator(np.random.PCG64(dn.SEED_DENOISER + 12))
    x = 0.05 * rng.standard_normal((1, n, n, 3))
    p = D.init_params(dn.SEED_DENOISER + 7)
    for _ in range(warmup):
        D.loss_and_grads(p, x, 0.5 * x)
    t0 = time.perf_counter()
    for _ in range(steps):
        D.loss_and_grads(p, x, 0.5 * x)
    dt = time.perf_counter() - t0
    return 3 * dn.forward_flops(n, n) * steps / dt / 1e12, dt


def run_reference_denoiser_train(args, world):
    """Reference arm of the training workloads: the FP64 numpy oracle's loss
    and gradients on a bounded 32x32 sample, in the same unit."""
    n = 32
    value, dt = oracle_train_rate(n, args.steps, args.warmup)
    print(json.dumps({
        "impl": "reference", "metric": "denoiser training throughput", "value": value,
        "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: the FP64 numpy oracle's loss and gradients of "
                                   f"one {n}x{n} sample"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_denoiser_train(args, rank, world, local_rank):
    """Training throughput of the denoiser: K steps (forward, backward through
    every layer, Adam) on one batch of synthetic currents resident in HBM;
    each call synchronises, so the CUDA events bracket whole steps.  End to
    end, the same steps from host buffers (the library stages the batch and
    returns the loss)."""
    import torch
    from paper_2501_14795_gb300 import denoise as dn
    from paper_2501_14795_gb300 import pic

    torch.cuda.set_device(local_rank)
    kw = WORKLOADS[args.workload]["kw"]
    nx, ny, B = kw["nx"], kw["ny"], kw["batch"]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(dn.SEED_DENOISER + 12)
    jn = 0.05 * torch.randn((B, 3, ny, nx), device="cuda", generator=gen)
    jc = 0.5 * jn
    net = pic.Denoiser(nx, ny, B, 0.05)
    net.set_params(dn.init_params(dn.SEED_DENOISER + 7).astype(np.float32))
    for _ in range(args.warmup):
        net.train_step(jn, jc, 1e-4)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            net.train_step(jn, jc, 1e-4)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    jn_h, jc_h = jn.cpu().numpy(), jc.cpu().numpy()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        net.train_step(jn_h, jc_h, 1e-4)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    net.close()
    ms, e2e_ms = max_over_ranks(ms, e2e_ms)
    if rank != 0:
        return
    flops = 3 * dn.forward_flops(nx, ny, B)
    achieved = flops / (ms * 1e-3) / 1e12
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = float(json.load(open(p))["bf16_tflops"]) if os.path.exists(p) else 1900.0
    line = {
        "metric": "denoiser training throughput", "value": achieved * world, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (accumulate f32)", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [nx, ny], "batch": B,
                   "flops_per_step": flops,
                   "l2": "inputs larger than L2 (the level-0 activations of a batch exceed 129 MB)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "whole training step (forward, backward, Adam)",
                     "peak_source": "measured bf16_tflops" if os.path.exists(p) else "fallback"},
        "e2e": {"value": flops / (e2e_ms * 1e-3) / 1e12 * world, "unit": "TFLOP/s",
                "h2d_bytes_per_step": jn_h.nbytes + jc_h.nbytes, "d2h_bytes_per_step": 8},
        "gpu_launches": TRAIN_LAUNCHES * args.steps,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        n = 32
        v, _ = oracle_train_rate(n, 2)
        line["cpu_baseline"] = {"value": v, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                                "sample": f"2 steps of the FP64 numpy oracle's loss and "
                                          f"gradients on one {n}x{n} sample"}
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local_rank):
    """The batched workload: 64 simulations, each step one graph for all of
    them, against the same simulations stepped one after another (each its own
    graph) in the same run."""
    import torch
    from paper_2501_14795_gb300 import pic
    from paper_2501_14795_gb300 import workloads as wl

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    nm = WORKLOADS["batched_64"]["kw"]["members"]
    members = [wl.batch_member(s) for s in range(nm)]
    n = sum(w.n_particles for w in members)
    cells = sum(w.nx * w.ny for w in members)
    sims = [pic.Simulation.from_workload(w, tile=16, threads=args.threads, device=True,
                                         stream=stream.cuda_stream) for w in members]
    t0 = time.perf_counter()
    choices = {}
    for w, s in zip(members, sims):
        T, nthr, _ = s.autotune(steps=3)
        choices[f"{w.nx}x{w.ny}/{w.meta.get('ppc')}ppc"] = [T, nthr]
    tune_s = time.perf_counter() - t0

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # sequential: every simulation its own step graph, one after another
    for s in sims:
        s.step(args.warmup)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        for s in sims:
            s.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    seq_ms = ev0.elapsed_time(ev1)

    batch = pic.Batch(sims, stream.cuda_stream)
    batch.step(args.warmup)
    batch.sync()
    l0, per_step = batch.kernel_launches()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        batch.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    batch.sync()
    launches = batch.kernel_launches()[0] - l0
    leavers = sum(s.diagnostics()["leavers"] for s in sims)
    batch.close()
    for s in sims:
        s.close()
    del sims

    # ---- end to end through the C ABI from pinned host buffers ----
    host = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in w.species[0].arrays()]
            for w in members]
    outs = [torch.empty(3 * w.nx * w.ny, dtype=torch.float32).pin_memory() for w in members]
    h2d = sum(t.numel() * t.element_size() for h in host for t in h)
    d2h = sum(o.numel() * 4 for o in outs) + 96 * nm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cfgs = [pic.config_for(w, 16, args.threads, 0) for w in members]
    e2e_sims = pic.Simulation.init_batch(cfgs, stream.cuda_stream)
    for s, arrs in zip(e2e_sims, host):
        pic.pic_load_particles(s.h, 0, *arrs)
        s.autotune(steps=3)  # cached: applies the choice made above
    eb = pic.Batch(e2e_sims, stream.cuda_stream)
    eb.step(args.steps)
    for s, o in zip(e2e_sims, outs):
        pic.pic_get_fields(s.h, pic.FIELD_E, o)
        pic.pic_diagnostics(s.h)
    e2e_s = time.perf_counter() - t0
    eb.close()
    for s in e2e_sims:
        s.close()
    ms, e2e_ms, seq_ms = max_over_ranks(ms, e2e_s * 1e3, seq_ms)
    e2e_s = e2e_ms * 1e-3
    if rank != 0:
        return
    value = whole_job_rate(n, world, args.steps, ms)
    peak, peak_kind = read_peaks()
    f_leave = leavers / n
    step_bytes = 48.0 + 48.0 * f_leave + 96.0 * cells / n
    achieved = step_bytes * n * args.steps / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched_64", "members": nm, "particles": n, "cells": cells,
                   "tile": "autotuned per (grid, ppc)", "autotune": choices,
                   "autotune_s": tune_s,
                   "l2": f"inputs larger than L2 (particle state {n * 24 / 1e6:.0f} MB > 129 MB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "sequential": {"value": whole_job_rate(n, world, args.steps, seq_ms), "ms_per_step": seq_ms / args.steps,
                       "what": "the same simulations stepped one after another, each its own "
                               "step graph"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "whole batched step (algorithmic bytes of all stages)",
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "e2e": {"value": whole_job_rate(n, world, args.steps, e2e_s * 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
        "gpu_launches": int(launches),
        "launches_per_step": per_step,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# passes of the denoiser's low-wavenumber restoration evaluated beside the
# plain network
LOW_K_PASSES = (2, 4, 8)


def run_denoiser(args, rank, world, local_rank):
    """Learned denoiser: pairs from 64-ppc runs, training on the GPU, then true
    4-ppc runs with the network in the current-filter slot against plain 64-ppc
    and 4-ppc runs of the same draws (growth rate, field-energy history, step
    time)."""
    import torch
    from paper_2501_14795_gb300 import denoise as dn
    from paper_2501_14795_gb300 import pic

    torch.cuda.set_device(local_rank)
    kw = WORKLOADS["denoiser"]["kw"]
    nx, ny, B = kw["nx"], kw["ny"], kw["batch"]
    t0 = time.perf_counter()
    every = max(1, 600 // kw["pairs_per_draw"])
    Jn, Jc = dn.make_pairs(dn.draws(kw["draws"]), nx, ny, steps=600, every=every)
    pair_s = time.perf_counter() - t0
    n_pairs = int(Jn.shape[0])
    Vn, Vc = dn.make_pairs(dn.draws(2, offset=400), nx, ny, steps=600, every=20)
    scale = float(Jc.pow(2).mean().sqrt())
    net = pic.Denoiser(nx, ny, B, scale)
    net.set_params(dn.init_params(dn.SEED_DENOISER + 999))
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ev0.record(stream)
    losses = dn.train(net, Jn, Jc, kw["iters"], B, lr=1e-3, lr_min=5e-5, seed=11)
    ev1.record(stream)
    torch.cuda.synchronize()
    train_ms = ev0.elapsed_time(ev1)
    raw, den = dn.mse_gain(net, Vn, Vc, B)
    del Jn, Jc
    # forward pass alone, one sample (the in-loop use)
    x = Vn[:1].contiguous()
    o = torch.empty_like(x)
    for _ in range(3):
        pic.pic_denoiser_forward(net.d, x, o, 1)
    torch.cuda.synchronize()
    ev0.record(stream)
    nf = 50
    for _ in range(nf):
        pic.pic_denoiser_forward(net.d, x, o, 1)
    ev1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(ev1) / nf

    # where the network shrinks the coherent current: shell-by-shell gains on
    # the validation pairs, without and with the low-wavenumber restoration
    spectral = {}
    for n in (0,) + LOW_K_PASSES:
        net.set_low_k_restore(n)
        spectral[f"low_k_{n}"] = dn.spectral_gain(net, Vn, Vc, B)
    net.set_low_k_restore(0)
    del Vn, Vc

    steps = args.steps
    variants = [("ppc64", 8, False, 0, 0), ("ppc4", 2, False, 0, 0),
                ("ppc4_denoised", 2, True, 0, 0), ("ppc4_binomial", 2, False, 1, 0)]
    variants += [(f"ppc4_denoised_low_k_{n}", 2, True, 0, n) for n in LOW_K_PASSES]
    results = []
    for d in dn.draws(3, offset=500):
        theory = dn.kinetic_growth_rate(d.drift, d.u_th, nx * 0.1)
        row = {"seed": d.seed, "drift": d.drift, "u_th": d.u_th, "theory_gamma": theory,
               "eligible": theory > 0.05}
        runs = {}
        for name, k, use, binom, lowk in variants:
            net.set_low_k_restore(lowk)
            w = dn.workload(d, nx, ny, k, steps)
            we, _, diag, spec = dn.field_energy_run(w, steps, net if use else None, modes=True,
                                                     binomial=binom)
            _, ms, _, _ = dn.field_energy_run(w, steps, net if use else None, binomial=binom)
            runs[name] = (we, spec, ms, diag)
        m = int(np.argmax(runs["ppc64"][1][:, 1:].max(axis=0))) + 1
        lw64 = np.log(np.maximum(runs["ppc64"][0][1:], 1e-300))   # W_E(0) = 0
        for name, (we, spec, ms, diag) in runs.items():
            gm, _ = dn.mode_growth_rate(spec, 0.05, m)
            ge, _ = dn.growth_rate(we, 0.05)
            row[name] = {"gamma_mode": gm, "gamma_WE": ge, "ms_per_step": ms,
                         "W_E_max": float(we.max()),
                         "lnWE_rms_diff_vs_64": float(np.sqrt(np.mean(
                             (np.log(np.maximum(we[1:], 1e-300)) - lw64) ** 2))),
                         "continuity_max": diag["continuity_max"]}
        row["mode"] = m
        g64 = row["ppc64"]["gamma_mode"]
        for name, *_ in variants[1:]:
            row[name]["gamma_mode_rel_err"] = abs(row[name]["gamma_mode"] - g64) / g64
        results.append(row)
    net.set_low_k_restore(0)
    # the same trained network on larger grids (it is translation invariant):
    # step times of 64 ppc, 4 ppc and denoised 4 ppc
    by_grid = {}
    d0 = dn.draws(1, offset=500)[0]
    for side in (512, 1024, 2048):
        big = pic.Denoiser(side, side, 1, scale)
        big.set_params(net.params())
        row = {}
        for name, k, use, lowk in (("ppc64", 8, False, 0), ("ppc4", 2, False, 0),
                                   ("ppc4_denoised", 2, True, 0),
                                   (f"ppc4_denoised_low_k_{LOW_K_PASSES[-1]}", 2, True,
                                    LOW_K_PASSES[-1])):
            big.set_low_k_restore(lowk)
            w = dn.workload(d0, side, side, k, 60)
            _, ms, _, _ = dn.field_energy_run(w, 60, big if use else None)
            row[name] = ms
        row["speedup"] = row["ppc64"] / row["ppc4_denoised"]
        by_grid[f"{side}x{side}"] = row
        big.close()
    ms64 = float(np.mean([r["ppc64"]["ms_per_step"] for r in results]))
    msnn = float(np.mean([r["ppc4_denoised"]["ms_per_step"] for r in results]))
    msbin = float(np.mean([r["ppc4_binomial"]["ms_per_step"] for r in results]))
    ms4 = float(np.mean([r["ppc4"]["ms_per_step"] for r in results]))
    flops = dn.forward_flops(nx, ny)
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peak = float(json.load(open(p))["bf16_tflops"])
    achieved = flops / (fwd_ms * 1e-3) / 1e12
    train_tflops = 3 * flops * B * kw["iters"] / (train_ms * 1e-3) / 1e12
    if rank != 0:
        return
    elig = [r for r in results if r["eligible"]]
    line = {
        "metric": "denoised 4-ppc vs 64-ppc", "value": ms64 / msnn,
        "unit": "x (64-ppc step time / denoised 4-ppc step time)", "n_gpus": world,
        "steps": steps, "warmup": 2, "ms_per_step": msnn, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (network) / f32 (PIC)",
        "data": "synthetic",
        "config": {"workload": "denoiser", "grid": [nx, ny], "train_pairs": n_pairs,
                   "iters": kw["iters"], "batch": B, "scale": scale},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "kernel": "denoiser forward, one 256x256 sample (all launches)",
                     "flops_per_launch": flops, "launch_ms": fwd_ms,
                     "peak_source": "measured bf16_tflops" if peak else None},
        "training": {"pair_gen_s": pair_s, "train_ms": train_ms,
                     "train_tflops": train_tflops, "loss_first": losses[0],
                     "loss_last50": float(np.mean(losses[-50:]))},
        "validation_mse": {"raw_4ppc": raw, "denoised": den, "ratio": den / raw},
        "step_ms": {"ppc64": ms64, "ppc4": ms4, "ppc4_denoised": msnn, "ppc4_binomial": msbin},
        "speedup_by_grid": by_grid,
        "growth": results,
        "growth_within_5pct": [r["ppc4_denoised"]["gamma_mode_rel_err"] < 0.05 for r in elig],
        "growth_within_5pct_binomial": [r["ppc4_binomial"]["gamma_mode_rel_err"] < 0.05
                                        for r in elig],
        "growth_within_5pct_low_k": {n: [r[f"ppc4_denoised_low_k_{n}"]["gamma_mode_rel_err"] < 0.05
                                         for r in elig] for n in LOW_K_PASSES},
        "spectral_gain_validation": spectral,
    }
    print(json.dumps(line), flush=True)


# kernels of one forward pass from 2^18 pixels on: the input packing, eleven
# convolutions and two poolings (counted from an ncu launch list at 2048^2)
FWD_LAUNCHES = 14


def run_denoiser_fwd(args, rank, world, local_rank):
    """Tensor-core throughput of the denoiser's forward pass on one large
    sample: K forwards timed with CUDA events on the launching stream, the
    input resident in HBM; end to end, the same forwards from a host buffer
    (the library stages it and copies the result back)."""
    import torch
    from paper_2501_14795_gb300 import denoise as dn
    from paper_2501_14795_gb300 import pic

    torch.cuda.set_device(local_rank)
    kw = WORKLOADS[args.workload]["kw"]
    nx, ny = kw["nx"], kw["ny"]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(dn.SEED_DENOISER + 11)
    x = 0.03 * torch.randn((1, 3, ny, nx), device="cuda", generator=gen)
    o = torch.empty_like(x)
    net = pic.Denoiser(nx, ny, 1, 0.03)
    params = dn.init_params(dn.SEED_DENOISER + 7)
    rng = np.random.Generator(np.random.PCG64(dn.SEED_DENOISER + 8))
    params[-(9 * 32 * 3 + 3):] = rng.uniform(-0.05, 0.05, 9 * 32 * 3 + 3)  # a live last layer
    net.set_params(params.astype(np.float32))
    for _ in range(args.warmup):
        pic.pic_denoiser_forward(net.d, x, o, 1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            pic.pic_denoiser_forward(net.d, x, o, 1)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    xh = x.cpu().numpy()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oh = net.forward(xh)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    net.close()
    ms, e2e_ms = max_over_ranks(ms, e2e_ms)
    if rank != 0:
        return
    flops = dn.forward_flops(nx, ny)
    achieved = flops / (ms * 1e-3) / 1e12
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = float(json.load(open(p))["bf16_tflops"]) if os.path.exists(p) else 1900.0
    line = {
        "metric": "denoiser forward throughput", "value": achieved * world, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (accumulate f32)", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [nx, ny], "batch": 1,
                   "flops_per_forward": flops,
                   "l2": "inputs larger than L2 (one full-resolution activation 268 MB > 129 MB)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": f"whole forward pass ({FWD_LAUNCHES} launches)",
                     "peak_source": "measured bf16_tflops" if os.path.exists(p) else "fallback"},
        "e2e": {"value": flops / (e2e_ms * 1e-3) / 1e12 * world, "unit": "TFLOP/s",
                "h2d_bytes_per_step": xh.nbytes, "d2h_bytes_per_step": oh.nbytes},
        "gpu_launches": FWD_LAUNCHES * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2501_14795_gb300 import pic

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    w = make_workload(args.workload)
    if args.tile:
        w.tile = args.tile
    n = w.n_particles
    flags = pic.PIC_TIMING
    sim = pic.Simulation.from_workload(w, tile=w.tile, threads=args.threads, flags=flags,
                                       device=True, stream=stream.cuda_stream)
    sim.step(args.warmup)
    pic.pic_sync(sim.h)
    pic.pic_timing(sim.h, reset=True)
    l0 = pic.pic_kernel_launches(sim.h)
    n_start = sum(sim.diagnostics()["n_particles"])   # changes with a moving window
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    pic.pic_sync(sim.h)
    (adv_ms, sort_ms, field_ms), adv_n = pic.pic_timing_stages(sim.h, reset=True)
    launches = pic.pic_kernel_launches(sim.h) - l0
    d = sim.diagnostics()
    sim.close()
    del sim

    n_end = sum(d["n_particles"])
    if w.window is not None:
        n = 0.5 * (n_start + n_end)   # the count grows about linearly with the injection

    # ---- end to end through the C ABI from pinned host buffers ----
    host = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in sp.arrays()]
            for sp in w.species]
    fields_out = torch.empty(3 * w.nx * w.ny, dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for h in host for t in h)
    d2h = 2 * fields_out.numel() * 4 + 96
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    sim = pic.Simulation(pic.config_for(w, w.tile, args.threads, 0), stream.cuda_stream)
    if w.window is not None:
        sim.set_moving_window(w.window)
    for k, h in enumerate(host):
        pic.pic_load_particles(sim.h, k, *h)
    for laser in w.lasers:
        sim.add_laser(**laser)
    sim.step(args.steps)
    pic.pic_get_fields(sim.h, pic.FIELD_E, fields_out)
    pic.pic_get_fields(sim.h, pic.FIELD_B, fields_out)
    pic.pic_diagnostics(sim.h)
    e2e_s = time.perf_counter() - t0
    sim.close()

    # ---- max over ranks ----
    ms, e2e_ms = max_over_ranks(ms, e2e_s * 1e3)
    if rank != 0:
        return
    total = n * world
    value = whole_job_rate(n, world, args.steps, ms)
    peak, peak_kind = read_peaks()
    T = w.tile
    cells = w.nx * w.ny
    # algorithmic bytes of one particle-advance launch: each particle's 24 B
    # state read and written once, each cell's E|B (24 B) read and J (12 B)
    # written once
    alg_push = 48.0 * n + 36.0 * cells
    per_launch_s = (adv_ms / max(adv_n, 1)) * 1e-3
    achieved = alg_push / per_launch_s / 1e9
    leavers = d["leavers"]
    f_leave = leavers / n if n else 0.0
    step_bytes = 48.0 + 48.0 * f_leave + 96.0 * cells / n
    config = dict(workload_config(args.workload, w, args.threads),
                  parallelism=f"replicas x{world}" if world > 1 else "single GPU")
    if w.window is not None:
        config.update(moving_window=True, particles_start=n_start, particles_end=n_end,
                      window_moves=d.get("window_moves"),
                      particles="mean of start and end (the window injects plasma)")
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(args.workload),
                     "kernel": "k_push (gather+Boris+move+deposit+leaver emission)",
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "bytes_per_launch": alg_push, "launch_ms": per_launch_s * 1e3},
        # the same kernel against its own ceiling, instruction issue
        "issue_roofline": issue_roofline(args.workload, n / per_launch_s, clocks["sm_mhz"]),
        "step_hbm": {"bytes_per_particle": step_bytes, "leaver_fraction_last_step": f_leave,
                     "achieved_gbs": step_bytes * value / world / 1e9,
                     "frac": step_bytes * value / world / 1e9 / peak},
        # CUDA events on the simulation's stream around each stage of every
        # timed step (per step, in ms); re-sort algorithmic bytes: each
        # leaver's 24 B state read and written once more (2 S_p f_leave of the
        # step's bytes per particle)
        # "field_not_hidden": the field advance runs beside the re-sort's
        # eviction and fill; this is the part of it that ends after the fill
        "stages_ms_per_step": {"advance": adv_ms / max(adv_n, 1), "resort": sort_ms / max(adv_n, 1),
                               "field_not_hidden": field_ms / max(adv_n, 1)},
        "resort_hbm": {"moved_particles_last_step": leavers,
                       "bytes_per_step": 48.0 * leavers,
                       "achieved_gbs": 48.0 * leavers / (sort_ms / max(adv_n, 1) * 1e-3) / 1e9
                       if sort_ms > 0 else None},
        "e2e": {"value": total * args.steps / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "status_bits": d["status_bits"],
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="thermal_2048", choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--tile", type=int, default=0, help="override the workload's tile size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "batched_64":
            run_batched(args, rank, world, local_rank)
        elif args.workload == "denoiser":
            run_denoiser(args, rank, world, local_rank)
        elif WORKLOADS[args.workload]["kind"] == "denoiser_fwd":
            run_denoiser_fwd(args, rank, world, local_rank)
        elif WORKLOADS[args.workload]["kind"] == "denoiser_train":
            run_denoiser_train(args, rank, world, local_rank)
        else:
            run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
