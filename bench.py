#!/usr/bin/env python
"""Benchmark of the reactive lattice Boltzmann step on one GB300 (or N independent replicas).

Default workload: 3D reactive dissolution, 256^3 seeded random-sphere packing (porosity 0.4),
D3Q19 MRT flow + D3Q7 solute, wet-node reaction, solid consumption with geometry flips, FP32.
A "step" is one time step of the whole path (fused collide-stream, interface detection and
flips, monitors every N_mon steps).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload dissolution|droplet|channel|combustion] [--precision fp32|fp16|bf16|fp64|fp16s32|bf16s32]
                  [--size S] [--no-e2e] [--no-cpu]
  python bench.py --workload dissolution --size 128 --to-steady 1e-6
                  (time to steady state from rest, geometry frozen; its own JSON line)
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2502_12955_gb300 import inputs  # noqa: E402

PEAK_FALLBACK_GBS = 6800.0
PROFILES = os.path.join(ROOT, "profiles")


# ------------------------------------------------------------------ workloads

def workload(name, size, precision):
    """(cfg, geom, fields, label) of a bench workload."""
    if name == "dissolution":
        n = size or 256
        cfg, geom, fields = inputs.dissolution_3d(n=n, precision=precision)
        label = f"dissolution3d_{n}^3_d3q19mrt_d3q7_{precision}"
    elif name == "droplet":
        n = size or 128
        cfg, geom, fields = inputs.droplet_3d(n=n, radius=n / 8.0, precision=precision)
        label = f"droplet3d_{n}^3_2x_d3q19_shanchen_{precision}"
    elif name == "channel":
        cfg, geom, fields = inputs.reactive_channel_2d(precision=precision)
        label = f"channel2d_128x64_d2q9_d2q5_{precision}"
    elif name == "combustion":
        # the paper's reactive porous channel (Sec. 3.4) at its 420 x 80: velocity inlet, O2,
        # temperature and CO2 lattices, temperature-dependent rate, conduction in the solid
        cfg, geom, fields = inputs.combustion_channel_2d(precision=precision)
        label = f"combustion2d_420x80_d2q9_3xd2q5_conjugate_{precision}"
    else:
        raise SystemExit(f"unknown workload {name}")
    cfg = dict(cfg, precision=precision, N_mon=100)
    return cfg, geom, fields, label


L2_BYTES = 129e6   # GB300 L2

# bytes per stored (flow, scalar) population of each storage mode; the *s32 modes keep the
# scalar lattices in FP32
ELEM = {"fp64": (8, 8), "fp32": (4, 4), "fp16": (2, 2), "bf16": (2, 2), "fp16s32": (2, 4), "bf16s32": (2, 4)}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f16 storage, f32 math", "bf16": "bf16 storage, f32 math",
         "fp16s32": "f16 flow / f32 scalar storage, f32 math", "bf16s32": "bf16 flow / f32 scalar storage, f32 math"}


def bytes_per_fluid_node(cfg):
    """Algorithmic HBM bytes per fluid node and step of the step kernel: one read and one write of
    every population of every fluid lattice (the reaction product's included).  The solid
    thermal lattice of conduction in the solid lives at solid nodes and has its own kernel."""
    q = 19 if cfg["dim"] == 3 else 9
    qc = 7 if cfg["dim"] == 3 else 5
    ef, es = ELEM[cfg["precision"]]
    n_lat = cfg.get("n_scal", 0) + (1 if cfg.get("product") else 0)
    return 2 * (ef * q * cfg.get("n_comp", 1) + es * qc * n_lat)


def source_hash():
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2502_12955_gb300", "csrc", "*.cu*"))):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(label):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it was
    taken on the current kernel sources; else None."""
    path = os.path.join(PROFILES, f"k_step_{label.split('_')[0]}_{label.split('_')[-1]}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != source_hash():
        return None
    return float(m_b.group(1))


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(path))["hbm_gbs"])
        return v, "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.device)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(name, precision, seconds=10.0, sample_n=64, steps=None, warmup=2):
    """Time the FP64 oracle (single thread) on a bounded sample of the workload."""
    from oracle.oracle import Oracle

    if name == "dissolution":
        cfg, geom, fields = inputs.dissolution_3d(n=sample_n, precision="fp64")
        sample = f"dissolution 3D {sample_n}^3 seeded packing (same recipe), MRT + D3Q7, FP64 oracle"
    elif name == "droplet":
        cfg, geom, fields = inputs.droplet_3d(n=sample_n, radius=sample_n / 8.0, precision="fp64")
        sample = f"droplet 3D {sample_n}^3, two components, FP64 oracle"
    elif name == "combustion":
        cfg, geom, fields = inputs.combustion_channel_2d(precision="fp64")
        sample = "combustion channel 2D 420x80 (the same input), FP64 oracle"
    else:
        cfg, geom, fields = inputs.reactive_channel_2d(precision="fp64")
        sample = "channel 2D 128x64, FP64 oracle"
    o = Oracle(cfg)
    o.set_geometry(geom)
    rho, u, C = fields
    o.set_fields(rho, u, C if o.p.n_scal else None)
    o.step(warmup)
    n = 0
    t0 = time.perf_counter()
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if steps is not None and n >= steps:
            break
        if steps is None and el >= seconds and n >= 3:
            break
    nodes = geom.size
    return {"value": nodes * n / el / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{sample}, {n} steps after {warmup} warm-up, {el:.1f} s",
            "steps": n, "seconds": el}


def oracle_full_size(name, size, steps=2, warmup=1):
    """The single-thread FP64 oracle on the benchmark's own input at full size (a few steps)."""
    from oracle.oracle import Oracle

    cfg, geom, fields, label = workload(name, size, "fp64")
    o = Oracle(dict(cfg, precision="fp64"))
    o.set_geometry(geom)
    rho, u, C = fields
    o.set_fields(rho, u, C if o.p.n_scal else None)
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    return {"value": geom.size * steps / el / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{label} at full size ({geom.size} nodes), FP64 oracle, {steps} steps after "
                      f"{warmup} warm-up, {el:.1f} s", "steps": steps, "seconds": el}


def _oracle_full_worker(job):
    return oracle_full_size(*job)


def _oracle_worker(job):
    name, precision, seconds, sample_n, steps, warmup = job
    return oracle_sample(name, precision, seconds=seconds, sample_n=sample_n, steps=steps, warmup=warmup)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_all_cores(name, precision, seconds=10.0, sample_n=64, steps=None, warmup=2, cores=None):
    """The single-thread FP64 oracle, unchanged, run as one independent replica per host core at
    once (spawned processes, no shared state): the aggregate MLUPS of the host's cores, next to
    one core's."""
    import multiprocessing as mp

    cores = cores or host_cores()
    job = (name, precision, seconds, sample_n, steps, warmup)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [job] * cores)
    total = sum(r["value"] for r in res)
    per_step_s = max(r["seconds"] / r["steps"] for r in res)
    one = res[0]
    return {"value": total, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent replicas (one per host core) of: {one['sample']}",
            "single_core_value": min(r["value"] for r in res), "steps": one["steps"],
            "seconds": max(r["seconds"] for r in res), "seconds_per_step": per_step_s}


# ------------------------------------------------------------------ main

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="dissolution",
                    choices=["dissolution", "droplet", "channel", "combustion", "ensemble", "nn"])
    ap.add_argument("--members", type=int, default=32,
                    help="ensemble workload: members, half 2D squares and half 3D cubes (512 = the full set)")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--size", type=int, default=0)
    ap.add_argument("--block-x", type=int, default=0)
    ap.add_argument("--l2-fetch", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-full-cpu", action="store_true",
                    help="skip the single-thread oracle steps on the full-size input")
    ap.add_argument("--to-steady", type=float, default=None,
                    help="instead of the timed steps: run from rest to residual <= this tolerance")
    ap.add_argument("--max-steps", type=int, default=2_000_000)
    ap.add_argument("--warm-start", action="store_true",
                    help="with --to-steady: train the encoder-decoder on solver steady states, then compare "
                         "time to steady state from rest and from its prediction on held-out geometries")
    ap.add_argument("--train-samples", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--test-samples", type=int, default=4)
    ap.add_argument("--net-width", default="",
                    help="warm start: channel widths of the encoder levels and the bottleneck, e.g. 16,32,64,160")
    ap.add_argument("--no-augment", action="store_true",
                    help="warm start: train on the samples only, without their y-z symmetric copies")
    return ap.parse_args()


def reduce_over_ranks(dist, device, seconds, units):
    """Whole-job figures of a replica run: the slowest rank's time and the units all ranks
    processed (each rank steps its own independent problem; no data-path collective)."""
    if dist is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    n = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    precision = args.precision or ("fp64" if args.workload == "channel" else "fp32")
    if args.workload == "ensemble":
        # the ensemble's members are independent 2D / 3D runs: sample the oracle on a 3D one
        args.workload = "dissolution"
        label = f"ensemble_{args.members}_members_{precision}"
    else:
        cfg, geom, fields, label = workload(args.workload, args.size, precision)
    # each timed step is one oracle step, on every host core at once, of a bounded sample of the
    # workload (48^3 in 3D)
    res = oracle_sample_all_cores(args.workload, precision, steps=args.steps, sample_n=48, warmup=args.warmup)
    value = res["value"]
    ms = res["seconds_per_step"] * 1e3
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": label, "reference": "FP64 CPU oracle (oracle/lbm_oracle.c)",
                       "sample": res["sample"]},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"], "single_core_value": res["single_core_value"]},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ensemble(args, dist, ws, rank, local):
    """Uneven ensemble (2D squares and 3D cubes of random porous media), every member advanced
    by the persistent tile-list kernel; one lattice per ensemble, both in the timed region."""
    import torch
    from paper_2502_12955_gb300.lbm import Ensemble

    precision = args.precision or "fp16"
    n2d = args.members // 2
    n3d = args.members - n2d
    sets = inputs.ensemble_members(n2d, n3d, seed0=1000 * local, precision=precision)
    stream = torch.cuda.Stream(device=local)
    ens, nodes, fluid, bpn = [], 0, 0, 0.0
    ef, es = ELEM[precision]
    for members in sets:
        if not members:
            continue
        e = Ensemble([dict(c, device=local, N_mon=0) for c, _, _ in members], stream=stream.cuda_stream)
        for (cfg, geom, fields), m in zip(members, e.members):
            m.set_geometry(geom)
            m.set_fields(*fields)
            nf = int((geom == 0).sum())
            nodes += geom.size
            fluid += nf
            q, qc = (19, 7) if cfg["dim"] == 3 else (9, 5)
            bpn += nf * 2 * (ef * q + es * qc)
        ens.append(e)
    tiles = [e.autotune(steps=4) for e in ens]
    for e in ens:
        e.step(args.warmup + (args.warmup & 1))
    torch.cuda.synchronize()
    launches0 = sum(e.launch_count() for e in ens)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for e in ens:
        e.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = sum(e.launch_count() for e in ens) - launches0
    sec, nodes_all = reduce_over_ranks(dist, f"cuda:{local}", ms_total * 1e-3, nodes * args.steps)
    ms_step = sec * 1e3 / args.steps
    peak, peak_src = measured_peak()
    achieved = bpn / (ms_step * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": nodes_all / sec / 1e6, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[precision],
            "data": "synthetic (seeded porous geometries, inputs.ensemble_members)",
            "config": {"workload": f"ensemble_{args.members}_members_{n2d}x2d_{n3d}x3d_{precision}",
                       "nodes": nodes, "fluid_nodes": fluid, "tile_threads": tiles,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": f"population state {bpn / 2 / 1e9:.2f} GB > 0.13 GB L2: no flush needed"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                         "kernel": "k_step_tiles (whole step time: one tile-list launch per step)",
                         "algorithmic_bytes_per_launch": bpn},
            "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    for e in ens:
        e.close()
    if dist:
        dist.destroy_process_group()


def run_to_steady(args, local):
    """Time to steady state of plain LBM from rest (the baseline a warm start is compared
    against): the geometry update is frozen, the residual r (relative L2 change of u and C over
    N_mon = 100 steps, the larger of the two) is evaluated on the device every 100 steps, and
    the run stops at the first evaluation with r <= tol.  Wall time between CUDA events on the
    solver's stream, including the host reads of r."""
    import torch
    from paper_2502_12955_gb300.lbm import Solver

    precision = args.precision or ("fp64" if args.workload == "channel" else "fp32")
    cfg, geom, fields, label = workload(args.workload, args.size, precision)
    cfg = dict(cfg, device=local, geo_mode="none", N_mon=100)
    stream = torch.cuda.Stream(device=local)
    s = Solver(cfg, stream=stream.cuda_stream)
    s.set_geometry(geom)
    rho, u, C = fields
    s.set_fields(rho, u, C if s.n_scal else None)
    s.sync()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps, r = 0, float("inf")
    while steps < args.max_steps:
        s.step(100)
        steps += 100
        r = s.monitors()["residual"]
        if 0.0 <= r <= args.to_steady:
            break
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    clk = clocks.stop()
    line = {"metric": "time_to_steady", "value": sec, "unit": "s", "n_gpus": 1, "steps": steps,
            "higher_is_better": False, "converged": bool(0.0 <= r <= args.to_steady),
            "residual": r, "tol": args.to_steady, "start": "rest (uniform density, zero velocity)",
            "dtype": DTYPE[precision],
            "data": "synthetic (seeded geometry, inputs/ recipe), geometry update frozen",
            "config": {"workload": label, "nodes": int(geom.size), "fluid_nodes": int((geom == 0).sum())},
            "mlups": geom.size * steps / sec / 1e6, "clocks": clk}
    print(json.dumps(line), flush=True)
    s.close()


def measured_tensor_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops"]), "measured (burst)"
    except Exception:
        return 1900.0, "fallback"


def run_nn(args, local):
    """The warm-start network's training step at 128^3 (forward, backward, Adam; BF16 tensor-core
    GEMMs) on the seed-0 packing's features with synthetic targets, and the tcgen05 GEMM alone on
    a square-ish BF16 problem against the measured BF16 tensor peak."""
    import torch
    from paper_2502_12955_gb300 import surrogate

    torch.cuda.set_device(local)
    n = args.size or 128
    _, geom, _ = inputs.dissolution_3d(n=n)
    net = surrogate.WarmStartNet(device=local)
    x = surrogate.features(geom, device=local)
    rng = np.random.default_rng(0)
    t = torch.tensor(rng.standard_normal((geom.size, 4)).astype(np.float32), device=f"cuda:{local}")
    fl = torch.tensor((geom == 0).reshape(-1).astype(np.uint8), device=f"cuda:{local}")
    nf = int((geom == 0).sum())
    for _ in range(max(3, args.warmup)):
        net.train_step(x, t, fl, nf, geom.shape, lr=1e-4)
    net.check()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        net.train_step(x, t, fl, nf, geom.shape, lr=1e-4)
    e1.record(st)
    torch.cuda.synchronize()
    net.check()
    ms = e0.elapsed_time(e1) / args.steps
    # the GEMM alone, a compute-bound shape: M x N x K = 38912 x 1024 x 4096 (128 x 256 tiles, four
    # along N sharing each A tile in L2, 1216 tiles = 8 waves over 152 SMs), BF16 in, FP32
    # accumulate, BF16 out
    M, N, K = 38912, 1024, 4096
    A = torch.randn((M, K), device=f"cuda:{local}").to(torch.bfloat16)
    B = torch.randn((N, K), device=f"cuda:{local}").to(torch.bfloat16)
    C = torch.empty((M, N), device=f"cuda:{local}", dtype=torch.bfloat16)
    for _ in range(3):
        surrogate.lbm_nn_gemm_tn(A, B, C, N, M, N, K, 1, surrogate.OUT_BF16, None)
    reps = 20
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        surrogate.lbm_nn_gemm_tn(A, B, C, N, M, N, K, 1, surrogate.OUT_BF16, None)
    e1.record(st)
    torch.cuda.synchronize()
    net.check()
    gms = e0.elapsed_time(e1) / reps
    tflops = 2.0 * M * N * K / (gms * 1e-3) / 1e12
    peak, src = measured_tensor_peak()
    line = {"metric": "train_steps_per_s", "value": 1e3 / ms, "unit": "steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "dtype": "bf16 weights and activations, f32 accumulate and master weights",
            "data": "synthetic targets on the seed-0 packing's features",
            "config": {"workload": f"warm_start_net_{n}^3_train_step", "params": net.n_params,
                       "width": list(net.width)},
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "traffic": None, "peak_source": src,
                         "kernel": "k_gemm_tn<256>", "shape": [M, N, K], "kernel_ms": gms}}
    print(json.dumps(line), flush=True)


def run_warm_start(args, local):
    """Learned warm start against plain LBM from rest (the dissolution workload's recipe at the
    given size, default 128^3): generate solver steady states (r <= 1e-5) on seeded training
    geometries with Pe and Da drawn log-uniform in [5, 10] and [0.05, 0.2], train the encoder-decoder, then on held-out
    seeds run to r <= tol from rest and from the prediction.  value = mean warm time to steady
    (network inference included); the rest time, step counts and the speed-up are beside it."""
    import torch
    from paper_2502_12955_gb300 import surrogate, warmstart

    n = args.size or 128
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    samples, gen = warmstart.generate(args.train_samples, n=n, tol=1e-5, device=local)
    t_gen = time.perf_counter() - t0
    width = tuple(int(v) for v in args.net_width.split(",")) if args.net_width else (16, 32, 64, 160)
    net = surrogate.WarmStartNet(width=width, device=local)
    t0 = time.perf_counter()
    hist = warmstart.train(net, samples, args.epochs, augment=not args.no_augment)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del samples
    seeds = [20_000 + i for i in range(args.test_samples)]
    rows = warmstart.compare(net, seeds, n=n, tol=args.to_steady, max_steps=args.max_steps, device=local)
    # a warm run that failed (non-finite, or another end state) falls back to the rest run's cost
    for r in rows:
        if not r["converged_warm"]:
            r["warm_s"] = r["rest_s"] + r["warm_s"]
            r["warm_steps"] = r["rest_steps"] + r["warm_steps"]
    rest_s = float(np.mean([r["rest_s"] for r in rows]))
    warm_s = float(np.mean([r["warm_s"] for r in rows]))
    rest_k = float(np.mean([r["rest_steps"] for r in rows]))
    warm_k = float(np.mean([r["warm_steps"] for r in rows]))
    speed = rest_s / warm_s
    line = {"metric": "time_to_steady", "value": warm_s, "unit": "s", "n_gpus": 1,
            "higher_is_better": False, "start": "learned warm start (encoder-decoder prediction)",
            "rest_value": rest_s, "speedup_time": speed, "speedup_steps": rest_k / warm_k,
            "warm_steps_mean": warm_k, "rest_steps_mean": rest_k, "tol": args.to_steady,
            "target_speedup": 3.0, "target_met": bool(speed >= 3.0),
            "all_converged": all(r["converged"] for r in rows),
            "dtype": "f32 LBM; network bf16 weights and activations, f32 accumulate",
            "data": "synthetic (seeded sphere packings, dissolution recipe), geometry update frozen",
            "config": {"workload": f"dissolution3d_{n}^3_warm_start", "train_samples": args.train_samples,
                       "epochs": args.epochs, "params": net.n_params, "held_out_seeds": seeds, "width": list(width),
                       "augment_yz_symmetries": not args.no_augment},
            "train_loss_first_last": [hist[0], hist[-1]], "generate_s": t_gen, "train_s": t_train,
            "train_steps_mean": float(np.mean([g["steps"] for g in gen if g["converged"]])),
            "train_cases_skipped": [g for g in gen if not g["converged"]],
            "cases": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod

        dist_mod.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = dist_mod

    from paper_2502_12955_gb300.lbm import Solver

    if args.workload == "ensemble":
        run_ensemble(args, dist, ws, rank, local)
        return
    if args.workload == "nn":
        if rank == 0:
            run_nn(args, local)
        return
    if args.warm_start and args.to_steady is None:
        args.to_steady = 1e-6   # the warm start is judged by the time to r <= 1e-6
    if args.to_steady is not None:
        if rank == 0:
            (run_warm_start if args.warm_start else run_to_steady)(args, local)
        return
    precision = args.precision or ("fp64" if args.workload == "channel" else "fp32")
    cfg, geom, fields, label = workload(args.workload, args.size, precision)
    cfg = dict(cfg, device=local, block_x=args.block_x, l2_fetch_bytes=args.l2_fetch)
    stream = torch.cuda.Stream(device=local)
    s = Solver(cfg, stream=stream.cuda_stream)
    s.set_geometry(geom)
    rho, u, C = fields
    s.set_fields(rho, u, C if s.n_scal else None)
    N = geom.size
    Nf = int((geom == 0).sum())
    s.step(args.warmup)
    s.sync()

    # ---------------- timed region: K steps, inputs resident in HBM
    def barrier():
        if dist:
            dist.barrier()

    launches0 = s.launch_count()
    # a state smaller than L2 would stay cached between steps: then L2 is flushed before every
    # timed step (a 256 MB write on the same stream, outside the timed intervals)
    bpn = bytes_per_fluid_node(cfg)
    state_bytes = N * bpn / 2
    flush = state_bytes <= L2_BYTES
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}") if flush else None
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    if flush:
        ms_total = 0.0
        evs = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush_buf.zero_()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            s.step(1)
            a1.record(stream)
            evs.append((a0, a1))
        torch.cuda.synchronize()
        ms_total = sum(a0.elapsed_time(a1) for a0, a1 in evs)
    else:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_total = e0.elapsed_time(e1)
    barrier()
    clk = clocks.stop()
    launches = s.launch_count() - launches0
    s.sync()
    # per-launch duration of the fused step kernel: a separate pass with CUDA events around every
    # k_step launch on the solver's stream (kept out of the timed region above)
    rsteps = max(2, 2 * (min(args.steps, 100) // 2))
    s.profile(True)
    s.profile_read()
    s.step(rsteps)
    kern_ms, kern_n = s.profile_read()
    s.profile(False)
    s.sync()
    dev = f"cuda:{local}"
    sec, nodes_all = reduce_over_ranks(dist, dev, ms_total * 1e-3, N * args.steps)
    _, fluid_all = reduce_over_ranks(dist, dev, 0.0, Nf * args.steps)
    ms_total = sec * 1e3
    ms_step = ms_total / args.steps
    mlups = nodes_all / sec / 1e6
    mflups = fluid_all / sec / 1e6
    mon = s.monitors()

    # roofline of the fused step kernel (per launch, CUDA events on the launching stream)
    algo_bytes = Nf * bpn
    kavg_ms = kern_ms / max(1, kern_n)
    achieved = algo_bytes / (kavg_ms * 1e-3) / 1e9
    peak, peak_src = measured_peak()
    # with Shan-Chen forces the timed population pass is the psi pass plus the fused step, and the
    # bytes are the step's (one read and one write of every population of both components)
    sc_on = any(v != 0 for row in cfg.get("G", [[0.0, 0.0], [0.0, 0.0]]) for v in row)
    kernel = "k_psi + k_step" if sc_on else "k_step"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": profile_traffic(label),
                "peak_source": peak_src, "kernel": kernel, "kernel_ms": kavg_ms,
                "algorithmic_bytes_per_launch": algo_bytes,
                "bytes_per_fluid_node": bpn}

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        ke = max(10, min(args.steps, 100))
        flags_h = torch.from_numpy(np.ascontiguousarray(geom, dtype=np.uint8)).pin_memory().numpy()
        rho_h = torch.from_numpy(np.ascontiguousarray(rho)).pin_memory().numpy()
        u_h = torch.from_numpy(np.ascontiguousarray(u)).pin_memory().numpy()
        C_h = torch.from_numpy(np.ascontiguousarray(C)).pin_memory().numpy() if s.n_scal else None
        # the read-back lands in preallocated pinned buffers (Solver.fields(out=...))
        sh = tuple(s.shape)

        def pinned(shape, dt):
            return torch.empty(shape, dtype=dt).pin_memory().numpy()

        out_h = {"rho": pinned((s.n_comp,) + sh, torch.float64), "u": pinned((3,) + sh, torch.float64),
                 "C": pinned((s.n_scal,) + sh, torch.float64), "flags": pinned(sh, torch.uint8),
                 "acc": pinned(sh, torch.float64)}
        phases = {}

        def e2e_pass(k):
            ts = [time.perf_counter()]
            s.set_geometry(flags_h)
            ts.append(time.perf_counter())
            s.set_fields(rho_h, u_h, C_h)
            ts.append(time.perf_counter())
            for _ in range(k):
                s.step(1)
                s.sync()          # per-step read of the device status word (4 bytes)
            ts.append(time.perf_counter())
            o = s.fields(out=out_h)
            ts.append(time.perf_counter())
            phases.update({n: 1e3 * (b - a) for n, a, b in
                           zip(("set_geometry", "set_fields", "steps", "get_fields"), ts[:-1], ts[1:])})
            return o

        e2e_pass(2)               # untimed warm-up of the host path (first use of the pinned buffers)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = e2e_pass(ke)
        torch.cuda.synchronize()
        barrier()
        el, e2e_nodes = reduce_over_ranks(dist, dev, time.perf_counter() - t0, N * ke)
        h2d = geom.nbytes + rho.nbytes + u[: (3 if cfg["dim"] == 3 else 2)].nbytes + (C.nbytes if s.n_scal else 0)
        d2h = 4 * ke + sum(v.nbytes for v in out.values())
        e2e = {"value": e2e_nodes / el / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / ke,
               "d2h_bytes_per_step": d2h / ke, "steps": ke, "phases_ms": phases,
               "includes": "set_geometry + set_fields from pinned host memory, per-step lbm_step + "
                           "lbm_sync (4-byte status read), final lbm_get_fields into pinned host memory; "
                           "after one untimed pass of the same calls with 2 steps"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_sample_all_cores(args.workload, precision, seconds=12.0)
        if args.workload == "dissolution" and not args.no_full_cpu:
            import multiprocessing as mp

            with mp.get_context("spawn").Pool(1) as pool:
                cpu["full_size_single_thread"] = pool.map(_oracle_full_worker,
                                                          [(args.workload, args.size, 2, 1)])[0]

    q = 19 if cfg["dim"] == 3 else 9
    qc = 7 if cfg["dim"] == 3 else 5
    state_gb = state_bytes / 1e9   # one stored copy of every population of every node
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[precision],
            "data": "synthetic (seeded geometry, inputs/ recipe)",
            "config": {"workload": label, "nodes": N, "fluid_nodes": Nf,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": (f"population state {state_gb:.4f} GB <= L2: L2 flushed (256 MB write) before "
                              "every timed step, each step timed alone" if flush else
                              f"population state {state_gb:.2f} GB > 0.13 GB L2: no flush needed"),
                       "mflups": mflups, "achieved_gbs_step": Nf * bpn / (ms_step * 1e-3) / 1e9,
                       "mass": mon["mass0"], "n_solid": mon["nsolid"], "nonfinite": mon["nonfinite"]},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
