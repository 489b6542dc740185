#!/usr/bin/env python3
"""Benchmark of the GB300 Wilson-Dirac hot path (one JSON line on stdout).

Workload (default): mixed-precision even-odd CG on a 32^3x64 lattice,
kappa = 0.1245, links exp(0.25 i H), Gaussian source, FP16 per-site-scaled
spinor and FP16 link storage with FP32 arithmetic, FP64 reliable updates when
the inner residual drops by delta = 0.1, FP64 reductions, 1e-10 true relative
residual.  One step = one complete solve through the C ABI (source packing,
the CG with every Dslash, the reliable updates, unpacking of x), inputs
resident in HBM.  The metric is the sustained Wilson Dslash rate over the
solve, 1320 flop per output site per parity apply, next to the plain FP64 CG
on the same inputs and the isolated FP16 Dslash kernel against the HBM
roofline.

The oracle (plain numpy FP64) is timed on the host cores after the GPU
work, on one core and on every core, per parity apply and per CG iteration
for each workload (cpu_baseline).  --impl reference times the same oracle on
the headline workload: each step is one parity Dslash of the 32^3x64 lattice
over every host core.
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 64)
KAPPA = 0.1245
EPS = 0.25
BC = (1.0, 1.0, 1.0, -1.0)
DELTA = 0.1
TOL = 1e-10
CONFIG_ID = 2
FLOP_PER_SITE = 1320
WORKLOAD = "eo-mixed-fp16-cg-32x32x32x64"
METRIC = "Wilson Dslash GFLOP/s & HBM GB/s; mixed-vs-FP64 CG time at 1e-10 residual"
# algorithmic bytes per output site of one parity apply (FP16 storage, 12-real links):
# 8 links x 24 B + input spinor 48 B + its FP32 scale + output 48 B + scale
BYTES_PER_SITE_F16 = 8 * 24 + 52 + 52
BYTES_PER_SITE_F32 = 8 * 48 + 96 + 96
# FP64 peak of this part derived from its unit counts and clock, reported
# beside the measured one: 152 SMs x 2 DFMA per SM per cycle (the peak of
# ncu's DFMA instruction counter) x 2 flop x 2.07 GHz maximum SM clock.
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per launch of the hopping kernel at 32^3x64 from
# one ncu capture, with the digest of the kernel sources at capture time: the
# figure is reported only while the sources still have that digest, else the
# traffic is null (the kernel changed since the counters were taken).
KERNEL_SOURCES = ["cola_internal.cuh", "cola_impl.h", "dslash_kernel.cuh", "dslash.cu"]
NCU_TRAFFIC = {"f64": (1.6092e9, "a662dc36afcc8273"), "f16": (299.8e6, "a662dc36afcc8273")}


def kernel_source_digest():
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2302_00850_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(prec):
    nbytes, digest = NCU_TRAFFIC[prec]
    return nbytes if digest is not None and digest == kernel_source_digest() else None


FP64_PEAK_MEASURED = [FP64_PEAK_DERIVED_TFLOPS]  # replaced by the measurement of this run


def measure_fp64_peak(cola, dev, stream, reps=5):
    """FP64 arithmetic rate of this GPU now: independent DFMA chains (the
    library's probe kernel) on 8 blocks per SM, timed with CUDA events on the
    launching stream after a warm-up launch; best of `reps` launches."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, steps = 8 * sms, 256, 4096
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    cola.api.probe_fp64_fma(out, blocks, threads, steps)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flop = cola.api.probe_fp64_fma(out, blocks, threads, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        tf = flop / (e0.elapsed_time(e1) * 1e-3) / 1e12
        best = tf if best is None else max(best, tf)
    return best


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def aggregate_ranks(t_ms, units, device=None):
    """Whole-job timing over the ranks of a replicas run: (max time, summed units).

    Every rank solves its own copy of the workload (no data-path collective);
    only these two scalars cross ranks.  Without an initialised process group
    this is the identity.
    """
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_ms), float(units)
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------ CPU oracle --
# The oracle (plain numpy FP64) timed on the host cores, on one core and on
# every core.  The all-core figure splits one parity apply into disjoint site
# chunks and runs the oracle's own hop_sites on each in a process pool.  The
# pool is started by fork from a process that has made no CUDA call (the
# bench runs this study in a child process after its GPU work, and the
# reference arm never touches the GPU), so the children inherit the inputs
# without copies.

# (name, lattices, link scale eps, kappa, seed config, right-hand sides per lattice)
CPU_CONFIGS = [
    ("4x4x4x4", [(4, 4, 4, 4)], 0.3, 0.12, 0, 1),
    ("16x16x16x32", [(16, 16, 16, 32)], 0.3, 0.125, 1, 1),
    ("32x32x32x64", [(32, 32, 32, 64)], 0.25, 0.1245, 2, 1),
    ("24x24x24x48-12-point-sources", [(24, 24, 24, 48)], 0.3, 0.124, 3, 12),
    ("batch-8^4+12^3x24+16^3x32+24^3x48-x4", [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), (24, 24, 24, 48)],
     0.3, 0.124, 3, 4),
]
_CPU_FIELDS = {}  # lattice key -> (u, psi); set before the pool forks


def _lat_key(dims):
    return "x".join(map(str, dims))


def _cpu_hop_chunk(task):
    """One site chunk of a parity apply (runs in a pool worker)."""
    import numpy as np

    import oracle

    key, sites = task
    u, psi = _CPU_FIELDS[key]
    return float(np.abs(oracle.hop_sites(u, psi, BC, sites)).sum())


def host_cpu_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform

    return {"cpu_model": model or "unknown", "machine": platform.machine(),
            "nproc": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()}


def _parity_sites(dims, parity=0):
    import numpy as np

    import oracle

    return np.nonzero(oracle.parity_of_sites(dims).ravel() == parity)[0].astype(np.int64)


def _cpu_vector_ops_s(dims):
    """One CG iteration's vector operations of the oracle's cg on one field."""
    import numpy as np

    from oracle import solve

    lx, ly, lz, lt = dims
    rng = np.random.default_rng(0)
    shape = (lt, lz, ly, lx, 4, 3)
    p, q, r, x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(4))
    t0 = time.perf_counter()
    pq = solve.vdot(p, q).real
    x = x + (1.0 / pq) * p
    r = r - (1.0 / pq) * q
    rho = solve.norm2(r)
    p = r + (rho / pq) * p
    return time.perf_counter() - t0


def oracle_cpu_study(fields, fp64_iters, full=False, pool_procs=None):
    """Oracle timings on this host.

    fields: lattice key -> (u, psi) canonical numpy arrays (may be memory
    mapped); fp64_iters: config name -> iterations of the plain FP64 GPU solve
    of that workload (for the labelled extrapolations).  full: also run the
    whole oracle solve of the 16^3x32 workload (minutes on one core).
    """
    import multiprocessing as mp

    import numpy as np

    import oracle

    info = host_cpu_info()
    nproc = pool_procs or info["nproc"]
    _CPU_FIELDS.clear()
    _CPU_FIELDS.update(fields)
    apply1, applyn, vec = {}, {}, {}
    pool = mp.get_context("fork").Pool(nproc)
    try:
        for key, (u, psi) in fields.items():
            dims = tuple(int(v) for v in key.split("x"))
            sites = _parity_sites(dims)
            tasks = [(key, c) for c in np.array_split(sites, nproc)]
            pool.map(_cpu_hop_chunk, tasks)  # pages the inputs in
            t0 = time.perf_counter()
            oracle.hop_sites(u, psi, BC, sites)
            apply1[key] = time.perf_counter() - t0
            t0 = time.perf_counter()
            pool.map(_cpu_hop_chunk, tasks)
            applyn[key] = time.perf_counter() - t0
            vec[key] = _cpu_vector_ops_s(dims)
    finally:
        pool.close()
        pool.join()
    out = {}
    for name, lats, eps, kappa, cfg, nrhs in CPU_CONFIGS:
        keys = [_lat_key(d) for d in lats]
        if not all(k in fields for k in keys):
            continue
        vh = sum(int(np.prod(d)) // 2 for d in lats)
        a1 = nrhs * sum(apply1[k] for k in keys)
        an = nrhs * sum(applyn[k] for k in keys)
        vv = nrhs * sum(vec[k] for k in keys)
        row = {"sites_per_parity": vh, "rhs": nrhs,
               "apply_s_1core": a1, "apply_s_allcore": an,
               "gflops_1core": FLOP_PER_SITE * vh * nrhs / a1 / 1e9,
               "gflops_allcore": FLOP_PER_SITE * vh * nrhs / an / 1e9,
               "iter_s_1core": 4 * a1 + vv, "iter_s_allcore": 4 * an + vv,
               "iter_kind": "derived: 4 parity applies (hop_sites) + the CG's vector operations timed on one core"}
        iters = fp64_iters.get(name)
        if iters:
            row["fp64_iters_gpu"] = iters
            row["solve_s_1core_extrapolated"] = iters * row["iter_s_1core"]
            row["solve_s_allcore_extrapolated"] = iters * row["iter_s_allcore"]
        out[name] = row
    # whole oracle solves (the oracle's own cg, one core)
    if "4x4x4x4" in fields:
        u, b = fields["4x4x4x4"]
        t0 = time.perf_counter()
        _, it, res = oracle.solve_normal_full(np.asarray(u), np.asarray(b), 0.12, BC, tol=TOL)
        dt = time.perf_counter() - t0
        out["4x4x4x4"].update({"solve_s_1core_measured": dt, "solve_iters": it, "solve_true_rel_resid": res,
                               "solve_kind": "oracle.solve_normal_full (CG on D^dag D), one core"})
    if full and "16x16x16x32" in fields:
        u, b = fields["16x16x16x32"]
        t0 = time.perf_counter()
        _, it, res = oracle.solve_normal_eo(np.asarray(u), np.asarray(b), 0.125, BC, tol=TOL)
        dt = time.perf_counter() - t0
        out["16x16x16x32"].update({"solve_s_1core_measured": dt, "solve_iters": it, "solve_true_rel_resid": res,
                                   "iter_s_1core_measured": dt / max(it, 1),
                                   "solve_kind": "oracle.solve_normal_eo (CG on Mhat^dag Mhat), one core"})
    info.update({"pool_processes": nproc, "configs": out})
    return info


def cpu_study_inputs(device):
    """Inputs of the CPU study on `device` (numpy on the host): lattice key ->
    (links, source), the links and sources of each workload."""
    import synth

    fields = {}
    for name, lats, eps, kappa, cfg, nrhs in CPU_CONFIGS:
        for k, d in enumerate(lats):
            key = _lat_key(d)
            if key in fields:
                continue
            seed_u = synth.seed_for(cfg, 0) if len(lats) == 1 else synth.seed_for(cfg, 4 + k)
            u = synth.gauge_field_device(d, eps, seed_u, device=device).cpu().numpy()
            b = synth.gaussian_spinor_device(d, synth.seed_for(cfg, 1), device=device).cpu().numpy()
            fields[key] = (u, b)
    return fields


def config1_fp64_iters(cola, dev):
    """Iterations of the plain FP64 even-odd GPU solve of the 16^3x32 workload."""
    import synth

    d = (16, 16, 16, 32)
    u = synth.gauge_field_device(d, 0.3, synth.seed_for(1, 0), device=dev)
    b = synth.gaussian_spinor_device(d, synth.seed_for(1, 1), device=dev)
    g = cola.Gauge(u, d, 0.125, BC, precisions=("f64",), recon={"f64": 12})
    _, info = cola.cg_solve(g, b, tol=TOL, op="eo", inner="f64", use_graph=True)
    return info[0].iters


def run_cpu_study_child(args):
    """--cpu-study DIR: the oracle timings on inputs saved under DIR (a
    process without CUDA), one JSON line on stdout."""
    import numpy as np

    spec = json.load(open(os.path.join(args.cpu_study, "spec.json")))
    fields = {}
    for key in spec["lattices"]:
        fields[key] = (np.load(os.path.join(args.cpu_study, f"u_{key}.npy")),
                       np.load(os.path.join(args.cpu_study, f"b_{key}.npy")))
    print(json.dumps(oracle_cpu_study(fields, spec["fp64_iters"], full=args.cpu_full)), flush=True)


def cpu_baseline_from_study(study):
    """The bench line's cpu_baseline object: the headline workload's parity
    apply on every core, with the whole study beside it."""
    head = study["configs"]["32x32x32x64"]
    return {"value": head["gflops_allcore"], "unit": "GFLOP/s", "cores": study["pool_processes"], "kind": "oracle",
            "sample": "one oracle parity Dslash (hop_sites, numpy FP64) over the 1,048,576 even sites of 32^3x64, "
                      f"in {study['pool_processes']} site chunks on as many processes; per-config table beside it",
            "cpu_model": study["cpu_model"], "nproc": study["nproc"],
            "one_core_gflops": head["gflops_1core"], "configs": study["configs"]}


def run_cpu_study_from_gpu_arm(cola_iters, full=False):
    """Save the study's inputs (drawn on the GPU) and time the oracle in a child process."""
    import shutil

    import numpy as np
    import torch

    d = tempfile.mkdtemp(prefix="cola_cpu_study_")
    try:
        fields = cpu_study_inputs(torch.device("cuda", torch.cuda.current_device()))
        for key, (u, b) in fields.items():
            np.save(os.path.join(d, f"u_{key}.npy"), u)
            np.save(os.path.join(d, f"b_{key}.npy"), b)
        del fields
        with open(os.path.join(d, "spec.json"), "w") as f:
            json.dump({"lattices": [_lat_key(l) for _, lats, *_ in CPU_CONFIGS for l in lats],
                       "fp64_iters": cola_iters}, f)
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-study", d] + (["--cpu-full"] if full else [])
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=3600)
        if r.returncode != 0:
            return {"error": f"cpu study exited {r.returncode}: {r.stderr[-400:]}"}
        return json.loads(r.stdout.strip().splitlines()[-1])
    finally:
        shutil.rmtree(d, ignore_errors=True)


def run_reference(args):
    """--impl reference: the oracle on the host cores, on the bench's workload.

    Each step is a bounded sample of the same workload: one parity Dslash of
    the 32^3x64 eo solve (the operator the solve applies four times per
    iteration), by the oracle's hop_sites over disjoint site chunks on every
    host core.  No GPU is used: the inputs are drawn by the seeded generator
    with torch on the CPU.
    """
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp

    import numpy as np

    import oracle
    import synth

    u = synth.gauge_field_device(DIMS, EPS, synth.seed_for(CONFIG_ID, 0), device="cpu").numpy()
    psi = synth.gaussian_spinor_device(DIMS, synth.seed_for(CONFIG_ID, 1), device="cpu").numpy()
    key = _lat_key(DIMS)
    _CPU_FIELDS.clear()
    _CPU_FIELDS[key] = (u, psi)
    info = host_cpu_info()
    nproc = info["nproc"]
    sites = _parity_sites(DIMS)
    vh = len(sites)
    tasks = [(key, c) for c in np.array_split(sites, nproc)]
    pool = mp.get_context("fork").Pool(nproc)
    try:
        for _ in range(args.warmup):
            pool.map(_cpu_hop_chunk, tasks)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_cpu_hop_chunk, tasks)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    value = FLOP_PER_SITE * vh * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(world),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": nproc, "kind": "oracle",
                         "sample": f"each step one oracle parity Dslash (hop_sites, numpy FP64) over the {vh} even "
                                   f"sites of 32^3x64 in {nproc} site chunks on as many processes",
                         "cpu_model": info["cpu_model"], "nproc": info["nproc"]},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def make_inputs(device):
    import torch

    import synth

    u = synth.gauge_field(DIMS, EPS, synth.seed_for(CONFIG_ID, 0), device=device, as_numpy=False)
    b = torch.from_numpy(synth.gaussian_spinor(DIMS, synth.seed_for(CONFIG_ID, 1))).to(device)
    return u, b


def bench_config(world):
    return {"workload": WORKLOAD, "lattice": "32x32x32x64", "kappa": KAPPA, "links": "exp(0.25 i H)",
            "inner": "f16 (per-site scale), 12-real links", "delta": DELTA, "tol": TOL,
            "l2": "inputs larger than L2 (FP16 links 201 MB, FP64 source 403 MB)",
            "parallelism": f"replicas{world}"}


def run_cola(args):
    import torch
    import torch.distributed as dist

    import paper_2302_00850_gb300 as cola

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    lx, ly, lz, lt = DIMS
    vol = lx * ly * lz * lt
    vh = vol // 2

    u, b = make_inputs(dev)
    g = cola.Gauge(u, DIMS, KAPPA, BC, precisions=("f64", "f16"), recon={"f64": 18, "f16": 12})

    use_graph = not args.host_loop

    def solve(inner="f16", bb=b, gg=g):
        return cola.cg_solve(gg, bb, tol=TOL, op="eo", inner=inner, delta=DELTA, use_graph=use_graph)

    for _ in range(args.warmup):
        x, info = solve()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    if args.profile_range:
        torch.cuda.profiler.start()
    ev0.record(stream)
    for _ in range(args.steps):
        x, info = solve()
        infos.append(info[0])
    ev1.record(stream)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    iters = [i.iters for i in infos]
    rus = [i.reliable_updates for i in infos]
    # parity Dslash applies per solve: 4 per iteration (inner precision) + 4 per FP64 residual
    n_ds = [4 * it + 4 * ru for it, ru in zip(iters, rus)]
    t_ms, flops = aggregate_ranks(ev0.elapsed_time(ev1), sum(FLOP_PER_SITE * vh * n for n in n_ds), dev)
    value = flops / (t_ms * 1e-3) / 1e9
    # kernels per solve: 9 set-up/finish launches (packing, |b|^2 and its
    # finishing kernel, the zero-guess check, initial residual and finisher,
    # final accumulate, unpacking), 10 per iteration (4 Dslash, the last of
    # which also reduces <p,Ap>, its finishing kernel, the x/r update and its
    # finishing kernel, the p update, 2 graph-control kernels) and 7 per
    # reliable update after the first (accumulate, 4 FP64 Dslash, residual
    # and its finishing kernel)
    launches = sum(9 + 10 * it + 7 * (ru - 1) for it, ru in zip(iters, rus))

    # plain FP64 CG on the same inputs (the comparison of the metric)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    x64, info64 = solve("f64")
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    mixed_ms = t_ms / args.steps

    # isolated FP16 parity Dslash (dominant kernel): chained applies p -> t -> p
    p16 = cola.pack(g, b, "f16")
    t16 = g.empty_packed("f16")
    for _ in range(5):
        cola.dslash(g, t16, p16, parity=1, prec="f16")
        cola.dslash(g, p16, t16, parity=0, prec="f16")
    nrep = 100
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    d0.record(stream)
    for _ in range(nrep):
        cola.dslash(g, t16, p16, parity=1, prec="f16")
        cola.dslash(g, p16, t16, parity=0, prec="f16")
    d1.record(stream)
    torch.cuda.synchronize()
    ds_us = d0.elapsed_time(d1) * 1e3 / (2 * nrep)
    ds_bytes = BYTES_PER_SITE_F16 * vh
    achieved = ds_bytes / (ds_us * 1e-6) / 1e9
    peak, peak_kind = measured_peak_hbm()

    # isolated FP64 parity Dslash (reliable updates; FP64-ALU bound on this part)
    p64 = cola.pack(g, b, "f64")
    t64 = g.empty_packed("f64")
    cola.dslash(g, t64, p64, parity=1, prec="f64")
    torch.cuda.synchronize()
    d0.record(stream)
    for _ in range(10):
        cola.dslash(g, t64, p64, parity=1, prec="f64")
        cola.dslash(g, p64, t64, parity=0, prec="f64")
    d1.record(stream)
    torch.cuda.synchronize()
    ds64_us = d0.elapsed_time(d1) * 1e3 / 20
    fp64_peak = measure_fp64_peak(cola, dev, stream)
    FP64_PEAK_MEASURED[0] = fp64_peak

    # isolated FP32 parity Dslash (the FP32-storage solver's kernel), own handle
    g32 = cola.Gauge(u, DIMS, KAPPA, BC, precisions=("f32",), recon={"f32": 12})
    p32 = cola.pack(g32, b, "f32")
    t32 = g32.empty_packed("f32")
    for _ in range(3):
        cola.dslash(g32, t32, p32, parity=1, prec="f32")
        cola.dslash(g32, p32, t32, parity=0, prec="f32")
    torch.cuda.synchronize()
    d0.record(stream)
    for _ in range(50):
        cola.dslash(g32, t32, p32, parity=1, prec="f32")
        cola.dslash(g32, p32, t32, parity=0, prec="f32")
    d1.record(stream)
    torch.cuda.synchronize()
    ds32_us = d0.elapsed_time(d1) * 1e3 / 100
    ds32_gbs = BYTES_PER_SITE_F32 * vh / (ds32_us * 1e-6) / 1e9
    del g32, p32, t32

    # the sections beside the headline: a failure is reported in its place, never
    # fatal; they run in single-process runs only (a replica run measures the headline)
    def section(skip, fn, *a):
        if skip or world > 1:
            return None
        try:
            return fn(*a)
        except Exception as e:  # noqa: BLE001
            torch.cuda.synchronize()
            return {"error": f"{type(e).__name__}: {e}"}

    multi = section(args.skip_multi_rhs, multi_rhs_measurements, cola, dev)
    clover = section(args.skip_clover, clover_measurements, cola, dev, u, b)
    hmc = section(args.skip_hmc, hmc_measurements, cola, dev)
    multishift = section(args.skip_multishift, multishift_measurements, cola, dev, u, b)
    eig = section(args.skip_eig, eig_measurements, cola, dev)

    # end to end through the public API with host buffers: every step copies
    # the canonical links and the source from pinned host memory, re-packs the
    # links into the (reused) gauge handle, solves and copies x back.  Copies
    # run on their own stream, double-buffered, so step k+1's inputs and step
    # k-1's result move while step k solves; all of them are inside the timed
    # region.
    u_host = u.cpu().pin_memory()
    b_host = b.cpu().pin_memory()
    e2e_steps = max(2, args.steps)
    x_host = [torch.empty_like(b_host).pin_memory() for _ in range(2)]
    ud = [torch.empty_like(u) for _ in range(2)]
    bd = [torch.empty_like(b) for _ in range(2)]
    copy = torch.cuda.Stream(device=dev)
    main = torch.cuda.current_stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    with torch.cuda.stream(copy):
        ud[0].copy_(u_host, non_blocking=True)
        bd[0].copy_(b_host, non_blocking=True)
        ev_in[0].record(copy)
    e2e_ds = 0
    for k in range(e2e_steps):
        cur, nxt = k % 2, (k + 1) % 2
        if k + 1 < e2e_steps:
            with torch.cuda.stream(copy):
                ud[nxt].copy_(u_host, non_blocking=True)
                bd[nxt].copy_(b_host, non_blocking=True)
                ev_in[nxt].record(copy)
        main.wait_event(ev_in[cur])
        g.update(ud[cur])
        xe, ie = cola.cg_solve(g, bd[cur], tol=TOL, op="eo", inner="f16", delta=DELTA, use_graph=True)
        e2e_ds += 4 * ie[0].iters + 4 * ie[0].reliable_updates
        copy.wait_stream(main)
        with torch.cuda.stream(copy):
            x_host[cur].copy_(xe, non_blocking=True)
        # the caching allocator may reuse x's memory once the copy stream has read it
        xe.record_stream(copy)
        del xe
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - w0) / e2e_steps
    e2e_ms, e2e_flops = aggregate_ranks(e2e_s * 1e3, FLOP_PER_SITE * vh * e2e_ds / e2e_steps, dev)
    e2e_s = e2e_ms * 1e-3
    e2e_value = e2e_flops / e2e_s / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # iterations of the plain FP64 GPU solves, for the oracle study's
        # labelled whole-solve extrapolations
        fp64_iters = {"32x32x32x64": info64[0].iters, "16x16x16x32": config1_fp64_iters(cola, dev)}
        if multi and "point_sources_24x24x24x48" in multi:
            fp64_iters["24x24x24x48-12-point-sources"] = multi["point_sources_24x24x24x48"]["fp64_iters"]
        study = run_cpu_study_from_gpu_arm(fp64_iters, full=args.cpu_full)
        cpu = study if "error" in study else cpu_baseline_from_study(study)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mixed_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16-storage/f32-math/f64-reliable", "data": "synthetic",
            "config": bench_config(world),
            "solve": {"iters": iters[-1], "reliable_updates": rus[-1],
                      "true_rel_resid": infos[-1].true_rel_resid, "mixed_ms": mixed_ms},
            "fp64_cg": {"ms": fp64_ms, "iters": info64[0].iters, "true_rel_resid": info64[0].true_rel_resid,
                        "mixed_over_fp64_time": mixed_ms / fp64_ms},
            "dslash_f16": {"us_per_parity_apply": ds_us, "gflops": FLOP_PER_SITE * vh / (ds_us * 1e-6) / 1e9,
                           "algorithmic_gbs": achieved},
            "dslash_f64": {"us_per_parity_apply": ds64_us, "gflops": FLOP_PER_SITE * vh / (ds64_us * 1e-6) / 1e9},
            "dslash_f32": {"us_per_parity_apply": ds32_us, "gflops": FLOP_PER_SITE * vh / (ds32_us * 1e-6) / 1e9,
                           "algorithmic_gbs": ds32_gbs, "hbm_frac": ds32_gbs / peak},
            # dominant kernel by time share: the FP64 hopping term of the reliable
            # updates (about half of the solve), bound by the FP64 pipe
            "roofline": {"bound": "alu", "achieved": FLOP_PER_SITE * vh / (ds64_us * 1e-6) / 1e12,
                         "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": FLOP_PER_SITE * vh / (ds64_us * 1e-6) / 1e12 / fp64_peak,
                         "traffic": ncu_traffic("f64"), "kernel": "dslash_kernel<F64,18> parity apply",
                         "peak_kind": "measured in this run: independent FP64 FMA chains (cola_probe_fp64_fma), "
                                      "CUDA events, best of 5; 1320 algorithmic flop per site",
                         "peak_derived": FP64_PEAK_DERIVED_TFLOPS,
                         "frac_of_derived": FLOP_PER_SITE * vh / (ds64_us * 1e-6) / 1e12 / FP64_PEAK_DERIVED_TFLOPS},
            # the inner-iteration kernel, bound by HBM
            "roofline_inner": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "traffic": ncu_traffic("f16"),
                               "kernel": "dslash_kernel<F16,12> parity apply",
                               "peak_kind": f"{peak_kind} hbm_gbs (burst, kernel timed alone)"},
            "e2e": {"value": e2e_value, "unit": "GFLOP/s",
                    "h2d_bytes_per_step": u_host.numel() * 16 + b_host.numel() * 16,
                    "d2h_bytes_per_step": x_host[0].numel() * 16, "ms_per_step": e2e_s * 1e3,
                    "overlap": "copies double-buffered on a copy stream, overlapping the previous and next solve"},
            "multi_rhs": multi,
            "clover": clover,
            "hmc": hmc,
            "multishift": multishift,
            "eig": eig,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def multi_rhs_measurements(cola, dev):
    """Multi-RHS and batched solves (not part of the timed step).

    (a) the 12 spin-colour point sources at the origin on 24^3x48, kappa 0.124,
        links exp(0.3 i H), FP32 storage with FP64 reliable updates, solved as
        one 12-RHS graph-captured solve, against plain FP64 CG of one source;
    (b) one batched solve of 8^4, 12^3x24, 16^3x32, 24^3x48 with 4 Gaussian
        sources each, same parameters.
    """
    import torch

    import synth

    kappa = 0.124
    out = {}
    d24 = (24, 24, 24, 48)
    u24 = synth.gauge_field(d24, 0.3, synth.seed_for(3, 0), device=dev, as_numpy=False)
    g24 = cola.Gauge(u24, d24, kappa, BC, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
    pts = torch.from_numpy(synth.point_sources(d24)).to(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    ms12, (x12, i12) = timed(lambda: cola.cg_solve(g24, pts, tol=TOL, op="eo", inner="f32", delta=DELTA,
                                                   use_graph=True))
    ms64, (x64, i64) = timed(lambda: cola.cg_solve(g24, pts[0], tol=TOL, op="eo", inner="f64", use_graph=True))
    # the same 12 sources as 12 single-right-hand-side solves of the same kind
    cola.cg_solve(g24, pts[0], tol=TOL, op="eo", inner="f32", delta=DELTA, use_graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    singles = [cola.cg_solve(g24, pts[k], tol=TOL, op="eo", inner="f32", delta=DELTA, use_graph=True)[1][0]
               for k in range(12)]
    e1.record()
    torch.cuda.synchronize()
    ms1x12 = e0.elapsed_time(e1)
    # the FP32 parity hopping term alone: 12 right-hand sides in one launch against one
    def hop_us(nrhs, reps=20):
        pin = cola.pack(g24, pts[:nrhs] if nrhs > 1 else pts[0], "f32")
        pout = g24.empty_packed("f32", nrhs)
        cola.dslash(g24, pout, pin, parity=1, prec="f32", nrhs=nrhs)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record()
        for _ in range(reps):
            cola.dslash(g24, pout, pin, parity=1, prec="f32", nrhs=nrhs)
        h1.record()
        torch.cuda.synchronize()
        return h0.elapsed_time(h1) * 1e3 / reps
    us1, us12 = hop_us(1), hop_us(12)
    vh24 = 24 ** 3 * 48 // 2
    out["point_sources_24x24x24x48"] = {
        "nrhs": 12, "mixed_f32_ms": ms12, "mixed_ms_per_rhs": ms12 / 12,
        "max_iters": max(i.iters for i in i12), "max_true_rel_resid": max(i.true_rel_resid for i in i12),
        "single_rhs_f32_solves_ms": ms1x12, "single_rhs_f32_ms_per_rhs": ms1x12 / 12,
        "single_rhs_max_true_rel_resid": max(i.true_rel_resid for i in singles),
        "per_rhs_ratio_vs_single_rhs_f32": ms12 / ms1x12,
        "fp64_single_rhs_ms": ms64, "fp64_iters": i64[0].iters,
        "per_rhs_ratio_vs_fp64": (ms12 / 12) / ms64,
        "dslash_f32_us_1rhs": us1, "dslash_f32_us_per_rhs_12rhs": us12 / 12,
        # algorithmic bytes per output site and right-hand side: spinor in and out
        # (2 x 96 B) plus the 8 links (8 x 48 B) shared by the right-hand sides of a launch
        "dslash_f32_12rhs_algorithmic_gbs": (12 * 192 + 384) * vh24 / (us12 * 1e-6) / 1e9}
    dims_list = [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), d24]
    gauges, bs = [], []
    for k, d in enumerate(dims_list):
        u = u24 if d == d24 else synth.gauge_field(d, 0.3, synth.seed_for(3, 4 + k), device=dev, as_numpy=False)
        gauges.append(g24 if d == d24 else cola.Gauge(u, d, kappa, BC, precisions=("f64", "f32"),
                                                      recon={"f64": 18, "f32": 12}))
        bs.append(torch.from_numpy(synth.gaussian_spinor(d, synth.seed_for(3, 8 + k), nrhs=4)).to(dev))
    msb, (xb, ib) = timed(lambda: cola.cg_solve_batched(gauges, bs, tol=TOL, op="eo", inner="f32", delta=DELTA,
                                                         use_graph=True))
    # (c) the HMC force: phi = D^dag eta on 24^3x48 (links exp(0.3 i H), kappa 0.124),
    #     X = (D^dag D)^-1 phi by FP32-inner CG on the whole lattice, Y = D X, force
    u4 = synth.gauge_field(d24, 0.3, synth.seed_for(4, 0), device=dev, as_numpy=False)
    g4 = cola.Gauge(u4, d24, kappa, BC, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
    eta = torch.from_numpy(synth.gaussian_spinor(d24, synth.seed_for(4, 1))).to(dev)
    phi = cola.apply_dirac(g4, eta, dagger=True)
    msx, (X, ix) = timed(lambda: cola.cg_solve(g4, phi, tol=TOL, op="full", inner="f32", delta=DELTA,
                                               use_graph=True))
    Y = cola.apply_dirac(g4, X)
    msf, F = timed(lambda: cola.fermion_force(g4, X, Y))
    out["force_24x24x24x48"] = {"solve_ms": msx, "iters": ix[0].iters, "true_rel_resid": ix[0].true_rel_resid,
                                "force_kernel_ms": msf, "links": 4 * 24 ** 3 * 48}
    del g4, u4
    out["batched_4_lattices_x4"] = {
        "lattices": ["8^4", "12^3x24", "16^3x32", "24^3x48"], "nrhs": 4, "ms": msb,
        "max_iters": max(i.iters for row in ib for i in row),
        "max_true_rel_resid": max(i.true_rel_resid for row in ib for i in row)}
    return out


CSW = 1.0
# algorithmic bytes per even site of one FP16 even-odd normal-operator apply
# (4 parity launches): hopping reads and writes as above, the xpay input of the
# two even-parity launches, and one 6x6-block pair of A or A^-1 (72 halves =
# 144 B) per output site in each launch with a clover term
BYTES_MDAGM_F16_WILSON = 2 * BYTES_PER_SITE_F16 + 2 * (BYTES_PER_SITE_F16 + 52)
BYTES_MDAGM_F16_CLOVER = BYTES_MDAGM_F16_WILSON + 4 * 144


def clover_measurements(cola, dev, u, b):
    """Clover-improved operator on the benchmark's lattice (not part of the timed step).

    c_sw = 1 on the same links and source: the construction of A and A^-1
    (FP64, once per gauge field), the FP16 even-odd normal operator
    Mhat^dag Mhat (4 hopping launches with clover epilogues) next to the
    Wilson one, and the mixed FP16 solve of the same normal system next to
    plain FP64 CG.  The operator is applied repeatedly to one input (its 55 MB
    FP16 spinor may stay in L2; links and clover fields, 503 MB, do not).
    """
    import torch

    vh = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2
    g = cola.Gauge(u, DIMS, KAPPA, BC, precisions=("f64", "f16"), recon={"f64": 18, "f16": 12})
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.attach_clover(CSW)
    build_ms = (time.perf_counter() - t0) * 1e3

    def op_us(gg, reps=50):
        p16 = cola.pack(gg, b, "f16")
        q16 = gg.empty_packed("f16")
        for _ in range(3):
            cola.mdagm(gg, q16, p16, op="eo", prec="f16")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            cola.mdagm(gg, q16, p16, op="eo", prec="f16")
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    us_clover = op_us(g)
    gw = cola.Gauge(u, DIMS, KAPPA, BC, precisions=("f16",), recon={"f16": 12})
    us_wilson = op_us(gw)
    del gw

    def solve(inner):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, info = cola.cg_solve(g, b, tol=TOL, op="eo", inner=inner, delta=DELTA, use_graph=True)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), info[0]

    solve("f16")
    ms16, i16 = solve("f16")
    ms64, i64 = solve("f64")
    peak, _ = measured_peak_hbm()
    gbs = BYTES_MDAGM_F16_CLOVER * vh / (us_clover * 1e-6) / 1e9
    return {
        "csw": CSW, "construction_ms": build_ms,
        "mdagm_eo_f16": {"us_clover": us_clover, "us_wilson": us_wilson, "clover_over_wilson": us_clover / us_wilson,
                         "algorithmic_gbs": gbs, "hbm_frac": gbs / peak,
                         "bytes_per_even_site": BYTES_MDAGM_F16_CLOVER},
        "mixed_f16_solve": {"ms": ms16, "iters": i16.iters, "reliable_updates": i16.reliable_updates,
                            "true_rel_resid": i16.true_rel_resid},
        "fp64_cg": {"ms": ms64, "iters": i64.iters, "true_rel_resid": i64.true_rel_resid,
                    "mixed_over_fp64_time": ms16 / ms64},
    }


# FP64 flop per link of the Wilson gauge force: 6 staples of 2 SU(3) products
# each, the product U V, and the staple sums (3x3 complex product = 27 complex
# multiply-adds = 216 flop)
GAUGE_FORCE_FLOP_PER_LINK = 13 * 216 + 5 * 18
# clover force per link (18-real FP64 links): for each of the three planes
# through it, two plaquettes of 8 products of 3x3 complex matrices each in
# nested form, 4 of them with the Hermitian insertion matrix (real diagonal:
# 180 instead of 216 flop), then U S+ and S- U^dag
CLOVER_FORCE_FLOP_PER_LINK = 3 * 2 * (4 * 216 + 4 * 180) + 2 * 216


def hmc_measurements(cola, dev):
    """One HMC trajectory on 24^3x48 (not part of the timed step).

    kappa 0.124, beta 5.6, links exp(0.3 i H), Gaussian momenta and
    pseudofermion source, tau = 0.5 in 5 Omelyan steps (11 force
    evaluations), force solves with FP64 reliable updates to 1e-8, final
    action to 1e-12.  The same trajectory with the force solves as CG on
    D^dag D or as two even-odd Dirac-system solves (the same X), each with
    FP32 or FP16 inner iterations, after one warm-up trajectory of each; the
    fastest is reported in front.  Also the isolated gauge-force and
    link-update kernels, the fermion force with and without the clover term,
    and the trajectory with the clover term (c_sw = 1).
    """
    import torch

    import synth

    d24 = (24, 24, 24, 48)
    vol = 24 ** 3 * 48
    u = synth.gauge_field(d24, 0.3, synth.seed_for(5, 0), device=dev, as_numpy=False)
    mom = torch.from_numpy(synth.su3_direction(d24, synth.seed_for(5, 1))).to(dev)
    eta = torch.from_numpy(synth.gaussian_spinor(d24, synth.seed_for(5, 2))).to(dev)
    g = cola.Gauge(u, d24, 0.124, BC, precisions=("f64", "f32", "f16"), recon={"f64": 18, "f32": 12, "f16": 12})
    torch.cuda.synchronize()
    u0, mom0 = u.clone(), mom.clone()

    def trajectory(md_op, md_inner):
        u.copy_(u0)
        mom.copy_(mom0)
        g.update(u)
        return cola.hmc_trajectory(g, u, mom, eta, 5.6, 0.5, 5, "omelyan", uniform=0.0, md_tol=1e-8,
                                   md_inner=md_inner, action_tol=1e-12, md_op=md_op)

    # force solves: CG on D^dag D, or two even-odd Dirac-system solves; FP32 or FP16 inner iterations
    keys = [(op, inner) for op in ("full", "eo") for inner in ("f32", "f16")]
    for k in keys:  # warm-up: launch-shape tuning and solve-graph capture per configuration
        trajectory(*k)
    variants = {k: trajectory(*k) for k in keys}
    best = min(variants, key=lambda k: variants[k].seconds)
    info = variants[best]

    def kernel_us(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    gf_us = kernel_us(lambda: cola.gauge_force(g, 5.6))
    zero = torch.zeros_like(mom)
    lu_us = kernel_us(lambda: cola.link_update(g, u, zero, 0.0))
    gf_tflops = GAUGE_FORCE_FLOP_PER_LINK * 4 * vol / (gf_us * 1e-6) / 1e12
    # the fermion force without and with the clover term (c_sw = 1), and the
    # trajectory with the clover term in the fastest solve configuration
    ff_us = kernel_us(lambda: cola.fermion_force(g, eta, eta))
    g.attach_clover(1.0)
    ffc_us = kernel_us(lambda: cola.fermion_force(g, eta, eta))
    trajectory(*best)  # warm-up of the clover kernels' launch shapes
    info_c = trajectory(*best)
    g.attach_clover(0.0)
    cf_us = ffc_us - ff_us
    cf_tflops = CLOVER_FORCE_FLOP_PER_LINK * 4 * vol / (cf_us * 1e-6) / 1e12
    return {
        "lattice": "24x24x24x48", "beta": 5.6, "kappa": 0.124, "tau": 0.5, "steps": 5, "integrator": "omelyan",
        "md_solves": f"{best[0]} ({'CG on D^dag D' if best[0] == 'full' else 'D W = g5 phi, D X = g5 W'}), "
                     f"{best[1]} inner iterations, FP64 reliable updates, 1e-8",
        "trajectory_s": info.seconds, "force_evals": info.force_evals, "cg_iters": info.cg_iters, "dH": info.dH,
        "accepted": info.accepted, "plaquette": info.plaquette,
        "variants_s": {f"{k[0]}/{k[1]}": v.seconds for k, v in variants.items()},
        "gauge_force_us": gf_us, "gauge_force_fp64_tflops": gf_tflops, "gauge_force_frac_fp64": gf_tflops / FP64_PEAK_MEASURED[0],
        "link_update_and_repack_us": lu_us,
        "fermion_force_us": ff_us, "clover_force_us": cf_us, "clover_force_fp64_tflops": cf_tflops,
        "clover_force_frac_fp64": cf_tflops / FP64_PEAK_MEASURED[0],
        "clover_trajectory": {"csw": 1.0, "trajectory_s": info_c.seconds, "cg_iters": info_c.cg_iters,
                              "dH": info_c.dH, "accepted": info_c.accepted},
    }


def multishift_measurements(cola, dev, u, b):
    """Multi-shift CG on the benchmark's lattice (not part of the timed step).

    Ten shifts sigma_i = 1e-4 x 10^(0.6 i) (1e-4 .. 25, the spread of a
    rational approximation's poles) on Mhat^dag Mhat of the 32^3x64 workload,
    to 1e-10 per shift: FP32 phase 1 (to 1e-7) plus the FP16-inner refinement
    with FP64 reliable updates at delta = 0.01, against the same ten systems
    solved one at a time by the same mixed solver, and against the plain FP64
    multi-shift recurrence.
    """
    import torch

    shifts = [1e-4 * 10 ** (0.6 * i) for i in range(10)]
    g = cola.Gauge(u, DIMS, KAPPA, BC, precisions=("f64", "f32", "f16"), recon={"f64": 18, "f32": 12, "f16": 12})

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    # warm-up of every variant timed below: launch-shape tuning and solve-graph capture per shape
    mixed = dict(tol=TOL, op="eo", inner="f16", delta=0.01, use_graph=True)
    cola.multishift_solve(g, b, shifts, **mixed)
    cola.multishift_solve(g, b, shifts, tol=TOL, op="eo", inner="f64")
    cola.multishift_solve(g, b, shifts[:1], **mixed)
    ms16, (x16, i16) = timed(lambda: cola.multishift_solve(g, b, shifts, **mixed))
    ms64, (x64, i64) = timed(lambda: cola.multishift_solve(g, b, shifts, tol=TOL, op="eo", inner="f64"))
    sep = 0.0
    for sg in shifts:
        t, _ = timed(lambda sg=sg: cola.multishift_solve(g, b, [sg], **mixed))
        sep += t
    return {
        "lattice": "32x32x32x64", "nshift": len(shifts), "shifts": [shifts[0], shifts[-1]], "tol": TOL,
        "delta": 0.01, "phase1": "fp32 to 1e-7", "refinement": "fp16 inner, fp64 reliable updates",
        "mixed_f16_ms": ms16, "max_true_rel_resid": max(i.true_rel_resid for i in i16),
        "iters_smallest_shift": i16[0].iters, "iters_largest_shift": i16[-1].iters,
        "fp64_ms": ms64, "separate_mixed_solves_ms": sep, "multishift_over_separate": ms16 / sep,
    }


def eig_measurements(cola, dev):
    """Lowest eigenmodes on the 16^3x32 workload (not part of the timed step).

    kappa 0.125, links exp(0.3 i H), Gaussian starting vectors: the twelve
    lowest eigenpairs of Mhat^dag Mhat (four guard vectors) to a relative
    residual of 1e-8 by the Kalkreuter-Simma accelerated CG in FP64.
    """
    import torch

    import synth

    d16 = (16, 16, 16, 32)
    u = synth.gauge_field(d16, 0.3, synth.seed_for(1, 0), device=dev, as_numpy=False)
    v0 = torch.from_numpy(synth.gaussian_spinor(d16, synth.seed_for(1, 5), nrhs=16)).to(dev)
    g = cola.Gauge(u, d16, 0.125, BC, precisions=("f64",), recon={"f64": 18})
    cola.eig_lowest(g, v0[:2], op="eo", tol=1e-6, max_sweeps=2, raise_on_error=False)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vals, _, info = cola.eig_lowest(g, v0, nev=12, op="eo", tol=1e-8)
    secs = time.perf_counter() - t0
    # FP64 normal operator applications dominate: 4 parity hops each
    return {"lattice": "16x16x16x32", "nev": 12, "nextra": 4, "tol": 1e-8, "seconds": secs, "sweeps": info.sweeps,
            "operator_applications": info.applications, "max_rel_resid": info.max_rel_resid,
            "lambda_min": float(vals[0]), "lambda_12": float(vals[-1]),
            "ms_per_application": secs * 1e3 / info.applications}


def run_dslash_only(args):
    """Chained parity Dslash applies only (the case profiled with ncu): the
    32^3x64 workload, or with --clover the clover normal operator on
    --lattice, or with --nrhs > 1 that many point sources of 24^3x48 in one
    multi-right-hand-side launch."""
    import torch

    import paper_2302_00850_gb300 as cola

    torch.cuda.set_device(0)
    dims = DIMS
    if args.clover:
        import synth

        # a smaller lattice keeps the FP64 links and clover fields of the
        # profiled process to about 1.5 GB (still well above L2)
        dims = tuple(int(v) for v in args.lattice.split("x"))
        dev = torch.device("cuda", 0)
        u = synth.gauge_field(dims, EPS, synth.seed_for(CONFIG_ID, 0), device=dev, as_numpy=False)
        b = torch.from_numpy(synth.gaussian_spinor(dims, synth.seed_for(CONFIG_ID, 1))).to(dev)
    elif args.nrhs > 1:
        import synth

        # the 12 point sources of the multi-RHS workload (24^3x48, kappa 0.124, links exp(0.3 i H))
        dims = (24, 24, 24, 48)
        dev = torch.device("cuda", 0)
        u = synth.gauge_field(dims, 0.3, synth.seed_for(3, 0), device=dev, as_numpy=False)
        b = torch.from_numpy(synth.point_sources(dims)[:args.nrhs]).to(dev)
    else:
        u, b = make_inputs(torch.device("cuda", 0))
    prec = args.prec
    if args.clover:
        # the even-odd normal operator with clover epilogues (4 launches per apply)
        g = cola.Gauge(u, dims, KAPPA, BC, precisions=("f64", prec), recon={"f64": 18, prec: args.recon})
        g.attach_clover(CSW)
    else:
        g = cola.Gauge(u, dims, KAPPA, BC, precisions=(prec,), recon={prec: args.recon})
    del u
    nrhs = max(args.nrhs, 1)
    p = cola.pack(g, b, prec)
    t = g.empty_packed(prec, nrhs)
    for _ in range(args.reps):
        if args.clover:
            cola.mdagm(g, t, p, op="eo", prec=prec)
        else:
            cola.dslash(g, t, p, parity=1, prec=prec, nrhs=nrhs)
            cola.dslash(g, p, t, parity=0, prec=prec, nrhs=nrhs)
    torch.cuda.synchronize()
    print(json.dumps({"dslash_only": prec, "recon": args.recon, "reps": args.reps, "clover": bool(args.clover),
                      "nrhs": nrhs, "lattice": "x".join(map(str, dims))}))


def run_gauge_only(args):
    """Gauge force and link update kernels only on --lattice (the case profiled with ncu);
    with --clover also the fermion force of a handle with a clover term (c_sw = 1)."""
    import torch

    import paper_2302_00850_gb300 as cola
    import synth

    torch.cuda.set_device(0)
    dims = tuple(int(v) for v in args.lattice.split("x"))
    dev = torch.device("cuda", 0)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(5, 0), device=dev, as_numpy=False)
    mom = torch.from_numpy(synth.su3_direction(dims, synth.seed_for(5, 1))).to(dev)
    g = cola.Gauge(u, dims, 0.124, BC, precisions=("f64",), recon={"f64": 18})
    for _ in range(args.reps):
        cola.gauge_force(g, 5.6)
        cola.link_update(g, u, mom, 0.01)
    if args.clover:
        x = torch.from_numpy(synth.gaussian_spinor(dims, synth.seed_for(5, 2))).to(dev)
        y = torch.from_numpy(synth.gaussian_spinor(dims, synth.seed_for(5, 3))).to(dev)
        g.attach_clover(1.0)
        for _ in range(args.reps):
            cola.fermion_force(g, x, y)
    torch.cuda.synchronize()
    print(json.dumps({"gauge_only": args.lattice, "reps": args.reps, "clover_force": bool(args.clover)}))


def run_solve_only(args):
    """One mixed-precision even-odd solve on a smaller lattice (the case profiled with ncu)."""
    import torch

    import paper_2302_00850_gb300 as cola
    import synth

    torch.cuda.set_device(0)
    dims = tuple(int(v) for v in args.lattice.split("x"))
    dev = torch.device("cuda", 0)
    u = synth.gauge_field(dims, EPS, synth.seed_for(CONFIG_ID, 0), device=dev, as_numpy=False)
    b = torch.from_numpy(synth.gaussian_spinor(dims, synth.seed_for(CONFIG_ID, 1))).to(dev)
    g = cola.Gauge(u, dims, KAPPA, BC, precisions=("f64", args.prec), recon={"f64": 18, args.prec: 12})
    del u
    for _ in range(args.reps):
        x, info = cola.cg_solve(g, b, tol=TOL, op="eo", inner=args.prec, delta=DELTA, use_graph=False)
    torch.cuda.synchronize()
    print(json.dumps({"solve_only": args.lattice, "prec": args.prec, "iters": info[0].iters,
                      "true_rel_resid": info[0].true_rel_resid}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--solve-only", action="store_true", help="run host-loop solves on --lattice and exit")
    ap.add_argument("--lattice", default="24x24x24x48")
    ap.add_argument("--dslash-only", action="store_true", help="run chained parity Dslash applies and exit")
    ap.add_argument("--gauge-only", action="store_true", help="run gauge-force and link-update kernels and exit")
    ap.add_argument("--prec", default="f16")
    ap.add_argument("--clover", action="store_true",
                    help="with --dslash-only: the clover normal operator; with --gauge-only: also the clover force")
    ap.add_argument("--recon", type=int, default=12)
    ap.add_argument("--nrhs", type=int, default=1,
                    help="with --dslash-only: that many of the 12 point sources of 24^3x48 per launch")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cola", choices=["cola", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="the oracle study also runs the whole 16^3x32 oracle solve (minutes on one core)")
    ap.add_argument("--cpu-study", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-study-only", action="store_true",
                    help="run only the oracle study on the host cores (inputs drawn on the GPU) and print it")
    ap.add_argument("--skip-multi-rhs", action="store_true", help="skip the multi-RHS and batched solves")
    ap.add_argument("--skip-clover", action="store_true", help="skip the clover-operator measurements")
    ap.add_argument("--skip-hmc", action="store_true", help="skip the HMC trajectory measurement")
    ap.add_argument("--skip-multishift", action="store_true", help="skip the multi-shift CG measurement")
    ap.add_argument("--skip-eig", action="store_true", help="skip the eigensolver measurement")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the CG loop from the host instead of one conditional CUDA graph (ncu cannot "
                         "profile kernels inside graphs with conditional nodes)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.cpu_study:
        run_cpu_study_child(args)
    elif args.cpu_study_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps(run_cpu_study_from_gpu_arm({}, full=args.cpu_full)), flush=True)
    elif args.dslash_only:
        run_dslash_only(args)
    elif args.gauge_only:
        run_gauge_only(args)
    elif args.solve_only:
        run_solve_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_cola(args)


if __name__ == "__main__":
    main()
