#!/usr/bin/env python
"""Benchmark of the diagonal-budgeted Trotterization hot path on GB300.

One bench step = the whole hot path over one synthetic instance: factor
build from the Pauli terms (host planning + FP64 GPU build), the n_steps x G
factor applications of the evolution, and the FP64 overlap/norm reduction.

Metric: amplitude-updates/s = sum over the step of n_steps * G * N * R (one
update = one output amplitude of one factor application to one state).
The default workload is the largest single-GPU configuration: weighted MaxCut
on 24 qubits with the transverse mixer, 16 states, 50 steps, complex64 (the
complex128 run of the same workload is reported beside it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload maxcut24|heis16|batch256|...]
                  [--impl ours|reference] [--no-cpu-baseline] [--no-c128]

Under torchrun (N > 1) every rank evolves its own replica of the instance
(the path has no exchange step: replicas only) and rank 0 prints one JSON line
with value = updates of all ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "amplitude-updates/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="maxcut24",
                    choices=["heis16", "maxcut24", "tfim10", "batch256", "serve", "taylor16", "anneal24"])
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-rate", type=float, default=500.0)
    ap.add_argument("--serve-find-rate", action="store_true",
                    help="serve: search the highest Poisson rate whose queue stays bounded over 20 s and report "
                         "p50/p99 there, at half of it and at --serve-rate")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--e2e-chunks", type=int, default=0,
                    help="end-to-end step: chunks of states pipelined with the copies (0: library default of the bench)")
    ap.add_argument("--batch-jobs", type=int, default=256)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c128", action="store_true")
    ap.add_argument("--method", type=int, default=0)
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--rhs-block", type=int, default=0)
    ap.add_argument("--graph", type=int, default=0)
    ap.add_argument("--order", type=int, default=1, choices=[1, 2, 4],
                    help="product formula: 1 (first order), 2 (Strang), 4 (Suzuki)")
    ap.add_argument("--qubits", type=int, default=0,
                    help="maxcut24 only: a smaller instance of the same family (profiling cases)")
    return ap.parse_args()


def make_job(name, dtype=None, qubits=0):
    from paper_2606_16959_gb300 import workloads as W
    if name == "maxcut24" and qubits:
        job = W.maxcut24(n=qubits)
        desc = (f"weighted MaxCut random 3-regular n={qubits} (seed 1003) + 0.5 sum X, 16 states (|+> and Gaussians), "
                "t=2, 50 steps, budget 4")
    elif name == "heis16":
        job = W.heis16(dtype or "c64")
        desc = "Heisenberg XXX periodic chain n=16, J_i~U[0.5,1.5] (seed 1002), Gaussian state, t=1, 100 steps, budget 8"
    elif name == "anneal24":
        job = W.anneal24()
        desc = ("MaxCut annealing H(s) = (1-s) 0.5 sum X + s H_C on the n=24 weighted random 3-regular graph "
                "(seed 1003), linear ramp s = t/T at step midpoints, T=2, 50 steps, 16 states (|+> and Gaussians), "
                "budget 4; factors of the driven terms rebuilt on the GPU every step")
    elif name == "maxcut24":
        job = W.maxcut24()
        desc = ("weighted MaxCut random 3-regular n=24 (seed 1003) + 0.5 sum X, 16 states (|+> and Gaussians), "
                "t=2, 50 steps, budget 4")
    else:
        job = W.tfim10()
        desc = "TFIM open chain n=10, J=h=1, |0..0>, t=1, 10 steps, budget 4"
    if dtype:
        job.dtype = dtype
    return job, desc


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


TUNE_CACHE = os.path.join(ROOT, "paper_2606_16959_gb300", "_build", "autotune_bench.json")
# Committed ncu summaries are named <kernel>_<workload>.md (profiles/).
# Device-code sources of each kernel: a summary's DRAM figures count only while
# these are unchanged since the capture.
KERNEL_SOURCES = {"sweep_kernel": ("apply.cu", "sweep_core.cuh", "hs_internal.h"),
                  "qsweep_kernel": ("qsweep.cu", "qsweep.h", "qplan.cpp", "sweep_core.cuh", "bounds.cuh", "hs_internal.h"),
                  "batch_level_kernel": ("batch.cu", "sweep_core.cuh", "hs_internal.h"),
                  "qlevel_kernel": ("qsweep.cu", "qsweep.h", "qplan.cpp", "batch.cu", "sweep_core.cuh", "bounds.cuh", "hs_internal.h"),
                  "spmv_kernel": ("dia.cu",)}


def sweep_kernel_name(opts, n_sweeps):
    """The kernel an evolution's fused launches run under these options."""
    if not n_sweeps:
        return "apply_plain_kernel"
    return "qsweep_kernel" if opts.get("method") == 3 else "sweep_kernel"


def kernel_source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2606_16959_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, kernel):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None if there is none or the kernel's sources changed since."""
    if kernel not in KERNEL_SOURCES:
        return None
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.strip().startswith(("kernel_source_sha256", "dram_bytes_per_launch")):
                k, v = line.strip().strip("`").split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != kernel_source_hash(kernel):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def dram_fields(traffic, launch_s, peak):
    """DRAM bytes actually moved per launch (ncu) over the live launch time: the
    roofline figure that a fused sweep, which keeps the state on chip across
    several factors, cannot beat by construction."""
    if traffic is None:
        return {}
    a = traffic / launch_s / 1e9
    return {"dram_achieved": a, "dram_frac": a / peak}


def load_tune_cache():
    """Autotuner choices of earlier runs on this machine (so that a run under a
    profiler replays the configuration measured without it)."""
    try:
        with open(TUNE_CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_tune_cache(cache):
    os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
    with open(TUNE_CACHE, "w") as fh:
        json.dump(cache, fh)


def algorithmic_bytes(f, job, n_rhs):
    """Per factor application: s * S_g (factor read once for all states) + 2 s N R
    (state read and write); summed over the n_steps x G applications."""
    s = 8 if f.dtype == "c64" else 16
    N = 1 << f.n_qubits
    per_step = 0
    for g in f.sequence:
        _, _, offs, _ = f.factor(g, values=False)
        S = int(np.sum(N - np.abs(offs)))
        per_step += s * S + 2 * s * N * n_rhs
    return per_step * job.n_steps


def build_job(hs, job, dtype, order):
    """The job's factor set: static, or time-dependent when the job has a drive."""
    if job.drive is not None:
        x, z, n = hs.hs_parse_terms(job.ham.labels)
        return hs.hs_build_factors_td(x, z, job.ham.a, job.ham.b, n, job.t, job.n_steps, job.budget, dtype,
                                      order=order)
    return hs.hs_build_factors(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.budget, dtype, order=order)


def evolve_job(hs, f, psi, job, **opts):
    if job.drive is not None:
        hs.hs_evolve_td(f, psi, job.drive, **opts)
    else:
        hs.hs_evolve_ex(f, psi, job.n_steps, **opts)


def time_ours(job, args, world, dtype, rank):
    """Device-timed steps with inputs resident in HBM.  Returns dict."""
    import torch
    from paper_2606_16959_gb300 import hs
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    psi0 = torch.from_numpy(np.ascontiguousarray(job.psi0)).to(dev, tdt)
    if psi0.dim() == 1:
        psi0 = psi0.unsqueeze(0)
    R, N = psi0.shape
    work = torch.empty_like(psi0)
    out4 = torch.zeros(4, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    opts = dict(method=args.method, tile_bits=args.tile_bits, rhs_block=args.rhs_block, use_graph=bool(args.graph))
    E = torch.cuda.Event

    def step(keep):
        work.copy_(psi0)
        f = build_job(hs, job, dtype, args.order)
        e0, e1 = E(enable_timing=True), E(enable_timing=True)
        e0.record()
        evolve_job(hs, f, work, job, **opts)
        e1.record()
        hs.hs_inner_device(psi0[0], work[0], out4)
        keep.append(f)
        return e0, e1

    tuned = None
    if args.autotune and not any((args.method, args.tile_bits, args.rhs_block)):
        key = f"{args.workload}:{job.ham.n_qubits}:o{args.order}:{dtype}:{torch.cuda.get_device_name()}"
        cache = load_tune_cache()
        if key in cache:
            tuned = cache[key]
        else:
            ft = build_job(hs, job, dtype, args.order)
            tuned = hs.hs_autotune(ft, psi0, min(job.n_steps, 10))
            ft.close()
            cache[key] = tuned
            save_tune_cache(cache)
        opts = dict(method=tuned["method"], tile_bits=tuned["tile_bits"], rhs_block=tuned["rhs_block"],
                    low_bits=tuned["low_bits"], max_fuse=tuned.get("max_fuse", 0), smem_kb=tuned.get("smem_kb", 0),
                    reg_bits=tuned.get("reg_bits", 0), use_graph=bool(args.graph))
    args.tuned_opts = opts
    keep = []
    for _ in range(args.warmup):
        step(keep)
    torch.cuda.synchronize()
    f0 = keep[0]
    if job.drive is not None:
        n_sweeps, n_plain, tb, rb = hs.hs_evolve_td_plan(f0, R, job.n_steps, **opts)
    else:
        n_sweeps, n_plain, tb, rb = hs.hs_evolve_plan(f0, R, job.n_steps, **opts)
    alg = algorithmic_bytes(f0, job, R)
    for f in keep:
        f.close()
    keep = []
    step_ms, evolve_ms = [], []
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    l0 = hs.hs_kernel_launches()
    for _ in range(args.steps):
        flush.zero_()
        s0, s1 = E(enable_timing=True), E(enable_timing=True)
        s0.record()
        e0, e1 = step(keep)
        s1.record()
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        evolve_ms.append(e0.elapsed_time(e1))
        keep[-1].close()
    launches = hs.hs_kernel_launches() - l0
    clocks = sampler.stop() if sampler else None
    barrier(world)
    fid = out4.cpu().numpy()
    G = len(f0.sequence)  # factor applications per step (n_factors for the first-order formula)
    units = job.n_steps * G * N * R
    total_ms = max_over_ranks(sum(step_ms), world)
    return dict(units=units, G=G, R=R, N=N, step_ms=step_ms, evolve_ms=evolve_ms, total_ms=total_ms,
                n_sweeps=n_sweeps, n_plain=n_plain, tile_bits=tb, rhs_block=rb, alg_bytes=alg,
                launches=launches, clocks=clocks, overlap=fid, tuned=tuned)


def time_e2e(job, args, dtype):
    """Same metric through the public API with pinned host buffers: H2D of the
    initial states, build, evolve, norm reduction, D2H of the final states."""
    import torch
    from paper_2606_16959_gb300 import hs
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    host_in = torch.from_numpy(np.ascontiguousarray(job.psi0)).to(tdt)
    if host_in.dim() == 1:
        host_in = host_in.unsqueeze(0)
    host_in = host_in.pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    work = torch.empty(host_in.shape, dtype=tdt, device=dev)
    out4 = torch.zeros(4, dtype=torch.float64, device=dev)
    out4_h = torch.zeros(4, dtype=torch.float64).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    opts = getattr(args, "tuned_opts", None) or dict(method=args.method, tile_bits=args.tile_bits,
                                                     rhs_block=args.rhs_block, use_graph=bool(args.graph))

    # States are independent: with several states the step runs in chunks of
    # states, each chunk's upload overlapping the previous chunk's evolution
    # and each download the next one's (a copy stream beside the compute
    # stream); one state runs as one piece.  Fewer, larger chunks keep the
    # sweeps' grids full.
    R = host_in.shape[0]
    n_chunks = args.e2e_chunks or 2  # (measured on maxcut24: 2 chunks 2.11e12, 4: 2.09e12, 8: 1.75e12)
    if R % n_chunks or R < 2 * n_chunks:
        n_chunks = 1
    cs = R // n_chunks
    main = torch.cuda.current_stream()
    copy_s = torch.cuda.Stream()

    def step():
        if n_chunks == 1:
            work.copy_(host_in, non_blocking=True)
            f = build_job(hs, job, dtype, args.order)
            evolve_job(hs, f, work, job, **opts)
            hs.hs_inner_device(work[0], work[0], out4)
            host_out.copy_(work, non_blocking=True)
            out4_h.copy_(out4, non_blocking=True)
            return f
        copy_s.wait_stream(main)
        ins, outs = [], []
        with torch.cuda.stream(copy_s):
            for c in range(n_chunks):
                work[c * cs:(c + 1) * cs].copy_(host_in[c * cs:(c + 1) * cs], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_s)
                ins.append(ev)
        f = build_job(hs, job, dtype, args.order)
        for c in range(n_chunks):
            main.wait_event(ins[c])
            evolve_job(hs, f, work[c * cs:(c + 1) * cs], job, **opts)
            ev = torch.cuda.Event()
            ev.record(main)
            outs.append(ev)
        hs.hs_inner_device(work[0], work[0], out4)
        with torch.cuda.stream(copy_s):
            for c in range(n_chunks):
                copy_s.wait_event(outs[c])
                host_out[c * cs:(c + 1) * cs].copy_(work[c * cs:(c + 1) * cs], non_blocking=True)
        main.wait_stream(copy_s)
        out4_h.copy_(out4, non_blocking=True)
        return f

    fs = [step() for _ in range(max(1, args.warmup))]
    torch.cuda.synchronize()
    for f in fs:
        f.close()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        f = step()
        s1.record()
        torch.cuda.synchronize()
        times.append(s0.elapsed_time(s1))
        f.close()
    m = len(job.ham.labels)
    term_bytes = 28 * m + 256  # masks, coefficients and group tables uploaded by the build
    if job.drive is not None:
        term_bytes += 8 * m + 8 * len(job.drive)  # H1 coefficients and drive samples
    return dict(ms=statistics.mean(times), h2d=int(host_in.numel() * host_in.element_size()) + term_bytes,
                d2h=int(host_out.numel() * host_out.element_size()) + 32)


def batch_jobs(args, dtype="c64"):
    from paper_2606_16959_gb300 import workloads as W
    jobs = W.batch256(n_jobs=args.batch_jobs, dtype=dtype)
    desc = (f"{len(jobs)} instances: TFIM open / Heisenberg periodic chains 50/50, n~U{{12..20}}, J~U[0.5,1.5], "
            "h~U[0,2], steps~U{20..200}, budget~U{4..16}, Gaussian states, t=1 (seed 1004)")
    return jobs, desc


_BUILD_POOL = None


_BUILD_STREAMS = {}


def build_all(jobs, dtype):
    """Factor sets of independent jobs, built from host threads, each thread on
    a stream of its own (the jobs' host planning runs in parallel and their
    small build kernels overlap on the device); the current stream then waits
    for every build stream."""
    global _BUILD_POOL
    import threading
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2606_16959_gb300 import hs
    if _BUILD_POOL is None:
        _BUILD_POOL = ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)))
    main = torch.cuda.current_stream()

    def one(j):
        tid = threading.get_ident()
        st = _BUILD_STREAMS.get(tid)
        if st is None:
            st = _BUILD_STREAMS[tid] = torch.cuda.Stream()
        st.wait_stream(main)  # inputs and freed memory of earlier work on the main stream
        with torch.cuda.stream(st):
            f = hs.hs_build_factors(j.ham.labels, j.ham.coeffs, j.t, j.n_steps, j.budget, dtype)
        return f, st

    out = list(_BUILD_POOL.map(one, jobs))
    for st in {id(st): st for _, st in out}.values():
        main.wait_stream(st)
    return [f for f, _ in out]


def batch_options(jobs, views, args, dtype):
    """Batch options from the batch autotuner (kept in the autotune cache so that
    a later run, e.g. under a profiler, replays the same configuration)."""
    from paper_2606_16959_gb300 import hs
    import torch
    if args.method or args.tile_bits:  # given on the command line (profiling cases)
        return {k: v for k, v in (("method", args.method), ("tile_bits", args.tile_bits)) if v}
    if not args.autotune:
        return {}
    key = f"batch{len(jobs)}:{dtype}:{torch.cuda.get_device_name()}"
    cache = load_tune_cache()
    if key not in cache:
        facs = build_all(jobs, dtype)
        cache[key] = hs.hs_batch_autotune([(f, v, j.n_steps) for f, v, j in zip(facs, views, jobs)])
        for f in facs:
            f.close()
        save_tune_cache(cache)
    return cache[key]


def time_batch(jobs, args, world, rank, dtype):
    """Device-timed batch steps: build every job's factors, plan the batch, one
    batched launch sequence, and each job's FP64 norm; states resident."""
    import torch
    from paper_2606_16959_gb300 import hs
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    sizes = [1 << j.ham.n_qubits for j in jobs]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    host = np.concatenate([np.asarray(j.psi0).ravel() for j in jobs])
    init = torch.from_numpy(host).to(dev, tdt)
    work = torch.empty_like(init)
    views = [work[int(offs[k]):int(offs[k + 1])] for k in range(len(jobs))]
    outs = torch.zeros(len(jobs), 4, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    E = torch.cuda.Event
    bopts = batch_options(jobs, views, args, dtype)

    def step():
        work.copy_(init)
        facs = build_all(jobs, dtype)
        b = hs.hs_batch_create([(f, v, j.n_steps) for f, v, j in zip(facs, views, jobs)], use_graph=False, **bopts)
        e0, e1 = E(enable_timing=True), E(enable_timing=True)
        e0.record()
        hs.hs_batch_launch(b)
        e1.record()
        for k, v in enumerate(views):
            hs.hs_inner_device(v, v, outs[k])
        return facs, b, e0, e1

    for _ in range(args.warmup):
        facs, b, _, _ = step()
        torch.cuda.synchronize()
        info = (b.n_levels, b.n_ctas, b.n_updates, b.n_separate)
        alg = sum(algorithmic_bytes(f, j, 1) for f, j in zip(facs, jobs))
        state_bytes = 0
        if bopts.get("method") == 3:  # levels each register-batched job takes part in x its state in and out
            T, B = bopts.get("tile_bits") or 13, bopts.get("reg_bits") or 5
            for f, j in zip(facs, jobs):
                n = j.ham.n_qubits
                if n >= B + 5:
                    n_lv = hs.hs_evolve_plan(f, 1, j.n_steps, method=3, tile_bits=min(T, n),
                                             low_bits=bopts.get("low_bits") or 2, reg_bits=B)[0]
                    state_bytes += n_lv * 2 * 8 * (1 << n)
        b.close()
        for f in facs:
            f.close()
    step_ms, launch_ms = [], []
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    l0 = hs.hs_kernel_launches()
    for _ in range(args.steps):
        flush.zero_()
        s0, s1 = E(enable_timing=True), E(enable_timing=True)
        s0.record()
        facs, b, e0, e1 = step()
        s1.record()
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        launch_ms.append(e0.elapsed_time(e1))
        b.close()
        for f in facs:
            f.close()
    clocks = sampler.stop() if sampler else None
    barrier(world)
    norms = outs[:, 2].cpu().numpy()
    total_ms = max_over_ranks(sum(step_ms), world)
    return dict(units=info[2], levels=info[0], ctas=info[1], separate=info[3], step_ms=step_ms, launch_ms=launch_ms,
                total_ms=total_ms, alg_bytes=alg, state_bytes=state_bytes, clocks=clocks,
                max_norm_drift=float(np.max(np.abs(norms - 1.0))),
                launches=hs.hs_kernel_launches() - l0, bopts=bopts,
                kernel="qlevel_kernel" if bopts.get("method") == 3 else "batch_level_kernel")


def time_batch_e2e(jobs, args, dtype, bopts):
    import torch
    from paper_2606_16959_gb300 import hs
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    sizes = [1 << j.ham.n_qubits for j in jobs]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    host_in = torch.from_numpy(np.concatenate([np.asarray(j.psi0).ravel() for j in jobs])).to(tdt).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    work = torch.empty(host_in.shape, dtype=tdt, device=dev)
    views = [work[int(offs[k]):int(offs[k + 1])] for k in range(len(jobs))]
    outs = torch.zeros(len(jobs), 4, dtype=torch.float64, device=dev)
    outs_h = torch.zeros(len(jobs), 4, dtype=torch.float64).pin_memory()
    times = []
    for it in range(1 + args.steps):
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        work.copy_(host_in, non_blocking=True)
        facs = build_all(jobs, dtype)
        b = hs.hs_batch_create([(f, v, j.n_steps) for f, v, j in zip(facs, views, jobs)], use_graph=False, **bopts)
        hs.hs_batch_launch(b)
        for k, v in enumerate(views):
            hs.hs_inner_device(v, v, outs[k])
        host_out.copy_(work, non_blocking=True)
        outs_h.copy_(outs, non_blocking=True)
        s1.record()
        torch.cuda.synchronize()
        if it:
            times.append(s0.elapsed_time(s1))
        b.close()
        for f in facs:
            f.close()
    m = sum(len(j.ham.labels) for j in jobs)
    return dict(ms=statistics.mean(times), h2d=int(host_in.numel() * host_in.element_size()) + 28 * m + 256 * len(jobs),
                d2h=int(host_out.numel() * host_out.element_size()) + 32 * len(jobs))


def oracle_batch_sample(jobs, budget_s=15.0):
    """FP64 oracle on the batch's jobs in order (whole jobs, single thread),
    until about budget_s seconds of work."""
    import oracle
    done_units, t_total, n_done = 0, 0.0, 0
    for j in jobs:
        x, z, n = oracle.parse_terms(j.ham.labels)
        G = len(oracle.group_terms(x, j.budget))
        t0 = time.perf_counter()
        oracle.evolve_direct(x, z, j.ham.coeffs, j.t, j.n_steps, j.psi0)
        t_total += time.perf_counter() - t0
        done_units += j.n_steps * G * (1 << n)
        n_done += 1
        if t_total >= budget_s:
            break
    return dict(value=done_units / t_total, seconds=t_total,
                sample=f"the first {n_done} of {len(jobs)} instances, whole evolutions, direct term-by-term FP64, "
                       "single thread; units counted as steps x G x N per instance")


def oracle_sample(job, G, budget_s=15.0, order=1):
    """Time the FP64 oracle (single-threaded) on a bounded sample of the same
    workload: whole Trotter steps of state 0, as many as fit ~budget_s."""
    import oracle
    x, z, n = oracle.parse_terms(job.ham.labels)
    psi = np.asarray(job.psi0)
    psi = psi[0] if psi.ndim == 2 else psi
    N = 1 << n
    dt = job.t / job.n_steps

    def run(k):
        if job.drive is not None:
            return oracle.evolve_direct_td(x, z, job.ham.a, job.ham.b, job.drive[:k], dt * k, psi, order)
        if order == 1:
            return oracle.evolve_direct(x, z, job.ham.coeffs, dt * k, k, psi)
        return oracle.evolve_direct_order(x, z, job.ham.coeffs, dt * k, k, psi, order)

    t0 = time.perf_counter()
    run(1)
    t1 = time.perf_counter() - t0
    k = int(max(1, min(job.n_steps, budget_s // max(t1, 1e-9))))
    if k > 1:
        t0 = time.perf_counter()
        run(k)
        t1 = time.perf_counter() - t0
    else:
        k = 1
    units = k * G * N
    R = np.asarray(job.psi0).shape[0] if np.asarray(job.psi0).ndim == 2 else 1
    kind = "first-order" if order == 1 else f"order-{order} product-formula"
    if job.drive is not None:
        kind += " time-dependent"
    return dict(value=units / t1, seconds=t1, steps=k,
                sample=f"{k} of {job.n_steps} {kind} steps of state 0 (of {R}), direct term-by-term FP64 "
                       f"evolution, single thread; units counted as steps x {G} factor applications x N={N}")


def oracle_fanout_sample(job, G, steps, order=1):
    """The same oracle on every host core at once: one spawned process per core,
    each evolving `steps` whole steps of one state of the workload (states
    taken in order, repeated when there are more cores than states)."""
    import oracle
    from oracle import fanout
    x, z, n = oracle.parse_terms(job.ham.labels)
    psi = np.asarray(job.psi0)
    rows = psi if psi.ndim == 2 else psi[None, :]
    cores = fanout.host_cores()
    dt = job.t / job.n_steps
    tasks = []
    for c in range(cores):
        p0 = rows[c % rows.shape[0]]
        if job.drive is not None:
            tasks.append(("td", (x, z, job.ham.a, job.ham.b, job.drive[:steps], dt * steps, p0, order)))
        elif order == 1:
            tasks.append(("direct", (x, z, job.ham.coeffs, dt * steps, steps, p0)))
        else:
            tasks.append(("order", (x, z, job.ham.coeffs, dt * steps, steps, p0, order)))
    t0 = time.perf_counter()
    fanout.run_many(tasks, workers=cores)
    wall = time.perf_counter() - t0
    units = cores * steps * G * (1 << n)
    return dict(value=units / wall, seconds=wall, cores=cores,
                sample=f"{cores} spawned processes, one per host core, each {steps} whole step(s) of one of the "
                       f"{rows.shape[0]} states (direct term-by-term FP64, unchanged oracle); wall time includes "
                       "process start-up; units counted as processes x steps x "
                       f"{G} factor applications x N={1 << n}")


def oracle_batch_fanout(jobs, budget_s=15.0):
    """Whole batch instances on every host core at once (one spawned process
    per instance, as many instances as fit ~budget_s of single-core work)."""
    import oracle
    from oracle import fanout
    cores = fanout.host_cores()
    tasks, units = [], 0
    for j in jobs[: 4 * cores]:
        x, z, n = oracle.parse_terms(j.ham.labels)
        G = len(oracle.group_terms(x, j.budget))
        tasks.append(("direct", (x, z, j.ham.coeffs, j.t, j.n_steps, j.psi0)))
        units += j.n_steps * G * (1 << n)
    t0 = time.perf_counter()
    fanout.run_many(tasks, workers=cores)
    wall = time.perf_counter() - t0
    return dict(value=units / wall, seconds=wall, cores=cores,
                sample=f"the first {len(tasks)} of {len(jobs)} instances, whole evolutions, on {cores} spawned "
                       "processes (one per host core, direct term-by-term FP64, unchanged oracle)")


def cpu_baseline_of(job, G, order=1):
    """Single-thread oracle on a bounded sample, and the all-cores fan-out."""
    cb = oracle_sample(job, G, order=order)
    fo = oracle_fanout_sample(job, G, cb["steps"], order=order)
    return {"value": cb["value"], "unit": METRIC, "cores": 1, "kind": "oracle", "sample": cb["sample"],
            "all_cores": {"value": fo["value"], "unit": METRIC, "cores": fo["cores"], "kind": "oracle",
                          "sample": fo["sample"]}}


def config_of(args, job, desc, res=None):
    c = {"workload": args.workload, "description": desc, "n_qubits": job.ham.n_qubits, "n_terms": len(job.ham.labels),
         "n_steps": job.n_steps, "diag_budget": job.budget, "n_rhs": int(np.asarray(job.psi0).shape[0]) if np.asarray(job.psi0).ndim == 2 else 1,
         "t": job.t, "l2": "flushed (512 MiB write) before every timed step"}
    if getattr(args, "order", 1) != 1:
        c["product_formula_order"] = args.order
    if job.drive is not None:
        c["time_dependent"] = "H0 + f(t) H1, f frozen per step at the caller's sample"
        c["driven_terms"] = int(np.count_nonzero(job.ham.b))
    if res:
        c.update({"factor_applications_per_step": res["G"], "tile_bits": res["tile_bits"], "rhs_block": res["rhs_block"],
                  "sweep_launches_per_step": res["n_sweeps"], "plain_launches_per_step": res["n_plain"]})
    return c


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # Each reference step: the unchanged FP64 oracle on every host core at once
    # (one spawned process per core, independent states or instances), a
    # bounded sample of the workload sized so that the run ends in minutes.
    per_step_budget = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    if args.workload == "batch256":
        jobs, desc = batch_jobs(args)
        job = jobs[0]
        sample = lambda: oracle_batch_fanout(jobs, per_step_budget)
        cfg = {"workload": "batch256", "description": desc, "n_jobs": len(jobs)}
    else:
        job, desc = make_job(args.workload)
        import oracle as _o
        x, z, n = _o.parse_terms(job.ham.labels)
        G = len(_o.group_terms(x, job.budget)) * (1 if args.order == 1 else 2 if args.order == 2 else 10)
        probe = oracle_sample(job, G, per_step_budget, order=args.order)
        sample = lambda: oracle_fanout_sample(job, G, probe["steps"], order=args.order)
        cfg = config_of(args, job, desc)
    for _ in range(args.warmup):
        sample()
    vals, secs = [], []
    for _ in range(args.steps):
        r = sample()
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = len(vals) / sum(1.0 / x for x in vals)
    line = {"metric": METRIC, "value": v, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic", "impl": "reference",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch
    rank, world, local = dist_setup(args)
    from paper_2606_16959_gb300 import hs
    hs.lib()
    if args.workload == "batch256":
        return run_batch(args, rank, world)
    if args.workload == "serve":
        return run_serve(args, rank, world)
    if args.workload == "taylor16":
        return run_taylor(args, rank, world)
    job, desc = make_job(args.workload, qubits=args.qubits)
    dtype = job.dtype
    res = time_ours(job, args, world, dtype, rank)
    K = args.steps
    value = res["units"] * K * world / (res["total_ms"] / 1000.0)
    ms = res["total_ms"] / K
    e2e = time_e2e(job, args, dtype)
    hbm, peak_kind = peaks()
    launches_evolve = res["n_sweeps"] + res["n_plain"]
    avg_launch_s = statistics.mean(res["evolve_ms"]) / 1000.0 / max(1, launches_evolve)
    model_bytes = res["alg_bytes"] / max(1, launches_evolve)
    kernel = sweep_kernel_name(args.tuned_opts, res["n_sweeps"])
    # A register sweep reads no stored factor value (it generates them), so its
    # algorithmic bytes per launch are the state in and out once; the per
    # factor-application figure of the staged paths stays beside it (model_*).
    s_bytes = 8 if dtype == "c64" else 16
    per_launch_bytes = 2 * s_bytes * res["N"] * res["R"] if kernel == "qsweep_kernel" else model_bytes
    achieved = per_launch_bytes / avg_launch_s / 1e9
    traffic = profiled_traffic(args.workload, kernel) if not args.qubits else None
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic", "config": config_of(args, job, desc, res),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic, "peak_source": peak_kind,
                         "kernel": kernel,
                         "algorithmic_bytes_per_launch": per_launch_bytes,
                         "model_bytes_per_launch": model_bytes, "model_frac": model_bytes / avg_launch_s / 1e9 / hbm,
                         "avg_launch_us": avg_launch_s * 1e6, **dram_fields(traffic, avg_launch_s, hbm),
                         **({"note": "evolution time per sweep launch, including the launches that "
                                     "compute the driven factors' records and values"}
                            if job.drive is not None else {})},
            "e2e": {"value": res["units"] / (e2e["ms"] / 1000.0), "unit": METRIC,
                    "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]},
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "evolve_ms_per_step": statistics.mean(res["evolve_ms"]), "autotuned": res["tuned"]}
    if args.workload in ("heis16", "maxcut24") and not args.qubits and not args.no_c128 and world >= 1:
        r2 = time_ours(make_job(args.workload, "c128")[0], args, world, "c128", rank)
        line["c128"] = {"value": r2["units"] * K * world / (r2["total_ms"] / 1000.0),
                        "ms_per_step": r2["total_ms"] / K, "evolve_ms_per_step": statistics.mean(r2["evolve_ms"])}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_of(job, res["G"], order=args.order)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args, rank, world):
    import torch
    jobs, desc = batch_jobs(args)
    dtype = "c64"
    res = time_batch(jobs, args, world, rank, dtype)
    K = args.steps
    value = res["units"] * K * world / (res["total_ms"] / 1000.0)
    e2e = time_batch_e2e(jobs, args, dtype, res["bopts"])
    hbm, peak_kind = peaks()
    launch_s = statistics.mean(res["launch_ms"]) / 1000.0
    model_bytes = res["alg_bytes"] / max(1, res["levels"])
    # register-sweep levels: the states of the level's jobs in and out (see run_ours)
    total_bytes = res["state_bytes"] if res.get("kernel") == "qlevel_kernel" else res["alg_bytes"]
    per_launch_bytes = total_bytes / max(1, res["levels"])
    achieved = total_bytes / launch_s / 1e9
    traffic = profiled_traffic("batch256", res.get("kernel", "batch_level_kernel")) if args.batch_jobs == 256 else None
    cfg = {"workload": "batch256", "description": desc, "n_jobs": len(jobs), "levels_per_step": res["levels"],
           "ctas_per_step": res["ctas"], "separate_jobs": res["separate"], "batch_options": res["bopts"],
           "l2": "flushed (512 MiB write) before every timed step"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": res["total_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic, "peak_source": peak_kind, "kernel": res["kernel"],
                         "algorithmic_bytes_per_launch": per_launch_bytes,
                         "model_bytes_per_launch": model_bytes,
                         "model_frac": res["alg_bytes"] / launch_s / 1e9 / hbm,
                         "avg_launch_us": launch_s * 1e6 / max(1, res["levels"]),
                         **dram_fields(traffic, launch_s / max(1, res["levels"]), hbm)},
            "e2e": {"value": res["units"] / (e2e["ms"] / 1000.0), "unit": METRIC,
                    "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]},
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "batch_launch_ms_per_step": statistics.mean(res["launch_ms"]), "max_norm_drift": res["max_norm_drift"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_batch_sample(jobs)
        fo = oracle_batch_fanout(jobs)
        line["cpu_baseline"] = {"value": cb["value"], "unit": METRIC, "cores": 1, "kind": "oracle", "sample": cb["sample"],
                                "all_cores": {"value": fo["value"], "unit": METRIC, "cores": fo["cores"],
                                              "kind": "oracle", "sample": fo["sample"]}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


TAYLOR_DESC = ("single-factor Taylor mode (Alg. 3): TFIM open chain n={n}, J=1, h=0.1, Gaussian state, t=1, "
               "diagonal budget {b}; H to the compact layout, budgeted step search, SpME (FP64), complex64 SpMV "
               "evolution, FP64 norm")


def taylor_job(args):
    from paper_2606_16959_gb300 import workloads as W
    n = args.qubits or 16
    job = W.taylor_tfim(n=n)
    return job, TAYLOR_DESC.format(n=n, b=job.budget)


def time_taylor(job, args, world, rank):
    """Device-timed Alg. 3 steps: every step rebuilds H, searches r, builds U and
    evolves r SpMVs; the SpMV evolution is also timed on its own."""
    import torch
    from paper_2606_16959_gb300 import hs
    dev = torch.device("cuda", torch.cuda.current_device())
    psi0 = torch.from_numpy(np.ascontiguousarray(job.psi0)).to(dev, torch.complex64)
    work = torch.empty_like(psi0)
    out4 = torch.zeros(4, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    E = torch.cuda.Event
    info = {}

    def step():
        work.copy_(psi0)
        H = hs.hs_dia_from_terms(job.ham.labels, job.ham.coeffs)
        r = hs.hs_estimate_timesteps(H, job.t, job.budget)
        U, K, ok = hs.hs_spme(H, job.t / r)
        Uc = hs.hs_dia_convert(U, "c64")
        e0, e1 = E(enable_timing=True), E(enable_timing=True)
        e0.record()
        hs.hs_dia_evolve(Uc, work, r)
        e1.record()
        hs.hs_inner_device(work, work, out4)
        info.update(r=r, K=K, converged=ok, D=U.n_diags, H_diags=H.n_diags,
                    S=int(sum(Uc.N - abs(int(d)) for d in Uc.offsets())))
        return (H, U, Uc), e0, e1

    for _ in range(args.warmup):
        keep, _, _ = step()
        torch.cuda.synchronize()
    step_ms, evolve_ms = [], []
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    l0 = hs.hs_kernel_launches()
    for _ in range(args.steps):
        flush.zero_()
        s0, s1 = E(enable_timing=True), E(enable_timing=True)
        s0.record()
        keep, e0, e1 = step()
        s1.record()
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        evolve_ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop() if sampler else None
    barrier(world)
    N = 1 << job.ham.n_qubits
    return dict(units=info["r"] * N, step_ms=step_ms, evolve_ms=evolve_ms,
                total_ms=max_over_ranks(sum(step_ms), world), clocks=clocks, info=info,
                norm2=float(out4[2].item()), N=N, launches=hs.hs_kernel_launches() - l0)


def oracle_taylor_sample(budget_s=15.0):
    """The oracle's whole Alg. 3 pipeline (H in the compact layout, step search,
    Taylor exponential, r SpMVs) on the 10-qubit instance of the same family at
    the same diagonal-budget fraction of 2N-1, repeated for ~budget_s seconds."""
    import oracle as _o
    from oracle import taylor as OT
    from paper_2606_16959_gb300 import workloads as W
    n = 10
    job = W.taylor_tfim(n=n, budget=256)
    x, z, _ = _o.parse_terms(job.ham.labels)
    units, t_total, reps = 0, 0.0, 0
    while t_total < budget_s or reps == 0:
        t0 = time.perf_counter()
        A = OT.ham_dia(x, z, job.ham.coeffs, n)
        r = OT.estimate_timesteps(A, job.t, job.budget)
        U, _, _ = OT.expm_taylor(A, job.t / r)
        OT.evolve(U, job.psi0, r)
        t_total += time.perf_counter() - t0
        units += r * (1 << n)
        reps += 1
    return dict(value=units / t_total, seconds=t_total,
                sample=f"{reps} run(s) of the oracle's whole Alg. 3 pipeline on the {n}-qubit TFIM chain "
                       f"(h=0.1, budget {job.budget} of 2N-1={2 * (1 << n) - 1}, r={r}), FP64 numpy, "
                       "single thread; units r x N")


def run_taylor(args, rank, world):
    import torch
    job, desc = taylor_job(args)
    res = time_taylor(job, args, world, rank)
    K = args.steps
    info = res["info"]
    value = res["units"] * K * world / (res["total_ms"] / 1000.0)
    hbm, peak_kind = peaks()
    launch_s = statistics.mean(res["evolve_ms"]) / 1000.0 / max(1, info["r"])
    per_launch = 8 * info["S"] + 2 * 8 * res["N"]
    achieved = per_launch / launch_s / 1e9
    traffic = profiled_traffic("taylor16", "spmv_kernel") if not args.qubits else None
    cfg = {"workload": "taylor16", "description": desc, "n_qubits": job.ham.n_qubits, "n_terms": len(job.ham.labels),
           "diag_budget": job.budget, "t": job.t, "n_rhs": 1, "H_diags": info["H_diags"], "n_steps": info["r"],
           "U_diags": info["D"], "taylor_terms": info["K"], "l2": "flushed (512 MiB write) before every timed step"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": res["total_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic, "peak_source": peak_kind, "kernel": "spmv_kernel",
                         "algorithmic_bytes_per_launch": per_launch, "avg_launch_us": launch_s * 1e6,
                         **dram_fields(traffic, launch_s, hbm)},
            "e2e": None, "gpu_launches": res["launches"], "clocks": res["clocks"],
            "evolve_ms_per_step": statistics.mean(res["evolve_ms"]), "final_norm2": res["norm2"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_taylor_sample()
        line["cpu_baseline"] = {"value": cb["value"], "unit": METRIC, "cores": 1, "kind": "oracle",
                                "sample": cb["sample"]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def serve_batch_opts(jobs, n=16):
    """Batch options for served groups: hs_batch_autotune on a group of the
    stream's first requests (factors and seeded states built on the device)."""
    import torch
    from paper_2606_16959_gb300 import hs
    sel = jobs[:n]
    facs, states = [], []
    for j in sel:
        facs.append(hs.hs_build_factors(j.ham.labels, j.ham.coeffs, j.t, j.n_steps, j.budget, "c64"))
        g = torch.Generator(device="cuda")
        g.manual_seed(int(j.seed))
        st = torch.complex(torch.randn(1 << j.ham.n_qubits, generator=g, device="cuda"),
                           torch.randn(1 << j.ham.n_qubits, generator=g, device="cuda"))
        states.append(st / torch.linalg.vector_norm(st))
    opts = hs.hs_batch_autotune([(f, st, j.n_steps) for f, st, j in zip(facs, states, sel)])
    for f in facs:
        f.close()
    torch.cuda.synchronize()
    return opts


def serve_trial(rate, seconds, opts, seed=1005):
    """One realtime Poisson stream through a fresh server; its stats with the
    offered rate and whether the queue stayed bounded (the median latency of
    the last quarter of the requests within 1.2x that of the second quarter
    plus 25 ms)."""
    from paper_2606_16959_gb300 import serve, workloads as W
    reqs = serve.requests_from_jobs(W.serve_stream(rate=rate, duration=seconds, seed=seed))
    st = serve.Server(batch_opts=opts).run(reqs, realtime=True)
    st.update(rate=rate, seconds=seconds, bounded=bool(st["p50_q4_ms"] <= 1.2 * st["p50_q2_ms"] + 25.0))
    return st


def find_serve_rate(args, opts):
    """Highest bounded rate over 20-s streams: start from the capacity of an
    all-at-once run, step by 1.25x until the boundary, then report p50/p99 at
    that rate, at half of it and at --serve-rate."""
    from paper_2606_16959_gb300 import serve, workloads as W
    probe = serve.requests_from_jobs(W.serve_stream(rate=args.serve_rate, duration=2.0, seed=1005))
    for r in probe:
        r.arrival = 0.0
    cap = serve.Server(batch_opts=opts).run(probe, realtime=False)
    capacity = cap["n"] / max(cap["makespan_s"], 1e-9)
    trials = []
    rate = 0.8 * capacity
    st = serve_trial(rate, 20.0, opts)
    trials.append(st)
    step = 1.25 if st["bounded"] else 1 / 1.25
    for _ in range(6):
        nxt = serve_trial(rate * step, 20.0, opts)
        trials.append(nxt)
        if nxt["bounded"] != st["bounded"]:
            break
        rate, st = rate * step, nxt
    good = [t for t in trials if t["bounded"]]
    best = max(good, key=lambda t: t["rate"]) if good else None
    half = serve_trial(best["rate"] / 2, 20.0, opts) if best else None
    conf = serve_trial(args.serve_rate, 20.0, opts)
    keys = ("rate", "n", "p50_ms", "p99_ms", "mean_ms", "bounded", "backlog_at_last_arrival", "drain_s",
            "p50_q2_ms", "p50_q4_ms", "throughput", "peak_bytes")
    pick = lambda t: None if t is None else {k: t[k] for k in keys}
    return dict(capacity_req_s=capacity, capacity_run={"n": cap["n"], "makespan_s": cap["makespan_s"]},
                sustainable=pick(best), half=pick(half), configured=pick(conf), trials=[pick(t) for t in trials])


def run_serve(args, rank, world):
    """A step = serving one Poisson request stream (arrivals over --serve-seconds,
    then the drain).  Value = amplitude updates of all requests / (last
    completion - first arrival); p50/p99 arrival-to-completion latency beside it."""
    import torch
    from paper_2606_16959_gb300 import serve, workloads as W
    jobs = W.serve_stream(rate=args.serve_rate, duration=args.serve_seconds, seed=1005)
    jobs = serve.shard_jobs(jobs, rank, world)
    desc = (f"Poisson stream {args.serve_rate:g} req/s for {args.serve_seconds:g} s (seed 1005): TFIM, Heisenberg, "
            "MaxCut (n~U{12..24}) and one-hot TSP (16 qubits), t~U[0.5,2], steps~U{10..100}, complex64, "
            "per-family budgets; HBM admission")
    bopts = serve_batch_opts(jobs)
    for _ in range(args.warmup):
        warm = serve.requests_from_jobs(jobs[:8])
        for r in warm:
            r.arrival = 0.0
        serve.Server(batch_opts=bopts).run(warm, realtime=False)
    if args.serve_find_rate:
        if rank == 0:
            res = find_serve_rate(args, bopts)
            print(json.dumps({"workload": "serve", "search": "sustainable Poisson rate", "batch_options": bopts,
                              "description": desc.replace(f" {args.serve_rate:g} req/s for {args.serve_seconds:g} s",
                                                          ""), **res}))
        return
    runs = []
    barrier(world)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    from paper_2606_16959_gb300 import hs
    l0 = hs.hs_kernel_launches()
    for _ in range(args.steps):
        reqs = serve.requests_from_jobs(jobs)
        runs.append(serve.Server(batch_opts=bopts).run(reqs, realtime=True))
    served_launches = hs.hs_kernel_launches() - l0
    clocks = sampler.stop() if sampler else None
    barrier(world)
    updates = sum(r["updates"] for r in runs)
    span = max_over_ranks(sum(r["makespan_s"] for r in runs), world)
    value = updates * world / span
    p50 = statistics.median([r["p50_ms"] for r in runs])
    p99 = max(r["p99_ms"] for r in runs)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * span / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "serve", "description": desc, "requests_per_step": len(jobs),
                       "l2": "inputs larger than L2 (factor sets up to 16 GB)", "batch_options": bopts},
            "latency_ms": {"p50": p50, "p99": p99, "mean": statistics.mean([r["mean_ms"] for r in runs])},
            "queue": {"backlog_at_last_arrival": max(r["backlog_at_last_arrival"] for r in runs),
                      "drain_s": max(r["drain_s"] for r in runs),
                      "p50_q2_ms": statistics.median([r["p50_q2_ms"] for r in runs]),
                      "p50_q4_ms": statistics.median([r["p50_q4_ms"] for r in runs])},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 32 * len(jobs)},
            "gpu_launches": served_launches, "clocks": clocks, "peak_admitted_bytes": max(r["peak_bytes"] for r in runs)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
