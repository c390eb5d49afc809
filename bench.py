#!/usr/bin/env python
"""Benchmark: particle-steps/s of the PM+PP force + KDK step on one GB300.

Workload (default): 256^3 particles in a 256 Mpc/h box, two PM levels (coarse
128^3 + fine 512^3), FP32 velocities, seeded Zel'dovich ICs at z = 49
(BBKS spectrum), the 50-step constant-Delta-a KDK schedule to z = 0.  A step is
one kdk_step of that schedule over the whole box (drift + re-bin, deposit on
both meshes, both Poisson solves, interpolation, PP, both kicks).

Timing: W warm-up steps from the ICs; then the whole schedule runs once from
the ICs (untimed for the headline, reported as ``full_schedule``), keeping
the states at K step indices spread evenly over it; the timed region runs
those K steps, each from its kept state (restored outside its CUDA-event
pair), so the headline covers the early (PM-bound) and late (PP-bound)
parts of the schedule in proportion.  value = K N / summed step durations.

Also reported on the same JSON line:
  roofline      dominant kernel class: algorithmic work per launch / its mean
                CUDA-event duration inside the timed region, against the
                measured HBM copy bandwidth, or for PP the FP32 FMA rate the
                library's probe kernel measures on this device
  e2e           the same steps through cube2_kdk_step_host with the particle
                state in pinned host memory (H2D + step + D2H every step)
  adjoint       adjoint/forward time ratio of the differentiation workload
  cpu_baseline  the FP64 oracle on all host cores, on a bounded sample of the
                same recipe
  clocks        nvidia-smi samples taken during the timed region

--impl reference times the FP64 oracle alone (this project's reference arm).
With torchrun (N > 1) every rank runs an independent realisation of the box
(another seed of the same recipe; the single box does not shard, so there
are replicas only and no data-path collective); the units all ranks
processed over the slowest rank's time set the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/sec (PM+PP force + KDK) on 1 GB300; adjoint/forward ratio"
UNIT = "particle-steps/s"
HBM_FALLBACK_GBS = 6800.0
SAMPLE_NP = 32          # oracle sample: same recipe as the workload at 32^3 particles


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cube2", choices=["cube2", "reference"])
    ap.add_argument("--workload", default="pm2-256c-128x512mesh")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward sub-record")
    ap.add_argument("--streams", type=int, default=16, help="graph branches of the ensemble workload")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Ranks:
    """The job's ranks as bench.py uses them: reductions of per-rank scalars
    (the slowest rank's time, the units all ranks processed) and barriers.
    ``dist`` is torch.distributed with an initialised group, or None for one
    rank; ``device`` is where the reduction tensors live ("cuda" under NCCL,
    "cpu" under gloo)."""

    def __init__(self, dist=None, device="cpu"):
        self.dist, self.device = dist, device
        self.world = dist.get_world_size() if dist else 1
        self.rank = dist.get_rank() if dist else 0

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def _reduce(self, x, op):
        if not self.dist:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX if self.dist else None)

    def sum(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM if self.dist else None)


def replica_workload(w, rank):
    """The box rank ``rank`` simulates: the workload itself on rank 0, an
    independent realisation (another seed of the same recipe) elsewhere."""
    return w if rank == 0 else w.with_(seed=w.seed + 7919 * rank)


def ensemble_share(ws, world, rank):
    """Indices of the ensemble boxes rank ``rank`` simulates: the boxes are
    split over the ranks by the library's LPT placement of its per-box cost
    estimate (largest first, to the least loaded rank)."""
    from paper_2512_12629_gb300 import cube2
    costs = [cube2.config_cost(cube2.make_config(w)) for w in ws]
    bins = cube2.lpt_partition(costs, world)
    return [i for i, b in enumerate(bins) if b == rank]


def job_throughput(units_all_ranks, seconds_slowest):
    """Whole-job particle-steps/s: units processed by all ranks / slowest rank."""
    return units_all_ranks / seconds_slowest


# ----------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.bus_id:
                cmd += ["-i", self.bus_id]
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def numa_cpus(bus_id, root="/sys"):
    """(node, CPUs) of the NUMA node sysfs names for the PCI device `bus_id`
    ("DDDDDDDD:BB:DD.F" as torch reports it), or None."""
    try:
        dom, bus, devfn = bus_id.lower().split(":")
        node = int(open(f"{root}/bus/pci/devices/{dom[-4:]}:{bus}:{devfn}/numa_node").read())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"{root}/devices/system/node/node{node}/cpulist").read().strip().split(","):
            if part:
                lo, _, hi = part.partition("-")
                cpus.update(range(int(lo), int(hi or lo) + 1))
        return (node, cpus) if cpus else None
    except (OSError, ValueError, AttributeError):
        return None


def bind_local_numa(bus_id):
    """Restrict this process to the CPUs of the NUMA node the GPU hangs off (as
    sysfs reports it), so that pinned host buffers allocated afterwards are
    local to that node; returns the node or None (nothing changed)."""
    found = numa_cpus(bus_id)
    if not found:
        return None
    try:
        os.sched_setaffinity(0, found[1])
    except OSError:
        return None
    return found[0]


def bus_id_of(dev):
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ------------------------------------------------------ algorithmic bytes
def algorithmic_bytes(w, n_part, cls, level):
    """Compulsory HBM bytes of one launch group of a kernel class (each array once)."""
    N, C = n_part, w.n_ios ** 3
    meshes = [lv.n_mesh for lv in w.levels]
    n = meshes[level] if level < len(meshes) else meshes[-1]
    half = n * n * (n // 2 + 1)
    m = n // 2 + 1
    green_len = m * (m + 1) * (m + 2) // 6           # the symmetry-reduced Green's table
    tsc = getattr(w, "assign_order", 2) == 3
    table = {
        # CIC: both levels in one pass; TSC: one launch group per level (fill, atomic deposit)
        "deposit": 10 * N + 4 * n ** 3 if tsc else 6 * N + 8 * C + sum(4 * m ** 3 for m in meshes),
        "fft_x_fwd": 4 * n ** 3 + 8 * half,
        "fft_y_fwd": 16 * half,
        "fft_z_green": 16 * half + 4 * green_len,
        "fft_y_inv": 16 * half,
        "fft_x_inv": 8 * half + 4 * n ** 3,
        "interp": 4 * n ** 3 + 22 * N if tsc else sum(4 * m ** 3 for m in meshes) + 22 * N,
        "pp": 58 * N + 8 * C,
        "kick": 36 * N,
        "kick_drift": 68 * N + 4 * C,
        "scan": 8 * C,
        "scatter": 16 * N,
        "sort": 8 * C + 8 * N,
        "gather": 48 * N,
        "cellid": 8 * C + 4 * N,
        "green": 4 * green_len,
        "prep": 26 * N,
        "pp_order": 4 * C + 26 * N,
        "sort_big": 8 * N,
    }
    # the third level's classes move data-dependent amounts (the refined
    # subtiles' local boxes): no algorithmic figure
    return table.get(cls)


# FP32 operations (an FMA counts 2) of one in-range PP pair, as the roofline
# counts them: the separation 3, r^2 5, the reciprocal square root and the
# scaled distance u = r / b 3, one shell polynomial of R_PP in Horner form 14,
# the 1/r^3 scaling and the product with the force factor 2, accumulation of
# the three components 3: 30.  The kernel as written also evaluates the second
# shell polynomial and forms the powers of v = 1 - u (45 in all), and tests
# every candidate (separation 3 and r^2 - b^2 6); both are reported beside it.
PP_FLOPS_PAIR = 30
PP_FLOPS_PAIR_AS_WRITTEN = 45
PP_FLOPS_CANDIDATE = 9


def fp32_peak_derived(sms, sm_mhz):
    """SMs x 128 FP32 lanes x 2 (FMA) x clock, TFLOP/s."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def measure_fp32_peak(cube2, torch, reps=3):
    """FP32 FMA rate of this device from the library's probe kernel (8 blocks
    of 256 threads per SM, 8 independent FMA chains per thread), timed with
    CUDA events; the best of ``reps`` launches of ~20 ms, TFLOP/s."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    out = torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream()
    blocks, threads = sms * 8, 256
    cube2.fma_probe(out, blocks, threads, 64, stream)
    iters = 2000
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = cube2.fma_probe(out, blocks, threads, iters, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best, sms


def pp_roofline(pairs, cands, launches, per_launch_ms, peak_tflops, sms, sm_mhz, traffic=None):
    """Roofline record of the PP kernel class: in-range pair work (PP_FLOPS_PAIR
    per ordered pair) per launch over the mean launch time, against the FP32
    FMA rate measured by the probe kernel."""
    flops = pairs * PP_FLOPS_PAIR / launches
    sec = per_launch_ms / 1e3
    achieved = flops / sec / 1e12
    return {"bound": "alu", "kernel": "pp_kernel (shared-stream and per-lane paths)", "achieved": achieved,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "peak_source": f"measured: FP32 FMA probe kernel (cube2_fma_probe), CUDA events, {sms} SMs",
            "peak_derived": fp32_peak_derived(sms, sm_mhz), "peak_derived_note":
            f"{sms} SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz (median SM clock in the timed region)",
            "flops_per_pair": PP_FLOPS_PAIR, "algorithmic_flops_per_launch": flops,
            "achieved_as_written": pairs * PP_FLOPS_PAIR_AS_WRITTEN / launches / sec / 1e12,
            "achieved_with_candidate_tests": (pairs * PP_FLOPS_PAIR_AS_WRITTEN + cands * PP_FLOPS_CANDIDATE)
            / launches / sec / 1e12,
            "pairs_per_launch": pairs / launches, "candidates_per_launch": cands / launches,
            "mean_launch_ms": per_launch_ms, "traffic": traffic}


def traffic_record(kernel):
    """ncu DRAM bytes per launch for `kernel` from profiles/traffic.json, if the
    kernel's source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
        if not rec:
            return None
        src = os.path.join(ROOT, "paper_2512_12629_gb300", "csrc", rec["source"])
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return rec["bytes_per_launch"] if digest == rec["sha256_16"] else None
    except Exception:
        return None


# ------------------------------------------------------------- CPU oracle
def sampled_steps(n_steps, k):
    """Indices of the k timed steps, spread evenly over the n_steps-step
    schedule (the middle of k equal stretches); the whole schedule, repeated,
    when k >= n_steps."""
    reps, rest = divmod(k, n_steps)
    idx = list(range(n_steps)) * reps
    idx += [int((j + 0.5) * n_steps / rest) for j in range(rest)]
    return sorted(idx)


def oracle_sample_workload(w):
    """The workload's recipe scaled to SAMPLE_NP^3 particles (same resolution)."""
    from inputs.workloads import Level
    scale = SAMPLE_NP / w.n_p
    return w.with_(name=w.name + "-sample", n_p=SAMPLE_NP, box=w.box * scale, n_ios=int(w.n_ios * scale),
                   levels=tuple(Level(int(lv.n_mesh * scale), lv.beta) for lv in w.levels))


def _oracle_worker(job):
    """One host core: run the FP64 oracle through the schedule of the sample
    workload ``sw`` (untimed), keep the states at the steps in ``idx``, then
    time one oracle KDK step from each kept state.  Returns (seconds, steps,
    particles per step)."""
    sw, idx = job
    from inputs.zeldovich import zeldovich_ios
    from oracle import kdk as okdk
    from oracle import mesh as omesh
    st = zeldovich_ios(sw)
    greens = omesh.green_tables(sw)
    state = dict(off=st["off"], count=st["count"], start=st["start"], vel=st["vel"].astype("float64"))
    state["acc"] = okdk.total_force(st["off"], st["count"], st["start"], sw, greens)
    a = sw.scale_factors()
    keep = {}
    last = max(idx)
    for i in range(last + 1):
        if i in idx:
            keep[i] = dict(state)
        if i < last:
            state = okdk.kdk_step(state, sw, a[i], a[i + 1], greens)
    el = 0.0
    for i in idx:
        t0 = time.perf_counter()
        okdk.kdk_step(keep[i], sw, a[i], a[i + 1], greens)
        el += time.perf_counter() - t0
    return el, len(idx), sw.n_particles


def host_cpu():
    """(model name, logical cores) of this host, from lscpu."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model, os.cpu_count() or 1


def oracle_timing(w, idx, procs=None):
    """The FP64 oracle as it stands, timed on the host cores: ``procs``
    independent processes (default: one per core), each an independent
    realisation of the workload's recipe at SAMPLE_NP^3 particles timed on the
    steps ``idx`` of its schedule (_oracle_worker).  Returns a dict with the
    aggregate particle-steps/s (all particle-steps over the slowest process's
    timed seconds), the single-core rate (median over processes), the core
    count and CPU model, and the sample's description."""
    import multiprocessing as mp
    model, ncpu = host_cpu()
    procs = procs or ncpu
    sw = oracle_sample_workload(w)
    jobs = [(sw.with_(seed=sw.seed + 7919 * j), list(idx)) for j in range(procs)]
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, jobs)
    slowest = max(r[0] for r in res)
    units = sum(r[1] * r[2] for r in res)
    single = statistics.median(r[1] * r[2] / r[0] for r in res)
    desc = (f"FP64 numpy oracle as it stands: {procs} processes on {procs} host cores, each an independent "
            f"realisation of the workload recipe scaled to {SAMPLE_NP}^3 particles (box {sw.box:g} Mpc/h, meshes "
            f"{[lv.n_mesh for lv in sw.levels]}, IOS {sw.n_ios}^3), one KDK step timed from each of the schedule "
            f"states {sorted(set(idx))} (reached untimed); Green's tables built outside the timing")
    return {"value": units / slowest, "single_core_value": single, "cores": procs, "cpu_model": model,
            "seconds": slowest, "steps_per_process": len(idx), "sample": desc}


def run_reference(args, w):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    idx = sampled_steps(w.n_steps, args.steps)
    t = oracle_timing(w, idx)
    value = t["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t["seconds"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Zel'dovich ICs, BBKS spectrum)", "config": workload_config(w, idx),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": t["cores"], "kind": "oracle", "sample": t["sample"],
                         "cpu_model": t["cpu_model"], "single_core_value": t["single_core_value"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w, idx=None):
    cfg = {"workload": w.name, "particles": w.n_particles, "box_mpc_h": w.box,
           "meshes": [lv.n_mesh for lv in w.levels], "ios_cells": w.n_ios,
           "schedule": f"{w.n_steps} KDK steps z={w.z_init:g}->{w.z_final:g}, constant Delta a",
           "l2": "inputs larger than L2 (>= 2 GB resident working set); each timed step starts after a "
                 "checkpoint restore larger than L2", "parallelism": "replicas"}
    if idx is not None:
        a = w.scale_factors()
        cfg["timed_steps"] = sorted(set(idx))
        cfg["timed_a_range"] = [a[min(idx)], a[max(idx) + 1]]
        cfg["timing"] = ("each timed step is one kdk_step of the schedule from the state the untimed run "
                         "reached there; value = steps x particles / summed CUDA-event step durations")
    return cfg


# ------------------------------------------------------------------ main
ENSEMBLE = "c4-ensemble-64x20"


def run_ensemble(args):
    """The 64-box ensemble (inputs.workloads.c4_ensemble), every box's 20 KDK
    steps recorded as one CUDA graph; a step of this bench is one launch of
    that graph (64 boxes x 20 steps), timed with CUDA events after the
    particle states are reset to the initial conditions.  Two recordings of
    the same work are timed the same way: per-box launches on concurrent
    graph branches, and step by step with one persistent PP kernel over every
    box fed by the cost-ordered device queue, its knobs chosen by the
    library's autotuner (cube2_ensemble_autotune)."""
    import numpy as np
    import torch
    from inputs.workloads import c4_ensemble
    from inputs.zeldovich import zeldovich_ios
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    ranks = Ranks(dist, "cuda")
    from paper_2512_12629_gb300 import build as pkg_build
    if rank == 0:
        pkg_build.build()
    ranks.barrier()
    pkg_build.build()
    from paper_2512_12629_gb300 import cube2
    ws = c4_ensemble()
    mine = [ws[i] for i in ensemble_share(ws, world, rank)]
    ctxs, states, ics = [], [], []
    for w in mine:
        st = zeldovich_ios(w)
        ctx = cube2.init_mesh(cube2.make_config(w, n_particles=int(st["count"].sum())))
        ctx.set_green(0)
        p = cube2.IOSState.from_numpy(st)
        ctx.force(p)
        ctxs.append(ctx)
        states.append(p)
        ics.append(p.clone())
    for c in ctxs:
        c.check()
    torch.cuda.synchronize()
    sched = np.array([w.scale_factors() for w in mine])
    stream = torch.cuda.current_stream()

    def reset():
        for p, q in zip(states, ics):
            for x, y in zip((p.off, p.count, p.start, p.vel, p.acc), (q.off, q.count, q.start, q.vel, q.acc)):
                x.copy_(y, non_blocking=True)

    def timed(ens, k, clocks=None):
        for _ in range(args.warmup):
            reset()
            ens.launch(stream)
        ens.check(stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        if clocks:
            clocks.start()
        ranks.barrier()
        torch.cuda.synchronize()
        for e0, e1 in evs:
            reset()
            e0.record(stream)
            ens.launch(stream)
            e1.record(stream)
        torch.cuda.synchronize()
        ranks.barrier()
        clk = clocks.stop() if clocks else None
        ens.check(stream)
        return sum(e0.elapsed_time(e1) for e0, e1 in evs), clk

    t0 = time.perf_counter()
    reset()
    best, tune_ms = cube2.ensemble_autotune(ctxs, states, sched, trials=2, stream=stream,
                                            start=cube2.ensemble_opts(n_streams=args.streams, persistent_pp=True,
                                                                      pp_ctas_per_sm=8))
    tune_s = time.perf_counter() - t0
    ens = cube2.Ensemble(ctxs, states, sched, opts=best)
    kernels, psteps = ens.info()
    ms, clk = timed(ens, args.steps, ClockSampler(bus_id_of(torch.cuda.current_device())))
    ens.close()
    for c in ctxs:
        c.check()
    # the same work as per-box launches on concurrent graph branches
    ens_b = cube2.Ensemble(ctxs, states, sched, opts=cube2.ensemble_opts(n_streams=args.streams))
    kernels_b, _ = ens_b.info()
    ms_b, _ = timed(ens_b, args.steps)
    ens_b.close()
    ms_max = ranks.max(ms)
    units = ranks.sum(psteps * args.steps)
    value = job_throughput(units, ms_max / 1e3)
    value_b = job_throughput(units, ranks.max(ms_b) / 1e3)
    if rank == 0:
        line = {
            "metric": "ensemble particle-steps/sec (64 independent boxes x 20 KDK steps, one CUDA graph)",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Zel'dovich ICs, BBKS spectrum)",
            "config": {"workload": ENSEMBLE, "boxes": len(ws), "boxes_this_rank": len(mine),
                       "particles": int(sum(w.n_particles for w in ws)), "kdk_steps_per_box": ws[0].n_steps,
                       "recording": "step by step: boxes' steps up to their PP inputs on LPT-placed graph branches, "
                                    "then one persistent PP kernel over all boxes (cost-ordered device queue)",
                       "autotuned": {"n_streams": best.n_streams, "pp_ctas_per_sm": best.pp_ctas_per_sm,
                                     "pp_wmax": best.pp_wmax, "tuning_s": tune_s, "tuned_ms": tune_ms},
                       "step": "one graph launch = every box's 20 steps; states reset to the ICs before each",
                       "l2": "inputs larger than L2 (~1 GB of particles and meshes)", "parallelism": "boxes split over ranks"},
            "per_box_graph": {"value": value_b, "unit": UNIT, "ms_per_launch": ms_b / args.steps,
                              "kernel_nodes": kernels_b, "n_streams": args.streams,
                              "what": "the same steps as each box's own launches on concurrent graph branches"},
            "gpu_launches": kernels * args.steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


ADJOINT = "c3-adjoint-128c-256mesh"


def adjoint_measure(reps, warmup, breakdown=True):
    """Adjoint/forward time ratio on the differentiation workload (128^3
    particles, one 256^3 level, 10 KDK steps z = 9 -> 0): forward = the 10
    steps plus the final density loss; adjoint = the same steps with a
    checkpoint and re-bin map per step, the loss gradient, and the reverse
    sweep (one force product per step), giving dL/dx0 and dL/dv0.  The target
    is the final overdensity of an independent realisation (seed 4).  Wall
    clock with a device synchronisation on both sides, median per repetition.
    Runs on the current device; returns a dict."""
    import torch
    from inputs.workloads import WORKLOADS
    from inputs.zeldovich import zeldovich_ios
    from paper_2512_12629_gb300 import cube2
    w = WORKLOADS["pm1-128c-256mesh"]
    a = w.scale_factors()
    st = zeldovich_ios(w)
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    ctx.set_green(0)
    ctx.adjoint_init()
    pt = cube2.IOSState.from_numpy(zeldovich_ios(w.with_(seed=4)))
    ctx.force(pt)
    for k in range(len(a) - 1):
        ctx.kdk_step(pt, a[k], a[k + 1])
    ctx.deposit(0, pt)
    target = ctx.get_density(0).clone()
    p0 = cube2.IOSState.from_numpy(st)
    ctx.force(p0)
    torch.cuda.synchronize()

    def forward():
        p = p0.clone()
        for k in range(len(a) - 1):
            ctx.kdk_step(p, a[k], a[k + 1])
        return ctx.density_mse_vjp(0, p, target)[0]

    def adjoint():
        return cube2.loss_gradient(ctx, p0, target, a)

    for _ in range(max(1, warmup)):
        forward()
        adjoint()
    tf, ta = [], []
    for _ in range(max(1, reps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = forward()
        torch.cuda.synchronize()
        tf.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        loss_a, gx, gv = adjoint()
        torch.cuda.synchronize()
        ta.append(time.perf_counter() - t0)
    ctx.check()
    fwd, adj = statistics.median(tf), statistics.median(ta)
    out = {"ratio": adj / fwd, "forward_ms": 1e3 * fwd, "adjoint_ms": 1e3 * adj, "loss": loss,
           "loss_in_adjoint_run": loss_a, "grad_x_rms": float(gx.pow(2).mean().sqrt()),
           "grad_v_rms": float(gv.pow(2).mean().sqrt()), "particles": n_part, "mesh": 256, "kdk_steps": len(a) - 1,
           "z": f"{w.z_init:g} -> {w.z_final:g}", "repetitions": len(tf),
           "timing": "median wall clock per repetition, synchronised"}
    if breakdown:
        # per-class kernel time of one more repetition of each, CUDA events, outside the timing
        bd = {}
        for name, fn in (("forward", forward), ("adjoint", adjoint)):
            ctx.profile(capacity=5000)
            fn()
            prof = ctx.profile_read()
            ctx.profile(0)
            bd[name] = {f"{c}/{l}": round(ms, 3) for (c, l), (ms, _n) in sorted(prof.items(), key=lambda kv: -kv[1][0])}
        out["kernels_ms_per_repetition"] = bd
    ctx.close()
    return out


def run_adjoint(args):
    """The differentiation workload alone (see adjoint_measure)."""
    import torch
    world, rank, _ = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(0)
    from paper_2512_12629_gb300 import build as pkg_build
    pkg_build.build()
    r = adjoint_measure(args.steps, args.warmup)
    line = {
        "metric": "adjoint/forward time ratio (128^3 particles, 256^3 mesh, 10 KDK steps, density MSE loss)",
        "value": r["ratio"], "unit": "ratio", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "forward_ms": r["forward_ms"], "adjoint_ms": r["adjoint_ms"], "loss": r["loss"],
        "loss_in_adjoint_run": r["loss_in_adjoint_run"], "grad_x_rms": r["grad_x_rms"], "grad_v_rms": r["grad_v_rms"],
        "kernels_ms_per_repetition": r.get("kernels_ms_per_repetition"), "dtype": "f32",
        "data": "synthetic (seeded Zel'dovich ICs, BBKS spectrum; target = seed 4 final overdensity)",
        "config": {"workload": ADJOINT, "particles": r["particles"], "mesh": 256, "kdk_steps": r["kdk_steps"],
                   "z": r["z"], "gradient": "dL/dx0 and dL/dv0", "timing": r["timing"]},
    }
    print(json.dumps(line), flush=True)


LARGE = "c5-force-1024c-512x2048mesh"


def run_large(args):
    """One force evaluation of the large workload (1024^3 particles, 512^3 +
    2048^3 meshes, 1024^3 IOS cells, Zel'dovich displacement to z = 0, initial
    conditions from the device generator): W warm-up and K timed evaluations,
    CUDA events on the library's stream, with the per-class profile."""
    import torch
    from inputs.workloads import WORKLOADS
    from inputs.zeldovich_gpu import zeldovich_ios_torch
    world, rank, _ = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(0)
    from paper_2512_12629_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2512_12629_gb300 import cube2
    w = WORKLOADS["pm2-1024c-512x2048mesh"]
    st = zeldovich_ios_torch(w)
    torch.cuda.empty_cache()
    n_part = w.n_particles
    p = cube2.IOSState(st["off"], st["count"], st["start"], torch.zeros((3, 1), device="cuda"),
                       torch.zeros((3, n_part), device="cuda"))
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    t0 = time.perf_counter()
    for l in range(len(w.levels)):
        ctx.set_green(l)
    torch.cuda.synchronize()
    green_s = time.perf_counter() - t0
    for _ in range(max(1, args.warmup)):
        ctx.force(p)
    ctx.check()
    torch.cuda.synchronize()
    stream = ctx.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(capacity=64 * (args.steps + 2))
    launches0 = ctx.launch_count()
    clocks = ClockSampler(bus_id_of(torch.cuda.current_device()))
    clocks.start()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.force(p)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    ctx.profile(0)
    ctx.check()
    launches = ctx.launch_count() - launches0
    # PP work of the same evaluation, counted in an untimed pass (counting costs PP time)
    ctx.pp_count(True)
    ctx.pp_stats()
    ctx.force(p)
    pairs, cands = (v * args.steps for v in ctx.pp_stats())
    ctx.pp_count(False)
    total_prof = sum(v[0] for v in prof.values())
    kernels = {f"{c}/{l}": {"share": v[0] / total_prof, "ms_per_launch": v[0] / v[1], "launches": v[1]}
               for (c, l), v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    (cls, lvl), (dms, dcount) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_ms = dms / dcount
    if cls == "pp":
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        fpk, sms = measure_fp32_peak(cube2, torch)
        roofline = pp_roofline(pairs, cands, dcount, per_launch_ms, fpk, sms, mhz)
    else:
        peak, kind = peaks()
        alg = algorithmic_bytes(w, n_part, cls, lvl)
        achieved = alg / (per_launch_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"{cls}[level {lvl}]", "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "peak_source": kind,
                    "algorithmic_bytes_per_launch": alg, "mean_launch_ms": per_launch_ms, "traffic": None}
    line = {
        "metric": "particle-force evaluations/sec (1024^3 particles, 512^3 + 2048^3 meshes, PM + PP)",
        "value": n_part * args.steps / (ms / 1e3), "unit": "particle-forces/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (device-generated Zel'dovich displacement to z = 0, BBKS spectrum)",
        "config": {"workload": LARGE, "particles": n_part, "meshes": [lv.n_mesh for lv in w.levels],
                   "ios_cells": w.n_ios, "step": "one force evaluation (deposit, two solves, interp, PP)",
                   "l2": "inputs larger than L2", "green_tables_s": green_s},
        "roofline": roofline, "gpu_launches": launches, "clocks": clk, "kernels": kernels,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.workload == LARGE:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the large workload has no oracle arm (host memory)"}))
            return
        run_large(args)
        return
    if args.workload == ADJOINT:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the adjoint workload has no oracle arm"}))
            return
        run_adjoint(args)
        return
    if args.workload == ENSEMBLE:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the ensemble workload has no oracle arm"}))
            return
        run_ensemble(args)
        return
    from inputs.workloads import WORKLOADS
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
        return
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    ranks = Ranks(dist, "cuda")
    from paper_2512_12629_gb300 import build as pkg_build
    if rank == 0:
        pkg_build.build()
    ranks.barrier()
    pkg_build.build()
    from inputs.zeldovich import zeldovich_ios
    from paper_2512_12629_gb300 import cube2

    w = replica_workload(w, rank)
    st = zeldovich_ios(w)
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    for l in range(len(w.levels)):
        ctx.set_green(l)
    if w.pm3 is not None:
        ctx.set_green(cube2.LEVEL_PM3)
    p0 = cube2.IOSState.from_numpy(st)
    ctx.force(p0)
    p = p0.clone()
    a = w.scale_factors()
    S = w.n_steps
    idx = sampled_steps(S, args.steps)
    stream = ctx.stream

    def load(dst, src):
        for x, y in zip((dst.off, dst.count, dst.start, dst.vel, dst.acc),
                        (src.off, src.count, src.start, src.vel, src.acc)):
            x.copy_(y)

    # warm-up: W steps from the initial conditions
    for k in range(args.warmup):
        i = k % S
        ctx.kdk_step(p, a[i], a[i + 1])
    ctx.check()
    # the whole schedule from the initial conditions (untimed for the headline):
    # per-step CUDA events and the states the timed steps start from
    load(p, p0)
    ckpt = {}
    sched_ms, sched_pm3 = [], []
    for i in range(S):
        if i in idx:
            ckpt[i] = p.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.kdk_step(p, a[i], a[i + 1])
        e1.record(stream)
        e1.synchronize()
        sched_ms.append(e0.elapsed_time(e1))
        if w.pm3 is not None:
            sched_pm3.append(ctx.pm3_stats()[0])
    ctx.check()
    # the same schedule again with the PP work counters on (they cost PP time,
    # so no timed pass counts): pairs and candidates of every step
    load(p, p0)
    sched_pairs, sched_cands = [], []
    ctx.pp_count(True)
    ctx.pp_stats()
    for i in range(S):
        ctx.kdk_step(p, a[i], a[i + 1])
        pc = ctx.pp_stats()
        sched_pairs.append(pc[0])
        sched_cands.append(pc[1])
    ctx.pp_count(False)
    ctx.check()
    torch.cuda.synchronize()

    # timed region: K steps, each from its checkpoint (the restore is outside the event pair)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in idx]
    ctx.profile(capacity=64 * (args.steps + 2))
    launches = 0
    clocks = ClockSampler(bus_id_of(torch.cuda.current_device()))
    clocks.start()
    ranks.barrier()
    torch.cuda.synchronize()
    for (e0, e1), i in zip(evs, idx):
        load(p, ckpt[i])
        l0 = ctx.launch_count()
        e0.record(stream)
        ctx.kdk_step(p, a[i], a[i + 1])
        e1.record(stream)
        launches += ctx.launch_count() - l0
    torch.cuda.synchronize()
    ranks.barrier()
    clk = clocks.stop()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    prof = ctx.profile_read()
    ctx.profile(0)
    ctx.check()
    # the timed steps repeat schedule steps from their checkpoints (bitwise)
    pp_pairs = sum(sched_pairs[i] for i in idx)
    pp_cands = sum(sched_cands[i] for i in idx)
    ms_max = ranks.max(ms)
    units = ranks.sum(n_part * args.steps)
    value = job_throughput(units, ms_max / 1e3)

    # dominant kernel class -> roofline (PP counts both of its kernels)
    peak, peak_kind = peaks()
    total_prof = sum(v[0] for v in prof.values())
    # the roofline is taken for the dominant class with an algorithmic figure
    # (the third level's classes move data-dependent amounts); the overall
    # dominant class is named beside it
    (top_cls, top_lvl), (top_ms, _) = max(prof.items(), key=lambda kv: kv[1][0])
    rated = {k: v for k, v in prof.items() if k[0] == "pp" or algorithmic_bytes(w, n_part, k[0], k[1]) is not None}
    (cls, lvl), (dms, dcount) = max(rated.items(), key=lambda kv: kv[1][0])
    per_launch_ms = dms / dcount
    kname = f"{cls}[level {lvl}]" if cls.startswith("fft") else cls
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    fpk, sms = measure_fp32_peak(cube2, torch)
    if cls == "pp":
        roofline = pp_roofline(pp_pairs, pp_cands, dcount, per_launch_ms, fpk, sms, mhz, traffic_record("pp"))
    else:
        alg = algorithmic_bytes(w, n_part, cls, lvl)
        achieved = alg / (per_launch_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": alg, "mean_launch_ms": per_launch_ms,
                    "traffic": traffic_record(cls)}
    roofline["dominant_class_overall"] = {"class": f"{top_cls}/{top_lvl}", "share": top_ms / total_prof}
    kernels = {}
    for (c, l), (kms, kc) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        b = algorithmic_bytes(w, n_part, c, l)
        gbps = None if b is None else b / (kms / kc / 1e3) / 1e9
        kernels[f"{c}/{l}"] = {"share": kms / total_prof, "ms_per_launch": kms / kc, "launches": kc,
                               "GBps_alg": gbps, "frac_hbm": None if gbps is None else gbps / peak}
    kernels["pp_work"] = {"pairs_per_step": pp_pairs / args.steps, "candidates_per_step": pp_cands / args.steps}
    if sched_pm3:
        full_pm3 = {"refined_subtiles_each": sched_pm3, "subtile_ios_cells": w.pm3.tile,
                    "rho_min": w.pm3.rho_min, "refine": w.pm3.refine, "beta3": w.pm3.beta}
    else:
        full_pm3 = None
    full = {"steps": S, "pm3": full_pm3, "ms_per_step": sum(sched_ms) / S, "value": n_part * S / (sum(sched_ms) / 1e3),
            "ms_first_last_10": [sum(sched_ms[:10]) / 10, sum(sched_ms[-10:]) / 10],
            "pp_pairs_first_last_step": [sched_pairs[0], sched_pairs[-1]],
            "ms_per_step_each": [round(x, 3) for x in sched_ms],
            "pp_pairs_each": sched_pairs,
            "what": "the whole schedule from the initial conditions, per-step CUDA events (untimed run)"}

    # end to end through the host-buffer entry point, on the same steps
    e2e = None
    if not args.no_e2e:
        cpus_before = os.sched_getaffinity(0)
        numa = bind_local_numa(bus_id_of(torch.cuda.current_device()))
        host = cube2.IOSState(*(x.cpu().pin_memory() for x in (p0.off, p0.count, p0.start, p0.vel, p0.acc)))
        pe = p0.clone()
        bytes_down = sum(x.numel() * x.element_size() for x in (host.off, host.count, host.start, host.vel, host.acc))
        bytes_up = bytes_down - host.start.numel() * host.start.element_size()   # start is formed on the device
        ctx.kdk_step_host(pe, host, a[0], a[1])                # warm
        el = 0.0
        ranks.barrier()
        for i in idx:
            load(host, ckpt[i])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.kdk_step_host(pe, host, a[i], a[i + 1])
            el += time.perf_counter() - t0
        el = ranks.max(el)
        os.sched_setaffinity(0, cpus_before)
        e2e = {"value": job_throughput(units, el), "unit": UNIT,
               "h2d_bytes_per_step": bytes_up, "d2h_bytes_per_step": bytes_down,
               "api": "cube2_kdk_step_host (pinned host state, H2D + step + D2H each step), the same steps",
               "host_numa_node": numa}
    del ckpt

    # cuFFT (through torch.fft), timed only as a comparison with the library's own
    # FFT passes of the finest level: r2c + c2r of the same n^3 FP32 grid
    cufft = None
    adjoint = None
    if rank == 0:
        nf = w.levels[-1].n_mesh
        own = sum(kms / kc for (c, l), (kms, kc) in prof.items() if c.startswith("fft_") and l == len(w.levels) - 1)
        grid = torch.randn((nf, nf, nf), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
        for _ in range(2):
            torch.fft.irfftn(torch.fft.rfftn(grid), s=grid.shape)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            torch.fft.irfftn(torch.fft.rfftn(grid), s=grid.shape)
        e1.record()
        torch.cuda.synchronize()
        cufft = {"n": nf, "torch_cufft_r2c_c2r_ms": e0.elapsed_time(e1) / reps, "own_fft_passes_ms": own,
                 "note": "own passes include the Green's multiply (fused into the z pass); cuFFT is not on the path"}
        del grid
        if not args.no_adjoint:
            adjoint = adjoint_measure(5, 3, breakdown=False)
            adjoint["workload"] = ADJOINT

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t = oracle_timing(w, sampled_steps(w.n_steps, min(args.steps, 6)))
        cpu = {"value": t["value"], "unit": UNIT, "cores": t["cores"], "kind": "oracle", "sample": t["sample"],
               "cpu_model": t["cpu_model"], "single_core_value": t["single_core_value"], "seconds": t["seconds"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Zel'dovich ICs, BBKS spectrum)", "config": workload_config(w, idx),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "full_schedule": full, "adjoint": adjoint, "kernels": kernels,
            "cufft_comparison": cufft,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
