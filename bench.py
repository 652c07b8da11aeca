#!/usr/bin/env python
"""Benchmark of the Spectral Quadrature hot path on one GB300 (or N replicas).

One step = one SCF-iteration's worth of the path on the whole grid:
  sq_spectral_bounds (Lanczos) -> sq_moments (Chebyshev recurrence) ->
  sq_fermi_level (weights + bisection) -> sq_density_energy.
Metric: node-moments/s = N_d * n_pl / (seconds per step), whole job.

Workload (default): the scale case, 8x8x8 FCC cells (2048 atoms), 128^3 grid
(2.1M nodes), h = 0.478125 bohr, R_cut = 7 bohr (29^3 regions), n_pl = 64,
kT = 0.1 Ha, s + 3p Gaussian KB projectors, 6144 electrons, FP32 recurrence
with FP64 moments; synthetic, seeded inputs.  The line also carries the FP64
form against the FP32 form on the 3x3x3-cell workload (al108_48, 25^3 regions;
FP64 regions above 25^3 do not fit one CTA): both step times and the FP32
error against the FP64 result.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
                  [--workload al108_48|al2048_128|...] [--impl reference]
  python bench.py --workload batch16          (16 uneven systems as one CUDA graph;
                                               --batch-plan auto|streams|share|queue, --nodes-per-item k)
  python bench.py --workload force_al108_48   (nonlocal atomic forces; --precision fp32|fp64)
  python bench.py --workload scf_al256_64     (SCF to 1e-6: Kerker-preconditioned Anderson mixing,
                                               FP32 then FP64 from --refine-at 1e-5; --reuse-bounds w,
                                               --fresh-below r)
  python bench.py --workload warmstart_c4     (train the warm-start network, then SCF
                                               iterations to 1e-6 on al256_64 with and without it)
  python bench.py --n-lanczos K --margin M    (ablation of the bounds' cost; --save-rho path)

Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (the path has no data exchange between replicas); the JSON line
reports the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "al2048_128"
METRIC = "node-moments/s (nodes x Chebyshev degree per second, whole SCF-iteration step)"
UNIT = "node-moments/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_PATH = os.path.join(ROOT, "profiles", "roofline_counters.json")
FP32_LANES_PER_SM = 128        # FP32 FMA lanes per SM per clock (Blackwell)
SM_COUNT_GB300 = 152


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--cpu-sample", type=int, default=0, help="oracle sample size (nodes); 0 = automatic")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-context", action="store_true", help="skip the FP64-vs-FP32 comparison on al108_48")
    p.add_argument("--n-lanczos", type=int, default=0,
                   help="override the workload's Lanczos step count (an ablation; 0: the workload's)")
    p.add_argument("--margin", type=float, default=0.0,
                   help="with --n-lanczos: the bounds' relative widening (0: the workload's)")
    p.add_argument("--save-rho", default="", help="write the last step's density (float32 .npy) to this path")
    p.add_argument("--fresh-below", default="none",
                   help="scf_*, warmstart_c4: residual below which bounds are no longer reused (none: reuse to the end)")
    p.add_argument("--refine-at", default="1e-5",
                   help="scf_*, warmstart_c4: residual at which an FP64 context takes over (none: FP32 throughout)")
    p.add_argument("--batch-plan", choices=["auto", "streams", "share", "queue"], default="auto",
                   help="batch16: launch plan (auto: the autotuner times them and keeps the fastest)")
    p.add_argument("--nodes-per-item", type=int, default=1, help="batch16 with --batch-plan queue: nodes per work item")
    p.add_argument("--train-geometries", type=int, default=250, help="warmstart_c4: seeded training geometries")
    p.add_argument("--train-iters", type=int, default=8, help="warmstart_c4: SCF iterations kept per geometry")
    p.add_argument("--train-steps", type=int, default=1000, help="warmstart_c4: Adam steps")
    p.add_argument("--max-scf", type=int, default=80, help="warmstart_c4, scf_*: SCF iteration limit")
    p.add_argument("--kerker", default="0.5,0.1", help="scf_*: k0,amin of the preconditioner, or 'none'")
    p.add_argument("--history", type=int, default=16, help="scf_*: mixing history")
    p.add_argument("--beta", type=float, default=0.3, help="scf_*: mixing parameter")
    p.add_argument("--period", type=int, default=1, help="scf_*: Pulay period (1: Anderson every step)")
    p.add_argument("--reuse-bounds", default="none",
                   help="scf_*: w_max (Ha) -- reuse the last Lanczos bounds, widened by max|V - V_ref| <= w_max")
    return p.parse_args()


# --------------------------------------------------------------------------
# algorithmic work per unit (flops), used for the roofline
# --------------------------------------------------------------------------
LOCAL_FLOPS_RECUR = 52    # per region point per Chebyshev step (stencil, diagonal, update, two dots)
LOCAL_FLOPS_LANCZOS = 56  # per region point per Lanczos step (stencil, diagonal, -beta v_old, alpha, w-alpha v, |w|^2, scale)
# per (region point, atom support) pair per step, for the plain evaluation of the
# nonlocal term: 4 projectors (s, p_x, p_y, p_z), each one multiply-add in its
# inner product and one in its update (2 + 2 flops); about 55 flops per point at
# the FCC-Al atom density.  The kernels evaluate the projectors separably and do
# fewer, so this is the algorithmic count the roofline fraction is taken against.
NL_FLOPS_PER_PAIR = 16


def nl_pairs_per_point(wl):
    """Mean number of atom supports covering a grid point."""
    if not wl.nonlocal_:
        return 0.0
    return wl.n_atoms / wl.L ** 3 * (4.0 / 3.0) * math.pi * synth.PROJ_RNL ** 3


def flops_moments(wl):
    S = 2 * wl.m + 1
    per_point = LOCAL_FLOPS_RECUR + NL_FLOPS_PER_PAIR * nl_pairs_per_point(wl)
    return wl.n_nodes * (wl.npl // 2) * S ** 3 * per_point


def flops_lanczos(wl):
    S = 2 * wl.m + 1
    per_point = LOCAL_FLOPS_LANCZOS + NL_FLOPS_PER_PAIR * nl_pairs_per_point(wl)
    return wl.n_nodes * wl.n_lanczos * S ** 3 * per_point


# the sources that define the region kernels (their counters are recorded
# against this hash, so any change to these files voids them)
KERNEL_SOURCES = ("sq_internal.cuh", "sq_region.cuh", "sq_region_dispatch.cuh", "sq_region_f32.cu",
                  "sq_region_f64.cu")


def source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1708_07913_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------
# clocks sampling (nvidia-smi) during the timed region
# --------------------------------------------------------------------------
SMI_FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            # raw samples go to the temp directory; the JSON line carries their summary
            self.path = os.path.join(tempfile.gettempdir(), f"sq_bench_clocks_gpu{self.gpu}_{os.getpid()}.csv")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(SMI_FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < len(SMI_FIELDS):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same workload)
# --------------------------------------------------------------------------
_W = {}


def _oracle_init(name):
    import oracle
    s = synth.make_system(name)
    _W["wl"] = s.wl
    _W["osys"] = oracle.OracleSystem.from_synth(s)


def _oracle_chunk(nodes):
    wl, osys = _W["wl"], _W["osys"]
    t0 = time.perf_counter()
    chi, zeta = osys.bounds(nodes, wl.n_lanczos, wl.margin)
    osys.moments(nodes, chi, zeta, wl.npl)
    return time.perf_counter() - t0


class OraclePool:
    """Spawned worker processes, each holding the workload in oracle form."""

    def __init__(self, name, cores):
        import multiprocessing as mp
        import oracle
        oracle.build()
        self.name, self.cores = name, cores
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(name,))

    def rate(self, sample, seed=1234):
        """node-moments/s of the oracle (bounds + moments, >99% of its per-step
        cost) on a seeded node sample split over the workers; the slowest
        worker's own compute time is the step time."""
        wl = synth.WORKLOADS[self.name]
        nodes = synth.sample_nodes(wl.n_nodes, sample, seed=seed)
        chunks = [c for c in np.array_split(nodes, self.cores) if len(c)]
        t = max(self.pool.map(_oracle_chunk, chunks))
        return len(nodes) * wl.npl / t, t, len(chunks)

    def close(self):
        self.pool.close()
        self.pool.join()


def workload_desc(name, wl):
    """The config.workload string of both arms."""
    return (f"{name}: {wl.cells}^3 FCC cells ({wl.n_atoms} atoms), {wl.n}^3 grid (h={wl.h:.6f}), "
            f"{2 * wl.m + 1}^3 regions (R_cut={wl.r_cut}), n_pl={wl.npl}, kT={wl.kT}, "
            f"{'s+3p KB projectors' if wl.nonlocal_ else 'local potential only'}, {int(wl.n_electrons)} electrons")


def oracle_rates(name, cores, sample, seed=1234):
    """(all-core rate, its seconds, processes used, serial rate, serial sample,
    serial seconds): node-moments/s of the oracle on a seeded node sample of the
    workload, spread over `cores` spawned processes, and on one process over a
    smaller sample."""
    pool = OraclePool(name, cores)
    rate, t, used = pool.rate(sample, seed=seed)
    pool.close()
    ser_n = max(1, min(sample // max(1, cores), 64))
    one = OraclePool(name, 1)
    srate, st, _ = one.rate(ser_n, seed=seed + 1)
    one.close()
    return rate, t, used, srate, ser_n, st


def auto_sample(name, cores, target_s=15.0):
    """Sample size for ~target_s seconds of oracle work per worker."""
    per_node = {"al4_16": 0.005, "al108_48": 0.08, "al2048_128": 0.15}.get(name, 0.1)
    return max(cores, min(int(target_s / per_node) * cores, synth.WORKLOADS[name].n_nodes))


# --------------------------------------------------------------------------
def run_reference(a):
    """The oracle as it stands, timed on the host cores, same metric and unit.
    Each step is a seeded node sample of the workload (bounds + moments, >99 %
    of the oracle's per-step cost) spread over all host cores; ms_per_step is
    that sample's measured time, and the full-grid time it extrapolates to is
    reported separately."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = synth.WORKLOADS[a.workload]
    cores = os.cpu_count() or 1
    per_node = {"al4_16": 0.005, "al108_48": 0.08, "al2048_128": 0.15}.get(a.workload, 0.15)
    sample = a.cpu_sample or max(cores, int(4.0 / per_node) * cores)
    sample = min(sample, wl.n_nodes)
    pool = OraclePool(a.workload, cores)
    rates = []
    for i in range(a.warmup + a.steps):
        r, t, used = pool.rate(sample, seed=1234 + i)
        if i >= a.warmup:
            rates.append((r, t))
    pool.close()
    ser_n = max(1, min(sample // cores, 64))
    one = OraclePool(a.workload, 1)
    srate, st, _ = one.rate(ser_n, seed=999)
    one.close()
    value = statistics.median(r for r, _ in rates)
    t_sample = statistics.median(t for _, t in rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_sample * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded FCC Al-like crystal, Gaussian V and KB projectors)",
        "config": {"workload": workload_desc(a.workload, wl), "sample_nodes_per_step": sample,
                   "step": f"{sample} seeded nodes of the workload (Lanczos bounds + moments) on {used} processes"},
        "extrapolated_full_grid_ms": wl.n_nodes * wl.npl / value * 1e3,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{sample} seeded nodes per step (bounds + moments), per-node rate",
                         "serial": {"value": srate, "cores": 1, "sample": f"{ser_n} seeded nodes, {st:.1f} s"}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def replica_times(times, dist):
    """Each timing (seconds) maximised over the ranks (the slowest replica
    sets the job's time); unchanged on one rank (dist None)."""
    if dist is None:
        return [float(t) for t in times]
    import torch
    tt = torch.tensor([float(t) for t in times], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return [float(x) for x in tt]


def replica_value(units_per_rank, world, t_max):
    """Whole-job throughput: the units every rank processed over the
    slowest rank's time."""
    return units_per_rank * world / t_max


def run_gb300(a):
    import torch
    from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQSolver, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    build()
    prec = SQ_FP32 if a.precision == "fp32" else SQ_FP64
    s = synth.make_system(a.workload)
    wl = s.wl
    if a.n_lanczos > 0:                                    # ablation of the bounds' cost
        wl = dataclasses.replace(wl, n_lanczos=a.n_lanczos, margin=a.margin if a.margin > 0 else wl.margin)
    solver = SQSolver.from_workload(wl, s.positions, precision=prec, device=str(dev))
    Vh = torch.from_numpy(s.V.ravel().copy()).pin_memory()
    V = Vh.to(dev)
    rho_h = torch.empty(wl.n_nodes, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(timed=None):
        e = [ev() for _ in range(5)]
        e[0].record(stream)
        solver.bounds(V, wl.n_lanczos, wl.margin)
        e[1].record(stream)
        solver.compute_moments(V)
        e[2].record(stream)
        mu = solver.fermi_level(wl.n_electrons, wl.kT)
        e[3].record(stream)
        eb, es, ne = solver.density_energy(mu, wl.kT)
        e[4].record(stream)
        if timed is not None:
            timed.append(e)
        return mu, eb, es, ne

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = solver.launches
    timed = []
    for _ in range(a.steps):
        flush.fill_(1.0)                                   # evict L2 between steps (not timed)
        step(timed)
    torch.cuda.synchronize()
    launches = solver.launches - launches0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # end-to-end through host buffers: V from pinned host memory, rho and the
    # scalars back to the host, copies inside the timed region
    e2e_t = []
    for _ in range(max(1, a.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        V.copy_(Vh, non_blocking=True)
        step()
        rho_h.copy_(solver.rho, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    clk = clocks.stop()
    if a.save_rho:
        np.save(a.save_rho, rho_h.numpy().astype(np.float32))

    per = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in timed])   # ms
    step_ms = per.sum(axis=1)
    t_step = float(step_ms.mean()) / 1e3
    t_e2e = float(np.median(e2e_t))
    t_step, t_e2e = replica_times([t_step, t_e2e], dist)
    units = wl.n_nodes * wl.npl * world
    value = replica_value(wl.n_nodes * wl.npl, world, t_step)
    t_bounds, t_mom, t_fermi, t_dens = (float(x) / 1e3 for x in per.mean(axis=0))

    # roofline for the dominant kernel (FP32/FP64 CUDA-core pipe, "alu" bound)
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if prec == SQ_FP32:
        peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    else:
        peak = 1.25 * sms / SM_COUNT_GB300 * sm_max / 2070.0     # FP64 at GB300's published 1.25 TFLOP/s
    kern = {"lanczos_kernel": (flops_lanczos(wl), t_bounds), "moments_kernel": (flops_moments(wl), t_mom)}
    dom = max(kern, key=lambda k: kern[k][1])
    achieved = kern[dom][0] / kern[dom][1] / 1e12
    traffic = None
    if os.path.exists(PROFILE_PATH):
        prof = json.load(open(PROFILE_PATH))
        key = f"{dom}:{a.workload}:{a.precision}"
        if key in prof and prof[key].get("source_sha") == source_sha():
            traffic = prof[key].get("dram_bytes_per_launch")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == SQ_FP32 else "f64",
        "data": "synthetic (seeded FCC Al-like crystal, Gaussian V and KB projectors)",
        "config": {"workload": workload_desc(a.workload, wl),
                   "precision": ("FP32 recurrence/Lanczos vectors, FP64 moments, weights, Fermi level, energies"
                                 if prec == SQ_FP32 else "FP64 throughout"),
                   "n_lanczos": wl.n_lanczos, "margin": wl.margin,
                   "lanczos_override": a.n_lanczos > 0, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "breakdown_s": {"bounds": t_bounds, "moments": t_mom, "fermi": t_fermi, "density": t_dens},
        "moments_only_node_moments_per_s": wl.n_nodes * wl.npl * world / t_mom,
        "s_per_scf_iteration": t_step,
        "roofline": {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": (f"{'FP32' if prec == SQ_FP32 else 'FP64'} CUDA-core pipe at "
                                    f"{sm_max:.0f} MHz x {sms} SMs (derived from unit counts and clock)")},
        "e2e": {"value": units / t_e2e, "unit": UNIT, "h2d_bytes_per_step": wl.n_nodes * 8,
                "d2h_bytes_per_step": wl.n_nodes * 8 + 4 * 8},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sample = a.cpu_sample or auto_sample(a.workload, cores)
        try:
            rate, t, used, srate, ser_n, st = oracle_rates(a.workload, cores, sample)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                                    "sample": f"{sample} seeded nodes of {a.workload} (Lanczos bounds + moments, "
                                              f"{t:.1f} s on {used} processes), per-node rate",
                                    "serial": {"value": srate, "cores": 1,
                                               "sample": f"{ser_n} seeded nodes, {st:.1f} s on one process"}}
        except Exception as exc:   # the CPU leg must not hide the GPU result
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                                    "sample": f"failed: {exc}"}
    solver.close()
    if rank == 0 and world == 1 and prec == SQ_FP32 and not a.no_fp64_context:
        try:
            line["fp64_vs_fp32"] = fp64_context(dev, flush)
        except Exception as exc:   # context only: must not hide the main result
            line["fp64_vs_fp32"] = {"failed": str(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def fp64_context(dev, flush, name="al108_48"):
    """The whole step in FP64 and in FP32 on al108_48 (25^3 regions, the
    largest the FP64 form holds in one CTA): step seconds of each (FP32: one
    warm-up, then one timed step; FP64: one timed step, whose ~20 s dwarf any
    first-call cost), the speed-up, and the FP32 result's error against the
    FP64 one (density 2-norm and max-norm relative, energies per atom, Fermi
    level, electron count)."""
    import torch
    from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQSolver
    s = synth.make_system(name)
    wl = s.wl
    V = torch.from_numpy(s.V.ravel().copy()).to(dev)
    stream = torch.cuda.current_stream()
    res = {}
    for label, prec, warm in (("fp32", SQ_FP32, 1), ("fp64", SQ_FP64, 0)):
        sv = SQSolver.from_workload(wl, s.positions, precision=prec, device=str(dev))
        for _ in range(warm):
            sv.solve(V, wl.n_electrons, wl.kT, wl.n_lanczos, wl.margin)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = sv.solve(V, wl.n_electrons, wl.kT, wl.n_lanczos, wl.margin)
        e1.record(stream)
        torch.cuda.synchronize()
        res[label] = dict(s=e0.elapsed_time(e1) / 1e3, rho=out["rho"].cpu().numpy().copy(), mu=out["mu"],
                          e_band=out["e_band"], e_ent=out["e_ent"], n_elec=out["n_elec"])
        sv.close()
    f, d = res["fp32"], res["fp64"]
    return {
        "workload": workload_desc(name, wl),
        "fp64_step_s": d["s"], "fp32_step_s": f["s"], "speedup_fp32_over_fp64": d["s"] / f["s"],
        "fp64_node_moments_per_s": wl.n_nodes * wl.npl / d["s"], "fp32_node_moments_per_s": wl.n_nodes * wl.npl / f["s"],
        "fp32_error_vs_fp64": {
            "rho_rel_2norm": float(np.linalg.norm(f["rho"] - d["rho"]) / np.linalg.norm(d["rho"])),
            "rho_rel_max": float(np.abs(f["rho"] - d["rho"]).max() / d["rho"].max()),
            "e_band_ha_per_atom": abs(f["e_band"] - d["e_band"]) / wl.n_atoms,
            "e_ent_ha_per_atom": abs(f["e_ent"] - d["e_ent"]) / wl.n_atoms,
            "mu_ha": abs(f["mu"] - d["mu"]), "n_elec_abs": abs(f["n_elec"] - wl.n_electrons)},
        "timing": "one FP32 warm-up then one timed step; one timed FP64 step; L2 flushed before each",
    }


def run_batch(a):
    """16 uneven seeded systems (synth.batch_workloads) as one CUDA-graph
    launch per step (sq_batch_*), FP32; the same metric summed over the
    systems, and the same systems run one after another through the
    single-system calls for comparison."""
    import torch
    from paper_1708_07913_gb300 import SQ_FP32, SQBatch, SQSolver, build, sq

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    build()
    wls = synth.batch_workloads()
    systems = [synth.make_system(w) for w in wls]
    margin, n_lz = wls[0].margin, wls[0].n_lanczos
    Vh = [torch.from_numpy(s.V.ravel().copy()).pin_memory() for s in systems]
    Vs = [v.to(dev) for v in Vh]
    solvers = [SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP32, device=str(dev)) for s in systems]
    Ne, kT = [w.n_electrons for w in wls], [w.kT for w in wls]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # sequential reference: the single-system calls, one system after another
    def seq():
        for s, sv, V in zip(systems, solvers, Vs):
            sv.solve(V, s.wl.n_electrons, s.wl.kT, n_lz, margin)
    seq()
    flush.fill_(1.0)
    e0, e1 = ev(), ev()
    e0.record(stream)
    seq()
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    batch = SQBatch(solvers)
    plans = {"auto": sq.SQ_BATCH_AUTO, "streams": sq.SQ_BATCH_STREAMS, "share": sq.SQ_BATCH_STREAMS_SHARE,
             "queue": sq.SQ_BATCH_QUEUE}
    if a.batch_plan != "auto":
        batch.set_plan(plans[a.batch_plan], a.nodes_per_item)
    t0 = time.perf_counter()
    batch.run(Vs, Ne, kT, n_lz, margin)                      # first call: autotune + capture
    batch.results()
    t_tune = time.perf_counter() - t0
    for _ in range(a.warmup):
        batch.run(Vs, Ne, kT, n_lz, margin)
        batch.results()
    clocks = ClockSampler(0)
    clocks.start()
    times = []
    for _ in range(a.steps):
        flush.fill_(1.0)
        e0, e1 = ev(), ev()
        e0.record(stream)
        batch.run(Vs, Ne, kT, n_lz, margin)
        e1.record(stream)
        batch.results()
        times.append(e0.elapsed_time(e1) / 1e3)
    e2e = []
    for _ in range(max(2, a.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for v, vh in zip(Vs, Vh):
            v.copy_(vh, non_blocking=True)
        batch.run(Vs, Ne, kT, n_lz, margin)
        batch.results()
        rho_h = [sv.rho.to("cpu", non_blocking=True) for sv in solvers]
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    clk = clocks.stop()
    t = float(np.mean(times))
    units = sum(w.n_nodes * w.npl for w in wls)
    flops = sum(flops_moments(w) + flops_lanczos(w) for w in wls)
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    plan, npi = batch.plan()
    plan_name = {v: k for k, v in plans.items()}[plan]
    # kernels per system in one graph: weights, Fermi-state init, bracket, two end counts and 201
    # bisection counts, density, tridiagonal extremes; per system potential copy, Lanczos and moments
    # (stream plans), or per group of systems with one region size a Lanczos and a moments queue kernel
    post = len(wls) * (1 + 1 + 1 + 2 + 201 + 1 + 1)
    if plan == sq.SQ_BATCH_QUEUE:
        n_groups = sum(-(-c // 8) for c in collections.Counter(w.m for w in wls).values())
        per_graph = post + 2 * n_groups
    else:
        per_graph = post + 3 * len(wls)
    line = {
        "metric": METRIC, "value": units / t, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (16 seeded FCC Al-like crystals, Gaussian V and KB projectors)",
        "config": {"workload": "batch16: " + "; ".join(
            f"{w.cells}^3 cells {w.n}^3 grid h={w.h:.3f} {2 * w.m + 1}^3 regions n_pl={w.npl} kT={w.kT:.3f}"
            for w in wls),
            "precision": "FP32 recurrence/Lanczos vectors, FP64 moments, weights, Fermi level, energies",
            "n_lanczos": n_lz, "margin": margin,
            "launch": ("one CUDA graph per step: persistent queue kernels per group of systems with one region "
                       f"size, {npi} node(s) per work item" if plan == sq.SQ_BATCH_QUEUE else
                       "one CUDA graph per step, one stream per system"),
            "plan": plan_name if a.batch_plan != "auto" else f"{plan_name} (autotuned)",
            "l2": "flushed between timed steps (256 MB write)", "parallelism": "single GPU"},
        "sequential_s": t_seq, "batch_speedup_vs_sequential": t_seq / t, "autotune_first_call_s": t_tune,
        "blocks_per_system": batch.blocks(),
        "roofline": {"kernel": "all region kernels of the batch", "bound": "alu", "achieved": flops / t / 1e12,
                     "peak": peak, "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak, "traffic": None,
                     "peak_basis": f"FP32 CUDA-core pipe at {sm_max:.0f} MHz x {sms} SMs"},
        "e2e": {"value": units / float(np.median(e2e)), "unit": UNIT,
                "h2d_bytes_per_step": sum(w.n_nodes * 8 for w in wls),
                "d2h_bytes_per_step": sum(w.n_nodes * 8 + 4 * 8 for w in wls)},
        "gpu_launches": per_graph * a.steps,
        "graph_launches": a.steps,
        "clocks": clk,
        "cpu_baseline": {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                         "sample": "not timed for the batch (see the single-workload line)"},
    }
    batch.close()
    for sv in solvers:
        sv.close()
    print(json.dumps(line), flush=True)


FORCE_METRIC = "force node-steps/s (nodes inside a projector support x n_pl per second, one force evaluation)"
FORCE_UNIT = "node-steps/s"
FORCE_FLOPS_PER_POINT = 50   # per region point per step: stencil, diagonal, shift/scale, three-term update, D update


def touched_nodes(wl, positions):
    """Nodes inside some projector support (|x - R - image| < r_nl): the
    nodes the force visits."""
    n, h, rnl = wl.n, wl.h, synth.PROJ_RNL
    mark = np.zeros((n, n, n), dtype=bool)
    for R in positions:
        lo = [int(math.ceil((R[d] - rnl) / h)) for d in range(3)]
        hi = [int(math.floor((R[d] + rnl) / h)) for d in range(3)]
        g = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
        dx = [g[d] * h - R[d] for d in range(3)]
        inside = (dx[2][:, None, None] ** 2 + dx[1][None, :, None] ** 2 + dx[0][None, None, :] ** 2) < rnl * rnl
        iz, iy, ix = np.nonzero(inside)
        mark[np.mod(g[2][iz], n), np.mod(g[1][iy], n), np.mod(g[0][ix], n)] = True
    return int(mark.sum())


def _oracle_force_chunk(nodes):
    wl, osys = _W["wl"], _W["osys"]
    chi, zeta = osys.bounds(nodes, wl.n_lanczos, wl.margin)
    t0 = time.perf_counter()
    osys.nl_force(nodes, chi, zeta, wl.npl, float(np.median(chi)), wl.kT)
    return time.perf_counter() - t0


def run_force(a):
    """Nonlocal atomic forces (sq_nl_forces; recurrence in the --precision
    given, FP32 by default) on the workload named after ``force_``, with the
    spectral bounds and Fermi level of one SQ step computed first (not
    timed).  One step = one force evaluation."""
    import torch
    from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQSolver, build

    name = a.workload[len("force_"):]
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    build()
    s = synth.make_system(name)
    wl = s.wl
    prec = SQ_FP32 if a.precision == "fp32" else SQ_FP64
    solver = SQSolver.from_workload(wl, s.positions, precision=prec, device=str(dev))
    Vh = torch.from_numpy(s.V.ravel().copy()).pin_memory()
    V = Vh.to(dev)
    out = solver.solve(V, wl.n_electrons, wl.kT, wl.n_lanczos, wl.margin)
    mu = out["mu"]
    chi_h, zeta_h = solver.chi.cpu().pin_memory(), solver.zeta.cpu().pin_memory()
    F_h = torch.empty(wl.n_atoms * 3, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(a.warmup):
        solver.nl_forces(V, mu, wl.kT)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = solver.launches
    times = []
    for _ in range(a.steps):
        flush.fill_(1.0)
        e0, e1 = ev(), ev()
        e0.record(stream)
        F = solver.nl_forces(V, mu, wl.kT)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    launches = solver.launches - launches0
    e2e = []
    for _ in range(max(2, a.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        V.copy_(Vh, non_blocking=True)
        solver.chi.copy_(chi_h, non_blocking=True)
        solver.zeta.copy_(zeta_h, non_blocking=True)
        F = solver.nl_forces(V, mu, wl.kT)
        F_h.copy_(F.reshape(-1), non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    clk = clocks.stop()
    t = float(np.mean(times))
    nt = touched_nodes(wl, s.positions)
    S = 2 * wl.m + 1
    units = nt * wl.npl
    flops = nt * wl.npl * S ** 3 * (FORCE_FLOPS_PER_POINT + NL_FLOPS_PER_PAIR * nl_pairs_per_point(wl))
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if prec == SQ_FP32:
        peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        basis = f"FP32 CUDA-core pipe at {sm_max:.0f} MHz x {sms} SMs (derived from unit counts and clock)"
    else:
        peak = 1.25 * sms / SM_COUNT_GB300 * sm_max / 2070.0
        basis = f"FP64 at GB300's published 1.25 TFLOP/s scaled to {sm_max:.0f} MHz x {sms} SMs"
    line = {
        "metric": FORCE_METRIC, "value": units / t, "unit": FORCE_UNIT, "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == SQ_FP32 else "f64",
        "data": "synthetic (seeded FCC Al-like crystal, Gaussian V and KB projectors)",
        "config": {"workload": f"{a.workload}: nonlocal forces on {name} ({wl.n_atoms} atoms, {wl.n}^3 grid, "
                               f"{S}^3 regions, n_pl={wl.npl}, kT={wl.kT}); {nt} of {wl.n_nodes} nodes inside "
                               f"a projector support",
                   "precision": ("FP32 recurrence, D and projector sums; FP64 coefficients and contraction"
                                 if prec == SQ_FP32 else "FP64 throughout"),
                   "kernel": ("first form, current vector in shared memory (SQ_FORCE_KERNEL=legacy, SQ_FORCE_SMEM=1)"
                              if os.environ.get("SQ_FORCE_KERNEL") == "legacy" and os.environ.get("SQ_FORCE_SMEM") == "1"
                              else "first form, vectors in global scratch (SQ_FORCE_KERNEL=legacy)"
                              if os.environ.get("SQ_FORCE_KERNEL") == "legacy"
                              else "region form (the region kernels' recurrence with D in global scratch)"),
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "single GPU"},
        "forces_max_abs": float(F.abs().max().item()),
        "roofline": {"kernel": ("nl_force_kernel" if os.environ.get("SQ_FORCE_KERNEL") == "legacy"
                                else "force_region_kernel"),
                     "bound": "alu", "achieved": flops / t / 1e12, "peak": peak,
                     "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak, "traffic": None, "peak_basis": basis},
        "e2e": {"value": units / float(np.median(e2e)), "unit": FORCE_UNIT,
                "h2d_bytes_per_step": 3 * wl.n_nodes * 8, "d2h_bytes_per_step": wl.n_atoms * 3 * 8},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not a.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sample = a.cpu_sample or cores * 8
        try:
            pool = OraclePool(name, cores)
            nodes = synth.sample_nodes(wl.n_nodes, sample, seed=4321)
            chunks = [c for c in np.array_split(nodes, cores) if len(c)]
            tc = max(pool.pool.map(_oracle_force_chunk, chunks))
            pool.close()
            line["cpu_baseline"] = {"value": len(nodes) * wl.npl / tc, "unit": FORCE_UNIT, "cores": len(chunks),
                                    "kind": "oracle",
                                    "sample": f"{len(nodes)} seeded nodes of {name} (or_nl_force after the "
                                              f"oracle's own bounds; force part timed), per-node rate"}
        except Exception as exc:
            line["cpu_baseline"] = {"value": None, "unit": FORCE_UNIT, "cores": 0, "kind": "oracle",
                                    "sample": f"failed: {exc}"}
    solver.close()
    print(json.dumps(line), flush=True)


def run_scf(a):
    """The SCF loop (SQSCF: SQ path, CG Poisson, X-alpha, mixing) on the
    workload named after ``scf_``, FP32 recurrence, to a 1e-6 residual.
    Value: seconds per SCF iteration (device time of the whole loop divided
    by its iterations)."""
    import torch
    from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQSCF, SQSolver, build

    name = a.workload[len("scf_"):]
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    build()
    s = synth.make_system(name)
    wl = s.wl
    prec = SQ_FP32 if a.precision == "fp32" else SQ_FP64
    solver = SQSolver.from_workload(wl, s.positions, precision=prec, device=str(dev))
    V_loc = torch.from_numpy(s.V.ravel().copy()).to(dev)
    kerker = None if a.kerker == "none" else tuple(float(x) for x in a.kerker.split(","))
    reuse = None if a.reuse_bounds == "none" else float(a.reuse_bounds)
    fine = None
    refine_at = None if a.refine_at == "none" else float(a.refine_at)
    if refine_at is not None:
        fine = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=str(dev))
    fresh = None if a.fresh_below == "none" else float(a.fresh_below)
    scf = SQSCF(solver, V_loc, wl.n_electrons, wl.kT, beta=a.beta, history=a.history, margin=wl.margin,
                kerker=kerker, period=a.period, reuse_bounds=reuse, fresh_below=fresh,
                refine=None if fine is None else (fine, refine_at))
    solver.solve(V_loc, wl.n_electrons, wl.kT, wl.n_lanczos, wl.margin)      # warm-up (not timed)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = solver.launches + (fine.launches if fine is not None else 0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stamps = []
    t0 = time.perf_counter()
    e0.record(stream)
    out = scf.run(tol=1e-6, max_iter=a.max_scf,
                  on_step=lambda V, rho, mu: stamps.append(time.perf_counter()))
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    it = out["iterations"]
    line = {
        "metric": "seconds per SCF iteration (SQ step, Poisson, X-alpha, mixing)", "value": t / it, "unit": "s",
        "n_gpus": 1, "steps": it, "warmup": 1, "ms_per_step": t / it * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == SQ_FP32 else "f64",
        "data": "synthetic (seeded FCC Al-like crystal, Gaussian V and KB projectors)",
        "config": {"workload": f"{a.workload}: {wl.cells}^3 cells ({wl.n_atoms} atoms), {wl.n}^3 grid, "
                               f"{2 * wl.m + 1}^3 regions, n_pl={wl.npl}, kT={wl.kT}",
                   "mixing": {"beta": a.beta, "history": a.history, "period": a.period, "kerker": kerker},
                   "reuse_bounds": reuse, "fresh_bounds_below": fresh, "fp64_from_residual": refine_at,
                   "tolerance": 1e-6, "parallelism": "single GPU"},
        "iterations": it, "converged": out["converged"], "residuals": [float(r) for r in out["residuals"]],
        "lanczos_runs": out["lanczos_runs"], "fp64_from_iteration": out["refined_at"],
        "iteration_wall_s": [b - a_ for a_, b in zip([t0] + stamps[:-1], stamps)],
        "poisson_iterations": out["poisson_iterations"], "wall_s": wall,
        "roofline": None, "e2e": None, "cpu_baseline": None,
        "gpu_launches": int(solver.launches + (fine.launches if fine is not None else 0) - launches0),
        "clocks": clk,
    }
    scf.close()
    solver.close()
    if fine is not None:
        fine.close()
    print(json.dumps(line), flush=True)


def run_warmstart(a):
    """The learned warm start on the 4x4x4-cell system (al256_64): training
    pairs from SCF iterations of seeded one-cell geometries with the same
    grid spacing, region, degree and temperature; two networks trained on
    them with their own kernels (input V, and input V - mu with mu fixed by
    the electron count at inference); then the SCF of al256_64 to 1e-6 from
    V_loc and from each warm start.  Value: SCF iterations with the better
    warm start."""
    import torch
    from paper_1708_07913_gb300 import SQCNN, build
    from paper_1708_07913_gb300 import warmstart as wsm

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    build()
    target = synth.WORKLOADS["al256_64"]
    tmpl = synth.custom_workload("ws_train", cells=1, n=16, r_cut=target.r_cut, npl=target.npl, kT=target.kT,
                                 sigma_disp=target.sigma_disp, nonlocal_=True, seed=0)
    clocks = ClockSampler(0)
    clocks.start()
    pairs, t_data = wsm.training_pairs(tmpl, a.train_geometries, a.train_iters, seed=5000, device=str(dev),
                                       mu_offsets=(-0.1, -0.05, 0.0, 0.05, 0.1))
    nets, t_train, losses = {}, {}, {}
    for label, fermi in (("warm_V", False), ("warm_V_minus_mu", True)):
        use = pairs if fermi else wsm.scf_pairs(pairs)
        net = SQCNN(True, 0, *wsm.input_scales(use, fermi_referenced=fermi), device=str(dev))
        losses[label], t_train[label] = wsm.train(net, use, a.train_steps, fermi_referenced=fermi)
        nets[label] = (net, fermi)
    reuse = None if a.reuse_bounds == "none" else float(a.reuse_bounds)
    refine_at = None if a.refine_at == "none" else float(a.refine_at)
    fresh = None if a.fresh_below == "none" else float(a.fresh_below)
    res = wsm.compare(nets, target, tol=1e-6, max_iter=a.max_scf, device=str(dev), reuse_bounds=reuse,
                      fresh_below=fresh, refine_at=refine_at)
    clk = clocks.stop()
    for net, _ in nets.values():
        net.close()
    best = min(("warm_V", "warm_V_minus_mu"), key=lambda k: (not res[k]["converged"], res[k]["iterations"]))
    line = {
        "metric": "SCF iterations to a 1e-6 residual (al256_64) with the learned warm start",
        "value": res[best]["iterations"], "unit": "iterations", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": res[best]["seconds"] * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 network (FP32 accumulation), FP32 SQ recurrence with FP64 moments",
        "data": "synthetic (seeded FCC Al-like crystals, Gaussian V and KB projectors)",
        "config": {"workload": "warmstart_c4: target al256_64 (4^3 cells, 256 atoms, 64^3 grid, 25^3 regions, "
                               "n_pl=48, kT=0.05); training on one-cell 16^3 geometries",
                   "training_pairs": len(pairs), "training_geometries": a.train_geometries,
                   "fermi_level_offsets": [-0.1, -0.05, 0.0, 0.05, 0.1],
                   "scf_iterations_per_geometry": a.train_iters, "adam_steps": a.train_steps,
                   "mixing": "Anderson, history 16, beta 0.3, Kerker (0.5, 0.1)", "best": best,
                   "reuse_bounds": reuse, "fresh_bounds_below": fresh, "fp64_from_residual": refine_at,
                   "parallelism": "single GPU"},
        "plain_iterations": res["plain"]["iterations"], "plain_converged": res["plain"]["converged"],
        "results": res,
        "seconds": {"training_data": t_data, "training": t_train},
        "loss_first_last": {k: [v[0], v[-1]] for k, v in losses.items()},
        "roofline": None, "e2e": None, "cpu_baseline": None, "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.warmup < 3:
        a.warmup = 3
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch16":
        run_batch(a)
    elif a.workload.startswith("force_"):
        run_force(a)
    elif a.workload == "warmstart_c4":
        run_warmstart(a)
    elif a.workload.startswith("scf_"):
        run_scf(a)
    else:
        run_gb300(a)


if __name__ == "__main__":
    main()
