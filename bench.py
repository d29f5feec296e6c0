#!/usr/bin/env python
"""Benchmark of the PIC-MCC/PPPM step on one GB300 (or N independent replicas).

One bench step = one full time step of the particle cycle (gather, push with
MD subcycling near grains, absorption, MCC, deposit, Poisson solve).  The
headline workload is the large mixed-precision case: 256x256x1024 cells of
0.2 mm, 5e8 macroparticles (2.5e8 e + 2.5e8 Ar+, drawn on the device from the
seed), a 100-grain seeded cluster, 100 V at 13.56 MHz, argon at 2 Pa.
Particle arrays (16 GB mixed, 32 GB FP64) far exceed the 129 MB L2.

Prints one JSON line.  ``value`` is mixed-precision particle-steps/s summed
over ranks; the FP64 path on the same workload, Poisson solves/s, the push
kernel's roofline, an end-to-end figure through the C ABI from host arrays,
the paper-scale 128x128x512 cluster (2e8 particles) and the 64x64x256 rf
sheath (1e7 particles, with Coulomb collisions, diagnostics and the 48-run
ensemble as extra legs), and the CPU oracle on a bounded sample ride along.
``--impl reference`` times the CPU oracle alone (rank 0) on the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and Poisson solves/s, mixed vs FP64, 1 GB300, % HBM roof"
BYTES_MIXED = 64     # per particle-step: float4 pos + float4 vel, read and written
BYTES_FP64 = 128     # double4 pos + double4 vel, read and written
SORT_EVERY = 5       # counting-sort interval (steps) when not autotuned
TUNE_STEPS = 12      # steps per candidate of the autotuner (tile shape, window margin, sort interval)
TUNE_CACHE = os.path.join(tempfile.gettempdir(), "pic_tune_cache.json")


# Poisson: algorithmic bytes per mesh node per refinement iteration: the
# V(2,2) cycle (4 red-black sweeps x 12 B + residual/restriction 8.5 B +
# prolongation 8.5 B, x 8/7 for the coarser levels) plus the refinement's
# residual and update (40 B)
BYTES_NODE_MIXED = 74 + 40
BYTES_NODE_FP64 = 148 + 40
DIAG_PHASES = 16           # rf phase bins of the diagnostics run
# committed ncu summary of the push kernel on the headline workload (DRAM traffic per launch)
PUSH_PROFILE = "k_push32_w4_256x256x1024_5e8.md"


def poisson_block(pr, cold, wl, bytes_node, peak, peak_kind, precision):
    solves = max(pr["solves"], 1)
    ms = pr["solve_ms"] / solves
    iters = pr["solve_iterations"] / solves
    nodes = wl.nx * wl.ny * (wl.nz + 1)
    gbs = iters * bytes_node * nodes / (ms / 1000.0) / 1e9 if ms > 0 else 0.0
    return {"solves_per_s": 1000.0 / ms if ms > 0 else None, "iterations_per_solve": iters, "ms_per_solve": ms,
            "bytes_per_node_iteration": bytes_node, "achieved_gbs": gbs, "frac": gbs / peak, "peak_kind": peak_kind,
            "precision": precision, "warm": "from the previous step's potential, inside the step loop",
            "cold": cold}


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=4, help="headline workload (inputs.workload index)")
    ap.add_argument("--no-f64-residual", action="store_true", help="skip the FP64-residual solve leg")
    ap.add_argument("--fp64-steps", type=int, default=6)
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--eager", action="store_true", help="no CUDA graphs (for profilers)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="fixed sort interval (no autotuning)")
    ap.add_argument("--no-coulomb", action="store_true", help="skip the run with Coulomb collisions")
    ap.add_argument("--no-diag", action="store_true", help="skip the run with every diagnostic on")
    ap.add_argument("--no-extra", action="store_true", help="headline workload only (no 128x128x512 and "
                                                            "64x64x256 legs)")
    ap.add_argument("--grains", type=int, default=None,
                    help="keep only the first N grains of the headline workload (for profiling: fewer launches "
                         "for the grain tables at init)")
    ap.add_argument("--particles", type=float, default=None,
                    help="macroparticles of the headline workload (both species; the weight keeps the density); "
                         "for profiling a smaller case")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return None
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            t = [x.strip() for x in line.split(",")]
            if len(t) < 9:
                continue
            try:
                sm.append(float(t[1]))
                mx.append(float(t[2]))
            except ValueError:
                continue
            for n, v in zip(names, t[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_gpu(P, I, wl, parts, prec, steps, warmup, stream, gpu, flags=0, tune=True, sort_every=SORT_EVERY,
            tuning=None, **run_kw):
    import torch
    run = P.Run(wl, parts, prec=prec, stream=stream, sort_every=sort_every, flags=flags, **run_kw)
    if tuning is not None and not tune:
        run.set_tuning(tuning)
        sort_every = tuning["sort_every"]
    # tile shape, deposit-window margin and sort interval autotuned on the run
    # itself before the timed region (pic_tune; fixed choices otherwise)
    tuning = run.tune(TUNE_STEPS, cache_path=TUNE_CACHE) if tune else run.tuning()
    sort_every = tuning["sort_every"]
    # warm-up covers two sorts, so that the step graphs of both particle-buffer
    # parities are captured before the timed region
    run.step(max(warmup, 2 * sort_every + 1))
    _, c0 = run.counts()
    run.profile(1)
    k0 = run.profile_read()["kernels"]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(gpu)
    with clk:
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize()
        start.record(torch.cuda.current_stream())
        torch.cuda.nvtx.range_push("timed")
        run.step(steps)
        torch.cuda.nvtx.range_pop()
        end.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
    ms = start.elapsed_time(end)
    prof = run.profile_read()
    n, c1 = run.counts()
    cold = cold_solves(run)
    run.close()
    return dict(ms=ms, pushed=c1["pushed"] - c0["pushed"], prof=prof, kernels=prof["kernels"] - k0,
                live=[int(x) for x in n], clocks=clk.summary(), counters=c1, cold=cold, sort_every=sort_every,
                steps=steps, tuning=tuning)


def cold_solves(run, reps=3):
    """Solve-only loop from a zero potential on the last step's charge density
    (the warm solves are the ones inside the timed step loop)."""
    import numpy as np
    import torch
    zero = np.zeros_like(run.phi())
    times, iters = [], []
    for _ in range(reps):
        run.set_phi(zero)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(torch.cuda.current_stream())
        it, _ = run.solve()
        e.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
        iters.append(it)
    return {"ms_per_solve": statistics.median(times), "iterations_per_solve": statistics.median(iters)}


def kernel_source_hash(kernel_source, kernel):
    """sha256 of a source file from its start to the end of `kernel`'s body: the
    kernel and every helper defined above it (shared headers are not included)."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1801_00972_gb300", "csrc", kernel_source)).read()
    start = src.index(kernel + "(")
    end = src.index("\n}\n", start) + 3
    return hashlib.sha256(src[:end].encode()).hexdigest()


def traffic_from_profile(kernel_source, name, kernel="k_push32"):
    """DRAM bytes per launch of the push kernel from its committed ncu summary,
    or None when the kernel's source has changed since that capture."""
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
        digest = kernel_source_hash(kernel_source, kernel)
    except (OSError, ValueError):
        return None
    vals = dict(line.split(":", 1) for line in text.splitlines() if line.startswith(("traffic_bytes_per_launch:",
                                                                                    "source_sha256:")))
    if vals.get("source_sha256", "").strip() != digest:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def e2e(P, I, wl, prec, steps, stream, sort_every):
    """Through the public API from host buffers: pic_init from host particle
    arrays (validation, conversion and the host->device copy), then each step
    followed by a device->host read of the grain charges (the step's result).
    The host arrays are drawn before the timed region."""
    import torch
    parts = I.sample_particles(wl)
    h2d = sum(p[0].nbytes + p[1].nbytes + p[2].nbytes for p in parts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run = P.Run(wl, parts, prec=prec, stream=stream, sort_every=sort_every)
    t_init = time.perf_counter() - t0
    del parts
    _, c0 = run.counts()
    t1 = time.perf_counter()
    for _ in range(steps):
        run.step(1)
        run.grains()
    _, c1 = run.counts()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    run.close()
    d2h = (2 * 8 + 8) * len(wl.grain_r)
    ps = c1["pushed"] - c0["pushed"]
    return {"value": ps / (t2 - t0), "unit": "particle-steps/s", "h2d_bytes_per_step": int(h2d // steps),
            "d2h_bytes_per_step": int(d2h), "seconds": t2 - t0, "steps": steps, "init_s": t_init,
            "steps_value": ps / (t2 - t1),
            "note": "pic_init from host arrays (timed, its H2D bytes spread over the steps) + per step "
                    "pic_step(1) and a pic_grain_charges read; steps_value excludes pic_init"}


def batch_bench(P, I, steps, warmup):
    """The 48-run ensemble stepped concurrently (pic_batch_step).  pic_batch_step
    returns after every run's stream has finished, so host timestamps around
    it bracket the device work."""
    import torch
    wls = I.ensemble()
    parts = [I.sample_particles(w) for w in wls]
    b = P.Batch(wls, parts, prec=P.PIC_MIXED, sort_every=SORT_EVERY)
    b.step(warmup)
    c0 = sum(P.pic_counts(r)[1]["pushed"] for r in b.runs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    t = time.perf_counter() - t0
    c1 = sum(P.pic_counts(r)[1]["pushed"] for r in b.runs)
    b.close()
    return {"workload": f"{len(wls)} independent runs, meshes 32^3..64x64x128, "
                        f"{sum(w.n_e + w.n_i for w in wls):.3g} particles in all, 1-10 Pa, 1-19 grains",
            "value": (c1 - c0) / t, "unit": "particle-steps/s", "steps": steps, "ms_per_step": 1000 * t / steps,
            "timing": "host clock around pic_batch_step (synchronises all run streams)"}


def oracle_sample(wl, n_particles, steps, seed=1, threads=None):
    """The CPU oracle, as it stands, on a bounded sample of the workload: the same
    mesh, grains and gas with n_particles macroparticles (init excluded), on
    `threads` host threads (None: all)."""
    import dataclasses

    import oracle as O
    from paper_1801_00972_gb300 import inputs as I
    half = n_particles // 2
    w = dataclasses.replace(wl, n_e=half, n_i=half, weight=wl.weight * wl.n_e / max(half, 1))
    parts = I.sample_particles(w, seed=seed)
    O.set_threads(threads or 0)
    s = O.Sim(w, parts)
    n0 = s.count(0) + s.count(1)
    t0 = time.perf_counter()
    done = 0
    for _ in range(steps):
        done += s.count(0) + s.count(1)
        s.step()
    t = time.perf_counter() - t0
    cores = O.threads()
    del s
    O.set_threads(0)
    return done / t, t, n0, cores


def replica_seed(seed, rank):
    """Replicas: every rank runs the same workload from its own seed."""
    return seed + 1000 * rank


def aggregate(ms, units, device):
    """Whole-job figures of a replicas run: the slowest rank's time and the
    units (particle-steps) of all ranks; the values themselves on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    m = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(m[0]), float(u[0])


def reference_arm(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1801_00972_gb300 import inputs as I
    wl = I.workload(a.workload)
    # a bounded sample: each oracle step also solves the whole mesh exactly
    n = 2_000_000 if wl.nodes > 10_000_000 else 600_000
    steps = a.warmup + a.steps
    if wl.nodes > 10_000_000:
        steps = min(steps, 12)
    value, t, n0, cores = oracle_sample(wl, n, steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(wl), "sample_particles": n0, "oracle_steps": steps},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n0} particles (the workload's {wl.n_e + wl.n_i:.0e}) on its full mesh "
                                       f"and grains, {steps} steps incl. the exact Poisson solve, init excluded"},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def describe(wl):
    return (f"{wl.nx}x{wl.ny}x{wl.nz} cells of {wl.dx * 1e3:.1f} mm, {wl.n_e + wl.n_i:.0e} macroparticles, "
            f"{len(wl.grain_r)} grains, {wl.v_rf:.0f} V at {wl.f_rf / 1e6:.2f} MHz, "
            f"argon {wl.n_gas * 1.380649e-23 * wl.t_gas:.0f} Pa")


def push_roofline(res, peak, peak_kind, profile_name):
    pr = res["prof"]
    push_s = pr["push_ms"] / 1000.0
    achieved = res["pushed"] * BYTES_MIXED / push_s / 1e9 if push_s > 0 else 0.0
    return {"bound": "hbm", "kernel": "k_push32 (fused gather/push/absorb/MCC test/deposit)",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
            "bytes_per_particle_step": BYTES_MIXED,
            "traffic": traffic_from_profile("particles_mixed.cu", profile_name) if profile_name else None,
            "timing": "CUDA events around each step's push phase, in which the electron and ion launches "
                      "overlap on two streams (the MD-region kernel on a third); achieved = both launches' "
                      "algorithmic bytes / the phase time",
            "phase_ms_per_step": pr["push_ms"] / max(res["steps"], 1),
            "launches": pr["push_launches"]}


def leg(P, I, wl, peak, peak_kind, steps, warmup, stream, gpu, flags, tune, profile_name=None, parts=None):
    """One mixed-precision workload: value, push roofline and Poisson figures."""
    r = run_gpu(P, I, wl, parts, P.PIC_MIXED, steps, warmup, stream, gpu, flags, tune=tune)
    return r, {"workload": describe(wl), "value": r["pushed"] / (r["ms"] / 1000.0), "unit": "particle-steps/s",
               "steps": steps, "ms_per_step": r["ms"] / steps, "tuning": r["tuning"],
               "roofline": push_roofline(r, peak, peak_kind, profile_name),
               "poisson": poisson_block(r["prof"], r["cold"], wl, BYTES_NODE_MIXED, peak, peak_kind, "mixed"),
               "gpu_launches": r["kernels"], "clocks": r["clocks"]}


def main():
    a = args()
    if a.impl == "reference":
        reference_arm(a)
        return
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    from paper_1801_00972_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_1801_00972_gb300 as P
    from paper_1801_00972_gb300 import inputs as I
    P.load()
    peak, peak_kind = peaks()
    wl = I.workload(a.workload)
    if a.particles:
        half = int(a.particles) // 2
        wl = I.workload(a.workload, n_e=half, n_i=half, weight=wl.weight * wl.n_e / half)
    if a.grains is not None:
        wl.grain_pos, wl.grain_r = wl.grain_pos[: a.grains], wl.grain_r[: a.grains]
    # replicas: each rank runs its own independent run (different seed)
    wl.seed = replica_seed(wl.seed, rank)
    stream = torch.cuda.current_stream().cuda_stream
    flags = P.PIC_F_NO_GRAPH if a.eager else 0
    # the headline: the initial plasma drawn on the device from the seed (pic_init_plasma)
    mixed = run_gpu(P, I, wl, None, P.PIC_MIXED, a.steps, a.warmup, stream, local, flags, tune=not a.no_tune)
    fp64 = None
    if not a.no_fp64:
        fp64 = run_gpu(P, I, wl, None, P.PIC_FP64, a.fp64_steps, min(a.warmup, 3), stream, local, flags,
                       tune=False, sort_every=mixed["sort_every"])
    # the same solve with the refinement residual in FP64 arithmetic instead of
    # double-float (PIC_F_F64_RESIDUAL), for the cost of that choice
    f64r = None
    if not a.no_f64_residual and world == 1:
        f64r = run_gpu(P, I, wl, None, P.PIC_MIXED, a.fp64_steps, min(a.warmup, 3), stream, local,
                       flags | P.PIC_F_F64_RESIDUAL, tune=False, tuning=mixed["tuning"])
    ee = None
    if not a.no_e2e and world == 1:
        ee = e2e(P, I, wl, P.PIC_MIXED, a.e2e_steps, stream, mixed["sort_every"])
    extra = {}
    if not a.no_extra and world == 1:
        # the paper-scale cluster: 128x128x512 cells, 50 grains, 2e8 particles
        w2 = I.workload(2)
        _, extra["config_128x128x512"] = leg(P, I, w2, peak, peak_kind, max(a.steps // 2, 20), a.warmup, stream,
                                             local, flags, not a.no_tune)
        # the rf sheath with the 7-grain cluster: 64x64x256 cells, 1e7 particles, with its extra legs
        w1 = I.workload(1)
        r1, extra["config_64x64x256"] = leg(P, I, w1, peak, peak_kind, 200, a.warmup, stream, local, flags,
                                            not a.no_tune)
        c2 = extra["config_64x64x256"]
        base_ms = r1["ms"] / 200
        if not a.no_coulomb:
            coul = run_gpu(P, I, w1, None, P.PIC_MIXED, 50, a.warmup, stream, local, flags | P.PIC_F_COULOMB,
                           tune=False, tuning=r1["tuning"])
            c2["coulomb"] = {"value": coul["pushed"] / (coul["ms"] / 1000.0), "unit": "particle-steps/s",
                             "steps": 50, "ms_per_step": coul["ms"] / 50,
                             "extra_ms_per_step": coul["ms"] / 50 - base_ms,
                             "note": "mixed, PIC_F_COULOMB (e-e, e-Ar+, Ar+-Ar+ binary collisions, lnL = 10)"}
        if not a.no_diag:
            import numpy as np
            h = 0.08 * w1.dx
            centre = np.asarray(w1.grain_pos).mean(0)
            diag = run_gpu(P, I, w1, None, P.PIC_MIXED, 50, a.warmup, stream, local, flags | P.PIC_F_MOMENTS,
                           tune=False, tuning=r1["tuning"], mom_phases=DIAG_PHASES, fine_n=(200, 200, 200),
                           fine_h=h, fine_origin=tuple(centre - 100 * h), eepf_bins=200, eepf_de_ev=0.1)
            c2["diagnostics"] = {"value": diag["pushed"] / (diag["ms"] / 1000.0), "unit": "particle-steps/s",
                                 "steps": 50, "ms_per_step": diag["ms"] / 50,
                                 "extra_ms_per_step": diag["ms"] / 50 - base_ms,
                                 "note": f"mixed, PIC_F_MOMENTS with T_e/T_i, {DIAG_PHASES} rf phase bins, 200^3 "
                                         "fine grid (0.08 dx) on the cluster, EEPF 200 x 0.1 eV per cell plane, "
                                         "sampled every step"}
        if not a.no_batch:
            extra["batch"] = batch_bench(P, I, 20, a.warmup)

    def agg(x):
        return None if x is None else aggregate(x["ms"], x["pushed"], "cuda")

    m_ms, m_tot = agg(mixed)
    f = agg(fp64)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC,
        "value": m_tot / (m_ms / 1000.0),
        "unit": "particle-steps/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": m_ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "mixed: f32 particle offsets and velocities with int cells, f32 multigrid V-cycles with "
                 "double-float (two-f32, about 48-bit) residual refinement and an f32 exact coarse-level "
                 "solve, int64 fixed-point charge",
        "data": "synthetic",
        "config": {"workload": describe(wl) + ", 100-grain seeded cluster, initial plasma drawn on the device "
                                              "from the seed",
                   "parallelism": "replicas only" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (particle arrays 16 GB mixed / 32 GB FP64)",
                   "tuning": mixed["tuning"],
                   "tuned": "fixed" if a.no_tune else "autotuned (pic_tune: tile shape, window margin, sort order, sort interval)",
                   "tol": 1e-10},
        "roofline": push_roofline(mixed, peak, peak_kind, PUSH_PROFILE),
        "poisson": poisson_block(mixed["prof"], mixed["cold"], wl, BYTES_NODE_MIXED, peak, peak_kind, "mixed"),
        "gpu_launches": mixed["kernels"],
        "clocks": mixed["clocks"],
        "live_particles_end": mixed["live"],
    }
    if fp64 is not None:
        fp = fp64["prof"]
        fpush = fp["push_ms"] / 1000.0
        fach = fp64["pushed"] * BYTES_FP64 / fpush / 1e9 if fpush > 0 else 0.0
        line["fp64"] = {"value": f[1] / (f[0] / 1000.0), "unit": "particle-steps/s", "steps": a.fp64_steps,
                        "ms_per_step": f[0] / a.fp64_steps,
                        "push_achieved_gbs": fach, "push_frac": fach / peak,
                        "poisson": poisson_block(fp, fp64["cold"], wl, BYTES_NODE_FP64, peak, peak_kind, "fp64"),
                        "mixed_speedup": (m_tot / m_ms) / (f[1] / f[0])}
    if f64r is not None:
        pb = poisson_block(f64r["prof"], f64r["cold"], wl, BYTES_NODE_MIXED, peak, peak_kind, "mixed")
        line["poisson"]["f64_residual"] = {
            "ms_per_solve": pb["ms_per_solve"], "iterations_per_solve": pb["iterations_per_solve"],
            "cold": pb["cold"], "steps": a.fp64_steps,
            "note": "the same mixed solve with the refinement residual in FP64 arithmetic (PIC_F_F64_RESIDUAL) "
                    "instead of double-float sums"}
    if ee is not None:
        line["e2e"] = ee
    line.update(extra)
    if not a.no_cpu:
        v, t, n0, cores = oracle_sample(wl, 2_000_000, 2)
        line["cpu_baseline"] = {"value": v, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"{n0} of the {wl.n_e + wl.n_i:.0e} particles on the full "
                                          f"{wl.nx}x{wl.ny}x{wl.nz} mesh with its {len(wl.grain_r)} grains, "
                                          f"2 steps incl. the exact Poisson solve, init excluded ({t:.1f} s)"}
        v1, t1, n1, _ = oracle_sample(wl, 500_000, 1, threads=1)
        line["cpu_baseline"]["one_core"] = {"value": v1, "cores": 1,
                                            "sample": f"{n1} particles, 1 step incl. the exact solve ({t1:.1f} s)"}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
