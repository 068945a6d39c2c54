"""Benchmark of the GB300 GL-ECSIM hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

One step = one full pass of the hot path: limited-LF coefficients, right-hand
side, FP64 FGMRES field solve, field advance, the fused mover + re-bin +
deposit kernel, and the grid-side assembly of rho, u, the comoving current and
the mass matrices.  The metric is particle-steps/s of push+deposit (the fused
particle kernel plus the moment assembly it feeds), timed with CUDA events on
the launching stream inside the timed steps; the field solve's time per step
is reported next to it.  Inputs are seeded synthetic plasmas (workloads/).

With --gpus N > 1 (launched by torch.distributed.run) every rank runs an
independent replica of the workload on its own GPU (the single-domain step has
no exchange to shard); value = particle-steps of all ranks / max rank time.

--impl reference times the FP64 CPU oracle (the reference arm of this project)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "particle-steps/s (push+deposit) & GMRES time/step, learned vs plain"
UNIT = "particle-steps/s"
ALG_BYTES_2D = 44          # per particle-step: read ox,oy,vx,vy,vz,w (24 B) + write ox,oy,vx,vy,vz (20 B)
ALG_BYTES_3D = 52          # per particle-step: read ox,oy,oz,vx,vy,vz,w (28 B) + write ox,oy,oz,vx,vy,vz (24 B)
# FP32 flops of the 3D push kernel per particle: mover 172 (corner weights 15, E and B
# gathered from 8 corners 96, rotation 55, position 6), deposit factors 214 (weights 15,
# B and u_ref gathered 96, alpha 25, alpha (v - u_ref) 21, pair weights 57), and the
# sums of 27 pair classes x 16 columns, 864
FLOP_3D = 1250
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12    # SMs x FP32 lanes x FMA x max SM clock: 80.5 TFLOP/s


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over all ranks: the whole job is
    as slow as its slowest replica."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_rate(world, units_per_rank, ms):
    """Units processed by all ranks per second of the slowest rank's time."""
    return world * units_per_rank / (ms / 1000.0)


def make_workload(name):
    if name == "harris":
        return workloads.harris(nx=512, ny=256, ppc=100), "2D Harris-sheet reconnection 512x256 cells, 100 ppc/species"
    if name == "harris_small":
        return workloads.harris(nx=128, ny=64, ppc=100), "2D Harris sheet 128x64 cells, 100 ppc/species"
    if name == "uniform":
        return workloads.uniform_drift(n=(32, 32, 1), ppc=64), "2D periodic 32x32, 64 ppc/species"
    if name == "shock_parallel":
        return (workloads.shock_1d("parallel", ny=8, ppc=256),
                "quasi-parallel shock from the printed states, 940x8 cells, 256 ppc/species, open x boundaries")
    if name == "shock_wall":
        return workloads.shock_wall(), "shock by reflection: inflow onto a reflecting wall, 1024x8 cells, 256 ppc"
    raise SystemExit(f"unknown workload {name}")


def drift3d_config(n=128, ppc=64):
    """The 3D periodic drifting plasma: n^3 cells of 0.1 d_i, electrons and ions
    (m_i/m_e 25) drawn on the device as drifting Maxwellians (u = 0.3 c along x,
    vth_e = 0.05 c, vth_i = 0.01 c, ppc per cell and species), B = 0.1 along z,
    E = -u x B / c, theta = 1/2, dt = 0.1 / omega_pe, comoving current and
    limited LF on, mixed-precision FGMRES to an FP64 true residual of 1e-8."""
    return dict(n=(n, n, n), dx=(0.1, 0.1, 0.1), ppc=ppc, u=(0.3, 0.0, 0.0), B=(0.0, 0.0, 0.1),
                vth_e=0.05, vth_i=0.01, mass_ratio=25.0, dt=0.02)


def drift3d_context(gx, n=128, ppc=64, seed=2024):
    c3 = drift3d_config(n, ppc)
    cfg = gx.make_config(c3["n"], c3["dx"], dt=c3["dt"], comoving=1, lf_on=1, gmres_tol=1e-8, seed=seed,
                         gmres_mixed=1)
    ctx = gx.Context(cfg)
    n0 = workloads.N0
    ctx.species_maxwellian(-1.0, 1.0 / c3["mass_ratio"], ppc, n0, c3["u"], c3["vth_e"])
    ctx.species_maxwellian(1.0, 1.0, ppc, n0, c3["u"], c3["vth_i"])
    u32 = np.asarray(c3["u"], np.float32).astype(np.float64)
    Em = -np.cross(u32, np.asarray(c3["B"], float))
    shape = (3, n, n, n)
    E = np.empty(shape)
    B = np.empty(shape)
    for d in range(3):
        E[d] = Em[d]
        B[d] = c3["B"][d]
    ctx.fields_set(E, B)
    return ctx, 2 * ppc * n ** 3


def run_drift3d(gx, ppc, warmup, steps, barrier, dist, world, n=128):
    """Push+deposit throughput of the 3D drifting plasma at `ppc` particles per
    cell and species, with the push kernel's HBM and FP32 fractions."""
    peak, peak_kind = load_peaks()
    ctx, npart = drift3d_context(gx, n, ppc)
    for _ in range(warmup):
        ctx.step(1, allow_noconv=True)
    ctx.timers(reset=True)
    ctx.kernel_timer(reset=True)
    iters = []
    barrier()
    for _ in range(steps):
        iters.append(ctx.step(1, allow_noconv=True).iters)
    barrier()
    tm = ctx.timers(reset=True)
    kt = ctx.kernel_timer(reset=True)
    ctx.close()
    pd_ms = (tm["push_ms"] + tm["moments_ms"]) / steps
    kms = kt["pd_kernel_ms"] / max(1, kt["pd_launches"])
    pd_ms, kms = max_over_ranks([pd_ms, kms], dist, "cuda")
    per_launch = npart / 2
    hbm = ALG_BYTES_3D * per_launch / (kms / 1000.0) / 1e9
    alu = FLOP_3D * per_launch / (kms / 1000.0) / 1e12
    return {"ppc": ppc, "particles": npart, "value": whole_job_rate(world, npart, pd_ms), "unit": UNIT,
            "push_deposit_ms_per_step": pd_ms, "push_kernel_ms_per_launch": kms,
            "solve_ms_per_step": tm["solve_ms"] / steps, "gmres_iters_per_step": statistics.mean(iters),
            "hbm": {"achieved": hbm, "peak": peak, "unit": "GB/s", "frac": hbm / peak, "peak_kind": peak_kind,
                    "alg_bytes_per_particle": ALG_BYTES_3D},
            "alu": {"achieved": alu, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": alu / FP32_PEAK_TFLOPS,
                    "flop_per_particle": FLOP_3D}}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic(summary_name, source):
    """DRAM bytes per launch of the dominant kernel from its committed ncu
    summary (profiles/<summary_name>.md, lines "- dram_bytes_per_launch: N" and
    "- kernel_source_sha256: H"), or None when there is none or the kernel's
    source has changed since the counters were taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", summary_name + ".md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        line = line.strip()
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, source), "rb").read()).hexdigest()
    except OSError:
        return None
    if vals.get("kernel_source_sha256") != sha:
        return None
    try:
        return int(float(vals["dram_bytes_per_launch"]))
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region:
    the sampler (every 20 ms, each line time-stamped) is started and seen running
    before the region begins; the summary keeps the samples taken inside it (or,
    when the region is shorter than the sampling interval, the ones nearest to
    it, and says so)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.p, self.out = dev, None, os.path.join("/tmp", f"gx_clocks_{os.getpid()}.csv")
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                       "-lms", "20", "-i", str(self.dev)], stdout=self.f, stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0
            while time.time() < deadline and os.path.getsize(self.out) == 0:
                time.sleep(0.02)
        except Exception:
            self.p = None
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        self.t1 = time.time()
        if self.p:
            time.sleep(0.05)                  # one sample past the region's end
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p or not os.path.exists(self.out):
            return None
        return summarize_clock_lines(open(self.out).read().splitlines(), self.t0, self.t1)


def summarize_clock_lines(lines, t0, t1):
    """Median SM clock, maximum clock and the throttle reasons seen, from
    nvidia-smi CSV lines (timestamp, index, clocks.sm, clocks.max.sm, power,
    active mask, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown,
    sw_power_cap), over the samples time-stamped within [t0, t1]; if there are
    none, over the sample nearest to either end ("window": "nearest")."""
    import datetime
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            sm, mx = float(parts[2]), float(parts[3])
        except ValueError:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        rows.append((ts, sm, mx, parts[6:10]))
    if not rows:
        return None
    timed = [r for r in rows if r[0] is not None]
    inside = [r for r in timed if t0 is not None and t1 is not None and t0 <= r[0] <= t1]
    window = "during"
    if not inside:
        ref = [t for t in (t0, t1) if t is not None]
        if timed and ref:
            window = "nearest"
            inside = [min(timed, key=lambda r: min(abs(r[0] - t) for t in ref))]
        else:
            window = "untimed"
            inside = rows
    reasons = set()
    for r in inside:
        for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[3]):
            if v.lower() == "active":
                reasons.add(name)
    return {"sm_mhz": statistics.median([r[1] for r in inside]), "sm_max_mhz": max(r[2] for r in inside),
            "reasons": sorted(reasons), "samples": len(inside), "window": window}


def oracle_push_deposit_rate(wl, budget_s=15.0, cells=(64, 32)):
    """The FP64 CPU oracle's push+deposit throughput (mover + bulk moments +
    deposit) on a bounded patch of the workload (single host thread)."""
    import oracle as O
    sub = make_sample(wl, cells)
    cfg = O.make_cfg(sub.n, sub.dx, **sub.grid_kwargs())
    pl = O.Plasma.from_species(sub.species)
    Bn = O.node_avg(cfg, sub.B0)
    Eth = sub.E0.copy()
    t0 = time.perf_counter()
    steps = 0
    while True:
        O.mover(cfg, pl, Eth, Bn)
        rm, P = O.bulk_moments(cfg, pl)
        u = O.bulk_velocity(cfg, rm, P)
        O.deposit(cfg, pl, Bn, u=u if sub.comoving else None)
        steps += 1
        if time.perf_counter() - t0 > budget_s or steps >= 50:
            break
    dt = time.perf_counter() - t0
    return pl.np * steps / dt, {"particles": pl.np, "steps": steps, "seconds": dt, "cells": list(cells)}


def _oracle_worker(args):
    """One host core's run of the oracle on the patch (a spawned process)."""
    sub, budget_s = args
    import oracle as O
    O.build()
    cfg = O.make_cfg(sub.n, sub.dx, **sub.grid_kwargs())
    pl = O.Plasma.from_species(sub.species)
    Bn = O.node_avg(cfg, sub.B0)
    Eth = sub.E0.copy()
    t0 = time.perf_counter()
    steps = 0
    while True:
        O.mover(cfg, pl, Eth, Bn)
        rm, P = O.bulk_moments(cfg, pl)
        u = O.bulk_velocity(cfg, rm, P)
        O.deposit(cfg, pl, Bn, u=u if sub.comoving else None)
        steps += 1
        if time.perf_counter() - t0 > budget_s or steps >= 200:
            break
    return pl.np * steps / (time.perf_counter() - t0)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def oracle_all_cores_rate(wl, budget_s=8.0, cells=(64, 32)):
    """The oracle as it stands, one process per host core, each on the same
    patch: the sum of their push+deposit throughputs (processes are spawned,
    so no CUDA state is inherited)."""
    import multiprocessing as mp
    sub = make_sample(wl, cells)
    ncores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(ncores) as pool:
        rates = pool.map(_oracle_worker, [(sub, budget_s)] * ncores)
    return float(sum(rates)), ncores


def make_sample(wl, cells):
    """A patch of the workload: the first cells[0] x cells[1] cells with their
    particles and fields, made periodic."""
    nx, ny = cells
    nx, ny = min(nx, wl.n[0]), min(ny, wl.n[1])
    Lx, Ly = nx * wl.dx[0], ny * wl.dx[1]
    species = []
    for s in wl.species:
        m = (s["x"] < Lx) & (s["y"] < Ly)
        species.append({k: (v[m] if isinstance(v, np.ndarray) else v) for k, v in s.items()})
    import copy
    sub = copy.copy(wl)
    sub.n = (nx, ny, 1)
    sub.species = species
    sub.E0 = np.ascontiguousarray(wl.E0[:, :, :ny, :nx])
    sub.B0 = np.ascontiguousarray(wl.B0[:, :, :ny, :nx])
    return sub


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl, desc = make_workload(args.workload)
    import oracle as O
    O.build()
    rates = []
    info = None
    for k in range(args.warmup + args.steps):
        r, info = oracle_push_deposit_rate(wl, budget_s=4.0)
        if k >= args.warmup:
            rates.append(r)
    single = statistics.median(rates)
    value, ncores = oracle_all_cores_rate(wl, budget_s=6.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample": f"{info['cells'][0]}x{info['cells'][1]}-cell patch"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "cpu_model": cpu_model(), "single_thread_value": single,
                             "sample": f"{info['particles']} particles of a {info['cells'][0]}x{info['cells'][1]}"
                                       f"-cell patch, mover+bulk+deposit; one unmodified oracle process per "
                                       f"core, throughputs summed; single thread: {info['steps']} steps per "
                                       f"timing"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_shock(gx, warmup, steps, barrier, dist, world, wall=False):
    """Push+deposit throughput on a shock-shaped plasma, timed like the main
    workload (library CUDA events over push, refill and moments): the paper's
    quasi-parallel shock (printed states, open boundaries refilled every step)
    over 940 x 8 cells of 0.4 d_i with 256 particles per cell and species (3.85 M
    particles), or with `wall` the shock by reflection (inflow at 0.2 c onto a
    reflecting conducting wall, 1024 x 8 cells of 0.1 d_i, 256 ppc, 4.16 M)."""
    import torch
    wl = workloads.shock_wall() if wall else workloads.shock_1d("parallel", ny=8, ppc=256)
    ctx = gx.from_workload(wl, gmres_mixed=1)
    for _ in range(warmup):
        ctx.step(1, allow_noconv=True)
    ctx.timers(reset=True)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        ctx.step(1, allow_noconv=True)
    ev1.record()
    barrier()
    tm = ctx.timers(reset=True)
    npart = sum(ctx.species_count(s) for s in range(len(wl.species)))
    ctx.close()
    pd_ms, step_ms = max_over_ranks([(tm["push_ms"] + tm["moments_ms"]) / steps, ev0.elapsed_time(ev1) / steps],
                                    dist, "cuda")
    return {"value": whole_job_rate(world, npart, pd_ms), "unit": UNIT, "push_deposit_ms_per_step": pd_ms,
            "ms_per_step": step_ms, "particles": npart,
            "workload": (f"{wl.name}: inflow at 0.2 c onto a reflecting conducting wall, m_i/m_e 100, "
                         f"{wl.n[0]}x{wl.n[1]} cells" if wall else
                         f"{wl.name}: the paper's 1D quasi-parallel shock (printed up/downstream states, M_A 7, "
                         f"m_i/m_e 25, c = 3000 km/s) on {wl.n[0]}x{wl.n[1]} cells, open x boundaries")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="harris")
    ap.add_argument("--impl", default="gx")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precond", action="store_true")
    ap.add_argument("--no-shock", action="store_true")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D drifting-plasma sweep")
    ap.add_argument("--n3d", type=int, default=128, help="cells per axis of the 3D drifting plasma")
    ap.add_argument("--sweep3d", default="8,16,32,64,128,256",
                    help="particles per cell and species of the 3D 128^3 sweep")
    ap.add_argument("--precond-workload", default="harris_1024x512",
                    help="plasma of the learned-vs-plain GMRES comparison: harris_1024x512 (the learned-"
                         "preconditioner configuration: Harris reconnection, 1024x512 cells, 100 ppc/species) "
                         "or 'same' (the main workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import paper_2506_11320_gb300 as gx
    if not os.path.exists(gx.LIB_PATH):
        from paper_2506_11320_gb300 import build as b
        b.build()
    wl, desc = make_workload(args.workload)
    Np = wl.n_particles

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
            torch.cuda.synchronize()

    # ------------------------------------------------------- device-timed run
    # the field solve: mixed-precision FGMRES (FP32 Arnoldi cycles between FP64
    # restarts); the relres the library reports is the FP64 true residual
    ctx = gx.from_workload(wl, gmres_tol=wl.gmres_tol, gmres_mixed=1)
    for _ in range(args.warmup):
        ctx.step(1, allow_noconv=True)
    ctx.timers(reset=True)
    ctx.kernel_timer(reset=True)
    iters, relres = [], []
    barrier()
    with Clocks(dev) as clk:
        t0 = time.perf_counter()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            st = ctx.step(1, allow_noconv=True)
            iters.append(st.iters)
            relres.append(st.relres)
        ev1.record()
        barrier()
        wall = time.perf_counter() - t0
    step_ms_dev = ev0.elapsed_time(ev1) / args.steps
    tm = ctx.timers(reset=True)
    kt = ctx.kernel_timer(reset=True)
    pd_ms = (tm["push_ms"] + tm["moments_ms"]) / args.steps
    solve_ms = tm["solve_ms"] / args.steps
    pd_ms_max, step_ms_max, _ = max_over_ranks([pd_ms, step_ms_dev, wall], dist, "cuda")
    value = whole_job_rate(world, Np, pd_ms_max)

    peak, peak_kind = load_peaks()
    # roofline of the dominant kernel: the fused mover + re-bin + deposit
    # kernel, one launch per species; algorithmic bytes of one launch = 44 B per
    # particle of that species; time = its own CUDA events (launch list share in
    # profiles/)
    n_launch = max(1, kt["pd_launches"])
    pd_kernel_ms = kt["pd_kernel_ms"] / n_launch
    alg_bytes = ALG_BYTES_2D * Np / len(wl.species)
    achieved = alg_bytes / (pd_kernel_ms / 1000.0) / 1e9
    traffic = load_traffic(f"k_pd_push_{args.workload}", "paper_2506_11320_gb300/csrc/gx_particles.cu")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "k_pd<push> (fused mover + re-bin + deposit), one launch per species",
                "alg_bytes_per_launch": alg_bytes, "ms_per_launch": pd_kernel_ms}
    push_kernel_ms = tm["push_ms"] / args.steps

    # ------------------------------------------------------- field solve: mixed vs all-FP64 FGMRES
    fp64 = gx.from_workload(wl, gmres_tol=wl.gmres_tol)
    for _ in range(args.warmup):
        fp64.step(1, allow_noconv=True)
    fp64.timers(reset=True)
    rr64 = []
    for _ in range(args.steps):
        rr64.append(fp64.step(1, allow_noconv=True).relres)
    solve64_ms = fp64.timers(reset=True)["solve_ms"] / args.steps
    fp64.close()
    mixed_cmp = {"mixed_ms_per_step": solve_ms, "fp64_ms_per_step": solve64_ms,
                 "speedup": solve64_ms / solve_ms if solve_ms > 0 else None,
                 "mixed_relres_max": max(relres), "fp64_relres_max": max(rr64), "gmres_tol": wl.gmres_tol}

    # ------------------------------------------------------- field solve: learned vs plain
    solve_cmp = None
    if not args.no_precond:
        if args.precond_workload == "same":
            pwl, pdesc = wl, desc
        else:
            pwl = workloads.harris(nx=1024, ny=512, ppc=100)
            pdesc = ("Harris double current sheet 1024x512 cells, dx 0.05 d_i, 100 particles/cell/species "
                     f"({pwl.n_particles / 1e6:.1f} M particles), mass ratio 100, Ti/Te 5, flow 0.5 v_A")
        solve_cmp = run_precond_compare(gx, pwl, args.steps, barrier)
        solve_cmp["workload"] = pdesc
        solve_cmp["cells"] = list(pwl.n[:2])
        del pwl

    # ------------------------------------------------------- shock-shaped plasma
    shock = shock_wall = None
    if not args.no_shock:
        shock = run_shock(gx, args.warmup, args.steps, barrier, dist, world)
        shock_wall = run_shock(gx, args.warmup, args.steps, barrier, dist, world, wall=True)

    # ------------------------------------------------------- 3D drifting plasma, 128^3, ppc sweep
    sweep3d = None
    if not args.no_3d:
        sweep3d = {"workload": f"3D periodic drifting Maxwellian plasma, {args.n3d}^3 cells of 0.1 d_i, u = 0.3 c along x, "
                               "vth_e 0.05 c, vth_i 0.01 c, m_i/m_e 25, B = 0.1 along z, comoving current and "
                               "limited LF on, particles drawn on the device",
                   "points": []}
        for ppc in [int(v) for v in args.sweep3d.split(",") if v]:
            sweep3d["points"].append(run_drift3d(gx, ppc, 1, 3, barrier, dist, world, n=args.n3d))

    # ------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(gx, wl, args.steps, barrier, dist, world)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            rate, info = oracle_push_deposit_rate(wl, budget_s=10.0)
            allc, ncores = oracle_all_cores_rate(wl, budget_s=8.0)
            cpu = {"value": allc, "unit": UNIT, "cores": ncores, "kind": "oracle", "cpu_model": cpu_model(),
                   "single_thread_value": rate,
                   "sample": f"{info['particles']} particles of a {info['cells'][0]}x{info['cells'][1]}-cell patch "
                             f"of the workload, FP64 mover+bulk moments+deposit; one unmodified oracle process per "
                             f"host core for 8 s, throughputs summed; single thread {info['steps']} steps in "
                             f"{info['seconds']:.1f} s"}
        except Exception as e:     # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 particles / f64 fields", "data": "synthetic",
            "config": {"workload": desc, "particles": Np, "cells": list(wl.n[:2]), "comoving": wl.comoving,
                       "lf": wl.lf_on, "ns_j": wl.ns_j, "gmres_tol": wl.gmres_tol, "precond": "none",
                       "gmres": "mixed precision (FP32 Arnoldi cycles, FP64 restarts and true residual)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 ({Np * 24 / 1e6:.0f} MB of particle state read per step, "
                             f"L2 129 MB); no flush"},
            "push_deposit_ms_per_step": pd_ms_max, "push_phase_ms_per_step": push_kernel_ms,
            "gmres_ms_per_step": solve_ms, "gmres_iters_per_step": statistics.mean(iters),
            "gmres_relres_max": max(relres), "gmres_mixed_vs_fp64": mixed_cmp,
            "wall_ms_per_step": 1000 * wall / args.steps,
            "gmres_learned_vs_plain": solve_cmp,
            "shock": shock, "shock_wall": shock_wall, f"drift3d_{args.n3d}": sweep3d,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(tm["launches"]),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_precond_compare(gx, wl, steps, barrier, collect_steps=24):
    """Field-solve time per step with the learned preconditioner against plain
    GMRES and block Jacobi on the same plasma.  Three contexts start from the
    same state and step together; the learned one keeps training pairs from its
    first `collect_steps` solves (each solve gives (r0, e) and six Krylov pairs,
    each pair cut into 122 windows of 40^2 nodes: 20,480 crops in a ring, the
    20k residual/solution pairs of the learned-preconditioner configuration),
    trains on the device, then all three are timed for `steps` steps (solve time
    from CUDA events in the library)."""
    kinds = (("plain", gx.GX_PRECOND_NONE), ("jacobi", gx.GX_PRECOND_JACOBI), ("learned", gx.GX_PRECOND_NET))
    ctxs = {k: gx.from_workload(wl, precond=p) for k, p in kinds}
    net = ctxs["learned"]
    crops, crop, per_pair = 20480, 32, 122
    net.precond_collect_crops(crops, crop, per_pair, seed=7)
    for _ in range(collect_steps):
        for c in ctxs.values():
            c.step(1, allow_noconv=True)
    barrier()
    t0 = time.perf_counter()
    losses = net.precond_train(npairs=512, crop=crop, batch=32, epochs=200, lr=2e-3, seed=7)
    barrier()
    train_s = time.perf_counter() - t0
    net.precond_collect(0)
    out = {}
    for k, c in ctxs.items():
        c.timers(reset=True)
    its = {k: [] for k in ctxs}
    for _ in range(steps):
        for k, c in ctxs.items():
            its[k].append(c.step(1, allow_noconv=True).iters)
    barrier()
    for k, c in ctxs.items():
        tm = c.timers(reset=True)
        out[k] = {"ms_per_step": tm["solve_ms"] / steps, "iters_per_step": statistics.mean(its[k])}
    out["learned_speedup_vs_plain"] = out["plain"]["ms_per_step"] / out["learned"]["ms_per_step"]
    out["training"] = {"pairs": net.precond_pairs(), "pair_kind": f"crops of {crop + 8}^2 nodes ({per_pair} per "
                       "field pair)", "collect_steps": collect_steps, "epochs": len(losses),
                       "samples_per_epoch": 512, "crop": crop, "seconds": train_s,
                       "loss_first": float(losses[0]), "loss_last": float(losses[-1])}
    out["note"] = ("solve = LF coefficients + right-hand side + FGMRES to 1e-8 relative residual + field "
                   "advance, FP64; learned = block Jacobi plus a BF16 conv-net correction trained on this "
                   "run's own solves")
    for c in ctxs.values():
        c.close()
    return out


def run_e2e(gx, wl, steps, barrier, dist=None, world=1):
    """Same metric through the public C ABI with host buffers: pinned host
    particle and field arrays are copied in (gx_species_add, gx_fields_set),
    every step's diagnostics (FP64 energies, momentum) are read back, and the
    final fields are copied out; all inside the timed region."""
    import torch
    host = []
    h2d = 0
    for s in wl.species:
        arrs = {}
        for k in ("x", "y", "z"):
            t = torch.from_numpy(np.ascontiguousarray(s[k], np.float64)).pin_memory()
            arrs[k] = t
            h2d += t.numel() * 8
        for k in ("vx", "vy", "vz", "w"):
            t = torch.from_numpy(np.ascontiguousarray(s[k], np.float32)).pin_memory()
            arrs[k] = t
            h2d += t.numel() * 4
        host.append((s["q"], s["m"], arrs))
    E0 = torch.from_numpy(np.ascontiguousarray(wl.E0)).pin_memory()
    B0 = torch.from_numpy(np.ascontiguousarray(wl.B0)).pin_memory()
    Eout = torch.empty_like(E0).pin_memory()
    Bout = torch.empty_like(B0).pin_memory()
    h2d += 2 * E0.numel() * 8
    cfg = gx.make_config(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, comoving=wl.comoving, lf_on=wl.lf_on,
                         lf_speed_c=wl.lf_speed_c, lf_beta=wl.lf_beta, ns_j=wl.ns_j, nsmooth_u=wl.nsmooth_u,
                         gmres_tol=wl.gmres_tol, gmres_mixed=1)
    barrier()
    t0 = time.perf_counter()
    ctx = gx.Context(cfg)
    for q, m, a in host:
        ctx.species_add(q, m, a["x"].numpy(), a["y"].numpy(), a["z"].numpy(), a["vx"].numpy(), a["vy"].numpy(),
                        a["vz"].numpy(), a["w"].numpy())
    ctx.fields_set(E0.numpy(), B0.numpy())
    d2h = 0
    for _ in range(steps):
        ctx.step(1, allow_noconv=True)
        ctx.diagnostics()
        d2h += 16 * 8
    ctx.get_fields(Eout.numpy(), Bout.numpy())
    d2h += 2 * Eout.numel() * 8
    barrier()
    wall_ms = max_over_ranks([1000.0 * (time.perf_counter() - t0)], dist, "cuda")[0]
    ctx.close()
    return {"value": whole_job_rate(world, wl.n_particles * steps, wall_ms), "unit": UNIT,
            "h2d_bytes_per_step": h2d // steps,
            "d2h_bytes_per_step": d2h // steps,
            "note": "context creation, binning of all particles from pinned host memory, every step's FP64 "
                    "diagnostics and the final fields read back are inside the timed region"}


if __name__ == "__main__":
    sys.exit(main())
