#!/usr/bin/env python
"""Throughput benchmark of the MFM step on the GB300 (one JSON line on stdout).

Workload: the subsonic turbulent box of 128^3 = 2,097,152 particles (seeded
synthetic initial conditions, gamma = 5/3, N_ngb = 32, rms Mach 0.5,
log-normal density sigma 0.3), FP32 mixed path, global CFL step.  A step is
one full gz_step: bin + sort, h-iteration, gradients + limiter, CFL step,
pairwise HLLC fluxes, update.  The working set (state, neighbour lists,
records: about 2 GB) is far larger than L2, so consecutive steps do not run
from cache.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp32|fp64] [--n 128]

Under torchrun (N > 1) the one 128^3 box is decomposed into N slab
subdomains, one per GPU (paper_1712_01294_gb300.decomp: ghost halos
exchanged and the step's minimum taken over NCCL every step): strong scaling,
the whole box's particle-updates/s over the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle (the only reference this
method has) on the host cores, on a bounded sample of the same workload.
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
sys.path.insert(0, ROOT)

METRIC = "MFM particle-updates/s at 128^3 (FP32 vs FP64 GPU, fwd & adjoint); % roofline"
UNIT = "particle-updates/s"
# Algorithmic FP32 operations per unordered flux pair (add, sub, mul, div and
# sqrt each count one; min/max/compare/select count zero), counted on the
# oracle's face routine: offsets 3, r^2 5, r 1, two kernel weights 28, two
# squares of H 2, two volumes 2, two B d 30, face area 15, |A| 6, s 2, v_f 9,
# normal 3, s_R 2, offsets 6, reconstruction 60, Hancock 37, v_f.n 5, u_L u_R
# 16, HLLC 30, rates 6, accumulation into both particles 8.
FLOPS_PER_PAIR = 276            # flux pass, per unordered pair
FLOPS_PER_DENSITY_TERM = 24     # density pass, per (particle, evaluation, neighbour)
FLOPS_PER_GRAD_NEIGHBOUR = 127  # gradient pass, per (particle, neighbour)
FLOPS_PER_GRAD_PARTICLE = 60    # gradient pass, per particle
# DRAM bytes (read + write) per work unit of each kernel, from the ncu capture
# summarised in TRAFFIC_SOURCE (64^3 turbulence, one launch each), scaled to a
# launch by the work units of the run; to be emptied whenever one of these
# kernels changes after that capture
TRAFFIC_PER_UNIT = {"density": 0.455, "gradients": 7.75, "fluxes": 20.41}
TRAFFIC_SOURCE = "profiles/kernels_turb64_fp32.md (64^3 capture, scaled by work units)"
FP32_LANES = 128  # FP32 lanes per SM (Blackwell)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--n", type=int, default=128, help="particles per axis")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cell-factor", type=float, default=None)
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="collectives of the decomposed box (N > 1); gloo moves the exchanges "
                         "through host memory, so that ranks may also share a GPU")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-path, adjoint and ensemble measurements")
    ap.add_argument("--extras", default="all", choices=["all", "adjoint", "variants", "hier"],
                    help="which extra measurements to run (adjoint: only the adjoint cost; "
                         "variants: only the MFV and exact-Riemann throughputs; hier: only the "
                         "hierarchical-timestep Sedov comparison)")
    return ap.parse_args()


def replica_aggregate(ms_local, dist=None, device="cpu"):
    """Max over ranks of the per-rank timings (each rank runs an independent
    replica of the workload; the slowest bounds the job).  ms_local: list of
    floats; returns the list of maxima (the input itself without dist)."""
    if dist is None:
        return list(ms_local)
    import torch
    t = torch.tensor(ms_local, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def replica_rate(world, n_per_rank, steps, ms_max):
    """Whole-job particle-updates/s: all ranks' particles over the slowest rank's time."""
    return world * n_per_rank * steps / (ms_max / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_decomposed(a, world, rank, local):
    """N > 1: the workload's box split into `world` slab subdomains, one per
    rank and GPU; warm-up, then K timed steps between barriers, CUDA events
    on each rank, the maximum over ranks."""
    import torch
    import torch.distributed as dist

    import paper_1712_01294_gb300 as gz
    from paper_1712_01294_gb300 import decomp as D
    from paper_1712_01294_gb300 import inputs as I

    ngpu = torch.cuda.device_count()
    dev = local % ngpu  # (more ranks than GPUs only with gloo: the ranks' kernels never wait on each other)
    if world > ngpu and a.dist_backend == "nccl":
        raise RuntimeError(f"{world} ranks on {ngpu} GPUs: NCCL needs one GPU per rank (--dist-backend gloo)")
    torch.cuda.set_device(dev)
    dist.init_process_group(a.dist_backend)
    prec = gz.GZ_FP64 if a.precision == "fp64" else gz.GZ_MIXED32
    p = I.turbulence(a.n, seed=1714)
    kw = {"precision": prec}
    if a.cell_factor:
        kw["cell_factor"] = a.cell_factor
    params = gz.default_params(**kw)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        box = D.DecomposedBox(gz.to_device(p, prec), p.N, world, D.DistComm(), params=params,
                              stream=stream)
        for _ in range(a.warmup):
            box.step()
        ctx = box.ctx[rank]
        st = ctx.status(reset=True)
        if not st["ok"]:
            raise RuntimeError(f"device status after warm-up: {st}")
        ctx.profile_read(reset=True)
        ctx.profile(True)
        launches0 = ctx.info()["launches"]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev) as clk:
            ev0.record(stream)
            for _ in range(a.steps):
                box.step()
            ev1.record(stream)
            torch.cuda.synchronize()
        dist.barrier()
        ms = ev0.elapsed_time(ev1)
        if box.ctx[rank] is not ctx:  # the subdomain outgrew its context during the timed steps
            ctx, launches0 = box.ctx[rank], 0
        launches = ctx.info()["launches"] - launches0
        prof = ctx.profile_read(reset=True)
        st = ctx.status(reset=True)
        if not st["ok"]:
            raise RuntimeError(f"device status after timed steps: {st}")
        held = int(box.owned[rank]["id"].numel())
    tmax = replica_aggregate([ms], dist, "cuda" if a.dist_backend == "nccl" else "cpu")[0]
    value = p.N * a.steps / (tmax / 1e3)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(tmax / a.steps, 4),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32" if prec == gz.GZ_MIXED32 else "f64", "data": "synthetic",
        "config": {"workload": f"turbulence {a.n}^3 = {p.N} particles, gamma 5/3, N_ngb 32, "
                               f"Mach 0.5, sigma_lnrho 0.3, CFL 0.2, global step",
                   "precision": a.precision, "parallelism": f"domain decomposition, {world} slabs",
                   "collectives": a.dist_backend, "gpus_seen": ngpu,
                   "owned_particles_rank0": held,
                   "l2": "working set far above the 129 MB L2; no flush needed"},
        "roofline": None,
        "pass_ms_per_step_rank0": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof.items() if v[1]},
        "e2e": {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "what": "measured at N = 1 (host-resident trajectories); the decomposed box stays "
                        "on the GPUs"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    box.close()
    dist.destroy_process_group()
    return line


def run_ours(a, world, rank, local):
    import numpy as np
    import torch

    import paper_1712_01294_gb300 as gz
    from paper_1712_01294_gb300 import inputs as I

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = gz.GZ_FP64 if a.precision == "fp64" else gz.GZ_MIXED32
    p = I.turbulence(a.n, seed=1714 + rank)
    N = p.N
    kw = {"precision": prec}
    if a.cell_factor:
        kw["cell_factor"] = a.cell_factor
    params = gz.default_params(**kw)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gz.Context([N], params, stream=stream)
        d0 = gz.to_device(p, prec)
        d = {k: v.clone() for k, v in d0.items()}
        dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(a.warmup):
            ctx.step(d, 0.0, dtu)
        st = ctx.status(reset=True)
        if not st["ok"]:
            raise RuntimeError(f"device status after warm-up: {st}")
        ctx.profile_read(reset=True)
        ctx.profile(True)
        launches0 = ctx.info()["launches"]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(a.steps):
                ctx.step(d, 0.0, dtu)
            ev1.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        launches = ctx.info()["launches"] - launches0
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        pairs = ctx.pair_count()
        # work units of the density and gradient passes: one density pass on a
        # copy of the state (the start of the next step), outside the timing
        dcopy = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in d.items()}
        _, iters = ctx.density(dcopy)
        nbr_counts, _ = ctx.neighbours(0)
        it64 = iters.to(torch.int64)
        nc64 = nbr_counts.to(torch.int64)
        work = {"density_eval_neighbours": int((it64 * nc64).sum()), "neighbours": int(nc64.sum()),
                "mean_iterations": round(float(it64.double().mean()), 3)}
        # the cell scan's candidates per true neighbour (overhead the density
        # pass's algorithmic FLOP count leaves out)
        sc = ctx.scan_stats()
        work["scan_candidates_per_particle"] = round(sc["candidates"] / p.N, 2)
        work["scan_candidates_per_neighbour"] = round(sc["candidates"] / max(sc["neighbours"], 1), 3)
        work["cached_per_particle"] = round(sc["within_cache_radius"] / p.N, 2)
        del dcopy
        st = ctx.status(reset=True)
        if not st["ok"]:
            raise RuntimeError(f"device status after timed steps: {st}")
        # end to end through the public API with host buffers: two independent
        # trajectories of the workload (this state and a second realisation)
        # live in pinned host memory and advance alternately; every step copies
        # its trajectory's current state in, steps it and copies the result
        # back over it, so the next step of that trajectory starts from there.
        # The copies of one trajectory run on a second stream while the other
        # trajectory's step computes (pipeline.pipelined_steps, one device
        # buffer per trajectory)
        from paper_1712_01294_gb300 import pipeline
        p2 = I.turbulence(a.n, seed=1714 + 1000 + rank)
        trajs = [{k: v.cpu().pin_memory() for k, v in d0.items()},
                 {k: v.cpu().pin_memory() for k, v in gz.to_device(p2, prec).items()}]
        h2d = sum(t.numel() * t.element_size() for t in trajs[0].values())
        d2h = sum(trajs[0][k].numel() * trajs[0][k].element_size() for k in pipeline.OUT_FIELDS)
        outs = [{k: t[k] for k in pipeline.OUT_FIELDS} for t in trajs]
        bufs = pipeline.device_buffers(trajs[0])
        cstream = torch.cuda.Stream()
        # one untimed pass through the pipeline (first use of the second buffer)
        pipeline.pipelined_steps(ctx, trajs, outs, 0.0, dtu, bufs, cstream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cstream.wait_event(e0)
        seq = [k % 2 for k in range(a.e2e_steps)]
        pipeline.pipelined_steps(ctx, [trajs[k] for k in seq], [outs[k] for k in seq], 0.0, dtu,
                                 bufs, cstream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1)
        st_e2e = ctx.status(reset=True)
        if not st_e2e["ok"]:
            raise RuntimeError(f"device status after the end-to-end steps: {st_e2e}")
        del bufs
        # the same steps launched as a CUDA graph: one step captured on a
        # second context and replayed (each replay a whole step, dt on the
        # device), from the state the timed loop started from; per-pass
        # profiling off, so no event records between the passes
        gctx = gz.Context([N], params, stream=stream)
        dg = {k: v.clone() for k, v in d0.items()}
        dtg = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(a.warmup):
            gctx.step(dg, 0.0, dtg)
        gctx.graph_capture(dg, 1, 0.0, dtg)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        g0.record(stream)
        for _ in range(a.steps):
            gctx.graph_launch()
        g1.record(stream)
        torch.cuda.synchronize()
        ms_graph = g0.elapsed_time(g1)
        st_g = gctx.status(reset=True)
        if not st_g["ok"]:
            raise RuntimeError(f"device status after the graph replays: {st_g}")
        gctx.close()
        del dg
        # measured throughput of the ALU pipes (outside every timed region):
        # context for the derived FP32 peak the roofline divides by
        alu = gz.measure_alu(stream)
        extras = {} if a.no_extras else measure_extras(a, ctx, d, dtu, stream, prec, p,
                                                       alu["fp64_fma_tflops"])
    tmax = ms
    if dist:
        tmax, ms_e2e, ms_graph = replica_aggregate([ms, ms_e2e, ms_graph], dist, "cuda")
    value = replica_rate(world, N, a.steps, tmax)
    e2e = replica_rate(world, N, a.e2e_steps, ms_e2e) if a.e2e_steps > 0 else None
    # roofline: each pair pass against the FP32 ALU peak, by its algorithmic
    # FLOP (counted on the oracle's routines); the dominant one by time is
    # the headline entry
    pk = peaks()
    clocks = clk.summary()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_fp32 = sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    flops = {"density": FLOPS_PER_DENSITY_TERM * work["density_eval_neighbours"],
             "gradients": FLOPS_PER_GRAD_NEIGHBOUR * work["neighbours"] + FLOPS_PER_GRAD_PARTICLE * N,
             "fluxes": FLOPS_PER_PAIR * (pairs // 2)}
    units = {"density": (work["density_eval_neighbours"], "particle-evaluation-neighbour terms",
                         FLOPS_PER_DENSITY_TERM),
             "gradients": (work["neighbours"], "particle-neighbour terms (+60 FLOP per particle)",
                           FLOPS_PER_GRAD_NEIGHBOUR),
             "fluxes": (pairs // 2, "unordered flux pairs", FLOPS_PER_PAIR)}
    kern = {"density": "k_density", "gradients": "k_gradients", "fluxes": "k_fluxes"}
    kernels = []
    for name in ("density", "gradients", "fluxes"):
        ms_k = prof[name][0] / max(prof[name][1], 1)
        ach = flops[name] / (ms_k / 1e3) / 1e12
        kernels.append({"kernel": kern[name], "bound": "alu", "achieved": round(ach, 3),
                        "peak": round(peak_fp32, 2), "unit": "TFLOP/s", "frac": round(ach / peak_fp32, 4),
                        "avg_launch_ms": round(ms_k, 4), "units_per_launch": units[name][0],
                        "unit_kind": units[name][1], "flop_per_unit": units[name][2],
                        "traffic": TRAFFIC_PER_UNIT.get(name) and round(TRAFFIC_PER_UNIT[name] * units[name][0]),
                        "traffic_source": TRAFFIC_SOURCE if name in TRAFFIC_PER_UNIT else None})
    roof = dict(max(kernels, key=lambda k: k["avg_launch_ms"]))
    dom = max(("density", "gradients", "fluxes", "sort", "update"), key=lambda k: prof[k][0])
    roof["peak_basis"] = f"{sms} SMs x {FP32_LANES} FP32 lanes x 2 x {sm_max:.0f} MHz (ALU, not tensor)"
    roof["peak_measured"] = alu["fp32_fma_tflops"]
    roof["frac_of_measured"] = round(roof["achieved"] / alu["fp32_fma_tflops"], 4)
    shares = {k: round(v[0] / max(sum(x[0] for x in prof.values()), 1e-9), 4) for k, v in prof.items()
              if v[1]}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(tmax / a.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == gz.GZ_MIXED32 else "f64", "data": "synthetic",
        "config": {"workload": f"turbulence {a.n}^3 = {N} particles, gamma 5/3, N_ngb 32, "
                               f"Mach 0.5, sigma_lnrho 0.3, CFL 0.2, global step",
                   "precision": a.precision, "particles_per_gpu": N,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set (~2 GB) far above the 129 MB L2; no flush needed"},
        "roofline": roof,
        "roofline_kernels": kernels,
        "work": work,
        "pass_ms_per_step": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof.items() if v[1]},
        "pass_share": shares, "dominant_pass": dom,
        "e2e": {"value": round(e2e, 1) if e2e else None, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": a.e2e_steps,
                "what": "two trajectories in pinned host memory advanced alternately: each step copies "
                        "its trajectory's state in, steps it, copies the result back over it; one "
                        "trajectory's copies overlap the other's step"},
        "gpu_launches": launches,
        "graph_replay": {"value": round(replica_rate(world, N, a.steps, ms_graph), 1), "unit": UNIT,
                         "ms_per_step": round(ms_graph / a.steps, 4), "steps": a.steps,
                         "what": "the same steps from the same state, one step captured as a CUDA graph "
                                 "and replayed (per-pass profiling off); the headline times plain "
                                 "gz_step calls with the per-pass CUDA-event profile on"},
        "alu_peaks_measured": dict(alu, how="gz_measure_alu: independent FMA / rsqrt chains, 64 warps "
                                            "per SM, best of 3 launches"),
        "clocks": clocks,
    }
    line.update(extras)
    if "fp64_path" in line:
        line["fp64_path"]["fp32_over_fp64"] = round(value / world / line["fp64_path"]["value"], 2)
    for key in ("mfv", "riemann_exact", "riemann_fallback"):
        if key in line:
            line[key]["ms_over_mfm"] = round(line[key]["ms_per_step"] / (tmax / a.steps), 3)
    if "adjoint" in line:
        adj = line["adjoint"]
        adj["forward_ms_per_step"] = round(tmax / a.steps, 4)
        # (forward that saves the checkpoint + backward) / plain forward, the
        # plain forward timed on the same states (those after the timed steps)
        adj["total_over_forward"] = round(
            (adj["forward_with_checkpoint_ms_per_step"] + adj["backward_ms_per_step"])
            / adj["forward_same_states_ms_per_step"], 3)
    # the metric's other arms on the same workload, kept beside the workload
    # description: the FP64 GPU path, the adjoint step and the graph replay
    comp = {}
    if "fp64_path" in line:
        f64 = line["fp64_path"]
        comp["fp64_path"] = {"value": f64["value"], "ms_per_step": f64["ms_per_step"],
                             "fp32_over_fp64": f64["fp32_over_fp64"]}
    if "adjoint" in line:
        adj = line["adjoint"]
        comp["adjoint"] = {"total_over_forward": adj["total_over_forward"],
                           "backward_ms_per_step": adj["backward_ms_per_step"],
                           "forward_with_checkpoint_ms_per_step": adj["forward_with_checkpoint_ms_per_step"],
                           "forward_same_states_ms_per_step": adj["forward_same_states_ms_per_step"]}
    comp["graph_replay"] = {"value": line["graph_replay"]["value"],
                            "ms_per_step": line["graph_replay"]["ms_per_step"]}
    line["config"]["companions"] = comp
    return line, p


def measure_extras(a, ctx, d, dtu, stream, prec, p, fp64_peak=None):
    """Adjoint cost, MFV and exact-Riemann throughputs, the evolved state, FP64-path throughput
    and the batched ensemble (CUDA graph)."""
    import numpy as np
    import torch

    import paper_1712_01294_gb300 as gz
    from paper_1712_01294_gb300 import autotune
    from paper_1712_01294_gb300 import inputs as I
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        if a.extras in ("all", "adjoint"):
            # adjoint of one step (same workload, same precision), dt frozen, in the
            # configuration MFMStep runs it: the forward fills the step checkpoint
            # (gz_step_checkpoint at GZ_CKPT_LISTS: rates, the gradient pass's
            # per-particle outputs, the sorted order, n and the neighbour lists)
            # and returns the converged H; the backward recomputes the reverse
            # lists and every pair quantity
            rng = np.random.default_rng(0)
            T = d["x"].dtype
            start = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in d.items()}
            level = gz.GZ_CKPT_LISTS
            ck = ctx.new_checkpoint(level)
            K = max(2, a.steps // 2)
            # the plain forward over the same K steps (the denominator of the
            # cost ratio: the same states as the checkpointing forward below)
            fwd = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in start.items()}
            ctx.step(fwd, 0.0, dtu)
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(K):
                ctx.step(fwd, 0.0, dtu)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_fwd_plain = e0.elapsed_time(e1) / K
            fwd = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in start.items()}
            ctx.step(fwd, 0.0, dtu, ck, level)
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(K):
                ctx.step(fwd, 0.0, dtu, ck, level)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_fwd_ckpt = e0.elapsed_time(e1) / K
            fwd = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in start.items()}
            ctx.step(fwd, 0.0, dtu, ck, level)
            dt = float(dtu.item())
            ckstate = dict(start)
            ckstate["h"] = fwd["h"]
            gend = {k: torch.as_tensor(rng.normal(size=p.N), dtype=T).cuda() for k in
                    ("x", "y", "z", "vx", "vy", "vz", "u")}
            gstart = {k: torch.zeros(p.N, dtype=T, device="cuda") for k in
                      ("x", "y", "z", "vx", "vy", "vz", "u", "m")}
            ctx.step_backward(ckstate, dt, gend, gstart, ck, level)
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(K):
                ctx.step_backward(ckstate, dt, gend, gstart, ck, level)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_bwd = e0.elapsed_time(e1) / K
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(K):
                ctx.step_backward(start, dt, gend, gstart)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_bwd_full = e0.elapsed_time(e1) / K
            st = ctx.status(reset=True)
            out["adjoint"] = {"backward_ms_per_step": round(ms_bwd, 4),
                              "forward_with_checkpoint_ms_per_step": round(ms_fwd_ckpt, 4),
                              "forward_same_states_ms_per_step": round(ms_fwd_plain, 4),
                              "checkpoint_bytes_per_particle": round(ctx.checkpoint_bytes(level) / p.N, 1),
                              "backward_full_recompute_ms_per_step": round(ms_bwd_full, 4),
                              "steps": K, "status_ok": st["ok"],
                              "what": "gz_step_backward from the MFMStep checkpoint at GZ_CKPT_LISTS "
                                      "(start state, converged H, n, rates, gradient-pass outputs, the "
                                      "sorted order and the lists' first 64 slots): the reverse pair "
                                      "lists and all pair quantities recomputed, then the adjoint "
                                      "passes"}
            del ck
        if a.extras == "adjoint":
            return out
        # the scheme variants on the same workload and precision: MFV (mass
        # fluxes through moving faces) and the MFM face with the exact Riemann
        # solver on every face; full steps, per-pass split
        variants = (("mfv", {"scheme": gz.GZ_MFV}), ("riemann_exact", {"riemann": gz.GZ_RIEMANN_EXACT}),
                    ("riemann_fallback", {"riemann": gz.GZ_RIEMANN_FALLBACK}))
        for key, kw in (variants if a.extras in ("all", "variants") else ()):
            if a.cell_factor:
                kw = dict(kw, cell_factor=a.cell_factor)
            cm = gz.Context([p.N], gz.default_params(precision=prec, **kw), stream=stream)
            dv = gz.to_device(p, prec)
            for _ in range(3):
                cm.step(dv, 0.0, dtu)
            cm.profile(True)
            K = max(3, a.steps)
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(K):
                cm.step(dv, 0.0, dtu)
            e1.record(stream)
            torch.cuda.synchronize()
            prof_m = cm.profile_read(reset=True)
            cm.profile(False)
            ms_m = e0.elapsed_time(e1) / K
            out[key] = {"value": round(p.N / (ms_m / 1e3), 1), "unit": UNIT,
                        "ms_per_step": round(ms_m, 4), "steps": K, "steps_before": 3,
                        "status_ok": cm.status(reset=True)["ok"],
                        "pass_ms_per_step": {k: round(v[0] / max(v[1], 1), 4)
                                             for k, v in prof_m.items() if v[1]}}
            cm.close()
            del dv
        if a.extras == "variants":
            return out
        if a.extras in ("all", "hier"):
            out["hierarchical"] = measure_hier(a, stream, prec)
        if a.extras == "all":
            # the other configured workloads at the same precision, one box
            # each: 10 steps from the initial state, after 2 steps on a copy
            cfg = {}
            for name in ("sod32", "sedov64", "kh64"):
                q = I.WORKLOADS[name]()
                c2 = gz.Context([q.N], gz.default_params(precision=prec), stream=stream)
                warm = gz.to_device(q, prec)
                for _ in range(2):
                    c2.step(warm)
                dd = gz.to_device(q, prec)
                t2 = torch.zeros(1, dtype=torch.float64, device="cuda")
                e0, e1 = ev(), ev()
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(10):
                    c2.step(dd, 0.0, t2)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 10
                cfg[name] = {"particles": q.N, "value": round(q.N / (ms / 1e3), 1), "unit": UNIT,
                             "ms_per_step": round(ms, 4), "steps": 10,
                             "status_ok": c2.status(reset=True)["ok"]}
                c2.close()
            out["configs"] = cfg
        if a.extras == "hier":
            return out
        # the same box further on: 20 more steps from the state the timed loop
        # left, when the particles have left the initial lattice (whose regular
        # cell occupancy the density scan profits from), then 10 timed
        ev_state = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in d.items()}
        for _ in range(20):
            ctx.step(ev_state, 0.0, dtu)
        ctx.profile_read(reset=True)
        ctx.profile(True)
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(10):
            ctx.step(ev_state, 0.0, dtu)
        e1.record(stream)
        torch.cuda.synchronize()
        prof_ev = ctx.profile_read(reset=True)
        ctx.profile(False)
        ms_ev = e0.elapsed_time(e1) / 10
        out["evolved_state"] = {"value": round(p.N / (ms_ev / 1e3), 1), "unit": UNIT,
                                "ms_per_step": round(ms_ev, 4), "steps_before": a.warmup + a.steps + 20,
                                "steps": 10, "status_ok": ctx.status(reset=True)["ok"],
                                "pass_ms_per_step": {k: round(v[0] / max(v[1], 1), 4)
                                                     for k, v in prof_ev.items() if v[1]}}
        del ev_state
        # FP64 path on the same workload
        if prec == gz.GZ_MIXED32:
            c64 = gz.Context([p.N], gz.default_params(precision=gz.GZ_FP64), stream=stream)
            d64 = gz.to_device(p, gz.GZ_FP64)
            c64.step(d64)
            c64.profile(True)
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(3):
                c64.step(d64)
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1) / 3
            prof64 = c64.profile_read(reset=True)
            c64.profile(False)
            pass64 = {k: round(v[0] / max(v[1], 1), 3) for k, v in prof64.items() if v[1]}
            # the flux pass against the measured FP64 FMA rate, by the same
            # algorithmic FLOP as the FP32 roofline
            pairs64 = c64.pair_count() // 2
            ach64 = pairs64 * FLOPS_PER_PAIR / (pass64["fluxes"] / 1e3) / 1e12
            out["fp64_path"] = {"value": round(p.N / (ms64 / 1e3), 1), "unit": UNIT,
                                "ms_per_step": round(ms64, 3), "steps": 3, "pass_ms_per_step": pass64,
                                "fluxes_roofline": {"bound": "alu (FP64)", "achieved": round(ach64, 4),
                                                    "peak_measured": fp64_peak, "unit": "TFLOP/s",
                                                    "frac": round(ach64 / fp64_peak, 4) if fp64_peak else None},
                                "status_ok": c64.status(reset=True)["ok"]}
            c64.close()
            del d64
        # batched ensemble: 256 boxes, 20 steps captured as one CUDA graph
        ens = I.ensemble(256, seed=1716)
        counts = [int(c) for c in ens.counts]
        # tuned on the configured run itself: its 20 steps from the initial state
        (cf, dc), tune_ms = autotune.tune(ens, gz.GZ_MIXED32, candidates=(0.85, 1.0, 1.2), caches=(40, 48),
                                          steps=20, warmup=0, use_cache=False)
        ce = gz.Context(counts, gz.default_params(precision=gz.GZ_MIXED32, cell_factor=cf, density_cache=dc),
                        stream=stream)
        d_init = gz.to_device(ens, gz.GZ_MIXED32)
        de = {k: v.clone() for k, v in d_init.items()}
        dte = torch.zeros(len(counts), dtype=torch.float64, device="cuda")
        ce.graph_capture(de, 20, 0.0, dte)
        # every replay is the configured run: the 20 steps from the initial
        # state (restored outside the timed region)
        R, msg = 3, 0.0
        l1 = None
        for r in range(R + 1):
            for k in de:
                de[k].copy_(d_init[k])
            if r == 1:
                l1 = ce.info()["launches"]
            e0, e1 = ev(), ev()
            e0.record(stream)
            ce.graph_launch()
            e1.record(stream)
            torch.cuda.synchronize()
            if r > 0:
                msg += e0.elapsed_time(e1) / R
        per_graph = (ce.info()["launches"] - l1) // R
        # the same 20 steps launched one kernel at a time, per-pass profile
        # (what a graph saves; where the time goes)
        for k in de:
            de[k].copy_(d_init[k])
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(20):
            ce.step(de, 0.0, dte)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_direct = e0.elapsed_time(e1)
        for k in de:
            de[k].copy_(d_init[k])
        ce.profile_read(reset=True)
        ce.profile(True)
        for _ in range(20):
            ce.step(de, 0.0, dte)
        prof_e = ce.profile_read(reset=True)
        ce.profile(False)
        ntot = sum(counts)
        out["ensemble"] = {"value": round(ntot * 20 / (msg / 1e3), 1), "unit": UNIT,
                           "direct_launch_ms": round(ms_direct, 3),
                           "pass_ms_per_step": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof_e.items()
                                                if v[1]},
                           "boxes": len(counts), "particles": ntot, "steps_per_graph": 20,
                           "ms_per_graph": round(msg, 3), "graph_replays": R,
                           "kernels_per_graph": per_graph,
                           "cell_factor": cf, "density_cache": dc,
                           "tuning_ms_per_step": {f"{k[0]},{k[1]}": round(v, 3) for k, v in tune_ms.items()},
                           "what": "each replay: the 20 steps of the configuration from the initial state",
                           "status_ok": ce.status(reset=True)["ok"]}
        ce.close()
    return out


def measure_hier(a, stream, prec, K=5, intervals=3):
    """Sedov blast at the workload's particle count: time to advance the same
    physical time with hierarchical power-of-two steps (gz_step_hier, K bins,
    `intervals` sync intervals) and with global CFL steps (gz_step)."""
    import torch

    import paper_1712_01294_gb300 as gz
    from paper_1712_01294_gb300 import inputs as I
    ev = lambda: torch.cuda.Event(enable_timing=True)
    sed = I.sedov(a.n)
    N = sed.N
    kw = {"cell_factor": a.cell_factor} if a.cell_factor else {}
    with torch.cuda.stream(stream):
        ch = gz.Context([N], gz.default_params(precision=prec, **kw), stream=stream)
        D = torch.zeros(1, dtype=torch.float64, device="cuda")
        dw = gz.to_device(sed, prec)
        ch.step_hier(dw, K, 0.0, D)  # warm-up (allocates the scratch)
        dh = gz.to_device(sed, prec)
        ch.profile_read(reset=True)
        ch.profile(True)
        e0, e1 = ev(), ev()
        e0.record(stream)
        t_h, active = 0.0, 0
        for _ in range(intervals):
            active += ch.step_hier(dh, K, 0.0, D)
            t_h += float(D.item())
        e1.record(stream)
        torch.cuda.synchronize()
        ms_h = e0.elapsed_time(e1)
        prof = ch.profile_read(reset=True)
        ch.profile(False)
        st_h = ch.status(reset=True)["ok"]
        cg = gz.Context([N], gz.default_params(precision=prec, **kw), stream=stream)
        dg = gz.to_device(sed, prec)
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        cg.step(dg, 0.0, dt)  # warm-up on a copy
        dg = gz.to_device(sed, prec)
        steps, t_g = 0, 0.0
        e0, e1 = ev(), ev()
        e0.record(stream)
        while t_g < t_h and steps < 2000:
            cg.step(dg, 0.0, dt)
            t_g += float(dt.item())
            steps += 1
        e1.record(stream)
        torch.cuda.synchronize()
        ms_g = e0.elapsed_time(e1)
        st_g = cg.status(reset=True)["ok"]
        ch.close()
        cg.close()
    return {"workload": f"Sedov blast {a.n}^3 = {N} particles, E = 1 in the 32 central particles",
            "K": K, "intervals": intervals, "physical_time": round(t_h, 8),
            "hier_ms": round(ms_h, 3), "global_steps": steps, "global_time": round(t_g, 8),
            "global_ms": round(ms_g, 3), "speedup": round(ms_g / ms_h, 2),
            "active_particle_substeps": active,
            "active_fraction": round(active / (N * intervals * (1 << K)), 4),
            "hier_pass_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
            "status_ok": st_h and st_g,
            "what": "wall time (CUDA events) to advance the same physical time; the hierarchical "
                    "call synchronises the host once per substep"}


def cpu_sample_rate(p, threads=None, sample_frac=1.0 / 8):
    """Oracle throughput on a bounded sample: every pass runs on the particles
    it needs for a cubic sub-box holding ~sample_frac of the particles (plus
    the halo that the pass's inputs need); rate = 1 / sum_pass (time / count)."""
    import numpy as np

    import oracle as O
    if threads:
        O.set_threads(threads)
    s = O.State.from_any(p.__dict__)
    prm = O.params()
    side = sample_frac ** (1.0 / 3.0)
    Hm = 1.3 * float(np.max(s.H))

    def region(pad):
        lo, hi = -pad, side + pad
        ok = np.ones(s.N, dtype=bool)
        for c in (s.x, s.y, s.z):
            w = np.where(c > 0.5 + side / 2, c - 1.0, c)
            ok &= (w >= lo) & (w < hi)
        return ok

    m_f, m_g, m_d = region(0.0), region(2.2 * Hm), region(4.4 * Hm)
    t = {}
    t0 = time.perf_counter()
    H, n, it, _ = O.density(s, prm, mask=m_d)
    t["density"] = (time.perf_counter() - t0, int(m_d.sum()))
    H = np.where(m_d, H, s.H)
    n = np.where(m_d, n, 1.0)
    t0 = time.perf_counter()
    g = O.gradients(s, H, n, prm, mask=m_g)
    t["gradients"] = (time.perf_counter() - t0, int(m_g.sum()))
    t0 = time.perf_counter()
    O.timestep(s, H, n, prm, mask=m_f)
    t["timestep"] = (time.perf_counter() - t0, int(m_f.sum()))
    t0 = time.perf_counter()
    dp, dE = O.fluxes(s, H, n, g["grad"], g["B"], 1e-4, prm, mask=m_f)
    t["fluxes"] = (time.perf_counter() - t0, int(m_f.sum()))
    t0 = time.perf_counter()
    O.update(s, dp, dE, 1e-4, prm)
    t["update"] = (time.perf_counter() - t0, s.N)
    per = sum(v[0] / max(v[1], 1) for v in t.values())
    total = sum(v[0] for v in t.values())
    return 1.0 / per, total, int(m_f.sum()), O.num_threads()


def main():
    a = parse()
    world, rank, local = dist_env()
    if a.impl == "reference":
        if rank != 0:
            return 0
        from paper_1712_01294_gb300 import inputs as I
        p = I.turbulence(a.n, seed=1714)
        rates, walls = [], []
        for _ in range(a.warmup):
            cpu_sample_rate(p)
        for _ in range(a.steps):
            t0 = time.perf_counter()
            r, secs, ns, cores = cpu_sample_rate(p)
            walls.append(time.perf_counter() - t0)
            rates.append(r)
        v = statistics.median(rates)
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT,
                "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": round(statistics.median(walls) * 1e3, 2), "sampled": True,
                "full_step_ms_extrapolated": round(p.N / v * 1e3, 2),
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"turbulence {a.n}^3 = {p.N} particles, gamma 5/3, N_ngb 32, "
                                       f"Mach 0.5, sigma_lnrho 0.3, CFL 0.2, global step",
                           "precision": "fp64 (the oracle)", "particles_per_gpu": p.N,
                           "parallelism": "single",
                           "sample": "each step is a bounded sample: every pass on a cubic sub-box of "
                                     "1/8 of the state (plus the halo it needs); ms_per_step is the "
                                     "wall time of that sample, value its rate"},
                "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"each pass on a cubic sub-box of ~{ns} particles plus its "
                                           f"halo; rate = 1/sum(time/particles) over passes"},
                "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        line = run_decomposed(a, world, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    line, p = run_ours(a, world, rank, local)
    if rank == 0:
        if world == 1 and not a.no_cpu_baseline:
            r, secs, ns, cores = cpu_sample_rate(p, sample_frac=1.0)
            line["cpu_baseline"] = {"value": round(r, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"one full oracle step of the same {ns}-particle state "
                                              f"(density, gradients, timestep, fluxes, update), "
                                              f"{secs:.1f} s of CPU wall time"}
            # the same oracle on one host core, on a cubic sub-box of 1/64 of
            # the state (each pass on the particles it needs there)
            import oracle as O
            r1, secs1, ns1, _ = cpu_sample_rate(p, threads=1, sample_frac=1.0 / 64)
            O.set_threads(cores)
            line["cpu_baseline_1thread"] = {"value": round(r1, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                                            "sample": f"one oracle step of a cubic sub-box of {ns1} particles "
                                                      f"of the same state, {secs1:.1f} s"}
            if "configs" in line:
                # the oracle on the other configured workloads: one full step
                # from each initial state on all host cores
                from paper_1712_01294_gb300 import inputs as I
                cb = {}
                for name, g in line["configs"].items():
                    rc, secsc, nsc, _ = cpu_sample_rate(I.WORKLOADS[name](), sample_frac=1.0)
                    cb[name] = {"value": round(rc, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"one full oracle step of the {nsc}-particle initial state, "
                                          f"{secsc:.1f} s",
                                "gpu_over_oracle": round(g["value"] / rc, 1)}
                line["cpu_baseline_configs"] = cb
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
