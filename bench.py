#!/usr/bin/env python
"""Throughput of distilled multi-time-step MD (Algorithm 1) on one GB300.

One timed step is one outer step of Algorithm 1 on the synthetic
12,288-atom water box (4,096 rigid-geometry waters, L = 49.7 A): n_inner
small-model (3.5 A) neighbour lists + force evaluations with their kicks and
drifts, then one big-model (5.0 A) neighbour list + force evaluation and the
closing half-kick, all through the C ABI (dmts_respa_step). The baseline is
plain 1 fs velocity Verlet with the big model alone, timed the same way.

Prints one JSON line. ``value`` is DMTS ns/day (whole job: with N GPUs every
rank runs its own replica, so simulated time adds up). The L2 cache (129 MB)
is flushed between timed steps by writing a 256 MB buffer on the same stream;
each step is timed with CUDA events on the library's stream.

``--impl reference`` times the FP64 CPU oracle (the plain definition of the
same step) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DMTS ns/day and atom-force evals/s vs plain 1 fs NNP MD on same GB300"
FS_PER_NS = 1e6
SEC_PER_DAY = 86400.0
# FP32 SIMT peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) at the
# maximum SM clock of 2,070 MHz.
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def measured_peak(key: str, fallback: float = 1900.0) -> float:
    """A figure from MEASURED_PEAKS.json (written per pod), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return fallback


def workload(name: str):
    from paper_2510_06562_gb300 import inputs as I
    if name == "water12288":
        return I.water_12288(0)
    if name == "water192":
        return I.water_192(0)
    raise SystemExit(f"unknown workload {name}")


def step_config(args, s, world: int) -> dict:
    """The timed workload: the water box by name and size, the RESPA split,
    the two models and how a step is measured. Both arms print this same
    object; the arithmetic each arm computes in is its ``dtype``."""
    return {"workload": f"{args.workload}: {s.n_atoms // 3:,} rigid waters, {s.n_atoms:,} atoms, "
                        f"L={s.box[0]:.1f} A, periodic",
            "outer_fs": args.outer_fs, "inner_fs": args.outer_fs / args.n_inner, "n_inner": args.n_inner,
            "small_model": "3.5 A, K=8, 1 layer, F=32", "big_model": "5.0 A, K=16, 2 layers, F=64",
            "state": "FP64 x, v",
            "l2": "GPU: flushed (256 MB write) before every timed step; host: not applicable",
            "parallelism": f"replicas{world}"}


def models(n_species: int):
    from paper_2510_06562_gb300 import inputs as I
    return (I.small_arch(n_species), I.init_params(I.small_arch(n_species), 2),
            I.big_arch(n_species), I.init_params(I.big_arch(n_species), 3))


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

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
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------- GPU arm
WINDOW_FS = 60.0


def time_steps(ctx, torch, stream, flush, n_steps, dt, n_inner, x0, v0):
    """Per-step CUDA-event times (ms) of n_steps single outer steps, with the
    L2 flushed before each step (outside the timed window).

    The random-init models conserve energy for ~120-200 fs before the system
    collapses into a dense many-neighbour well, so the timed steps are taken
    in windows of WINDOW_FS simulated fs that restart from the initial state
    (x0, v0); the restart and the first step after it (which re-evaluates
    both models) are not timed."""
    ms = []
    launches = 0
    per_window = max(1, int(WINDOW_FS / dt))
    for k in range(n_steps):
        if k % per_window == 0:
            ctx.set_state(x0, v0)
            ctx.respa_step(1, dt, n_inner, energies=False)
        with torch.cuda.stream(stream):
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        n0 = ctx.launch_count
        a.record(stream)
        ctx.respa_step(1, dt, n_inner, energies=False)
        b.record(stream)
        launches += ctx.launch_count - n0
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms, launches


def max_over_ranks(values, dist, device="cpu"):
    """Element-wise maximum of per-rank timings (every rank gets the result);
    with one process, the values themselves."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_ns_per_day(world, steps, dt_fs, t_max_s):
    """Whole-job simulated time per day of `world` independent replicas, each
    running `steps` steps of dt_fs in at most t_max_s seconds."""
    return world * steps * dt_fs / FS_PER_NS / t_max_s * SEC_PER_DAY


def measure(D, I, torch, s, models_, prec, args, flush, dt, n_inner, seed):
    """DMTS (dt / n_inner) and 1 fs STS throughput of one precision on one
    system, per-stage times and the dominant kernel's roofline."""
    sa, sp, ba, bp = models_
    v0 = I.maxwell_boltzmann(s.mass, 300.0, seed, s.atom_offset)
    N = s.n_atoms
    ctx = D.Context(s, ba, bp, sa, sp, precision=prec)
    sts = D.Context(s, ba, bp, precision=prec)
    stream = torch.cuda.ExternalStream(ctx.stream)
    sstream = torch.cuda.ExternalStream(sts.stream)
    ctx.set_state(s.x, v0)
    sts.set_state(s.x, v0)
    ctx.respa_step(args.warmup, dt, n_inner, energies=False)
    sts.respa_step(args.warmup, 1.0, 1, energies=False)
    torch.cuda.synchronize()
    ms_dmts, launches = time_steps(ctx, torch, stream, flush, args.steps, dt, n_inner, s.x, v0)
    ms_sts, _ = time_steps(sts, torch, sstream, flush, args.steps, 1.0, 1, s.x, v0)
    k6 = max(3, args.steps // 2)
    ctx.respa_step(3, 6.0, 6, energies=False)
    ms6, _ = time_steps(ctx, torch, stream, flush, k6, 6.0, 6, s.x, v0)
    out = {"t_dmts": sum(ms_dmts) / 1e3, "t_sts": sum(ms_sts) / 1e3, "t6": sum(ms6) / 1e3, "k6": k6,
           "launches": launches, "ctx": ctx, "sts": sts, "v0": v0}
    out["stages_big"] = ctx.time_stages(D.BIG, reps=20)
    out["stages_small"] = ctx.time_stages(D.SMALL, reps=20)
    out["pairs_big"] = int(ctx.neighbors(D.BIG)[0][-1])
    out["pairs_small"] = int(ctx.neighbors(D.SMALL)[0][-1])
    out["tuning"] = {"big": ctx.tuning(D.BIG), "small": ctx.tuning(D.SMALL)}
    return out


KERNEL_OF_STAGE = {
    # (precision is BF16, stage name or prefix) -> (kernel name in the ncu capture, source file);
    # the tensor-core backward pass has a layer-0 variant (two MMA groups per tile)
    (True, "edge_bwd_l0"): ("k_edge_bwd_grp<64,3,2,16,1>", "potential_bf16.cu"),
    (True, "edge_bwd"): ("k_edge_bwd_grp<64,3,2,16,0>", "potential_bf16.cu"),
    (True, "edge_fwd"): ("k_edge_fwd_bf16<64,16>", "potential_bf16.cu"),
    (False, "edge_bwd"): ("k_edge_bwd<64,16>", "potential_f32.cu"),
    (False, "edge_fwd"): ("k_edge_fwd<64,16>", "potential_f32.cu"),
}


def captured_traffic(kernel: str, source: str, pairs: int, root: str = ROOT):
    """DRAM bytes per launch of `kernel` (template arguments without spaces)
    from a committed ncu summary under profiles/ (a line `counters:
    kernel=... source_sha256=... dram_bytes_per_launch=... pairs=...`), or
    None when there is none, the kernel's source changed since the capture,
    or the capture was of another workload (pair count more than 1% away:
    the count of one box drifts a little with the dynamics)."""
    src = os.path.join(root, "paper_2510_06562_gb300", "csrc", source)
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    pdir = os.path.join(root, "profiles")
    for name in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        for line in open(os.path.join(pdir, name), errors="replace"):
            if "counters:" not in line:
                continue
            fields = dict(kv.split("=", 1) for kv in line.split("counters:", 1)[1].split() if "=" in kv)
            if (fields.get("kernel") == kernel and fields.get("source_sha256") == sha
                    and "dram_bytes_per_launch" in fields and "pairs" in fields
                    and abs(int(fields["pairs"]) - pairs) <= 0.01 * pairs):
                return float(fields["dram_bytes_per_launch"])
    return None


def roofline_of(D, prec, stages_big, E_big, ba):
    dom = max((k for k in stages_big if k.startswith("edge_")), key=lambda k: stages_big[k])
    K, F = ba.n_radial, ba.n_feat
    if prec == D.FP32:
        flop_edge = 2 * (2 * K * F + 2 * F * F) if dom.startswith("edge_bwd") else 2 * (K * F + F * F)
        peak, bound, src, kind = FP32_SIMT_TFLOPS, "alu", "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz", "FP32 SIMT"
    else:
        # the algorithmic edge-GEMM work per pair and layer, K padded to 16: one pass 2F(16 + F) forward,
        # two backward (the adjoint and the recomputed filter). The layer-0 backward kernel skips the
        # recomputation and issues 2 (2 * 16 F + F^2); the figure stays the algorithm's.
        flop_edge = 2 * (2 * 16 * F + 2 * F * F) if dom.startswith("edge_bwd") else 2 * (16 * F + F * F)
        peak, bound, src, kind = measured_peak("bf16_tflops"), "tensor", "MEASURED_PEAKS.json bf16_tflops (burst)", "BF16 tcgen05"
    achieved = flop_edge * E_big / (stages_big[dom] * 1e-3) / 1e12
    bf16 = prec != D.FP32
    kname, ksrc = KERNEL_OF_STAGE.get((bf16, dom)) or KERNEL_OF_STAGE[(bf16, dom[:8])]
    return {"kernel": f"{dom} (big model, {kind})", "bound": bound, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": captured_traffic(kname, ksrc, E_big),
            "algorithmic_flop_per_launch": flop_edge * E_big, "launch_ms": stages_big[dom], "peak_source": src}


def run_ours(args):
    import torch

    from paper_2510_06562_gb300 import build as B
    from paper_2510_06562_gb300 import dmts as D
    from paper_2510_06562_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    s = workload(args.workload)
    mdl = models(s.n_species)
    sa, sp, ba, bp = mdl
    N = s.n_atoms
    dt, n_inner = args.outer_fs, args.n_inner
    main_prec = D.BF16_MLP if args.precision == "bf16" else D.FP32
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    res = {main_prec: measure(D, I, torch, s, mdl, main_prec, args, flush, dt, n_inner, 1 + rank)}
    other = D.FP32 if main_prec == D.BF16_MLP else D.BF16_MLP
    if not args.single_precision:
        res[other] = measure(D, I, torch, s, mdl, other, args, flush, dt, n_inner, 1 + rank)
    torch.cuda.synchronize()
    clk = clocks.stop()

    def agg(r):
        t_dmts, t_sts, t6 = max_over_ranks([r["t_dmts"], r["t_sts"], r["t6"]], dist, "cuda")
        return {"dmts_ns_per_day": replica_ns_per_day(world, args.steps, dt, t_dmts),
                "sts_1fs_ns_per_day": replica_ns_per_day(world, args.steps, 1.0, t_sts),
                "dmts_6fs_ns_per_day": replica_ns_per_day(world, r["k6"], 6.0, t6),
                "atom_force_evals_per_s": world * args.steps * (n_inner + 1) * N / t_dmts,
                "ms_per_step": t_dmts * 1e3 / args.steps, "ms_per_step_sts": t_sts * 1e3 / args.steps}

    main = res[main_prec]
    m = agg(main)
    r = main["ctx"]
    # end to end through the public API with host buffers: upload state,
    # one outer step, read energies and state back (each step)
    xh = torch.tensor(s.x).pin_memory()
    vh = torch.tensor(main["v0"]).pin_memory()
    eh = torch.empty((1, s.n_systems, 3), dtype=torch.float64).pin_memory()
    k_e2e = max(3, args.steps // 4)
    # one untimed round trip: the first upload moves the atoms back to the
    # start, so that step re-evaluates both models (Algorithm 1's first step)
    r.set_state(xh, vh)
    r.respa_step(1, dt, n_inner, out=eh)
    r.get_state(xh, vh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        r.set_state(xh, vh)
        r.respa_step(1, dt, n_inner, out=eh)
        r.get_state(xh, vh)
    t_e2e = time.perf_counter() - t0
    e2e = {"value": world * k_e2e * dt / FS_PER_NS / t_e2e * SEC_PER_DAY, "unit": "ns/day",
           "h2d_bytes_per_step": 2 * N * 3 * 8, "d2h_bytes_per_step": 2 * N * 3 * 8 + 3 * 8 * s.n_systems,
           "steps": k_e2e,
           "note": ("every step: x and v uploaded from pinned host buffers (dmts_set_state), one outer step, "
                    "energies and x, v read back; positions equal to the device's keep the cached forces")}

    extras = {}
    if not args.single_precision:
        o = agg(res[other])
        o["stage_ms"] = {"big": res[other]["stages_big"], "small": res[other]["stages_small"]}
        o["roofline"] = roofline_of(D, other, res[other]["stages_big"], res[other]["pairs_big"], ba)
        o["speedup_vs_sts"] = o["dmts_ns_per_day"] / o["sts_1fs_ns_per_day"]
        extras["fp32" if other == D.FP32 else "bf16"] = o
    if args.extras and world == 1:
        extras["langevin_hmr_5fs"] = langevin_hmr(D, I, torch, s, mdl, main_prec, args, flush)
        extras["vacuum512"] = vacuum_batch(D, I, torch, main_prec, args, flush)
        extras["replicas8"] = replicas_batch(D, I, torch, main_prec, args, flush)
        extras["distill"] = distill_rate(D, I, torch, s, mdl, main_prec)
        extras["polymer100k"] = polymer(D, I, torch, main_prec, args, flush)

    if rank != 0:
        return None
    cpu = cpu_baseline(args, s, mdl, dt, n_inner) if world == 1 and not args.no_cpu else None
    line = {
        "metric": METRIC, "value": m["dmts_ns_per_day"], "unit": "ns/day", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if main_prec == D.BF16_MLP else "f32",
        "data": "synthetic",
        "config": step_config(args, s, world),
        "precision": args.precision + (" MLP operands on tcgen05, FP32 accumulation, geometry and sums; "
                                       "FP64 integrator state" if args.precision == "bf16" else ""),
        "atom_force_evals_per_s": m["atom_force_evals_per_s"], "sts_1fs_ns_per_day": m["sts_1fs_ns_per_day"],
        "speedup_vs_sts": m["dmts_ns_per_day"] / m["sts_1fs_ns_per_day"],
        "dmts_6fs_ns_per_day": m["dmts_6fs_ns_per_day"],
        "speedup_6fs_vs_sts": m["dmts_6fs_ns_per_day"] / m["sts_1fs_ns_per_day"],
        "ms_per_step_sts": m["ms_per_step_sts"],
        "pairs": {"small": main["pairs_small"], "big": main["pairs_big"]},
        "tuning": main["tuning"],
        "stage_ms": {"big": main["stages_big"], "small": main["stages_small"]},
        "roofline": roofline_of(D, main_prec, main["stages_big"], main["pairs_big"], ba),
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": main["launches"], "clocks": clk,
    }
    line.update(extras)
    return line


def vacuum_batch(D, I, torch, prec, args, flush):
    """512 independent non-periodic molecules of 10-60 atoms, one context,
    DMTS 3 fs / 1 fs vs 1 fs STS (each CUDA graph covers all molecules)."""
    s = I.make_vacuum_batch(512, 10, 60, seed=0)
    mdl = models(4)
    r = measure(D, I, torch, s, mdl, prec, argparse.Namespace(steps=max(10, args.steps // 2), warmup=3),
                flush, 3.0, 3, 1)
    k = max(10, args.steps // 2)
    return {"workload": f"512 vacuum molecules, {s.n_atoms} atoms", "steps": k,
            "dmts_ns_per_day_per_molecule_sum": k * 3.0 / FS_PER_NS / r["t_dmts"] * SEC_PER_DAY * 512,
            "dmts_ns_per_day": k * 3.0 / FS_PER_NS / r["t_dmts"] * SEC_PER_DAY,
            "sts_1fs_ns_per_day": k * 1.0 / FS_PER_NS / r["t_sts"] * SEC_PER_DAY,
            "ms_per_step": r["t_dmts"] * 1e3 / k, "ms_per_step_sts": r["t_sts"] * 1e3 / k,
            "pairs": {"small": r["pairs_small"], "big": r["pairs_big"]}}


def replicas_batch(D, I, torch, prec, args, flush, n_rep=8):
    """n_rep periodic replicas of the 1,536-atom water box (512 waters,
    L = 24.85 A, different orientations and velocities) in one context, one
    graph per outer step for all of them, against the same boxes each in its
    own context run one after another; DMTS 3 fs / 1 fs."""
    boxes = [I.make_water(8, 24.85, k) for k in range(n_rep)]
    s = I.replicas(boxes)
    mdl = models(2)
    k = max(10, args.steps // 2)
    r = measure(D, I, torch, s, mdl, prec, argparse.Namespace(steps=k, warmup=3), flush, 3.0, 3, 1)
    t_sep = 0.0
    for b in boxes[:2]:                                # two separate contexts, scaled to n_rep
        rb = measure(D, I, torch, b, mdl, prec, argparse.Namespace(steps=k, warmup=3), flush, 3.0, 3, 1)
        t_sep += rb["t_dmts"]
        rb["ctx"].close()
        rb["sts"].close()
    t_sep *= n_rep / 2
    r["ctx"].close()
    r["sts"].close()
    agg = n_rep * k * 3.0 / FS_PER_NS / r["t_dmts"] * SEC_PER_DAY
    return {"workload": f"{n_rep} periodic replicas of 1,536-atom water (L = 24.85 A), {s.n_atoms} atoms", "steps": k,
            "dmts_ns_per_day_sum_over_replicas": agg,
            "separate_contexts_ns_per_day_sum": n_rep * k * 3.0 / FS_PER_NS / t_sep * SEC_PER_DAY,
            "ms_per_step": r["t_dmts"] * 1e3 / k, "pairs": {"small": r["pairs_small"], "big": r["pairs_big"]}}


def langevin_hmr(D, I, torch, s, mdl, prec, args, flush, seed=1):
    """The paper's production setting on the water box: BAOAB-RESPA
    (Algorithm 1 with the Langevin thermostat, friction 1 ps^-1, 300 K),
    hydrogens repartitioned to 3.024 amu, 1 fs inner / 5 fs outer steps;
    against 1 fs BAOAB with the big model only and standard masses."""
    sa, sp, ba, bp = mdl
    m = D.hmr_masses(s.mass, s.bonds, 3.024)
    sh = I.System(x=s.x, species=s.species, mass=m, atom_offset=s.atom_offset, box=s.box,
                  n_species=s.n_species, name=s.name, bonds=s.bonds)
    opts = json.dumps({"langevin_friction": 1.0, "temperature": 300.0, "seed": seed})
    ctx = D.Context(sh, ba, bp, sa, sp, precision=prec, options=opts)
    sts = D.Context(s, ba, bp, precision=prec, options=opts)
    vh = I.maxwell_boltzmann(m, 300.0, seed, s.atom_offset)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, seed, s.atom_offset)
    ctx.set_state(s.x, vh)
    sts.set_state(s.x, v0)
    ctx.respa_step(3, 5.0, 5, energies=False)
    sts.respa_step(3, 1.0, 1, energies=False)
    k = max(6, args.steps // 4)
    ms, _ = time_steps(ctx, torch, torch.cuda.ExternalStream(ctx.stream), flush, k, 5.0, 5, s.x, vh)
    ms_s, _ = time_steps(sts, torch, torch.cuda.ExternalStream(sts.stream), flush, k, 1.0, 1, s.x, v0)
    # the same with the paper's force-difference monitor armed (150 kcal/mol/A)
    mon = D.Context(sh, ba, bp, sa, sp, precision=prec,
                    options=json.dumps({"langevin_friction": 1.0, "temperature": 300.0, "seed": seed,
                                        "fallback_threshold": 6.505}))
    mon.set_state(s.x, vh)
    mon.respa_step(3, 5.0, 5, energies=False)
    ms_m, _ = time_steps(mon, torch, torch.cuda.ExternalStream(mon.stream), flush, k, 5.0, 5, s.x, vh)
    t, t_s, t_m = sum(ms) / 1e3, sum(ms_s) / 1e3, sum(ms_m) / 1e3
    dmts = k * 5.0 / FS_PER_NS / t * SEC_PER_DAY
    sts_v = k * 1.0 / FS_PER_NS / t_s * SEC_PER_DAY
    mstat = mon.monitor()
    return {"workload": f"{s.name}, hydrogens 3.024 amu, Langevin 1 ps^-1 at 300 K", "steps": k,
            "dmts_5fs_hmr_ns_per_day": dmts, "sts_1fs_baoab_ns_per_day": sts_v, "speedup": dmts / sts_v,
            "ms_per_step": t * 1e3 / k, "ms_per_step_sts": t_s * 1e3 / k,
            "monitored": {"threshold_eV_per_A": 6.505, "dmts_5fs_hmr_ns_per_day": k * 5.0 / FS_PER_NS / t_m * SEC_PER_DAY,
                          "fallback_steps": mstat["n_fallback"], "max_df_eV_per_A": mstat["max_df"]}}


def polymer(D, I, torch, prec, args, flush):
    """~100k-atom solvated polymer (4 species), DMTS 3 fs / 1 fs vs 1 fs STS,
    with the dominant kernel's roofline at this size."""
    s = I.make_solvated_polymer()
    mdl = models(4)
    k = max(10, args.steps // 4)
    r = measure(D, I, torch, s, mdl, prec, argparse.Namespace(steps=k, warmup=3), flush, 3.0, 3, 1)
    return {"workload": f"solvated polymer, {s.n_atoms} atoms, L={s.box[0]:.2f} A", "steps": k,
            "dmts_ns_per_day": k * 3.0 / FS_PER_NS / r["t_dmts"] * SEC_PER_DAY,
            "sts_1fs_ns_per_day": k * 1.0 / FS_PER_NS / r["t_sts"] * SEC_PER_DAY,
            "ms_per_step": r["t_dmts"] * 1e3 / k, "ms_per_step_sts": r["t_sts"] * 1e3 / k,
            "atom_force_evals_per_s": k * 4 * s.n_atoms / r["t_dmts"],
            "pairs": {"small": r["pairs_small"], "big": r["pairs_big"]},
            "stage_ms": {"big": r["stages_big"], "small": r["stages_small"]},
            "roofline": roofline_of(D, prec, r["stages_big"], r["pairs_big"], mdl[2]),
            "tuning": r["tuning"]}


def distill_rate(D, I, torch, s, mdl, prec, n_frames=64, n_traj=8):
    """System-specific distillation on the water box: n_frames frames from
    big-model MD (n_traj trajectories, one frame every 10 fs), labelled with
    the big model's energies and forces, then the energy and force loss
    gradient of the small model over all frames (hand-written second-order
    adjoints through the forces, in the context's precision) and a full
    training step (gradient + Adam update)."""
    from paper_2510_06562_gb300 import distill as DS
    sa, sp, ba, bp = mdl
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    frames, f_ref, e_ref = DS.sample_frames(s, ba, bp, n_frames, n_traj, 10.0, precision=prec)
    t_sample = time.perf_counter() - t0
    ctx = D.Context(s, ba, bp, sa, sp, precision=prec)
    ctx.set_state(s.x)
    fd = torch.tensor(frames, device="cuda")
    rd = torch.tensor(f_ref, device="cuda")
    ed = torch.tensor(e_ref, device="cuda")
    loss0, _ = ctx.distill_grad(fd, rd, ed, 1.0)             # warm-up (sizes the capacities)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, g = ctx.distill_grad(fd, rd, ed, 1.0)
    t_grad = time.perf_counter() - t0
    m1, m2 = np.zeros(ctx.small_n_params), np.zeros(ctx.small_n_params)
    t0 = time.perf_counter()
    ctx.adam_step(D.SMALL, g, m1, m2, 1, 1e-3)
    t_adam = time.perf_counter() - t0
    loss1, _ = ctx.distill_grad(fd, rd, ed, 1.0)
    ctx.close()
    return {"workload": f"{n_frames} frames of the {s.n_atoms}-atom box from big-model MD ({n_traj} trajectories, "
                        f"10 fs apart), energy + force loss (lambda_e = 1)",
            "precision": ("frame forces and energies, and the per-pair MLP products and filter-weight "
                          "gradient sums of the second-order edge passes, BF16 operands on tcgen05 with FP32 "
                          "accumulation; geometry, per-atom pass and sums FP32" if prec == D.BF16_MLP
                          else "FP32 throughout"),
            "frames_per_s": n_frames / t_grad, "ms_per_frame": t_grad * 1e3 / n_frames,
            "ms_per_training_step": (t_grad + t_adam) * 1e3, "frame_sampling_s": t_sample,
            "loss": loss, "loss_after_one_step": loss1}


# ------------------------------------------------------------------- oracle
class OracleStep:
    """Outer steps of Algorithm 1 by the FP64 oracle (``oracle.integrate.respa``
    with ``oracle.model`` forces, O(N^2) pair search), carrying the forces
    between steps as the algorithm does."""

    def __init__(self, s, sa, sp, ba, bp, v0):
        from oracle import model as M
        self.s = s
        self.fs = lambda x: M.energy_forces(M.spec_of(sa), sp, x, s.species, s.atom_offset, s.box)[1]
        self.fb = lambda x: M.energy_forces(M.spec_of(ba), bp, x, s.species, s.atom_offset, s.box)[1]
        self.bpa = np.full(s.n_atoms, s.box[0])
        self.x, self.v = np.array(s.x, dtype=np.float64), np.array(v0, dtype=np.float64)
        self.F_small = self.F = None

    def step(self, dt, n_inner):
        """One outer step; returns its wall-clock seconds."""
        from oracle import integrate as G
        t0 = time.perf_counter()
        self.x, self.v, self.F_small, self.F, _ = G.respa(self.x, self.v, self.s.mass, self.fs, self.fb, dt,
                                                         n_inner, 1, box_per_atom=self.bpa,
                                                         F_small=self.F_small, F=self.F)
        return time.perf_counter() - t0


def _oracle_ns_per_day(s, mdl, dt, n_inner, n_steps=1):
    """ns/day of the oracle on system s: one untimed step (it evaluates both
    models at the start), then n_steps timed outer steps."""
    from paper_2510_06562_gb300 import inputs as I
    sa, sp, ba, bp = mdl
    o = OracleStep(s, sa, sp, ba, bp, I.maxwell_boltzmann(s.mass, 300.0, 1, s.atom_offset))
    o.step(dt, n_inner)
    t = sum(o.step(dt, n_inner) for _ in range(n_steps))
    return n_steps * dt / FS_PER_NS / t * SEC_PER_DAY, t / n_steps


def cpu_baseline(args, s, mdl, dt, n_inner):
    """The oracle as it stands on the host cores: one outer step of the timed
    workload (after one untimed step), plus the 192-atom box on all cores and
    on one thread."""
    import torch
    from paper_2510_06562_gb300 import inputs as I
    cores = torch.get_num_threads()
    value, t_step = _oracle_ns_per_day(s, mdl, dt, n_inner)
    small = I.water_192(0)
    v192, t192 = _oracle_ns_per_day(small, models(small.n_species), dt, n_inner, n_steps=5)
    torch.set_num_threads(1)
    try:
        v192_1, t192_1 = _oracle_ns_per_day(small, models(small.n_species), dt, n_inner, n_steps=5)
    finally:
        torch.set_num_threads(cores)
    return {"value": value, "unit": "ns/day", "cores": cores, "kind": "oracle",
            "sample": (f"one outer step of Algorithm 1 ({n_inner} small + 1 big FP64 force evaluations, O(N^2) "
                       f"pair search; {t_step:.2f} s) on the {s.n_atoms}-atom box after one untimed step"),
            "water192": {"ns_per_day": v192, "s_per_step": t192, "cores": cores, "steps": 5},
            "water192_single_thread": {"ns_per_day": v192_1, "s_per_step": t192_1, "cores": 1, "steps": 5}}


def run_reference(args):
    """The oracle arm: every step is one outer step of Algorithm 1 by the FP64
    oracle on the same workload, integrated (not extrapolated); W untimed
    warm-up steps first (the first evaluates both models at the start)."""
    import torch
    from paper_2510_06562_gb300 import inputs as I
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    s = workload(args.workload)
    sa, sp, ba, bp = models(s.n_species)
    dt, n_inner = args.outer_fs, args.n_inner
    o = OracleStep(s, sa, sp, ba, bp, I.maxwell_boltzmann(s.mass, 300.0, 1, s.atom_offset))
    for _ in range(args.warmup):
        o.step(dt, n_inner)
    t = sum(o.step(dt, n_inner) for _ in range(args.steps))
    value = args.steps * dt / FS_PER_NS / t * SEC_PER_DAY
    sample = (f"{args.steps} outer steps of {dt:g} fs ({n_inner} small + 1 big FP64 force evaluations each, "
              f"O(N^2) pair search) on the {s.n_atoms}-atom box, integrated by the oracle after "
              f"{args.warmup} untimed steps")
    return {"metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": step_config(args, s, world), "precision": "fp64 (the oracle on the host cores)",
            "cpu_baseline": {"value": value, "unit": "ns/day", "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water12288")
    ap.add_argument("--outer-fs", type=float, default=3.0)
    ap.add_argument("--n-inner", type=int, default=3)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--single-precision", action="store_true", help="measure only --precision")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the vacuum-batch and distillation measurements")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
