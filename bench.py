"""Benchmark of the UGKS + adaptive-velocity-space hot path on GB300.

Workload (default): supersonic flow around a sphere in the slip regime
(paper Sec. 4.6 shape): spherical shell of 64 radial x 48 polar x 48
azimuthal cells, Ma 4.25, Kn 0.031, isothermal wall, global octree over
[-12, 12]^3 sqrt(R T_inf) with base 16^3 and up to 3 levels (~15-21k nodes),
mixed precision (f in FP32; moment sums, wall balance and correction in
FP64) with the learned adaptation proposer.  `--workload cylinder` runs the
Ma 5 cylinder (O-mesh 128 x 96, quadtree base 24^2, 4 levels).

One benchmark step = one pass of the whole hot path over one batch: the
Maxwellian start of the flow from the device-resident initial field, `nu`
(= 50, the adaptation interval) explicit UGKS steps and one adaptation of the
velocity mesh (moments, criterion, marks + scan compaction, consanguinity
remap, conservation correction).  Metric: cell-velocity-node updates per
second, sum over the UGKS steps of Nc * Nv divided by the time.  The line
also carries the same workload with the plain criterion (ablation of the
proposer), the plain FP64 GPU form, the end-to-end rate through the C ABI
with host buffers, the HBM roofline of the UGKS step and the CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs its own replica (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-velocity-node updates/s"
UNIT = "cell-node updates/s"
NU = 50


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--nu", type=int, default=NU)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU (oracle) baseline leg")
    ap.add_argument("--no-ablation", action="store_true", help="skip the plain-criterion ablation leg")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="form of the timed leg: mixed (the benchmark) or the plain FP64 form (profiling)")
    ap.add_argument("--workload", default="sphere", choices=sorted(WORKLOADS),
                    help="sphere (the benchmark case) or another configuration")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="host threads of the CPU oracle (default: all cores)")
    ap.add_argument("--implicit", type=float, default=0.0, metavar="CFL",
                    help="time the implicit IUGKS step (60 macro + 2 micro SGS iterations) at this CFL instead")
    ap.add_argument("--sweep", action="store_true",
                    help="kernel sweep over cell and node counts (FP32 and FP64 steps), one JSON line per case")
    ap.add_argument("--sweep-precision", default="both", choices=["both", "mixed", "fp64"],
                    help="forms the sweep runs")
    return ap.parse_args()


WORKLOADS = {
    # supersonic cylinder, O-mesh 128 radial x 96 circumferential (the benchmark case)
    "cylinder": ("cylinder", dict()),
    # same flow and velocity mesh on the inner 64 radial rows (profiling case, f > L2)
    "cylinder-r64": ("cylinder", dict(n_r=64)),
    # lid-driven cavity 32 x 32 (config of the FP64 full-run parity)
    "cavity": ("cavity", dict()),
    # blunt wedge 240 x 160, Ma 8, Kn 0.01, 5 levels
    "wedge": ("blunt_wedge", dict()),
    # sphere 64 x 48 x 48, Ma 4.25, Kn 0.031, octree 16^3 with 3 levels
    "sphere": ("sphere", dict()),
    # the sphere's inner 8 radial shells (profiling case, f > L2)
    "sphere-r8": ("sphere", dict(n_r=8)),
    # the sphere's inner 4 radial shells (detailed ncu captures: f = 0.55 GB, a few GB on the device)
    "sphere-r4": ("sphere", dict(n_r=4)),
    # the sphere's inner 2 radial shells (captures of the FP64 form: f = 0.8 GB in FP64)
    "sphere-r2": ("sphere", dict(n_r=2)),
    # the cylinder with the velocity space of the adaptive-parameter rules (zones, C1(Ma))
    "cylinder-zones": ("cylinder_zones", dict()),
    # the cylinder with a diatomic gas (Rykov model: G, H, R)
    "cylinder-rykov": ("cylinder", dict(model="rykov")),
    # the same on the inner 64 radial rows (profiling case)
    "cylinder-rykov-r64": ("cylinder", dict(n_r=64, model="rykov")),
}
_WL = "sphere"


def _build(fn, kw, precision):
    """A workload by builder name; the key `model` selects the gas model."""
    from paper_2212_05645_gb300 import workloads as wl
    kw = dict(kw)
    model = kw.pop("model", "shakhov")
    w = getattr(wl, fn)(precision=precision, **kw)
    w.model = model
    return w


def _workload(precision="mixed"):
    fn, kw = WORKLOADS[_WL]
    return _build(fn, kw, precision)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- ranks
def aggregate(ms, updates, ws, device=None):
    """Whole-job numbers over ranks: the slowest rank's time and the sum of
    the cell-node updates (replicas, weak scaling).  Uses torch.distributed
    when ws > 1 (NCCL on the GPU, gloo on the CPU)."""
    if ws <= 1:
        return float(ms), float(updates)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms), float(updates)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


# ---------------------------------------------------------------- peaks
def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _traffic(family, Nc, Nv):
    """DRAM bytes per UGKS step (the step kernels, one ncu pass) from the
    committed record of this workload family, scaled to this step by
    cell-nodes; None when the step's kernel sources changed since the
    counters were taken or no record exists."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "step_kernel_dram.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    h = hashlib.sha256()
    for f in ("avs_step.cu", "avs_dev.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2212_05645_gb300", "csrc", f), "rb").read())
    sha = h.hexdigest()[:16]
    e = d.get(family)
    if not e or e.get("src_sha") != sha:
        return None
    return e["dram_bytes"] * (Nc * Nv) / (e["Nc"] * e["Nv"])


# ---------------------------------------------------------------- CPU baseline (oracle)
ORACLE_SAMPLES = {
    # workload -> (builder, reduced mesh arguments, what the sample is)
    "cylinder": ("cylinder", dict(n_r=12), "the first 12 radial rows (1152 cells)"),
    "cylinder-r64": ("cylinder", dict(n_r=12), "the first 12 radial rows (1152 cells)"),
    "cavity": ("cavity", dict(), "the whole 32 x 32 cavity"),
    "wedge": ("blunt_wedge", dict(n_r=8, learned=False), "the first 8 wall-normal rows (1920 cells)"),
    "sphere": ("sphere", dict(n_r=2, learned=False), "the first 2 radial shells (4608 cells)"),
    "sphere-r8": ("sphere", dict(n_r=2, learned=False), "the first 2 radial shells (4608 cells)"),
    "sphere-r4": ("sphere", dict(n_r=2, learned=False), "the first 2 radial shells (4608 cells)"),
    "sphere-r2": ("sphere", dict(n_r=2, learned=False), "the first 2 radial shells (4608 cells)"),
    "cylinder-zones": ("cylinder_zones", dict(), "the whole 128 x 96 O-mesh (12288 cells)"),
    "cylinder-rykov": ("cylinder", dict(n_r=12, model="rykov"), "the first 12 radial rows (1152 cells)"),
    "cylinder-rykov-r64": ("cylinder", dict(n_r=12, model="rykov"), "the first 12 radial rows (1152 cells)"),
}


def cpu_baseline(seconds=12.0, nu=NU):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same
    workload (the rows of cells next to the body, the full velocity tree);
    UGKS steps until about `seconds` of CPU time, at most `nu`."""
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle as O
    from paper_2212_05645_gb300 import workloads as wl
    fn, kw, what = ORACLE_SAMPLES[_WL]
    w = _build(fn, kw, "fp64")
    r = O.Run(w)
    r.init_field()
    dt = r.dt()
    r.step(dt)                                     # warm-up
    n, t0 = 0, time.perf_counter()
    while True:
        r.step(dt)
        n += 1
        if time.perf_counter() - t0 > seconds or n >= nu:
            break
    el = time.perf_counter() - t0
    val = w.mesh.Nc * r.Nv * n / el
    return {"value": val, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
            "sample": f"{n} UGKS steps of {what} x {r.Nv} velocity nodes, FP64",
            "seconds": el}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    t0 = time.perf_counter()
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(seconds=1.0, nu=2)
    for _ in range(args.steps):
        vals.append(cpu_baseline(seconds=8.0, nu=args.nu))
    el = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    w = _workload()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "oracle_sample": vals[0]["sample"]},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"], "value": v,
                             "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    from paper_2212_05645_gb300 import avs as A
    from paper_2212_05645_gb300 import build as B

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    B.build()
    stream = torch.cuda.current_stream()
    w = _workload("mixed")
    # headline form: mixed precision with the learned proposer (full criterion every 4th adaptation)
    learned = True
    nu = args.nu
    W0 = torch.from_numpy(np.ascontiguousarray(w.W_init)).to("cuda")
    Nc = w.mesh.Nc

    def advance(ctx, n):
        if args.implicit > 0:
            ctx.step_implicit(n, cfl=args.implicit)
        else:
            ctx.step(n)

    # Every bench step is one batch: a flow started from the initial field W0
    # (device-resident here, uploaded from pinned host memory in the e2e
    # leg), nu UGKS steps and one adaptation, so that every timed bench step
    # is the same job; the velocity mesh carries over from the previous
    # batch's adaptation (the flows themselves run stably for thousands of
    # steps; tests/test_gpu_long_runs.py).
    def bench_step(ctx, updates, n=nu):
        ctx.init_field(W0)
        advance(ctx, n)
        updates.append(Nc * ctx.Nv * n)
        return ctx.adapt()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def field_after_steps(ctx):
        """W and heat flux q after nu UGKS steps from the initial field on the
        context's current velocity mesh (untimed)."""
        ctx.init_field(W0)
        advance(ctx, nu)
        return ctx.moments()

    # inputs below twice the L2 size: a 256 MB write between timed bench steps
    # (outside their events) so that no step starts from a warm L2
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size

    def make(precision, learned_, **kw):
        return A.AVS(w, precision=precision, stream=stream.cuda_stream, learned=learned_, full_every=4, **kw)

    # ---- headline: mixed + learned, device-timed (--precision fp64: the plain
    # FP64 form instead, for profiling)
    main_fp64 = args.precision == "fp64"
    if main_fp64:
        learned = False
    g = make("fp64" if main_fp64 else "mixed", learned)
    NA, NW = g.NA, g.NW
    esize = 8 if main_fp64 else 4
    f_bytes = Nc * NA * g.Nv * esize
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if f_bytes < 2 * l2 else None
    for _ in range(args.warmup):
        bench_step(g, [])
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    upd = []
    ev = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_s, ev_e, wb_s, wb_e = ev(), ev(), ev(), ev()
    step_cells = []
    barrier()
    torch.cuda.synchronize()
    l0 = g.launches
    astats = []
    for j in range(args.steps):
        if flush is not None:
            flush.fill_(j & 255)
        wb_s[j].record(stream)
        g.init_field(W0)
        ev_s[j].record(stream)
        advance(g, nu)
        ev_e[j].record(stream)
        upd.append(Nc * g.Nv * nu)
        step_cells.append(Nc * g.Nv)
        astats.append(g.adapt())
        wb_e[j].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = g.launches - l0
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in zip(wb_s, wb_e))
    step_ms = [a.elapsed_time(b) for a, b in zip(ev_s, ev_e)]
    t_max, tot_updates = aggregate(ms, float(sum(upd)), ws, device="cuda")
    value = tot_updates / (t_max * 1e-3)
    Nv_last = g.Nv
    # the proposer's misses judged on the fields: the learned run's W and q
    # after one more bench step's UGKS steps, against the plain run's below
    field_learned = field_after_steps(g) if learned and not args.no_ablation else None
    nodes_learned = g.Nv
    g.close()
    del g

    # roofline of the UGKS step (the step kernels; 90+ % of a bench step):
    # algorithmic traffic = 1 read + 1 write of f in FP32 per cell-node
    bytes_per_cn = 2 * NA * esize
    kern_ms = sum(step_ms) / (args.steps * nu)
    cn_per_launch = statistics.mean(step_cells)
    achieved = bytes_per_cn * cn_per_launch / (kern_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    family = "sphere" if _WL.startswith("sphere") else "cylinder" if _WL.startswith("cylinder") else None
    traffic = (_traffic(family, Nc, cn_per_launch / Nc)
               if family and args.implicit <= 0 and w.model == "shakhov" else None)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "kernel": (f"implicit Rykov UGKS step: k_grad + rk_face + rk_imp_setup + rk_imp_macro + rk_imp_res"
                       f" + rk_imp_micro + rk_imp_finish <{w.D},float>" if args.implicit > 0 and w.model == "rykov" else
                       f"implicit UGKS step: k_foot + k_face + k_imp_setup + k_imp_macro + k_imp_state + k_imp_res"
                       f" + k_imp_micro + k_imp_finish <{w.D},float>" if args.implicit > 0 else
                       f"Rykov UGKS step: k_grad + rk_face + rk_cell <{w.D},float>" if w.model == "rykov" else
                       f"UGKS step: k_foot + k_face + k_cell_state + k_cell <{w.D},{'double' if main_fp64 else 'float'}>"),
            "peak_source": peak_kind,
            "algorithmic_bytes_per_cell_node": bytes_per_cn, "kernel_ms": kern_ms,
            "peak_spec_gbs": 8000.0, "frac_of_spec": achieved / 8000.0}

    # ---- end to end through the public API with host buffers: a fresh
    # context through the same warm-up, so that its steps see the same
    # sequence of velocity meshes and of full and learned adaptations
    e2e = None
    if rank == 0 or ws > 1:
        Wp = torch.from_numpy(np.ascontiguousarray(w.W_init)).pin_memory()
        Wout = torch.zeros((Nc, NW), dtype=torch.float64).pin_memory()   # D + 2, or D + 3 (Rykov)
        ge = make("mixed", learned)
        for _ in range(args.warmup):
            bench_step(ge, [])
        ke = min(args.steps, 6)
        torch.cuda.synchronize()
        e_upd = []
        te0 = time.perf_counter()
        for j in range(ke):
            if flush is not None:     # the same cold L2 as the device-timed steps
                flush.fill_(j & 255)
            ge.init_field(Wp)         # h2d of the step's input W
            advance(ge, nu)
            e_upd.append(Nc * ge.Nv * nu)
            ge.adapt()
            ge.moments(out_W=Wout)    # d2h of the step's result
        torch.cuda.synchronize()
        te = time.perf_counter() - te0
        ge.close()
        del ge
        e2e = {"value": sum(e_upd) / te, "unit": UNIT, "h2d_bytes_per_step": int(Wp.numel() * 8),
               "d2h_bytes_per_step": int(Wout.numel() * 8), "steps": ke,
               "velocity_nodes": [int(u // (Nc * nu)) for u in e_upd]}

    # ---- ablation: the same workload and bench steps with the plain
    # criterion on every adaptation (no proposer)
    ablation = None
    if learned and not args.no_ablation:
        ga = make("mixed", False)
        for _ in range(min(args.warmup, 2)):
            bench_step(ga, [])
        ka = min(args.steps, 6)
        ua = []
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        ta = 0.0
        crit = []
        for j in range(ka):
            if flush is not None:
                flush.fill_(j & 255)
            a0.record(stream)
            bench_step(ga, ua)
            a1.record(stream)
            torch.cuda.synchronize()
            ta += a0.elapsed_time(a1)
        field_plain = field_after_steps(ga)
        nodes_plain = ga.Nv
        ga.close()
        del ga
        ablation = {"form": "mixed, plain criterion on every adaptation", "value": sum(ua) / (ta * 1e-3),
                    "unit": UNIT, "steps": ka, "mean_velocity_nodes": sum(ua) / (ka * nu * Nc),
                    "learned_over_plain": value / ws / (sum(ua) / (ta * 1e-3)),
                    "fields": dict(_field_gaps(w, field_learned, field_plain), velocity_nodes_learned=nodes_learned,
                                   velocity_nodes_plain=nodes_plain,
                                   what=f"W and wall heat flux after {nu} UGKS steps from the initial field on each "
                                        "run's last velocity mesh: learned against plain")}

    # ---- plain FP64 GPU form on the same workload: the same kind of bench
    # step with fewer UGKS steps where the workload is large (about 20 s of
    # FP64 work; the step count is in the line); device memory permitting
    fp64 = None
    if not args.no_fp64:
        n64 = int(max(1, min(nu, 2.6e10 / (2.0 * Nc * Nv_last))))
        try:
            gd = make("fp64", False)
            bench_step(gd, [], n64)
            torch.cuda.synchronize()
            u = []
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            kd = 2 if n64 == nu else 1
            a.record(stream)
            for _ in range(kd):
                bench_step(gd, u, n64)
            b.record(stream)
            torch.cuda.synchronize()
            fms = a.elapsed_time(b)
            fp64 = {"value": sum(u) / (fms * 1e-3), "ms_per_step": fms / kd, "steps": kd,
                    "ugks_steps_per_step": n64}
            gd.close()
            del gd
        except A.AVSError as exc:
            fp64 = {"value": None, "unavailable": str(exc)}

    alu = {"fp32_fma_gflops": A.fma_peak_gflops(0), "fp64_fma_gflops": A.fma_peak_gflops(1, iters=2000),
           "fp32x2_fma_gflops": A.fma_peak_gflops(2),
           "kind": "measured: independent FMA chains, bench.py start-up"}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    if rank == 0:
        f_mb = f_bytes / 1e6
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if main_fp64 else "f32+f64", "data": "synthetic",
                "config": {"workload": w.name, "cells": Nc, "velocity_nodes": Nv_last,
                           "ugks_steps_per_step": nu,
                           "precision": "FP64" if main_fp64 else "mixed (f FP32, sums FP64)",
                           "time_step": (f"implicit IUGKS, CFL {args.implicit}, 60 macro + 2 micro SGS iterations"
                                         if args.implicit > 0 else "explicit, CFL 0.8"),
                           "adaptation": ("learned proposer, full criterion every 4th adaptation" if learned
                                          else "plain criterion every adaptation"),
                           "gas": ("Rykov (diatomic: G, H, R)" if w.model == "rykov" else
                                   "Shakhov (monatomic: G, H)" if w.D == 2 else "Shakhov (monatomic: G)"),
                           "l2": (f"L2 flushed before each timed step (f = {f_mb:.0f} MB per buffer)"
                                  if flush is not None else f"inputs larger than L2 (f = {f_mb:.0f} MB per buffer)"),
                           "parallelism": f"replicas x{ws}"},
                "roofline": roof, "alu_peaks": alu, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks, "fp64_form": fp64, "ablation": ablation,
                "adaptation": {"full": sum(a["full"] for a in astats), "learned": sum(1 - a["full"] for a in astats),
                               "mean_checked_cells": statistics.mean(a["checked_cells"] for a in astats),
                               "checked_fraction_learned": (statistics.mean(
                                   a["checked_cells"] / Nc for a in astats if not a["full"])
                                   if any(not a["full"] for a in astats) else None),
                               "missed_nodes_on_full_steps": [a["missed_nodes"] for a in astats if a["full"]],
                               "nodes": [a["Nv"] for a in astats],
                               "step_velocity_nodes": [int(c // Nc) for c in step_cells]},
                "speedup_vs_fp64_form": (value / ws / fp64["value"]) if fp64 and fp64.get("value") else None}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _field_gaps(w, learned, plain):
    """L1 gap of the conserved moments and of the wall heat flux q . n (cells
    next to wall faces), relative to the plain run's (the measure of the
    proposer's misses)."""
    from paper_2212_05645_gb300 import workloads as wl
    (Wl, ql), (Wp, qp) = learned, plain
    m = w.mesh
    out = {"l1_moment_gap": float(np.abs(Wl - Wp).sum() / np.abs(Wp).sum()), "wall_heat_flux_gap": None}
    b = np.nonzero(m.faceR < 0)[0]
    b = b[m.bc[-1 - m.faceR[b], 0].astype(int) == wl.BC_WALL]
    if len(b):
        n = m.An[b] / np.linalg.norm(m.An[b], axis=1, keepdims=True)
        hl = (ql[m.faceL[b]] * n).sum(1)
        hp = (qp[m.faceL[b]] * n).sum(1)
        out["wall_heat_flux_gap"] = float(np.abs(hl - hp).sum() / np.abs(hp).sum())
    return out


# ---------------------------------------------------------------- kernel sweep
SWEEP_CELLS_2D = [(32, 32), (128, 128), (256, 256), (448, 448)]
SWEEP_CELLS_3D = [(10, 10, 10), (20, 20, 20), (40, 40, 40), (58, 58, 58)]
SWEEP_BASE_2D = [16, 32, 64, 128, 180]          # 256 .. 32400 nodes (uniform quadtree)
SWEEP_BASE_3D = [8, 16, 24, 32]                 # 512 .. 32768 nodes (uniform octree)
SWEEP_MAX_BYTES = 200e9                         # skip states above 200 GB


def run_sweep(args):
    """One JSON line per (cells, nodes, precision): the UGKS step alone on a
    periodic box with the smooth synthetic field, its cell-node updates/s and
    the algorithmic HBM fraction (1 read + 1 write of f per cell-node)."""
    import torch
    from paper_2212_05645_gb300 import avs as A
    from paper_2212_05645_gb300 import build as B
    from paper_2212_05645_gb300 import workloads as wl
    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.current_stream()
    peak, peak_kind = _peaks()
    cases = [(n, b) for n in SWEEP_CELLS_2D for b in SWEEP_BASE_2D] + \
            [(n, b) for n in SWEEP_CELLS_3D for b in SWEEP_BASE_3D]
    import dataclasses
    meshes = {}
    for n, b in cases:
        D = len(n)
        Nc = int(np.prod(n))
        Nv = b ** D
        if n not in meshes:
            meshes[n] = wl.sweep_box(n, base=(b,) * D, max_refine=0)     # mesh and field built once per size
        forms = ("mixed", "fp64") if args.sweep_precision == "both" else (args.sweep_precision,)
        for precision in forms:
            es = 4 if precision == "mixed" else 8
            NA = 2 if D == 2 else 1
            # f twice and the face rows of foot values / fluxes (D faces per cell)
            state = Nc * Nv * NA * es * (2 + D)
            if state > SWEEP_MAX_BYTES:
                continue
            w = dataclasses.replace(meshes[n], base=(b,) * D, precision=precision)
            g = A.AVS(w, precision=precision, stream=stream.cuda_stream, learned=False)
            g.init_field()
            dt = g.dt()
            g.step(2, dt=dt)
            torch.cuda.synchronize()
            work = Nc * g.Nv
            k = max(3, min(20, int((1e10 if precision == "mixed" else 5e8) / work)))
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.step(k, dt=dt)
            e.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(e) / k
            rate = work / (ms * 1e-3)
            alg = 2 * NA * es
            print(json.dumps({"sweep": True, "D": D, "cells": Nc, "velocity_nodes": g.Nv, "precision": precision,
                              "ms_per_step": ms, "value": rate, "unit": UNIT, "steps": k,
                              "achieved_gbs": alg * rate / 1e9, "peak_gbs": peak, "peak_source": peak_kind,
                              "frac": alg * rate / 1e9 / peak}), flush=True)
            g.close()
            del g


def main():
    global _WL
    args = _args()
    _WL = args.workload
    if args.oracle_threads > 0:
        os.environ["OMP_NUM_THREADS"] = str(args.oracle_threads)
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
