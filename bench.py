"""Benchmark: H-IDBF-LU solves/s at relative residual 1e-6 on one GB300.

Workload (one "step" = one batched solve: every right-hand side of the batch
driven through the whole hot path -- H-IDBF apply, L~/U~ sweeps, Krylov
iteration -- to true relative residual 1e-6):
  PEC semicircular open arc, arc length 6553.6 lambda (R = 6553.6/pi),
  N = 262,144 pulse segments (40 per wavelength), leaf 64, eps = 1e-6,
  256 plane waves phi_i = 180 i / 256 deg solved as one block; chosen form =
  split-BF16 (HB_SPLIT_BF16): the leaves' entry and exit contractions of the
  apply on the tensor cores (bf16 hi/lo parts, FP32 accumulation), the inner
  butterfly steps and the L~/U~ sweeps in complex FP32, inside FP64 flexible
  GMRES with iterative refinement.  The plain FP64 form (complex128 factors,
  FP64 GMRES on the split system) runs on the same columns for the comparison.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank solves its own 256-angle block (angles offset by
rank; replicas, weak scaling); value = all ranks' solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "H-IDBF-LU solves/s at rel. residual 1e-6 (chosen form vs plain FP64)"
UNIT = "solves/s"
RTOL = 1e-6
RESTART = 30
MAXIT = 600
NRHS = 256
PLAIN_NRHS = 32        # right-hand sides of the like-for-like FP64 / FP32 comparison
PLAIN_REPS = 1         # timed solves of each form in the comparison
SAMPLE_N = 4096        # bounded CPU-oracle sample of the same curve family


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _arc_params(n):
    # same curve family: semicircle at 40 segments per wavelength
    return ((n / 40.0) / math.pi, 0.0, math.pi)


# ----------------------------------------------------------------------------
# CPU oracle leg (bounded sample of the same curve family, measured as is)
# ----------------------------------------------------------------------------
class OracleSample:
    """The oracle's split-preconditioned GMRES on the N=SAMPLE_N member of the semicircle
    family (same 40 segments per wavelength, leaf, eps and rtol).  Construction (dense
    assembly + naive H-IDBF) runs once, untimed, like the GPU factor; a step is one
    right-hand side solved to rtol, the plane waves taken in turn from the workload's
    256 angles."""

    def __init__(self):
        from oracle import efie, idbf
        wl = W.SEMICIRCLE_N262144
        self.params = _arc_params(SAMPLE_N)
        t0 = time.perf_counter()
        self.p = efie.Problem(W.ARC, self.params, SAMPLE_N)
        self.h = idbf.HIDBF(self.p.dense(), wl.leaf, wl.eps)
        self.build_s = time.perf_counter() - t0
        self.phis = W.incidence_angles_deg(wl)
        self.k = 0

    def step(self):
        from oracle import krylov
        phi = self.phis[(17 + 37 * self.k) % len(self.phis)]
        self.k += 1
        b = self.p.plane_wave([phi])[:, 0] * self.p.scale
        x, info = krylov.gmres_split(self.h.apply, self.h.solve_lower, self.h.solve_upper, b, rtol=RTOL,
                                     restart=RESTART, maxit=MAXIT)
        return info["iters"]


def _host_threads():
    cores = os.cpu_count() or 1
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        pass
    return int(cores)


def oracle_timed(steps, warmup):
    """Measured oracle throughput on the bounded sample: `steps` timed solves after `warmup`."""
    o = OracleSample()
    for _ in range(warmup):
        o.step()
    iters = []
    t0 = time.perf_counter()
    for _ in range(steps):
        iters.append(o.step())
    dt = time.perf_counter() - t0
    wl = W.SEMICIRCLE_N262144
    value = steps / dt
    sample = (f"oracle (numpy fp64, naive H-IDBF + GMRES({RESTART}) on L~^-1 A U~^-1, rtol {RTOL:g}) on the "
              f"semicircle family member N={SAMPLE_N} (40 segments per wavelength, leaf {wl.leaf}, eps {wl.eps:g}), "
              f"one plane wave per step, {steps} timed steps after {warmup} warm-up: {dt / steps:.2f} s per solve, "
              f"{int(np.mean(iters))} iterations; construction {o.build_s:.1f} s untimed")
    # labelled model, not a measurement: the same per-iteration cost scaled by N log^2 N
    ratio = (wl.n * math.log2(wl.n) ** 2) / (SAMPLE_N * math.log2(SAMPLE_N) ** 2)
    return dict(value=value, unit=UNIT, cores=_host_threads(), kind="oracle", sample=sample,
                ms_per_step=1e3 * dt / steps, iters=int(np.mean(iters)),
                model_estimate={"value": value / ratio, "unit": UNIT,
                                "how": f"N log^2 N scaling of the measured sample to N={wl.n} ({ratio:.1f}x), "
                                       "same iteration count; an estimate, not a measurement"})


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hb_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
# dram__bytes_read.sum + dram__bytes_write.sum per launch (256 columns, semicircle N = 262,144)
# from one ncu capture, keyed by the SHA-256 (first 16 hex digits) of the kernel's sources at
# capture time; a kernel whose sources changed since has no traffic figure (None).
MEASURED_TRAFFIC = {
    # profiles/k_sweep_coop_semicircle_N262144_traffic.md (autotuned 256-column launch)
    "k_sweep": {"sha": "b4653ac2957de173", "bytes": 2247096576 + 2686350592},
    # profiles/k_sweep_cols_semicircle_N262144.md (256-column launch, 128 CTAs x 2 columns)
    "k_sweep_cols": {"sha": "7197c23169dc946a", "bytes": 2364800000 + 2608399104},
}
KERNEL_SOURCES = {
    "k_sweep": ["hb_sweep_impl.cuh", "hb_sweep.cu", "hb_sweep_f32w.cu", "hb_sweep_launch.h"],
    "k_apply1": ["hb_apply1.cu", "hb_plan.cpp"],
    "k_sweep_cols": ["hb_sweep_cols.cu", "hb_swsched.cpp", "hb_sweep_launch.h", "hb_internal.h"],
}


def source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_1901_11371_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    rec = MEASURED_TRAFFIC.get(kernel)
    if rec is None or rec["sha"] != source_hash(kernel):
        return None
    return rec["bytes"]


def shard_angles(rank, world):
    """Incidence angles (deg) of this rank's block: every rank solves NRHS plane waves,
    rank r's angles offset by r * 180 / (NRHS * world) so that the ranks' sets interleave
    without overlap (replicas of the factor, right-hand sides sharded; no collective on the
    data path)."""
    base = W.incidence_angles_deg(W.SEMICIRCLE_N262144)
    return base + (rank * 180.0 / NRHS / world if world > 1 else 0.0)


def max_over_ranks(ms, world, device):
    """Largest timed-region length over the ranks (the job's time)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args, rank, world):
    import torch

    import paper_1901_11371_gb300 as hb
    from paper_1901_11371_gb300 import build as hb_build

    if rank == 0:
        hb_build.build()
    if world > 1:
        torch.distributed.barrier()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = W.SEMICIRCLE_N262144
    stream = torch.cuda.current_stream()
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    t0 = time.perf_counter()
    f32 = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_SPLIT_BF16, seed=0)
    hb.hb_set_gmres_graph(f32, args.gmres_graph)
    t_build = time.perf_counter() - t0
    st = hb.hb_factor_info(f32)
    tuned = hb.hb_autotune(f32, NRHS)
    tune_ms = hb.hb_autotune_times(f32, NRHS)
    phis = shard_angles(rank, world)
    b = hb.hb_rhs_plane_wave(f32, phis)
    x = torch.empty_like(b)

    def solve(fac, bb, out):
        return hb.hb_gmres(fac, bb, restart=RESTART, rtol=RTOL, maxit=MAXIT, out=out)

    def step(bb, out):
        # one step: batched solve, then the monostatic far field at every incidence angle
        _, inf = solve(f32, bb, out)
        mono = hb.hb_monostatic(f32, out, phis)
        return inf, mono

    # kernel timing on from the warm-up on: the solver's restart-cycle graph is
    # captured (with its timing events) during the warm-up, not in the timed region
    hb.hb_profile(f32, True)
    for _ in range(args.warmup):
        info, mono = step(b, x)
    # ---- timed region: device events on the launching stream
    hb.hb_profile(f32, True)   # (already on: resets the counts only)
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        info, mono = step(b, x)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    n_apply, ms_apply = hb.hb_profile_read(f32, 0)
    n_sweep, ms_sweep = hb.hb_profile_read(f32, 1)
    n_launch, _ = hb.hb_profile_read(f32, 2)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = world * args.steps * NRHS / (ms_max / 1e3)
    iters = int(np.mean([i["iters"] for i in infos]))
    ir_steps = int(np.mean([i["ir_steps"] for i in infos]))
    graph_launches = int(np.mean([i["graph_launches"] for i in infos]))
    res = max(i["true_rel_res"] for i in infos)

    # ---- end-to-end through the public API with host buffers (pinned), copies inside the region
    b_host = b.cpu().pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    b_dev = torch.empty_like(b)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        b_dev.copy_(b_host, non_blocking=True)
        _, mono = step(b_dev, x)
        x_host.copy_(x, non_blocking=True)
        mono_host = mono.cpu()
        torch.cuda.synchronize()
    e_s = time.perf_counter() - e0
    e2e = {"value": args.steps * NRHS / e_s, "unit": UNIT, "h2d_bytes_per_step": int(b.numel() * 16),
           "d2h_bytes_per_step": int(x.numel() * 16 + NRHS * 16)}
    hb.hb_profile(f32, False)

    # ---- single-column apply of the same factor (the persistent kernel), outside the timed
    # region: CUDA events on the launching stream over 20 applies after 3 warm-up applies
    x1 = b[0].to(torch.complex64).contiguous()
    y1 = torch.empty_like(x1)
    for _ in range(3):
        hb.hb_apply(f32, x1, out=y1)
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(20):
        hb.hb_apply(f32, x1, out=y1)
    eb.record(stream)
    torch.cuda.synchronize()
    apply1_ms = ea.elapsed_time(eb) / 20

    mono_np = mono.cpu().numpy()
    out = dict(value=value, ms=ms_max, iters=iters, ir_steps=ir_steps, graph_launches=graph_launches, res=res, st=st, t_build=t_build, clocks=clk, e2e=e2e, tuned=tuned, tune_ms=tune_ms,
               mono_db=[float(v) for v in 20 * np.log10(np.abs(mono_np[::32]) + 1e-300)],
               n_apply=n_apply, ms_apply=ms_apply, n_sweep=n_sweep, ms_sweep=ms_sweep, n_launch=n_launch,
               apply1_ms=apply1_ms,
               x=x)
    # ---- like-for-like form comparison (rank 0 only, outside the contract's timed region):
    # the plain FP64 form and the chosen form on the same PLAIN_NRHS right-hand sides,
    # each timed with CUDA events on the launching stream over the same number of solves
    if rank == 0 and not args.no_plain:
        f64 = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C128, seed=0)
        hb.hb_autotune(f64, PLAIN_NRHS)
        hb.hb_autotune(f32, PLAIN_NRHS)
        bp = b[:PLAIN_NRHS].contiguous()
        cmp = {}
        xs = {}
        for name, fac in (("fp64", f64), ("chosen", f32)):
            xo = torch.empty_like(bp)
            solve(fac, bp, xo)                                   # warm-up
            torch.cuda.synchronize()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            infs = [solve(fac, bp, xo)[1] for _ in range(PLAIN_REPS)]
            eb.record(stream)
            torch.cuda.synchronize()
            t = ea.elapsed_time(eb) / 1e3
            cmp[name] = {"value": PLAIN_REPS * PLAIN_NRHS / t, "unit": UNIT, "iters": infs[-1]["iters"],
                         "true_rel_res": max(i["true_rel_res"] for i in infs), "nrhs": PLAIN_NRHS,
                         "solves_timed": PLAIN_REPS * PLAIN_NRHS}
            xs[name] = xo.cpu().numpy()
        cmp["fp64"]["form"] = "complex128 factors, FP64 GMRES(30) on the split system"
        cmp["chosen"]["form"] = "the bench's chosen form (same kernels and solver as the timed region)"
        cmp["angles"] = f"the first {PLAIN_NRHS} of the workload's 256 plane waves"
        cmp["speedup"] = cmp["chosen"]["value"] / cmp["fp64"]["value"]
        out["plain"] = cmp
        out["err_vs_fp64"] = float(max(np.linalg.norm(xs["chosen"][r] - xs["fp64"][r]) / np.linalg.norm(xs["fp64"][r])
                                       for r in range(PLAIN_NRHS)))
        del f64
        hb.hb_autotune(f32, NRHS)
    return out


def run_kernels(args):
    """Kernel timings (no Krylov loop): hb_apply, one L~ sweep and one U~ sweep on one workload,
    and the three adjoint counterparts, with algorithmic bytes per launch and the fraction of
    the measured HBM copy bandwidth."""
    import torch

    import paper_1901_11371_gb300 as hb
    from paper_1901_11371_gb300 import build as hb_build
    hb_build.build()
    wl = {"spiral": W.SPIRAL_N65536, "semicircle": W.SEMICIRCLE_N262144, "strips": W.STRIPS8_N131072, "strip": W.STRIP_N1024}[args.workload]
    R = args.nrhs
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    form = {"c64": hb.HB_C64, "c128": hb.HB_C128, "split": hb.HB_SPLIT_BF16}[args.form]
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=form)
    tuned, times = None, {}
    if args.grid_min:
        hb.lib().hb_set_sweep_grid_min(f._h, args.grid_min)
    if args.sweep_kernel >= 0:
        hb.hb_set_sweep_kernel(f, args.sweep_kernel)
    elif not args.grid_min:
        tuned = hb.hb_autotune(f, R)
        times = hb.hb_autotune_times(f, R)
    st = hb.hb_factor_info(f)
    dt = torch.complex128 if args.form == "c128" else torch.complex64
    x = torch.randn((R, wl.n) if R > 1 else (wl.n,), dtype=dt, device="cuda")

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    hbm, src = _peaks()
    ms_a = timed(lambda: hb.hb_apply(f, x), args.steps)
    ms_l = timed(lambda: hb.hb_lower_solve(f, x), args.steps)
    ms_u = timed(lambda: hb.hb_upper_solve(f, x), args.steps)
    # adjoint (Sec. 3 operators conjugate-transposed): A^H, L~^{-H} and U~^{-H}
    ms_ah = timed(lambda: hb.hb_apply(f, x, op=hb.HB_OP_H), args.steps)
    ms_lh = timed(lambda: hb.hb_lower_solve(f, x, hb.HB_OP_H), args.steps)
    ms_uh = timed(lambda: hb.hb_upper_solve(f, x, hb.HB_OP_H), args.steps)
    eb = 16 if args.form == "c128" else 8
    vec_extra = 2 * wl.n * (R - 1) * eb
    out = {"mode": "kernels", "workload": wl.name, "nrhs": R, "form": args.form,
           "grid_min": args.grid_min or tuned, "sweep_kernel": args.sweep_kernel, "autotune_ms": times,
           "apply_ms": ms_a, "lower_ms": ms_l, "upper_ms": ms_u,
           "adjoint_apply_ms": ms_ah, "adjoint_lower_ms": ms_lh, "adjoint_upper_ms": ms_uh,
           "apply_GBps": (st["apply_bytes"] + vec_extra) / ms_a / 1e6,
           "lower_GBps": (st["lower_bytes"] + vec_extra) / ms_l / 1e6,
           "apply_frac": (st["apply_bytes"] + vec_extra) / ms_a / 1e6 / hbm, "peak_GBps": hbm, "peak_source": src,
           "apply_bytes": st["apply_bytes"], "lower_bytes": st["lower_bytes"], "kmax": st["kmax"],
           "kavg": st["kavg"], "device_bytes": st["device_bytes"]}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="solve", choices=["solve", "kernels"])
    ap.add_argument("--workload", default="spiral", choices=["spiral", "semicircle", "strips", "strip"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--form", default="c64", choices=["c64", "c128", "split"])
    ap.add_argument("--grid-min", type=int, default=0)
    ap.add_argument("--sweep-kernel", type=int, default=-1, choices=[-1, 0, 1],
                    help="kernels mode: -1 autotune, 0 cooperative, 1 column-partitioned")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--gmres-graph", type=int, default=1, choices=[0, 1],
                    help="1: every restart cycle one CUDA graph launch; 0: the host-driven Arnoldi loop "
                         "(the same kernels, launched one by one: what ncu can list kernel by kernel)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.mode == "kernels":
        run_kernels(args)
        return

    if args.impl == "reference":
        # the oracle as it stands, timed on this host's cores (rank 0 only)
        if rank != 0:
            return
        r = oracle_timed(steps=args.steps, warmup=args.warmup)
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": f"semicircle_N{SAMPLE_N}: the bench workload's curve family (40 segments "
                                       f"per wavelength, leaf 64, eps 1e-6) at N={SAMPLE_N}, one plane wave per step",
                           "full_workload": "semicircle_N262144 (256 plane waves) is out of the oracle's reach"},
                "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "model_estimate": r["model_estimate"],
                "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    out = run_gpu(args, rank, world)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    st = out["st"]
    hbm, peak_kind = _peaks()
    # dominant kernel: the sweep kernel (two per iteration) vs the apply sequence
    sweep_ms = out["ms_sweep"] / max(out["n_sweep"], 1)
    apply_ms = out["ms_apply"] / max(out["n_apply"], 1)
    # algorithmic bytes of one launch over the NRHS-column block: every factor and
    # index entry once, every right-hand side's vector read and written once
    # (hb_factor_info reports the single-column figure)
    vec_extra = 2 * st["n"] * (NRHS - 1) * 8
    sweep_bytes = 0.5 * (st["lower_bytes"] + st["upper_bytes"]) + vec_extra
    apply_bytes = st["apply_bytes"] + vec_extra
    sweep_kernel = "k_sweep_cols" if out["tuned"] == 0 else "k_sweep"
    dominant = sweep_kernel if out["ms_sweep"] >= out["ms_apply"] else "apply (k_apply_*)"
    if dominant == sweep_kernel:
        achieved = sweep_bytes / (sweep_ms / 1e3) / 1e9
        algo = sweep_bytes
        avg_ms = sweep_ms
    else:
        achieved = apply_bytes / (apply_ms / 1e3) / 1e9
        algo = apply_bytes
        avg_ms = apply_ms
    # DRAM bytes of one launch from an ncu capture of the same kernel revision on this
    # workload (profiles/k_sweep_coop_semicircle_N262144_traffic.md); None when no capture
    # of the current revision exists
    traffic = measured_traffic(dominant.split()[0])
    line = {
        "metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": out["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16x3->f32 (tensor-core leaf contractions) + c64 (butterfly steps, sweeps) + f64 (Krylov, residuals)",
        "data": "synthetic",
        "config": {"workload": "semicircle_N262144: R = 6553.6/pi lambda, phi in [0, pi], N=262144, leaf 64, "
                               "eps 1e-6, 256 plane waves phi_i = 180 i/256 deg per step",
                   "form": f"split-BF16: FP64 FGMRES({RESTART}) + IR around U~^-1 L~^-1 (complex FP32) and A_F "
                           "(leaf contractions on tcgen05 tensor cores, butterfly steps complex FP32)",
                   "rhs_per_step": NRHS, "sweep_grid_min": out["tuned"],
                   "sweep_kernel": "column-partitioned (k_sweep_cols)" if out["tuned"] == 0
                                   else f"cooperative (k_sweep_coop, grid_min {out['tuned']})",
                   "sweep_autotune_ms": {str(k): round(v, 3) for k, v in out["tune_ms"].items()},
                   "krylov_cycle": f"one CUDA graph launch per restart cycle ({out['graph_launches']} per solve)"
                                   if out["graph_launches"] else "host-driven Arnoldi loop",
                   "l2": f"inputs larger than L2: factor {st['device_bytes'] / 1e6:.0f} MB",
                   "kmax": st["kmax"], "kavg": round(st["kavg"], 2), "build_s": round(out["t_build"], 2)},
        "iters_per_solve": out["iters"], "ir_steps_per_solve": out["ir_steps"], "true_rel_res": out["res"],
        "monostatic_dB_every_32nd_angle": out["mono_db"],
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "algorithmic_bytes_per_launch": algo,
                     "avg_launch_ms": avg_ms, "peak_source": peak_kind,
                     "sweep_launches": out["n_sweep"], "sweep_ms_total": out["ms_sweep"],
                     "apply_calls": out["n_apply"], "apply_ms_total": out["ms_apply"],
                     "apply_GBps": apply_bytes / (apply_ms / 1e3) / 1e9 if out["n_apply"] else None,
                     "us_per_leaf_step": sweep_ms * 1e3 / (st["n"] // st["leaf"])},
        "roofline_single_column_apply": {
            "bound": "hbm", "kernel": "k_apply1 (one column, complex64 factors, same factor)",
            "achieved": st["apply_bytes"] / (out["apply1_ms"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": st["apply_bytes"] / (out["apply1_ms"] / 1e3) / 1e9 / hbm,
            "algorithmic_bytes_per_launch": st["apply_bytes"], "avg_launch_ms": out["apply1_ms"],
            "traffic": measured_traffic("k_apply1"), "peak_source": peak_kind},
        "gpu_launches": out["n_launch"],
        "clocks": out["clocks"],
        "e2e": out["e2e"],
    }
    if "plain" in out:
        line["form_comparison"] = out["plain"]
        line["err_vs_fp64"] = out["err_vs_fp64"]
    if not args.no_cpu:
        try:
            r = oracle_timed(steps=8, warmup=1)
            line["cpu_baseline"] = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
            line["cpu_baseline"]["model_estimate"] = r["model_estimate"]
        except Exception as e:  # the oracle leg must never hide the GPU result
            line["cpu_baseline"] = {"error": str(e)[:200]}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
