#!/usr/bin/env python
"""Benchmark of the GB300 pressure-correction path.

One step = one full FP64 RK3 / Crank-Nicolson time step of the Rayleigh-Benard
workload (Ra = 1e8, Pr = 1, 512 x 512 x 384 cells, tanh-stretched wall-normal
grid): the CFL reduction (Listing 1) and three substeps, each with the
explicit terms, four Crank-Nicolson wall-normal sweeps and the pressure
correction (divergence fused into the forward x FFT, y FFT, Thomas sweeps,
inverse FFTs, projection). Inputs are seeded synthetic fields resident in HBM
(each field is 805 MB, larger than L2, so no flush is needed between steps).

Printed: one JSON line (rank 0) with the headline grid-points/s, the roofline
of the dominant kernel family (CUDA events around every launch group inside
the timed region), the FP64 oracle timed on the host cores on a bounded
sample, the end-to-end number with host buffers, clocks sampled during the
timed region, and side measurements (Poisson solve alone, FP64 vs mixed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# Nominal FP64 issue rate of this part, for context only: 2 FP64 operations
# (add, multiply or fused multiply-add alike) per clock per SM x 152 SMs x the
# 2070 MHz maximum SM clock. The ALU roofline of the FP64 kernels uses the rate
# measured in the same run by afid_probe_fp64_rate (FMA chains, an FMA counted
# as one operation), each add, multiply or FMA of a kernel's formulation
# counted once against it.
FP64_OPS_NOMINAL = 2 * 152 * 2.070e9 / 1e12          # 0.629 T FP64 ops/s
# The mixed-precision solve is measured at the accuracy it is held to: a
# relative error of 1e-10 against the FP64 solve (its stopping rule's target).
MIXED_TOL = 1e-10


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rb512")
    ap.add_argument("--no-extra", action="store_true", help="skip the side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--poisson-only", action="store_true",
                    help="only the Poisson-solve side measurement (FP64 and mixed)")
    ap.add_argument("--no-tma", action="store_true",
                    help="use the plain y-transform kernel instead of the TMA-staged one")
    ap.add_argument("--fuse", default="auto", choices=["auto", "on", "off"],
                    help="mixed: the small-nz kernel fusing the y transforms and the Thomas sweeps "
                         "(auto: where measured faster; on: wherever it fits; off: never)")
    ap.add_argument("--multires-only", action="store_true",
                    help="only the refined-temperature-grid coupled step (2x2x2, afid_mr_step)")
    ap.add_argument("--grid", default=None,
                    help="override the workload's cells as NXxNYxNZ (profiling smaller cases)")
    return ap.parse_args(argv)


def workload_from(args):
    import synth
    w = synth.workload(args.workload)
    if args.grid:
        nx, ny, nz = (int(t) for t in args.grid.lower().split("x"))
        w.nx, w.ny, w.nz = nx, ny, nz
    return w


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if sm:
            top = max(sm)
            loaded = [s for s in sm if s >= 0.5 * top] or sm
            out = {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ------------------------------------------------------------------ work model
def fft_ops(n: int) -> float:
    """FP64 operations per complex point of one n-point transform with the
    library's pass sequence (radix 8 first, untwiddled, then twiddled radix-8
    passes, then one radix-4 or radix-2 pass): 6.5, 8.25, 7, 4 per point (a
    radix-8 butterfly is 52 operations with its 1/sqrt(2) scalings fused into
    FMAs; the twiddled radix-8 passes take their seven twiddles in tangent form,
    kappa (1 + i t), two FMAs each, the kappas folded into the butterfly's
    additions: 66 per butterfly; a complex twiddle of the last radix-4 or
    radix-2 pass 4; the last radix-4 pass of a power-of-two length of at least
    64 also takes the tangent form: 22 per butterfly, 5.5 per point). The
    tangent form is used for power-of-two lengths of at least 64; other
    lengths take 10 per twiddled radix-8 pass."""
    tangent = n >= 64 and n & (n - 1) == 0
    ops, p = 0.0, 1
    while n // p >= 8:
        ops += 6.5 if p == 1 else (8.25 if tangent else 10.0)
        p *= 8
    if n // p == 4:
        ops += 5.5 if tangent else 7.0
    elif n // p == 2:
        ops += 4.0
    return ops


def family_work(fam: str, w):
    """Algorithmic work of one launch group of a kernel family on grid w:
    (bytes, fp64_ops). Bytes: compulsory HBM traffic of the kernel's own inputs
    and outputs. FP64 operations: the formulation's arithmetic, each add,
    multiply or FMA counted once (per grid point unless noted):
      r2c_x  divergence 6 + packed real FFT fft_ops(nx/2)/2 + unpacking 3 (its
             halves folded into FMAs and a halved twiddle table)
      c2r_x  packing 3 (the 1/(nx ny) normalisation folded in) + fft_ops(nx/2)/2
      fft_y  fft_ops(ny) per complex point (nx/2+1 complex per row)
      thomas 7 per complex point (4 forward, 3 backward)
      project 9; rhs 104 (shared face fluxes 25, u 20, v 20, w 20, T 16, per-plane
      factors 3; the recomputed fluxes of the warp- and block-edge neighbours are
      overhead, not counted); crank_nicolson 8 (4 fields: one forward-elimination
      FMA, the reciprocal pivot being folded into the right-hand side the
      explicit-terms kernel writes, and one back-substitution FMA each on the
      FP64 pipe; the q += dq addition is an atomic done in L2);
      cfl_reduce 6 (|.| is an operand modifier; the maximum is taken on the bit
      patterns with integer instructions)."""
    nx, ny, nz = w.nx, w.ny, w.nz
    n = nx * ny * nz
    M1 = nx // 2 + 1
    nc = M1 * ny * nz
    if fam == "r2c_x":
        return 24 * n + 16 * nc, (6 + fft_ops(nx // 2) / 2 + 3) * n
    if fam == "c2r_x":
        return 16 * nc + 8 * n, (3 + fft_ops(nx // 2) / 2) * n
    if fam == "fft_y":
        return 32 * nc, fft_ops(ny) * nc
    if fam == "thomas":
        return 32 * nc + 8 * M1 * (ny // 2 + 1) * nz, 7 * nc
    if fam == "project":
        return 72 * n, 9 * n
    if fam == "rhs":
        return 136 * n, 104 * n
    if fam == "crank_nicolson":
        return 4 * 24 * n, 8 * n
    if fam == "cfl_reduce":
        return 24 * n, 6 * n
    return None


# the translation unit holding each captured kernel family
FAMILY_SOURCE = {"r2c_x": "k_spectral.cu", "fft_y": "k_spectral.cu", "thomas": "k_spectral.cu",
                 "zero_mode": "k_spectral.cu", "c2r_x": "k_spectral.cu", "project": "k_physical.cu",
                 "crank_nicolson": "k_physical.cu", "cn_tables": "k_physical.cu", "rhs": "k_rhs.cu"}


def src_hash(fam: str) -> str:
    """Hash of the sources a family's kernels are compiled from: its translation
    unit and the two internal headers every kernel includes."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1705_01423_gb300", "csrc")
    for f in (FAMILY_SOURCE[fam], "afid_internal.cuh", "fft.cuh"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(fam: str, w):
    """DRAM bytes per launch group from the committed ncu summary, scaled to the
    workload; None when missing or taken on different sources of that family."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p) or fam not in FAMILY_SOURCE:
        return None
    e = json.load(open(p)).get("families", {}).get(fam)
    if not e or e.get("src_hash") != src_hash(fam):
        return None
    return e["bytes_per_point"] * w.nx * w.ny * w.nz


# ------------------------------------------------------------------ oracle baseline
def oracle_step_time(nx, ny, nz, steps=1, warmup=0):
    import torch
    import synth
    from oracle import Grid, timestep as ts
    w = synth.workload("rb512", nx=nx, ny=ny, nz=nz)
    g = Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces())
    ph = ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, T_bot=w.T_bot, T_top=w.T_top)
    st = tuple(torch.as_tensor(a) for a in synth.rb_initial(w, 0))
    H = None
    from oracle import operators as op
    for _ in range(warmup):
        st, H = ts.step(g, ph, op.cfl_dt(g, st[0], st[1], st[2], w.cfl, w.dt_max), st, H)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        dt = op.cfl_dt(g, st[0], st[1], st[2], w.cfl, w.dt_max)
        st, H = ts.step(g, ph, dt, st, H)
        times.append(time.perf_counter() - t0)
    return times, torch.get_num_threads()


# ------------------------------------------------------------------ main (ours)
def run_poisson_only(args):
    """Poisson solve alone on the workload grid: FP64 direct and mixed FP32 +
    FP64 refinement, contexts created one after the other (the 2048^2 x 1024
    grid needs about 110 GB for the FP64 context and 132 GB for the mixed one)."""
    import torch
    import synth
    from paper_1705_01423_gb300 import Context
    w = workload_from(args)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    pts = w.nx * w.ny * w.nz
    if w.name == "poisson2048":
        bh, _ = synth.manufactured_rhs(w, seed=0)
        b = torch.from_numpy(bh).to(dev)
        del bh
    else:
        b = torch.as_tensor(synth.noise((w.nz, w.ny, w.nx), seed=123)).to(dev)
    out = {}
    tma = not args.no_tma
    ctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), poisson_only=True, tma=tma)
    phi64 = torch.empty_like(b)
    ms64 = timed(lambda: ctx.poisson_solve(b, phi64), 5, stream)
    ctx.profile(True)
    ctx.profile_read()
    ctx.poisson_solve(b, phi64)
    fam64 = {k: v[0] for k, v in ctx.profile_read().items() if v[1]}
    ctx.close()
    del ctx
    torch.cuda.synchronize()
    out["poisson_fp64"] = {"ms": ms64, "grid_points_per_s": pts / (ms64 / 1e3), "families_ms": fam64}
    mctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), precision="mixed", refine_tol=MIXED_TOL,
                   refine_max_iter=6, poisson_only=True, tma=tma,
                   fuse={"auto": None, "on": True, "off": False}[args.fuse])
    phim = torch.empty_like(b)
    _, info = mctx.poisson_solve(b, phim, info=True)
    msm = timed(lambda: mctx.poisson_solve(b, phim), 5, stream)
    mctx.profile(True)
    mctx.profile_read()
    mctx.poisson_solve(b, phim)
    famm = {k: v[0] for k, v in mctx.profile_read().items() if v[1]}
    err = float((phim - phi64).norm() / phi64.norm())
    out["poisson_mixed"] = {"ms": msm, "grid_points_per_s": pts / (msm / 1e3), "iters": info["iters"],
                            "refine_tol": MIXED_TOL, "rel_l2_vs_fp64_gpu": err,
                            "err_estimate": info["err_estimate"], "speedup_vs_fp64": ms64 / msm,
                            "families_ms": famm}
    print(json.dumps({"workload": "%s %dx%dx%d" % (w.name, w.nx, w.ny, w.nz), "tma_y": tma,
                      "fuse": args.fuse, "poisson": out}))


def run_multires_only(args):
    """The refined-temperature-grid measurement alone on the workload grid."""
    import torch
    from paper_1705_01423_gb300 import Context, Physics
    w = workload_from(args)
    dev = torch.device("cuda", 0)
    ph = Physics(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                 T_bot=w.T_bot, T_top=w.T_top)
    ctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), phys=ph)
    peak, _ = fp64_probe(ctx, 0)
    out = multires_measurement(ctx, w, dev, fp64_peak=peak)
    print(json.dumps({"workload": "%s %dx%dx%d" % (w.name, w.nx, w.ny, w.nz), "multires": out}))


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (the whole job ends when it does)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def whole_job_rate(points_per_replica: int, world: int, steps: int, ms: float) -> float:
    """Grid points of every replica and step per second of the slowest rank."""
    return points_per_replica * world * steps / (ms / 1e3)


def replica_state(w, rank: int):
    """Host fields (u, v, w, T or None, p) of one replica: the workload's start
    state drawn with the rank as seed, so replicas solve different problems."""
    import synth
    if w.has_T:
        return synth.rb_initial(w, seed=rank)
    u0, v0, w0, p0 = synth.couette_initial(w, seed=rank)
    return (u0, v0, w0, None, p0)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_1705_01423_gb300 import Context, Physics

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = workload_from(args)
    ph = Physics(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                 T_bot=w.T_bot, T_top=w.T_top)
    ctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), phys=ph, tma=not args.no_tma)
    host = replica_state(w, rank)
    S = [torch.as_tensor(a).to(dev) if a is not None else None for a in host]
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]),
         torch.zeros_like(S[3]) if S[3] is not None else None]

    def step():
        ctx.cfl(S[0], S[1], S[2], w.cfl, w.dt_max)
        for l in range(3):
            ctx.rk3_substep(l, -1.0, *S, *H)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    fp64_peak, probe = fp64_probe(ctx, local)
    ctx.profile(True)
    ctx.profile_read()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    l0 = ctx.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    launches = ctx.kernel_launches() - l0
    fams = ctx.profile_read()
    ctx.profile(False)
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_step = ms / args.steps
    pts = w.nx * w.ny * w.nz
    value = whole_job_rate(pts, world, args.steps, ms)
    # state sanity: still divergence free
    mdiv = float(ctx.max_divergence(S[0], S[1], S[2]))

    # ---- roofline of the dominant kernel family
    peaks, peak_src = measured_peaks()
    top = max((f for f in fams if family_work(f, w)), key=lambda f: fams[f][0])
    tms, tn = fams[top]
    per_launch_ms = tms / max(tn, 1)
    bytes_, ops = family_work(top, w)
    t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9)
    t_alu = ops / (fp64_peak * 1e12)
    if t_alu > t_hbm:
        ach = ops / (per_launch_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak, "traffic": traffic_for(top, w),
                "kernel": top, "launch_ms": per_launch_ms,
                "peak_source": "measured in this run: afid_probe_fp64_rate (independent FP64 FMA chains, "
                               "FMA = 1 operation), best of %d launches at a median SM clock of %s MHz; "
                               "FLOP here = one FP64 add, mul or FMA of the kernel's formulation"
                               % (probe["launches"], probe["sm_mhz"]),
                "peak_nominal": FP64_OPS_NOMINAL, "fp64_probe": probe,
                "hbm_gbs_algorithmic": bytes_ / (per_launch_ms / 1e3) / 1e9,
                "hbm_frac_of_measured": (bytes_ / (per_launch_ms / 1e3) / 1e9) / peaks["hbm_gbs"]}
    else:
        ach = bytes_ / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic_for(top, w), "kernel": top,
                "launch_ms": per_launch_ms, "peak_source": peak_src + " copy bandwidth"}
    fam_report = {}
    tot_ms = max(sum(x[0] for x in fams.values()), 1e-9)
    for f, v in fams.items():
        if not v[1]:
            continue
        e = {"ms_per_step": v[0] / args.steps, "launch_groups_per_step": v[1] / args.steps,
             "share": v[0] / tot_ms}
        fw = family_work(f, w)
        if fw:
            t = v[0] / v[1] / 1e3
            e["fp64_ops_frac"] = fw[1] / t / 1e12 / fp64_peak
            e["hbm_frac_algorithmic"] = fw[0] / t / 1e9 / peaks["hbm_gbs"]
        fam_report[f] = e

    # ---- end to end with host buffers (same metric through the API). Every
    # step uploads its input state from pinned host memory and reads its result
    # back, inside the timed region. Pipelined: two device state buffers, the
    # next step's upload and the previous step's read-back on their own copy
    # streams while the current step computes; the serial form (copy, step,
    # copy) is reported beside it.
    e2e = None
    if rank == 0 or world > 1:
        hS = [torch.as_tensor(a).pin_memory() if a is not None else None for a in host]
        oS = [torch.empty_like(a).pin_memory() if a is not None else None for a in hS]
        bi = sum(a.numel() * 8 for a in hS if a is not None)
        k2 = max(2, min(args.steps, 10))
        S2 = [torch.empty_like(a) if a is not None else None for a in S]
        bufs = [S, S2]

        def step_on(St):
            ctx.cfl(St[0], St[1], St[2], w.cfl, w.dt_max)
            for l in range(3):
                ctx.rk3_substep(l, -1.0, *St, *H)

        def copy_all(dst, src):
            for d_, s_ in zip(dst, src):
                if d_ is not None:
                    d_.copy_(s_, non_blocking=True)

        def e2e_serial():
            for _ in range(k2):
                copy_all(S, hS)
                step_on(S)
                copy_all(oS, S)

        def e2e_pipelined():
            h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
            ev_in = [torch.cuda.Event() for _ in range(k2)]
            ev_done = [torch.cuda.Event() for _ in range(k2)]
            ev_out = [torch.cuda.Event() for _ in range(k2)]
            start = torch.cuda.Event()
            start.record(stream)
            h2d.wait_event(start)
            d2h.wait_event(start)

            def upload(i):
                with torch.cuda.stream(h2d):
                    if i >= 2:  # the buffer's previous result has been read back
                        h2d.wait_event(ev_out[i - 2])
                    copy_all(bufs[i % 2], hS)
                    ev_in[i].record(h2d)

            upload(0)
            for i in range(k2):
                if i + 1 < k2:
                    upload(i + 1)
                stream.wait_event(ev_in[i])
                step_on(bufs[i % 2])
                ev_done[i].record(stream)
                with torch.cuda.stream(d2h):
                    d2h.wait_event(ev_done[i])
                    copy_all(oS, bufs[i % 2])
                    ev_out[i].record(d2h)
            stream.wait_event(ev_out[k2 - 1])

        times = {}
        for name, fn in (("serial", e2e_serial), ("pipelined", e2e_pipelined)):
            e2 = torch.cuda.Event(enable_timing=True)
            e3 = torch.cuda.Event(enable_timing=True)
            barrier()
            torch.cuda.synchronize()
            e2.record(stream)
            fn()
            e3.record(stream)
            torch.cuda.synchronize()
            times[name] = max_over_ranks(e2.elapsed_time(e3), world, dev)
        # the host link alone: one state upload and one read-back, each by itself
        link = {}
        for name, fn in (("h2d", lambda: copy_all(S, hS)), ("d2h", lambda: copy_all(oS, S))):
            e2 = torch.cuda.Event(enable_timing=True)
            e3 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e2.record(stream)
            fn()
            e3.record(stream)
            torch.cuda.synchronize()
            link[name + "_gbs"] = bi / (e2.elapsed_time(e3) / 1e3) / 1e9
        e2e = {"value": whole_job_rate(pts, world, k2, times["pipelined"]), "unit": "grid-points/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bi, "steps": k2,
               "serial_value": whole_job_rate(pts, world, k2, times["serial"]), "host_link": link,
               "note": "every step uploads its state from pinned host memory and reads its result back; "
                       "value: uploads and read-backs on two copy streams overlapping the neighbouring "
                       "steps (two device state buffers); serial_value: copy, step, copy in order"}
        del S2, bufs

    # ---- side measurements: Poisson solve alone, FP64 vs mixed
    extra = {}
    if not args.no_extra and rank == 0:
        extra = side_measurements(ctx, w, dev, tma=not args.no_tma, state=S, fp64_peak=fp64_peak)

    # ---- the large mixed-precision Poisson solve (2048 x 2048 x 1024), after
    # the step's context and fields are released (it needs about 255 GB)
    if not args.no_extra and rank == 0:
        ctx.close()
        del S, H
        torch.cuda.empty_cache()
        try:
            extra["poisson2048"] = poisson2048_measurement(dev)
        except Exception as e:  # report, do not hide
            extra["poisson2048"] = {"error": str(e)}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = 256
        ts_, thr = oracle_step_time(ns, ns, w.nz, steps=2)
        cpu = {"value": ns * ns * w.nz * len(ts_) / sum(ts_), "unit": "grid-points/s", "cores": thr,
               "kind": "oracle", "host_cpus": os.cpu_count(),
               "sample": "two FP64 oracle RK3 steps (CFL + 3 substeps each) of the same Rayleigh-Benard "
                         "workload on %dx%dx%d cells (1/4 of the horizontal points), %.1f s"
                         % (ns, ns, w.nz, sum(ts_))}

    if rank == 0:
        out = {
            "metric": "grid-points/s per FP64 RK3/CN time step (Rayleigh-Benard Ra=1e8, 512x512x384)",
            "value": value, "unit": "grid-points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: conduction profile T = 1 - z plus seeded U(-1e-3, 1e-3) noise, velocity 0 at start",
            "config": {"workload": "rb512: Rayleigh-Benard Ra=1e8 Pr=1 aspect 1, %dx%dx%d cells, tanh-stretched z (s=1.5), "
                                   "FP64 RK3/CN step = CFL + 3 x (explicit terms, 4 CN sweeps, pressure correction)"
                                   % (w.nx, w.ny, w.nz),
                       "l2": "inputs larger than L2 (805 MB per field), no flush needed",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "kernel_families": fam_report, "max_div_after": mdiv, "extra": extra,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def fp64_probe(ctx, gpu_index, launches=12, iters=20000):
    """The FP64 rate this GPU delivers (afid_probe_fp64_rate), best of
    `launches` timed launches, with the SM clock sampled meanwhile: the peak
    of the ALU roofline, in T FP64 operations per second."""
    clk = ClockSampler(gpu_index)
    clk.start()
    rates = [ctx.probe_fp64_rate(iters) for _ in range(launches)]
    c = clk.stop()
    best = max(r for r, _ in rates)
    return best / 1e12, {"ops_per_s": best, "launches": launches, "ms_per_launch": min(m for _, m in rates),
                         "sm_mhz": c["sm_mhz"], "reasons": c["reasons"],
                         "per_clock_per_sm": (best / (c["sm_mhz"] * 1e6 * 152)) if c["sm_mhz"] else None}


def poisson2048_measurement(dev, reps=3):
    """The large mixed-precision Poisson solve: 2048 x 2048 x 1024 cells,
    tanh-stretched z, rhs = seeded N(0,1) noise + 8 manufactured modes
    cos(2 pi a x) cos(2 pi b y) cos(pi m z). FP64 direct solve and mixed FP32
    solve with FP64 refinement to 1e-10, their times and speedup; the errors of
    both against the sampled-mode FP64 oracle (16 (kx, ky) columns: the 8
    manufactured pairs, (0,0), the lowest and Nyquist pairs, seeded others; a
    direct DFT of the whole rhs and FP64 Thomas per column), of the mixed
    solve against the FP64 solve, and of the modes-only solve against the
    continuum closed form -sum cos cos cos / (4 pi^2 (a^2 + b^2) + pi^2 m^2)
    (the second-order discretisation error)."""
    import numpy as np
    import torch
    import synth
    from oracle import Grid, sampled
    from paper_1705_01423_gb300 import Context
    w = synth.workload("poisson2048")
    free, _ = torch.cuda.mem_get_info()
    need = 255e9
    if free < need:
        return {"skipped": "needs about %.0f GB of free device memory, %.0f GB free" % (need / 1e9, free / 1e9)}
    stream = torch.cuda.current_stream()
    g = Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces())
    t0 = time.perf_counter()
    bh, modes = synth.manufactured_rhs(w, seed=0)
    B = torch.from_numpy(bh).to(dev)
    t_gen = time.perf_counter() - t0
    pairs = [(a, b) for a, b, _ in modes]
    for p in sampled.default_pairs(g, seed=2, count=10):
        if p not in pairs:
            pairs.append(p)
    t0 = time.perf_counter()
    ref = sampled.solve_modes(g, bh, pairs)
    t_oracle = time.perf_counter() - t0
    del bh

    def sampled_err(phi):
        got = sampled.mode_columns(g, phi, pairs)
        num = sum(np.linalg.norm(got[p] - ref[p]) ** 2 for p in pairs)
        den = sum(np.linalg.norm(ref[p]) ** 2 for p in pairs)
        return math.sqrt(num / den)

    pts = w.nx * w.ny * w.nz
    ctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), poisson_only=True)
    phi64 = torch.empty_like(B)
    ms64 = timed(lambda: ctx.poisson_solve(B, phi64), reps, stream)
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
    err64 = sampled_err(phi64)
    mctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), precision="mixed", refine_tol=MIXED_TOL,
                   refine_max_iter=6, poisson_only=True)
    phim = torch.empty_like(B)
    _, info = mctx.poisson_solve(B, phim, info=True)
    msm = timed(lambda: mctx.poisson_solve(B, phim), reps, stream)
    errm = sampled_err(phim)
    err_m64 = float((phim - phi64).norm() / phi64.norm())
    del phi64
    torch.cuda.empty_cache()
    # modes only (deterministic cosines built on the device), against the closed form
    zc = torch.as_tensor(g.zc.numpy(), device=dev)
    xc = (torch.arange(w.nx, device=dev, dtype=torch.float64) + 0.5) * (w.lx / w.nx)
    yc = (torch.arange(w.ny, device=dev, dtype=torch.float64) + 0.5) * (w.ly / w.ny)
    B.zero_()
    for a, b, m in modes:
        B += (torch.cos(math.pi * m * zc)[:, None, None] * torch.cos(2 * math.pi * b * yc / w.ly)[None, :, None]
              * torch.cos(2 * math.pi * a * xc / w.lx)[None, None, :])
    mctx.poisson_solve(B, phim)
    exact = B
    exact.zero_()
    for a, b, m in modes:
        lam = 4 * math.pi ** 2 * (a ** 2 / w.lx ** 2 + b ** 2 / w.ly ** 2) + math.pi ** 2 * m ** 2
        exact -= (torch.cos(math.pi * m * zc)[:, None, None] * torch.cos(2 * math.pi * b * yc / w.ly)[None, :, None]
                  * torch.cos(2 * math.pi * a * xc / w.lx)[None, None, :]) / lam
    dzc = torch.as_tensor(g.dzc.numpy(), device=dev)[:, None, None]
    exact -= float((dzc * exact).sum() / (dzc.sum() * w.nx * w.ny))
    err_closed = float((phim - exact).norm() / exact.norm())
    mctx.close()
    del mctx, B, phim, exact
    torch.cuda.empty_cache()
    return {"grid": [w.nx, w.ny, w.nz], "fp64_ms": ms64, "mixed_ms": msm, "speedup": ms64 / msm,
            "fp64_grid_points_per_s": pts / (ms64 / 1e3), "mixed_grid_points_per_s": pts / (msm / 1e3),
            "mixed_iters": info["iters"], "refine_tol": MIXED_TOL, "err_estimate": info["err_estimate"],
            "fp64_rel_l2_vs_sampled_oracle": err64, "mixed_rel_l2_vs_sampled_oracle": errm,
            "mixed_rel_l2_vs_fp64_gpu": err_m64, "modes_only_rel_l2_vs_closed_form": err_closed,
            "sampled_pairs": len(pairs), "host_rhs_generation_s": t_gen, "sampled_oracle_s": t_oracle}


def timed(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def mixed_step_measurement(ctx, w, dev, state, tma=True, reps=3):
    """The whole RK3/CN step with the mixed-precision Poisson solve (FP32
    transforms and sweeps, FP64 residual refinement to 1e-10) against the FP64
    step: time per step, and the relative L2 difference of every field after
    one step of each from the same state with the same dt."""
    import torch
    from paper_1705_01423_gb300 import Context, Physics
    stream = torch.cuda.current_stream()
    ph = Physics(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                 T_bot=w.T_bot, T_top=w.T_top)
    mctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), precision="mixed", refine_tol=MIXED_TOL,
                   refine_max_iter=6, phys=ph, tma=tma)
    dt = float(w.dt_max)
    clone = lambda xs: [x.clone() if x is not None else None for x in xs]
    zeros = lambda xs: [torch.zeros_like(x) if x is not None else None for x in xs[:4]]
    S64, Sm = clone(state), clone(state)
    H64, Hm = zeros(state[:3] + [state[3]]), zeros(state[:3] + [state[3]])
    ctx.rk3_step(S64, H64, dt)
    mctx.rk3_step(Sm, Hm, dt)
    torch.cuda.synchronize()
    names = ["u", "v", "w", "T", "p"]
    err = {n: float((a - b).norm() / max(float(b.norm()), 1e-300))
           for n, a, b in zip(names, Sm, S64) if a is not None}
    Sw, Hw = clone(state), zeros(state[:3] + [state[3]])
    ms_m = timed(lambda: mctx.rk3_step(Sw, Hw, dt), reps, stream)
    ms_64 = timed(lambda: ctx.rk3_step(Sw, Hw, dt), reps, stream)
    mctx.close()
    pts = w.nx * w.ny * w.nz
    return {"ms_per_step_mixed": ms_m, "ms_per_step_fp64": ms_64, "speedup": ms_64 / ms_m,
            "grid_points_per_s_mixed": pts / (ms_m / 1e3), "refine_tol": MIXED_TOL,
            "rel_l2_vs_fp64_step": err, "dt": dt,
            "note": "one step from the benchmark's state after its timed steps, fixed dt = dt_max"}


def workload_measurements(dev, reps=5):
    """The other workloads of the benchmark set, each on its own context:
    the pressure correction on 64^3 (L2-resident and latency-bound: reported,
    not held to a roofline), the plane Couette RK3 step at 1024x512x256 with
    its FP64 and mixed Poisson solves, and the adjoint rollout (forward and
    backward of dNu/dT0 over 20 steps, checkpoints every 5) at 256x256x128."""
    import torch
    import synth
    from paper_1705_01423_gb300 import Context, Physics
    from paper_1705_01423_gb300.autodiff import nusselt_gradient, _run_step
    stream = torch.cuda.current_stream()
    out = {}
    phys = lambda w: Physics(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                             T_bot=w.T_bot, T_top=w.T_top)
    # plain FP64 pressure correction, 64^3
    w = synth.workload("pc64")
    ctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), poisson_only=True)
    U, V, W = (torch.as_tensor(a).to(dev) for a in synth.velocity_noise(w, 0))
    P = torch.zeros(ctx.cell, dtype=torch.float64, device=dev)
    info = ctx.project(U, V, W, P, info=True)
    ms = timed(lambda: ctx.project(U, V, W, P), 20, stream)
    out["pc64_pressure_correction"] = {"ms": ms, "grid_points_per_s": w.nx * w.ny * w.nz / (ms / 1e3),
                                       "max_div_after_first": info["max_div"]}
    ctx.close()
    # plane Couette, 1024 x 512 x 256: RK3 step (CFL dt on the device), FP64 and mixed solves
    w = synth.workload("couette1024")
    ctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), phys=phys(w))
    S = [torch.as_tensor(a).to(dev) if a is not None else None for a in replica_state(w, 0)]
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]), None]

    def cstep():
        ctx.cfl(S[0], S[1], S[2], w.cfl, w.dt_max)
        for l in range(3):
            ctx.rk3_substep(l, -1.0, *S, *H)

    for _ in range(3):
        cstep()
    ms = timed(cstep, reps, stream)
    b = torch.as_tensor(synth.noise((w.nz, w.ny, w.nx), seed=7)).to(dev)
    phi = torch.empty_like(b)
    ms64 = timed(lambda: ctx.poisson_solve(b, phi), reps, stream)
    mctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), precision="mixed", refine_tol=MIXED_TOL,
                   refine_max_iter=6, poisson_only=True)
    phim = torch.empty_like(b)
    _, minfo = mctx.poisson_solve(b, phim, info=True)
    msm = timed(lambda: mctx.poisson_solve(b, phim), reps, stream)
    out["couette1024"] = {"rk3_step_ms": ms, "grid_points_per_s": w.nx * w.ny * w.nz / (ms / 1e3),
                          "poisson_fp64_ms": ms64, "poisson_mixed_ms": msm, "mixed_speedup": ms64 / msm,
                          "mixed_iters": minfo["iters"],
                          "mixed_rel_l2_vs_fp64": float((phim - phi).norm() / phi.norm())}
    mctx.close()
    ctx.close()
    del S, H, b, phi, phim
    torch.cuda.empty_cache()
    # adjoint rollout: Ra = 1e7, 256 x 256 x 128, 20 steps, checkpoints every 5
    w = synth.workload("adj256")
    ctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), phys=phys(w))
    st = [torch.as_tensor(a).to(dev) for a in synth.rb_initial(w, 0)]
    S = [a.clone() for a in st]
    dts = []
    for _ in range(w.steps):  # the rollout's dt sequence (CFL), frozen for the adjoint
        cflm = float(ctx.cfl(S[0], S[1], S[2], w.cfl, w.dt_max))
        dts.append(min(w.cfl / cflm, w.dt_max))
        _run_step(ctx, dts[-1], S)
    ra = w.extra["Ra"]
    nusselt_gradient(ctx, st, dts, ra, 1.0, checkpoint_every=w.extra["checkpoint_every"])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nu, gT = nusselt_gradient(ctx, st, dts, ra, 1.0, checkpoint_every=w.extra["checkpoint_every"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    S = [a.clone() for a in st]
    fwd = timed(lambda: [_run_step(ctx, dt, S) for dt in dts], 1, stream)
    out["adj256_nusselt_gradient"] = {"ms_forward_and_adjoint": ms, "ms_forward_only": fwd,
                                      "adjoint_over_forward": ms / fwd, "steps": w.steps,
                                      "checkpoint_every": w.extra["checkpoint_every"], "nu": nu,
                                      "grad_max_abs": float(gT.abs().max())}
    ctx.close()
    torch.cuda.empty_cache()
    return out


def tridiag_regime_measurement(dev, reps=20):
    """The warp-partitioned FP64 tridiagonal solver against one system per
    thread in the regime it is for: long wall-normal columns and few
    wavenumber pairs (the paper's Table 3 Ra = 1e11 grid has 1296 wall-normal
    points). FP64 Poisson solves of N(0,1) rhs on 64 x 64 x 1296, 32 x 32 x
    2048 and 128 x 128 x 1296 cells, tanh-stretched z: the Thomas-family time
    per solve with each solver, and the relative L2 difference of the two
    solutions."""
    import torch
    import synth
    from paper_1705_01423_gb300 import Context
    stream = torch.cuda.current_stream()
    out = {}
    for nx, ny, nz in ((64, 64, 1296), (32, 32, 2048), (128, 128, 1296)):
        w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
        b = torch.as_tensor(synth.noise((nz, ny, nx), seed=nz)).to(dev)
        res = {}
        phis = {}
        for name, warp in (("per_thread", False), ("warp_partitioned", True)):
            ctx = Context(nx, ny, nz, w.lx, w.ly, w.faces(), poisson_only=True, warp_tridiag=warp)
            phi = torch.empty_like(b)
            ms = timed(lambda: ctx.poisson_solve(b, phi), reps, stream)
            ctx.profile(True)
            ctx.profile_read()
            for _ in range(reps):
                ctx.poisson_solve(b, phi)
            fam = ctx.profile_read()
            ctx.close()
            res[name] = {"solve_ms": ms, "tridiag_ms": fam["thomas"][0] / reps}
            phis[name] = phi
        res["warp_over_per_thread_tridiag_time"] = (res["warp_partitioned"]["tridiag_ms"]
                                                    / res["per_thread"]["tridiag_ms"])
        res["rel_l2_between"] = float((phis["warp_partitioned"] - phis["per_thread"]).norm()
                                      / phis["per_thread"].norm())
        out["%dx%dx%d" % (nx, ny, nz)] = res
    return out


def small_nz_measurement(dev, shapes=((512, 512, 8), (256, 256, 16), (512, 512, 32)), reps=20):
    """The fused small-nz kernel (y transforms and wall-normal solves of one
    kx column in shared memory) against the separate passes, mixed Poisson
    solve at refine_tol 1e-10 on small-nz grids (stretched z; the FP32
    spectral arrays are L2-resident): time per solve, the time of the middle
    stages (the fused kernel against the forward y transform, the Thomas
    sweeps, the (0,0) mode and the inverse y transform), the error of each
    against the FP64 solve, and which form the context chooses by itself."""
    import torch
    import synth
    from paper_1705_01423_gb300 import Context
    stream = torch.cuda.current_stream()
    res = {}
    for shape in shapes:
        nx, ny, nz = shape
        w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
        b = torch.as_tensor(synth.noise((nz, ny, nx), seed=32)).to(dev)
        ctx = Context(nx, ny, nz, w.lx, w.ly, w.faces(), poisson_only=True)
        ref = ctx.poisson_solve(b)
        ctx.close()
        out = {}
        for name, fuse in (("fused", True), ("separate", False), ("default", None)):
            m = Context(nx, ny, nz, w.lx, w.ly, w.faces(), precision="mixed", refine_tol=MIXED_TOL,
                        refine_max_iter=6, poisson_only=True, fuse=fuse)
            phi = torch.empty_like(b)
            _, info = m.poisson_solve(b, phi, info=True)
            ms = timed(lambda: m.poisson_solve(b, phi), reps, stream)
            m.profile(True)
            m.profile_read()
            for _ in range(reps):
                m.poisson_solve(b, phi)
            fam = {k: v[0] / reps for k, v in m.profile_read().items() if v[1]}
            mid = sum(fam.get(k, 0.0) for k in ("yfft_thomas", "fft_y", "thomas", "zero_mode"))
            m.close()
            out[name] = {"solve_ms": ms, "middle_stages_ms": mid, "iters": info["iters"],
                         "rel_l2_vs_fp64": float((phi - ref).norm() / ref.norm()),
                         "fused": "yfft_thomas" in fam}
        out["solve_speedup"] = out["separate"]["solve_ms"] / out["fused"]["solve_ms"]
        out["middle_stages_speedup"] = (out["separate"]["middle_stages_ms"]
                                        / max(out["fused"]["middle_stages_ms"], 1e-9))
        out["default_is_fused"] = out["default"]["fused"]
        res["%dx%dx%d" % shape] = out
    return res


def side_measurements(ctx, w, dev, tma=True, state=None, fp64_peak=FP64_OPS_NOMINAL):
    """Poisson solve alone on the same grid: FP64 direct vs mixed FP32 + FP64
    refinement, with the mixed error against the FP64 GPU solve; the whole
    step with the mixed solve; the refined temperature grid."""
    import torch
    import synth
    from paper_1705_01423_gb300 import Context
    stream = torch.cuda.current_stream()
    pts = w.nx * w.ny * w.nz
    b = torch.as_tensor(synth.noise((w.nz, w.ny, w.nx), seed=123)).to(dev)
    phi64 = torch.empty_like(b)
    ms64 = timed(lambda: ctx.poisson_solve(b, phi64), 5, stream)
    out = {"poisson_fp64": {"ms": ms64, "grid_points_per_s": pts / (ms64 / 1e3)}}
    try:
        mctx = Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), precision="mixed", refine_tol=MIXED_TOL,
                       refine_max_iter=6, poisson_only=True, tma=tma)
        phim = torch.empty_like(b)
        _, info = mctx.poisson_solve(b, phim, info=True)
        msm = timed(lambda: mctx.poisson_solve(b, phim), 5, stream)
        err = float((phim - phi64).norm() / phi64.norm())
        out["poisson_mixed"] = {"ms": msm, "grid_points_per_s": pts / (msm / 1e3), "iters": info["iters"],
                                "refine_tol": MIXED_TOL, "rel_l2_vs_fp64_gpu": err,
                                "err_estimate": info["err_estimate"], "speedup_vs_fp64": ms64 / msm}
        mctx.profile(True)
        mctx.profile_read()
        mctx.poisson_solve(b, phim)
        out["poisson_mixed"]["families_ms"] = {k: v[0] for k, v in mctx.profile_read().items() if v[1]}
        mctx.close()
    except Exception as e:  # report, do not hide
        out["poisson_mixed"] = {"error": str(e)}
    ctx.profile(True)
    ctx.profile_read()
    ctx.poisson_solve(b, phi64)
    out["poisson_fp64"]["families_ms"] = {k: v[0] for k, v in ctx.profile_read().items() if v[1]}
    ctx.profile(False)
    out["cufft_comparison"] = cufft_comparison(b, out, stream)
    del b, phi64
    try:
        out["workloads"] = workload_measurements(dev)
    except Exception as e:  # report, do not hide
        out["workloads"] = {"error": str(e)}
    try:
        out["tridiag_regime"] = tridiag_regime_measurement(dev)
    except Exception as e:  # report, do not hide
        out["tridiag_regime"] = {"error": str(e)}
    try:
        out["small_nz_fused"] = small_nz_measurement(dev)
    except Exception as e:  # report, do not hide
        out["small_nz_fused"] = {"error": str(e)}
    if state is not None:
        try:
            out["rk3_step_mixed"] = mixed_step_measurement(ctx, w, dev, state, tma=tma)
        except Exception as e:  # report, do not hide
            out["rk3_step_mixed"] = {"error": str(e)}
    try:
        out["multires"] = multires_measurement(ctx, w, dev, fp64_peak=fp64_peak)
    except Exception as e:  # report, do not hide
        out["multires"] = {"error": str(e)}
    return out


def multires_measurement(ctx, w, dev, r=(2, 2, 2), n_sub=1, reps=3, fp64_peak=FP64_OPS_NOMINAL):
    """Coupled step with the temperature on a grid refined r times (afid_mr_step):
    the momentum step on the workload's grid with the restricted buoyancy, then
    n_sub refined RK3/CN temperature steps on the fine grid."""
    import torch
    import synth
    from paper_1705_01423_gb300 import MultiRes
    stream = torch.cuda.current_stream()
    m = MultiRes(ctx, *r)
    zf = m.faces()
    Tf = torch.as_tensor(synth.conduction_temperature(zf, m.ny, m.nx, w.T_bot, w.T_top, 11, amp=1e-3)).to(dev)
    vel = [torch.as_tensor(a).to(dev) for a in synth.velocity_noise(w, 12, sigma=0.05)]
    p = torch.zeros(ctx.cell, dtype=torch.float64, device=dev)
    H = [torch.zeros(ctx.cell, dtype=torch.float64, device=dev), torch.zeros(ctx.cell, dtype=torch.float64, device=dev),
         torch.zeros(ctx.face, dtype=torch.float64, device=dev)]
    dt = 1e-3
    ctx.project(*vel, p)  # a solenoidal start

    def step():
        m.step(dt, n_sub, *vel, p, *H, Tf)

    ms = timed(step, reps, stream)
    ctx.profile(True)
    ctx.profile_read()
    step()
    fams = {k: v[0] for k, v in ctx.profile_read().items() if v[1]}
    ctx.profile(False)
    l0 = ctx.kernel_launches()
    step()
    torch.cuda.synchronize()
    launches = ctx.kernel_launches() - l0
    fine = m.nx * m.ny * m.nz
    nsubst = 3 * n_sub  # refined substeps per coupled step
    # FP64 operation model per fine point and substep: the temperature terms
    # with shared face fluxes (30: own x and y face fluxes 8, the block-edge
    # fluxes 2 + 1 (64-wide rows, 4 rows), z flux 3, divergence 6, horizontal
    # diffusion with kappa folded into its weights, forming H, 5, CN explicit
    # side 3, R 2) and the prolongation (per
    # component a z interpolation, 2, plus per coarse plane a y interpolation,
    # 2, and the column's share of the block's x interpolations of 8/ry + 1
    # coarse rows, 2 (8/ry + 1) / 8, shared by rz fine levels)
    ops_rhs = 30.0 * fine * nsubst
    ops_pro = 3 * (2.0 + (2.0 + 2.0 * (8.0 / r[1] + 1.0) / 8.0) / r[2]) * fine * nsubst
    peak = fp64_peak * 1e12
    out = {"refinement": list(r), "n_sub": n_sub, "fine_grid": [m.nx, m.ny, m.nz],
           "ms_per_coupled_step": ms, "fine_grid_points_per_s": fine / (ms / 1e3),
           "kernel_launches_per_step": launches, "families_ms": fams,
           "fp64_ops_frac": {"mr_scalar_rhs": ops_rhs / (fams.get("mr_scalar_rhs", 1e9) / 1e3) / peak,
                             "mr_prolong": ops_pro / (fams.get("mr_prolong", 1e9) / 1e3) / peak},
           "refined_workspace_gb": m.workspace_bytes / 1e9,
           "note": "momentum %dx%dx%d (FP64 RK3/CN step, buoyancy from the restricted T), temperature "
                   "%dx%dx%d (%d refined RK3/CN step(s) per momentum step)" % (w.nx, w.ny, w.nz, m.nx, m.ny, m.nz, n_sub)}
    m.close()
    del Tf, vel, p, H
    # the single-grid step at the fine resolution, for the saving of the refined grid
    try:
        from paper_1705_01423_gb300 import Context, Physics
        ph = Physics(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                     T_bot=w.T_bot, T_top=w.T_top)
        fctx = Context(out["fine_grid"][0], out["fine_grid"][1], out["fine_grid"][2], w.lx, w.ly, zf, phys=ph)
        shp_c, shp_f = fctx.cell, fctx.face
        S = [torch.zeros(shp_c, dtype=torch.float64, device=dev), torch.zeros(shp_c, dtype=torch.float64, device=dev),
             torch.zeros(shp_f, dtype=torch.float64, device=dev),
             torch.as_tensor(synth.conduction_temperature(zf, shp_c[1], shp_c[2], w.T_bot, w.T_top, 13, amp=1e-3)).to(dev),
             torch.zeros(shp_c, dtype=torch.float64, device=dev)]
        HS = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]), torch.zeros_like(S[3])]
        ms_f = timed(lambda: fctx.rk3_step(S, HS, dt), 2, stream)
        out["single_grid_step_at_fine_resolution_ms"] = ms_f
        out["saving_vs_single_grid"] = ms_f / ms
        fctx.close()
        del S, HS
    except Exception as e:  # report, do not hide
        out["single_grid_step_at_fine_resolution_ms"] = {"error": str(e)}
    torch.cuda.empty_cache()
    return out


def cufft_comparison(b, out, stream):
    """Timing comparison only (never on the product path): the library's batched
    2-D real FFT pair (forward rfft2 + inverse irfft2 over the z planes, through
    torch.fft) next to this build's transform kernels inside one solve (the x
    transforms with their fused divergence/scaling plus the two y passes)."""
    import torch
    res = {}
    fams64 = out["poisson_fp64"].get("families_ms", {})
    ours64 = sum(fams64.get(k, 0.0) for k in ("r2c_x", "fft_y", "c2r_x"))
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        x = b.to(dt)
        ms = timed(lambda: torch.fft.irfft2(torch.fft.rfft2(x), s=x.shape[-2:]), 5, stream)
        res[name] = {"library_rfft2_irfft2_ms": ms}
        del x
    res["fp64"]["this_build_fft_passes_ms"] = ours64
    res["fp64"]["ratio_library_over_this_build"] = res["fp64"]["library_rfft2_irfft2_ms"] / max(ours64, 1e-9)
    fm = out.get("poisson_mixed", {}).get("families_ms")
    if fm:
        it = max(out["poisson_mixed"].get("iters", 1), 1)
        ours32 = sum(fm.get(k, 0.0) for k in ("r2c_x", "fft_y", "c2r_x")) / it
        res["fp32"]["this_build_fft_passes_ms_per_iteration"] = ours32
        res["fp32"]["ratio_library_over_this_build"] = res["fp32"]["library_rfft2_irfft2_ms"] / max(ours32, 1e-9)
    return res


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle (plain FP64 PyTorch CPU) as the reference arm: each step is one
    oracle RK3 step of the same workload on a bounded 64x64 x nz sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload_from(args)
    nx = ny = 64
    times, thr = oracle_step_time(nx, ny, w.nz, steps=args.steps, warmup=args.warmup)
    tot = sum(times)
    pts = nx * ny * w.nz
    value = pts * len(times) / tot
    out = {"impl": "reference",
           "metric": "grid-points/s per FP64 RK3/CN time step (Rayleigh-Benard Ra=1e8, 512x512x384)",
           "value": value, "unit": "grid-points/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "rb512 (oracle on a bounded %dx%dx%d sample per step)" % (nx, ny, w.nz)},
           "cpu_baseline": {"value": value, "unit": "grid-points/s", "cores": thr, "kind": "oracle",
                            "sample": "each step: one FP64 oracle RK3 step on %dx%dx%d cells of the Rayleigh-Benard workload" % (nx, ny, w.nz)},
           "e2e": {"value": value, "unit": "grid-points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.poisson_only:
        run_poisson_only(args)
    elif args.multires_only:
        run_multires_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
