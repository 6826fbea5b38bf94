"""Implicit-stage throughput of the hybridized FR stage on GB300.

One step = one hybridized implicit stage of the workload (default vortex256: 2D Navier-Stokes
isentropic vortex with 1e-3 seeded noise, 256x256 quads, p = 4, 6,553,600 implicit DOF, blocks
100x100 / 80x80; or vortex64: 64x64 quads, p = 3, 262,144 DOF), SDIRK2 stage 1 at 10x the
explicit CFL limit, solved from the standard initial guess to a relative Newton residual of 1e-8,
through the C ABI (imex_stage stages 0 and 1).  The headline ``value`` is the mixed-precision path (FP32 element
blocks, inverse, condensation, trace operator and Krylov basis; FP64 residuals, Newton updates,
Hessenberg / Givens and the trace solution); the plain FP64 path is timed in the same run and
reported beside it.  Both paths stop on the same FP64 Newton residual test.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: replicas only (one independent stage per rank, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HFR implicit-stage DOF/s at 1e-8 resid: mixed-prec batched vs FP64, one GB300"
WORKLOADS = {
    "vortex256": ("vortex256: 2D compressible Navier-Stokes isentropic vortex, M=0.5, gamma=1.4, Re=1e4, periodic "
                  "[0,10]^2, 256x256 quads, p=4 (blocks A 100x100, S 80x80), + U(-1e-3,1e-3) noise (seed 1234), "
                  "SDIRK2 stage 1 at 10x explicit CFL, Newton to 1e-8"),
    "vortex64": ("vortex64: 2D compressible Navier-Stokes isentropic vortex, M=0.5, gamma=1.4, Re=1e4, periodic "
                 "[0,10]^2, 64x64 quads, p=3 (blocks 64x64), SDIRK2 stage 1 at 10x explicit CFL, Newton to 1e-8"),
}
PATCH = {"vortex256": 14, "vortex64": 16, "vortex64p4": 10, "vortex128p4": 12}
# profiling aid: the p = 4 kernels of vortex256 on a 64x64 mesh (a few GB on the device)
WORKLOADS["vortex64p4"] = "vortex64p4: vortex256's physics, p = 4 and noise on 64x64 quads (profiling size)"
# profiling aid: 128x128, so that the trace operator's S blocks (420 MB) exceed the 129 MB L2
WORKLOADS["vortex128p4"] = "vortex128p4: vortex256's physics, p = 4 and noise on 128x128 quads (profiling size)"  # oracle sample: PATCH x PATCH elements at the workload's spacing
NEWTON_TOL = 1e-8
GMRES_RTOL = 1e-4
FP32_PEAK_PER_SM_CLK = 256.0  # 128 FP32 FMA lanes x 2 flops
FP64_PEAK_PER_SM_CLK = 4.0    # 2 FP64 FMA per clock per SM (1.25 TFLOP/s at 2.07 GHz, 152 SMs)
TF32_PER_BF16 = 0.5           # dense TF32 tensor rate / dense BF16 rate
NUM_SMS = 152


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hfr_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_max(values, dist=None, device="cpu"):
    """Max over ranks of per-rank timings (replicas: each rank runs the whole workload)."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_value(world, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def flush_l2(buf):
    buf.add_(1.0)  # writes a buffer larger than L2 (129 MB)


def run_stage(ctx, dt, u_n, u_stage, uhat, uhat0, R_hist):
    uhat.copy_(uhat0)
    ctx.imex_stage(0, dt, u_n, u_stage, uhat, R_hist, newton_tol=NEWTON_TOL, gmres_rtol=GMRES_RTOL)
    return ctx.imex_stage(1, dt, u_n, u_stage, uhat, R_hist, newton_tol=NEWTON_TOL, newton_maxit=30,
                          gmres_rtol=GMRES_RTOL, gmres_maxit=3000, refine=ctx.refine)


JAC_POLICY = {"every": 0, "once": 1}


def time_path(pkg, torch, w, precision, refine, steps, warmup, dev, l2buf, jac="every", barrier=None, graph=False,
              autotune=True, cond_mode=None):
    ctx = pkg.Context(w.mesh, w.physics, precision=precision, tableau=pkg.FR_TAB_SDIRK2)
    ctx.refine = refine
    ctx.imex_set_jacobian_policy(JAC_POLICY[jac])
    if graph:
        ctx.imex_stage_set_graph(True)
    stream = torch.cuda.current_stream()
    u_n = torch.tensor(w.u0, device=dev)
    uhat0 = ctx.hfr_initial_trace(u_n)
    uhat = uhat0.clone()
    tune = None
    if autotune and precision == pkg.FR_PREC_FP32:  # pick the condensation form and GMRES cycle on this workload
        tune = ctx.hfr_autotune(u_n, uhat0, u_n, w.dt * (1.0 - 0.5 ** 0.5))
    if cond_mode is not None:
        ctx.hfr_condense_set_mode(cond_mode)
    R_hist = ctx.empty(3, *ctx.state_shape)
    u_stage = ctx.empty(*ctx.state_shape)
    stats = None
    for _ in range(warmup):
        stats = run_stage(ctx, w.dt, u_n, u_stage, uhat, uhat0, R_hist)
    torch.cuda.synchronize()
    if barrier is not None:
        barrier()
    ctx.fr_profile_enable(True)
    l0 = ctx.kernel_launches()
    times = []
    for _ in range(steps):
        flush_l2(l2buf)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = run_stage(ctx, w.dt, u_n, u_stage, uhat, uhat0, R_hist)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if barrier is not None:
        barrier()
    launches = ctx.kernel_launches() - l0
    prof = ctx.fr_profile_read()
    ctx.fr_profile_enable(False)
    result = {"ms": times, "stats": stats, "profile": prof, "launches": launches, "ctx": ctx,
              "u": u_stage.clone(), "uhat0": uhat0, "tune": tune}
    return result


def time_e2e(pkg, torch, ctx, w, steps, dev):
    """Same stage through the C ABI with HOST buffers: pinned H2D of u_n and the initial trace,
    the stage, D2H of u_stage and the trace, all inside the timed region."""
    u_host = torch.tensor(w.u0).pin_memory()
    uhat_host = ctx.hfr_initial_trace(torch.tensor(w.u0, device=dev)).cpu().pin_memory()
    u_out = torch.empty_like(u_host).pin_memory()
    uh_out = torch.empty_like(uhat_host).pin_memory()
    u_n = torch.empty(u_host.shape, dtype=torch.float64, device=dev)
    uhat = torch.empty(uhat_host.shape, dtype=torch.float64, device=dev)
    R_hist = ctx.empty(3, *ctx.state_shape)
    u_stage = ctx.empty(*ctx.state_shape)
    stream = torch.cuda.current_stream()
    times = []
    # one untimed stage on these buffers (a graph context captures its stage graph here)
    u_n.copy_(u_host)
    uhat.copy_(uhat_host)
    ctx.imex_stage(0, w.dt, u_n, u_stage, uhat, R_hist, newton_tol=NEWTON_TOL, gmres_rtol=GMRES_RTOL)
    ctx.imex_stage(1, w.dt, u_n, u_stage, uhat, R_hist, newton_tol=NEWTON_TOL, newton_maxit=30,
                   gmres_rtol=GMRES_RTOL, gmres_maxit=3000, refine=ctx.refine)
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u_n.copy_(u_host, non_blocking=True)
        uhat.copy_(uhat_host, non_blocking=True)
        ctx.imex_stage(0, w.dt, u_n, u_stage, uhat, R_hist, newton_tol=NEWTON_TOL, gmres_rtol=GMRES_RTOL)
        ctx.imex_stage(1, w.dt, u_n, u_stage, uhat, R_hist, newton_tol=NEWTON_TOL, newton_maxit=30,
                       gmres_rtol=GMRES_RTOL, gmres_maxit=3000, refine=ctx.refine)
        u_out.copy_(u_stage, non_blocking=True)
        uh_out.copy_(uhat, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3))
    bi = u_host.numel() * 8 + uhat_host.numel() * 8
    bo = u_out.numel() * 8 + uh_out.numel() * 8
    return float(np.mean(times)), bi, bo


def jacobian_reuse(pkg, torch, ctx, w, dev, nsteps=3):
    """Whole IMEX steps (imex_steps) with the condensation held across stages and steps
    (FR_JAC_KEEP, the paper's practice of refreshing the Jacobian every 100 steps): one untimed step
    makes the linearisation, the timed steps are chord-Newton steps that reuse it."""
    kw = dict(newton_tol=NEWTON_TOL, newton_maxit=60, gmres_rtol=GMRES_RTOL, gmres_maxit=3000)
    ctx.imex_set_jacobian_policy(pkg.FR_JAC_KEEP)
    try:
        u = torch.tensor(w.u0, device=dev)
        uh = ctx.hfr_initial_trace(u)
        ctx.imex_steps(1, w.dt, u, uh, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = ctx.imex_steps(nsteps, w.dt, u, uh, **kw)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        ctx.imex_set_jacobian_policy(pkg.FR_JAC_EVERY_NEWTON)
    stages = nsteps * ctx.info.nstages
    return {"steps": nsteps, "ms_per_step": ms / nsteps, "ms_per_implicit_stage": ms / stages,
            "value": w.dofs_implicit * stages / (ms * 1e-3), "unit": "implicit-stage DOF/s",
            "newton_iterations_per_stage": st["newton_iterations"] / stages,
            "gmres_iterations_per_stage": st["gmres_iterations"] / stages,
            "jacobian_refreshes": st["jacobian_refreshes"], "converged": st["converged"],
            "note": "SDIRK2 steps at the bench dt from the vortex, explicit stage and final combination "
                    "included; the linearisation made in the untimed first step is reused by every timed "
                    "stage (Newton to the same 1e-8 FP64 test)"}


def uneven_condense(pkg, torch, dev, n_elem=40000, steps=3):
    """Condensation of a seeded batch of Navier-Stokes element blocks of uneven degree (p drawn
    uniformly from 2..5: blocks 36/48, 64/64, 100/80, 144/96) in one persistent launch
    (hfr_condense_uneven, FP32), against the same kernel launched once per degree class.  Synthetic
    blocks A = 4 I + N(0,1)/sqrt(nA), B, C, D, r, s ~ N(0, 1), generated on the device."""
    g = torch.Generator(device=dev)
    g.manual_seed(2024)
    ps = torch.randint(2, 6, (n_elem,), generator=g, device=dev).cpu().tolist()
    shapes = [(4 * (p + 1) ** 2, 16 * (p + 1)) for p in ps]

    def make(shp):
        nA = [a for a, _ in shp]
        nT = [t for _, t in shp]
        A = torch.cat([(4.0 * torch.eye(a, device=dev) + torch.randn(a, a, generator=g, device=dev) / a ** 0.5).reshape(-1)
                       for a in nA]).float()
        sb = sum(a * t for a, t in shp)
        sd = sum(t * t for t in nT)
        B = torch.randn(sb, generator=g, device=dev)
        C = torch.randn(sb, generator=g, device=dev)
        D = torch.randn(sd, generator=g, device=dev)
        r = torch.randn(sum(nA), generator=g, device=dev, dtype=torch.float64)
        s = torch.randn(sum(nT), generator=g, device=dev, dtype=torch.float64)
        return nA, nT, (A, B, C, D, r, s)

    def timed(args_list):
        for a in args_list:  # warm-up
            pkg.hfr_condense_uneven(a[0], a[1], *a[2], precision=pkg.FR_PREC_FP32)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(steps):
            t0 = time.perf_counter()
            for a in args_list:
                pkg.hfr_condense_uneven(a[0], a[1], *a[2], precision=pkg.FR_PREC_FP32)
            torch.cuda.synchronize()
            best = min(best, (time.perf_counter() - t0) * 1e3)
        return best

    whole = make(shapes)
    ms_one = timed([whole])
    per_class = [make([sh for sh in shapes if sh == c]) for c in sorted(set(shapes))]
    ms_cls = timed(per_class)
    flop = sum(2.0 * a ** 3 + 2.0 * a * a * (t + 1) + 2.0 * t * a * (t + 1) for a, t in shapes)
    return {"elements": n_elem, "degrees": "p uniform in 2..5 (seed 2024)", "ms_one_launch": ms_one,
            "ms_per_class_launches": ms_cls, "gflops_one_launch": flop / (ms_one * 1e-3) / 1e9,
            "note": "wall time of the call (host shape table, stream-ordered work buffer, one kernel, "
                    "synchronise); FP32 shared-memory Gauss-Jordan + products"}


def measure_pipe_peaks(pkg):
    """FP64 / FP32 FMA and TF32 tensor-core rates of this GPU, measured now by the library's loop
    kernels (fr_measure_peak, CUDA events): the denominators of the ALU- and tensor-bound
    fractions.  Reported, never fatal."""
    out = {}
    for key, which in (("fp64_tflops_measured", 0), ("fp32_tflops_measured", 1), ("tf32_tflops_measured", 2)):
        try:
            out[key] = float(pkg.fr_measure_peak(which))
        except Exception as exc:
            out[key] = f"error: {exc}"
    out["how"] = ("fr_measure_peak: FP64/FP32 8 independent FMA chains per thread, 8 CTAs x 256 threads per SM; "
                  "TF32 tcgen05.mma kind::tf32 M=128 N=256 K=8 back to back, 2 CTAs per SM; CUDA events, after a "
                  "warm-up launch")
    return out


def tight_agreement(pkg, torch, w, ctx_mixed, ctx_fp64, dev, tol=1e-11, refines=(0, 1)):
    """The precision error of the mixed path, separated from the Newton tolerance: both paths
    converge the same stage to a relative FP64 Newton residual of ``tol``; the mixed one with 0 and
    1 FP64 refinement sweeps of its local solves.  Differences relative to the stage increment
    (max norm over all DOF)."""
    kw = dict(newton_tol=tol, newton_maxit=40, gmres_rtol=1e-6, gmres_maxit=5000)

    def solve(ctx, refine):
        u_n = torch.tensor(w.u0, device=dev)
        uh = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist, **kw)
        st = ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, refine=refine, **kw)
        return us, st

    graph = ctx_mixed.imex_stage_get_graph()
    ref, st64 = solve(ctx_fp64, 0)
    inc = (ref - torch.tensor(w.u0, device=dev)).abs().max().item()
    out = {"newton_tol": tol, "gmres_rtol": kw["gmres_rtol"], "fp64_newton_iterations": st64["newton_iterations"]}
    for refine in refines:
        us, st = solve(ctx_mixed, refine)
        out[f"refine{refine}"] = {"max_rel_diff": (us - ref).abs().max().item() / inc,
                                  "newton_iterations": st["newton_iterations"],
                                  "gmres_iterations": st["gmres_iterations"], "converged": st["converged"]}
    assert graph == ctx_mixed.imex_stage_get_graph()
    return out


GENERAL_WORKLOADS = {
    "boundary_layer": ("boundary_layer: 2D Navier-Stokes Re=1.7e6 M=0.2, 400x500 quads, wall-normal growth 1.15 from "
                       "1e-5 to isotropic 1e-2 (aspect ratio to 1e3), p uniform random in 2..5 per element (seed 2024), "
                       "wall below, far field above, 20% stiffest elements implicit (40 000), SDIRK2 stage 1 with the "
                       "ERK partner, Newton to 1e-8"),
    "channel3d": ("channel3d: 3D Navier-Stokes Re=1.6e3 M=0.1 Taylor-Green-like field, 64x32x48 hexahedra, tanh "
                  "clustering beta=2.5, walls at y=+-1, periodic x and z, p=3 (blocks 320 / 480), three implicit wall "
                  "layers per wall (18 432 elements), SDIRK2 stage 1 with the ERK partner, Newton to 1e-8"),
    "efr_vortex256": ("efr_vortex256: the vortex256 workload (256x256 periodic quads, p=4, all implicit, seeded 1e-3 "
                      "noise, SDIRK2 stage 1 at 10x explicit CFL, Newton to 1e-8) with the EFR trace: continuous at the "
                      "Gauss-Lobatto points of the trace faces (Sec. 2.2), 458 752 trace nodes x 4 variables"),
}


def general_leg(pkg, torch, dev, l2buf, name, steps=(3, 2), warmup=(2, 1), peaks=None, paths=("mixed", "fp64")):
    """A workload of the general-mesh path (boundary_layer: mixed degree, wall, far field; channel3d:
    hexahedra with walls), mixed precision against FP64, each stage timed with CUDA events (steps /
    warm-ups per path as given).  Rooflines of its two largest phases from their algorithmic work:
    the condensation (2/3 nA^3 + 2 nA^2 (nT + 1) + 2 nT nA (nT + 1) flop per element, FP32 FMA
    roof) and the trace GMRES (per iteration the S_k blocks, the gathered and scattered trace values
    and the orthogonalisation, HBM roof)."""
    from workloads import make_config

    efr = name.startswith("efr_")
    w = make_config(name[len("efr_"):] if efr else name)
    tkind = pkg.FR_TRACE_EFR if efr else pkg.FR_TRACE_HFR
    peaks = peaks or {}
    out = {"workload": GENERAL_WORKLOADS[name], "implicit_dofs": w.dofs_implicit, "elements": w.mesh.nelem}
    res = {}
    for pi, (label, prec) in enumerate((("mixed", pkg.FR_PREC_FP32), ("fp64", pkg.FR_PREC_FP64))):
        if label not in paths:
            continue
        ctx = pkg.Context(w.mesh, w.physics, precision=prec, tableau=pkg.FR_TAB_SDIRK2, trace_kind=tkind)
        u0 = w.u0 if isinstance(w.u0, list) else list(w.u0)
        u_n = torch.tensor(ctx.pack_state(u0), device=dev)
        uh0 = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        stream = torch.cuda.current_stream()

        def run():
            uh = uh0.clone()
            ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist, newton_tol=NEWTON_TOL)
            return ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, newton_tol=NEWTON_TOL, newton_maxit=30,
                                  gmres_rtol=GMRES_RTOL, gmres_maxit=20000)

        for _ in range(warmup[pi]):
            st = run()
        torch.cuda.synchronize()
        ctx.fr_profile_enable(True)
        l0 = ctx.kernel_launches()
        times = []
        for _ in range(steps[pi]):
            flush_l2(l2buf)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = run()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = ctx.fr_profile_read()
        ctx.fr_profile_enable(False)
        res[label] = {"ms": float(np.mean(times)), "stats": st, "prof": prof, "steps": steps[pi],
                      "launches": (ctx.kernel_launches() - l0) // steps[pi], "u": (us - u_n).clone(),
                      "nA": ctx.blk_nA.astype(np.float64), "nT": ctx.blk_nT.astype(np.float64),
                      "nh": int(ctx.info.trace_values)}
        if label == "mixed" and steps[pi] > 0:
            # the same stage as one CUDA graph (the per-phase times above come from the stream form)
            ctx.imex_stage_set_graph(True)
            for _ in range(max(warmup[pi], 1)):
                run()
            torch.cuda.synchronize()
            l1 = ctx.kernel_launches()
            gt = []
            for _ in range(steps[pi]):
                flush_l2(l2buf)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                gst = run()
                e1.record(stream)
                torch.cuda.synchronize()
                gt.append(e0.elapsed_time(e1))
            res[label].update({"graph_ms": float(np.mean(gt)), "graph_launches": (ctx.kernel_launches() - l1) // steps[pi],
                               "graph_stats": gst, "u_graph": (us - u_n).clone()})
            ctx.imex_stage_set_graph(False)
        ctx.close()
        del R_hist, us, uh0, u_n
        torch.cuda.empty_cache()
    if "fp64" not in res:  # profiling aid: the mixed path alone
        m = res["mixed"]
        return {"workload": out["workload"], "ms": m["ms"], "graph_ms": m.get("graph_ms"), "stats": m["stats"],
                "launches": m["launches"], "phases_ms_total": {k: round(v[0], 3) for k, v in m["prof"].items()}}
    m, f = res["mixed"], res["fp64"]
    inc = f["u"].abs().max().item()
    nA, nT = m["nA"], m["nT"]
    flop = float(np.sum(2.0 / 3.0 * nA ** 3 + 2 * nA ** 2 * (nT + 1) + 2 * nT * nA * (nT + 1)))
    ms, cnt = m["prof"]["condense_factor"]
    cond_a = flop / (ms / max(cnt, 1) * 1e-3) / 1e12
    fp32 = peaks.get("fp32_tflops_measured") or NUM_SMS * FP32_PEAK_PER_SM_CLK * 2070e6 / 1e12
    gms, gcnt = m["prof"]["gmres"]
    # GMRES solves of one stage: one per Newton iteration (the profile counts every timed stage)
    its = m["stats"]["gmres_iterations"] / max(m["stats"]["newton_iterations"], 1)
    k_its = int(round(its))
    alg = k_its * float(np.sum(nT * nT) * 4 + np.sum(nT) * 2 * 8) + sum((k + 2) * m["nh"] * 8 for k in range(1, k_its + 1))
    g_a = alg / (gms / max(gcnt, 1) * 1e-3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    cond_kernel = ("k_big_lu_panel + k_big_gemm (blocked LU), k_big_solve (column-block solve), k_big_gemm_tc "
                   "(S on tcgen05), k_big_xr" if name == "channel3d" else
                   "k_inverse_tc + k_products_tc (tensor-core shape classes), k_condense_uneven<float> (shared-memory "
                   "Gauss-Jordan bundles, nA <= 64), the blocked-LU kernels (larger blocks)")
    out.update({
        "value": w.dofs_implicit / (m["graph_ms"] * 1e-3), "unit": "implicit-stage DOF/s", "ms_per_step": m["graph_ms"],
        "stage_execution": "one CUDA graph per stage (mixed); the FP64 path and the per-phase times: stream form",
        "stream_stage": {"ms_per_step": m["ms"], "value": w.dofs_implicit / (m["ms"] * 1e-3),
                         "gpu_launches": int(m["launches"]),
                         "graph_equals_stream": bool(torch.equal(m["u"], m["u_graph"]))},
        "steps": m["steps"], "newton_iterations": m["graph_stats"]["newton_iterations"],
        "gmres_iterations": m["graph_stats"]["gmres_iterations"], "gpu_launches": int(m["graph_launches"]),
        "fp64": {"value": w.dofs_implicit / (f["ms"] * 1e-3), "ms_per_step": f["ms"], "steps": f["steps"],
                 "newton_iterations": f["stats"]["newton_iterations"], "gmres_iterations": f["stats"]["gmres_iterations"],
                 "phases_ms_total": {k: round(v[0], 3) for k, v in f["prof"].items()}},
        "mixed_over_fp64": f["ms"] / m["graph_ms"],
        "mixed_vs_fp64_max_rel_diff": (m["u"] - f["u"]).abs().max().item() / inc,
        "phases_ms_total": {k: round(v[0], 3) for k, v in m["prof"].items()},
        "rooflines": {
            "condense": {"kernel": cond_kernel, "bound": "alu", "achieved": cond_a, "peak": fp32,
                         "unit": "TFLOP/s", "frac": cond_a / fp32, "avg_launch_ms": ms / max(cnt, 1),
                         "algorithmic_flop": flop},
            "gmres": {"kernel": "multi-kernel GMRES cycle (k_gen_matvec_elem, k_gen_gather_sum, k_gen_precond_apply, k_cgs)",
                      "bound": "hbm", "achieved": g_a, "peak": hbm, "unit": "GB/s", "frac": g_a / hbm,
                      "avg_solve_ms": gms / max(gcnt, 1), "iterations_per_solve": k_its, "algorithmic_bytes": alg},
        },
        "l2": "flushed between timed steps (256 MB write)",
    })
    if efr:
        out["trace_values"] = m["nh"]
        out["hfr_trace_values"] = int(2 * w.mesh.nelem * (w.p + 1) * 4)
    return out


def cpu_baseline(workload="vortex256", npatch=None):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: the stage-1
    Newton solve of the same vortex on a PATCH x PATCH periodic patch (or npatch x npatch) at the
    workload's element size, p and time step, direct trace solve."""
    from oracle.fr import Discretisation
    from oracle.physics import make_physics
    from oracle.stepping import TABLEAUX, newton_stage
    from workloads import make_config
    from workloads.states import isentropic_vortex, sample_points

    full = make_config(workload)
    npatch = npatch or PATCH[workload]
    nfull = int(round(np.sqrt(full.mesh.nelem)))
    w = make_config("vortex", n=npatch, p=full.p)
    scale = (10.0 / nfull) / (10.0 / npatch)
    mesh = w.mesh
    mesh.verts = mesh.verts * scale
    u0 = isentropic_vortex(sample_points(mesh, full.p), center=(5.0 * scale, 5.0 * scale))
    d = Discretisation(mesh, make_physics(full.physics))
    a = TABLEAUX["sdirk2"]["a"][0, 0]
    t0 = time.perf_counter()
    _, _, info = newton_stage(d, u0, u0, d.initial_trace(u0), a * full.dt, tol=NEWTON_TOL)
    el = time.perf_counter() - t0
    dofs = mesh.nelem * (full.p + 1) ** 2 * 4
    cores = _threads()
    return {"value": dofs / el, "unit": "DOF/s", "cores": cores, "kind": "oracle", "dofs": dofs,
            "sample": f"stage-1 Newton solve (to 1e-8, {info['iterations']} iterations, direct trace solve) of the "
                      f"vortex on a {npatch}x{npatch} periodic patch at the {workload} spacing, p={full.p}, same dt: "
                      f"{mesh.nelem} elements, {dofs} DOF, {el:.1f} s"}


def cpu_baseline_single_core(workload="vortex256", npatch=8):
    """The same oracle sample on one host core: a child process with every BLAS / OpenMP pool
    limited to one thread before numpy loads (a smaller patch keeps it to seconds)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    code = ("import json, bench; r = bench.cpu_baseline(%r, npatch=%d); r['cores'] = 1; print(json.dumps(r))"
            % (workload, npatch))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        return {"error": out.stderr.strip().splitlines()[-1] if out.stderr.strip() else "failed"}
    return json.loads(out.stdout.strip().splitlines()[-1])


def _threads():
    try:
        from threadpoolctl import threadpool_info

        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


# DRAM bytes per launch (read + write) of the current kernels, from one ncu capture each
# (summaries under profiles/), per workload; None where not captured or the kernel changed since
# vortex256: captured on the same kernels over 64x64 elements (p = 4) and scaled by the element
# count (x16) where the traffic is per element (factorisation, products, Jacobian)
NCU_TRAFFIC_BYTES = {"vortex256": {"k_inverse_tc": 16 * (165.51e6 + 109.29e6),
                                   "k_products_tc": 16 * (539.59e6 + 209.25e6),
                                   "k_inverse_rq": 16 * (169.68e6 + 109.01e6),
                                   "k_products_x": 16 * (299.90e6 + 101.01e6),
                                   "k_products_s": 16 * (372.94e6 + 85.81e6),
                                   "k_jacobian": 16 * (82.50e6 + 528.51e6)},
                     "vortex64": {}}


# DRAM bytes (read + write) of k_gmres_cycle<float, 80, 20> per element and GMRES iteration, from
# one ncu capture of the three cycle launches of a vortex128p4 stage (16 384 elements, 60 GMRES
# iterations, 31.28 GB in all; profiles/vortex128p4_gmres_cycle_traffic.md), keyed by nT; a full
# launch is that times its elements and iterations (the cycle's traffic grows with both)
GMRES_TRAFFIC_PER_ELEM_ITER = {80: (30827120896 + 452353536) / (16384 * 60)}


def kernel_rooflines(prof, stats, w, peaks, clocks, workload, cond_mode=2):
    """Roofline of every single-kernel phase of the timed step, from the live CUDA-event phase
    timings (average launch duration), and the dominant one (largest total time).
    Algorithmic work per launch (E elements, nA = 4 n^2, nT = 16 n, face blocks bs = 4 n, ntrace = 2E faces,
    n_t = 16 ntrace trace unknowns, k = GMRES iterations per solve):
      k_gmres_cycle       HBM: k (S_k blocks E nT^2 4 B + face inverses ntrace bs^2 4 B
                          + Krylov passes 4 (k/2 + 1) n_t 4 B + z, w 2 n_t 4 B)
      k_inverse_tc        Gauss-Jordan inverse 2 nA^3 flop per element, against the FP32 FMA roof (the
                          panel eliminations on the FP32 pipes set its time; the rank-16 trailing
                          updates run on the tensor cores)
      k_products_tc       HBM 4 (nA^2 + 2 nA nT + nT^2) B in + 4 (nA nT + nT^2) B out per element, or the
                          TF32 tensor roof for 2 (nA^2 (nT+1) + nT nA (nT+1)) flop per element,
                          whichever fraction is higher
      k_jacobian          ALU: (nA+nT)^2 (2n+4) 2 flop per element (n = p + 1)
    """
    E = w.mesh.nelem
    n = w.p + 1
    nA, nT, bs = 4 * n * n, 16 * n, 4 * n
    ntrace = 2 * E
    nt_u = ntrace * bs
    mhz = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu_peak = peaks.get("fp32_tflops_measured") or NUM_SMS * FP32_PEAK_PER_SM_CLK * mhz * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    tf32_peak = peaks.get("tf32_tflops_measured") or float(peaks.get("bf16_tflops", 1900.0)) * TF32_PER_BF16
    its = stats["gmres_iterations"] / max(stats["newton_iterations"], 1)
    out = {}

    def avg(ph):
        ms, cnt = prof[ph]
        return ms, ms / max(cnt, 1)

    def entry(kern, bound, achieved, peak, unit, total_ms, avg_ms):
        tw = NCU_TRAFFIC_BYTES.get(workload, {})
        t = sum(tw[kk] for kk in kern.split("+")) if all(tw.get(kk) for kk in kern.split("+")) else None
        src = {"GB/s": "MEASURED_PEAKS.json hbm_gbs",
               "TFLOP/s": ("fr_measure_peak FP32 FMA loop, this run" if peaks.get("fp32_tflops_measured")
                           else f"FP32 lanes x {mhz:.0f} MHz x {NUM_SMS} SMs"),
               "TF32 TFLOP/s": ("fr_measure_peak TF32 tcgen05 loop, this run" if peaks.get("tf32_tflops_measured")
                                else f"MEASURED_PEAKS.json bf16_tflops x {TF32_PER_BF16} (nominal TF32 / BF16 ratio)")}[unit]
        return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit.replace("TF32 ", ""),
                "frac": achieved / peak, "traffic": t, "kernel": kern, "avg_launch_ms": avg_ms, "total_ms": total_ms,
                "peak_source": src}

    tot, a = avg("gmres")
    # algorithmic bytes of one restart cycle of its iterations: per iteration the S_k blocks
    # (E nT^2 4 B) and the gathered / scattered trace vectors (E 2 nT 8 B), and at iteration
    # k = 1..its the orthogonalisation's (k + 2) n_t 8 B
    k_its = int(round(its))
    alg = k_its * (E * nT * nT * 4 + E * 2 * nT * 8) + sum((k + 2) * nt_u * 8 for k in range(1, k_its + 1))
    # bytes this implementation moves beyond those: the face-block inverses of the preconditioner
    # (ntrace bs^2 4 B per iteration) and the deferred second Gram-Schmidt pass over the FP32 basis
    extra = k_its * ntrace * bs * bs * 4 + sum((k + 1) * nt_u * 4 for k in range(1, k_its + 1))
    out["gmres"] = entry("k_gmres_cycle", "hbm", alg / (a * 1e-3) / 1e9, hbm_peak, "GB/s", tot, a)
    per = GMRES_TRAFFIC_PER_ELEM_ITER.get(nT)
    out["gmres"]["traffic"] = per * E * k_its if per else None
    out["gmres"]["iterations_per_launch"] = k_its
    out["gmres"]["algorithmic_bytes"] = alg
    out["gmres"]["implementation_extra_bytes"] = extra
    tot, a = avg("condense_factor")
    inv = "k_inverse_tc" if cond_mode >= 2 else ("k_inverse_warp" if nA <= 64 else "k_inverse_rq")
    out["condense_factor"] = entry(inv, "alu", E * 2.0 * nA**3 / (a * 1e-3) / 1e12, alu_peak, "TFLOP/s", tot, a)
    tot, a = avg("condense_products")
    fl = E * 2.0 * (nA * nA * (nT + 1) + nT * nA * (nT + 1)) / (a * 1e-3) / 1e12
    by = E * (4.0 * (nA * nA + 2 * nA * nT + nT * nT) + 4.0 * (nA * nT + nT * nT)) / (a * 1e-3) / 1e9
    if cond_mode >= 1:
        pk, fpk, funit = "k_products_tc", tf32_peak, "TF32 TFLOP/s"
    else:
        pk, fpk, funit = ("k_condense_products" if nA <= 64 else "k_products_x+k_products_s"), alu_peak, "TFLOP/s"
    if by / hbm_peak > fl / fpk:
        out["condense_products"] = entry(pk, "hbm", by, hbm_peak, "GB/s", tot, a)
    else:
        out["condense_products"] = entry(pk, "tensor" if cond_mode >= 1 else "alu", fl, fpk, funit, tot, a)
    tot, a = avg("jacobian")
    out["jacobian"] = entry("k_jacobian", "alu", E * (nA + nT) ** 2 * (2 * n + 4) * 2.0 / (a * 1e-3) / 1e12,
                            alu_peak, "TFLOP/s", tot, a)
    dom = max(out, key=lambda k: out[k]["total_ms"])
    return dom, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refine", type=int, default=0,
                    help="FP64 refinement sweeps of the local solves in the back-substitution")
    ap.add_argument("--workload", default="vortex256", choices=list(WORKLOADS))
    ap.add_argument("--jacobian", default="every", choices=["every", "once"],
                    help="re-linearise at every Newton iterate, or once per stage (chord iterations)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", default="both", choices=["both", "mixed", "fp64"],
                    help="profiling aid: time only one precision path")
    ap.add_argument("--no-e2e", action="store_true", help="profiling aid: skip the host-buffer e2e leg")
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven-degree condensation leg")
    ap.add_argument("--no-reuse", action="store_true", help="skip the Jacobian-reuse (imex_steps) leg")
    ap.add_argument("--no-tf32", action="store_true", help="skip the single-pass TF32 condensation leg")
    ap.add_argument("--no-channel", action="store_true", help="skip the hexahedral channel leg")
    ap.add_argument("--no-efr", action="store_true", help="skip the EFR-trace leg on the vortex256 mesh")
    ap.add_argument("--general-only", default=None, choices=list(GENERAL_WORKLOADS),
                    help="profiling aid: time only this general-mesh workload's mixed path")
    ap.add_argument("--no-boundary-layer", action="store_true",
                    help="skip the boundary-layer (mixed degree, walls, far field) leg")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16 trace-operator leg")
    ap.add_argument("--no-tight", action="store_true",
                    help="skip the tight-tolerance agreement leg of the mixed and FP64 stages")
    ap.add_argument("--no-autotune", action="store_true",
                    help="profiling aid: keep the default kernel forms (timings under a profiler would mislead the tuner)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch

    import paper_2401_16632_gb300 as pkg
    from paper_2401_16632_gb300.build import build
    from workloads import make_config

    build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if args.workload in ("vortex64p4", "vortex128p4"):
        w = make_config("vortex", n=64 if args.workload == "vortex64p4" else 128, p=4, noise=1.0e-3, seed=1234)
    else:
        w = make_config(args.workload)
    l2buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB
    pipe_peaks = measure_pipe_peaks(pkg)
    if args.general_only:  # profiling aid: one general-mesh workload, mixed path, no JSON contract line
        print(json.dumps(general_leg(pkg, torch, dev, l2buf, args.general_only, steps=(args.steps, 0),
                                     warmup=(args.warmup, 0), paths=("mixed",))))
        return
    if args.paths != "both":  # profiling aid: one path, no JSON contract line
        prec = pkg.FR_PREC_FP32 if args.paths == "mixed" else pkg.FR_PREC_FP64
        r = time_path(pkg, torch, w, prec, args.refine if args.paths == "mixed" else 0, args.steps, args.warmup,
                      dev, l2buf, args.jacobian, autotune=not args.no_autotune)
        print(json.dumps({"path": args.paths, "ms": r["ms"], "stats": r["stats"],
                          "phases_ms_total": r["profile"], "launches": r["launches"]}))
        return
    barrier = dist.barrier if dist is not None else None
    with ClockSampler(local) as clk:
        mixed = time_path(pkg, torch, w, pkg.FR_PREC_FP32, args.refine, args.steps, args.warmup, dev, l2buf,
                          args.jacobian, barrier, autotune=not args.no_autotune)
        fp64 = time_path(pkg, torch, w, pkg.FR_PREC_FP64, 0, args.steps, args.warmup, dev, l2buf, args.jacobian,
                         barrier)
        # the same mixed stage as one CUDA graph (no per-kernel phases: timed as a whole)
        tf32 = None
        if not args.no_tf32:
            try:  # the same stream stage with the single-pass TF32 condensation (not the headline)
                tf32 = time_path(pkg, torch, w, pkg.FR_PREC_FP32, args.refine, args.steps, args.warmup, dev, l2buf,
                                 args.jacobian, barrier, autotune=not args.no_autotune,
                                 cond_mode=pkg.FR_CONDENSE_TENSOR_TF32)
            except Exception as exc:  # reported, never fatal
                tf32 = {"error": str(exc)}
        bf16 = None
        if not args.no_bf16:
            try:  # the same stream stage with the trace operator in BF16 (FR_PREC_BF16)
                bf16 = time_path(pkg, torch, w, pkg.FR_PREC_BF16, args.refine, args.steps, args.warmup, dev, l2buf,
                                 args.jacobian, barrier, autotune=False)
            except Exception as exc:  # reported, never fatal
                bf16 = {"error": str(exc)}
        graph = None
        if args.jacobian == "every":
            graph = time_path(pkg, torch, w, pkg.FR_PREC_FP32, args.refine, args.steps, args.warmup, dev, l2buf,
                              args.jacobian, barrier, graph=True, autotune=not args.no_autotune)
    clocks = clk.summary()
    ms_mixed, ms_fp64 = replica_max([np.mean(mixed["ms"]), np.mean(fp64["ms"])], dist, dev)
    ms_graph = replica_max([np.mean(graph["ms"])], dist, dev)[0] if graph else None
    # headline: the graph stage where it exists (same kernels and results as the stream path, whose
    # per-phase CUDA-event timings give the per-kernel rooflines)
    head, ms_head = (graph, ms_graph) if graph else (mixed, ms_mixed)
    dofs = w.dofs_implicit
    # agreement of the two converged stages (same equations, same tolerance)
    inc = (fp64["u"] - torch.tensor(w.u0, device=dev)).abs().max().item()
    diff = (mixed["u"] - fp64["u"]).abs().max().item() / inc
    if args.no_e2e:
        e2e_ms, bi, bo = float("nan"), 0, 0
    else:
        e2e_ms, bi, bo = time_e2e(pkg, torch, head["ctx"], w, max(3, args.steps // 2), dev)
        e2e_ms = replica_max([e2e_ms], dist, dev)[0]
    peaks, peak_src = _peaks()
    peaks = dict(peaks)
    peaks.update({k: v for k, v in pipe_peaks.items() if isinstance(v, float)})
    pm = {k: v[0] for k, v in mixed["profile"].items()}
    dom, kroofs = kernel_rooflines(mixed["profile"], mixed["stats"], w, peaks, clocks, args.workload,
                                   mixed["ctx"].hfr_condense_get_mode())
    roof = {k: v for k, v in kroofs[dom].items() if k != "total_ms"}
    line = {
        "metric": METRIC,
        "value": job_value(world, dofs, ms_head),
        "unit": "DOF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_head,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "implicit_dofs": dofs, "elements": w.mesh.nelem,
                   "newton_tol": NEWTON_TOL, "gmres_rtol": GMRES_RTOL, "refine_sweeps": args.refine,
                   "jacobian": args.jacobian,
                   "stage_execution": "one CUDA graph per stage" if graph else "stream, kernel by kernel",
                   "autotune": ({k: v for k, v in mixed["tune"].items()} if mixed.get("tune") else None),
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "fp64": {"value": job_value(world, dofs, ms_fp64), "ms_per_step": ms_fp64, "dtype": "f64",
                 "newton_iterations": fp64["stats"]["newton_iterations"],
                 "gmres_iterations": fp64["stats"]["gmres_iterations"],
                 "phases_ms_total": {k: round(v[0], 3) for k, v in fp64["profile"].items()}},
        "stream_stage": {"ms_per_step": ms_mixed, "value": job_value(world, dofs, ms_mixed),
                         "gpu_launches": int(mixed["launches"] // max(args.steps, 1)),
                         "note": "the same mixed stage launched kernel by kernel from the host (per-phase "
                                 "CUDA events: the per-kernel rooflines)"},
        "mixed_over_fp64": ms_fp64 / ms_mixed,
        "mixed_vs_fp64_max_rel_diff": diff,
        "newton_iterations": mixed["stats"]["newton_iterations"],
        "gmres_iterations": mixed["stats"]["gmres_iterations"],
        "phases_ms_total": {k: round(v, 3) for k, v in pm.items()},
        "dominant_phase": dom,
        "roofline": roof,
        "kernel_rooflines": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                             for k, v in kroofs.items()},
        "e2e": {"value": job_value(world, dofs, e2e_ms), "unit": "DOF/s", "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo},
        "gpu_launches": int(head["launches"] // max(args.steps, 1)),
        "gpu_launches_note": "kernels of libhfr.so executed per timed step (mixed path)",
        "clocks": clocks,
        "peaks_source": peak_src,
        "pipe_peaks_measured": pipe_peaks,
    }
    if not args.no_tight:
        try:
            line["mixed_vs_fp64_tight"] = tight_agreement(pkg, torch, w, mixed["ctx"], fp64["ctx"], dev)
        except Exception as exc:  # reported, never fatal
            line["mixed_vs_fp64_tight"] = {"error": str(exc)}
    if tf32 is not None:
        if "error" in tf32:
            line["tf32_single_pass"] = tf32
        else:
            ms_t = replica_max([np.mean(tf32["ms"])], dist, dev)[0]
            line["tf32_single_pass"] = {
                "value": job_value(world, dofs, ms_t), "ms_per_step": ms_t,
                "newton_iterations": tf32["stats"]["newton_iterations"],
                "gmres_iterations": tf32["stats"]["gmres_iterations"], "converged": tf32["stats"]["converged"],
                "max_rel_diff_vs_fp64": (tf32["u"] - fp64["u"]).abs().max().item() / inc,
                "note": "stream stage with FR_CONDENSE_TENSOR_TF32 (one TF32 product per term in the tensor-core "
                        "factorisation and products); compare stream_stage"}
    if bf16 is not None:
        if "error" in bf16:
            line["bf16_trace_operator"] = bf16
        else:
            ms_b = replica_max([np.mean(bf16["ms"])], dist, dev)[0]
            line["bf16_trace_operator"] = {
                "value": job_value(world, dofs, ms_b), "ms_per_step": ms_b,
                "newton_iterations": bf16["stats"]["newton_iterations"],
                "gmres_iterations": bf16["stats"]["gmres_iterations"], "converged": bf16["stats"]["converged"],
                "max_rel_diff_vs_fp64": (bf16["u"] - fp64["u"]).abs().max().item() / inc,
                "phases_ms_total": {k: round(v[0], 3) for k, v in bf16["profile"].items()},
                "note": "stream stage with FR_PREC_BF16: S_k stored in BF16 for the single-launch GMRES mat-vecs "
                        "(FP32 accumulation), everything else as the mixed path; compare stream_stage"}
            if not args.no_tight:
                try:
                    line["bf16_trace_operator"]["tight"] = tight_agreement(pkg, torch, w, bf16["ctx"], fp64["ctx"], dev,
                                                                           refines=(0,))
                except Exception as exc:
                    line["bf16_trace_operator"]["tight"] = {"error": str(exc)}
    if not args.no_reuse:
        try:
            line["jacobian_reuse"] = jacobian_reuse(pkg, torch, mixed["ctx"], w, dev)
        except Exception as exc:  # reported, never fatal
            line["jacobian_reuse"] = {"error": str(exc)}
    # the vortex256 contexts are done: release their device memory before the general-mesh legs
    for r in (mixed, fp64, tf32, bf16, graph):
        if isinstance(r, dict) and r.get("ctx") is not None:
            r["ctx"].close()
    torch.cuda.empty_cache()
    if not args.no_boundary_layer:
        try:
            line["boundary_layer"] = general_leg(pkg, torch, dev, l2buf, "boundary_layer", peaks=peaks)
        except Exception as exc:  # reported, never fatal
            line["boundary_layer"] = {"error": str(exc)}
    if not args.no_channel:
        try:
            line["channel3d"] = general_leg(pkg, torch, dev, l2buf, "channel3d", steps=(2, 1), warmup=(1, 1), peaks=peaks)
        except Exception as exc:  # reported, never fatal
            line["channel3d"] = {"error": str(exc)}
    if not args.no_efr:
        try:
            line["efr_vortex256"] = general_leg(pkg, torch, dev, l2buf, "efr_vortex256", steps=(3, 1), warmup=(1, 1),
                                                peaks=peaks)
        except Exception as exc:  # reported, never fatal
            line["efr_vortex256"] = {"error": str(exc)}
    if not args.no_uneven:
        try:
            line["uneven_condense"] = uneven_condense(pkg, torch, dev)
        except Exception as exc:  # reported, never fatal
            line["uneven_condense"] = {"error": str(exc)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        except Exception as exc:  # reported, never fatal
            line["cpu_baseline"] = {"error": str(exc)}
        try:
            line["cpu_baseline"]["single_core"] = cpu_baseline_single_core(args.workload)
        except Exception as exc:  # reported, never fatal
            line["cpu_baseline"]["single_core"] = {"error": str(exc)}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def reference_arm(args, rank, world):
    """The oracle (FP64 CPU, as it stands) on the host cores, on bounded samples of the same
    workload (see cpu_baseline)."""
    if rank != 0:
        return
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args.workload)
        if i >= args.warmup:
            vals.append(cb["value"])
            info = cb
    v = float(np.mean(vals))
    line = {
        "metric": METRIC,
        "value": v,
        "unit": "DOF/s",
        "n_gpus": 0,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": info["dofs"] / v * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "impl": "reference",
        "config": {"workload": WORKLOADS[args.workload], "sample": info["sample"]},
        "cpu_baseline": {"value": v, "unit": "DOF/s", "cores": info["cores"], "kind": "oracle",
                         "sample": info["sample"]},
        "e2e": {"value": v, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
