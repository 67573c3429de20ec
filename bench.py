#!/usr/bin/env python3
"""Throughput of the TENO finite-volume hot path on one GB300.

Default workload: the periodic shear layer on [0,1]^2 (density 2 inside
|y - 0.5| < 0.25 and 1 outside, u = -+0.5 with tanh thickness 0.01, p = 2.5,
an 8-mode seeded v perturbation) on a jittered 2048x2048 split-quad mesh
(8,388,608 triangles), 6th-order TENO (large stencil of 42 cells, three
directional stencils of 12), HLL flux, SSP-RK3 with the CFL step (0.4)
reduced on the device.  One "step" = one SSP-RK3 step = 3 residual stages,
each running every step of the path (stencil differences, matvecs,
smoothness indicators, cutoff and selection, Gauss-point evaluation, face
fluxes, residual gather, RK update) plus the CFL reduction.  Metric:
cell-stage updates per second = n_cell * 3 * steps / time.  The per-cell
reconstruction matrices (68 GB in FP64) are far larger than L2, so no flush
is needed between steps.

The primary line is the FP64 path on the FP64 pipe (dtype f64).  Labelled
legs: fp64_pairs (the FP64-accurate double-float path, ~48-bit
significands), fp32_mixed, the adjoint, CWENO and the end-to-end call with
host buffers.  Every leg reports its residual error against the oracle on
sampled cells (per variable) and its selection flip rate against the FP64
path, both at the initial state.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload shear|vortex] [--n N] [--order P]

--impl reference times the CPU oracle (oracle/) on the host cores on a bounded
sample of the same workload.  Under torchrun every rank runs an independent
replica (the path needs no collective on one mesh); rank 0 prints one JSON
line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/sec at 1 GB300 (FP64 vs FP32-mixed), % HBM roofline; adjoint/forward time"
UNIT = "cell-stage/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
KERNELS_SRC = os.path.join(ROOT, "paper_2105_02127_gb300", "csrc", "teno_kernels.cu")
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the
# dominant kernel per cell, keyed by (path, order), with the sha256 prefix of
# csrc/teno_kernels.cu the capture was taken with (summaries in profiles/); a
# launch's traffic is this times the cells it processes.  An entry whose
# source hash differs from the current file's is stale and reported as null.
# Captured on the 131,072-cell shear layer (TENO6; matrices ~2 GB, above L2)
# and scaled by the cells of a launch: the streamed bytes are per cell.
NCU_TRAFFIC_PER_CELL = {
    ("fp64_native", 6): (8033.0, "0b2213304e9869b8"),
    ("fp64_pairs", 6): (8047.6, "0b2213304e9869b8"),
    ("fp32_mixed", 6): (4420.2, "0b2213304e9869b8"),
    ("adjoint_vjp", 6): (3629.6, "0b2213304e9869b8"),
}


def kernels_hash():
    with open(KERNELS_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(path, order, n_cell):
    e = NCU_TRAFFIC_PER_CELL.get((path, order))
    if e is None or e[1] != kernels_hash():
        return None
    return e[0] * n_cell


def parse():
    """Command line; workload-dependent defaults are filled in after parsing."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed SSP-RK3 steps (default 20 on the shear layer, 50 on the vortex)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shear", choices=["shear", "vortex"],
                    help="shear: periodic shear layer on [0,1]^2 (default); vortex: isentropic "
                         "vortex on [0,10]^2")
    ap.add_argument("--n", type=int, default=None,
                    help="quads per side, 2 n^2 triangles (shear 2048, vortex 512)")
    ap.add_argument("--order", type=int, default=None, help="TENO order (shear 6, vortex 5)")
    ap.add_argument("--extras", default="pairs,mixed,adjoint,cweno,e2e,cpu",
                    help="comma list of extra legs: pairs, mixed, adjoint, cweno, e2e, cpu, "
                         "charvar (characteristic-variable TENO on the pair path; not in the "
                         "default list)")
    ap.add_argument("--no-extras", action="store_true", help="the primary line only")
    ap.add_argument("--primary", default="native", choices=["native", "pairs", "mixed"],
                    help="path timed as the primary line: native FP64 (default), the "
                         "double-float FP64-accurate path, or FP32-mixed")
    a = ap.parse_args()
    if a.n is None:
        a.n = 2048 if a.workload == "shear" else 512
    if a.order is None:
        a.order = 6 if a.workload == "shear" else 5
    if a.steps is None:
        a.steps = 20 if a.workload == "shear" else 50
    a.extra_set = set() if a.no_extras else {e for e in a.extras.split(",") if e}
    return a


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload(n, order, kind="shear"):
    from paper_2105_02127_gb300 import inputs
    if kind == "shear":
        mesh = inputs.jittered_mesh(n, n, 1.0, 1.0, seed=1005)
        U = inputs.cell_average(mesh, inputs.shear_layer(seed=2005), n_quad=3)
        return mesh, U
    mesh = inputs.jittered_mesh(n, n, 10.0, 10.0, seed=1002)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    return mesh, U


def workload_name(args, n_cell):
    if args.workload == "shear":
        return (f"periodic shear layer on [0,1]^2 (density 2/1, u = -+0.5, 8-mode seeded v "
                f"perturbation), jittered {args.n}x{args.n} split quads = {n_cell} triangles, "
                f"TENO{args.order}, HLL, SSP-RK3, CFL 0.4 (device dt)")
    return (f"isentropic vortex, periodic [0,10]^2, jittered {args.n}x{args.n} split quads = "
            f"{n_cell} triangles, TENO{args.order}, HLL, SSP-RK3, CFL 0.4 (device dt)")


def sizes(order):
    r = order - 1
    m = (r + 1) * (r + 2) // 2 - 1
    ns = 2 * (m + 1)
    return m, ns, m * ns + 3 * 12 * 5


def algorithmic_bytes(order, n_var, precision):
    """Bytes one cell-stage must move (the per-unit figure of the hot-path
    table): the per-cell reconstruction matrices (FP64 or FP32), the
    (N_s + 36) int32 stencil ids, the state and RK operands (U^(s) and U^n
    read, U^(s+1) written: 3 n_var doubles), the cell's geometry (1/|V| and
    its three face ids; per face, shared by two cells, nx, ny, |A| as doubles,
    two int32 cells and two int8 local edges) and the selection and stencil
    mask bytes.  Gauss-point values and face fluxes are implementation
    overhead and not counted."""
    m, ns, entries = sizes(order)
    esz = 4 if precision == "fp32_mixed" else 8
    geometry = 8 + 3 * 4 + 1.5 * (3 * 8 + 2 * 4 + 2)
    return entries * esz + (ns + 36) * 4 + 3 * n_var * 8 + geometry + n_var + 1


def algorithmic_vjp_bytes(order, nq):
    """Bytes one tiled reconstruction-VJP launch must move per cell (Euler,
    FP64 path, large stencil kept): the per-cell W = Psi' G pairs, the halo
    positions of the large-stencil slots, Uq_bar at the 3 nq Gauss points,
    the selection bytes and the cell's own dU_0 term.  The per-tile halo
    partial sums are implementation overhead and not counted; tiles where a
    cell keeps a directional stencil also stream its (hi, lo) matrices."""
    m, ns, _ = sizes(order)
    nq3 = 3 * nq
    return ns * nq3 * 8 + ns * 2 + nq3 * 4 * 8 + 4 + 4 * 8


def algorithmic_fp64_flops(order, n_var, nq):
    """FP64 flops per cell of the native reconstruction in the W form (the
    default native kernel, recon_tma_w_kernel<native>): per variable the
    N_s + 36 stencil differences, the Gauss-point values U_0 + W d as
    N_s x 3 N_q multiply-adds (2 flops each) and 3 N_q additions.  The
    smoothness indicators and the cutoff run on the FP32 pipe (with the FP64
    fallback where their error bound does not decide), so they are not FP64
    work; the direct evaluation of the hot-path table (coefficients, beta,
    evaluation: about 14.4k flops at TENO6) is the same mathematics."""
    m, ns, entries = sizes(order)
    per_var = (ns + 36) + 2 * ns * 3 * nq + 3 * nq
    return per_var * n_var


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.index = index
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader",
                                       "-i", str(self.index), "-lms", "50"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def timed_steps(t, steps, stream, barrier):
    import torch
    t.profile(True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t.rk3_steps(steps, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    kms, launches = t.profile_read()
    t.profile(False)
    return ms, kms, launches


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2105_02127_gb300 import replicas

    rank, world, local = replicas.world()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    barrier = replicas.barrier

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, device="cuda")

    import __graft_entry__ as g
    g.build()
    from paper_2105_02127_gb300 import teno

    peaks, peak_src = load_peaks()
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    dev = torch.cuda.current_device()
    # measured FMA pipe peaks of this GPU (before any context holds memory)
    fp64_peak = teno.fma_peak(1, device=dev) / 1e12
    fp32_peak = teno.fma_peak(0, device=dev) / 1e12
    mesh, U = workload(args.n, args.order, args.workload)
    n_cell = mesh.n_cell
    stream = torch.cuda.current_stream()
    Ud = torch.from_numpy(U).cuda()
    nq = 2 if args.order <= 4 else 3
    code = {"native": teno.FP64_NATIVE, "pairs": teno.FP64, "mixed": teno.FP32_MIXED}
    key = {"native": "fp64_native", "pairs": "fp64_pairs", "mixed": "fp32_mixed"}
    dtypes = {"native": "f64",
              "pairs": "f64-pairs (double-float fp32x2 arithmetic, ~48-bit significands, for "
                       "matvecs, Gauss values and fluxes; f64 cutoff decision near C_T, residual "
                       "accumulation and update)",
              "mixed": "f32 matvecs and fluxes; f64 cutoff decision near C_T, residual "
                       "accumulation and update"}
    rng = np.random.default_rng(0)
    cells = np.sort(rng.choice(n_cell, min(n_cell, 2000), replace=False))
    cells_t = torch.from_numpy(cells).cuda()

    def make(path, scheme="teno"):
        t = teno.Teno(device=dev, stream=stream).load(mesh)
        kw = {"charvar": 1} if scheme == "charvar" else {"scheme": scheme}
        t.precompute_stencils(order=args.order, n_var=4, flux=teno.FLUX_HLL,
                              precision=code[path], **kw)
        t.set_state(Ud)
        return t

    def roofline(path, scheme, rec_ms):
        nbytes = algorithmic_bytes(args.order, 4, key[path]) * n_cell
        gbs = nbytes / (rec_ms / 1e3) / 1e9
        if path == "native":
            kernel = f"recon_tma_w_kernel <fp64 native> order {args.order}"
        elif path == "pairs":
            kernel = {"teno": f"recon_tma_w_kernel <fp64 pairs> order {args.order}",
                      "cweno": f"recon_tma_kernel <fp64 pairs, CWENO> order {args.order}",
                      "charvar": f"recon_tma_kernel <fp64 pairs, coefficients> + "
                                 f"char_finish_kernel order {args.order}"}[scheme]
        else:
            kernel = f"recon_tma_kernel <fp32_mixed> order {args.order}"
        traffic = ncu_traffic(key[path], args.order, n_cell) if scheme == "teno" else None
        if path == "native":
            fl = algorithmic_fp64_flops(args.order, 4, nq) * n_cell / (rec_ms / 1e3) / 1e12
            return {"bound": "alu", "achieved": fl, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": fl / fp64_peak, "traffic": traffic, "kernel": kernel,
                    "peak_source": "FP64 FMA rate measured in this run (teno_fma_peak: "
                                   "independent DFMA chains on every SM)",
                    "flops_per_cell": algorithmic_fp64_flops(args.order, 4, nq),
                    "hbm_achieved_gbs": gbs, "hbm_frac": gbs / hbm_gbs}
        return {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s",
                "frac": gbs / hbm_gbs, "traffic": traffic, "kernel": kernel,
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)",
                "bytes_per_cell": algorithmic_bytes(args.order, 4, key[path])}

    def leg(path, scheme="teno", steps=None, clocks=False, after=None):
        steps = steps or args.steps
        t = make(path, scheme)
        # the initial state's residual and selection (outside the timed region)
        R = torch.empty_like(Ud)
        sel = torch.empty(Ud.shape, dtype=torch.uint8, device="cuda")
        t.residual(out=R, sel=sel)
        t.check_state()
        res = {"_R_cells": R.index_select(1, cells_t).cpu().numpy(),
               "_R_scale": R.abs().amax(dim=1).cpu().numpy(), "_sel": sel.cpu().numpy()}
        del R, sel
        t.rk3_steps(args.warmup, 0.0)
        t.check_state()
        clk = Clocks(dev) if clocks else None
        if clk:
            clk.__enter__()
        ms, kms, launches = timed_steps(t, steps, stream, barrier)
        if clk:
            clk.__exit__()
        t.check_state()
        ms = max_over_ranks(ms)
        rec_ms = kms[0] / max(1, launches[0])
        res.update({"value": n_cell * 3 * steps * world / (ms / 1e3), "unit": UNIT,
                    "ms_per_step": ms / steps, "steps": steps,
                    "roofline": roofline(path, scheme, rec_ms), "kernel_ms": kms.tolist(),
                    "launches": launches.tolist(), "recon_ms_per_launch": rec_ms,
                    "dtype": dtypes[path]})
        if clk:
            res["clocks"] = clk.summary()
        if after:
            after(t, res)
        Uf = torch.empty_like(Ud)
        t.get_state(Uf)
        res["_rho_final"] = Uf[0].cpu().numpy()
        t.close()
        torch.cuda.synchronize()
        return res

    def adjoint_leg(t, res):
        # the adjoint of one SSP-RK3 step: from a recorded step (the reverse
        # sweep of a checkpointed adjoint, whose segment replay records its
        # steps), and with its own replay of the forward stages
        lam = torch.from_numpy(np.ones_like(U)).cuda()
        lam_out = torch.empty_like(lam)
        dt_a = 1e-4
        na = max(2, args.steps // 4)
        t.set_state(Ud)
        t.tape_reserve(1)
        t.rk3_step_record(0, dt_a)  # warm-up
        t.adjoint_step_tape(0, lam, lam_out)
        torch.cuda.synchronize()

        def timed(fn):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t.profile(True)
            e0.record(stream)
            for _ in range(na):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            kms, kl = t.profile_read()
            t.profile(False)
            return e0.elapsed_time(e1) / na, kms / na, kl

        rec_ms, _, _ = timed(lambda: t.rk3_step_record(0, dt_a))
        tape_ms, akms, alaunch = timed(lambda: t.adjoint_step_tape(0, lam, lam_out))
        t.tape_reserve(0)
        t.set_state(Ud)
        t.adjoint_step(dt_a, lam, lam_out)
        replay_ms, _, _ = timed(lambda: t.adjoint_step(dt_a, lam, lam_out))
        vjp_ms = akms[6] * na / max(1, alaunch[6])
        vjp_gbs = algorithmic_vjp_bytes(args.order, nq) * n_cell / (vjp_ms / 1e3) / 1e9
        fwd = res["ms_per_step"]
        res["adjoint"] = {
            "ms_per_step": tape_ms, "forward_ms_per_step": fwd,
            "adjoint_over_forward": tape_ms / fwd,
            "record_ms_per_step": rec_ms, "record_over_forward": rec_ms / fwd,
            "with_replay_ms_per_step": replay_ms, "with_replay_over_forward": replay_ms / fwd,
            "roofline": {"bound": "hbm", "achieved": vjp_gbs, "peak": hbm_gbs, "unit": "GB/s",
                         "frac": vjp_gbs / hbm_gbs,
                         "traffic": ncu_traffic("adjoint_vjp", args.order, n_cell),
                         "kernel": f"recon_vjp_tma_kernel <fp64 pairs> order {args.order}",
                         "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)",
                         "ms_per_launch": vjp_ms},
            "kernel_ms_per_step": akms.tolist(),
            "note": "FP64 pair path.  ms_per_step: the adjoint of a recorded step "
                    "(teno_adjoint_step_tape: three flux and reconstruction VJPs, no "
                    "reconstruction), the reverse sweep of a checkpointed adjoint; its segment "
                    "replay records each step (record_ms_per_step, the forward step plus the "
                    "copies of the stage states).  with_replay: teno_adjoint_step, which "
                    "replays the step's forward stages itself."}

    def e2e_leg(t, res):
        # end to end through the C ABI with pinned host buffers
        hin = torch.from_numpy(U.copy()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        n_e2e = max(2, min(args.steps, 10))
        for _ in range(2):
            t.set_state(hin)
            t.rk3_step(0.0, sync=False)
            t.get_state(hout)
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(n_e2e):
            t.set_state(hin)
            t.rk3_step(0.0, sync=False)
            t.get_state(hout)
        torch.cuda.synchronize()
        w1 = time.perf_counter()
        barrier()
        e2e_s = max_over_ranks(w1 - w0)
        nbytes = U.size * 8
        res["e2e"] = {"value": n_cell * 3 * n_e2e * world / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                      "steps": n_e2e}

    ex = args.extra_set
    legs = {}
    legs[args.primary] = leg(args.primary, clocks=True,
                             after=(lambda t, r: (e2e_leg(t, r) if "e2e" in ex else None,
                                                  adjoint_leg(t, r) if "adjoint" in ex and
                                                  args.primary == "pairs" else None)))
    for path in ("pairs", "mixed", "native"):
        if path == args.primary or path not in ex:
            continue
        legs[path] = leg(path, after=(adjoint_leg if path == "pairs" and "adjoint" in ex
                                      else None))
    cweno = None
    if "cweno" in ex:
        cweno = leg("pairs", scheme="cweno", steps=max(2, args.steps // 4))
    charvar = None
    if "charvar" in ex:
        charvar = leg("pairs", scheme="charvar", steps=max(2, args.steps // 4))
    # selection flips against the FP64 path on the same (initial) state
    ref = legs.get("native", legs[args.primary])["_sel"]
    for r in list(legs.values()) + ([cweno] if cweno else []):
        r["flip_rate_vs_fp64"] = float((r["_sel"] != ref).mean())
    # the oracle on the host cores: CPU baseline and each leg's error on sampled cells
    cpu = None
    if rank == 0 and world == 1 and "cpu" in ex:
        cpu, Ro, selo, mg, fsc = cpu_baseline(args, mesh, U, cells)
        for r in list(legs.values()) + ([cweno] if cweno else []):
            diff = np.abs(r["_R_cells"].T - Ro)
            d = diff.max(axis=0) / np.maximum(r["_R_scale"], 1e-300)
            dk = (diff / np.maximum(fsc, 1e-300)).max(axis=0)
            r["err_vs_oracle"] = {
                "per_variable": d.tolist(), "max": float(d.max()), "cells": len(cells),
                "norm": "max over sampled cells of |R - R_oracle| / max over the field of |R|, "
                        "per conservative variable",
                "flux_relative_per_variable": dk.tolist(), "flux_relative_max": float(dk.max()),
                "flux_relative_norm": "max over sampled cells of |R - R_oracle| / (sum over the "
                                      "cell's faces of |K_f|, over |V|): rounding measured "
                                      "against the terms that cancel in R",
                "cancellation": (fsc.max(axis=0) / np.maximum(r["_R_scale"], 1e-300)).tolist()}
            own = r["_sel"][:, cells].T
            r["sel_mismatch_vs_oracle"] = int(((own != selo) & (mg > 1e-10)).sum())
    main = legs[args.primary]
    for r in legs.values():
        if r is not main:
            r["l1_rho_diff_vs_primary_after_steps"] = float(
                np.abs(r["_rho_final"] - main["_rho_final"]).mean())
    if cweno:
        cweno["scheme"] = "CWENO, d'_K = 1e4, eps = 1e-14"
        cweno["cweno_over_teno_time"] = cweno["ms_per_step"] / legs["pairs"]["ms_per_step"] \
            if "pairs" in legs else None
    if charvar:
        # selections are per edge and field in this mode (the residual reports 8)
        # and the oracle legs above reconstruct conservative variables
        charvar["scheme"] = "TENO in characteristic variables per edge"
        charvar["charvar_over_teno_time"] = \
            charvar["ms_per_step"] / legs["pairs"]["ms_per_step"] if "pairs" in legs else None

    def public(r):
        return {k: v for k, v in r.items() if not k.startswith("_") and k not in ("e2e",)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": main["dtype"], "data": "synthetic",
            "config": {"workload": workload_name(args, n_cell),
                       "n_cell": n_cell, "order": args.order, "primary_path": key[args.primary],
                       "l2": "inputs larger than L2 (a reconstruction launch reads %.1f GB of "
                             "matrices on the FP64 paths, %.1f GB FP32-mixed)" % (
                                 algorithmic_bytes(args.order, 4, "fp64_native") * n_cell / 1e9,
                                 algorithmic_bytes(args.order, 4, "fp32_mixed") * n_cell / 1e9),
                       "parallelism": f"replicas x{world}"},
            "roofline": main["roofline"], "gpu_launches": int(sum(main["launches"])),
            "kernel_ms": main["kernel_ms"],
            "kernel_kinds": ["recon", "face_flux", "gather_rk", "cfl", "other", "flux_vjp",
                             "recon_vjp", "reverse_gather"],
            "clocks": main.get("clocks"),
            "fma_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak,
                                 "how": "teno_fma_peak in this run"},
            "flip_rate_vs_fp64": main["flip_rate_vs_fp64"],
        }
        if "err_vs_oracle" in main:
            line["err_vs_oracle"] = main["err_vs_oracle"]
            line["sel_mismatch_vs_oracle"] = main["sel_mismatch_vs_oracle"]
        for path, r in legs.items():
            if r is not main:
                line[key[path]] = public(r)
        if "adjoint" in line.get("fp64_pairs", {}):
            line["adjoint"] = line["fp64_pairs"].pop("adjoint")
        elif "adjoint" in main:
            line["adjoint"] = main["adjoint"]
        if cweno:
            line["cweno"] = public(cweno)
        if charvar:
            line["charvar"] = public(charvar)
        if "e2e" in main:
            line["e2e"] = main["e2e"]
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def oracle_sample_rate(o, U, cells, min_seconds):
    """Residuals of the sampled cells, repeated until min_seconds have passed;
    returns (cell-stage/s, R, sel, margin)."""
    R, sel, mg, sc = o.residual_cells(U, cells, flux_scale=True)  # untimed: builds stencils
    n, t0 = 0, time.perf_counter()
    while True:
        o.residual_cells(U, cells)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            return len(cells) * n / dt, R, sel, mg, sc


def cpu_baseline(args, mesh, U, cells):
    """The oracle, untouched, on the host cores, on a bounded sample of the
    same workload: the residuals of sampled cells (each needs the
    reconstructions of the cell and of its three face neighbours).  Also
    returns the oracle's residual, selection, cutoff margin and flux-sum
    scale sum |K_f| / |V| there, from which each leg's error is taken."""
    from oracle.oracle import Oracle
    o = Oracle(mesh, order=args.order, n_var=4, flux=1)
    o.prepare(cells)
    rate, R, sel, mg, sc = oracle_sample_rate(o, U, cells, 10.0)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"residuals of {len(cells)} sampled cells of the {mesh.n_cell}-cell mesh, "
                     "repeated for 10 s after an untimed stencil build; each sampled residual "
                     "reconstructs the cell and its three face neighbours, so per cell this "
                     "is about 3-4x slower than the oracle's full-mesh residual (full_mesh)",
           "cpu_model": cpu_model(), "full_mesh": cpu_full_mesh(args)}
    del o
    return out, R, sel, mg, sc


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


_FULL = """
import sys, time
sys.path.insert(0, {root!r})
import bench
from oracle.oracle import Oracle
mesh, U = bench.workload({n}, {order}, {kind!r})
o = Oracle(mesh, order={order}, n_var=4, flux=1)
o.prepare()
o.residual(U)
t0 = time.perf_counter()
o.residual(U)
print(mesh.n_cell / (time.perf_counter() - t0))
"""


def cpu_full_mesh(args):
    """The oracle's full-mesh residual rate on a 256x256 mesh of the same
    workload (131,072 cells), all cores and one core (fresh processes)."""
    n = 256 if args.workload == "shear" else 128
    out = {"mesh": f"{n}x{n} split quads = {2 * n * n} cells, same workload and order"}
    for label, threads in (("all_cores", None), ("one_core", "1")):
        env = dict(os.environ)
        if threads:
            env["OMP_NUM_THREADS"] = threads
        try:
            r = subprocess.run([sys.executable, "-c",
                                _FULL.format(root=ROOT, n=n, order=args.order, kind=args.workload)],
                               capture_output=True, text=True, timeout=600, env=env)
            out[label] = float(r.stdout.strip().splitlines()[-1])
        except (OSError, subprocess.SubprocessError, ValueError, IndexError):
            out[label] = None
    out["unit"] = UNIT
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        # rank 0 alone runs the oracle: give it the host cores it has at N = 1
        # (the launcher sets one OpenMP thread per rank by default)
        os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    from oracle import build as ob
    ob.build()
    from oracle.oracle import Oracle
    mesh, U = workload(args.n, args.order, args.workload)
    rng = np.random.default_rng(0)
    cells = np.sort(rng.choice(mesh.n_cell, min(mesh.n_cell, 8192), replace=False))
    o = Oracle(mesh, order=args.order, n_var=4, flux=1)
    o.prepare(cells)
    for _ in range(args.warmup):
        o.residual_cells(U, cells)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _s in range(3):
            o.residual_cells(U, cells)
    dt = time.perf_counter() - t0
    value = len(cells) * 3 * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"residuals of {len(cells)} sampled cells of the {mesh.n_cell}-cell mesh, 3 per "
              "step; each sampled residual reconstructs the cell and its three face neighbours, "
              "so per cell this is about 3-4x slower than the oracle's full-mesh residual")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args, mesh.n_cell), "n_cell": mesh.n_cell,
                       "order": args.order, "parallelism": "oracle on the host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
