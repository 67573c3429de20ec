#!/usr/bin/env python3
"""Throughput of the TENO finite-volume hot path on one GB300.

Workload: the periodic isentropic vortex on [0,10]^2 (strength 5, free stream
(1,1,1,1), gamma 1.4) on a jittered 512x512 split-quad mesh (524,288
triangles), 5th-order TENO (large stencil of 30 cells, three directional
stencils of 12), HLL flux, SSP-RK3 with the CFL step (0.4) reduced on the
device.  One "step" = one SSP-RK3 step = 3 residual stages, each running every
step of the path (stencil differences, matvecs, smoothness indicators, cutoff
and selection, Gauss-point evaluation, face fluxes, residual gather, RK
update) plus the CFL reduction.  Metric: cell-stage updates per second =
n_cell * 3 * steps / time.  The per-cell reconstruction matrices (2.5 GB in
FP64) are larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/) on the host cores on a bounded
sample of the same workload.  Under torchrun every rank runs an independent
replica (the path needs no collective on one mesh); rank 0 prints one JSON
line.
"""
from __future__ import annotations

import argparse
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
# FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the
# dominant kernel per cell, (path, order) -> bytes, from the small-case
# captures summarised in profiles/ (64,800-cell vortex mesh; "adjoint_vjp":
# the tiled reconstruction VJP); a launch's traffic is this times the cells
# it processes.  Absent when the kernel changed since the capture.
NCU_TRAFFIC_PER_CELL = {("fp64", 5): 5228.4, ("fp32_mixed", 5): 2668.1, ("fp64_native", 5): 5213.7,
                        ("adjoint_vjp", 5): 2601.9}


def ncu_traffic(precision, order, n_cell):
    b = NCU_TRAFFIC_PER_CELL.get((precision, order))
    return None if b is None else b * n_cell


def parse():
    """Command line; workload-dependent defaults are filled in after parsing."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vortex", choices=["vortex", "shear"],
                    help="vortex: isentropic vortex on [0,10]^2 (default); shear: periodic "
                         "shear layer on [0,1]^2")
    ap.add_argument("--n", type=int, default=None,
                    help="quads per side, 2 n^2 triangles (vortex 512, shear 2048)")
    ap.add_argument("--order", type=int, default=None, help="TENO order (vortex 5, shear 6)")
    ap.add_argument("--extras", default="mixed,native,cweno,adjoint,e2e,cpu",
                    help="comma list of extra legs: mixed, native, cweno, adjoint, e2e, cpu")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed, adjoint, e2e and CPU-baseline legs")
    ap.add_argument("--recon-variant", type=int, default=2, choices=[0, 1, 2],
                    help="reconstruction kernel: 0 halo-staged, 1 direct gathers, 2 TMA-staged")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="path timed as the primary line (the other one is an extra)")
    a = ap.parse_args()
    if a.n is None:
        a.n = 512 if a.workload == "vortex" else 2048
    if a.order is None:
        a.order = 5 if a.workload == "vortex" else 6
    a.extra_set = set() if a.no_extras else {e for e in a.extras.split(",") if e}
    return a


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload(n, order, kind="vortex"):
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


def algorithmic_bytes(order, n_var, precision):
    """Bytes one recon launch must move per cell: the per-cell matrices, the
    stencil ids, the cell's own state and selection byte; neighbour states are
    the same state array (read once).  Gauss-point values are implementation
    overhead and not counted."""
    r = order - 1
    m = (r + 1) * (r + 2) // 2 - 1
    ns = 2 * (m + 1)
    entries = m * ns + 3 * 12 * 5
    esz = 8 if precision == "fp64" else 4
    return entries * esz + (ns + 36) * 4 + n_var * 8 + 1 + n_var


def algorithmic_vjp_bytes(order, nq):
    """Bytes one tiled reconstruction-VJP launch must move per cell (Euler,
    FP64 path, large stencil kept): the per-cell W = Psi' G pairs, the halo
    positions of the large-stencil slots, Uq_bar at the 3 nq Gauss points,
    the selection bytes and the cell's own dU_0 term.  The per-tile halo
    partial sums are implementation overhead and not counted; tiles where a
    cell keeps a directional stencil also stream its (hi, lo) matrices."""
    r = order - 1
    m = (r + 1) * (r + 2) // 2 - 1
    ns = 2 * (m + 1)
    nq3 = 3 * nq
    return ns * nq3 * 8 + ns * 2 + nq3 * 4 * 8 + 4 + 4 * 8


def algorithmic_fp64_flops(order, n_var, nq):
    """FP64 flops per cell of the recon kernel's FP64 path: differences,
    matvecs, beta, selection and Gauss-point evaluation."""
    r = order - 1
    m = (r + 1) * (r + 2) // 2 - 1
    ns = 2 * (m + 1)
    entries = m * ns + 3 * 12 * 5
    per_var = (ns + 36) + 2 * entries + 2 * (m + 15) + 25 + 2 * 3 * nq * m + 3 * nq
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
    mesh, U = workload(args.n, args.order, args.workload)
    n_cell = mesh.n_cell
    stream = torch.cuda.current_stream()
    Ud = torch.from_numpy(U).cuda()
    nq = 2 if args.order <= 4 else 3
    prec_code = {"fp64": teno.FP64, "fp32_mixed": teno.FP32_MIXED,
                 "fp64_native": teno.FP64_NATIVE}

    def make(precision, scheme="teno"):
        t = teno.Teno(device=torch.cuda.current_device(), stream=stream).load(mesh)
        t.precompute_stencils(order=args.order, n_var=4, flux=teno.FLUX_HLL,
                              precision=prec_code[precision], recon_variant=args.recon_variant,
                              scheme=scheme)
        t.set_state(Ud)
        return t

    def measure(precision, clocks=False, scheme="teno"):
        t = make(precision, scheme)
        t.rk3_steps(args.warmup, 0.0)
        t.check_state()
        clk = Clocks(torch.cuda.current_device()) if clocks else None
        if clk:
            clk.__enter__()
        ms, kms, launches = timed_steps(t, args.steps, stream, barrier)
        if clk:
            clk.__exit__()
        t.check_state()
        ms = max_over_ranks(ms)
        rec_ms = kms[0] / max(1, launches[0])
        store = "fp32_mixed" if precision == "fp32_mixed" else "fp64"
        nbytes = algorithmic_bytes(args.order, 4, store) * n_cell
        gbs = nbytes / (rec_ms / 1e3) / 1e9
        var = args.recon_variant
        if precision == "fp64_native" and var == 2:
            var = 0  # the TMA kernel covers the double-float and mixed paths only;
            # variant 2 takes the halo kernel there
        vname = ["recon_halo_kernel", "recon_kernel (direct)", "recon_tma_kernel"][var]
        if precision == "fp64" and var == 2 and scheme == "teno":
            vname = "recon_tma_w_kernel"  # the W form of the pair path
        kernel = f"{vname} <{precision}> order {args.order}"
        roof_hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": gbs / hbm_gbs,
                    "traffic": ncu_traffic(precision, args.order, n_cell) if scheme == "teno" else None,
                    "kernel": kernel, "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)"}
        if precision == "fp64_native":
            fl = algorithmic_fp64_flops(args.order, 4, nq) * n_cell / (rec_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": fl / FP64_PEAK_TFLOPS, "traffic": ncu_traffic(precision, args.order, n_cell),
                    "kernel": kernel,
                    "peak_source": "FP64 pipe: 152 SMs x 4 flop/clk x 2.07 GHz",
                    "hbm_achieved_gbs": gbs, "hbm_frac": gbs / hbm_gbs}
        else:
            roof = roof_hbm
        res = {"value": n_cell * 3 * args.steps * world / (ms / 1e3), "unit": UNIT,
               "ms_per_step": ms / args.steps, "roofline": roof, "kernel_ms": kms.tolist(),
               "launches": launches.tolist(), "recon_ms_per_launch": rec_ms}
        if clk:
            res["clocks"] = clk.summary()
        return t, res

    primary = "fp32_mixed" if args.precision == "mixed" else "fp64"
    t_main, main = measure(primary, clocks=True)
    extras = {}
    ex = args.extra_set
    t64 = t_main
    if ex:
        U_main = t_main.get_state()
        for other, key in (("fp32_mixed", "mixed"), ("fp64_native", "native")):
            if other == primary or key not in ex:
                continue
            t_o, r = measure(other)
            r["l1_rho_diff_vs_primary_after_steps"] = float(np.abs(t_o.get_state()[0] - U_main[0]).mean())
            extras[other] = r
            t_o.close()
    if "cweno" in ex and primary == "fp64":
        # ---- the comparison scheme on the same stencils (the paper's TENO vs
        # CWENO cost comparison, Sec. 5): FP64 path, same workload
        t_c, r = measure("fp64", scheme="cweno")
        r["scheme"] = "CWENO, d'_K = 1e4, eps = 1e-14"
        r["cweno_over_teno_time"] = r["ms_per_step"] / main["ms_per_step"]
        extras["cweno"] = r
        t_c.close()
    if "adjoint" in ex:
        # ---- adjoint / forward (FP64 path)
        lam = torch.from_numpy(np.ones_like(U)).cuda()
        lam_out = torch.empty_like(lam)
        t64.set_state(Ud)
        t64.adjoint_step(0.001, lam, lam_out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        na = max(2, args.steps // 4)
        t64.profile(True)
        e0.record(stream)
        for _ in range(na):
            t64.adjoint_step(0.001, lam, lam_out)
        e1.record(stream)
        torch.cuda.synchronize()
        adj_ms = e0.elapsed_time(e1) / na
        akms, alaunch = t64.profile_read()
        t64.profile(False)
        # dominant adjoint kernel: the tiled reconstruction VJP (kind 6)
        vjp_ms = akms[6] / max(1, alaunch[6])
        vjp_gbs = algorithmic_vjp_bytes(args.order, nq) * n_cell / (vjp_ms / 1e3) / 1e9
        vjp_roof = {"bound": "hbm", "achieved": vjp_gbs, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": vjp_gbs / hbm_gbs,
                    "traffic": ncu_traffic("adjoint_vjp", args.order, n_cell),
                    "kernel": f"recon_vjp_tma_kernel <fp64> order {args.order}",
                    "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)",
                    "ms_per_launch": vjp_ms}
        extras["adjoint"] = {"ms_per_step": adj_ms, "forward_ms_per_step": main["ms_per_step"],
                             "adjoint_over_forward": adj_ms / main["ms_per_step"],
                             "roofline": vjp_roof,
                             "kernel_ms_per_step": (akms / na).tolist(),
                             "note": "one adjoint SSP-RK3 step, including the replay of its two "
                                     "forward stages"}
    if "e2e" in ex:
        # ---- end to end through the C ABI with pinned host buffers
        hin = torch.from_numpy(U.copy()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        for _ in range(2):
            t64.set_state(hin)
            t64.rk3_step(0.0, sync=False)
            t64.get_state(hout)
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            t64.set_state(hin)
            t64.rk3_step(0.0, sync=False)
            t64.get_state(hout)
        torch.cuda.synchronize()
        w1 = time.perf_counter()
        barrier()
        e2e_s = max_over_ranks(w1 - w0)
        nbytes = U.size * 8
        extras["e2e"] = {"value": n_cell * 3 * args.steps * world / e2e_s, "unit": UNIT,
                         "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    cpu = None
    if rank == 0 and world == 1 and "cpu" in ex:
        cpu = cpu_baseline(mesh, U, args.order, samples=20)

    if rank == 0:
        dtype = {"fp64": "f64 (reconstruction and flux in double-float fp32x2 arithmetic, "
                         "~48-bit; residual accumulation and RK update in f64)",
                 "fp32_mixed": "f32 matvec/flux, f64 selection/update"}[primary]
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic",
            "config": {"workload": workload_name(args, n_cell),
                       "n_cell": n_cell, "order": args.order,
                       "l2": "inputs larger than L2 (a reconstruction launch reads %.2f GB "
                             "on the FP64 path, %.2f GB FP32-mixed)" % (
                                 algorithmic_bytes(args.order, 4, "fp64") * n_cell / 1e9,
                                 algorithmic_bytes(args.order, 4, "fp32_mixed") * n_cell / 1e9),
                       "parallelism": f"replicas x{world}"},
            "roofline": main["roofline"], "gpu_launches": int(sum(main["launches"])),
            "kernel_ms": main["kernel_ms"],
            "kernel_kinds": ["recon", "face_flux", "gather_rk", "cfl", "other", "flux_vjp",
                             "recon_vjp", "reverse_gather"],
            "clocks": main.get("clocks"),
        }
        for k in ("fp32_mixed", "fp64_native", "cweno", "adjoint", "e2e"):
            if k in extras:
                line[k] = extras[k]
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(mesh, U, order, samples=1):
    """The oracle, untouched, on the host cores: full-mesh residual stages of
    the same workload after its own (untimed) stencil precompute."""
    from oracle.oracle import Oracle
    o = Oracle(mesh, order=order, n_var=4, flux=1)
    o.prepare()
    t0 = time.perf_counter()
    for _ in range(samples):
        o.residual(U)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": mesh.n_cell * samples / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{samples} full residual stage(s) of the {mesh.n_cell}-cell mesh "
                      f"({dt:.1f} s), stencils precomputed beforehand",
            "cpu_model": cpu_model(), "single_thread": cpu_single_thread(order)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


_SINGLE = """
import sys, time, numpy as np
sys.path.insert(0, {root!r})
import bench
from oracle.oracle import Oracle
mesh, U = bench.workload(128, {order})
o = Oracle(mesh, order={order}, n_var=4, flux=1)
o.prepare()
t0 = time.perf_counter()
o.residual(U)
print(mesh.n_cell / (time.perf_counter() - t0))
"""


def cpu_single_thread(order):
    """The same oracle on one core (OMP_NUM_THREADS=1, a fresh process): one
    full residual stage of the 128x128 vortex mesh (32,768 cells)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", _SINGLE.format(root=ROOT, order=order)],
                           capture_output=True, text=True, timeout=300, env=env)
        v = float(r.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": v, "unit": UNIT, "cores": 1,
            "sample": "one full residual stage of the 128x128 vortex mesh (32,768 cells)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    from oracle.oracle import Oracle
    mesh, U = workload(args.n, args.order, args.workload)
    rng = np.random.default_rng(0)
    cells = np.sort(rng.choice(mesh.n_cell, min(mesh.n_cell, 65536), replace=False))
    o = Oracle(mesh, order=args.order, n_var=4, flux=1)
    nb = mesh.tri  # neighbours are prepared inside residual_cells
    del nb
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
    sample = (f"{len(cells)} sampled cells of the {mesh.n_cell}-cell mesh, 3 residual stages "
              "per step")
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
