"""Double Mach reflection (Sec. 5) as a time run on one GPU.

The Mach-10 shock at 60 degrees to a reflecting wall on [0,4]x[0,1], run to
t = 0.2 with TENO (default TENO6), HLLC, SSP-RK3 at CFL 0.4 and the
positivity scaling of the reconstruction, in FP64 (the double-float path),
FP32-mixed and, when asked for, FP64 on the FP64 pipe (leg fp64_native).  At
sampled steps of the double-float run the selections of the FP64 and
FP32-mixed paths are evaluated on the same stage input states (U^n, U^(1),
U^(2)); their flip rate per stage is the fraction of (cell, variable)
selections that differ.  At the same steps of every run the largest
deviation from the pre-shock state ahead of the incident shock (more than
0.05 ahead of its exact position and above y = 0.5, clear of the Mach stem:
there the exact solution is that state) is recorded with its location.
Prints one JSON object.

  python -m paper_2105_02127_gb300.shock_run [--nx 2048] [--ny 512] [--order 6]
                                             [--t-end 0.2] [--sample-every 50] [--cfl 0.4]
                                             [--legs fp64_pairs,fp32_mixed,fp64_native]
                                             [--dump PREFIX]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(nx: int, ny: int, order: int, t_end: float, sample_every: int, flux: int | None = None,
        dump: str | None = None, cfl: float = 0.4, legs=("fp64_pairs", "fp32_mixed")):
    import torch

    from . import build, inputs, teno
    build.build()
    if flux is None:
        flux = teno.FLUX_HLLC
    mesh = inputs.jittered_mesh(nx, ny, 4.0, 1.0, seed=1003, periodic=False,
                                bc_tagger=inputs.dmr_bc_tagger)
    U0 = inputs.cell_average(mesh, inputs.dmr_state, n_quad=3)
    n_cell = mesh.n_cell

    def ctx(precision):
        t = teno.Teno(device=0).load(mesh)
        t.precompute_stencils(order=order, n_var=4, flux=flux, precision=precision, positivity=1,
                              cfl=cfl)
        return t

    out = {"workload": f"double Mach reflection, [0,4]x[0,1], jittered {nx}x{ny} split quads = "
                       f"{n_cell} triangles, TENO{order}, "
                       f"{'HLLC' if flux == teno.FLUX_HLLC else 'HLL'}, SSP-RK3, CFL {cfl}, "
                       f"positivity scaling, t_end {t_end}",
           "n_cell": n_cell}
    probes = (ctx(teno.FP64), ctx(teno.FP32_MIXED))
    cen = torch.from_numpy(mesh.unwrapped_vertices().mean(axis=1)).cuda()
    pre = torch.tensor([1.4, 0.0, 0.0, 2.5], dtype=torch.float64, device="cuda")[:, None]

    def ahead_dev(Us, time_):
        # ahead of the incident shock x_s(y, t) = 1/6 + (y + 20 t) / sqrt(3),
        # above the Mach stem (which runs ahead of it along the wall)
        ahead = (cen[:, 0] > 0.1667 + (cen[:, 1] + 20.0 * time_) / 1.732 + 0.05) & (cen[:, 1] > 0.5)
        d = (Us - pre).abs().amax(dim=0) * ahead
        i = int(torch.argmax(d).item())
        return [float(d[i].item()), float(cen[i, 0].item()), float(cen[i, 1].item())]
    Rb = torch.empty((4, n_cell), dtype=torch.float64, device="cuda")
    sels = [torch.empty((4, n_cell), dtype=torch.uint8, device="cuda") for _ in range(2)]

    def flips(Us, time_):
        for p, sel in zip(probes, sels):
            p.set_time(time_)
            p.set_state(Us)
            p.residual(out=Rb, sel=sel)
        return float((sels[0] != sels[1]).double().mean().item())

    rho64 = None
    for name, precision in (("fp64_pairs", teno.FP64), ("fp32_mixed", teno.FP32_MIXED),
                            ("fp64_native", teno.FP64_NATIVE)):
        if name not in legs:
            continue
        t = ctx(precision)
        Ud = torch.from_numpy(U0).cuda()
        t.set_state(Ud)
        Un, U1, U2, prev = (torch.empty_like(Ud) for _ in range(4))
        tm, n, per_stage, dev = 0.0, 0, [], []
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        step_s = 0.0
        failure = None
        while tm < t_end - 1e-14:
            dt = min(t.cfl_dt(), t_end - tm)
            sample = name == "fp64_pairs" and n % sample_every == 0
            t.get_state(prev)
            if n % sample_every == 0:
                dev.append([n, tm] + ahead_dev(prev, tm))
            if sample:
                Un.copy_(prev)
            s0 = time.perf_counter()
            try:
                t.rk3_step(dt)
            except teno.TenoError as e:
                failure = _failure(mesh, t, prev, n, tm, dt, str(e), dump, name)
                break
            step_s += time.perf_counter() - s0
            if sample:
                t.stage_state(1, U1)
                t.stage_state(2, U2)
                per_stage.append([n, tm] + [flips(Us, tm) for Us in (Un, U1, U2)])
            tm += dt
            n += 1
        if failure is None:
            t.check_state()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        U = t.get_state()
        rho = U[0]
        p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
        rec = {"steps": n, "t": tm, "wall_s": wall,
               "cell_stage_per_s_in_steps": n_cell * 3 * n / max(step_s, 1e-30),
               "failure": failure,
               "finite": bool(np.isfinite(U).all()), "rho_min": float(rho.min()),
               "p_min": float(p.min()), "rho_max": float(rho.max())}
        dv = np.array([r[2] for r in dev]) if dev else np.zeros(1)
        rec["ahead_of_shock_deviation"] = {
            "every": sample_every, "max": float(dv.max()), "final": float(dv[-1]),
            "samples": dev[::max(1, len(dev) // 40)] + dev[-1:]}
        if name == "fp64_pairs" and per_stage:
            fl = np.array([r[2:] for r in per_stage])
            rec["flip_rate_per_stage"] = {
                "sampled_steps": len(per_stage), "every": sample_every,
                "mean": fl.mean(axis=0).tolist(), "max": fl.max(axis=0).tolist(),
                "overall_max": float(fl.max()), "overall_mean": float(fl.mean()),
                "samples": [[int(r[0]), float(r[1])] + r[2:] for r in per_stage]}
        if name == "fp64_pairs":
            rho64 = rho.copy()
        elif rho64 is not None:
            rec["mean_abs_rho_diff_vs_fp64_pairs_over_mean_rho"] = float(
                np.abs(rho - rho64).mean() / np.abs(rho64).mean())
        out[name] = rec
        t.close()
    for p in probes:
        p.close()
    return out


def _failure(mesh, t, prev, n, tm, dt, msg, dump, name):
    """Where a step produced a non-physical state: the step, the time, the
    stage (1, 2: the stage outputs U^(1), U^(2); 3: the new state), the first
    non-physical cells and their centroids; the state before the step goes to
    `dump` (npz) when given."""
    def bad_cells(U):
        rho = U[0]
        p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
        return np.where(~(np.isfinite(U).all(axis=0) & (rho > 0) & (p > 0)))[0]
    bad, stage = np.array([], dtype=np.int64), 0
    for k, U in ((1, t.stage_state(1)), (2, t.stage_state(2)), (3, t.get_state())):
        b = bad_cells(U)
        if len(b):
            bad, stage = b, k
            break
    cen = mesh.unwrapped_vertices().mean(axis=1)
    out = {"step": n, "t": tm, "dt": dt, "message": msg, "stage": stage, "n_bad": int(len(bad)),
           "bad_cells": bad[:20].tolist(), "centroids": cen[bad[:20]].tolist()}
    if dump and len(bad):
        # the state before the step within 0.1 of the failing cells: all that
        # the residual of those cells depends on
        Up = prev.cpu().numpy()
        d2 = np.full(len(cen), np.inf)
        for c in bad[:50]:
            d2 = np.minimum(d2, ((cen - cen[c]) ** 2).sum(axis=1))
        near = np.where(d2 < 0.01)[0]
        np.savez_compressed(f"{dump}_{name}.npz", cells=near, U=Up[:, near], t=tm, dt=dt,
                            step=n, bad=bad)
        out["dump"] = f"{dump}_{name}.npz"
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--order", type=int, default=6)
    ap.add_argument("--t-end", type=float, default=0.2)
    ap.add_argument("--sample-every", type=int, default=50)
    ap.add_argument("--dump", default=None,
                    help="path prefix: where a step fails, the state before it (npz)")
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--legs", default="fp64_pairs,fp32_mixed")
    a = ap.parse_args()
    print(json.dumps(run(a.nx, a.ny, a.order, a.t_end, a.sample_every, dump=a.dump, cfl=a.cfl,
                         legs=tuple(a.legs.split(",")))))


if __name__ == "__main__":
    main()
