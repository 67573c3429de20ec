"""GPU runs of the workload configurations beyond single residuals.

- isentropic vortex (Sec. 5.2) advected for one period (t = 10) on 32k and 128k
  jittered triangles, TENO5/HLL: L1 density error against the exact solution
  (the initial state), its decrease with resolution, and the FP32-mixed result
  against the FP64 one;
- the adjoint configuration: gradient of J = sum over cells with centroid in
  [4,6]^2 of |V| rho^2 at t = 1 w.r.t. the initial state, 128k triangles,
  TENO5, 200 SSP-RK3 steps of dt = 0.005 with checkpoints every 20 steps,
  against central differences (eps = 1e-6) along 50 seeded directions.
"""
import numpy as np
import pytest

from paper_2105_02127_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_02127_gb300 import autograd, build, teno
    build.build()
    teno.lib()
    return torch, teno, autograd


def _areas(mesh):
    V = mesh.unwrapped_vertices()
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    return 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]), V.mean(axis=1)


def _run_vortex(torch, teno, n, precision, t_end=10.0):
    mesh = inputs.jittered_mesh(n, n, 10.0, 10.0, seed=1002)
    U0 = inputs.cell_average(mesh, inputs.isentropic_vortex)
    t = teno.Teno(device=0).load(mesh)
    t.precompute_stencils(order=5, n_var=4, flux=teno.FLUX_HLL, precision=precision)
    t.set_state(U0)
    dt = t.cfl_dt()
    steps = int(np.ceil(t_end / dt))
    t.rk3_steps(steps, t_end / steps)
    t.check_state()
    U = t.get_state()
    area, _ = _areas(mesh)
    return mesh, U0, U, float(np.sum(area * np.abs(U[0] - U0[0])) / np.sum(area))


def test_vortex_one_period(env):
    torch, teno, _ = env
    errs = {}
    for n in (128, 256):
        _, _, U64, e64 = _run_vortex(torch, teno, n, teno.FP64)
        _, _, Umx, emx = _run_vortex(torch, teno, n, teno.FP32_MIXED)
        errs[n] = e64
        diff = float(np.abs(Umx[0] - U64[0]).mean())
        print(f"vortex {2 * n * n} cells: L1(rho) FP64 {e64:.3e}, mixed {emx:.3e}, "
              f"mean |mixed - FP64| {diff:.2e}")
        assert abs(emx - e64) <= max(0.25 * e64, 1e-6)
    rate = np.log2(errs[128] / errs[256])
    print(f"L1 rate 128^2 -> 256^2 quads: {rate:.2f}")
    assert errs[256] < errs[128] and rate > 3.0


def _adjoint_setup(env, linear):
    torch, teno, ag = env
    mesh = inputs.jittered_mesh(256, 256, 10.0, 10.0, seed=1004)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    area, cen = _areas(mesh)
    inside = (cen[:, 0] >= 4) & (cen[:, 0] <= 6) & (cen[:, 1] >= 4) & (cen[:, 1] <= 6)
    wm = torch.from_numpy(inside * area).cuda()
    t = teno.Teno(device=0).load(mesh)
    t.precompute_stencils(order=5, n_var=4, flux=teno.FLUX_HLL, linear=int(linear))
    dt, n = 0.005, 200

    def J(U0):
        out = ag.trajectory(U0, t, dt, n, checkpoint_every=20)
        return (wm * out[0] ** 2).sum()

    Ud = torch.from_numpy(U).cuda().requires_grad_(True)
    J(Ud).backward()
    grad = Ud.grad.detach()
    t.check_state()
    scale = torch.from_numpy(np.abs(U).max(axis=1, keepdims=True)).cuda()
    return mesh, U, wm, t, dt, n, J, grad, scale


def _adjoint_fd(env, linear, n_dirs):
    torch, teno, ag = env
    mesh, U, wm, t, dt, n, J, grad, scale = _adjoint_setup(env, linear)
    errs = []
    with torch.no_grad():
        Ub = torch.from_numpy(U).cuda()
        for d in inputs.random_directions(3000, n_dirs, U.size):
            v = torch.from_numpy(d.reshape(U.shape)).cuda() * scale
            eps = 1e-6
            fd = (J(Ub + eps * v) - J(Ub - eps * v)).item() / (2 * eps)
            errs.append(abs(fd - (grad * v).sum().item()) / max(abs(fd), 1e-30))
    return np.array(errs)


def test_adjoint_config_full(env):
    """Linear scheme (large stencil everywhere, a differentiable map): the
    checkpointed adjoint of 200 steps on 131,072 cells against central FD on 50
    seeded cell-wise random directions."""
    errs = _adjoint_fd(env, linear=True, n_dirs=50)
    print("adjoint config, linear scheme: FD relative errors median %.2e max %.2e"
          % (np.median(errs), errs.max()))
    assert np.median(errs) < 1e-5 and (errs < 1e-4).mean() >= 0.9


def test_adjoint_config_teno_selection_masks(env):
    """TENO scheme: the checkpointed adjoint of 200 steps on 131,072 cells
    (frozen selections) against central FD (eps = 1e-6) along 12 seeded
    smooth directions (low-wavenumber Fourier modes per variable).  The
    selection of every one of the 600 stages is recorded in the unperturbed
    run and in both perturbed runs; FD equals the derivative only where no
    selection flips under +-eps v, so the masks are compared stage by stage.
    Cell-wise random directions roughen the nearly uniform far field at the
    scale of eps, where the smoothness indicators are ~eps = 1e-12, and flip
    selections there; smooth directions do not."""
    torch, teno, ag = env
    mesh, U, wm, t, dt, n, J, grad, scale = _adjoint_setup(env, False)
    probe = teno.Teno(device=0).load(mesh)
    probe.precompute_stencils(order=5, n_var=4, flux=teno.FLUX_HLL)
    R = torch.empty((4, mesh.n_cell), dtype=torch.float64, device="cuda")

    def run(U0, record=None, compare=None):
        """J(U0) by plain steps, with each stage's selection recorded or
        compared with a recorded run (returns the flip count)"""
        t.set_state(U0)
        Un, U1, U2 = (torch.empty_like(U0) for _ in range(3))
        flips = torch.zeros((), dtype=torch.int64, device="cuda")
        for s in range(n):
            t.get_state(Un)
            t.rk3_step(dt, sync=False)
            t.stage_state(1, U1)
            t.stage_state(2, U2)
            for k, Us in enumerate((Un, U1, U2)):
                sel = torch.empty((4, mesh.n_cell), dtype=torch.uint8, device="cuda")
                probe.set_state(Us)
                probe.residual(out=R, sel=sel)
                if record is not None:
                    record.append(sel)
                else:
                    flips += (sel != compare[3 * s + k]).sum()
        out = torch.empty_like(U0)
        t.get_state(out)
        return (wm * out[0] ** 2).sum().item(), int(flips.item())

    with torch.no_grad():
        Ub = torch.from_numpy(U).cuda()
        base = []
        run(Ub, record=base)
        res = []
        for d in inputs.smooth_directions(3000, 12, mesh, 4):
            v = torch.from_numpy(d).cuda() * scale
            eps = 1e-6
            Jp, fp = run(Ub + eps * v, compare=base)
            Jm, fm = run(Ub - eps * v, compare=base)
            fd = (Jp - Jm) / (2 * eps)
            res.append((fp + fm, abs(fd - (grad * v).sum().item()) / max(abs(fd), 1e-30)))
    res = np.array(res)
    clean = res[:, 0] == 0
    print("adjoint config, TENO: %d of %d smooth directions without a selection flip; "
          "FD relative errors there median %.2e max %.2e"
          % (clean.sum(), len(res), np.median(res[clean, 1]), res[clean, 1].max()))
    assert clean.sum() >= 10
    assert res[clean, 1].max() < 1e-8


def test_solid_body_rotation_one_turn(env):
    """Solid-body rotation (Sec. 5): the three bodies advected by
    v = (0.5 - y, x - 0.5) for one turn (t = 2 pi) on 14,792 jittered
    triangles of the periodic unit square (the paper: 14,860 with h = 1/80),
    scalar upwind flux, CFL 0.4.  The rotation is tapered to zero between
    r = 0.45 and 0.5 (the bodies stay within r = 0.4), which makes the field
    periodic; the untapered field jumps across the periodic seam, where it is
    not divergence-free in the discrete sense and small tails grow there.
    Mass is conserved to rounding, the solution stays bounded, the L1
    distance to the initial field (the exact solution) falls from TENO3 to
    TENO5/6, and the FP32-mixed run stays close to the FP64 one."""
    torch, teno, _ = env
    mesh = inputs.jittered_mesh(86, 86, 1.0, 1.0, seed=1006)
    U0 = inputs.cell_average(mesh, inputs.solid_bodies)
    area, _ = _areas(mesh)
    res = {}
    for order, prec in [(3, teno.FP64), (5, teno.FP64), (6, teno.FP64), (5, teno.FP32_MIXED)]:
        t = teno.Teno(device=0).load(mesh)
        t.precompute_stencils(order=order, n_var=1, flux=teno.FLUX_UPWIND, precision=prec,
                              rotation=(0.5, 0.5, 1.0, 0.45, 0.5), cfl=0.4)
        t.set_state(U0)
        dt = t.cfl_dt()
        n = int(np.ceil(2 * np.pi / dt))
        t.rk3_steps(n, 2 * np.pi / n)
        t.check_state()
        U = t.get_state()
        m0, m1 = float(np.sum(area * U0[0])), float(np.sum(area * U[0]))
        assert abs(m1 - m0) <= 1e-12 * abs(m0)
        assert U.min() > -0.2 and U.max() < 1.2
        res[(order, prec)] = (U, float(np.sum(area * np.abs(U[0] - U0[0])) / np.sum(area)))
        print(f"rotation TENO{order} precision {prec}: {n} steps, L1 {res[(order, prec)][1]:.4e}, "
              f"min {U.min():.3e} max {U.max():.3e}")
    e3, e5, e6 = (res[(o, teno.FP64)][1] for o in (3, 5, 6))
    assert e5 < e3 and e6 < e3
    d = float(np.abs(res[(5, teno.FP32_MIXED)][0] - res[(5, teno.FP64)][0]).mean())
    print(f"mean |mixed - FP64| TENO5: {d:.2e}")
    assert d < 1e-3


def test_dmr_initial_residual(env, oracle_mod):
    """Shock case (Sec. 5, DMR) on 1024x256 jittered quads of [0,4]x[0,1] =
    524,288 triangles with its four boundary conditions, TENO6, HLLC, at the
    initial state: the FP64 residual against the oracle on 1,000 sampled cells
    (the few cells whose Gauss states are non-physical give NaN on both sides,
    and the sets must agree), the selection-flip rate of the FP32-mixed path
    against FP64, and the residual throughput of both paths.  Without the
    positivity option some Gauss states at the incident front are non-physical
    (negative pressure from the directional quadratics across the 116:1
    jump), so the time run uses the option (test_dmr_time_run)."""
    torch, teno, _ = env
    mesh = inputs.jittered_mesh(1024, 256, 4.0, 1.0, seed=1003, periodic=False,
                                bc_tagger=inputs.dmr_bc_tagger)
    U = inputs.cell_average(mesh, inputs.dmr_state, n_quad=3)
    out = {}
    for prec in (teno.FP64, teno.FP32_MIXED):
        t = teno.Teno(device=0).load(mesh)
        t.precompute_stencils(order=6, n_var=4, flux=teno.FLUX_HLLC, precision=prec)
        Ud = torch.from_numpy(U).cuda()
        t.set_state(Ud)
        R, sel = t.residual(want_sel=True)
        Rd = torch.empty_like(Ud)
        for _ in range(3):
            t.residual(out=Rd)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            t.residual(out=Rd)
        e1.record()
        torch.cuda.synchronize()
        rate = 20 * mesh.n_cell / (e0.elapsed_time(e1) / 1e3)
        out[prec] = (R, sel, rate)
        t.close()
    R64, sel64, r64 = out[teno.FP64]
    Rmx, selmx, rmx = out[teno.FP32_MIXED]
    flips = float((sel64 != selmx).mean())
    bad = ~np.isfinite(R64).all(axis=0)
    print(f"DMR t=0, 524,288 cells, TENO6 HLLC: residual {r64:.3e} cell-stage/s (FP64), "
          f"{rmx:.3e} (mixed); mixed/FP64 selection flips {flips:.2e}; "
          f"non-finite residual cells {int(bad.sum())}")
    assert flips < 1e-2
    o = oracle_mod.Oracle(mesh, order=6, n_var=4, flux=2)
    cells = np.random.default_rng(11).choice(mesh.n_cell, 1000, replace=False)
    Ro, selo, mg = o.residual_cells(U, cells)
    Rg = R64[:, cells].T
    fin_o, fin_g = np.isfinite(Ro).all(axis=1), np.isfinite(Rg).all(axis=1)
    assert np.array_equal(fin_o, fin_g)
    ok = np.all((sel64[:, cells].T == selo) | (mg <= 1e-10), axis=1)
    assert ok.all()
    scale = np.abs(R64[:, ~bad]).max()
    assert np.abs(Rg[fin_g] - Ro[fin_g]).max() / scale <= 1e-11


def _flip_probe(teno, mesh, order, flux):
    """FP64 and FP32-mixed contexts that evaluate the selection of a given
    state (the flip rate compares the two on the same input state)."""
    probes = []
    for prec in (teno.FP64, teno.FP32_MIXED):
        p = teno.Teno(device=0).load(mesh)
        p.precompute_stencils(order=order, n_var=4, flux=flux, precision=prec, positivity=1)
        probes.append(p)
    return probes


def _stage_flips(torch, probes, states, time):
    """Fraction of (cell, variable) selections of the mixed path that differ
    from the FP64 path, per stage input state."""
    out = []
    for Us in states:
        sels = []
        for p in probes:
            p.set_time(time)
            p.set_state(Us)
            R = torch.empty_like(Us)
            sel = torch.empty(Us.shape, dtype=torch.uint8, device="cuda")
            p.residual(out=R, sel=sel)
            sels.append(sel)
        out.append(float((sels[0] != sels[1]).double().mean().item()))
    return out


def test_dmr_time_run(env, oracle_mod):
    """Shock case (Sec. 5, DMR) as a time run to t = 0.2 on 64x16 jittered
    quads (2,048 triangles), TENO6, HLLC, CFL 0.4, positivity scaling on, in
    FP64 and FP32-mixed.  Both runs stay physical.  At every stage of the FP64
    run the FP32-mixed selection on the same state differs from the FP64 one
    in under 1 % of (cell, variable) pairs.  The oracle runs the same steps;
    every 20th state of its run is checked against the library's residual
    (the parity rules of the positivity test: 1e-11 away from Gauss points held
    at the pressure floor).  The two trajectories themselves part at the
    rounding level where the floor and the cutoff margin decide, so their end
    states are compared only loosely."""
    from test_gpu_parity import FLOOR_TOL, TOL, positivity_parity
    torch, teno, _ = env
    mesh = inputs.jittered_mesh(64, 16, 4.0, 1.0, seed=1003, periodic=False,
                                bc_tagger=inputs.dmr_bc_tagger)
    U0 = inputs.cell_average(mesh, inputs.dmr_state)
    order, flux, t_end = 6, teno.FLUX_HLLC, 0.2
    runs = {}
    probes = _flip_probe(teno, mesh, order, flux)
    flips = []
    for prec in (teno.FP64, teno.FP32_MIXED):
        t = teno.Teno(device=0).load(mesh)
        t.precompute_stencils(order=order, n_var=4, flux=flux, precision=prec, positivity=1)
        Ud = torch.from_numpy(U0).cuda()
        t.set_state(Ud)
        time, n, dts = 0.0, 0, []
        while time < t_end - 1e-14:
            dt = min(t.cfl_dt(), t_end - time)
            if prec == teno.FP64:
                Un = torch.empty_like(Ud)
                t.get_state(Un)
            t.rk3_step(dt)
            if prec == teno.FP64:
                U1, U2 = t.stage_state(1, torch.empty_like(Ud)), t.stage_state(2, torch.empty_like(Ud))
                flips.append(_stage_flips(torch, probes, (Un, U1, U2), time))
            time += dt
            n += 1
            dts.append(dt)
        t.check_state()
        U = t.get_state()
        rho = U[0]
        p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
        assert np.isfinite(U).all() and rho.min() > 0 and p.min() > 0
        runs[prec] = (U, n, np.array(dts))
    flips = np.array(flips)
    U64, n64, dts64 = runs[teno.FP64]
    Umx, nmx, _ = runs[teno.FP32_MIXED]
    # the oracle's run with the FP64 run's steps, and parity along it
    o = oracle_mod.Oracle(mesh, order=order, n_var=4, flux=flux, positivity=True)
    tp = teno.Teno(device=0).load(mesh)
    tp.precompute_stencils(order=order, n_var=4, flux=flux, precision=teno.FP64, positivity=1)
    Uo, time, worst = U0.copy(), 0.0, (0.0, 0.0)
    for k, dt in enumerate(dts64):
        if k % 20 == 0:
            far, at, _ = positivity_parity(tp, o, Uo, time, 0)
            worst = (max(worst[0], far), max(worst[1], at))
        Uo = o.rk3_step(Uo, dt, time=time)
        time += dt
    d_or = float(np.abs(U64[0] - Uo[0]).mean() / np.abs(Uo[0]).mean())
    d_mx = float(np.abs(Umx[0] - U64[0]).mean() / np.abs(U64[0]).mean())
    print(f"DMR 2,048 cells TENO6 HLLC to t = 0.2: FP64 {n64} steps, mixed {nmx} steps; "
          f"residual parity along the oracle run {worst[0]:.2e} (next to floor cells "
          f"{worst[1]:.2e}); end states: mean |rho_fp64 - rho_oracle| / mean rho {d_or:.2e}, "
          f"mixed vs FP64 {d_mx:.2e}; flip rate per stage: mean {flips.mean():.2e}, "
          f"max {flips.max():.2e}")
    assert worst[0] <= TOL and worst[1] <= FLOOR_TOL
    assert flips.max() < 1e-2
    assert d_or < 1e-2 and d_mx < 5e-2
