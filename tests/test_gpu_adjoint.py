"""GPU tests of the differentiable RK3 loop (torch.autograd over libteno's
discrete adjoint with RK-state checkpointing).

- one step: TenoStep.backward against the oracle's SSP-RK3 adjoint;
- a checkpointed trajectory (segments shorter than the run, a ragged last
  segment) against the chained oracle adjoint on the oracle's own forward
  states;
- the vortex objective J = sum over cells with centroid in [4,6]^2 of
  |V| rho^2 at the final time, gradient w.r.t. the initial state, against
  central finite differences (eps = 1e-6) along seeded directions.
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


def _solver(teno, mesh, order=5):
    t = teno.Teno(device=0).load(mesh)
    t.precompute_stencils(order=order, n_var=4, flux=teno.FLUX_HLL)
    return t


def test_step_backward_vs_oracle(env, oracle_mod):
    torch, teno, ag = env
    mesh = inputs.jittered_mesh(14, 13, 10.0, 10.0, seed=1004)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    t = _solver(teno, mesh)
    Ud = torch.from_numpy(U).cuda().requires_grad_(True)
    out = ag.TenoStep.apply(Ud, t, 0.02)
    g = torch.from_numpy(inputs.random_directions(3001, 1, U.size)[0].reshape(U.shape)).cuda()
    (out * g).sum().backward()
    o = oracle_mod.Oracle(mesh, order=5, n_var=4, flux=1)
    ref = o.rk3_vjp(U, g.cpu().numpy(), 0.02)
    assert np.abs(Ud.grad.cpu().numpy() - ref).max() / np.abs(ref).max() <= 1e-10
    assert np.abs(out.detach().cpu().numpy() - o.rk3_step(U, 0.02)).max() <= 1e-11 * np.abs(U).max()


def test_checkpointed_trajectory_vs_oracle(env, oracle_mod):
    torch, teno, ag = env
    mesh = inputs.jittered_mesh(12, 12, 10.0, 10.0, seed=1005)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    t = _solver(teno, mesh)
    dt, n = 0.03, 7
    Ud = torch.from_numpy(U).cuda().requires_grad_(True)
    out = ag.trajectory(Ud, t, dt, n, checkpoint_every=3)
    g = inputs.random_directions(3002, 1, U.size)[0].reshape(U.shape)
    (out * torch.from_numpy(g).cuda()).sum().backward()
    o = oracle_mod.Oracle(mesh, order=5, n_var=4, flux=1)
    states = [U]
    for _ in range(n):
        states.append(o.rk3_step(states[-1], dt))
    assert np.abs(out.detach().cpu().numpy() - states[-1]).max() <= 1e-11 * np.abs(U).max()
    lam = g
    for k in range(n - 1, -1, -1):
        lam = o.rk3_vjp(states[k], lam, dt)
    assert np.abs(Ud.grad.cpu().numpy() - lam).max() / np.abs(lam).max() <= 1e-10


def test_vortex_objective_gradient_vs_fd(env):
    """Config-4 shape at reduced size (64^2 quads, 40 steps of dt = 0.005,
    checkpoint every 10): adjoint gradient vs central FD along 10 seeded
    directions."""
    torch, teno, ag = env
    mesh = inputs.jittered_mesh(64, 64, 10.0, 10.0, seed=1004)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    V = mesh.unwrapped_vertices()
    cen = V.mean(axis=1)
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    wmask = ((cen[:, 0] >= 4) & (cen[:, 0] <= 6) & (cen[:, 1] >= 4) & (cen[:, 1] <= 6)) * area
    wm = torch.from_numpy(wmask).cuda()
    t = _solver(teno, mesh)
    dt, n = 0.005, 40

    def J(U0):
        out = ag.trajectory(U0, t, dt, n, checkpoint_every=10)
        return (wm * out[0] ** 2).sum()

    Ud = torch.from_numpy(U).cuda().requires_grad_(True)
    J(Ud).backward()
    grad = Ud.grad.detach()
    dirs = inputs.random_directions(3000, 10, U.size)
    errs = []
    with torch.no_grad():
        for d in dirs:
            v = torch.from_numpy(d.reshape(U.shape)).cuda() * torch.from_numpy(
                np.abs(U).max(axis=1, keepdims=True)).cuda()
            eps = 1e-6
            Up = torch.from_numpy(U).cuda() + eps * v
            Um = torch.from_numpy(U).cuda() - eps * v
            fd = (J(Up) - J(Um)).item() / (2 * eps)
            adj = (grad * v).sum().item()
            errs.append(abs(fd - adj) / max(abs(fd), 1e-30))
    errs = np.array(errs)
    print("FD relative errors:", np.array2string(errs, precision=2))
    assert np.median(errs) < 1e-5 and (errs < 1e-4).mean() >= 0.8


@pytest.mark.parametrize("precision,order,flux", [(0, 5, 1), (0, 6, 2), (2, 5, 1)],
                         ids=["pairs-teno5", "pairs-teno6-hllc", "native-teno5"])
def test_tape_adjoint_equals_replayed_adjoint(env, precision, order, flux):
    """The adjoint of recorded steps (teno_adjoint_step_tape: no
    reconstruction) is the same bits as teno_adjoint_step, which replays the
    step's stages from its initial state."""
    torch, teno, ag = env
    mesh = inputs.jittered_mesh(17, 16, 10.0, 10.0, seed=1005)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    t = teno.Teno(device=0).load(mesh)
    t.precompute_stencils(order=order, n_var=4, flux=flux, precision=precision)
    dt = 0.02
    t.set_state(U)
    t.tape_reserve(3)
    states = []
    for k in range(3):
        states.append(t.get_state())
        t.rk3_step_record(k, dt)
    end = t.get_state()
    lam = inputs.random_directions(3006, 1, U.size)[0].reshape(U.shape)
    taped, l = [], lam
    for k in (2, 1, 0):
        l = t.adjoint_step_tape(k, l)
        taped.append(l)
    assert np.array_equal(t.get_state(), end)  # the taped adjoint leaves the state alone
    ref, l = [], lam
    for k in (2, 1, 0):
        t.set_state(states[k])
        l = t.adjoint_step(dt, l)
        ref.append(l)
    for a, b in zip(taped, ref):
        assert np.array_equal(a, b)
    # the recorded forward steps are the plain steps
    t.set_state(U)
    for _ in range(3):
        t.rk3_step(dt)
    assert np.array_equal(t.get_state(), end)
    t.tape_reserve(0)
