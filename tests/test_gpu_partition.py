"""Partitioned meshes on one GPU: P = 2 and 4 parts of one mesh, each a
context with its own device buffers, driven in one process with the
copy-based halo exchange after every RK stage (teno_group_rk3_step) and the
reverse exchange of the adjoint (teno_group_residual_vjp).  Every part uses
the whole mesh's stencils, matrices, slot order and face orientation, so its
owned cells' residual and RK3 update must equal the whole-mesh results bit
for bit; the VJP sums the same terms in another order (equal to rounding)."""
import numpy as np
import pytest

from paper_2105_02127_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_02127_gb300 import build, teno
    build.build()
    teno.lib()
    return teno


def _blast(mesh):
    def f(x, y):
        inside = (np.abs(x - 5.0) < 2.0) & (np.abs(y - 5.0) < 2.0)
        return inputs.prim_to_cons(np.where(inside, 1.0, 0.5), 0.3 * np.ones_like(x),
                                   -0.2 * np.ones_like(x), np.where(inside, 1.0, 0.7), 1.4)
    return inputs.cell_average(mesh, f)


def _contexts(T, mesh, P, **kw):
    whole = T.Teno(device=0).load(mesh)
    whole.precompute_stencils(**kw)
    parts = [T.Teno(device=0).load(mesh).precompute_partition(P, p, **kw) for p in range(P)]
    return whole, parts


def _assemble(parts, arrays, n_var, n_cell):
    out = np.full((n_var, n_cell), np.nan)
    for t, a in zip(parts, arrays):
        out[:, t.partition_cells()] = a
    return out


@pytest.mark.parametrize("P", [2, 4])
@pytest.mark.parametrize("precision", [0, 2, 1], ids=["pairs", "native", "mixed"])
@pytest.mark.parametrize("order,flux", [(5, 1), (6, 2)])
def test_partitioned_steps_bit_equal(T, P, precision, order, flux):
    """Residual, selections and three SSP-RK3 steps at the CFL step of the
    parts equal the whole mesh's, bit for bit (discontinuous periodic state:
    directional stencils in use)."""
    mesh = inputs.jittered_mesh(40, 40, 10.0, 10.0, seed=1007)
    U = _blast(mesh)
    kw = dict(order=order, n_var=4, flux=flux, precision=precision)
    whole, parts = _contexts(T, mesh, P, **kw)
    whole.set_state(U)
    for t in parts:
        t.set_state(U)
    R, sel = whole.residual(want_sel=True)
    res = [t.residual(want_sel=True) for t in parts]
    assert np.array_equal(_assemble(parts, [r for r, _ in res], 4, mesh.n_cell), R)
    assert np.array_equal(_assemble(parts, [s for _, s in res], 4, mesh.n_cell), sel)
    for _ in range(3):
        dt_w = whole.rk3_step(0.0)
        dt_p = T.group_rk3_step(parts, 0.0)
        assert dt_p == dt_w
    Uw = whole.get_state()
    Up = _assemble(parts, [t.get_state() for t in parts], 4, mesh.n_cell)
    assert np.array_equal(Up, Uw)
    for t in parts:
        t.check_state()


@pytest.mark.parametrize("P", [2, 4])
@pytest.mark.parametrize("precision", [0, 2], ids=["pairs", "native"])
def test_partitioned_vjp(T, P, precision):
    """The residual VJP (frozen selection) with the reverse halo exchange
    equals the whole mesh's to rounding."""
    mesh = inputs.jittered_mesh(40, 40, 10.0, 10.0, seed=1007)
    U = _blast(mesh)
    whole, parts = _contexts(T, mesh, P, order=5, n_var=4, flux=1, precision=precision)
    whole.set_state(U)
    for t in parts:
        t.set_state(U)
    w = inputs.random_directions(3005, 1, U.size)[0].reshape(U.shape)
    v = whole.residual_vjp(w)
    vp = T.group_residual_vjp(parts, w)
    err = np.abs(vp - v).max(axis=1) / np.abs(v).max(axis=1)
    print(f"partitioned VJP P={P} precision {precision}: per-variable rel err {err.max():.2e}")
    assert err.max() <= 1e-13


@pytest.mark.parametrize("P", [2, 3])
def test_partitioned_vjp_boundaries(T, P):
    """The residual VJP on the shock-case boundaries (wall, inflow, outflow
    layer, moving top state) on a smooth state, HLL: the parts with the
    reverse halo exchange equal the whole mesh to rounding."""
    mesh = inputs.jittered_mesh(48, 12, 4.0, 1.0, seed=1003, periodic=False,
                                bc_tagger=inputs.dmr_bc_tagger)

    def f(x, y):
        return inputs.prim_to_cons(1.4 + 0.3 * np.sin(3 * x + 2 * y), 0.2 + 0.1 * np.cos(2 * y),
                                   -0.1 + 0.05 * x, 1.0 + 0.2 * np.sin(x * y), 1.4)
    U = inputs.cell_average(mesh, f)
    whole, parts = _contexts(T, mesh, P, order=4, n_var=4, flux=1)
    for t in [whole] + parts:
        t.set_time(0.05)
        t.set_state(U)
    w = inputs.random_directions(3006, 1, U.size)[0].reshape(U.shape)
    v = whole.residual_vjp(w)
    vp = T.group_residual_vjp(parts, w)
    err = np.abs(vp - v).max(axis=1) / np.abs(v).max(axis=1)
    assert err.max() <= 1e-13


def test_partitioned_shock_case(T):
    """Shock-case geometry (non-periodic, the four boundary conditions, the
    time-dependent top state), TENO6, HLLC, positivity scaling: two parts step
    bit for bit with the whole mesh for ten CFL steps."""
    mesh = inputs.jittered_mesh(64, 16, 4.0, 1.0, seed=1003, periodic=False,
                                bc_tagger=inputs.dmr_bc_tagger)
    U = inputs.cell_average(mesh, inputs.dmr_state)
    kw = dict(order=6, n_var=4, flux=2, positivity=1)
    whole, parts = _contexts(T, mesh, 2, **kw)
    whole.set_state(U)
    for t in parts:
        t.set_state(U)
    for _ in range(10):
        assert T.group_rk3_step(parts, 0.0) == whole.rk3_step(0.0)
    Up = _assemble(parts, [t.get_state() for t in parts], 4, mesh.n_cell)
    assert np.array_equal(Up, whole.get_state())


def test_partition_refusals(T):
    mesh = inputs.jittered_mesh(24, 24, 10.0, 10.0, seed=1002)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    t = T.Teno(device=0).load(mesh).precompute_partition(2, 0, order=3, n_var=4, flux=1)
    t.set_state(U)
    for call in (lambda: t.rk3_step(0.01), lambda: t.residual_vjp(np.zeros_like(U)),
                 lambda: t.adjoint_step(0.01, np.zeros_like(U))):
        with pytest.raises(T.TenoError) as e:
            call()
        assert e.value.code == T.TENO_EINVAL
