"""teno_cfl_dt_noalloc: the CFL step for callers that cannot allocate device
memory (a framework's caching allocator owns the GPU, a fixed device-memory
budget, no allocation-induced synchronisation allowed).  It must give the
same step as the allocating entry point teno_cfl_dt, call after call: the
scratch it uses is one device array shared by all calls, which keeps the last
call's contents.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2105_02127_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-13  # both sides take an exact maximum; only the per-cell lengths may round differently


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_02127_gb300 import build, teno
    build.build()
    teno.lib()
    return torch, teno


def _cell_len(mesh):
    V = mesh.unwrapped_vertices()
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    perim = sum(np.hypot(*(V[:, (k + 1) % 3] - V[:, k]).T) for k in range(3))
    return 4.0 * area / perim


def test_noalloc_matches_allocating_entry_point(env):
    torch, teno = env
    mesh = inputs.jittered_mesh(61, 37, 10.0, 10.0, seed=1018)  # 4,514 cells: ragged last block
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    t = teno.Teno(device=0).load(mesh)
    t.precompute_stencils(order=3, n_var=4, flux=teno.FLUX_HLL, cfl=0.4)
    lens = torch.from_numpy(_cell_len(mesh)).cuda()
    states = [U, U * np.array([1.0, 1.3, -0.7, 1.2])[:, None]]  # two different states
    for k, Uk in enumerate(states):
        t.set_state(Uk)
        ref = t.cfl_dt()
        Ud = torch.from_numpy(np.ascontiguousarray(Uk)).cuda()
        got_host = teno.cfl_dt_noalloc(Ud, lens, gamma=1.4, cfl=0.4)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        teno.cfl_dt_noalloc(Ud, lens, dt_out=out, gamma=1.4, cfl=0.4)
        torch.cuda.synchronize()
        got_dev = float(out.item())
        assert abs(got_host - ref) <= RTOL * ref, (k, got_host, ref)
        assert abs(got_dev - ref) <= RTOL * ref, (k, got_dev, ref)
    # scalar advection: the speed is |a| everywhere
    t1 = teno.Teno(device=0).load(mesh)
    t1.precompute_stencils(order=3, n_var=1, flux=teno.FLUX_UPWIND, cfl=0.3, adv=(1.0, 1.0))
    u = inputs.cell_average(mesh, inputs.advection_sine)
    t1.set_state(u)
    ref = t1.cfl_dt()
    for _ in range(2):
        got = teno.cfl_dt_noalloc(torch.from_numpy(u).cuda(), lens, adv=(1.0, 1.0), cfl=0.3)
        assert abs(got - ref) <= RTOL * ref


def test_noalloc_many_blocks_and_no_allocation(env):
    """605,000 cells = 296 partial maxima (more than one per thread of the
    final reduction block), two calls in a row against the allocating entry
    point; after a first call (which loads the kernels), further calls leave
    the device's free memory unchanged."""
    torch, teno = env
    mesh = inputs.jittered_mesh(550, 550, 10.0, 10.0, seed=1020)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex, n_quad=3)
    t = teno.Teno(device=0).load(mesh)
    t.precompute_stencils(order=3, n_var=4, flux=teno.FLUX_HLL, cfl=0.4)
    t.set_state(U)
    ref = t.cfl_dt()
    Ud = torch.from_numpy(U).cuda()
    lens = torch.from_numpy(_cell_len(mesh)).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    got = teno.cfl_dt_noalloc(Ud, lens, gamma=1.4, cfl=0.4)
    assert abs(got - ref) <= RTOL * ref
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert abs(teno.cfl_dt_noalloc(Ud, lens, gamma=1.4, cfl=0.4) - ref) <= RTOL * ref
        teno.cfl_dt_noalloc(Ud, lens, dt_out=out, gamma=1.4, cfl=0.4)
        torch.cuda.synchronize()
        assert abs(float(out.item()) - ref) <= RTOL * ref
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_nonphysical_state(env):
    """A cell with negative pressure or NaN has no CFL step: the host-result
    call returns TENO_ENONPHYS like teno_cfl_dt, the device-result call
    writes NaN."""
    torch, teno = env
    mesh = inputs.jittered_mesh(21, 17, 10.0, 10.0, seed=1021)
    U = inputs.cell_average(mesh, inputs.isentropic_vortex)
    lens = torch.from_numpy(_cell_len(mesh)).cuda()
    t = teno.Teno(device=0).load(mesh)
    t.precompute_stencils(order=3, n_var=4, flux=teno.FLUX_HLL, cfl=0.4)
    for k, val in ((3, -1.0), (0, float("nan"))):
        Ub = U.copy()
        Ub[k, 100] = val
        t.set_state(Ub)
        with pytest.raises(teno.TenoError) as e:
            t.cfl_dt()
        assert e.value.code == teno.TENO_ENONPHYS
        Ud = torch.from_numpy(Ub).cuda()
        with pytest.raises(teno.TenoError) as e:
            teno.cfl_dt_noalloc(Ud, lens, gamma=1.4, cfl=0.4)
        assert e.value.code == teno.TENO_ENONPHYS
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        teno.cfl_dt_noalloc(Ud, lens, dt_out=out, gamma=1.4, cfl=0.4)
        torch.cuda.synchronize()
        assert np.isnan(float(out.item()))
    # the same buffers give the step again once the state is physical
    Ud = torch.from_numpy(U).cuda()
    t.set_state(U)
    assert abs(teno.cfl_dt_noalloc(Ud, lens, gamma=1.4, cfl=0.4) - t.cfl_dt()) <= RTOL * t.cfl_dt()


def test_noalloc_keeps_current_device(env):
    """The call restores the calling thread's current device, also when it
    fails on a device that does not exist."""
    torch, teno = env
    import ctypes
    U = torch.ones((4, 64), dtype=torch.float64, device="cuda")
    U[3] = 2.5
    lens = torch.ones(64, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    L = teno.lib()
    stream = torch.cuda.current_stream().cuda_stream
    before = torch.cuda.current_device()
    for dev in range(torch.cuda.device_count()):
        with torch.cuda.device(dev):
            Ud, ld = U.to(f"cuda:{dev}"), lens.to(f"cuda:{dev}")
            cur = torch.cuda.current_device()
            rc = L.teno_cfl_dt_noalloc(dev, torch.cuda.current_stream().cuda_stream, 4, 64,
                                       Ud.data_ptr(), ld.data_ptr(), 1.4, 1.0, 1.0, 0.4,
                                       ctypes.addressof(out), 0)
            assert rc == teno.TENO_OK and out.value > 0
            assert torch.cuda.current_device() == cur
    rc = L.teno_cfl_dt_noalloc(torch.cuda.device_count() + 7, stream, 4, 64, U.data_ptr(),
                               lens.data_ptr(), 1.4, 1.0, 1.0, 0.4, ctypes.addressof(out), 0)
    assert rc == teno.TENO_ECUDA
    assert torch.cuda.current_device() == before
    rc = L.teno_cfl_dt_noalloc(before, stream, 4, 64, U.data_ptr(), lens.data_ptr(), 1.4, 1.0,
                               1.0, 0.4, ctypes.addressof(out), 0)
    assert rc == teno.TENO_OK


def test_noalloc_rejects_oversize(env):
    torch, teno = env
    U = torch.ones((4, 8), dtype=torch.float64, device="cuda")
    U[3] = 2.5  # rho = 1, u = v = 1, p = 0.6
    lens = torch.ones(8, dtype=torch.float64, device="cuda")
    import ctypes
    out = ctypes.c_double()
    L = teno.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # sizes are checked before anything is launched
    rc = L.teno_cfl_dt_noalloc(0, stream, 4, teno.NOALLOC_MAX_CELLS + 1, U.data_ptr(),
                               lens.data_ptr(), 1.4, 1.0, 1.0, 0.4, ctypes.addressof(out), 0)
    assert rc == teno.TENO_EINVAL
    rc = L.teno_cfl_dt_noalloc(0, stream, 4, 0, U.data_ptr(), lens.data_ptr(), 1.4, 1.0, 1.0,
                               0.4, ctypes.addressof(out), 0)
    assert rc == teno.TENO_EINVAL
    rc = L.teno_cfl_dt_noalloc(0, stream, 4, 8, U.data_ptr(), lens.data_ptr(), 1.4, 1.0, 1.0,
                               0.4, ctypes.addressof(out), 0)
    assert rc == teno.TENO_OK and out.value > 0
