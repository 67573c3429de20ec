"""Partitioned meshes on CPU ranks: two gloo ranks, each with a host-only
context of its part (no GPU).  The receive lists are exchanged at set-up
(partition.link); a halo exchange of host arrays by those lists delivers every
halo value from its owner; the CFL step reduced over the parts (partition.
cfl_dt) equals the oracle's step on the whole mesh."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _mesh_and_state():
    from paper_2105_02127_gb300 import inputs
    mesh = inputs.jittered_mesh(24, 22, 10.0, 10.0, seed=1002)
    return mesh, inputs.cell_average(mesh, inputs.isentropic_vortex)


def _cell_len(mesh):
    V = mesh.unwrapped_vertices()
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    perim = sum(np.hypot(*(V[:, (k + 1) % 3] - V[:, k]).T) for k in range(3))
    return 4.0 * area / perim


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2105_02127_gb300 import partition, teno
    mesh, U = _mesh_and_state()
    t = teno.Teno(device=-1).load(mesh)
    t.precompute_partition(world, rank, order=5, n_var=4, flux=teno.FLUX_HLL)
    partition.link(t, rank, world)
    owned = t.partition_cells()
    _, _, recv, send = t.partition_sizes()
    # every rank holds its own version of the state on its owned cells
    Ur = U + 0.01 * (rank + 1)
    # halo exchange of host arrays by the library's lists
    peer = 1 - rank
    # the cells the peer receives from this rank: its receive list, declared here
    send_ids = t.send_users[peer]
    assert set(send_ids.tolist()) <= set(owned.tolist())
    sbuf = torch.from_numpy(np.ascontiguousarray(Ur[:, send_ids]))
    rbuf = torch.empty((4, int(recv[peer])), dtype=torch.float64)
    ops = [dist.P2POp(dist.isend, sbuf, peer), dist.P2POp(dist.irecv, rbuf, peer)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()
    recv_ids = t.partition_recv_cells(peer)
    expect = U[:, recv_ids] + 0.01 * (peer + 1)  # the owner's values
    ok_halo = bool(np.array_equal(rbuf.numpy(), expect)) and int(send[peer]) == sbuf.shape[1]
    # the CFL step: largest speed over the owned cells, reduced over the ranks
    L = _cell_len(mesh)[owned]
    rho, mx, my, E = U[:, owned]
    u, v = mx / rho, my / rho
    p = 0.4 * (E - 0.5 * rho * (u * u + v * v))
    lam = float(np.max((np.hypot(u, v) + np.sqrt(1.4 * p / rho)) / L))
    dt = partition.cfl_dt(lam, 0.4)
    out[rank] = (ok_halo, dt, len(owned), int(recv[peer]), len(send_ids))
    dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_rank_halo_lists_and_cfl_reduction(oracle_mod):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(170)
        assert p.exitcode == 0
    mesh, U = _mesh_and_state()
    dt_or = oracle_mod.Oracle(mesh, order=5, n_var=4, flux=1).cfl_dt(U, 0.4)
    for r in range(2):
        ok, dt, n_own, n_recv, _ = out[r]
        assert ok
        assert n_recv > 0
        assert dt == pytest.approx(dt_or, rel=1e-14)
    assert out[0][2] + out[1][2] == mesh.n_cell
