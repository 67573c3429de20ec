"""Partitioned meshes across processes: one rank per part.

Host logic around the library's partition entry points (teno_precompute_
partition and friends): the exchange of receive lists at set-up, the halo
exchange of a stage (pack on the owner, send, receive, unpack), the CFL step
reduced over all parts, and an SSP-RK3 step with an exchange after every
stage.  The communicator is torch.distributed (NCCL between GPUs; the list
and reduction logic also runs over gloo on CPU ranks).  Within one process,
teno_group_rk3_step and teno_group_residual_vjp drive several parts on one
GPU with device-to-device copies instead.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def link(t, rank: int, world: int) -> None:
    """Tell every peer which of its cells this rank receives, and declare the
    cells each peer receives from this rank (t.partition_set_send)."""
    mine = {q: torch.from_numpy(t.partition_recv_cells(q).astype(np.int64))
            for q in range(world) if q != rank}
    counts_out = {q: torch.tensor([len(mine[q])], dtype=torch.int64) for q in mine}
    counts_in = {q: torch.zeros(1, dtype=torch.int64) for q in mine}
    ops = []
    for q in mine:
        ops.append(dist.P2POp(dist.isend, counts_out[q], q))
        ops.append(dist.P2POp(dist.irecv, counts_in[q], q))
    for w in dist.batch_isend_irecv(ops):
        w.wait()
    theirs = {q: torch.zeros(int(counts_in[q].item()), dtype=torch.int64) for q in mine}
    ops = []
    for q in mine:
        if len(mine[q]):
            ops.append(dist.P2POp(dist.isend, mine[q], q))
        if len(theirs[q]):
            ops.append(dist.P2POp(dist.irecv, theirs[q], q))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()
    t.send_users = {}
    for q in mine:
        t.send_users[q] = theirs[q].numpy().astype(np.int32)
        t.partition_set_send(q, t.send_users[q])


def exchange(t, what: int, rank: int, world: int) -> None:
    """Halo exchange of state `what` (0 U^n, 1 U^(1), 2 U^(2)) with every
    peer: pack the cells each peer receives, send, receive, unpack."""
    _, _, recv, send = t.partition_sizes()
    nv = t.n_var
    out = {q: torch.empty((nv, int(send[q])), dtype=torch.float64, device="cuda")
           for q in range(world) if q != rank and send[q]}
    inb = {q: torch.empty((nv, int(recv[q])), dtype=torch.float64, device="cuda")
           for q in range(world) if q != rank and recv[q]}
    for q, b in out.items():
        t.halo_pack(q, what, b)
    torch.cuda.current_stream().synchronize()
    ops = [dist.P2POp(dist.isend, b, q) for q, b in out.items()]
    ops += [dist.P2POp(dist.irecv, b, q) for q, b in inb.items()]
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()
    for q, b in inb.items():
        t.halo_unpack(q, what, b)


def max_over_ranks(x: float) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    v = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def cfl_dt(local_max_speed: float, cfl: float) -> float:
    """The CFL step of the whole mesh: cfl over the largest speed of all parts."""
    return cfl / max_over_ranks(local_max_speed)


def rk3_step(t, rank: int, world: int, dt: float = 0.0) -> float:
    """One SSP-RK3 step of this rank's part: the CFL step reduced over all
    parts when dt <= 0, and a halo exchange after every stage."""
    if dt <= 0.0:
        dt = cfl_dt(t.local_max_speed(), t.params.cfl)
    for stage in (1, 2, 3):
        t.rk3_stage(stage, dt)
        exchange(t, stage if stage < 3 else 0, rank, world)
    return dt
