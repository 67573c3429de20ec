"""torch.autograd bindings of the discrete adjoint (no counterpart in the paper).

`TenoStep` differentiates one SSP-RK3 step; `trajectory` differentiates n
steps with RK-state checkpointing: the forward keeps the state every
`checkpoint_every` steps, the backward replays one segment at a time from its
checkpoint, recording every step on the library's adjoint tape (stage states,
Gauss-point values, selections; the tape is reserved once for a segment), and
runs the adjoint steps of the segment in reverse from the tape, so that no
reconstruction is repeated.  Every step of the forward and of the backward
runs in libteno; the stencil selection and the flux branches of each stage are
frozen at their forward values.
"""
from __future__ import annotations

import torch


class TenoStep(torch.autograd.Function):
    """U^{n+1} = RK3(U^n) with a fixed step dt."""

    @staticmethod
    def forward(ctx, U, solver, dt: float):
        solver.set_state(U.contiguous())
        solver.rk3_step(dt, sync=False)
        out = torch.empty_like(U)
        solver.get_state(out)
        ctx.solver, ctx.dt = solver, dt
        ctx.save_for_backward(U)
        return out

    @staticmethod
    def backward(ctx, grad):
        (U,) = ctx.saved_tensors
        ctx.solver.set_state(U.contiguous())
        lam = torch.empty_like(U)
        ctx.solver.adjoint_step(ctx.dt, grad.contiguous(), lam)
        return lam, None, None


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, dt: float, n_steps: int, every: int):
        solver.set_state(U0.contiguous())
        checkpoints = [U0.detach().clone()]
        for k in range(1, n_steps + 1):
            solver.rk3_step(dt, sync=False)
            if k % every == 0 and k < n_steps:
                buf = torch.empty_like(U0)
                solver.get_state(buf)
                checkpoints.append(buf)
        out = torch.empty_like(U0)
        solver.get_state(out)
        ctx.solver, ctx.dt, ctx.n, ctx.every = solver, dt, n_steps, every
        ctx.checkpoints = checkpoints
        return out

    @staticmethod
    def backward(ctx, grad):
        solver, dt, n, every = ctx.solver, ctx.dt, ctx.n, ctx.every
        lam = grad.contiguous().clone()
        nxt = torch.empty_like(lam)
        solver.tape_reserve(min(every, n))
        for seg in range(len(ctx.checkpoints) - 1, -1, -1):
            start = seg * every
            stop = min(n, start + every)
            # replay the segment on the tape
            solver.set_state(ctx.checkpoints[seg])
            for k in range(stop - start):
                solver.rk3_step_record(k, dt)
            for k in range(stop - start - 1, -1, -1):
                solver.adjoint_step_tape(k, lam, nxt)
                lam, nxt = nxt, lam
        solver.tape_reserve(0)
        return lam, None, None, None, None


def trajectory(U0: torch.Tensor, solver, dt: float, n_steps: int, checkpoint_every: int = 20):
    """U(t = n_steps*dt) from U0 with a differentiable, checkpointed SSP-RK3 loop."""
    return _Trajectory.apply(U0, solver, float(dt), int(n_steps), int(checkpoint_every))
