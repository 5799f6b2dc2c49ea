"""Gradients through SSP-RK3 trajectories with the library's discrete adjoint.

Checkpointing (revolve-style, one level): the forward sweep keeps the state every
`every` steps; the reverse sweep replays each segment from its checkpoint (storing
the segment's states) and runs ``dg_adjoint_step`` back through it.  Every step and
every adjoint step runs in the library's kernels; this module only orders the calls
and keeps the checkpoints (device memory).
"""
from __future__ import annotations

import torch


def forward(solver, w0, dt: float, nsteps: int, every: int = 20):
    """Advance a copy of w0 by nsteps steps; return the final state and the checkpoints
    {step: state} taken every `every` steps (step 0 included)."""
    work = w0.clone()
    ckpt = {0: w0.clone()}
    done = 0
    while done < nsteps:
        k = min(every, nsteps - done)
        solver.dg_step(work, dt, k)
        done += k
        if done < nsteps:
            ckpt[done] = work.clone()
    return work, ckpt


def backward(solver, ckpt, lam_N, dt: float, nsteps: int, every: int = 20, tape: bool = True):
    """lam_0 = (d w_N / d w_0)^T lam_N by segment replay and adjoint steps.

    tape=True replays each segment with dg_step_tape (the stages and face traces of every
    step are kept) and reverses with dg_adjoint_step_tape; tape=False keeps only the states
    and lets dg_adjoint_step recompute the stages."""
    lam = lam_N.clone()
    work = torch.empty_like(lam)
    starts = sorted(s for s in ckpt if s < nsteps)
    seg_states, tapes = [], []
    tl = solver.dg_tape_len() if tape else 0
    for s0 in reversed(starts):
        s1 = min(s0 + every, nsteps)
        m = s1 - s0
        while len(seg_states) < m:
            seg_states.append(torch.empty_like(lam))
            if tape:
                tapes.append(torch.empty(tl, dtype=lam.dtype, device=lam.device))
        # replay the segment from its checkpoint, keeping w_{s0}, ..., w_{s1-1} (and the tapes)
        work.copy_(ckpt[s0])
        for j in range(m):
            seg_states[j].copy_(work)
            if tape:
                solver.dg_step_tape(work, dt, tapes[j])
            elif j < m - 1:
                solver.dg_step(work, dt, 1)
        for j in reversed(range(m)):
            if tape:
                solver.dg_adjoint_step_tape(seg_states[j], tapes[j], lam, dt, lam_n=lam)
            else:
                solver.dg_adjoint_step(seg_states[j], lam, dt, lam_n=lam)
    return lam


class DGTrajectory(torch.autograd.Function):
    """w_N = Phi^N(w_0) as a differentiable torch op (FP64 contexts without viscous / surface terms)."""

    @staticmethod
    def forward(ctx, w0, solver, dt, nsteps, every):
        wN, ckpt = forward(solver, w0.detach(), dt, nsteps, every)
        ctx.solver, ctx.ckpt, ctx.dt, ctx.nsteps, ctx.every = solver, ckpt, dt, nsteps, every
        return wN

    @staticmethod
    def backward(ctx, grad_wN):
        lam0 = backward(ctx.solver, ctx.ckpt, grad_wN.contiguous(), ctx.dt, ctx.nsteps, ctx.every)
        return lam0, None, None, None, None
