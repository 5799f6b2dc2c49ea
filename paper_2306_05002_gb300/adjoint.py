"""Gradients through SSP-RK3 trajectories with the library's discrete adjoint.

Checkpointing (revolve-style, one level): the forward sweep keeps the state every
`every` steps; the reverse sweep replays each segment from its checkpoint (storing
the segment's states and tapes) and runs the adjoint steps back through it, one
``dg_adjoint_segment`` call per segment.  Every step and every adjoint step runs in
the library's kernels; this module only orders the calls and keeps the checkpoints
(device memory).
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

    tape=True runs each checkpoint segment through dg_adjoint_segment (one call, one captured
    graph per segment length: the replay with dg_step_tape keeping every step's start and tape,
    then dg_adjoint_step_tape back through them); tape=False keeps only the states and lets
    dg_adjoint_step recompute the stages, one call per step."""
    starts = sorted(s for s in ckpt if s < nsteps)
    if tape:
        # The segment graphs are captured with the addresses of the states, tapes and adjoint
        # buffers, so these live on the solver and are reused by every sweep of the same shape
        # (new buffers in each sweep would mean a new capture in each sweep).
        m_max = min(every, nsteps)
        key = (m_max, tuple(lam_N.shape), lam_N.dtype, lam_N.device)
        ws = getattr(solver, "_adjoint_workspace", None)
        if ws is None or ws[0] != key:
            ws = (key,
                  torch.empty((m_max + 1,) + tuple(lam_N.shape), dtype=lam_N.dtype, device=lam_N.device),
                  torch.empty((m_max, solver.dg_tape_len()), dtype=lam_N.dtype, device=lam_N.device),
                  torch.empty_like(lam_N))
            solver._adjoint_workspace = ws
        _, states, tapes, lam = ws
        lam.copy_(lam_N)
        for s0 in reversed(starts):
            m = min(s0 + every, nsteps) - s0
            solver.dg_adjoint_segment(ckpt[s0], m, dt, states, tapes, lam)
        return lam.clone()
    lam = lam_N.clone()
    work = torch.empty_like(lam)
    seg_states = []
    for s0 in reversed(starts):
        m = min(s0 + every, nsteps) - s0
        while len(seg_states) < m:
            seg_states.append(torch.empty_like(lam))
        # replay the segment from its checkpoint, keeping w_{s0}, ..., w_{s1-1}
        work.copy_(ckpt[s0])
        for j in range(m):
            seg_states[j].copy_(work)
            if j < m - 1:
                solver.dg_step(work, dt, 1)
        for j in reversed(range(m)):
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


class DGRHS(torch.autograd.Function):
    """L = M^-1 R(w), one right-hand side, as a differentiable torch op: backward is the library's
    hand-written reverse mode, dg_rhs_vjp (FP64 contexts without viscous / surface terms or a
    pressure boundary)."""

    @staticmethod
    def forward(ctx, w, solver):
        ctx.solver = solver
        w = w.detach().contiguous()
        ctx.save_for_backward(w)
        return solver.dg_rhs(w)

    @staticmethod
    def backward(ctx, grad_L):
        (w,) = ctx.saved_tensors
        return ctx.solver.dg_rhs_vjp(w, grad_L.contiguous()), None
