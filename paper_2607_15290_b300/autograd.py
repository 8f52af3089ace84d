"""Differentiable midpoint trajectories: gradients of a loss of m(T) with respect to
the damping alpha, the uniform applied field h and the initial magnetisation m0.

The backward pass is the hand-written adjoint of the library (llg_adjoint_step):
for every converged midpoint step it solves the transposed Jacobian system with
the transposed FFT--HSS preconditioner on the GPU and propagates mbar, d/dalpha
and d/dh.  Forward states are not kept for every step: the forward keeps a
checkpoint (m, v^{n-1/2}) every `checkpoint` steps and the backward recomputes
each segment from its checkpoint before walking it in reverse (uniform
checkpointing; memory = one segment of states).

This module is orchestration only: each step, solve and adjoint runs through the
C ABI; the host adds the per-step scalar contributions to d/dalpha and d/dh.
"""
from __future__ import annotations

import torch

from . import Context, Opts, Params, llg_adjoint_step, llg_step_midpoint


def _run_segment(ctx, prm, opts, m, vprev, nsteps, keep):
    """Advance nsteps midpoint steps from (m, vprev); if keep, return the per-step
    (m_n, x_n) needed by the adjoint."""
    states = []
    for _ in range(nsteps):
        m_next, x, _ = llg_step_midpoint(ctx, prm, opts, m, vprev)
        if keep:
            states.append((m, x))
        vprev = x[:3].contiguous()
        m = m_next
    return m, vprev, states


class MidpointTrajectory(torch.autograd.Function):
    """m_T = Phi^nsteps(m0; alpha, h) with the converged midpoint map of Sec. 3.3."""

    @staticmethod
    def forward(fctx, m0, alpha, h, context: Context, k: float, lam: float, c_ex: float, exchange: int,
                opts: Opts, nsteps: int, checkpoint: int):
        prm = Params(alpha=float(alpha), c_ex=c_ex, k=k, theta=0.5, lam=lam,
                     h_ext=tuple(float(v) for v in h.detach().cpu()), exchange=exchange)
        m = m0.detach().contiguous()
        vprev = None
        ckpts = []
        done = 0
        while done < nsteps:
            seg = min(checkpoint, nsteps - done)
            ckpts.append((m, vprev, seg))
            m, vprev, _ = _run_segment(context, prm, opts, m, vprev, seg, keep=False)
            done += seg
        fctx.context, fctx.prm, fctx.opts, fctx.ckpts = context, prm, opts, ckpts
        fctx.alpha_meta = (alpha.dtype, alpha.device)
        fctx.h_meta = (h.dtype, h.device)
        return m.clone()

    @staticmethod
    def backward(fctx, grad_mT):
        ctx, prm, opts = fctx.context, fctx.prm, fctx.opts
        mbar = grad_mT.detach().contiguous().to(torch.float64)
        dalpha = 0.0
        dh = [0.0, 0.0, 0.0]
        for m_ck, v_ck, seg in reversed(fctx.ckpts):
            _, _, states = _run_segment(ctx, prm, opts, m_ck, v_ck, seg, keep=True)
            for m_n, x_n in reversed(states):
                mbar, da, dhh, _ = llg_adjoint_step(ctx, prm, opts, m_n, x_n, mbar)
                dalpha += da
                dh = [a + b for a, b in zip(dh, dhh)]
        adt, adev = fctx.alpha_meta
        hdt, hdev = fctx.h_meta
        g_alpha = torch.tensor(dalpha, dtype=adt, device=adev)
        g_h = torch.tensor(dh, dtype=hdt, device=hdev)
        return mbar, g_alpha, g_h, None, None, None, None, None, None, None, None


def midpoint_trajectory(context: Context, m0, alpha, h, k, nsteps, lam=0.5, c_ex=1.0, exchange=0, opts=None,
                        checkpoint=4):
    """Differentiable m(T) after `nsteps` midpoint steps of size k.  m0: (3, *grid) float64
    CUDA tensor; alpha: 0-dim tensor; h: (3,) tensor.  Gradients flow to all three.
    Use tight solver tolerances (rtol, picard_tol ~1e-13) when comparing with finite
    differences: the solver's own error enters the forward map at the tolerance level."""
    opts = opts or Opts(rtol=1e-12, picard_tol=1e-12, restart=30)
    return MidpointTrajectory.apply(m0, alpha, h, context, float(k), float(lam), float(c_ex), int(exchange), opts,
                                    int(nsteps), int(checkpoint))
