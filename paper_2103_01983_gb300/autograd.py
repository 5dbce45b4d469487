"""Differentiable Biot-Savart velocity and implicit rollouts (torch autograd).

* ``velocity(x, Gamma, delta)``: f of Eq. 2 through ``bs_velocity``; its
  backward is the hand-written adjoint kernel ``bs_vjp`` (positions and
  circulations).
* ``rollout(x0, Gamma, params, steps, every)``: ``steps`` implicit trapezoid
  steps (``fom_step``) returning x^steps; its backward runs ``fom_adjoint_step``
  (the implicit-function-theorem adjoint of each step) from the last step to
  the first, recomputing each segment of ``every`` steps from the state and
  velocity checkpointed at its start, so memory is O(steps / every + every)
  states.

All arithmetic runs in libptrom.so; torch supplies the tensors and autograd.
"""
from __future__ import annotations

import torch

from . import ptrom


class _Velocity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, Gamma, delta, prec):
        ctx.save_for_backward(x, Gamma)
        ctx.delta, ctx.prec = delta, prec
        return ptrom.bs_velocity(x.contiguous(), Gamma.contiguous(), delta, prec=prec)

    @staticmethod
    def backward(ctx, gf):
        x, Gamma = ctx.saved_tensors
        gx, gG = ptrom.bs_vjp(x, Gamma, ctx.delta, gf.contiguous(), want_x=ctx.needs_input_grad[0],
                              want_gamma=ctx.needs_input_grad[1], prec=ctx.prec)
        return gx, gG, None, None


def velocity(x, Gamma, delta, prec="fp32c"):
    """Differentiable f(x; Gamma) (Sec. 2, Eq. 2)."""
    return _Velocity.apply(x, Gamma, delta, prec)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, Gamma, params, steps, every):
        n = Gamma.numel()
        x = x0.detach().clone()
        G = Gamma.detach().contiguous()
        f = ptrom.bs_velocity(x, G, params.delta, prec=ptrom.FP64 if params.prec == ptrom.FP64 else "fp32c")
        work = ptrom.fom_workspace(params, n, x.device)
        ckpt = []
        for k in range(steps):
            if k % every == 0:
                ckpt.append((x.clone(), f.clone()))
            ptrom.fom_step(params, G, x, f, work=work)
        ctx.save_for_backward(Gamma)
        ctx.ckpt, ctx.params, ctx.steps, ctx.every = ckpt, params, steps, every
        return x

    @staticmethod
    def backward(ctx, gx):
        (Gamma,) = ctx.saved_tensors
        G = Gamma.detach().contiguous()
        p, steps, every = ctx.params, ctx.steps, ctx.every
        n = G.numel()
        lam = gx.detach().clone().contiguous()
        gG = torch.zeros_like(G)
        work = ptrom.fom_workspace(p, n, lam.device)
        awork = ptrom.fom_adjoint_workspace(p, n, lam.device)
        nseg = len(ctx.ckpt)
        for s in range(nseg - 1, -1, -1):
            x, f = ctx.ckpt[s][0].clone(), ctx.ckpt[s][1].clone()
            states = [x.clone()]
            for _ in range(min(every, steps - s * every)):
                ptrom.fom_step(p, G, x, f, work=work)
                states.append(x.clone())
            for k in range(len(states) - 1, 0, -1):
                ptrom.fom_adjoint_step(p, G, states[k], states[k - 1], lam, gG, work=awork)
        return lam, gG, None, None, None


def rollout(x0, Gamma, params, steps, every=10):
    """x^steps after ``steps`` implicit trapezoid steps, differentiable in x0
    and Gamma (checkpoint every ``every`` steps)."""
    return _Rollout.apply(x0, Gamma, params, steps, every)
