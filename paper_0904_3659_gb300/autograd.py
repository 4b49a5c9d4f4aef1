"""Differentiation through Eq. (gravity) and the leap-frog integrator.

NBForce is a torch.autograd.Function whose forward is nb_force and whose
backward is nb_force_vjp (the hand-written adjoint pair kernel), so gradients
of any loss of a_i, p_i reach the positions and masses. leapfrog() chains
kick-drift-kick steps (Section "Method", Eqs. (1)-(3) of Fujiwara & Nakasato,
arXiv:0904.3659) on FP64 state with the FP32 force, recomputing each segment
of `checkpoint_every` steps in the backward pass instead of storing it
(torch.utils.checkpoint), so memory grows with the number of segments, not
steps.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from . import NB_PLAIN, _default_context, nb_force, nb_force_vjp


class NBForce(torch.autograd.Function):
    """(a, p) = Eq. (gravity)(x, m) for CUDA float32 x [n,3], m [n]."""

    @staticmethod
    def forward(ctx, x, m, eps, mode=NB_PLAIN, nbctx=None):
        x = x.contiguous()
        m = m.contiguous()
        n = x.shape[0]
        if nbctx is None:
            nbctx = _default_context(x.device.index or 0)
        a = torch.empty((n, 3), dtype=torch.float32, device=x.device)
        p = torch.empty((n,), dtype=torch.float32, device=x.device)
        nb_force(nbctx, x, m, n, eps, a, p, mode)
        ctx.save_for_backward(x, m)
        ctx.eps = float(eps)
        ctx.nbctx = nbctx
        return a, p

    @staticmethod
    def backward(ctx, ga, gp):
        x, m = ctx.saved_tensors
        n = x.shape[0]
        ga = torch.zeros_like(x) if ga is None else ga.to(torch.float32).contiguous()
        gp = torch.zeros_like(m) if gp is None else gp.to(torch.float32).contiguous()
        gx = torch.empty_like(x)
        gm = torch.empty_like(m)
        nb_force_vjp(ctx.nbctx, x, m, n, ctx.eps, ga, gp, gx, gm)
        return gx, gm, None, None, None


def force(x, m, eps, mode=NB_PLAIN, nbctx=None):
    """Differentiable Eq. (gravity): returns (a, p)."""
    return NBForce.apply(x, m, eps, mode, nbctx)


def _segment(x, v, a, m, eps, dt, nsteps, mode, nbctx):
    for _ in range(nsteps):
        v = v + (0.5 * dt) * (-a.double())        # Eq. (1)
        x = x + dt * v                            # Eq. (2)
        a, _ = NBForce.apply(x.float(), m, eps, mode, nbctx)
        v = v + (0.5 * dt) * (-a.double())        # Eq. (3)
    return x, v, a


def leapfrog(x0, v0, m, eps, dt, nsteps, checkpoint_every=8, mode=NB_PLAIN, nbctx=None):
    """nsteps KDK steps from FP64 (x0, v0) with FP32 masses m; differentiable
    in x0, v0 and m. Returns (x, v) at the final time."""
    a, _ = NBForce.apply(x0.float(), m, eps, mode, nbctx)
    x, v = x0, v0
    done = 0
    while done < nsteps:
        k = min(checkpoint_every, nsteps - done) if checkpoint_every else nsteps - done
        if checkpoint_every and torch.is_grad_enabled():
            x, v, a = checkpoint(_segment, x, v, a, m, eps, dt, k, mode, nbctx, use_reentrant=False)
        else:
            x, v, a = _segment(x, v, a, m, eps, dt, k, mode, nbctx)
        done += k
    return x, v
