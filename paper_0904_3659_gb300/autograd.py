"""Differentiation through Eq. (gravity) and the leap-frog integrator.

NBForce is a torch.autograd.Function whose forward is nb_force and whose
backward is nb_force_vjp (the hand-written adjoint pair kernel), so gradients
of any loss of a_i, p_i reach the positions and masses.

leapfrog() integrates kick-drift-kick steps (Section "Method", Eqs. (1)-(3)
of Fujiwara & Nakasato, arXiv:0904.3659) on FP64 state with the FP32 force
through nb_leapfrog_step, one call per segment of `checkpoint_every` steps,
keeping only each segment's starting state. Its backward calls
nb_leapfrog_adjoint per segment, last segment first: the library replays
the segment and sweeps it in reverse with its own kernels, so memory grows
with the number of segments (plus one segment's positions), not with the
number of steps, and no step of the integrator runs as PyTorch arithmetic.
"""
from __future__ import annotations

import torch

from . import (NB_PLAIN, _default_context, nb_force, nb_force_vjp, nb_leapfrog_adjoint,
               nb_leapfrog_step)


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
        gp = None if gp is None else gp.to(torch.float32).contiguous()  # None: p unused
        gx = torch.empty_like(x)
        gm = torch.empty_like(m)
        nb_force_vjp(ctx.nbctx, x, m, n, ctx.eps, ga, gp, gx, gm)
        return gx, gm, None, None, None


def force(x, m, eps, mode=NB_PLAIN, nbctx=None):
    """Differentiable Eq. (gravity): returns (a, p)."""
    return NBForce.apply(x, m, eps, mode, nbctx)


class Trajectory(torch.autograd.Function):
    """(x, v) after nsteps leap-frog steps from FP64 (x0, v0) with FP32
    masses m, differentiable in x0, v0 and m."""

    @staticmethod
    def forward(ctx, x0, v0, m, eps, dt, nsteps, checkpoint_every, mode, nbctx):
        if nbctx is None:
            nbctx = _default_context(x0.device.index or 0)
        n = x0.shape[0]
        m = m.detach().contiguous()
        x = x0.detach().contiguous().clone()
        v = v0.detach().contiguous().clone()
        a = torch.empty((n, 3), dtype=torch.float32, device=x0.device)
        seg = int(checkpoint_every) if checkpoint_every else max(int(nsteps), 1)
        starts = []  # (x, v, a or None, steps) at each segment start
        done = 0
        while done < nsteps:
            k = min(seg, nsteps - done)
            first = not starts
            starts.append((x.clone(), v.clone(), None if first else a.clone(), k))
            nb_leapfrog_step(nbctx, x, v, m, a, None, n, eps, dt, k, 0 if first else 1, mode)
            done += k
        ctx.starts, ctx.m, ctx.nbctx = starts, m, nbctx
        ctx.args = (float(eps), float(dt), int(mode))
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        eps, dt, mode = ctx.args
        m, n = ctx.m, ctx.m.shape[0]
        dev = m.device
        lx = (torch.zeros((n, 3), dtype=torch.float64, device=dev) if gx is None
              else gx.to(torch.float64).contiguous().clone())
        lv = (torch.zeros((n, 3), dtype=torch.float64, device=dev) if gv is None
              else gv.to(torch.float64).contiguous().clone())
        la = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        lm = torch.zeros((n,), dtype=torch.float64, device=dev)
        for idx in reversed(range(len(ctx.starts))):
            xs, vs, as_, k = ctx.starts[idx]
            nb_leapfrog_adjoint(ctx.nbctx, xs, vs, as_, m, n, eps, dt, k, lx, lv, la, lm,
                                apply_first=(idx == 0), mode=mode)
        return lx, lv, lm.to(m.dtype), None, None, None, None, None, None


def leapfrog(x0, v0, m, eps, dt, nsteps, checkpoint_every=8, mode=NB_PLAIN, nbctx=None):
    """nsteps KDK steps from FP64 (x0, v0) with FP32 masses m; differentiable
    in x0, v0 and m. Returns (x, v) at the final time. checkpoint_every = 0
    keeps no intermediate state (the backward replays all steps at once)."""
    return Trajectory.apply(x0, v0, m, eps, dt, nsteps, checkpoint_every, mode, nbctx)
