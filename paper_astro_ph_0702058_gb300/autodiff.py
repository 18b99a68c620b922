"""torch.autograd.Function over the library's hand-written adjoint of a shared-step rollout.

``rollout(x0, v0, m, eps2=..., level=9, steps=256)`` returns the final
positions and velocities (x_T, v_T) of a Hermite rollout with one shared step
dt = 2^-level (FP32 pair math, FP64 state; nbody_rollout), and can sit inside
any larger differentiable program: its backward takes the incoming cotangents
of x_T and v_T and returns their vector-Jacobian product with respect to x0,
v0 and m (nbody_rollout_vjp: the forward run recomputed with checkpoints, then
the hand-written reverse sweep).

``rollout_loss(x0, v0, m, ...)`` is the fixed-loss convenience: the scalar
L = sum |x_final|^2 + E_pot(final), whose forward call computes the gradient
too (nbody_diff_rollout); its backward only scales it.  Argument marshalling
only.
"""
from __future__ import annotations

import torch

from . import MODES
from ._lib import nbody_diff_rollout, nbody_rollout, nbody_rollout_vjp


def _f64(t, dev):
    return t.detach().to(dev, torch.float64).contiguous()


def _stream(dev):
    return torch.cuda.current_stream(dev) if dev.type == "cuda" else None


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, eps2, level, steps, checkpoint_every, mode):
        dev = x0.device
        x, v, mm = _f64(x0, dev), _f64(v0, dev), _f64(m, dev)
        n = mm.shape[0]
        xT = torch.empty_like(x)
        vT = torch.empty_like(v)
        nbody_rollout(n, mm, x, v, eps2, level, steps, mode, xT, vT, _stream(dev))
        ctx.save_for_backward(x, v, mm)
        ctx.args = (eps2, level, steps, checkpoint_every, mode)
        return xT, vT

    @staticmethod
    def backward(ctx, g_xT, g_vT):
        x, v, mm = ctx.saved_tensors
        eps2, level, steps, checkpoint_every, mode = ctx.args
        dev = x.device
        gx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        gv = torch.empty_like(v) if ctx.needs_input_grad[1] else None
        gm = torch.empty_like(mm) if ctx.needs_input_grad[2] else None
        if gx is None and gv is None and gm is None:
            return None, None, None, None, None, None, None, None
        nbody_rollout_vjp(mm.shape[0], mm, x, v, eps2, level, steps, checkpoint_every, mode,
                          None if g_xT is None else _f64(g_xT, dev), None if g_vT is None else _f64(g_vT, dev),
                          gx, gv, gm, _stream(dev))
        return gx, gv, gm, None, None, None, None, None


class RolloutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, eps2, level, steps, checkpoint_every, mode):
        dev = x0.device
        x = x0.detach().to(torch.float64).contiguous()
        v = v0.detach().to(dev, torch.float64).contiguous()
        mm = m.detach().to(dev, torch.float64).contiguous()
        n = mm.shape[0]
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        gx = torch.zeros_like(x)
        gv = torch.zeros_like(v)
        gm = torch.zeros_like(mm)
        stream = torch.cuda.current_stream(dev) if dev.type == "cuda" else None
        nbody_diff_rollout(n, mm, x, v, eps2, level, steps, checkpoint_every, mode, loss, gx, gv, gm, stream)
        ctx.save_for_backward(gx, gv, gm)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        gx, gv, gm = ctx.saved_tensors
        return g * gx, g * gv, g * gm, None, None, None, None, None


def rollout_loss(x0, v0, m, *, eps2=(1.0 / 128) ** 2, level=9, steps=256, checkpoint_every=16, mode="plain"):
    return RolloutLoss.apply(x0, v0, m, float(eps2), int(level), int(steps), int(checkpoint_every),
                             MODES[mode] if isinstance(mode, str) else int(mode))


def rollout(x0, v0, m, *, eps2=(1.0 / 128) ** 2, level=9, steps=256, checkpoint_every=16, mode="plain"):
    """(x_T, v_T) of the shared-step rollout, differentiable with respect to x0, v0 and m."""
    return Rollout.apply(x0, v0, m, float(eps2), int(level), int(steps), int(checkpoint_every),
                         MODES[mode] if isinstance(mode, str) else int(mode))
