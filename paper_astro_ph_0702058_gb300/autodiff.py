"""torch.autograd.Function over the library's hand-written adjoint of a shared-step rollout.

``rollout_loss(x0, v0, m, eps2=..., level=9, steps=256)`` returns the scalar
L = sum |x_final|^2 + E_pot(final) of a Hermite rollout with one shared step
dt = 2^-level (FP32 pair math, FP64 state), and ``L.backward()`` delivers
dL/dx0, dL/dv0, dL/dm.  The forward call computes the gradient too (one
nbody_diff_rollout: forward with checkpoints, then the reverse sweep); the
backward only scales it by the incoming gradient.  Argument marshalling only.
"""
from __future__ import annotations

import torch

from . import MODES
from ._lib import nbody_diff_rollout


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
