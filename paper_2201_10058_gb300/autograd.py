"""torch.autograd.Function around the recorded kick-drift-kick integration.

Forward integrates nsteps steps of the original hybrid scheme (frozen
encounters recorded along the way, checkpoints every `checkpoint_every`
steps); backward runs the library's hand-written adjoint, giving gradients of
the final positions/velocities with respect to the initial state and the
masses.  Tensors are (3, n) component-major float64 CUDA tensors.
"""
from __future__ import annotations

import torch

from . import genga


class KickDriftKick(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, params, nsteps: int, checkpoint_every: int):
        pos = x0.detach().clone().contiguous()
        vel = v0.detach().clone().contiguous()
        mass = m.detach().clone().contiguous()
        sysm = genga.System(pos, vel, mass, params)
        sysm.adjoint_forward(nsteps, checkpoint_every)
        ctx.sysm = sysm
        return pos.clone(), vel.clone()

    @staticmethod
    def backward(ctx, gx, gv):
        sysm = ctx.sysm
        if sysm is None:
            raise RuntimeError("the recorded trajectory of KickDriftKick serves one backward pass "
                               "only (it is released after the first); run the forward again to "
                               "differentiate again")
        gx0, gv0, gm = sysm.adjoint_backward(gx.contiguous(), gv.contiguous())
        sysm.close()
        ctx.sysm = None
        return gx0, gv0, gm, None, None, None


def integrate(x0, v0, m, params, nsteps: int, checkpoint_every: int = 100):
    """Differentiable nsteps of the hybrid step (frozen encounters)."""
    return KickDriftKick.apply(x0, v0, m, params, nsteps, checkpoint_every)
