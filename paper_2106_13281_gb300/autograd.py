"""torch.autograd binding of the differentiable rollout (Sec. 1, Sec. 5 APG).

Forward: one persistent rollout launch that also writes the checkpoints the
reverse pass needs (every K steps).  Backward: the hand-written adjoint
kernel, which recomputes each checkpoint segment on chip and returns the
gradients with respect to the initial state and the action sequence.
"""
from __future__ import annotations

import torch


class BraxRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, system, state0, actions, K):
        state0 = state0.contiguous()
        actions = actions.contiguous()
        out = system.rollout(state0, actions, K=K, checkpoints=True, torso=True)
        ctx.system = system
        ctx.K = K
        ctx.save_for_backward(state0, actions, out["checkpoints"])
        return out["state_T"], out["torso"]

    @staticmethod
    def backward(ctx, g_state_T, g_torso):
        state0, actions, ckpt = ctx.saved_tensors
        if g_state_T is None:
            g_state_T = torch.zeros_like(state0)
        g_actions, g_state0 = ctx.system.rollout_backward(
            state0, actions, ckpt, g_state_T.contiguous(), None if g_torso is None else g_torso.contiguous(), K=ctx.K)
        return None, g_state0, g_actions, None


def rollout(system, state0, actions, K: int = 10):
    """Differentiable rollout: returns (state_T [N,B,13], torso [T,N,3])."""
    return BraxRollout.apply(system, state0, actions, K)
