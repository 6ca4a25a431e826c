"""Analytic policy gradients through the differentiable step (Sec. 5.1, APG).

The paper's stated use of differentiability: a policy is trained by
differentiating the return of short trajectories through the simulator
itself.  Here a small torch MLP maps each environment's observation to
torque actions; every step of the closed loop is one forward launch of the
library (brax_rollout, checkpointing the step's input) and, on the way back,
one launch of the hand-written adjoint (brax_rollout_backward), through the
torch.autograd binding.  The loss of a trajectory of T steps is
    L = mean over envs of [-(x_torso,T - x_torso,0)] + w_a * mean sum_t |a_t|^2,
a synthetic forward-progress reward with an action penalty.

Run `python -m paper_2106_13281_gb300.apg` on a GPU for a training curve.
"""
from __future__ import annotations

import torch

from .autograd import rollout


def observe(state: torch.Tensor) -> torch.Tensor:
    """Observation of each environment from its state [N, B, 13]: the root
    body's height, orientation, velocity and angular velocity, and every
    other body's position relative to the root, orientation and angular
    velocity (a differentiable function of the state)."""
    root = state[:, 0]
    rel = state[:, 1:, 0:3] - root[:, None, 0:3]
    parts = [root[:, 2:13], rel.flatten(1), state[:, 1:, 3:7].flatten(1), state[:, 1:, 10:13].flatten(1)]
    return torch.cat(parts, dim=1)


def obs_dim(n_bodies: int) -> int:
    return 11 + 10 * (n_bodies - 1)


class Policy(torch.nn.Module):
    """MLP policy: observation -> tanh -> actions in [-1, 1]."""

    def __init__(self, n_bodies: int, n_actions: int, hidden: int = 64):
        super().__init__()
        self.net = torch.nn.Sequential(torch.nn.Linear(obs_dim(n_bodies), hidden), torch.nn.Tanh(),
                                       torch.nn.Linear(hidden, hidden), torch.nn.Tanh(),
                                       torch.nn.Linear(hidden, n_actions))

    def forward(self, obs: torch.Tensor) -> torch.Tensor:
        return torch.tanh(self.net(obs))


def trajectory_loss(system, policy: torch.nn.Module, state0: torch.Tensor, T: int, action_weight: float = 1e-3):
    """Closed-loop rollout of T steps under `policy` and its loss (one
    forward launch per step; backward() runs one adjoint launch per step)."""
    s = state0
    penalty = state0.new_zeros(())
    for _ in range(T):
        a = policy(observe(s))
        penalty = penalty + (a * a).sum(dim=1).mean()
        s, _ = rollout(system, s, a[None].contiguous(), 1)
    progress = (s[:, 0, 0] - state0[:, 0, 0]).mean()
    return -progress + action_weight * penalty, progress


def train(system, state0: torch.Tensor, T: int = 10, iters: int = 200, lr: float = 1e-3, seed: int = 0,
          log=None):
    """Adam on the trajectory loss from the fixed start states; returns the
    policy and the list of (loss, progress) per iteration."""
    torch.manual_seed(seed)
    policy = Policy(system.B, system.A).to(state0.device)
    opt = torch.optim.Adam(policy.parameters(), lr=lr)
    hist = []
    for it in range(iters):
        opt.zero_grad(set_to_none=True)
        loss, prog = trajectory_loss(system, policy, state0, T)
        loss.backward()
        torch.nn.utils.clip_grad_norm_(policy.parameters(), 1.0)
        opt.step()
        hist.append((float(loss.detach()), float(prog.detach())))
        if log is not None and (it % 10 == 0 or it == iters - 1):
            log(f"iter {it:4d}  loss {hist[-1][0]: .4f}  forward progress {hist[-1][1]: .4f} m")
    return policy, hist


def _main():
    import numpy as np

    from . import scenes as S
    from .system import BraxSystem
    d = S.quadruped()
    sysm = BraxSystem(d)
    N = 1024
    rp, rr, ang = S.initial_conditions(d, N, 0, height_jitter=0.05)
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    st = sysm.default_qp(N, f32(rp), f32(rr), f32(ang))
    # let the quadruped settle on its feet before training
    st = sysm.rollout(st, torch.zeros((40, N, sysm.A), device="cuda"))["state_T"]
    train(sysm, st, T=10, iters=200, log=print)


if __name__ == "__main__":
    _main()
