"""FP64 oracle of the fused environment layer (the gym-like env of Sec. 4.2).

TEST INFRASTRUCTURE ONLY: the plain statement of what the library's
environment rollout computes, used by the tests to check it.  Only tests may
import it; the library never does.

The paper's env class keeps the book-keeping of a sequential decision
problem on top of the physics step: observing, rewarding, ending and
resetting episodes (Sec. 4.2; Table 1 gives the Ant's 8 actions).  It prints
no observation or reward formula, so this layer follows these readings:

  observation (after a step, before any reset), D = 11 + 2 * (joint DOF):
      the root body's height z, its quaternion (w, x, y, z), its velocity and
      its angular velocity; then every joint DOF's angle (joint order, axes
      0..dof-1) and every joint DOF's angular rate, (w_child - w_parent)
      along that axis in the world.
  reward of the step t -> t + 1 (MuJoCo-like locomotion reward; App. E notes
      that the Brax Ant drops the contact cost, as here):
      forward_weight * (x_root(t+1) - x_root(t)) / dt
      + healthy_reward * (not done) - ctrl_cost * sum_a clamp(a, -1, 1)^2.
  done: the root's height after the step lies outside [min_z, max_z].
  auto reset: a done environment continues from its reset state at the next
      step (its observation of this step is still the terminal one).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import oracle as orc


@dataclass
class EnvSpec:
    forward_weight: float = 1.0
    healthy_reward: float = 1.0
    ctrl_cost: float = 0.5
    min_z: float = 0.2
    max_z: float = 1.0
    auto_reset: bool = True


def obs_size(system) -> int:
    return 11 + 2 * int(np.sum(np.asarray(system["dof"])))


def observe(system, state):
    """Observation [N, D] of states [N, B, 13]."""
    state = np.asarray(state, dtype=np.float64)
    ang, rate = orc.joint_state(system, state)
    root = state[:, 0]
    return np.concatenate([root[:, 2:3], root[:, 3:7], root[:, 7:10], root[:, 10:13], ang, rate], axis=1)


def env_rollout(system, spec: EnvSpec, state0, reset_state, actions):
    """T steps of the environment: returns (state_T [N,B,13], obs [T,N,D],
    reward [T,N], done [T,N] bool)."""
    s = np.array(state0, dtype=np.float64)
    reset_state = np.asarray(reset_state, dtype=np.float64)
    actions = np.asarray(actions, dtype=np.float64)
    T, N = actions.shape[0], s.shape[0]
    dt = float(system["dt"])
    obs = np.zeros((T, N, obs_size(system)))
    reward = np.zeros((T, N))
    done = np.zeros((T, N), dtype=bool)
    for t in range(T):
        s1 = orc.rollout(system, s, actions[t:t + 1])
        z = s1[:, 0, 2]
        d = (z < spec.min_z) | (z > spec.max_z)
        ctrl = np.sum(np.clip(actions[t], -1.0, 1.0) ** 2, axis=1)
        reward[t] = (spec.forward_weight * (s1[:, 0, 0] - s[:, 0, 0]) / dt + spec.healthy_reward * (~d)
                     - spec.ctrl_cost * ctrl)
        obs[t] = observe(system, s1)
        done[t] = d
        if spec.auto_reset:
            s1[d] = reset_state[d]
        s = s1
    return s, obs, reward, done
