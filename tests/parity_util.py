"""Helpers shared by the GPU parity tests."""
import numpy as np

from oracle import oracle as orc


def decided_envs(desc, state0, actions, rel=1e-6, seed=0):
    """Environments whose every branch decision (contact activation, friction
    stick/slip, limits, clamps, inside/outside of a box) is the same for the
    given inputs and for inputs perturbed at FP32 rounding level (relative
    1e-6, both signs).  Elsewhere FP32 and FP64 may legitimately take
    different branches, so gradients and one-step states are compared only
    on decided environments."""
    rng = np.random.default_rng(seed)
    _, s0 = orc.rollout(desc, state0, actions, branch_signature=True)
    ok = np.ones(state0.shape[0], dtype=bool)
    for sign in (1.0, -1.0):
        pert = state0 * (1.0 + sign * rel * rng.uniform(0.5, 1.0, size=state0.shape))
        _, s1 = orc.rollout(desc, pert, actions, branch_signature=True)
        ok &= s1 == s0
    return ok
