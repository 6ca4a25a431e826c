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


def branch_consistent_envs(desc, gpu_starts, orc_starts, actions, window):
    """Environments along whose GPU trajectory the oracle takes the same
    branches as along its own: for every window of `window` steps, the
    oracle's branch signature from the GPU's state at the window's start
    (gpu_starts[w]) equals its signature from its own state there
    (orc_starts[w]).  Where they differ, FP32 rounding has moved the state
    across a contact, friction or limit threshold and the two trajectories
    legitimately part after it."""
    ok = np.ones(gpu_starts[0].shape[0], dtype=bool)
    for w in range(len(gpu_starts)):
        a = actions[w * window:(w + 1) * window]
        _, sg = orc.rollout(desc, gpu_starts[w], a, branch_signature=True)
        _, so = orc.rollout(desc, orc_starts[w], a, branch_signature=True)
        ok &= sg == so
    return ok
