"""The fused environment layer (GPU; Sec. 4.2 gym-like env): observation,
reward, done and auto reset written by the rollout kernel after every step,
checked against the oracle's statement of the same layer (oracle/env.py).

Step by step (one launch per step), the layer's outputs are compared with
the oracle's observation, reward and done of the GPU's own FP32 states, so
only the layer's arithmetic is under test; over a multi-step launch with
auto reset, they are compared with the oracle's environment rollout."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import env as oenv
from oracle import oracle as orc
from paper_2106_13281_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def brax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_13281_gb300.system import BraxSystem
    return BraxSystem


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


def settled(d, N, seed, drop=0.0, T=20):
    rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
    rp[:, 2] -= drop
    st = orc.default_qp(d, N, rp, rr, ang)
    a = S.actions(d, N, T, seed).astype(np.float64)
    return orc.rollout(d, st, a).astype(np.float32).astype(np.float64)


CASES = [("quadruped", 0.38), ("biped", 0.0), ("pendulum", 0.0), ("quadruped_2dof", 0.38)]


@pytest.mark.parametrize("name,drop", CASES)
def test_env_layer_each_step(brax, name, drop):
    """One launch per step, 8 steps: the observation equals the oracle's
    observation of the GPU's state after the step (root fields exactly,
    angles and rates to FP32 rounding), the reward and done are the oracle's
    formulas on the GPU's states before and after the step, and a done
    environment's next state is its reset state."""
    d = S.SCENES[name]()
    sysm = brax(d)
    N = 70  # two groups of 32 and a ragged tail
    st = settled(d, N, 301, drop)
    reset = settled(d, N, 302, drop)
    a_all = S.actions(d, N, 8, 303)
    D = sysm.env_obs_size()
    assert D == oenv.obs_size(d)
    root_z = st[:, 0, 2]
    spec = oenv.EnvSpec(forward_weight=1.25, healthy_reward=0.5, ctrl_cost=0.3,
                        min_z=float(np.quantile(root_z, 0.3)), max_z=float(np.quantile(root_z, 0.97)))
    lo, hi = np.float32(spec.min_z), np.float32(spec.max_z)
    cur = st
    n_done = 0
    for t in range(8):
        out = sysm.env_rollout(cuda(cur), cuda(a_all[t:t + 1]), reset_state=cuda(reset),
                               forward_weight=spec.forward_weight, healthy_reward=spec.healthy_reward,
                               ctrl_cost=spec.ctrl_cost, min_z=spec.min_z, max_z=spec.max_z, auto_reset=True)
        plain = sysm.rollout(cuda(cur), cuda(a_all[t:t + 1]))["state_T"].cpu().numpy().astype(np.float64)
        obs = out["obs"].cpu().numpy()[0].astype(np.float64)
        rew = out["reward"].cpu().numpy()[0].astype(np.float64)
        done = out["done"].cpu().numpy()[0].astype(bool)
        nxt = out["state_T"].cpu().numpy().astype(np.float64)
        z = plain[:, 0, 2].astype(np.float32)
        exp_done = (z < lo) | (z > hi)
        assert np.array_equal(done, exp_done), t
        ref = oenv.observe(d, plain)
        assert np.array_equal(obs[:, :11], ref[:, :11])  # the root's state, copied
        nd = (D - 11) // 2
        assert np.abs(obs[:, 11:11 + nd] - ref[:, 11:11 + nd]).max() < 2e-5  # angles (rad)
        rate_tol = 1e-5 * (1.0 + np.abs(ref[:, 11 + nd:]))
        assert (np.abs(obs[:, 11 + nd:] - ref[:, 11 + nd:]) <= rate_tol).all()  # rates (rad/s)
        ctrl = np.sum(np.clip(a_all[t].astype(np.float64), -1, 1) ** 2, axis=1)
        exp_rew = (spec.forward_weight * (plain[:, 0, 0] - cur[:, 0, 0]) / d["dt"] + spec.healthy_reward * (~exp_done)
                   - spec.ctrl_cost * ctrl)
        assert np.abs(rew - exp_rew).max() < 1e-5 * (1.0 + np.abs(exp_rew).max())
        # the physics is untouched, and a done environment restarts from its reset state
        assert np.array_equal(nxt[~done], plain[~done])
        assert np.array_equal(nxt[done], reset[done].astype(np.float32).astype(np.float64))
        n_done += done.sum()
        cur = nxt
    assert n_done > 0
    sysm.sync_status()


@pytest.mark.parametrize("name,drop", CASES[:1])
def test_env_rollout_matches_oracle(brax, name, drop):
    """One launch of 12 steps with auto reset against the oracle's
    environment rollout from the same inputs: done flags equal on every
    environment whose root height stays clear of the bounds by more than
    1e-4 m (the FP32 and FP64 trajectories are within ~1e-5 m), and there
    observations and rewards agree to FP32 trajectory accuracy."""
    d = S.SCENES[name]()
    sysm = brax(d)
    N, T = 96, 12
    st = settled(d, N, 311, drop)
    reset = settled(d, N, 312, drop)
    a = S.actions(d, N, T, 313)
    z0 = st[:, 0, 2]
    spec = oenv.EnvSpec(forward_weight=1.0, healthy_reward=1.0, ctrl_cost=0.5,
                        min_z=float(np.quantile(z0, 0.25)), max_z=float(z0.max() + 0.05))
    sT, obs_r, rew_r, done_r = oenv.env_rollout(d, spec, st, reset, a.astype(np.float64))
    out = sysm.env_rollout(cuda(st), cuda(a), reset_state=cuda(reset), forward_weight=spec.forward_weight,
                           healthy_reward=spec.healthy_reward, ctrl_cost=spec.ctrl_cost, min_z=spec.min_z,
                           max_z=spec.max_z, auto_reset=True)
    sysm.sync_status()
    obs = out["obs"].cpu().numpy().astype(np.float64)
    rew = out["reward"].cpu().numpy().astype(np.float64)
    done = out["done"].cpu().numpy().astype(bool)
    # environments whose root height never comes within 1e-4 m of a bound in the oracle run
    zr = obs_r[:, :, 0]
    clear = (np.minimum(np.abs(zr - spec.min_z), np.abs(zr - spec.max_z)) > 1e-4).all(axis=0)
    assert clear.mean() > 0.8
    assert done_r[:, clear].any()  # some environments end (and restart) within the rollout
    assert np.array_equal(done[:, clear], done_r[:, clear])
    assert np.abs(obs[:, clear, :11] - obs_r[:, clear, :11]).max() < 1e-3
    nd = (obs.shape[2] - 11) // 2
    assert np.abs(obs[:, clear, 11:11 + nd] - obs_r[:, clear, 11:11 + nd]).max() < 1e-3
    assert np.abs(rew[:, clear] - rew_r[:, clear]).max() < 1e-2


def test_env_rollout_edge_cases(brax):
    """Zero steps return the state unchanged; without auto reset a done
    environment keeps stepping from its own state (the physics of a plain
    rollout), while its done flags and rewards are still written; min_z above
    max_z is refused."""
    from paper_2106_13281_gb300.binding import BraxError
    d = S.quadruped()
    sysm = brax(d)
    N = 37
    st = settled(d, N, 321, 0.38)
    out = sysm.env_rollout(cuda(st), torch.zeros((0, N, sysm.A), device="cuda"))
    assert torch.equal(out["state_T"], cuda(st))
    a = S.actions(d, N, 6, 322)
    z0 = st[:, 0, 2]
    lo = float(np.quantile(z0, 0.5))
    out = sysm.env_rollout(cuda(st), cuda(a), min_z=lo, max_z=10.0, auto_reset=False)
    plain = sysm.rollout(cuda(st), cuda(a))["state_T"]
    assert torch.equal(out["state_T"], plain)
    assert out["done"].cpu().numpy().any()
    with pytest.raises(BraxError):
        sysm.env_rollout(cuda(st), cuda(a), min_z=1.0, max_z=0.5)
    sysm.sync_status()
