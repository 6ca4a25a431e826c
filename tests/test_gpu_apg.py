"""Analytic policy gradients through the differentiable step (GPU; Sec. 5.1
APG): a small MLP policy's gradient through a closed-loop rollout equals the
one assembled from the FP64 oracle's per-step vector-Jacobian products, and
training the policy through brax_rollout_backward raises the forward
progress of the quadruped."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2106_13281_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def quad():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_13281_gb300.system import BraxSystem
    d = S.quadruped()
    return d, BraxSystem(d)


def settled(d, N, seed, T=20):
    rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
    rp[:, 2] -= 0.38
    st = orc.default_qp(d, N, rp, rr, ang)
    a = S.actions(d, N, T, seed).astype(np.float64)
    return orc.rollout(d, st, a).astype(np.float32).astype(np.float64)


def test_apg_gradient_matches_oracle(quad):
    """Policy-parameter gradient of the trajectory loss on the GPU (forward
    and adjoint launches per step) against the same closed loop run by the
    oracle in FP64: forward steps by orc.rollout, and the reverse sweep
    chaining orc.vjp of each step with torch's gradient of the policy."""
    from paper_2106_13281_gb300.apg import Policy, observe, trajectory_loss
    d, sysm = quad
    N, T, w = 8, 3, 1e-3
    st = settled(d, N, 201)
    torch.manual_seed(5)
    pol = Policy(sysm.B, sysm.A).cuda()
    loss, _ = trajectory_loss(sysm, pol, torch.from_numpy(st.astype(np.float32)).cuda(), T, action_weight=w)
    loss.backward()
    g_gpu = torch.cat([p.grad.flatten() for p in pol.parameters()]).double().cpu().numpy()

    pol64 = copy.deepcopy(pol).double().cpu()
    for p in pol64.parameters():
        p.grad = None
    states, acts = [st], []
    with torch.no_grad():
        for _ in range(T):
            a = pol64(observe(torch.from_numpy(states[-1]))).numpy()
            acts.append(a)
            states.append(orc.rollout(d, states[-1], a[None]))
    g_s = np.zeros_like(st)
    g_s[:, 0, 0] = -1.0 / N
    for t in range(T - 1, -1, -1):
        g_a, g_prev = orc.vjp(d, states[t], acts[t][None], g_s)
        s_var = torch.from_numpy(states[t]).requires_grad_(True)
        a_var = pol64(observe(s_var))
        pen = w * (a_var * a_var).sum(dim=1).mean()
        torch.autograd.backward([a_var, pen], [torch.from_numpy(g_a[0]), torch.tensor(1.0, dtype=torch.float64)])
        g_s = g_prev + s_var.grad.numpy()
    g_ref = torch.cat([p.grad.flatten() for p in pol64.parameters()]).numpy()
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel < 1e-3, rel


def test_apg_training_raises_forward_progress(quad):
    """Adam through the adjoint for a few dozen iterations: the loss falls
    and the quadruped's forward progress over the 10-step (0.5 s) trajectory
    grows."""
    from paper_2106_13281_gb300.apg import train
    d, sysm = quad
    N = 512
    st = torch.from_numpy(settled(d, N, 202).astype(np.float32)).cuda()
    _, hist = train(sysm, st, T=10, iters=60, lr=3e-3, seed=0)
    loss = np.array([h[0] for h in hist])
    prog = np.array([h[1] for h in hist])
    assert np.isfinite(loss).all()
    assert loss[-10:].mean() < loss[:5].mean() - 0.01, (loss[:5], loss[-10:])
    assert prog[-10:].mean() > prog[:5].mean() + 0.01, (prog[:5], prog[-10:])
    sysm.sync_status()
