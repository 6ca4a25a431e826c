"""Parity of the CUDA adjoint with the FP64 oracle adjoint and with FP64
central finite differences (GPU).

The reverse pass differentiates the FP32 forward trajectory; the oracle's
tape differentiates the FP64 trajectory from the same FP32-rounded inputs.
Where a contact, limit or friction decision differs between the two
trajectories the gradients legitimately differ, so environments whose
active-contact counts differ, or whose oracle decisions change under an
FP32-sized perturbation of the inputs, are excluded (and bounded in number)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2106_13281_gb300 import scenes as S
from parity_util import decided_envs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def brax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_13281_gb300.system import BraxSystem
    return BraxSystem


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


def settled(d, N, seed, drop, T=20):
    rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
    rp[:, 2] -= drop
    st = orc.default_qp(d, N, rp, rr, ang)
    if len(d["parent"]) == 0:  # free bodies: random velocities instead of actuation, few steps
        rng = np.random.default_rng(seed)
        st[:, :, 7:10] += 0.3 * rng.normal(size=st[:, :, 7:10].shape)
        st[:, :, 10:13] += 2.0 * rng.normal(size=st[:, :, 10:13].shape)
        T = 1
    a = S.actions(d, N, T, seed).astype(np.float64)
    return orc.rollout(d, st, a).astype(np.float32).astype(np.float64)


def gpu_grad(sysm, st, a, gT, gtor, K):
    out = sysm.rollout(cuda(st), cuda(a), K=K, checkpoints=True, contact_count=True)
    ga, gs = sysm.rollout_backward(cuda(st), cuda(a), out["checkpoints"], cuda(gT),
                                   None if gtor is None else cuda(gtor), K=K)
    sysm.sync_status()
    return ga.cpu().numpy().astype(np.float64), gs.cpu().numpy().astype(np.float64), out["contact_count"].cpu().numpy()


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)


@pytest.mark.parametrize("name,drop,T", [("pendulum", 0.0, 5), ("quadruped", 0.38, 3), ("quadruped", 0.38, 10),
                                         ("biped", 0.0, 3), ("arm_box", 0.0, 3), ("capsule_on_box", 0.0, 1),
                                         ("capsule_in_box", 0.0, 2), ("quadruped_aniso", 0.38, 3)])
def test_adjoint_matches_oracle_tape(brax, name, drop, T):
    d = S.SCENES[name]()
    sysm = brax(d)
    N = 40  # a full group of 32 and a ragged tail
    st = settled(d, N, 11, drop)
    a = S.actions(d, N, T, 12).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(13)
    gT = rng.normal(size=st.shape).astype(np.float32).astype(np.float64)
    gtor = rng.normal(size=(T, N, 3)).astype(np.float32).astype(np.float64)
    ga, gs, cc = gpu_grad(sysm, st, a, gT, gtor, K=2)
    ga_ref, gs_ref = orc.vjp(d, st, a, gT, gtor)
    _, cc_ref = orc.rollout(d, st, a, contact_count=True)
    same = (cc == cc_ref) & decided_envs(d, st, a)
    assert same.mean() >= 0.8
    errs_a = np.array([rel_err(ga[:, n], ga_ref[:, n]) for n in range(N) if same[n]])
    errs_s = np.array([rel_err(gs[n], gs_ref[n]) for n in range(N) if same[n]])
    if name != "biped":
        assert errs_a.max() < 1e-3 and errs_s.max() < 1e-3, (errs_a.max(), errs_s.max())
    else:
        # 30 substeps of capsule-capsule contact between 17 bodies amplify the
        # FP32 rounding of the trajectory; most environments stay within 1e-3
        # and none leaves 1e-2
        assert np.mean(errs_a < 1e-3) >= 0.9 and np.mean(errs_s < 1e-3) >= 0.9, (sorted(errs_a)[-5:],
                                                                                  sorted(errs_s)[-5:])
        assert errs_a.max() < 1e-2 and errs_s.max() < 1e-2, (errs_a.max(), errs_s.max())


@pytest.mark.parametrize("name,drop", [("pendulum", 0.0), ("quadruped", 0.38), ("biped", 0.0), ("arm_box", 0.0),
                                       ("capsule_on_box", 0.0), ("capsule_in_box", 0.0), ("quadruped_aniso", 0.38)])
def test_single_substep_adjoint_exact(brax, name, drop):
    """One substep (dt = h): no trajectory divergence between FP32 and FP64
    can build up, so every environment's gradient matches the oracle tape
    to FP32 accuracy (relative error below 1e-3).  This isolates the hand-written vector-Jacobian
    products (joints, limits, actuators, all contact types) from the
    chaotic amplification of longer horizons."""
    d = S.SCENES[name]()
    d = dict(d, substeps=1, dt=float(d["dt"]) / int(d["substeps"]))
    sysm = brax(d)
    N = 64
    st = settled(d, N, 61, drop)
    a = S.actions(d, N, 1, 62).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(63)
    gT = rng.normal(size=st.shape).astype(np.float32).astype(np.float64)
    ga, gs, cc = gpu_grad(sysm, st, a, gT, None, K=1)
    ga_ref, gs_ref = orc.vjp(d, st, a, gT)
    _, cc_ref = orc.rollout(d, st, a, contact_count=True)
    ok = decided_envs(d, st, a) & (cc == cc_ref)
    assert ok.mean() >= 0.9
    for n in range(N):
        if not ok[n]:
            continue
        assert rel_err(gs[n], gs_ref[n]) < 1e-3, (n, rel_err(gs[n], gs_ref[n]))
        if a.shape[2]:
            assert rel_err(ga[:, n], ga_ref[:, n]) < 1e-3, (n, rel_err(ga[:, n], ga_ref[:, n]))


def test_adjoint_vs_fp64_central_differences(brax):
    """Quadruped, 8 envs, 20 steps, loss = -torso x displacement + 1e-3 sum |a|^2:
    GPU gradients vs FP64 central differences (h = 1e-4) of the oracle, on
    every entry whose +h and -h runs take the same branches (contact
    activation, friction stick/slip, limits, clamps) as the unperturbed run;
    and vs the oracle's tape gradient of the same loss."""
    d = S.quadruped()
    sysm = brax(d)
    N, T = 8, 20
    st = settled(d, N, 21, 0.38)
    a = S.actions(d, N, T, 22).astype(np.float32).astype(np.float64)
    gT = np.zeros_like(st)
    gT[:, 0, 0] = -1.0
    ga, gs, cc = gpu_grad(sysm, st, a, gT, None, K=5)
    ga = ga + 2e-3 * a
    ga_ref, gs_ref = orc.vjp(d, st, a, gT)
    ga_ref = ga_ref + 2e-3 * a
    _, cc_ref, sig0 = orc.rollout(d, st, a, contact_count=True, branch_signature=True)
    same = cc == cc_ref
    for n in range(N):
        if same[n]:
            assert rel_err(ga[:, n], ga_ref[:, n]) < 1e-3 and rel_err(gs[n], gs_ref[n]) < 1e-3, n

    def loss(s0, act):
        out, sig = orc.rollout(d, s0, act, branch_signature=True)
        return -(out[:, 0, 0] - s0[:, 0, 0]) + 1e-3 * np.sum(act ** 2, axis=(0, 2)), sig

    rng = np.random.default_rng(23)
    eps = 1e-4
    checked = skipped = 0
    for _ in range(40):
        t, k = rng.integers(0, T), rng.integers(0, a.shape[2])
        ap, am = a.copy(), a.copy()
        ap[t, :, k] += eps
        am[t, :, k] -= eps
        lp, sp_ = loss(st, ap)
        lm, sm_ = loss(st, am)
        fd = (lp - lm) / (2 * eps)
        for n in range(N):
            if not same[n] or sp_[n] != sig0[n] or sm_[n] != sig0[n]:
                skipped += 1
                continue
            g = ga[t, n, k]
            assert abs(fd[n] - g) <= 1e-3 * max(abs(fd[n]), abs(g)), (t, n, k, fd[n], g)
            checked += 1
    assert checked >= 100, (checked, skipped)
    for _ in range(10):
        b, j = rng.integers(0, st.shape[1]), rng.choice([0, 1, 2, 7, 8, 9, 10, 11, 12])
        sp, sm = st.copy(), st.copy()
        sp[:, b, j] += eps
        sm[:, b, j] -= eps
        lp, sp_ = loss(sp, a)
        lm, sm_ = loss(sm, a)
        fd = (lp - lm) / (2 * eps)
        for n in range(N):
            if not same[n] or sp_[n] != sig0[n] or sm_[n] != sig0[n]:
                continue
            g = gs[n, b, j]
            assert abs(fd[n] - g) <= 1e-3 * max(abs(fd[n]), abs(g)) + 1e-12, (b, j, n, fd[n], g)


@pytest.mark.parametrize("paired", [True, False])
def test_checkpoint_interval_does_not_change_gradients(brax, paired):
    """Recomputation from checkpoints is exact: K = 1, 4, 5 and T give
    bitwise identical gradients (the forward is deterministic), whichever
    kernel writes the checkpoints: the two-environments kernel (whose
    segments the reverse pass rebuilds with the same kernel) or the
    one-environment kernel (recomputed inside the reverse kernel)."""
    d = S.quadruped()
    sysm = brax(d)
    sysm.set_pair_launch(1 if paired else 0, 1, 0)
    N, T = 33, 12
    st = settled(d, N, 31, 0.38)
    a = S.actions(d, N, T, 32)
    gT = np.random.default_rng(33).normal(size=st.shape)
    ref = None
    for K in (1, 4, 5, T):
        ga, gs, _ = gpu_grad(sysm, st, a, gT, None, K)
        if ref is None:
            ref = (ga, gs)
        else:
            assert np.array_equal(ga, ref[0]) and np.array_equal(gs, ref[1])


@pytest.mark.parametrize("name,drop", [("quadruped_aniso", 0.38), ("biped", 0.0), ("arm_box", 0.0)])
def test_checkpoint_interval_general_kernel(brax, name, drop):
    """The four-barrier hinge kernel and the general kernel: the reverse
    pass recomputes a segment's steps with the checkpointing forward's
    substep arithmetic, and each body sums its body-body pairs' adjoints in
    its own pair order, so K = 1, 2 and 3, and a repeated run, give bitwise
    identical gradients."""
    d = S.SCENES[name]()
    sysm = brax(d)
    if name == "quadruped_aniso":
        sysm.set_pair_launch(0, 1, 0)  # the one-environment hinge kernel
    N, T = 40, 6
    st = settled(d, N, 35, drop)
    a = S.actions(d, N, T, 36)
    gT = np.random.default_rng(37).normal(size=st.shape)
    ref = None
    for K in (1, 2, 3, 1):
        ga, gs, _ = gpu_grad(sysm, st, a, gT, None, K)
        if ref is None:
            ref = (ga, gs)
        else:
            assert np.array_equal(ga, ref[0]) and np.array_equal(gs, ref[1]), K


@pytest.mark.parametrize("K,chunk", [(1, 3), (2, 2), (4, 1)])
def test_chunked_schedule_reverse_equals_static(brax, K, chunk):
    """The reverse pass under the chunked schedule (chunks of `chunk`
    checkpoint segments, last first; the state adjoint passes between chunks
    through the workspace), and the checkpointed forward under it: bitwise
    the static schedule's gradients."""
    d = S.quadruped()
    sysm = brax(d)
    N, T = 45, 13
    st = settled(d, N, 35, 0.38)
    a = S.actions(d, N, T, 36)
    rng = np.random.default_rng(37)
    gT = rng.normal(size=st.shape)
    gtor = rng.normal(size=(T, N, 3))
    sysm.set_schedule(0)
    ref = gpu_grad(sysm, st, a, gT, gtor, K)
    sysm.set_schedule(2, chunk)
    got = gpu_grad(sysm, st, a, gT, gtor, K)
    sysm.set_schedule(1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_chunked_schedule_reverse_general_kernel(brax):
    """The same for the biped (3-DOF joints, capsule pairs): its pair
    adjoints are summed with shared-memory atomics in no fixed order, so the
    gradients agree to rounding (relative norm 1e-4) rather than bitwise."""
    d = S.biped()
    sysm = brax(d)
    N, T, K = 40, 6, 1
    st = settled(d, N, 38, 0.0)
    a = S.actions(d, N, T, 39)
    gT = np.random.default_rng(40).normal(size=st.shape)
    sysm.set_schedule(0)
    ref = gpu_grad(sysm, st, a, gT, None, K)
    sysm.set_schedule(2, 2)
    got = gpu_grad(sysm, st, a, gT, None, K)
    sysm.set_schedule(1)
    for x, y in zip(got[:2], ref[:2]):
        assert np.linalg.norm(x - y) <= 1e-4 * np.linalg.norm(y)


def test_full_size_reverse_equals_sampled_solo(brax):
    """The headline size, 65,536 environments, 40 steps, K = 1: the
    checkpointed forward and the reverse pass run chunked (2,048 blocks are
    6.7 resident waves), and the gradients of 64 sampled environments equal
    those of a separate 64-environment run (one wave, static): an
    environment's gradient depends on its own inputs only (up to the sign of
    a zero that a lane masked out of a warp-wide branch may add)."""
    d = S.quadruped()
    sysm = brax(d)
    N, T, K = 65536, 40, 1
    rp, rr, ang = S.initial_conditions(d, N, 44, height_jitter=0.05)
    st = orc.default_qp(d, N, rp, rr, ang).astype(np.float32)
    a = S.actions(d, N, T, 45)
    gT = np.random.default_rng(46).normal(size=st.shape).astype(np.float32)
    ga, gs, _ = gpu_grad(sysm, st, a, gT, None, K)
    idx = np.unique(np.concatenate([[0, 31, 32, N - 1], np.random.default_rng(47).choice(N, 60, replace=False)]))
    ga1, gs1, _ = gpu_grad(sysm, st[idx], a[:, idx], gT[idx], None, K)
    for x, y in ((ga[:, idx], ga1), (gs[idx], gs1)):
        assert np.abs(x - y).max() <= 1e-6 * max(1.0, np.abs(y).max())
    assert np.isfinite(ga).all() and np.isfinite(gs).all()


def test_reverse_schedule_wait_gives_up_with_timeout_status(brax):
    """The reverse pass's bounded wait: with the counter started past chunk
    0 every item waits for a flag nothing sets; the status reads
    BRAX_ERR_TIMEOUT (6) and the next reverse pass runs normally."""
    from paper_2106_13281_gb300.binding import BraxError
    d = S.quadruped()
    sysm = brax(d)
    N, T, K = 70, 8, 1
    st = settled(d, N, 41, 0.38)
    a = S.actions(d, N, T, 42)
    gT = np.random.default_rng(43).normal(size=st.shape)
    units = (N + 31) // 32
    sysm.set_schedule(0)
    out = sysm.rollout(cuda(st), cuda(a), K=K, checkpoints=True)
    sysm.set_schedule(2, 2, units, 1_000_000)
    sysm.rollout_backward(cuda(st), cuda(a), out["checkpoints"], cuda(gT), None, K=K)
    with pytest.raises(BraxError) as ei:
        sysm.sync_status()
    assert ei.value.code == 6
    sysm.set_schedule(1)
    sysm.sync_status()
    ga, gs = sysm.rollout_backward(cuda(st), cuda(a), out["checkpoints"], cuda(gT), None, K=K)
    sysm.sync_status()
    assert torch.isfinite(ga).all() and torch.isfinite(gs).all()


def test_long_rollout_recomputation_is_exact(brax):
    """1000 steps: with checkpoints every 10 steps the reverse pass
    recomputes every step from its segment's checkpoint, with checkpoints
    every step it recomputes nothing but the substeps; both give bitwise the
    same gradients (the forward is deterministic), and they are finite."""
    d = S.quadruped()
    sysm = brax(d)
    N, T = 64, 1000
    rp, rr, ang = S.initial_conditions(d, N, 3, height_jitter=0.05)
    st = orc.default_qp(d, N, rp, rr, ang)
    a = S.actions(d, N, T, 3)
    gT = np.zeros_like(st)
    gT[:, 0, 0] = -1.0
    ga, gs, _ = gpu_grad(sysm, st, a, gT, None, 10)
    assert np.isfinite(ga).all() and np.isfinite(gs).all()
    assert np.abs(ga).max() > 0
    ga1, gs1, _ = gpu_grad(sysm, st, a, gT, None, 1)
    assert np.array_equal(ga, ga1) and np.array_equal(gs, gs1)


def test_autograd_function(brax):
    from paper_2106_13281_gb300.autograd import rollout
    d = S.quadruped()
    sysm = brax(d)
    N, T = 16, 6
    st = cuda(settled(d, N, 41, 0.38))
    a = cuda(S.actions(d, N, T, 42)).requires_grad_(True)
    s0 = st.clone().requires_grad_(True)
    sT, torso = rollout(sysm, s0, a, K=3)
    loss = -(sT[:, 0, 0] - s0[:, 0, 0]).sum() + 1e-3 * (a ** 2).sum() + torso[:, :, 2].sum()
    loss.backward()
    gT = torch.zeros_like(st)
    gT[:, 0, 0] = -1.0
    gtor = torch.zeros((T, N, 3), device="cuda")
    gtor[:, :, 2] = 1.0
    out = sysm.rollout(st, a.detach(), K=3, checkpoints=True)
    ga, gs = sysm.rollout_backward(st, a.detach(), out["checkpoints"], gT, gtor, K=3)
    assert torch.allclose(a.grad, ga + 2e-3 * a.detach(), atol=1e-6)
    gs[:, 0, 0] += 1.0
    assert torch.allclose(s0.grad, gs, atol=1e-6)
