"""Variants of the step (GPU): target-angle actuators (Sec. 3: actions are
"torques or target angles"), global damping, the gyroscopic torque, and the
planar masking of App. E, checked against the FP64 oracle like the default
step: one step from identical states, 50 steps, and the adjoint against the
oracle's tape (one substep, where it must be exact to FP32, and 3 steps)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2106_13281_gb300 import scenes as S
from parity_util import decided_envs

pytestmark = pytest.mark.gpu

SCENES = ["quadruped_variants", "quadruped_planar", "quadruped_2dof"]


@pytest.fixture(scope="module")
def brax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_13281_gb300.system import BraxSystem
    return BraxSystem


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def settled(d, N, seed, T=20):
    rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
    rp[:, 2] -= 0.38
    st = orc.default_qp(d, N, rp, rr, ang)
    return f32(orc.rollout(d, st, S.actions(d, N, T, seed).astype(np.float64)))


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)


@pytest.mark.parametrize("name", SCENES)
def test_variant_one_step_parity(brax, name):
    d = S.SCENES[name]()
    sysm = brax(d)
    N = 100
    st = settled(d, N, 401)
    a = S.actions(d, N, 1, 402)
    ref = orc.rollout(d, st, a.astype(np.float64))
    got = sysm.rollout(cuda(st), cuda(a))["state_T"].cpu().numpy().astype(np.float64)
    ok = decided_envs(d, st, a.astype(np.float64))
    assert ok.mean() >= 0.9
    for sl, tol in ((slice(0, 3), 1e-5), (slice(3, 7), 1e-4), (slice(7, 10), 2e-4), (slice(10, 13), 4e-3)):
        e = np.abs(got[ok][..., sl] - ref[ok][..., sl]).max()
        assert e <= tol, (sl, e)
    if name == "quadruped_planar":  # the plane and the single rotation axis hold exactly
        assert np.array_equal(got[..., 1], np.asarray(st[..., 1], dtype=np.float32).astype(np.float64))
        assert np.abs(got[..., [10, 12]]).max() == 0.0
    sysm.sync_status()


@pytest.mark.parametrize("name", SCENES)
def test_variant_fifty_step_parity(brax, name):
    d = S.SCENES[name]()
    sysm = brax(d)
    N, T = 128, 50
    rp, rr, ang = S.initial_conditions(d, N, 403)
    st = f32(orc.default_qp(d, N, rp, rr, ang))
    a = S.actions(d, N, T, 404)
    ref = orc.rollout(d, st, a.astype(np.float64))
    got = sysm.rollout(cuda(st), cuda(a))["state_T"].cpu().numpy().astype(np.float64)
    err = np.abs(got[..., 0:3] - ref[..., 0:3]).max(axis=(1, 2))
    ok = decided_envs(d, st, a.astype(np.float64))
    assert ok.mean() >= 0.9, ok.sum()
    assert err[ok].max() <= 1e-3, np.sort(err[ok])[-5:]
    sysm.sync_status()


@pytest.mark.parametrize("name", SCENES)
@pytest.mark.parametrize("T,substep", [(1, True), (3, False)])
def test_variant_adjoint_matches_oracle_tape(brax, name, T, substep):
    """The reverse pass of the variants (the target-angle actuator's angle
    and action terms, the damping factors, the gyroscopic torque's w and
    orientation terms) against the oracle's tape: one substep (dt = h) where
    every decided environment must agree to FP32 accuracy, and 3 steps."""
    d = S.SCENES[name]()
    if substep:
        d = dict(d, substeps=1, dt=float(d["dt"]) / int(d["substeps"]))
    sysm = brax(d)
    N = 48
    st = settled(d, N, 405)
    a = f32(S.actions(d, N, T, 406))
    rng = np.random.default_rng(407)
    gT = f32(rng.normal(size=st.shape))
    gtor = f32(rng.normal(size=(T, N, 3)))
    out = sysm.rollout(cuda(st), cuda(a), K=1, checkpoints=True, contact_count=True)
    ga, gs = sysm.rollout_backward(cuda(st), cuda(a), out["checkpoints"], cuda(gT), cuda(gtor), K=1)
    sysm.sync_status()
    ga, gs = ga.cpu().numpy().astype(np.float64), gs.cpu().numpy().astype(np.float64)
    ga_ref, gs_ref = orc.vjp(d, st, a, gT, gtor)
    _, cc_ref = orc.rollout(d, st, a, contact_count=True)
    ok = decided_envs(d, st, a) & (out["contact_count"].cpu().numpy() == cc_ref)
    assert ok.mean() >= 0.8
    ea = np.array([rel_err(ga[:, n], ga_ref[:, n]) for n in range(N) if ok[n]])
    es = np.array([rel_err(gs[n], gs_ref[n]) for n in range(N) if ok[n]])
    assert ea.max() < 1e-3 and es.max() < 1e-3, (ea.max(), es.max())
