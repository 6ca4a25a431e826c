"""Conservation checks of the CUDA step (GPU), measured with the oracle's
energy and momentum functions: the Sec. 6 "astronaut" protocol (no damping,
collisions or gravity).  The FP32 step must keep linear momentum to FP32
roundoff and must not drift in energy by more than twice the FP64 oracle's
own (time-discretisation) drift on the same inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def conservative(desc, damping=False):
    d = dict(desc)
    d["pair_a"] = np.zeros(0, dtype=np.int32)
    d["pair_b"] = np.zeros(0, dtype=np.int32)
    d["gravity"] = np.zeros(3)
    if not damping:
        d["spring_damping"] = np.zeros_like(d["spring_damping"])
        d["angular_damping"] = np.zeros_like(d["angular_damping"])
    return d


@pytest.mark.parametrize("name", ["biped", "quadruped"])
def test_energy_drift_within_twice_the_oracle(brax, name):
    """Actuators off, random 1 m/s kicks, 1 s (20 steps): GPU energy drift
    <= 2 x the oracle's drift on the same FP32-rounded inputs (+ 1e-4)."""
    d = conservative(S.SCENES[name]())
    N = 64
    rp, rr, ang = S.initial_conditions(d, N, 7, angle_sigma=0.05)
    st = orc.default_qp(d, N, rp, rr, ang)
    rng = np.random.default_rng(7)
    kick = rng.normal(size=(N, st.shape[1], 3))
    kick /= np.linalg.norm(kick, axis=-1, keepdims=True)
    st[:, :, 7:10] = kick
    st = st.astype(np.float32).astype(np.float64)
    a = np.zeros((20, N, len(d["gear"])))
    e0, _ = orc.energy_momentum(d, st)
    ref = orc.rollout(d, st, a)
    got = brax(d).rollout(cuda(st), cuda(a))["state_T"].cpu().numpy().astype(np.float64)
    e_ref, _ = orc.energy_momentum(d, ref)
    e_gpu, _ = orc.energy_momentum(d, got)
    drift_ref = np.mean(np.abs(e_ref - e0) / e0)
    drift_gpu = np.mean(np.abs(e_gpu - e0) / e0)
    assert drift_gpu <= 2.0 * drift_ref + 1e-4, (drift_gpu, drift_ref)


@pytest.mark.parametrize("name", ["biped", "quadruped"])
def test_linear_momentum_to_fp32_roundoff(brax, name):
    """Random actuation, damping on, no gravity or contacts: every joint and
    actuator term is equal and opposite, so sum m v stays constant up to FP32
    roundoff over 20 steps (200 substeps)."""
    d = conservative(S.SCENES[name](), damping=True)
    N = 64
    rp, rr, ang = S.initial_conditions(d, N, 8)
    st = orc.default_qp(d, N, rp, rr, ang)
    st[:, :, 7:13] = np.random.default_rng(8).normal(size=st[:, :, 7:13].shape)
    st = st.astype(np.float32).astype(np.float64)
    a = S.actions(d, N, 20, 8)
    _, m0 = orc.energy_momentum(d, st)
    got = brax(d).rollout(cuda(st), cuda(a))["state_T"].cpu().numpy().astype(np.float64)
    _, m1 = orc.energy_momentum(d, got)
    mass = float(np.sum(d["mass"]))
    vscale = np.abs(st[:, :, 7:10]).max() + 1.0
    assert np.abs(m1[:, :3] - m0[:, :3]).max() < 2e-4 * mass * vscale


def test_energy_drift_falls_with_step_size_on_the_gpu(brax):
    """The Sec. 6 conservation study as a sweep over the step size (Fig. 5:
    non-conservation against h): the astronaut protocol (the biped; actuators,
    damping, collisions and gravity off; random 1 m/s kicks) over 1 s at
    h = 5, 2.5 and 1.25 ms on the GPU.  The median energy drift over the
    environments falls as h falls, as the oracle's does, and stays within
    twice the oracle's at every h (the median: one of these 64 kicked
    configurations is unstable under the explicit springs in the oracle
    itself, at every h)."""
    base = conservative(S.biped())
    N = 64
    rp, rr, ang = S.initial_conditions(base, N, 9, angle_sigma=0.05)
    st = orc.default_qp(base, N, rp, rr, ang)
    rng = np.random.default_rng(9)
    kick = rng.normal(size=(N, st.shape[1], 3))
    kick /= np.linalg.norm(kick, axis=-1, keepdims=True)
    st[:, :, 7:10] = kick
    st = st.astype(np.float32).astype(np.float64)
    e0, _ = orc.energy_momentum(base, st)
    drifts = []
    for subs in (10, 20, 40):
        d = dict(base, substeps=subs)
        a = np.zeros((20, N, len(d["gear"])))
        got = brax(d).rollout(cuda(st), cuda(a))["state_T"].cpu().numpy().astype(np.float64)
        ref = orc.rollout(d, st, a)
        e_gpu, _ = orc.energy_momentum(d, got)
        e_ref, _ = orc.energy_momentum(d, ref)
        dg, dr = np.median(np.abs(e_gpu - e0) / e0), np.median(np.abs(e_ref - e0) / e0)
        assert dg <= 2.0 * dr + 1e-4, (subs, dg, dr)
        drifts.append(dg)
    assert drifts[2] < drifts[1] < drifts[0], drifts
