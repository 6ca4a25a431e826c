"""Parity of the CUDA forward path with the FP64 oracle (GPU).

Inputs are seeded and shared; the oracle runs on the same FP32-rounded
initial states.  Tolerances: one step <= 1e-5 m in position, 1e-4 in the
quaternion, 2e-4 m/s in velocity (the velocity that moves a body by the
position tolerance within one 0.05 s step) and 4e-3 rad/s in angular
velocity (the rate that turns it by the quaternion tolerance within one
step); 50 steps <= 1e-3 m in every environment; beyond the chaotic horizon
the torso displacement distributions agree (two-sample KS test and means
within 3 standard errors)."""
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


def f32(a):
    return np.asarray(a, dtype=np.float32)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(f32(a))).cuda()


def initial(desc, N, seed, jitter=0.0, drop=0.0):
    rp, rr, ang = S.initial_conditions(desc, N, seed, height_jitter=jitter)
    rp[:, 2] -= drop
    st = orc.default_qp(desc, N, rp, rr, ang)
    return f32(st).astype(np.float64), (rp, rr, ang)


SCENE_CASES = [("quadruped", 0.38), ("biped", 0.0), ("pendulum", 0.0), ("arm_box", 0.0), ("capsule_on_box", 0.0),
               ("capsule_in_box", 0.0)]


@pytest.mark.parametrize("name", [c[0] for c in SCENE_CASES[:4]])
def test_default_qp_matches_oracle(brax, name):
    d = S.SCENES[name]()
    sysm = brax(d)
    N = 70
    rp, rr, ang = S.initial_conditions(d, N, 1, height_jitter=0.05)
    ref = orc.default_qp(d, N, rp, rr, ang)
    got = sysm.default_qp(N, cuda(rp), cuda(rr), cuda(ang)).cpu().numpy()
    assert np.abs(got - ref).max() < 2e-6


def settled_states(d, name, N, seed, drop, T=30):
    """States after T oracle steps (contacts, limits and joints active).
    Free bodies (the capsule-box scenes) start tilted with random velocities
    and take one step only: once the capsule lies flat on a box face the
    closest segment point, hence the contact point, is not unique."""
    st, _ = initial(d, N, seed, jitter=0.05, drop=drop)
    if len(d["parent"]) == 0:
        rng = np.random.default_rng(seed)
        st[:, :, 7:10] += 0.3 * rng.normal(size=st[:, :, 7:10].shape)
        st[:, :, 10:13] += 2.0 * rng.normal(size=st[:, :, 10:13].shape)
        T = 1
    a = S.actions(d, N, T, seed).astype(np.float64)
    return f32(orc.rollout(d, st, a)).astype(np.float64)


@pytest.mark.parametrize("name,drop", SCENE_CASES)
def test_one_step_parity(brax, name, drop):
    """One step from identical states: max |dpos| <= 1e-5 m, |dvel| small."""
    d = S.SCENES[name]()
    sysm = brax(d)
    N = 100  # 3 full groups of 32 and a ragged tail of 4
    st = settled_states(d, name, N, 2, drop)
    a = S.actions(d, N, 1, 3)
    ref, cc_ref = orc.rollout(d, st, a.astype(np.float64), contact_count=True)
    out = sysm.rollout(cuda(st), cuda(a), contact_count=True)
    got = out["state_T"].cpu().numpy()
    assert np.isfinite(got).all()
    ok = decided_envs(d, st, a.astype(np.float64))
    assert ok.mean() >= 0.9
    dpos = np.abs(got[ok][..., 0:3] - ref[ok][..., 0:3]).max()
    assert dpos <= 1e-5, dpos
    dq = np.abs(got[ok][..., 3:7] - ref[ok][..., 3:7]).max()
    assert dq <= 1e-4, dq
    dv = np.abs(got[ok][..., 7:10] - ref[ok][..., 7:10]).max()
    assert dv <= 2e-4, dv
    dw = np.abs(got[ok][..., 10:13] - ref[ok][..., 10:13]).max()
    assert dw <= 4e-3, dw
    cc = out["contact_count"].cpu().numpy()
    assert cc_ref.sum() > 0 or name == "pendulum"
    if name.startswith("capsule_"):
        assert cc_ref.min() > 0
    # contact counts agree except where an activation threshold flips
    assert np.mean(cc == cc_ref) >= 0.9
    sysm.sync_status()


def test_step_equals_rollout_of_one(brax):
    d = S.quadruped()
    sysm = brax(d)
    N = 40
    st = settled_states(d, "quadruped", N, 4, 0.38)
    a = S.actions(d, N, 1, 4)
    r = sysm.rollout(cuda(st), cuda(a))["state_T"]
    s1 = sysm.step(cuda(st), cuda(a[0]))
    assert torch.equal(r, s1)


def test_fifty_step_parity_quadruped(brax):
    """Quadruped, 128 envs: after 50 steps every body of every environment
    is within 1e-3 m of the FP64 oracle (no environment excluded; the
    measured maximum is about 1.3e-5 m)."""
    d = S.quadruped()
    sysm = brax(d)
    N, T = 128, 50
    st, _ = initial(d, N, 0)
    a = S.actions(d, N, T, 0)
    ref = orc.rollout(d, st, a.astype(np.float64))
    got = sysm.rollout(cuda(st), cuda(a))["state_T"].cpu().numpy()
    err = np.abs(got[..., 0:3] - ref[..., 0:3]).max(axis=(1, 2))
    assert err.max() <= 1e-3, np.sort(err)[-10:]


def test_full_size_fifty_steps_sampled_parity(brax):
    """The headline size, 65,536 environments, in the launch the bench times
    (two environments per thread, one 64-environment group per block, the
    automatic chunked schedule), 50 steps as five launches of 10 (bitwise one
    launch of 50): 96 sampled environments (the first and last of the batch
    and of a block, the rest at random) within 1e-3 m of the FP64 oracle
    after 50 steps, every one along whose GPU trajectory the oracle takes its
    own branches (checked window by window from the GPU's state after every
    10 steps); at least 90 % of them."""
    from parity_util import branch_consistent_envs
    d = S.quadruped()
    sysm = brax(d)
    sysm.set_pair_launch(1, 1, 0)
    N, T, W = 65536, 50, 10
    st, _ = initial(d, N, 0)
    a = S.actions(d, N, T, 0)
    idx = np.unique(np.concatenate([[0, 1, 63, 64, N - 1], np.random.default_rng(1).choice(N, 91, replace=False)]))
    cur, gpu_starts = cuda(st), [st[idx]]
    for w in range(T // W):
        cur = sysm.rollout(cur, cuda(a[w * W:(w + 1) * W]), contact_count=(w == T // W - 1))
        cc = cur.get("contact_count")
        cur = cur["state_T"]
        gpu_starts.append(cur.cpu().numpy().astype(np.float64)[idx])
    sysm.sync_status()
    orc_starts = [st[idx]]
    for w in range(T // W):
        orc_starts.append(orc.rollout(d, orc_starts[-1], a[w * W:(w + 1) * W, idx].astype(np.float64)))
    ref, g = orc_starts[-1], gpu_starts[-1]
    err = np.abs(g[..., 0:3] - ref[..., 0:3]).max(axis=(1, 2))
    ok = branch_consistent_envs(d, gpu_starts[:-1], orc_starts[:-1], a[:, idx].astype(np.float64), W)
    assert ok.mean() >= 0.9, (ok.sum(), len(idx))
    assert err[ok].max() <= 1e-3, (np.sort(err[ok])[-5:], ok.sum(), len(idx))
    assert np.isfinite(cur.cpu().numpy()).all()
    assert (cc.cpu().numpy() > 0).mean() > 0.5  # the feet are on the ground


def test_distribution_after_1000_steps(brax):
    """Beyond the chaotic horizon: torso displacement distributions agree."""
    from scipy.stats import ks_2samp
    d = S.quadruped()
    sysm = brax(d)
    N, T = 128, 1000
    st, _ = initial(d, N, 0)
    a = S.actions(d, N, T, 0)
    ref = orc.rollout(d, st, a.astype(np.float64))
    got = sysm.rollout(cuda(st), cuda(a))["state_T"].cpu().numpy()
    assert np.isfinite(got).all()
    for k in (0, 1):
        dr = ref[:, 0, k] - st[:, 0, k]
        dg = got[:, 0, k] - st[:, 0, k]
        assert ks_2samp(dr, dg).pvalue > 0.01
        se = math.sqrt(dr.var() / N + dg.var() / N)
        assert abs(dr.mean() - dg.mean()) <= 3 * se + 1e-6
    sysm.sync_status()


def test_checkpoints_and_torso(brax):
    """Checkpoint k equals the state after kK steps; torso is body 0's
    position after every step (bitwise: the same kernel path)."""
    d = S.quadruped()
    sysm = brax(d)
    N, T, K = 45, 12, 5
    st, _ = initial(d, N, 5)
    a = cuda(S.actions(d, N, T, 5))
    out = sysm.rollout(cuda(st), a, K=K, checkpoints=True, torso=True)
    ck, tor = out["checkpoints"], out["torso"]
    assert ck.shape[0] == math.ceil(T / K)
    assert torch.equal(ck[0], cuda(st))
    # a checkpointing rollout runs the system's forward kernel (the one the
    # reverse pass rebuilds segments with): compare with rollouts of it
    for k in range(1, ck.shape[0]):
        part = sysm.rollout(cuda(st), a[:k * K].contiguous(), K=k * K, checkpoints=True)["state_T"]
        assert torch.equal(ck[k], part)
    part = sysm.rollout(cuda(st), a[:7].contiguous(), K=7, checkpoints=True)["state_T"]
    assert torch.equal(tor[6], part[:, 0, 0:3])
    assert torch.equal(tor[T - 1], out["state_T"][:, 0, 0:3])


def test_edge_sizes(brax):
    d = S.pendulum()
    sysm = brax(d)
    st, _ = initial(d, 1, 6)
    a = S.actions(d, 1, 3, 6)
    ref = orc.rollout(d, st, a.astype(np.float64))
    got = sysm.rollout(cuda(st), cuda(a))["state_T"].cpu().numpy()
    assert np.abs(got[..., :3] - ref[..., :3]).max() < 1e-5
    # T = 0 returns the initial state; N = 0 is a no-op
    z = sysm.rollout(cuda(st), torch.zeros((0, 1, sysm.A), device="cuda"))["state_T"]
    assert torch.equal(z, cuda(st))
    e = sysm.rollout(torch.zeros((0, sysm.B, 13), device="cuda"), torch.zeros((3, 0, sysm.A), device="cuda"))
    assert e["state_T"].shape == (0, sysm.B, 13)


def test_nonfinite_state_reported(brax):
    """A NaN in the input state sets the status word; no trap, context usable."""
    from paper_2106_13281_gb300.binding import BraxError
    d = S.quadruped()
    sysm = brax(d)
    st, _ = initial(d, 33, 7)
    st[17, 3, 8] = np.nan
    a = S.actions(d, 33, 2, 7)
    sysm.rollout(cuda(st), cuda(a))
    with pytest.raises(BraxError) as ei:
        sysm.sync_status()
    assert ei.value.code == 5
    # the flag is cleared and the context still works
    st[17, 3, 8] = 0.0
    sysm.rollout(cuda(st), cuda(a))
    sysm.sync_status()


@pytest.mark.parametrize("name,drop", [("quadruped", 0.38), ("pendulum", 0.0)])
def test_pair_kernel_matches_single_env_kernel(brax, name, drop):
    """Hinge-only systems run two environments per thread by default; the
    one-environment kernel computes the same step (rounding aside): one-step
    states within 1e-5, identical contact counts, checkpoints and torso
    output laid out alike, ragged tails (N = 37: one pair of half-empty
    lanes) included."""
    d = S.SCENES[name]()
    sysm = brax(d)
    for N in (37, 100):
        st, _ = initial(d, N, 11, drop=drop)
        a = cuda(S.actions(d, N, 1, 12))
        outs = []
        for mode in (1, 0):
            sysm.set_pair_launch(mode, 1, 0)
            outs.append(sysm.rollout(cuda(st), a, torso=True, contact_count=True))
            sysm.sync_status()
        p, q = outs
        dx = (p["state_T"] - q["state_T"]).abs()
        assert dx[..., :7].max().item() < 1e-5  # positions and orientations
        assert dx.max().item() < 1e-4           # velocities (m/s, rad/s)
        assert (p["torso"] - q["torso"]).abs().max().item() < 1e-5
        assert torch.equal(p["contact_count"], q["contact_count"])
    sysm.set_pair_launch(1, 1, 0)


def _rollout_outputs(sysm, st, a):
    out = sysm.rollout(st, a, torso=True, contact_count=True)
    sysm.sync_status()
    return out


@pytest.mark.parametrize("N,T,chunk", [(37, 10, 3), (100, 7, 1), (1000, 12, 5)])
def test_chunked_schedule_equals_static(brax, N, T, chunk):
    """Chunked schedule of the paired rollout (blocks take (chunk,
    environment block) items; a chunk starts from the state the previous one
    left in memory): bitwise the static schedule's final state, torso
    trajectory and contact counts, ragged tails and chunks that do not divide
    T included."""
    d = S.quadruped()
    sysm = brax(d)
    st, _ = initial(d, N, 21, drop=0.38)
    st, a = cuda(st), cuda(S.actions(d, N, T, 22))
    sysm.set_schedule(0)
    ref = _rollout_outputs(sysm, st, a)
    sysm.set_schedule(2, chunk)
    got = _rollout_outputs(sysm, st, a)
    sysm.set_schedule(1)
    for k in ("state_T", "torso", "contact_count"):
        assert torch.equal(got[k], ref[k]), k


def test_automatic_schedule_at_several_waves(brax):
    """40,000 environments are 625 blocks of 64, about two resident waves and
    a part-empty third: the automatic schedule chunks the rollout and still
    equals the static one bitwise."""
    d = S.quadruped()
    sysm = brax(d)
    N, T = 40000, 40
    st, _ = initial(d, N, 23, drop=0.38)
    st, a = cuda(st), cuda(S.actions(d, N, T, 24))
    sysm.set_pair_launch(1, 1, 0)
    sysm.set_schedule(0)
    ref = _rollout_outputs(sysm, st, a)
    sysm.set_schedule(1)
    got = _rollout_outputs(sysm, st, a)
    for k in ("state_T", "torso", "contact_count"):
        assert torch.equal(got[k], ref[k]), k


@pytest.mark.parametrize("name,drop", [("quadruped", 0.38), ("biped", 0.0)])
def test_chunked_schedule_one_env_kernel(brax, name, drop):
    """The one-environment kernel (rollouts with checkpoints; every system
    with 3-DOF joints or body-body pairs) under the chunked schedule:
    bitwise the static schedule's final state, checkpoints (K not dividing
    the chunk), torso trajectory and contact counts."""
    d = S.SCENES[name]()
    sysm = brax(d)
    N, T, K = 77, 11, 3
    st, _ = initial(d, N, 27, drop=drop)
    st, a = cuda(st), cuda(S.actions(d, N, T, 28))
    outs = []
    for mode, chunk in ((0, 0), (2, 4)):
        sysm.set_schedule(mode, chunk)
        outs.append(sysm.rollout(st, a, K=K, checkpoints=True, torso=True, contact_count=True))
        sysm.sync_status()
    sysm.set_schedule(1)
    for k in ("state_T", "checkpoints", "torso", "contact_count"):
        assert torch.equal(outs[0][k], outs[1][k]), k


@pytest.mark.parametrize("paired", [True, False])
@pytest.mark.parametrize("checkpoints", [False, True])
def test_schedule_wait_gives_up_with_timeout_status(brax, checkpoints, paired):
    """The bounded wait of the chunked schedule: when the counter starts past
    chunk 0, every item waits for a flag that nothing sets; after 1 ms each
    block gives up, the status reads BRAX_ERR_TIMEOUT (6), and the context
    still runs the next rollout."""
    from paper_2106_13281_gb300.binding import BraxError
    d = S.quadruped()
    sysm = brax(d)
    N, T = 100, 10
    st, _ = initial(d, N, 25, drop=0.38)
    st, a = cuda(st), cuda(S.actions(d, N, T, 26))
    if paired:  # two environments a thread: blocks of 64 environments
        sysm.set_pair_launch(1, 1, 0)
        units = (N + 63) // 64
    else:  # the one-environment kernel: blocks of 32 environments
        sysm.set_pair_launch(0, 1, 0)
        units = (N + 31) // 32
    sysm.set_schedule(2, 3, units, 1_000_000)
    sysm.rollout(st, a, checkpoints=checkpoints)
    with pytest.raises(BraxError) as ei:
        sysm.sync_status()
    assert ei.value.code == 6
    sysm.set_schedule(1)
    sysm.sync_status()  # the flag was cleared
    sysm.rollout(st, a, checkpoints=checkpoints)
    sysm.sync_status()


def test_pair_launch_rejected_for_general_systems(brax):
    from paper_2106_13281_gb300.binding import BraxError
    sysm = brax(S.biped())
    with pytest.raises(BraxError):
        sysm.set_pair_launch(1, 1, 0)
    sysm.set_pair_launch(0)


@pytest.mark.parametrize("name,drop", [("quadruped", 0.38), ("pendulum", 0.0)])
def test_rollout_streamed_equals_one_launch(brax, name, drop):
    """Actions streamed from pinned host memory in chunks (fixed, or
    doubling from a short first chunk; ragged last chunk) give bitwise the
    state of one launch over all steps."""
    d = S.SCENES[name]()
    sysm = brax(d)
    N, T = 100, 25
    st, _ = initial(d, N, 13, drop=drop)
    a = f32(S.actions(d, N, T, 14))
    ref = sysm.rollout(cuda(st), cuda(a))["state_T"].cpu()
    hs = torch.from_numpy(f32(st)).pin_memory()
    ha = torch.from_numpy(a).pin_memory()
    out = torch.empty((N, sysm.B, 13)).pin_memory()
    bufs = {}
    for chunk, first in ((10, 10), (7, 7), (25, 25), (100, 100), (10, 3), (8, 1), (100, 16)):
        n = sysm.rollout_streamed(hs, ha, out, chunk_steps=chunk, bufs=bufs, first_steps=first)
        torch.cuda.synchronize()
        sizes, t, k = [], 0, min(first, chunk, T)  # first_steps doubling up to chunk_steps
        while t < T:
            sizes.append(min(k, T - t))
            t, k = t + k, min(chunk, 2 * k)
        assert n == len(sizes), (chunk, first)
        assert torch.equal(out, ref), (chunk, first)
    # zero steps: the state comes back unchanged
    out.zero_()
    assert sysm.rollout_streamed(hs, ha[:0].clone().pin_memory(), out, chunk_steps=10, bufs=bufs) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, hs)
    # and so does a device rollout of zero steps (no action is read)
    z = sysm.rollout(cuda(st), torch.zeros((0, N, sysm.A), device="cuda"))["state_T"]
    assert torch.equal(z.cpu(), hs)
