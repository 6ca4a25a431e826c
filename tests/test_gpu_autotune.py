"""The autotuner (brax_autotune): it times real candidates, applies the
fastest, keeps results correct, and its JSON cache round-trips (GPU)."""
import os

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


@pytest.mark.parametrize("name", ["quadruped", "biped"])
def test_autotune_applies_a_timed_configuration(brax, name, tmp_path):
    d = S.SCENES[name]()
    sysm = brax(d)
    N, T = 2048, 20
    rp, rr, ang = S.initial_conditions(d, N, 3, height_jitter=0.05)
    st = orc.default_qp(d, N, rp, rr, ang)
    a = S.actions(d, N, T, 4)
    cache = os.path.join(tmp_path, "tune.json")
    r = sysm.autotune(cuda(st), cuda(a), reverse=True, cache=cache)
    assert not r["cached"] and r["n_candidates"] > 4
    assert r["fwd_ms"] > 0 and r["fwd_bwd_ms_per_step"] > 0
    assert 1 <= r["K"] <= T and r["bwd_variant"] in (0, 1, 2, 3, 4)
    if name == "biped":  # general systems have no two-environments kernel
        assert r["fwd_kernel"] == 0
    # the tuned configuration still computes the same step as the oracle
    st1 = st[:64]
    ref = orc.rollout(d, st1, a[:1, :64].astype(np.float64))
    got = sysm.rollout(cuda(st1), cuda(a[:1, :64]))["state_T"].cpu().numpy()
    assert np.abs(got[..., :3] - ref[..., :3]).max() < 1e-5
    # and its gradients match the default configuration's: the same arithmetic,
    # up to the order of the float atomics that sum body-body pair adjoints
    # (biped self-collision), which varies between runs
    K = r["K"]
    out = sysm.rollout(cuda(st1), cuda(a[:, :64]), K=K, checkpoints=True)
    g = torch.ones((64, sysm.B, 13), device="cuda")
    ga, gs = sysm.rollout_backward(cuda(st1), cuda(a[:, :64]), out["checkpoints"], g, None, K=K)
    fresh = brax(d)
    out2 = fresh.rollout(cuda(st1), cuda(a[:, :64]), K=K, checkpoints=True)
    ga2, gs2 = fresh.rollout_backward(cuda(st1), cuda(a[:, :64]), out2["checkpoints"], g, None, K=K)
    rel = lambda x, y: ((x - y).norm() / y.norm()).item()
    assert rel(ga, ga2) < 1e-4 and rel(gs, gs2) < 1e-4
    # a second system of the same description reads the cache without timing
    other = brax(d)
    r2 = other.autotune(cuda(st), cuda(a), reverse=True, cache=cache)
    assert r2["cached"] and r2["K"] == r["K"] and r2["fwd_kernel"] == r["fwd_kernel"]
    assert r2["fwd_groups"] == r["fwd_groups"] and r2["fwd_variant"] == r["fwd_variant"]


def test_autotune_respects_the_memory_budget(brax):
    """A budget too small for any checkpoint interval of the whole rollout is
    reported, not exceeded; a budget that admits only large K picks one of
    those."""
    from paper_2106_13281_gb300.binding import BraxError
    d = S.quadruped()
    sysm = brax(d)
    N, T = 1024, 40
    rp, rr, ang = S.initial_conditions(d, N, 5, height_jitter=0.05)
    st = cuda(orc.default_qp(d, N, rp, rr, ang))
    a = cuda(S.actions(d, N, T, 6))
    with pytest.raises(BraxError) as ei:
        sysm.autotune(st, a, reverse=True, forward=False, mem_budget=1024)
    assert ei.value.code == 4
    state_bytes = N * sysm.B * 13 * 4
    need = lambda K: -(-T // K) * state_bytes + sysm.workspace_size(N, T, K)
    budget = need(10)  # admits K = 10; K = 1 and 2 need more
    assert need(1) > budget and need(2) > budget
    r = sysm.autotune(st, a, reverse=True, forward=False, mem_budget=budget)
    assert r["K"] > 2 and need(r["K"]) <= budget
