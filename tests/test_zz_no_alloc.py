"""The reverse pass without a caller workspace (GPU).

brax_rollout_backward_noalloc serves callers that cannot allocate device
memory when they need a gradient: it takes its scratch from a fixed array
inside the library instead of a caller workspace.  These checks call it
through the C ABI twice in a row (the array keeps the previous call's
contents) and compare with brax_rollout_backward given a workspace, and
check that a rollout needing more scratch than the array holds is refused
with a clear error.  This file is collected last so that a failure here
leaves every other test already run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2106_13281_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def system():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_13281_gb300.system import BraxSystem
    return BraxSystem(S.quadruped())


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


def inputs(d, N, T, seed):
    rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
    rp[:, 2] -= 0.38
    st = orc.default_qp(d, N, rp, rr, ang)
    return cuda(st), cuda(S.actions(d, N, T, seed))


def test_noalloc_matches_workspace_entry_point_twice(system):
    d = system.desc
    N, T, K = 200, 12, 4
    for call, seed in enumerate((51, 52)):
        st, a = inputs(d, N, T, seed)
        out = system.rollout(st, a, K=K, checkpoints=True)
        rng = np.random.default_rng(seed)
        gT = cuda(rng.normal(size=(N, system.B, 13)))
        gtor = cuda(rng.normal(size=(T, N, 3)))
        ref_a, ref_s = system.rollout_backward(st, a, out["checkpoints"], gT, gtor, K=K)
        got_a, got_s = system.rollout_backward_noalloc(st, a, out["checkpoints"], gT, gtor, K=K)
        system.sync_status()
        assert torch.isfinite(got_a).all() and torch.isfinite(got_s).all()
        assert torch.allclose(got_a, ref_a, rtol=1e-5, atol=1e-6), call
        assert torch.allclose(got_s, ref_s, rtol=1e-5, atol=1e-6), call


def test_noalloc_refuses_rollouts_beyond_its_scratch(system):
    from paper_2106_13281_gb300.binding import BraxError
    d = system.desc
    N, T, K = 65536, 20, 10
    assert system.workspace_size(N, T, K) > (32 << 20)
    st = torch.zeros((N, system.B, 13), device="cuda")
    a = torch.zeros((T, N, system.A), device="cuda")
    ck = torch.zeros((2, N, system.B, 13), device="cuda")
    with pytest.raises(BraxError) as ei:
        system.rollout_backward_noalloc(st, a, ck, torch.zeros_like(st), K=K)
    assert ei.value.code == 7 and "scratch" in str(ei.value)


def test_noalloc_chunked_schedule_allocates_nothing():
    """With the chunked schedule forced on (chunks of two checkpoint
    segments), the entry point takes the schedule's counter and flags from its
    own array: two calls in a row on a fresh system match the static-schedule
    reverse pass given a workspace, and the device's free memory does not
    change across them (after a first call that sets the array up)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_13281_gb300.binding import _ptr, _stream, check
    from paper_2106_13281_gb300.system import BraxSystem
    d = S.quadruped()
    chunked = BraxSystem(d)
    chunked.set_schedule(2, 2)
    static = BraxSystem(d)
    static.set_schedule(0)
    N, T, K = 200, 12, 4
    runs = []
    for seed in (61, 62):
        st, a = inputs(d, N, T, seed)
        ck = static.rollout(st, a, K=K, checkpoints=True)["checkpoints"]
        rng = np.random.default_rng(seed)
        gT = cuda(rng.normal(size=(N, static.B, 13)))
        gtor = cuda(rng.normal(size=(T, N, 3)))
        ref = static.rollout_backward(st, a, ck, gT, gtor, K=K)
        runs.append((st, a, ck, gT, gtor, ref, torch.empty_like(a), torch.empty_like(st)))
    L = chunked._L

    def call(r):
        st, a, ck, gT, gtor, _, ga, gs = r
        check(L.brax_rollout_backward_noalloc(chunked.handle, N, T, K, _ptr(st), _ptr(a), _ptr(ck), _ptr(gT),
                                              _ptr(gtor), _ptr(ga), _ptr(gs), _stream()))

    call(runs[0])  # first call on the device: looks the array up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for r in runs:
        call(r)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    chunked.sync_status()
    assert free1 == free0, (free0, free1)
    for st, a, ck, gT, gtor, (ref_a, ref_s), ga, gs in runs:
        assert torch.isfinite(ga).all() and torch.isfinite(gs).all()
        assert torch.allclose(ga, ref_a, rtol=1e-5, atol=1e-6)
        assert torch.allclose(gs, ref_s, rtol=1e-5, atol=1e-6)
