"""Python front end of the C ABI: systems, rollouts and their gradients on
PyTorch CUDA tensors.  Argument marshalling only; the work runs in
libbrax_gb300.so."""
from __future__ import annotations

import ctypes as C
import hashlib
import json
import math
import os

import numpy as np
import torch

from .binding import (BRAX_TUNE_FORWARD, BRAX_TUNE_REVERSE, _ptr, _stream, brax_tune_result, check, load_library,
                      marshal_desc)


def _f32(t, shape=None, name="tensor"):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def stream_chunks(T: int, chunk_steps: int, first_steps: int = 16):
    """Step ranges [t0, t1) of a streamed rollout: the first chunk has
    first_steps steps, each next one twice the previous, up to chunk_steps;
    together they cover 0..T once, in order."""
    C = max(1, min(int(chunk_steps), T))
    chunks, t0, n = [], 0, max(1, min(int(first_steps), C))
    while t0 < T:
        chunks.append((t0, min(T, t0 + n)))
        t0, n = t0 + n, min(C, 2 * n)
    return chunks


class BraxSystem:
    """One system (Sec. 4.1 system specification) uploaded to the current GPU."""

    def __init__(self, desc: dict):
        L = load_library()
        d, keep = marshal_desc(desc)
        h = C.c_void_p()
        check(L.brax_system_create(C.byref(d), C.byref(h)))
        self._L = L
        self._h = h
        self.desc = desc
        B, A, D = C.c_int32(), C.c_int32(), C.c_int32()
        check(L.brax_system_info(h, C.byref(B), C.byref(A), C.byref(D)))
        self.B, self.A, self.D = B.value, A.value, D.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.brax_system_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def set_launch(self, groups: int, variant: int):
        """Launch of the one-environment-per-thread kernel (groups of 32
        environments per block, launch-bounds variant 0..3)."""
        check(self._L.brax_system_set_launch(self._h, groups, variant))

    def set_pair_launch(self, mode: int, groups: int = 1, variant: int = 0):
        """Two-environments-per-thread kernel of hinge-only systems: mode 1
        uses it for rollout/step (groups of 64 environments per block), mode 0
        falls back to the one-environment kernel."""
        check(self._L.brax_system_set_pair_launch(self._h, mode, groups, variant))

    def set_schedule(self, mode: int, chunk_steps: int = 0, first_item: int = 0, wait_ns: int = 2_000_000_000):
        """Chunked schedule of paired rollouts (resident blocks take (chunk,
        environment block) items so that the last wave is not part-empty):
        mode 1 automatic (default), 0 never, 2 always with chunks of
        chunk_steps steps.  first_item and wait_ns exist for the test of the
        bounded wait."""
        check(self._L.brax_system_set_schedule(self._h, mode, chunk_steps, first_item, wait_ns))

    # ---------------------------------------------------------------- autotuner
    def _desc_digest(self) -> str:
        h = hashlib.sha1()
        for k in sorted(self.desc):
            h.update(k.encode())
            h.update(np.ascontiguousarray(np.asarray(self.desc[k])).tobytes() if not isinstance(self.desc[k], str)
                     else self.desc[k].encode())
        return h.hexdigest()

    def autotune(self, state0, actions, reverse: bool = False, mem_budget: int = 0, cache: str | None = None,
                 forward: bool = True):
        """Time the workload sample (state0 [N,B,13], actions [T,N,A]) under
        every launch configuration and keep the fastest (brax_autotune); with
        reverse=True also pick the checkpoint interval K.  Results are cached
        in the JSON file `cache` (key: system, device, N, T, what), and a
        cache hit applies the stored configuration without timing.  Returns a
        dict with the chosen configuration (K for the reverse pass)."""
        N, T = state0.shape[0], actions.shape[0]
        _f32(state0, (N, self.B, 13), "state0")
        _f32(actions, (T, N, self.A), "actions")
        flags = (BRAX_TUNE_FORWARD if forward else 0) | (BRAX_TUNE_REVERSE if reverse else 0)
        if not flags:
            raise ValueError("autotune: nothing to tune")
        key = f"{self._desc_digest()}|{torch.cuda.get_device_name()}|{N}|{T}|{flags}"
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
        if key in table:
            r = table[key]
            if forward:
                self.set_launch(r["scalar_groups"], r["scalar_variant"])
                if r["fwd_kernel"] == 1:
                    self.set_pair_launch(1, r["fwd_groups"], r["fwd_variant"])
                elif self.paired:
                    self.set_pair_launch(0)
            if r.get("bwd_variant", -1) >= 0:
                self._L.brax_system_set_backward_launch(self._h, r["bwd_variant"])
            return dict(r, cached=True)
        out = brax_tune_result()
        check(self._L.brax_autotune(self._h, N, T, _ptr(state0), _ptr(actions), flags, mem_budget, _stream(),
                                    C.byref(out)))
        g, v = C.c_int32(), C.c_int32()
        check(self._L.brax_system_get_launch(self._h, C.byref(g), C.byref(v)))
        r = {k: getattr(out, k) for k, _ in brax_tune_result._fields_}
        r.update(scalar_groups=g.value, scalar_variant=v.value)
        if cache:
            table[key] = r
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1)
            os.replace(tmp, cache)
        return dict(r, cached=False)

    def last_rollout(self) -> dict:
        """Launch of the last rollout: blocks, chunks of the chunked schedule
        (0 = static) and steps per chunk."""
        g, c, k = C.c_int64(), C.c_int32(), C.c_int32()
        check(self._L.brax_system_last_rollout(self._h, C.byref(g), C.byref(c), C.byref(k)))
        return {"grid": g.value, "n_chunks": c.value, "chunk_steps": k.value}

    @property
    def paired(self) -> bool:
        """True when the system has the two-environments-per-thread kernel."""
        m = C.c_int32()
        check(self._L.brax_system_get_pair_launch(self._h, C.byref(m)))
        return m.value >= 0

    # ---------------------------------------------------------------- forward
    def default_qp(self, n_envs, root_pos=None, root_rot=None, angles=None):
        out = torch.empty((n_envs, self.B, 13), device="cuda", dtype=torch.float32)
        check(self._L.brax_default_qp(self._h, n_envs, _ptr(_f32(root_pos, (n_envs, 3), "root_pos")),
                                      _ptr(_f32(root_rot, (n_envs, 4), "root_rot")),
                                      _ptr(_f32(angles, (n_envs, self.D), "angles")), _ptr(out), _stream()))
        return out

    def step(self, state, actions, out=None):
        N = state.shape[0]
        _f32(state, (N, self.B, 13), "state")
        _f32(actions, (N, self.A), "actions")
        out = torch.empty_like(state) if out is None else _f32(out, (N, self.B, 13), "out")
        check(self._L.brax_step(self._h, N, _ptr(state), _ptr(actions), _ptr(out), _stream()))
        return out

    def rollout(self, state0, actions, K=1, checkpoints=False, torso=False, contact_count=False, state_T=None):
        """T steps in one persistent launch.  Returns a dict with state_T and
        the requested checkpoints [ceil(T/K),N,B,13], torso [T,N,3] and
        contact_count [N]."""
        N = state0.shape[0]
        T = actions.shape[0]
        _f32(state0, (N, self.B, 13), "state0")
        _f32(actions, (T, N, self.A), "actions")
        out = {"state_T": torch.empty_like(state0) if state_T is None else state_T}
        if checkpoints:
            out["checkpoints"] = torch.empty((math.ceil(T / K), N, self.B, 13), device="cuda", dtype=torch.float32)
        if torso:
            out["torso"] = torch.empty((T, N, 3), device="cuda", dtype=torch.float32)
        if contact_count:
            out["contact_count"] = torch.zeros((N,), device="cuda", dtype=torch.int32)
        check(self._L.brax_rollout(self._h, N, T, K, _ptr(state0), _ptr(actions), _ptr(out["state_T"]),
                                   _ptr(out.get("checkpoints")), _ptr(out.get("torso")),
                                   _ptr(out.get("contact_count")), _stream()))
        return out

    def env_obs_size(self) -> int:
        n = C.c_int32()
        check(self._L.brax_env_obs_size(self._h, C.byref(n)))
        return n.value

    def env_rollout(self, state0, actions, reset_state=None, forward_weight=1.0, healthy_reward=1.0, ctrl_cost=0.5,
                    min_z=0.2, max_z=1.0, auto_reset=True, state_T=None):
        """T steps of the gym-like environment layer (brax_env_rollout):
        returns a dict with state_T [N,B,13], obs [T,N,D], reward [T,N] and
        done [T,N] (uint8).  reset_state defaults to state0."""
        from .binding import brax_env_params
        N, T = state0.shape[0], actions.shape[0]
        _f32(state0, (N, self.B, 13), "state0")
        _f32(actions, (T, N, self.A), "actions")
        reset_state = state0 if reset_state is None else _f32(reset_state, (N, self.B, 13), "reset_state")
        D = self.env_obs_size()
        out = {"state_T": torch.empty_like(state0) if state_T is None else state_T,
               "obs": torch.empty((T, N, D), device="cuda", dtype=torch.float32),
               "reward": torch.empty((T, N), device="cuda", dtype=torch.float32),
               "done": torch.empty((T, N), device="cuda", dtype=torch.uint8)}
        p = brax_env_params(forward_weight, healthy_reward, ctrl_cost, min_z, max_z, 1 if auto_reset else 0)
        check(self._L.brax_env_rollout(self._h, C.byref(p), N, T, _ptr(state0), _ptr(reset_state), _ptr(actions),
                                       _ptr(out["state_T"]), _ptr(out["obs"]), _ptr(out["reward"]),
                                       _ptr(out["done"]), _stream()))
        return out

    def rollout_streamed(self, h_state0, h_actions, h_state_T, chunk_steps: int = 100, bufs: dict | None = None,
                         first_steps: int = 16):
        """Rollout whose inputs and output live in pinned host memory
        (brax_rollout_streamed): the actions stream to the device in chunks on
        the system's copy stream while the previous chunk is being stepped,
        and the final state is copied back into the pinned h_state_T.  Chunks
        start at `first_steps` steps and double up to `chunk_steps`; the
        result equals one launch over all steps.  `bufs` (a dict, filled on
        first use) keeps the device workspace between calls.  Returns the
        number of rollout launches."""
        N, T = h_state0.shape[0], h_actions.shape[0]
        if not all(t.is_pinned() for t in (h_state0, h_actions, h_state_T) if t.numel()):
            raise ValueError("rollout_streamed: host tensors must be pinned")
        for t, shape, name in ((h_state0, (N, self.B, 13), "h_state0"), (h_actions, (T, N, self.A), "h_actions"),
                               (h_state_T, (N, self.B, 13), "h_state_T")):
            if t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"{name}: expected a contiguous float32 tensor of shape {shape}")
        bufs = {} if bufs is None else bufs
        Cn = max(1, min(int(chunk_steps), max(T, 1)))
        nbytes = C.c_size_t()
        check(self._L.brax_streamed_workspace_size(self._h, N, Cn, C.byref(nbytes)))
        ws = bufs.get("ws")
        if ws is None or ws.numel() < nbytes.value:
            ws = bufs["ws"] = torch.empty((max(nbytes.value, 1),), device="cuda", dtype=torch.uint8)
        check(self._L.brax_rollout_streamed(self._h, N, T, h_state0.data_ptr(), h_actions.data_ptr(),
                                            h_state_T.data_ptr(), Cn, int(first_steps), _ptr(ws), ws.numel(),
                                            _stream()))
        return len(stream_chunks(T, Cn, first_steps)) if T > 0 else 0

    # ---------------------------------------------------------------- backward
    def workspace_size(self, n_envs, T, K):
        b = C.c_size_t()
        check(self._L.brax_workspace_size(self._h, n_envs, T, K, C.byref(b)))
        return b.value

    def rollout_backward(self, state0, actions, checkpoints, g_state_T, g_torso=None, K=1, workspace=None):
        N = state0.shape[0]
        T = actions.shape[0]
        _f32(state0, (N, self.B, 13), "state0")
        _f32(actions, (T, N, self.A), "actions")
        _f32(checkpoints, (math.ceil(T / K), N, self.B, 13), "checkpoints")
        _f32(g_state_T, (N, self.B, 13), "g_state_T")
        _f32(g_torso, (T, N, 3), "g_torso")
        nbytes = self.workspace_size(N, T, K)
        if workspace is None or workspace.numel() < nbytes:
            workspace = torch.empty((max(nbytes, 1),), device="cuda", dtype=torch.uint8)
        g_actions = torch.empty_like(actions)
        g_state0 = torch.empty_like(state0)
        check(self._L.brax_rollout_backward(self._h, N, T, K, _ptr(state0), _ptr(actions), _ptr(checkpoints),
                                            _ptr(g_state_T), _ptr(g_torso), _ptr(g_actions), _ptr(g_state0),
                                            _ptr(workspace), workspace.numel(), _stream()))
        return g_actions, g_state0

    def rollout_backward_noalloc(self, state0, actions, checkpoints, g_state_T, g_torso=None, K=1):
        """rollout_backward without a caller workspace: the library's own
        fixed scratch array is used (see brax_rollout_backward_noalloc in
        include/brax.h for its size limit and sharing rules).  Only the two
        output tensors are created here; the library allocates nothing."""
        N = state0.shape[0]
        T = actions.shape[0]
        _f32(state0, (N, self.B, 13), "state0")
        _f32(actions, (T, N, self.A), "actions")
        _f32(checkpoints, (math.ceil(T / K), N, self.B, 13), "checkpoints")
        _f32(g_state_T, (N, self.B, 13), "g_state_T")
        _f32(g_torso, (T, N, 3), "g_torso")
        g_actions = torch.empty_like(actions)
        g_state0 = torch.empty_like(state0)
        check(self._L.brax_rollout_backward_noalloc(self._h, N, T, K, _ptr(state0), _ptr(actions), _ptr(checkpoints),
                                                    _ptr(g_state_T), _ptr(g_torso), _ptr(g_actions), _ptr(g_state0),
                                                    _stream()))
        return g_actions, g_state0

    def sync_status(self):
        """Synchronise the current stream; raise if a kernel saw a non-finite state."""
        check(self._L.brax_sync_status(self._h, _stream()))


class BraxBatch:
    """Systems of different sizes stepped in one launch (forward and reverse).

    Arrays are concatenations over systems of the per-system arrays: state
    blocks [N_i, B_i, 13], action blocks [T, N_i, A_i], torso blocks
    [T, N_i, 3], checkpoint blocks [ceil(T/K), N_i, B_i, 13].
    """

    def __init__(self, systems, n_envs):
        L = load_library()
        self._L = L
        self.systems = list(systems)
        self.n_envs = [int(n) for n in n_envs]
        arr = (C.c_void_p * len(self.systems))(*[s.handle.value for s in self.systems])
        ns = (C.c_int64 * len(self.systems))(*self.n_envs)
        h = C.c_void_p()
        check(L.brax_batch_create(arr, ns, len(self.systems), C.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.brax_batch_destroy(h)
            self._h = None

    def set_schedule(self, mode: int, chunk_steps: int = 0):
        """Chunked schedule of the batch's forward rollouts (as
        BraxSystem.set_schedule): 1 automatic (default), 0 never, 2 always."""
        check(self._L.brax_batch_set_schedule(self._h, mode, chunk_steps))

    def sizes(self, T, K=1):
        """Total elements of the state, action, torso and checkpoint arrays."""
        st = sum(n * s.B * 13 for s, n in zip(self.systems, self.n_envs))
        ac = sum(T * n * s.A for s, n in zip(self.systems, self.n_envs))
        to = sum(T * n * 3 for n in self.n_envs)
        ck = sum(math.ceil(T / K) * n * s.B * 13 for s, n in zip(self.systems, self.n_envs))
        return st, ac, to, ck

    def offsets(self, T, K, i):
        o = [C.c_int64() for _ in range(4)]
        check(self._L.brax_batch_offsets(self._h, T, K, i, *[C.byref(x) for x in o]))
        return tuple(x.value for x in o)

    def rollout(self, state0, actions, T, K=1, checkpoints=False, torso=False):
        st_n, ac_n, to_n, ck_n = self.sizes(T, K)
        if state0.numel() != st_n or actions.numel() != ac_n:
            raise ValueError("batch arrays do not match the systems' sizes")
        out = {"state_T": torch.empty_like(state0)}
        if checkpoints:
            out["checkpoints"] = torch.empty((ck_n,), device="cuda", dtype=torch.float32)
        if torso:
            out["torso"] = torch.empty((to_n,), device="cuda", dtype=torch.float32)
        check(self._L.brax_batch_rollout(self._h, T, K, _ptr(state0), _ptr(actions), _ptr(out["state_T"]),
                                         _ptr(out.get("checkpoints")), _ptr(out.get("torso")), _stream()))
        return out

    def workspace_size(self, T, K):
        b = C.c_size_t()
        check(self._L.brax_batch_workspace_size(self._h, T, K, C.byref(b)))
        return b.value

    def autotune(self, state0, actions, T, K=10, reverse=False):
        """Pick the block size (warps per block) by timing this batch's own
        arrays (brax_batch_autotune); returns (warps, ms)."""
        w, ms = C.c_int32(), C.c_float()
        flags = BRAX_TUNE_FORWARD | (BRAX_TUNE_REVERSE if reverse else 0)
        check(self._L.brax_batch_autotune(self._h, T, K, _ptr(state0), _ptr(actions), flags, _stream(), C.byref(w),
                                          C.byref(ms)))
        return w.value, ms.value

    def rollout_backward(self, state0, actions, checkpoints, g_state_T, T, K=1, g_torso=None, workspace=None):
        nbytes = self.workspace_size(T, K)
        if workspace is None or workspace.numel() < nbytes:
            workspace = torch.empty((max(nbytes, 1),), device="cuda", dtype=torch.uint8)
        g_actions = torch.empty_like(actions)
        g_state0 = torch.empty_like(state0)
        check(self._L.brax_batch_rollout_backward(self._h, T, K, _ptr(state0), _ptr(actions), _ptr(checkpoints),
                                                  _ptr(g_state_T), _ptr(g_torso), _ptr(g_actions), _ptr(g_state0),
                                                  _ptr(workspace), workspace.numel(), _stream()))
        return g_actions, g_state0
