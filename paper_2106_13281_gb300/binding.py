"""ctypes binding of libbrax_gb300.so (the C ABI in include/brax.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  There is
no CPU fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbrax_gb300.so")

BRAX_DESC_VERSION = 2
STATUS = {0: "OK", 1: "INVALID_ARGUMENT", 2: "INVALID_DESCRIPTOR", 3: "CUDA", 4: "OUT_OF_MEMORY",
          5: "NONFINITE", 6: "TIMEOUT", 7: "WORKSPACE"}

# Every symbol include/brax.h declares.
EXPORTS = ["brax_system_create", "brax_system_destroy", "brax_system_info", "brax_default_qp", "brax_step",
           "brax_rollout", "brax_workspace_size", "brax_rollout_backward", "brax_batch_create",
           "brax_batch_destroy", "brax_batch_offsets", "brax_batch_rollout", "brax_batch_workspace_size",
           "brax_batch_rollout_backward", "brax_sync_status", "brax_last_error", "brax_rollout_backward_noalloc",
           "brax_autotune", "brax_batch_autotune", "brax_env_obs_size", "brax_env_rollout",
           "brax_streamed_workspace_size", "brax_rollout_streamed"]

BRAX_TUNE_FORWARD, BRAX_TUNE_REVERSE = 1, 2


class BraxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"brax error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code


class brax_env_params(C.Structure):
    _fields_ = [("forward_weight", C.c_float), ("healthy_reward", C.c_float), ("ctrl_cost", C.c_float),
                ("min_z", C.c_float), ("max_z", C.c_float), ("auto_reset", C.c_int32)]


class brax_tune_result(C.Structure):
    _fields_ = [("fwd_kernel", C.c_int32), ("fwd_groups", C.c_int32), ("fwd_variant", C.c_int32),
                ("fwd_ms", C.c_float), ("K", C.c_int32), ("bwd_variant", C.c_int32),
                ("fwd_bwd_ms_per_step", C.c_float), ("n_candidates", C.c_int32)]


class brax_desc(C.Structure):
    _fields_ = [
        ("version", C.c_int32), ("n_bodies", C.c_int32), ("n_joints", C.c_int32), ("n_actuators", C.c_int32),
        ("n_colliders", C.c_int32), ("n_pairs", C.c_int32), ("substeps", C.c_int32),
        ("dt", C.c_float), ("gravity", C.c_float * 3), ("baumgarte", C.c_float), ("contact_eps", C.c_float),
        ("average_contacts", C.c_int32),
        ("mass", C.c_void_p), ("inertia", C.c_void_p), ("rest_pos", C.c_void_p), ("rest_rot", C.c_void_p),
        ("frozen_pos", C.c_void_p), ("frozen_rot", C.c_void_p),
        ("parent", C.c_void_p), ("child", C.c_void_p), ("dof", C.c_void_p),
        ("parent_offset", C.c_void_p), ("child_offset", C.c_void_p),
        ("parent_frame", C.c_void_p), ("child_frame", C.c_void_p),
        ("stiffness", C.c_void_p), ("spring_damping", C.c_void_p), ("angular_stiffness", C.c_void_p),
        ("angular_damping", C.c_void_p), ("limit_lo", C.c_void_p), ("limit_hi", C.c_void_p),
        ("limit_stiffness", C.c_void_p),
        ("act_joint", C.c_void_p), ("act_axis", C.c_void_p), ("gear", C.c_void_p),
        ("col_body", C.c_void_p), ("col_type", C.c_void_p), ("col_pos", C.c_void_p), ("col_rot", C.c_void_p),
        ("radius", C.c_void_p), ("length", C.c_void_p), ("half_extents", C.c_void_p),
        ("friction", C.c_void_p), ("elasticity", C.c_void_p),
        ("pair_a", C.c_void_p), ("pair_b", C.c_void_p),
        ("linear_damping", C.c_float), ("angular_damping_global", C.c_float), ("gyroscopic", C.c_int32),
        ("act_type", C.c_void_p),
    ]


_F32 = ["mass", "inertia", "rest_pos", "rest_rot", "parent_offset", "child_offset", "parent_frame", "child_frame",
        "stiffness", "spring_damping", "angular_stiffness", "angular_damping", "limit_lo", "limit_hi",
        "limit_stiffness", "gear", "col_pos", "col_rot", "radius", "length", "half_extents", "friction", "elasticity"]
_I32 = ["parent", "child", "dof", "act_joint", "act_axis", "col_body", "col_type", "pair_a", "pair_b"]
_U8 = ["frozen_pos", "frozen_rot"]

_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbrax_gb300.so (build it with paper_2106_13281_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(path)
        P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.brax_last_error.restype = C.c_char_p
        L.brax_system_create.argtypes = [C.POINTER(brax_desc), C.POINTER(C.c_void_p)]
        L.brax_system_destroy.argtypes = [P]
        L.brax_system_destroy.restype = None
        L.brax_system_info.argtypes = [P, P, P, P]
        L.brax_default_qp.argtypes = [P, i64, P, P, P, P, P]
        L.brax_step.argtypes = [P, i64, P, P, P, P]
        L.brax_rollout.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, P]
        L.brax_workspace_size.argtypes = [P, i64, i32, i32, C.POINTER(C.c_size_t)]
        L.brax_rollout_backward.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, P, P, C.c_size_t, P]
        L.brax_batch_create.argtypes = [P, P, i32, C.POINTER(C.c_void_p)]
        L.brax_batch_destroy.argtypes = [P]
        L.brax_batch_destroy.restype = None
        L.brax_batch_offsets.argtypes = [P, i32, i32, i32, P, P, P, P]
        L.brax_batch_rollout.argtypes = [P, i32, i32, P, P, P, P, P, P]
        L.brax_batch_workspace_size.argtypes = [P, i32, i32, C.POINTER(C.c_size_t)]
        L.brax_batch_rollout_backward.argtypes = [P, i32, i32, P, P, P, P, P, P, P, P, C.c_size_t, P]
        L.brax_sync_status.argtypes = [P, P]
        L.brax_autotune.argtypes = [P, i64, i32, P, P, i32, C.c_size_t, P, C.POINTER(brax_tune_result)]
        L.brax_batch_autotune.argtypes = [P, i32, i32, P, P, i32, P, C.POINTER(i32), C.POINTER(C.c_float)]
        L.brax_rollout_backward_noalloc.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, P, P]
        L.brax_env_obs_size.argtypes = [P, C.POINTER(i32)]
        L.brax_streamed_workspace_size.argtypes = [P, i64, i32, C.POINTER(C.c_size_t)]
        L.brax_rollout_streamed.argtypes = [P, i64, i32, P, P, P, i32, i32, P, C.c_size_t, P]
        L.brax_env_rollout.argtypes = [P, C.POINTER(brax_env_params), i64, i32, P, P, P, P, P, P, P, P]
        if hasattr(L, "brax_system_set_launch"):
            L.brax_system_set_launch.argtypes = [P, i32, i32]
        if hasattr(L, "brax_system_set_pair_launch"):
            L.brax_system_set_pair_launch.argtypes = [P, i32, i32, i32]
            L.brax_system_get_launch.argtypes = [P, C.POINTER(i32), C.POINTER(i32)]
            L.brax_system_get_pair_launch.argtypes = [P, C.POINTER(i32)]
            L.brax_system_set_backward_launch.argtypes = [P, i32]
        if hasattr(L, "brax_system_last_rollout"):
            L.brax_system_last_rollout.argtypes = [P, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)]
        if hasattr(L, "brax_internal_atan2"):
            L.brax_internal_atan2.argtypes = [P, P, P, P, i64, P]
        if hasattr(L, "brax_system_set_schedule"):
            L.brax_system_set_schedule.argtypes = [P, i32, i32, i32, i64]
            L.brax_batch_set_schedule.argtypes = [P, i32, i32]
        _lib = L
        return L


def check(code: int):
    if code != 0:
        raise BraxError(code, load_library().brax_last_error().decode())


def last_error() -> str:
    return load_library().brax_last_error().decode()


def marshal_desc(desc: dict):
    """Build a brax_desc from a scene dict; returns (struct, keep-alive list)."""
    keep = []
    d = brax_desc()
    d.version = BRAX_DESC_VERSION
    d.n_bodies = len(desc["mass"])
    d.n_joints = len(desc["parent"])
    d.n_actuators = len(desc["act_joint"])
    d.n_colliders = len(desc["col_body"])
    d.n_pairs = len(desc["pair_a"])
    d.substeps = int(desc["substeps"])
    d.dt = float(desc["dt"])
    for i in range(3):
        d.gravity[i] = float(desc["gravity"][i])
    d.baumgarte = float(desc["baumgarte"])
    d.contact_eps = float(desc["contact_eps"])
    d.average_contacts = int(desc.get("average_contacts", 1))
    d.linear_damping = float(desc.get("linear_damping", 0.0))
    d.angular_damping_global = float(desc.get("angular_damping_global", 0.0))
    d.gyroscopic = int(desc.get("gyroscopic", 0))
    for keys, dt in ((_F32, np.float32), (_I32, np.int32), (_U8, np.uint8)):
        for k in keys:
            a = np.ascontiguousarray(np.asarray(desc[k]), dtype=dt)
            keep.append(a)
            setattr(d, k, a.ctypes.data if a.size else None)
    if "act_type" in desc and len(desc["act_type"]):
        a = np.ascontiguousarray(np.asarray(desc["act_type"]), dtype=np.int32)
        keep.append(a)
        d.act_type = a.ctypes.data
    return d, keep


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream
