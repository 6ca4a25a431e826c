"""Python wrapper of the FP64 oracle (ctypes over liborc.so).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, FP64 CPU statement
of the batched rigid-body step (Brax, Sec. 3 Algorithm 1) that the CUDA path
is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this module.  It shares no
code with the CUDA path and imports nothing from the product package.

Descriptors are plain dicts of numpy arrays (the seeded scene generators
produce them); arrays follow the QP layout: state [N, B, 13] with per body
(pos[3], quat[4] (w,x,y,z), vel[3], angvel[3]), actions [T, N, A].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liborc.so")
_SOURCES = ["oracle_capi.cpp", "oracle.hpp", "scalars.hpp"]
_lock = threading.Lock()
_lib = None

FLOP_CATEGORIES = ["body", "joint", "actuator", "detect", "response", "integrate", "other"]


def build(force: bool = False) -> str:
    """Compile liborc.so with g++ (portable flags: builds on x86_64 and aarch64)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB):
        t = os.path.getmtime(_LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    # -ffp-contract=off: no fused multiply-adds, so the FP64 results (and every
    # branch decision taken on them) are the same on x86_64 and aarch64.
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp,
           os.path.join(_HERE, "oracle_capi.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Desc(C.Structure):
    _fields_ = [
        ("n_bodies", C.c_int32), ("n_joints", C.c_int32), ("n_actuators", C.c_int32),
        ("n_colliders", C.c_int32), ("n_pairs", C.c_int32), ("substeps", C.c_int32),
        ("dt", C.c_double), ("gravity", C.c_double * 3), ("baumgarte", C.c_double),
        ("contact_eps", C.c_double), ("average_contacts", C.c_int32),
        ("mass", C.c_void_p), ("inertia", C.c_void_p), ("rest_pos", C.c_void_p), ("rest_rot", C.c_void_p),
        ("frozen_pos", C.c_void_p), ("frozen_rot", C.c_void_p),
        ("parent", C.c_void_p), ("child", C.c_void_p), ("dof", C.c_void_p),
        ("parent_offset", C.c_void_p), ("child_offset", C.c_void_p),
        ("parent_frame", C.c_void_p), ("child_frame", C.c_void_p),
        ("stiffness", C.c_void_p), ("spring_damping", C.c_void_p),
        ("angular_stiffness", C.c_void_p), ("angular_damping", C.c_void_p),
        ("limit_lo", C.c_void_p), ("limit_hi", C.c_void_p), ("limit_stiffness", C.c_void_p),
        ("act_joint", C.c_void_p), ("act_axis", C.c_void_p), ("gear", C.c_void_p),
        ("col_body", C.c_void_p), ("col_type", C.c_void_p), ("col_pos", C.c_void_p),
        ("col_rot", C.c_void_p), ("radius", C.c_void_p), ("length", C.c_void_p),
        ("half_extents", C.c_void_p), ("friction", C.c_void_p), ("elasticity", C.c_void_p),
        ("pair_a", C.c_void_p), ("pair_b", C.c_void_p),
        ("linear_damping", C.c_double), ("angular_damping_global", C.c_double), ("gyroscopic", C.c_int32),
        ("act_type", C.c_void_p),
    ]


_F64 = ["mass", "inertia", "rest_pos", "rest_rot", "parent_offset", "child_offset", "parent_frame",
        "child_frame", "stiffness", "spring_damping", "angular_stiffness", "angular_damping", "limit_lo",
        "limit_hi", "limit_stiffness", "gear", "col_pos", "col_rot", "radius", "length", "half_extents",
        "friction", "elasticity"]
_I32 = ["parent", "child", "dof", "act_joint", "act_axis", "col_body", "col_type", "pair_a", "pair_b"]
_U8 = ["frozen_pos", "frozen_rot"]


class OracleSystem:
    """A descriptor marshalled for the oracle (keeps its arrays alive)."""

    def __init__(self, desc: dict):
        self.desc = desc
        self._keep = {}
        d = _Desc()
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
        if "act_type" in desc:
            self._set(d, "act_type", np.ascontiguousarray(desc["act_type"], dtype=np.int32))
        for k in _F64:
            self._set(d, k, np.ascontiguousarray(desc[k], dtype=np.float64))
        for k in _I32:
            self._set(d, k, np.ascontiguousarray(desc[k], dtype=np.int32))
        for k in _U8:
            self._set(d, k, np.ascontiguousarray(desc[k], dtype=np.uint8))
        self.c = d
        self.B = d.n_bodies
        self.A = d.n_actuators
        self.D = int(np.sum(desc["dof"])) if d.n_joints else 0

    def _set(self, d, k, arr):
        self._keep[k] = arr
        setattr(d, k, arr.ctypes.data if arr.size else None)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            i64, i32 = C.c_int64, C.c_int32
            L.orc_rollout.argtypes = [P, i64, i32, P, P, P, P, P, P, i32]
            L.orc_flops.argtypes = [P, i64, i32, P, P, P, P]
            L.orc_vjp.argtypes = [P, i64, i32, P, P, P, P, P, P, i32]
            L.orc_reverse_flops.argtypes = [P, i64, i32, P, P, P, i32]
            L.orc_jvp.argtypes = [P, i64, i32, P, P, P, P, P, P, i32]
            L.orc_default_qp.argtypes = [P, i64, P, P, P, P]
            L.orc_joint_angles.argtypes = [P, i64, P, P]
            L.orc_joint_state.argtypes = [P, i64, P, P, P]
            L.orc_energy.argtypes = [P, i64, P, P, P]
            L.orc_contacts.argtypes = [P, P, i32, P, P]
            L.orc_segment_closest.argtypes = [P, P, P, P, P]
            L.orc_segment_closest.restype = None
            L.orc_capsule_box.argtypes = [P, P, C.c_double, P, P, P, P]
            L.orc_seg_box_param.argtypes = [P, P, P]
            L.orc_seg_box_param.restype = C.c_double
            _lib = L
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _sys(s):
    return s if isinstance(s, OracleSystem) else OracleSystem(s)


def _threads(n_threads):
    return n_threads if n_threads else (os.cpu_count() or 1)


def rollout(system, state0, actions, traj=False, n_threads=0, contact_count=False, branch_signature=False):
    """FP64 rollout.  state0 [N,B,13], actions [T,N,A] -> state_T [N,B,13]
    (+ traj [T,N,B,13] of states after every step, + active contacts [N],
    + a hash of every branch decision taken [N] (contact activation,
    friction stick/slip, limits, action clamps))."""
    s = _sys(system)
    state0 = _f64(state0)
    actions = _f64(actions)
    T, N = actions.shape[0], state0.shape[0]
    out = np.empty_like(state0)
    tr = np.empty((T, N, s.B, 13)) if traj else None
    cc = np.zeros(N, dtype=np.int64) if contact_count else None
    sig = np.zeros(N, dtype=np.uint64) if branch_signature else None
    lib().orc_rollout(C.byref(s.c), N, T, _p(state0), _p(actions), _p(out), _p(tr), _p(cc), _p(sig),
                      _threads(n_threads))
    res = [out]
    if traj:
        res.append(tr)
    if contact_count:
        res.append(cc)
    if branch_signature:
        res.append(sig)
    return res[0] if len(res) == 1 else tuple(res)


def flops(system, state0, actions):
    """Algorithmic flop counts of a rollout by category + active contact count."""
    s = _sys(system)
    state0 = _f64(state0)
    actions = _f64(actions)
    counts = np.zeros(7, dtype=np.int64)
    na = np.zeros(1, dtype=np.int64)
    lib().orc_flops(C.byref(s.c), state0.shape[0], actions.shape[0], _p(state0), _p(actions), _p(counts), _p(na))
    return dict(zip(FLOP_CATEGORIES, counts.tolist())), int(na[0])


def reverse_flops(system, state0, actions, n_threads=0):
    """Algorithmic flops of the reverse pass of a rollout (the tape's
    reverse-op count), summed over environments, and the tape's node count."""
    s = _sys(system)
    state0 = _f64(state0)
    actions = _f64(actions)
    out = np.zeros(2, dtype=np.int64)
    lib().orc_reverse_flops(C.byref(s.c), state0.shape[0], actions.shape[0], _p(state0), _p(actions), _p(out),
                            _threads(n_threads))
    return int(out[0]), int(out[1])


def vjp(system, state0, actions, g_state_T, g_torso=None, n_threads=0):
    """Reverse-mode gradient through the tape: returns (g_actions [T,N,A], g_state0 [N,B,13])."""
    s = _sys(system)
    state0, actions, g_state_T, g_torso = map(_f64, (state0, actions, g_state_T, g_torso))
    ga = np.zeros_like(actions)
    gs = np.zeros_like(state0)
    lib().orc_vjp(C.byref(s.c), state0.shape[0], actions.shape[0], _p(state0), _p(actions), _p(g_state_T),
                  _p(g_torso), _p(ga), _p(gs), _threads(n_threads))
    return ga, gs


def jvp(system, state0, actions, d_state0, d_actions, n_threads=0):
    """Forward-mode derivative: returns (d_state_T [N,B,13], d_torso [T,N,3])."""
    s = _sys(system)
    state0, actions, d_state0, d_actions = map(_f64, (state0, actions, d_state0, d_actions))
    T, N = actions.shape[0], state0.shape[0]
    ds = np.zeros_like(state0)
    dt = np.zeros((T, N, 3))
    lib().orc_jvp(C.byref(s.c), N, T, _p(state0), _p(actions), _p(d_state0), _p(d_actions), _p(ds), _p(dt),
                  _threads(n_threads))
    return ds, dt


def default_qp(system, n_envs, root_pos=None, root_rot=None, angles=None):
    """default_qp (Sec. 4.1): bodies placed in a valid joint configuration."""
    s = _sys(system)
    root_pos, root_rot, angles = map(_f64, (root_pos, root_rot, angles))
    out = np.zeros((n_envs, s.B, 13))
    lib().orc_default_qp(C.byref(s.c), n_envs, _p(root_pos), _p(root_rot), _p(angles), _p(out))
    return out


def joint_angles(system, state):
    s = _sys(system)
    state = _f64(state)
    out = np.zeros((state.shape[0], s.D))
    lib().orc_joint_angles(C.byref(s.c), state.shape[0], _p(state), _p(out))
    return out


def joint_state(system, state):
    """Joint angles [N, D] and joint angular rates [N, D] (w_c - w_p along each
    joint axis in the world)."""
    s = _sys(system)
    state = _f64(state)
    ang = np.zeros((state.shape[0], s.D))
    rate = np.zeros((state.shape[0], s.D))
    lib().orc_joint_state(C.byref(s.c), state.shape[0], _p(state), _p(ang), _p(rate))
    return ang, rate


def energy_momentum(system, state):
    """Energy [N] and momentum [N,6] (linear, angular about the origin)."""
    s = _sys(system)
    state = _f64(state)
    N = state.shape[0]
    e = np.zeros(N)
    m = np.zeros((N, 6))
    lib().orc_energy(C.byref(s.c), N, _p(state), _p(e), _p(m))
    return e, m


def contacts(system, state_env, max_out=256):
    """Active contacts of one environment's state [B,13]: list of (a, b, depth, n, p)."""
    s = _sys(system)
    st = _f64(state_env)
    bodies = np.zeros((max_out, 2), dtype=np.int32)
    geo = np.zeros((max_out, 7))
    n = lib().orc_contacts(C.byref(s.c), _p(st), max_out, _p(bodies), _p(geo))
    return [(int(bodies[i, 0]), int(bodies[i, 1]), geo[i, 0], geo[i, 1:4].copy(), geo[i, 4:7].copy())
            for i in range(min(n, max_out))]


def segment_closest(P1, Q1, P2, Q2):
    arrs = [_f64(np.asarray(a)) for a in (P1, Q1, P2, Q2)]
    out = np.zeros(2)
    lib().orc_segment_closest(*[_p(a) for a in arrs], _p(out))
    return float(out[0]), float(out[1])


def capsule_box(P, Q, r, c, q, he):
    """Capsule-box detection: None or (depth, n, p)."""
    arrs = [_f64(np.asarray(a)) for a in (P, Q, c, q, he)]
    out = np.zeros(7)
    hit = lib().orc_capsule_box(_p(arrs[0]), _p(arrs[1]), float(r), _p(arrs[2]), _p(arrs[3]), _p(arrs[4]), _p(out))
    if not hit:
        return None
    return float(out[0]), out[1:4].copy(), out[4:7].copy()


def seg_box_param(Pl, dl, he):
    arrs = [_f64(np.asarray(a)) for a in (Pl, dl, he)]
    return lib().orc_seg_box_param(*[_p(a) for a in arrs])
