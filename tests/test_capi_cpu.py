"""The C ABI library without a GPU: it loads, exports every symbol that
include/brax.h declares, and rejects invalid descriptors with status codes
and messages (validation runs before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2106_13281_gb300 import binding as bnd
from paper_2106_13281_gb300 import scenes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_13281_gb300 import build
    build.build()
    return bnd.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "brax.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(brax_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(names) == sorted(bnd.EXPORTS)


def create(lib, desc):
    d, keep = bnd.marshal_desc(desc)
    h = C.c_void_p()
    rc = lib.brax_system_create(C.byref(d), C.byref(h))
    return rc, h, lib.brax_last_error().decode()


@pytest.mark.parametrize("mutate,needle", [
    (lambda d: d.__setitem__("mass", np.array([0.0] + list(d["mass"][1:]))), "mass"),
    (lambda d: d.__setitem__("dof", np.array([4] * len(d["dof"]), dtype=np.int32)), "dof"),
    (lambda d: d.__setitem__("child", np.array([1] * len(d["child"]), dtype=np.int32)), "child"),
    (lambda d: d.__setitem__("act_axis", np.array([1] * len(d["act_axis"]), dtype=np.int32)), "act_axis"),
    (lambda d: d.__setitem__("pair_a", np.array([99] * len(d["pair_a"]), dtype=np.int32)), "pair"),
    (lambda d: d.__setitem__("substeps", 0), "substeps"),
    (lambda d: d.__setitem__("dt", -1.0), "dt"),
    (lambda d: d.__setitem__("radius", np.zeros_like(d["radius"])), "capsule"),
])
def test_invalid_descriptors_rejected(lib, mutate, needle):
    d = S.quadruped()
    mutate(d)
    rc, h, msg = create(lib, d)
    assert rc == 2, (rc, msg)
    assert needle in msg
    assert not h.value


def test_joint_cycle_rejected(lib):
    d = S.pendulum()
    d["parent"] = np.array([2, 1], dtype=np.int32)
    d["child"] = np.array([1, 2], dtype=np.int32)
    rc, h, msg = create(lib, d)
    assert rc == 2 and "cycle" in msg


def test_null_arguments(lib):
    assert lib.brax_system_create(None, None) == 1
    assert lib.brax_rollout(None, 1, 1, 1, None, None, None, None, None, None, None) == 1
    assert lib.brax_workspace_size(None, 1, 1, 1, None) == 1
    assert lib.brax_sync_status(None, None) == 1


def plan(lib, mode, chunk, units, T, slots, min_chunk=16):
    f = lib.brax_internal_plan_schedule
    f.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_int64, C.c_int32,
                  C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    n, s = C.c_int32(), C.c_int32()
    assert f(mode, chunk, units, T, slots, min_chunk, C.byref(n), C.byref(s)) == 0
    return n.value, s.value


def test_schedule_plan_host_logic(lib):
    """The chunked-schedule planner (host arithmetic, no GPU).  Whole
    resident waves (or a last wave at least 97 % full) keep the static
    launch; otherwise the chunk length (at least 16 steps) that fills the
    last round of items best, every step covered exactly once."""
    # the headline: 1,024 blocks of 64 environments on 304 resident blocks (3.37 waves)
    assert plan(lib, 1, 0, 1024, 1000, 304) == (8, 125)
    # whole waves, a full last wave, one wave or less: static
    assert plan(lib, 1, 0, 912, 1000, 304) == (0, 0)
    assert plan(lib, 1, 0, 1213, 1000, 304) == (0, 0)   # 1213 / 1216 = 99.8 % full
    assert plan(lib, 1, 0, 300, 1000, 304) == (0, 0)
    # short rollouts: chunks of at least 16 steps; fewer than two chunks stay static
    assert plan(lib, 1, 0, 1024, 100, 304) == (5, 20)  # 16.8 rounds of 20 steps, not 23.6 of 16
    assert plan(lib, 1, 0, 2048, 1000, 304) == (4, 250)  # the reverse pass at K = 1: 26.9 rounds
    assert plan(lib, 1, 0, 1024, 31, 304) == (2, 16)
    assert plan(lib, 1, 0, 1024, 16, 304) == (0, 0)
    assert plan(lib, 1, 0, 1024, 1, 304) == (0, 0)
    # the reverse pass: segments of K = 4 steps, at least 16 steps' worth per chunk
    assert plan(lib, 1, 0, 2048, 250, 304, 4) == (4, 63)
    # mode 0 never, mode 2 always with the given chunk
    assert plan(lib, 0, 0, 1024, 1000, 304) == (0, 0)
    assert plan(lib, 2, 3, 2, 10, 304) == (4, 3)
    assert plan(lib, 2, 10, 2, 10, 304) == (0, 0)   # one chunk: nothing to schedule
    # an item count that would not fit a launch grid stays static
    assert plan(lib, 2, 1, 1 << 24, 1000, 304) == (0, 0)
    for units, T, slots in [(1024, 1000, 304), (2048, 977, 456), (625, 40, 304), (5000, 333, 152)]:
        n, s = plan(lib, 1, 0, units, T, slots)
        if n:
            assert s >= 16 and (n - 1) * s < T <= n * s


def test_variant_fields_validated(lib):
    """Descriptor version 2 (the variants): invalid actuator kinds and
    negative damping are rejected before any CUDA call; an unknown version is
    rejected; a version-1 descriptor is read without the variant fields, so
    their (invalid) contents are never looked at."""
    d = S.quadruped()
    d["act_type"] = np.full(len(d["act_joint"]), 2, dtype=np.int32)
    rc, h, msg = create(lib, d)
    assert rc == 2 and "act_type" in msg
    d = S.quadruped()
    d["linear_damping"] = -1.0
    rc, h, msg = create(lib, d)
    assert rc == 2 and "damping" in msg
    for version, ok in ((3, False), (1, True)):
        dd = S.quadruped()
        dd["act_type"] = np.full(len(dd["act_joint"]), 7, dtype=np.int32)
        dd["angular_damping_global"] = -5.0
        desc, keep = bnd.marshal_desc(dd)
        desc.version = version
        hh = C.c_void_p()
        rc = lib.brax_system_create(C.byref(desc), C.byref(hh))
        msg = lib.brax_last_error().decode()
        if ok:  # validation passed (a GPU-less machine then fails at the first CUDA call)
            assert rc != 2, msg
            if rc == 0:
                lib.brax_system_destroy(hh)
        else:
            assert rc == 2 and "version" in msg
