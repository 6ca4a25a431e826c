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
    (lambda d: d.__setitem__("dof", np.array([2] * len(d["dof"]), dtype=np.int32)), "dof"),
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
