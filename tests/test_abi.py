"""The C-ABI library builds, loads and exports every symbol include/cn.h declares;
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_2205_00856_b300 as cnb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "cn.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cn_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = cnb.load()
    out = subprocess.run(["nm", "-D", "--defined-only", cnb.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    decl = declared_symbols()
    assert decl, "no declarations parsed"
    missing = [s for s in decl if s not in exported]
    assert not missing, missing
    for s in decl:
        assert hasattr(lib, s)
    assert set(cnb.EXPORTS) == set(decl)


def test_status_strings_and_version():
    lib = cnb.load()
    assert lib.cn_status_string(0) == b"ok"
    assert lib.cn_status_string(5) == b"device-side wait timed out"
    assert cnb.version().endswith("sm_103a")


def _desc(**kw):
    d = dict(n=100, dx=0.1, dt=0.01, x_min=0.0, pot=0, n_cos=0, V0=None, soft_s=2.0, cos_a=None, L=1.0,
             block=0, arith=0, flags=0, level_block=0, level1_block=0)
    d.update(kw)
    return cnb._Desc(*[d[f] for f, _ in cnb._Desc._fields_])


@pytest.mark.parametrize("kw", [dict(n=2), dict(n=-5), dict(dx=0.0), dict(dx=float("nan")), dict(dt=0.0),
                                dict(pot=9), dict(pot=1), dict(pot=2, soft_s=0.0), dict(pot=3, n_cos=17, L=1.0),
                                dict(pot=3, n_cos=2, L=1.0), dict(block=2), dict(block=33), dict(arith=3),
                                dict(flags=32), dict(flags=12), dict(level_block=2), dict(level_block=40), dict(level1_block=2),
                                dict(level1_block=33)])
def test_invalid_descriptor_rejected_on_host(kw):
    lib = cnb.load()
    h = C.c_void_p()
    rc = lib.cn_plan_create(C.byref(_desc(**kw)), C.byref(h))
    assert rc == 1 and not h.value


def test_null_arguments_rejected():
    lib = cnb.load()
    assert lib.cn_plan_create(None, None) == 1
    assert lib.cn_step(None, None, None, None, 1, None) == 1
    assert lib.cn_step_host(None, None, None, None, 1, None) == 1
    assert lib.cn_solve_tridiag(None, None, None, None, None, None, 10, None) == 1
    assert lib.cn_plan_status(None) == 1
    assert lib.cn_plan_destroy(None) == 0


@pytest.mark.parametrize("case", ["nsys0", "small_size", "cos_null", "bad_desc", "nan_xmin", "nan_cos"])
def test_invalid_batch_rejected_on_host(case):
    import numpy as np
    lib = cnb.load()
    h = C.c_void_p()
    sizes = np.array([100, 3, 5000], np.int64)
    xm = None
    cos = None
    d = _desc(n=0)
    nsys = 3
    if case == "nsys0":
        nsys = 0
    elif case == "small_size":
        sizes[1] = 2
    elif case == "cos_null":
        d = _desc(n=0, pot=3, n_cos=4, L=0.0)
    elif case == "bad_desc":
        d = _desc(n=0, dx=-1.0)
    elif case == "nan_xmin":
        xm = np.array([0.0, float("nan"), 1.0])
    elif case == "nan_cos":
        d = _desc(n=0, pot=3, n_cos=2, L=0.0)
        cos = np.array([[0.1, 0.2], [0.3, float("inf")], [0.0, 0.0]])
    rc = lib.cn_batch_create(C.byref(d), nsys, sizes.ctypes.data, None if xm is None else xm.ctypes.data,
                             None if cos is None else cos.ctypes.data, C.byref(h))
    assert rc == 1 and not h.value


def test_null_batch_arguments_rejected():
    lib = cnb.load()
    assert lib.cn_batch_create(None, 1, None, None, None, None) == 1
    assert lib.cn_batch_step(None, None, None, None, 1, None) == 1
    assert lib.cn_batch_offsets(None, None) == 1
    assert lib.cn_batch_status(None) == 1
    assert lib.cn_batch_destroy(None) == 0


@pytest.mark.parametrize("case", ["nslabs0", "rank_out", "joint_gap1", "joint_ends", "too_many"])
def test_invalid_slab_rejected_on_host(case):
    import numpy as np
    lib = cnb.load()
    h = C.c_void_p()
    d = _desc(n=100)
    G, r, J = 3, 0, None
    if case == "nslabs0":
        G = 0
    elif case == "rank_out":
        r = 3
    elif case == "joint_gap1":
        J = np.array([0, 10, 11, 99], np.int64)
    elif case == "joint_ends":
        J = np.array([1, 10, 50, 99], np.int64)
    else:
        G = cnb.SLAB_MAX + 1
    rc = lib.cn_slab_create(C.byref(d), G, r, None if J is None else J.ctypes.data, C.byref(h))
    assert rc == 1 and not h.value


def test_slab_calls_reject_null_and_plain_plans():
    lib = cnb.load()
    assert lib.cn_slab_reduce(None, None, None, None, None) == 1
    assert lib.cn_slab_finish(None, None, None, None) == 1
    assert lib.cn_slab_range(None, None, None) == 1
