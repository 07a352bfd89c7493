"""The C-ABI library builds, loads and exports every entry point include/lp2d.h
declares; host-side argument checks work without a GPU (no compute calls)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("lp2d.h", "lp3d.h", "lpnd.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1902_04995_gb300 import build

    build.build()
    import torch  # noqa: F401
    from paper_1902_04995_gb300 import lp2d

    return lp2d


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lp[23n]d_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("lp2d_solve_batch", "lp2d_solve_batch_ex", "lp2d_workspace_bytes", "lp2d_visit_order",
              "lp2d_last_error", "lp2d_read_device_error", "lp3d_solve_batch_ex", "lpnd_solve_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_options_and_workspace_sizes(lib):
    o = lib.default_options()
    assert (o.seed, o.precision, o.schedule, o.check_finite) == (0, lib.PREC_FP32, lib.SCHED_PERSISTENT, 1)
    assert lib.workspace_bytes(1000, o) >= 32
    assert lib.workspace_bytes(1000, lib.default_options(schedule=lib.SCHED_UNIFORM)) >= 32
    assert "sm_103a" in lib.version()


def test_host_side_validation(lib):
    L = lib._lib
    B = lib.Box
    # n_lp < 0
    assert L.lp2d_solve_batch_ex(None, None, None, None, -1, None, B(-1, 1, -1, 1), None, None, None, None, 0,
                                 None) == lib.ERR_INVALID_ARGUMENT
    assert "n_lp" in lib.last_error()
    # empty box
    assert L.lp2d_solve_batch_ex(None, None, None, None, 3, None, B(1, -1, -1, 1), None, None, None, None, 0,
                                 None) == lib.ERR_INVALID_ARGUMENT
    # NaN box
    assert L.lp2d_solve_batch_ex(None, None, None, None, 3, None, B(float("nan"), 1, -1, 1), None, None, None,
                                 None, 0, None) == lib.ERR_INVALID_ARGUMENT
    # NULL data
    assert L.lp2d_solve_batch_ex(None, None, None, None, 3, None, B(-1, 1, -1, 1), None, None, None, None, 0,
                                 None) == lib.ERR_INVALID_ARGUMENT
    # unknown precision / schedule
    o = lib.default_options(precision=7)
    assert L.lp2d_solve_batch_ex(None, None, None, None, 3, None, B(-1, 1, -1, 1), None, None, ctypes.byref(o),
                                 None, 0, None) == lib.ERR_INVALID_ARGUMENT
    o = lib.default_options(schedule=9)
    assert L.lp2d_solve_batch_ex(None, None, None, None, 3, None, B(-1, 1, -1, 1), None, None, ctypes.byref(o),
                                 None, 0, None) == lib.ERR_INVALID_ARGUMENT
    # n_lp == 0 is a no-op
    assert L.lp2d_solve_batch_ex(None, None, None, None, 0, None, B(-1, 1, -1, 1), None, None, None, None, 0,
                                 None) == lib.OK
    # misaligned pointer (never dereferenced: rejected on the host)
    fake = ctypes.c_void_p(0x1001)
    assert L.lp2d_solve_batch_ex(fake, fake, fake, fake, 3, fake, B(-1, 1, -1, 1), fake, fake, None, None, 0,
                                 None) == lib.ERR_INVALID_ARGUMENT
    # missing workspace for the persistent schedule
    al = ctypes.c_void_p(0x1000)
    assert L.lp2d_solve_batch_ex(al, al, al, al, 3, al, B(-1, 1, -1, 1), al, al, None, None, 0,
                                 None) == lib.ERR_WORKSPACE
    # visit order size checks
    assert L.lp2d_visit_order(0, -1, None, None) == lib.ERR_INVALID_ARGUMENT
    assert L.lp2d_visit_order(0, 0, None, None) == lib.OK


def test_host_entry_validation(lib):
    import numpy as np

    L = lib._lib
    B = lib.Box
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.lp2d_solve_batch_host.argtypes = [vp, vp, vp, vp, i64, vp, B, vp, vp, ctypes.POINTER(lib.Options), vp]
    L.lp2d_solve_batch_host.restype = ctypes.c_int
    box = B(-1, 1, -1, 1)
    a = np.zeros(8, dtype=np.float32)
    obj = np.zeros(6, dtype=np.float32)
    xy = np.zeros(6, dtype=np.float32)
    st = np.full(3, -5, dtype=np.int32)
    p = lambda arr: arr.ctypes.data_as(vp)  # noqa: E731
    # offsets that decrease are rejected on the host before anything is enqueued
    bad = np.array([0, 4, 2, 8], dtype=np.int64)
    assert L.lp2d_solve_batch_host(p(a), p(a), p(a), p(bad), 3, p(obj), box, p(xy), p(st), None,
                                   None) == lib.ERR_INVALID_ARGUMENT
    assert "decrease" in lib.last_error()
    assert (st == -5).all()
    neg = np.array([-1, 4, 6, 8], dtype=np.int64)
    assert L.lp2d_solve_batch_host(p(a), p(a), p(a), p(neg), 3, p(obj), box, p(xy), p(st), None,
                                   None) == lib.ERR_INVALID_ARGUMENT
    # n_lp < 0, bad box, NULL pointers, per-LP diagnostics (device outputs) unsupported
    good = np.array([0, 4, 6, 8], dtype=np.int64)
    assert L.lp2d_solve_batch_host(None, None, None, None, -1, None, box, None, None, None,
                                   None) == lib.ERR_INVALID_ARGUMENT
    assert L.lp2d_solve_batch_host(p(a), p(a), p(a), p(good), 3, p(obj), B(1, -1, -1, 1), p(xy), p(st), None,
                                   None) == lib.ERR_INVALID_ARGUMENT
    assert L.lp2d_solve_batch_host(None, p(a), p(a), p(good), 3, p(obj), box, p(xy), p(st), None,
                                   None) == lib.ERR_INVALID_ARGUMENT
    o = lib.default_options(out_nviol=0x1000)
    assert L.lp2d_solve_batch_host(p(a), p(a), p(a), p(good), 3, p(obj), box, p(xy), p(st), ctypes.byref(o),
                                   None) == lib.ERR_UNSUPPORTED
    o = lib.default_options(precision=lib.PREC_FP32_F64ISECT, schedule=lib.SCHED_UNIFORM)
    assert L.lp2d_solve_batch_host(p(a), p(a), p(a), p(good), 3, p(obj), box, p(xy), p(st), ctypes.byref(o),
                                   None) == lib.ERR_UNSUPPORTED
    assert L.lp2d_solve_batch_host(None, None, None, None, 0, None, box, None, None, None, None) == lib.OK
    assert (st == -5).all()


def test_3d_host_side_validation(lib):
    L = lib._lib
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    L.lp3d_solve_batch_ex.argtypes = [vp, vp, vp, vp, vp, i64, vp, lib.Box3, vp, vp, ctypes.POINTER(lib.Options), vp,
                                      sz, vp]
    L.lp3d_solve_batch_ex.restype = ctypes.c_int
    box = lib.Box3(-1, 1, -1, 1, -1, 1)
    call = lambda n, b=box, o=None, p=None, ws=None, wsb=0: L.lp3d_solve_batch_ex(  # noqa: E731
        p, p, p, p, p, n, p, b, p, p, ctypes.byref(o) if o else None, ws, wsb, None)
    assert call(-1) == lib.ERR_INVALID_ARGUMENT
    assert call(3, b=lib.Box3(-1, 1, 1, -1, -1, 1)) == lib.ERR_INVALID_ARGUMENT
    assert call(3, b=lib.Box3(-1, 1, -1, 1, -1, float("inf"))) == lib.ERR_INVALID_ARGUMENT
    assert call(3, o=lib.default_options(precision=lib.PREC_FP32_F64ISECT)) == lib.ERR_UNSUPPORTED
    assert call(3, o=lib.default_options(schedule=lib.SCHED_UNIFORM)) == lib.ERR_UNSUPPORTED
    assert call(0) == lib.OK
    assert call(3) == lib.ERR_INVALID_ARGUMENT  # NULL data
    al = ctypes.c_void_p(0x1000)
    assert call(3, p=al) == lib.ERR_WORKSPACE
    assert "workspace" in lib.last_error()


def test_nd_host_side_validation(lib):
    L = lib._lib
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    L.lpnd_solve_batch.argtypes = [ctypes.c_int, vp, vp, vp, i64, vp, vp, vp, vp, ctypes.POINTER(lib.Options), vp,
                                   sz, vp]
    L.lpnd_solve_batch.restype = ctypes.c_int

    def call(d, n, box=None, o=None, a=None, p=None, ws=None, wsb=0, no_box=False):
        vals = box if box is not None else [-1.0, 1.0] * d
        bx = None if no_box else (ctypes.c_float * len(vals))(*vals)
        return L.lpnd_solve_batch(d, a, p, p, n, p, bx, p, p, ctypes.byref(o) if o else None, ws, wsb, None)

    assert call(1, 3) == lib.ERR_INVALID_ARGUMENT and "d = 1" in lib.last_error()
    assert call(6, 3) == lib.ERR_INVALID_ARGUMENT
    assert call(4, -1) == lib.ERR_INVALID_ARGUMENT
    assert call(4, 3, no_box=True) == lib.ERR_INVALID_ARGUMENT
    assert call(4, 3, box=[-1, 1, -1, 1, 1, -1, -1, 1]) == lib.ERR_INVALID_ARGUMENT and "axis 2" in lib.last_error()
    assert call(5, 3, box=[-1, 1] * 4 + [-1, float("inf")]) == lib.ERR_INVALID_ARGUMENT
    assert call(4, 3, o=lib.default_options(precision=lib.PREC_FP32_F64ISECT)) == lib.ERR_UNSUPPORTED
    assert call(4, 3, o=lib.default_options(schedule=lib.SCHED_UNIFORM)) == lib.ERR_UNSUPPORTED
    assert call(4, 0) == lib.OK
    assert call(4, 3) == lib.ERR_INVALID_ARGUMENT  # NULL data
    al = 0x1000  # aligned fake device addresses: the host reads the pointer values only
    assert call(4, 3, a=(ctypes.c_void_p * 4)(al, al, al, al), p=ctypes.c_void_p(al)) == lib.ERR_WORKSPACE
    assert call(4, 3, a=(ctypes.c_void_p * 4)(al, al, None, al), p=ctypes.c_void_p(al)) == lib.ERR_INVALID_ARGUMENT
    assert "a[2]" in lib.last_error()
    assert call(4, 3, a=(ctypes.c_void_p * 4)(al, al, al, al + 2), p=ctypes.c_void_p(al)) == lib.ERR_INVALID_ARGUMENT
    assert lib.max_constraints_nd(5) == 8182 and lib.warp_stage_constraints_nd(5) == 1014


def test_autotune_host_side_validation(lib):
    L = lib._lib
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    L.lp2d_autotune.argtypes = [vp, vp, vp, vp, i64, vp, lib.Box, vp, vp, ctypes.POINTER(lib.Options), vp, sz,
                                ctypes.c_int, ctypes.POINTER(ctypes.c_float), vp]
    L.lp2d_autotune.restype = ctypes.c_int
    box = lib.Box(-1, 1, -1, 1)
    o = lib.default_options()
    assert L.lp2d_autotune(None, None, None, None, 0, None, box, None, None, None, None, 0, 2, None,
                           None) == lib.ERR_INVALID_ARGUMENT  # no options
    assert L.lp2d_autotune(None, None, None, None, 0, None, box, None, None, ctypes.byref(o), None, 0, 0, None,
                           None) == lib.ERR_INVALID_ARGUMENT  # reps < 1
    u = lib.default_options(schedule=lib.SCHED_UNIFORM)
    assert L.lp2d_autotune(None, None, None, None, 0, None, box, None, None, ctypes.byref(u), None, 0, 2, None,
                           None) == lib.ERR_UNSUPPORTED
    assert L.lp2d_autotune(None, None, None, None, -1, None, box, None, None, ctypes.byref(o), None, 0, 2, None,
                           None) == lib.ERR_INVALID_ARGUMENT
    assert L.lp2d_autotune(None, None, None, None, 0, None, box, None, None, ctypes.byref(o), None, 0, 2, None,
                           None) == lib.OK  # an empty batch has nothing to tune
    assert (o.ctas_per_sm, o.chunk_big, o.chunk_small) == (0, 0, 0)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1902_04995_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "seidel_oracle" not in text, f


def test_binding_fails_loudly_without_the_library(tmp_path):
    # a copy of the package without liblp2d.so: importing the binding must raise, never
    # fall back to anything else
    import shutil
    import subprocess
    import sys

    shutil.copytree(os.path.join(ROOT, "paper_1902_04995_gb300"), tmp_path / "paper_1902_04995_gb300",
                    ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_1902_04995_gb300.lp2d"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "is missing" in r.stderr
