"""FP64 CPU oracle for the batched 2-D LP solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The product path (``paper_1902_04995_gb300``) never imports
it, and it imports nothing from the product.

The arithmetic lives in ``seidel_oracle.c`` (plain serial Seidel in FP64, Sec. 2.1 of
the paper, Eqs. 1-4), ``seidel3_oracle.c`` (the same method in three dimensions, the
direction Sec. 6 names) and ``seidelN_oracle.c`` (any dimension up to five, as a
recursion over affine subspaces); this module only builds them with gcc and marshals
numpy arrays through ctypes.  ctypes drops the GIL during a call, so ``threads > 1`` splits a
batch by LP range over plain Python threads (one serial solve per LP, no change to
the arithmetic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("seidel_oracle.c", "seidel3_oracle.c", "seidelN_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OPTIMAL, INFEASIBLE, BOX_BOUNDED, BAD_INPUT = 0, 1, 2, 3
NONE_ID = -(2**31)
EPS_FP64 = 1e-12

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into liboracle.so next to them (portable flags only)."""
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _bind(lib):
    """Declare the C functions' signatures on a loaded copy of the oracle library."""
    u64, i64, i32, u32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_splitmix64.restype = u64
    lib.oracle_splitmix64.argtypes = [u64, u32]
    for name in ("oracle_perm_fwd", "oracle_perm_inv", "oracle_feistel_enc", "oracle_feistel_dec"):
        getattr(lib, name).restype = i64
        getattr(lib, name).argtypes = [u64, i64, i64]
    lib.oracle_feistel_half_bits.restype = i32
    lib.oracle_feistel_half_bits.argtypes = [i64]
    lib.oracle_perm_array.restype = None
    lib.oracle_perm_array.argtypes = [u64, i64, vp]
    lib.oracle_solve_batch.restype = None
    lib.oracle_solve_batch.argtypes = [vp, vp, vp, vp, i64, i64, vp, dbl, dbl, dbl, dbl, u64, dbl,
                                       vp, vp, vp, vp]
    lib.oracle_solve_batch3.restype = None
    lib.oracle_solve_batch3.argtypes = [vp, vp, vp, vp, vp, i64, i64, vp, vp, u64, dbl, vp, vp, vp, vp]
    lib.oracle_solve_batchN.restype = None
    lib.oracle_solve_batchN.argtypes = [ctypes.c_int, vp, vp, vp, i64, i64, vp, vp, u64, dbl, vp, vp, vp, vp]
    return lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def splitmix64(seed: int, r: int) -> int:
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), r))


def perm_fwd(seed: int, m: int, k: int) -> int:
    return int(_load().oracle_perm_fwd(seed & (2**64 - 1), m, k))


def perm_inv(seed: int, m: int, q: int) -> int:
    return int(_load().oracle_perm_inv(seed & (2**64 - 1), m, q))


def feistel_enc(seed: int, m: int, x: int) -> int:
    return int(_load().oracle_feistel_enc(seed & (2**64 - 1), m, x))


def feistel_dec(seed: int, m: int, x: int) -> int:
    return int(_load().oracle_feistel_dec(seed & (2**64 - 1), m, x))


def half_bits(m: int) -> int:
    return int(_load().oracle_feistel_half_bits(m))


def perm_array(seed: int, m: int) -> np.ndarray:
    out = np.empty(max(m, 0), dtype=np.int64)
    if m > 0:
        _load().oracle_perm_array(seed & (2**64 - 1), m, _ptr(out))
    return out


def solve_batch(ax, ay, b, offsets, obj, box, seed: int = 0, eps: float = EPS_FP64,
                threads: int = 1, lp_range=None, want_def: bool = False, want_nviol: bool = False):
    """Solve every LP of a CSR batch serially in FP64.

    ax, ay, b: float32 [n_constraints]; offsets: int64 [n_lp + 1]; obj: float32 [n_lp, 2]
    (or [2*n_lp]); box: (xmin, xmax, ymin, ymax).  LP l visits its constraints in the
    order pi_l with seed_l = seed + l.  Returns a dict with ``xy`` (float64 [n_lp, 2]),
    ``status`` (int32 [n_lp]) and optionally ``def`` (int32 [n_lp, 3]) and ``nviol``.
    With ``lp_range=(lo, hi)`` only those LPs are solved; the others stay zero.
    """
    lib = _load()
    ax = np.ascontiguousarray(ax, dtype=np.float32)
    ay = np.ascontiguousarray(ay, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    obj = np.ascontiguousarray(obj, dtype=np.float32).reshape(-1)
    n_lp = offsets.shape[0] - 1
    assert obj.shape[0] == 2 * n_lp
    xy = np.zeros((n_lp, 2), dtype=np.float64)
    status = np.zeros(n_lp, dtype=np.int32)
    dfn = np.zeros((n_lp, 3), dtype=np.int32) if want_def else None
    nviol = np.zeros(n_lp, dtype=np.int64) if want_nviol else None
    lo, hi = (0, n_lp) if lp_range is None else lp_range
    xmin, xmax, ymin, ymax = (float(np.float32(v)) for v in box)

    def run(a, z):
        lib.oracle_solve_batch(_ptr(ax), _ptr(ay), _ptr(b), _ptr(offsets), a, z, _ptr(obj),
                               xmin, xmax, ymin, ymax, seed & (2**64 - 1), eps,
                               _ptr(xy), _ptr(status), _ptr(dfn), _ptr(nviol))

    if threads <= 1 or hi - lo < 2 * threads:
        run(lo, hi)
    else:
        # Split by constraint count so that each thread gets similar work.
        csum = offsets[lo:hi + 1] - offsets[lo]
        pieces = threads * 8
        cuts = np.searchsorted(csum, np.linspace(0, csum[-1], pieces + 1)[1:-1]) + lo
        bounds = [lo] + sorted(set(int(c) for c in cuts if lo < c < hi)) + [hi]
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda ab: run(*ab), zip(bounds[:-1], bounds[1:])))
    out = {"xy": xy, "status": status}
    if want_def:
        out["def"] = dfn
    if want_nviol:
        out["nviol"] = nviol
    return out


def _split(offsets, lo, hi, threads):
    """LP ranges of similar constraint counts for `threads` workers."""
    csum = offsets[lo:hi + 1] - offsets[lo]
    cuts = np.searchsorted(csum, np.linspace(0, csum[-1], threads * 8 + 1)[1:-1]) + lo
    bounds = [lo] + sorted(set(int(c) for c in cuts if lo < c < hi)) + [hi]
    return list(zip(bounds[:-1], bounds[1:]))


def solve_batch3(ax, ay, az, b, offsets, obj, box, seed: int = 0, eps: float = EPS_FP64,
                 threads: int = 1, want_def: bool = False, want_nviol: bool = False):
    """Solve every 3-D LP of a CSR batch serially in FP64 (seidel3_oracle.c).

    ax, ay, az, b: float32 [n_constraints]; offsets: int64 [n_lp + 1]; obj: float32
    [n_lp, 3]; box: (xmin, xmax, ymin, ymax, zmin, zmax).  Returns a dict with ``xyz``
    (float64 [n_lp, 3]), ``status`` and optionally ``def`` (int32 [n_lp, 3]) and
    ``nviol`` (violations at the top level, each one a 2-D LP).
    """
    lib = _load()
    arrs = [np.ascontiguousarray(v, dtype=np.float32) for v in (ax, ay, az, b)]
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    obj = np.ascontiguousarray(obj, dtype=np.float32).reshape(-1)
    n_lp = offsets.shape[0] - 1
    assert obj.shape[0] == 3 * n_lp
    box6 = np.asarray([float(np.float32(v)) for v in box], dtype=np.float64)
    assert box6.shape[0] == 6
    xyz = np.zeros((n_lp, 3), dtype=np.float64)
    status = np.zeros(n_lp, dtype=np.int32)
    dfn = np.zeros((n_lp, 3), dtype=np.int32) if want_def else None
    nviol = np.zeros(n_lp, dtype=np.int64) if want_nviol else None

    def run(a, z):
        lib.oracle_solve_batch3(*(_ptr(v) for v in arrs), _ptr(offsets), a, z, _ptr(obj), _ptr(box6),
                                seed & (2**64 - 1), eps, _ptr(xyz), _ptr(status), _ptr(dfn), _ptr(nviol))

    if threads <= 1 or n_lp < 2 * threads:
        run(0, n_lp)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda ab: run(*ab), _split(offsets, 0, n_lp, threads)))
    out = {"xyz": xyz, "status": status}
    if want_def:
        out["def"] = dfn
    if want_nviol:
        out["nviol"] = nviol
    return out


def solve_batchN(a, b, offsets, obj, box, seed: int = 0, eps: float = EPS_FP64,
                 threads: int = 1, want_def: bool = False, want_nviol: bool = False):
    """Solve every d-dimensional LP of a CSR batch serially in FP64 (seidelN_oracle.c).

    a: float32 [d, n_constraints] (row t holds coefficient t of every constraint);
    b: float32 [n_constraints]; offsets: int64 [n_lp + 1]; obj: float32 [n_lp, d];
    box: (min_0, max_0, ..., min_{d-1}, max_{d-1}).  Returns a dict with ``x`` (float64
    [n_lp, d]), ``status`` and optionally ``def`` (int32 [n_lp, d]) and ``nviol``
    (violations in the whole space, each one an LP of dimension d - 1).
    """
    lib = _load()
    a = np.asarray(a, dtype=np.float32)
    d = a.shape[0]
    assert 1 <= d <= 5
    rows = np.ascontiguousarray(a.T)  # [n_constraints][d]
    b = np.ascontiguousarray(b, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    obj = np.ascontiguousarray(obj, dtype=np.float32).reshape(-1)
    n_lp = offsets.shape[0] - 1
    assert obj.shape[0] == d * n_lp
    boxd = np.asarray([float(np.float32(v)) for v in box], dtype=np.float64)
    assert boxd.shape[0] == 2 * d
    x = np.zeros((n_lp, d), dtype=np.float64)
    status = np.zeros(n_lp, dtype=np.int32)
    dfn = np.zeros((n_lp, d), dtype=np.int32) if want_def else None
    nviol = np.zeros(n_lp, dtype=np.int64) if want_nviol else None

    def run(lo, hi):
        lib.oracle_solve_batchN(d, _ptr(rows), _ptr(b), _ptr(offsets), lo, hi, _ptr(obj), _ptr(boxd),
                                seed & (2**64 - 1), eps, _ptr(x), _ptr(status), _ptr(dfn), _ptr(nviol))

    if threads <= 1 or n_lp < 2 * threads:
        run(0, n_lp)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda ab: run(*ab), _split(offsets, 0, n_lp, threads)))
    out = {"x": x, "status": status}
    if want_def:
        out["def"] = dfn
    if want_nviol:
        out["nviol"] = nviol
    return out
