"""Python binding of liblp2d.so: argument marshalling only.

Every function here has the name of the C entry point it wraps (without the
``lp2d_`` prefix) and forwards torch tensors as raw device pointers on the current
(or given) CUDA stream.  All compute runs in the library's CUDA kernels; there is
no CPU or PyTorch fallback: importing this module raises if the library has not
been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblp2d.so")

OPTIMAL, INFEASIBLE, BOX_BOUNDED, BAD_INPUT = 0, 1, 2, 3
OK, ERR_INVALID_ARGUMENT, ERR_CUDA, ERR_TIMEOUT, ERR_WORKSPACE, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
PREC_FP32, PREC_FP32_F64ISECT, PREC_FP64 = 0, 1, 2
SCHED_PERSISTENT, SCHED_UNIFORM = 0, 1
DEVERR_BAD_OFFSETS = 1


class Box(ctypes.Structure):
    _fields_ = [("xmin", ctypes.c_float), ("xmax", ctypes.c_float),
                ("ymin", ctypes.c_float), ("ymax", ctypes.c_float)]


class Options(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("chunk_big", ctypes.c_int32),
        ("chunk_small", ctypes.c_int32),
        ("check_finite", ctypes.c_int32),
        ("eps", ctypes.c_float),
        ("near_parallel_tau", ctypes.c_float),
        ("out_nviol", ctypes.c_void_p),
        ("out_def", ctypes.c_void_p),
        ("team_min_slots", ctypes.c_int32),
        ("l2_prefetch", ctypes.c_int32),
        ("lane_max_m", ctypes.c_int32),
    ]


class LP2DError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lp2d error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (__graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, u64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
    lib.lp2d_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.lp2d_default_options.restype = None
    lib.lp2d_workspace_bytes.argtypes = [i64, ctypes.POINTER(Options)]
    lib.lp2d_workspace_bytes.restype = sz
    lib.lp2d_workspace_init.argtypes = [vp, sz, vp]
    lib.lp2d_workspace_init.restype = ctypes.c_int
    lib.lp2d_solve_batch.argtypes = [vp, vp, vp, vp, i64, vp, Box, vp, vp, vp]
    lib.lp2d_solve_batch.restype = ctypes.c_int
    lib.lp2d_solve_batch_ex.argtypes = [vp, vp, vp, vp, i64, vp, Box, vp, vp, ctypes.POINTER(Options), vp, sz, vp]
    lib.lp2d_solve_batch_ex.restype = ctypes.c_int
    lib.lp2d_visit_order.argtypes = [u64, i64, vp, vp]
    lib.lp2d_visit_order.restype = ctypes.c_int
    lib.lp2d_read_device_error.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint32)]
    lib.lp2d_read_device_error.restype = ctypes.c_int
    lib.lp2d_last_error.argtypes = []
    lib.lp2d_last_error.restype = ctypes.c_char_p
    lib.lp2d_version.argtypes = []
    lib.lp2d_version.restype = ctypes.c_char_p
    return lib


_lib = _load()


def _check(rc):
    if rc != OK:
        raise LP2DError(rc, _lib.lp2d_last_error().decode())
    return rc


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


_dummy = {}


def _data_ptr(t):
    """Pointer for a constraint or objective array; an empty array (a batch whose LPs
    have no constraints) gets a one-element device buffer instead of NULL."""
    if t.numel() > 0:
        return ctypes.c_void_p(t.data_ptr())
    key = (t.device, t.dtype)
    if key not in _dummy:
        _dummy[key] = torch.zeros(4, dtype=t.dtype, device=t.device)
    return ctypes.c_void_p(_dummy[key].data_ptr())


def _need(t, dtype, name, numel=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")


def version() -> str:
    return _lib.lp2d_version().decode()


def last_error() -> str:
    return _lib.lp2d_last_error().decode()


def default_options(**kw) -> Options:
    o = Options()
    _lib.lp2d_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def workspace_bytes(n_lp: int, options: Options | None = None) -> int:
    return int(_lib.lp2d_workspace_bytes(n_lp, ctypes.byref(options) if options is not None else None))


def workspace_init(workspace: torch.Tensor, stream=None):
    _check(_lib.lp2d_workspace_init(_ptr(workspace), workspace.numel() * workspace.element_size(),
                                    _stream_handle(stream)))


def new_workspace(n_lp: int, options: Options | None = None, device=None, stream=None) -> torch.Tensor:
    """A zero-initialised workspace tensor of the size the options need (may be empty)."""
    n = workspace_bytes(n_lp, options)
    ws = torch.empty(max(n, 8), dtype=torch.uint8, device=device or "cuda")
    workspace_init(ws, stream)
    return ws


def _validate(ax, ay, b, offsets, obj, out_xy, out_status, out_dtype):
    n_lp = offsets.numel() - 1
    if n_lp < 0:
        raise ValueError("offsets needs n_lp + 1 entries")
    _need(ax, torch.float32, "ax")
    _need(ay, torch.float32, "ay", ax.numel())
    _need(b, torch.float32, "b", ax.numel())
    _need(offsets, torch.int64, "offsets")
    _need(obj, torch.float32, "obj_xy", 2 * n_lp)
    _need(out_xy, out_dtype, "out_xy", 2 * n_lp)
    _need(out_status, torch.int32, "out_status", n_lp)
    return n_lp


def solve_batch(ax, ay, b, offsets, obj, box, out_xy, out_status, stream=None):
    """lp2d_solve_batch: default options (seed 0, FP32, persistent schedule)."""
    n_lp = _validate(ax, ay, b, offsets, obj, out_xy, out_status, torch.float32)
    _check(_lib.lp2d_solve_batch(_data_ptr(ax), _data_ptr(ay), _data_ptr(b), _ptr(offsets), n_lp, _data_ptr(obj),
                                 Box(*box), _data_ptr(out_xy), _data_ptr(out_status), _stream_handle(stream)))


def solve_batch_ex(ax, ay, b, offsets, obj, box, out_xy, out_status, options: Options | None = None,
                   workspace: torch.Tensor | None = None, stream=None):
    """lp2d_solve_batch_ex: explicit options and a caller workspace (see new_workspace)."""
    opts = options if options is not None else default_options()
    out_dtype = torch.float64 if opts.precision == PREC_FP64 else torch.float32
    n_lp = _validate(ax, ay, b, offsets, obj, out_xy, out_status, out_dtype)
    wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.lp2d_solve_batch_ex(_data_ptr(ax), _data_ptr(ay), _data_ptr(b), _ptr(offsets), n_lp,
                                    _data_ptr(obj), Box(*box), _data_ptr(out_xy), _data_ptr(out_status),
                                    ctypes.byref(opts), _ptr(workspace), wbytes, _stream_handle(stream)))


def visit_order(seed_l: int, m: int, out: torch.Tensor, stream=None):
    """lp2d_visit_order: out[k] = pi(k) for one LP with m constraints, seed seed_l."""
    _need(out, torch.int64, "out", m)
    _check(_lib.lp2d_visit_order(seed_l & (2**64 - 1), m, _ptr(out), _stream_handle(stream)))


def read_device_error(workspace: torch.Tensor, stream=None) -> int:
    bits = ctypes.c_uint32(0)
    _check(_lib.lp2d_read_device_error(_ptr(workspace), _stream_handle(stream), ctypes.byref(bits)))
    return int(bits.value)


class Solver:
    """Device-resident solver for one batch layout: holds the workspace and output
    tensors so that repeated solves (and CUDA-graph capture) allocate nothing."""

    def __init__(self, n_lp: int, options: Options | None = None, device="cuda"):
        self.options = options if options is not None else default_options()
        self.n_lp = n_lp
        out_dtype = torch.float64 if self.options.precision == PREC_FP64 else torch.float32
        self.out_xy = torch.empty(2 * n_lp, dtype=out_dtype, device=device)
        self.out_status = torch.empty(n_lp, dtype=torch.int32, device=device)
        self.workspace = new_workspace(n_lp, self.options, device=device)

    def __call__(self, ax, ay, b, offsets, obj, box, stream=None):
        solve_batch_ex(ax, ay, b, offsets, obj, box, self.out_xy, self.out_status, self.options,
                       self.workspace, stream)
        return self.out_xy, self.out_status

    def autotune(self, ax, ay, b, offsets, obj, box, reps: int = 3, stream=None) -> float:
        """Pick this solver's schedule parameters for the given batch (lp2d_autotune);
        returns the winner's milliseconds per solve."""
        return autotune(ax, ay, b, offsets, obj, box, self.out_xy, self.out_status, self.options,
                        self.workspace, reps, stream)


_noalloc_ready = False


def solve_batch_noalloc(ax, ay, b, offsets, obj, box, out_xy, out_status, options: Options | None = None,
                        stream=None):
    """lp2d_solve_batch_noalloc: like solve_batch_ex, with the library's fixed device
    scratch array instead of a workspace (for callers that cannot allocate device
    memory).  Calls that overlap on the GPU race on that array."""
    global _noalloc_ready
    if not _noalloc_ready:
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        _lib.lp2d_solve_batch_noalloc.argtypes = [vp, vp, vp, vp, i64, vp, Box, vp, vp, ctypes.POINTER(Options), vp]
        _lib.lp2d_solve_batch_noalloc.restype = ctypes.c_int
        _noalloc_ready = True
    opts = options if options is not None else default_options()
    out_dtype = torch.float64 if opts.precision == PREC_FP64 else torch.float32
    n_lp = _validate(ax, ay, b, offsets, obj, out_xy, out_status, out_dtype)
    _check(_lib.lp2d_solve_batch_noalloc(_data_ptr(ax), _data_ptr(ay), _data_ptr(b), _ptr(offsets), n_lp,
                                         _data_ptr(obj), Box(*box), _data_ptr(out_xy), _data_ptr(out_status),
                                         ctypes.byref(opts), _stream_handle(stream)))


_host_ready = False


def _need_host(t, dtype, name, numel=None):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")


def solve_batch_host(ax, ay, b, offsets, obj, box, out_xy, out_status, options: Options | None = None,
                     stream=None):
    """lp2d_solve_batch_host: inputs and outputs are host tensors (pinned for full copy
    bandwidth).  The library copies the batch to the device in chunks, overlapping
    each chunk's copy with the previous chunk's solve, and copies the results back;
    synchronise `stream` before reading out_xy / out_status."""
    global _host_ready
    if not _host_ready:
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        _lib.lp2d_solve_batch_host.argtypes = [vp, vp, vp, vp, i64, vp, Box, vp, vp, ctypes.POINTER(Options), vp]
        _lib.lp2d_solve_batch_host.restype = ctypes.c_int
        _host_ready = True
    opts = options if options is not None else default_options()
    out_dtype = torch.float64 if opts.precision == PREC_FP64 else torch.float32
    n_lp = offsets.numel() - 1
    if n_lp < 0:
        raise ValueError("offsets needs n_lp + 1 entries")
    _need_host(ax, torch.float32, "ax")
    _need_host(ay, torch.float32, "ay", ax.numel())
    _need_host(b, torch.float32, "b", ax.numel())
    _need_host(offsets, torch.int64, "offsets")
    _need_host(obj, torch.float32, "obj_xy", 2 * n_lp)
    _need_host(out_xy, out_dtype, "out_xy", 2 * n_lp)
    _need_host(out_status, torch.int32, "out_status", n_lp)
    _check(_lib.lp2d_solve_batch_host(_ptr(ax), _ptr(ay), _ptr(b), _ptr(offsets), n_lp, _ptr(obj), Box(*box),
                                      _ptr(out_xy), _ptr(out_status), ctypes.byref(opts),
                                      _stream_handle(stream)))


_3d_ready = False
MAX_CONSTRAINTS_3D = 12282
DEVERR_TOO_LARGE = 4


class Box3(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")]


def solve_batch3d(ax, ay, az, b, offsets, obj, box, out_xyz, out_status, options: Options | None = None,
                  workspace: torch.Tensor | None = None, stream=None):
    """lp3d_solve_batch_ex: the batched 3-D solver.  obj: float32 [3*n_lp] (device);
    box: (xmin, xmax, ymin, ymax, zmin, zmax); out_xyz float32 [3*n_lp] (float64 for
    PREC_FP64); workspace as for solve_batch_ex (see new_workspace)."""
    global _3d_ready
    if not _3d_ready:
        vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
        _lib.lp3d_solve_batch_ex.argtypes = [vp, vp, vp, vp, vp, i64, vp, Box3, vp, vp, ctypes.POINTER(Options), vp,
                                             sz, vp]
        _lib.lp3d_solve_batch_ex.restype = ctypes.c_int
        _3d_ready = True
    opts = options if options is not None else default_options()
    out_dtype = torch.float64 if opts.precision == PREC_FP64 else torch.float32
    n_lp = offsets.numel() - 1
    if n_lp < 0:
        raise ValueError("offsets needs n_lp + 1 entries")
    _need(ax, torch.float32, "ax")
    for t, name in ((ay, "ay"), (az, "az"), (b, "b")):
        _need(t, torch.float32, name, ax.numel())
    _need(offsets, torch.int64, "offsets")
    _need(obj, torch.float32, "obj_xyz", 3 * n_lp)
    _need(out_xyz, out_dtype, "out_xyz", 3 * n_lp)
    _need(out_status, torch.int32, "out_status", n_lp)
    wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.lp3d_solve_batch_ex(_data_ptr(ax), _data_ptr(ay), _data_ptr(az), _data_ptr(b), _ptr(offsets), n_lp,
                                    _data_ptr(obj), Box3(*box), _data_ptr(out_xyz), _data_ptr(out_status),
                                    ctypes.byref(opts), _ptr(workspace), wbytes, _stream_handle(stream)))


_nd_ready = False
MAX_DIM = 5


def max_constraints_nd(d: int) -> int:
    """LPND_MAX_CONSTRAINTS(d): the largest LP the d-dimensional solver stages."""
    return 8192 - 2 * d


def warp_stage_constraints_nd(d: int) -> int:
    """The largest d-dimensional LP the main kernel stages (half of a CTA's stage); the
    one-warp large-LP kernel takes the larger ones."""
    return 1024 - 2 * d


def solve_batch_nd(a, b, offsets, obj, box, out_x, out_status, options: Options | None = None,
                   workspace: torch.Tensor | None = None, stream=None):
    """lpnd_solve_batch: the batched d-dimensional solver (2 <= d <= 5).

    a: float32 CUDA tensor [d, n_constraints] (row t: coefficient t of every
    constraint) or a sequence of d such 1-D tensors; b float32 [n_constraints];
    offsets int64 [n_lp + 1]; obj float32 [d*n_lp]; box: 2d floats (min_0, max_0,
    min_1, ...); out_x float32 [d*n_lp] (float64 for PREC_FP64); out_status int32
    [n_lp]; workspace as for solve_batch_ex (see new_workspace)."""
    global _nd_ready
    if not _nd_ready:
        vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
        _lib.lpnd_solve_batch.argtypes = [ctypes.c_int, vp, vp, vp, i64, vp, vp, vp, vp, ctypes.POINTER(Options),
                                          vp, sz, vp]
        _lib.lpnd_solve_batch.restype = ctypes.c_int
        _nd_ready = True
    cols = [a[t] for t in range(a.shape[0])] if isinstance(a, torch.Tensor) else list(a)
    d = len(cols)
    if not 2 <= d <= MAX_DIM:
        raise ValueError(f"d = {d} is outside 2..{MAX_DIM}")
    opts = options if options is not None else default_options()
    out_dtype = torch.float64 if opts.precision == PREC_FP64 else torch.float32
    n_lp = offsets.numel() - 1
    if n_lp < 0:
        raise ValueError("offsets needs n_lp + 1 entries")
    _need(cols[0], torch.float32, "a[0]")
    for t in range(1, d):
        _need(cols[t], torch.float32, f"a[{t}]", cols[0].numel())
    _need(b, torch.float32, "b", cols[0].numel())
    _need(offsets, torch.int64, "offsets")
    _need(obj, torch.float32, "obj", d * n_lp)
    _need(out_x, out_dtype, "out_x", d * n_lp)
    _need(out_status, torch.int32, "out_status", n_lp)
    if len(box) != 2 * d:
        raise ValueError(f"box needs {2 * d} values")
    ptrs = (ctypes.c_void_p * d)(*[_data_ptr(c).value for c in cols])
    box_c = (ctypes.c_float * (2 * d))(*[float(v) for v in box])
    wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.lpnd_solve_batch(d, ctypes.cast(ptrs, ctypes.c_void_p), _data_ptr(b), _ptr(offsets), n_lp,
                                 _data_ptr(obj), ctypes.cast(box_c, ctypes.c_void_p), _data_ptr(out_x),
                                 _data_ptr(out_status), ctypes.byref(opts), _ptr(workspace), wbytes,
                                 _stream_handle(stream)))


_lv_ready = False
LEAST_VIOLATION_TMAX_FACTOR = 8.0


def least_violation(ax, ay, b, offsets, box, status_in, out_xy, out_status, out_t=None,
                    options: Options | None = None, workspace: torch.Tensor | None = None, stream=None):
    """lp2d_least_violation: for every LP whose status_in is INFEASIBLE, the point of
    the box with the smallest largest violation (a 3-D LP in (x, y, t)); writes
    out_xy (2 per LP), out_status and, if given, out_t.  Other LPs are untouched."""
    global _lv_ready
    if not _lv_ready:
        vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
        _lib.lp2d_least_violation.argtypes = [vp, vp, vp, vp, i64, Box, vp, vp, vp, vp, ctypes.POINTER(Options), vp,
                                              sz, vp]
        _lib.lp2d_least_violation.restype = ctypes.c_int
        _lv_ready = True
    opts = options if options is not None else default_options()
    out_dtype = torch.float64 if opts.precision == PREC_FP64 else torch.float32
    n_lp = offsets.numel() - 1
    _need(ax, torch.float32, "ax")
    _need(ay, torch.float32, "ay", ax.numel())
    _need(b, torch.float32, "b", ax.numel())
    _need(offsets, torch.int64, "offsets")
    _need(status_in, torch.int32, "status_in", n_lp)
    _need(out_xy, out_dtype, "out_xy", 2 * n_lp)
    _need(out_status, torch.int32, "out_status", n_lp)
    if out_t is not None:
        _need(out_t, torch.float32, "out_t", n_lp)
    wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.lp2d_least_violation(_data_ptr(ax), _data_ptr(ay), _data_ptr(b), _ptr(offsets), n_lp, Box(*box),
                                     _data_ptr(status_in), _data_ptr(out_xy), _ptr(out_t), _data_ptr(out_status),
                                     ctypes.byref(opts), _ptr(workspace), wbytes, _stream_handle(stream)))


_tune_ready = False


def autotune(ax, ay, b, offsets, obj, box, out_xy, out_status, options: Options, workspace: torch.Tensor,
             reps: int = 3, stream=None) -> float:
    """lp2d_autotune: time a grid of (ctas_per_sm, chunk_big, chunk_small) on this batch
    and write the fastest into `options` (in place); returns ms per solve of the winner."""
    global _tune_ready
    if not _tune_ready:
        vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
        _lib.lp2d_autotune.argtypes = [vp, vp, vp, vp, i64, vp, Box, vp, vp, ctypes.POINTER(Options), vp, sz,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_float), vp]
        _lib.lp2d_autotune.restype = ctypes.c_int
        _tune_ready = True
    out_dtype = torch.float64 if options.precision == PREC_FP64 else torch.float32
    n_lp = _validate(ax, ay, b, offsets, obj, out_xy, out_status, out_dtype)
    best = ctypes.c_float(0.0)
    wbytes = workspace.numel() * workspace.element_size()
    _check(_lib.lp2d_autotune(_data_ptr(ax), _data_ptr(ay), _data_ptr(b), _ptr(offsets), n_lp, _data_ptr(obj),
                              Box(*box), _data_ptr(out_xy), _data_ptr(out_status), ctypes.byref(options),
                              _ptr(workspace), wbytes, int(reps), ctypes.byref(best), _stream_handle(stream)))
    return float(best.value)
