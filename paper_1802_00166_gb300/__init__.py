"""Python binding of libpcot.so (the GB300 stencil engine's C ABI).

Argument marshalling only: every function forwards to the C entry point of
the same name in ``include/pcot.h``; every step of the computation runs in the
library's CUDA kernels.  PyTorch is used for device memory and streams.  The
library must have been built (``python -m paper_1802_00166_gb300.build``);
importing this module without it raises, there is no other code path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcot.so")

PCOT_OK = 0
PCOT_ERR_INVALID_ARG = 1
PCOT_ERR_UNSUPPORTED = 2
PCOT_ERR_ALIGNMENT = 3
PCOT_ERR_CUDA = 4
PCOT_ERR_OOM = 5
PCOT_ERR_TIMEOUT = 6
PCOT_ERR_BOUNDS = 7

PCOT_DIRICHLET = 0
PCOT_PERIODIC = 1

PCOT_F32 = 0
PCOT_F64 = 1
PCOT_F64_EXACT = 2

PCOT_SWEEP = 0
PCOT_SLT = 1
PCOT_COT = 2
PCOT_AUTO = 3
PCOT_SKEW = 4

SCHEDULES = {"sweep": PCOT_SWEEP, "slt": PCOT_SLT, "cot": PCOT_COT, "auto": PCOT_AUTO, "skew": PCOT_SKEW}

PCOT_LA_LU = 0
PCOT_LA_CHOLESKY = 1
LA_KINDS = {"lu": PCOT_LA_LU, "cholesky": PCOT_LA_CHOLESKY}
DTYPES = {"f32": PCOT_F32, "f64": PCOT_F64, "f64_exact": PCOT_F64_EXACT}


class PcotError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class pcot_tile_params(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32 * 3), ("time_depth", ctypes.c_int32),
                ("cot_threshold", ctypes.c_int32 * 4)]


def tile_params(tile=(0, 0, 0), time_depth=0, cot_threshold=(0, 0, 0, 0)):
    p = pcot_tile_params()
    for i, v in enumerate(list(tile)[:3]):
        p.tile[i] = int(v)
    p.time_depth = int(time_depth)
    for i, v in enumerate(list(cot_threshold)[:4]):
        p.cot_threshold[i] = int(v)
    return p


_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_VP = ctypes.c_void_p
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_1802_00166_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    S = ctypes.c_int
    sig = {
        "pcot_status_string": (ctypes.c_char_p, [S]),
        "pcot_create": (S, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                            ctypes.c_int, ctypes.POINTER(_VP)]),
        "pcot_destroy": (S, [_VP]),
        "pcot_workspace_bytes": (S, [_VP, _I64P, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(pcot_tile_params), ctypes.POINTER(ctypes.c_size_t)]),
        "pcot_run": (S, [_VP, _VP, _VP, ctypes.c_size_t, _I64P, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                         ctypes.POINTER(pcot_tile_params), _VP]),
        "pcot_run_host": (S, [_VP, _VP, _VP, _VP, ctypes.c_size_t, _I64P, _I64P, ctypes.c_int64, ctypes.c_int,
                              ctypes.c_int, ctypes.POINTER(pcot_tile_params), _VP]),
        "pcot_check": (S, [_VP, _VP]),
        "pcot_plan_query": (S, [_VP, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(pcot_tile_params),
                                _I32P, _I32P, _I32P, _I64P, _I64P, _I32P, _I32P, ctypes.c_int64]),
        "pcot_test_wait_timeout": (S, [_VP, _VP, ctypes.c_int32, _VP]),
        "pcot_grid_sum": (S, [_VP, _VP, _I64P, _I64P, ctypes.c_int, _VP, _VP]),
        "pcot_launch_count": (S, [_VP, _I64P]),
        "pcot_batch_workspace_bytes": (S, [_VP, ctypes.c_int, _I64P, _I64P, _I64P, ctypes.c_int,
                                           ctypes.POINTER(pcot_tile_params), ctypes.POINTER(ctypes.c_size_t)]),
        "pcot_batch_create": (S, [_VP, ctypes.c_int, ctypes.POINTER(_VP), _I64P, _I64P, _I64P, ctypes.c_int,
                                  ctypes.POINTER(pcot_tile_params), _VP, ctypes.c_size_t, _VP, _VP,
                                  ctypes.POINTER(_VP)]),
        "pcot_batch_launch": (S, [_VP, _VP]),
        "pcot_batch_destroy": (S, [_VP]),
        "pcot_run_batched": (S, [_VP, ctypes.c_int, ctypes.POINTER(_VP), _I64P, _I64P, _I64P, ctypes.c_int,
                                 ctypes.POINTER(pcot_tile_params), _VP, ctypes.c_size_t, _VP, _VP]),
        "pcot_autotune": (S, [_VP, _VP, _VP, ctypes.c_size_t, _I64P, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(pcot_tile_params), ctypes.c_int,
                              ctypes.POINTER(ctypes.c_float), _VP]),
        "pcot_mlp_param_count": (ctypes.c_int, []),
        "pcot_mlp_scratch_bytes": (S, [ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
        "pcot_mlp_forward": (S, [_VP, _VP, ctypes.c_int, _VP, _VP]),
        "pcot_mlp_grad": (S, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
        "pcot_mlp_adam": (S, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, _VP]),
        "pcot_mlp_argmin": (S, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
        "pcot_features": (S, [_VP, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(pcot_tile_params),
                              ctypes.POINTER(ctypes.c_float)]),
        "pcot_run_noalloc": (S, [_VP, _VP, _I64P, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(pcot_tile_params), _VP]),
        "pcot_gs2d_workspace_bytes": (S, [_I64P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(pcot_tile_params),
                                          ctypes.POINTER(ctypes.c_size_t)]),
        "pcot_gs2d_run": (S, [_VP, _VP, _VP, ctypes.c_size_t, _I64P, _I64P, ctypes.c_int64, ctypes.c_int,
                              ctypes.c_int, ctypes.POINTER(pcot_tile_params), _VP]),
        "pcot_gs2d_plan_query": (S, [_I64P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(pcot_tile_params), _I32P,
                                     _I32P, _I64P, _I32P, _I32P, ctypes.c_int64]),
        "pcot_skew_plan_query": (S, [_I64P, ctypes.c_int64, ctypes.POINTER(pcot_tile_params), _I32P, _I32P, _I64P,
                                     _I32P, _I32P, ctypes.c_int64]),
        "pcot_fdtd2d_workspace_bytes": (S, [_I64P, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(pcot_tile_params), ctypes.POINTER(ctypes.c_size_t)]),
        "pcot_fdtd2d_run": (S, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _I64P, _I64P, ctypes.c_int64,
                                ctypes.c_int, ctypes.c_int, ctypes.POINTER(pcot_tile_params), _VP]),
        "pcot_la_workspace_bytes": (S, [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(pcot_tile_params),
                                        ctypes.POINTER(ctypes.c_size_t)]),
        "pcot_la_run": (S, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_int, ctypes.c_int, ctypes.POINTER(pcot_tile_params), _VP]),
        "pcot_la_plan_query": (S, [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(pcot_tile_params),
                                   _I32P, _I32P, _I64P, _I32P, _I32P, ctypes.c_int64]),
        "pcot_pick_among": (S, [_VP, _I64P, ctypes.c_int64, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(pcot_tile_params), _VP, ctypes.POINTER(ctypes.c_int), _VP]),
        "pcot_pick": (S, [_VP, _I64P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(pcot_tile_params)]),
        "pcot_picker_load": (S, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_float)]),
        "pcot_candidates": (S, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(pcot_tile_params), ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names declared in include/pcot.h that this binding marshals."""
    return ["pcot_gs2d_workspace_bytes", "pcot_gs2d_run", "pcot_gs2d_plan_query", "pcot_skew_plan_query",
            "pcot_fdtd2d_workspace_bytes", "pcot_fdtd2d_run",
            "pcot_la_workspace_bytes", "pcot_la_run", "pcot_la_plan_query",
            "pcot_status_string", "pcot_create", "pcot_destroy", "pcot_workspace_bytes", "pcot_run",
            "pcot_run_host", "pcot_check", "pcot_plan_query", "pcot_test_wait_timeout", "pcot_grid_sum",
            "pcot_launch_count", "pcot_batch_workspace_bytes", "pcot_batch_create", "pcot_batch_launch",
            "pcot_batch_destroy", "pcot_run_batched", "pcot_autotune", "pcot_mlp_param_count",
            "pcot_mlp_scratch_bytes", "pcot_mlp_forward", "pcot_mlp_grad", "pcot_mlp_adam", "pcot_mlp_argmin",
            "pcot_features", "pcot_pick", "pcot_pick_among", "pcot_picker_load", "pcot_candidates",
            "pcot_run_noalloc"]


def status_string(s):
    return _load().pcot_status_string(int(s)).decode()


def _chk(st, where):
    if st != PCOT_OK:
        raise PcotError(st, where)


def _i64(v):
    if v is None:
        return None
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
    return a


def _p64(a):
    return None if a is None else a.ctypes.data_as(_I64P)


def _ptr(t):
    """Device/host address of a tensor, array or integer."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _params(p):
    if p is None:
        return None
    if isinstance(p, pcot_tile_params):
        return ctypes.byref(p)
    if isinstance(p, dict):
        return ctypes.byref(tile_params(**p))
    raise TypeError("params must be pcot_tile_params, a dict or None")


def pcot_create(dims, radius, coeffs, boundary):
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    h = _VP()
    _chk(_load().pcot_create(int(dims), int(radius), c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             int(c.size), int(boundary), ctypes.byref(h)), "pcot_create")
    return h


def pcot_destroy(h):
    _chk(_load().pcot_destroy(h), "pcot_destroy")


def pcot_workspace_bytes(h, sizes, strides, T, dtype, schedule, params=None):
    n = ctypes.c_size_t()
    s, st = _i64(sizes), _i64(strides)
    _chk(_load().pcot_workspace_bytes(h, _p64(s), _p64(st), int(T), int(dtype), int(schedule), _params(params),
                                      ctypes.byref(n)), "pcot_workspace_bytes")
    return int(n.value)


def pcot_run(h, grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedule, params=None, stream=None):
    s, st = _i64(sizes), _i64(strides)
    _chk(_load().pcot_run(h, _ptr(grid), _ptr(workspace), int(workspace_bytes), _p64(s), _p64(st), int(T),
                          int(dtype), int(schedule), _params(params), _stream(stream)), "pcot_run")


def _header_define(name):
    """Integer value of a `#define NAME (expr)` of include/pcot.h (the C ABI
    header is the single source of the library's compile-time limits)."""
    import re
    with open(os.path.join(os.path.dirname(_HERE), "include", "pcot.h")) as f:
        m = re.search(r"#define\s+" + name + r"\s+\(([^)]*)\)", f.read())
    if not m:
        raise ImportError(f"{name} not found in include/pcot.h")
    return int(eval(re.sub(r"(\d+)u\b", r"\1", m.group(1)), {"__builtins__": {}}))


NOALLOC_MAX_BYTES = _header_define("PCOT_NOALLOC_MAX_BYTES")


def pcot_run_noalloc(h, grid, sizes, strides, T, dtype, schedule, params=None, stream=None):
    """pcot_run without a workspace: the library's fixed device array is the twin."""
    s, st = _i64(sizes), _i64(strides)
    _chk(_load().pcot_run_noalloc(h, _ptr(grid), _p64(s), _p64(st), int(T), int(dtype), int(schedule),
                                  _params(params), _stream(stream)), "pcot_run_noalloc")


def pcot_gs2d_workspace_bytes(sizes, T, schedule, params=None):
    n = ctypes.c_size_t()
    _chk(_load().pcot_gs2d_workspace_bytes(_p64(_i64(sizes)), int(T), int(schedule), _params(params),
                                           ctypes.byref(n)), "pcot_gs2d_workspace_bytes")
    return n.value


def pcot_gs2d_run(h, grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedule, params=None, stream=None):
    """Gauss-Seidel 2-D, in place on a device grid (see include/pcot.h)."""
    s, st = _i64(sizes), _i64(strides)
    _chk(_load().pcot_gs2d_run(h, _ptr(grid), _ptr(workspace), int(workspace_bytes), _p64(s), _p64(st), int(T),
                               int(dtype), int(schedule), _params(params), _stream(stream)), "pcot_gs2d_run")


def pcot_gs2d_plan_query(sizes, T, schedule, params=None, with_queue=True):
    lib = _load()
    s = _i64(sizes)
    lat = (ctypes.c_int32 * 3)()
    tl = (ctypes.c_int32 * 3)()
    nt = ctypes.c_int64()
    _chk(lib.pcot_gs2d_plan_query(_p64(s), int(T), int(schedule), _params(params), lat, tl, ctypes.byref(nt),
                                  None, None, 0), "pcot_gs2d_plan_query")
    out = dict(lattice=list(lat), tile=list(tl), n_tiles=nt.value)
    if with_queue:
        ncell = lat[0] * lat[1] * lat[2]
        cap = max(nt.value, ncell)
        qq = np.zeros(cap, dtype=np.int32)
        dd = np.zeros(cap, dtype=np.int32)
        _chk(lib.pcot_gs2d_plan_query(_p64(s), int(T), int(schedule), _params(params), None, None, None,
                                      qq.ctypes.data_as(_I32P), dd.ctypes.data_as(_I32P), cap), "pcot_gs2d_plan_query")
        out["queue"] = qq[:nt.value].copy()
        out["deps"] = dd[:ncell].copy()
    return out


def pcot_skew_plan_query(sizes, T, params=None):
    """PCOT_SKEW plan of a 2-D problem: lattice, tile, n_tiles, and the queue
    of lattice ids in execution order with each entry's predecessor count."""
    lib = _load()
    s = _i64(sizes)
    lat = (ctypes.c_int32 * 3)()
    tl = (ctypes.c_int32 * 3)()
    nt = ctypes.c_int64()
    _chk(lib.pcot_skew_plan_query(_p64(s), int(T), _params(params), lat, tl, ctypes.byref(nt), None, None, 0),
         "pcot_skew_plan_query")
    cap = max(nt.value, 1)
    qq = np.zeros(cap, dtype=np.int32)
    dd = np.zeros(cap, dtype=np.int32)
    _chk(lib.pcot_skew_plan_query(_p64(s), int(T), _params(params), None, None, None, qq.ctypes.data_as(_I32P),
                                  dd.ctypes.data_as(_I32P), cap), "pcot_skew_plan_query")
    return dict(lattice=list(lat), tile=list(tl), n_tiles=nt.value, queue=qq[:nt.value].copy(),
                deps=dd[:nt.value].copy())


def pcot_fdtd2d_workspace_bytes(sizes, strides, T, dtype, schedule, params=None):
    n = ctypes.c_size_t()
    _chk(_load().pcot_fdtd2d_workspace_bytes(_p64(_i64(sizes)), _p64(_i64(strides)), int(T), int(dtype),
                                             int(schedule), _params(params), ctypes.byref(n)),
         "pcot_fdtd2d_workspace_bytes")
    return n.value


def pcot_fdtd2d_run(h, ex, ey, hz, fict, workspace, workspace_bytes, sizes, strides, T, dtype, schedule,
                    params=None, stream=None):
    """FDTD-2D, the three device fields advanced in place (see include/pcot.h)."""
    s, st = _i64(sizes), _i64(strides)
    _chk(_load().pcot_fdtd2d_run(h, _ptr(ex), _ptr(ey), _ptr(hz), _ptr(fict), _ptr(workspace), int(workspace_bytes),
                                 _p64(s), _p64(st), int(T), int(dtype), int(schedule), _params(params),
                                 _stream(stream)), "pcot_fdtd2d_run")


def pcot_la_workspace_bytes(kind, n, schedule, params=None):
    b = ctypes.c_size_t()
    _chk(_load().pcot_la_workspace_bytes(int(kind), int(n), int(schedule), _params(params), ctypes.byref(b)),
         "pcot_la_workspace_bytes")
    return int(b.value)


def pcot_la_run(h, kind, A, workspace, workspace_bytes, n, lda, dtype, schedule, params=None, stream=None):
    """LU or Cholesky of the n x n device matrix A (row stride lda), in place
    (see include/pcot.h)."""
    _chk(_load().pcot_la_run(h, int(kind), _ptr(A), _ptr(workspace), int(workspace_bytes), int(n), int(lda),
                             int(dtype), int(schedule), _params(params), _stream(stream)), "pcot_la_run")


def pcot_la_plan_query(kind, n, schedule, params=None, with_queue=True):
    lib = _load()
    L = ctypes.c_int32()
    b = ctypes.c_int32()
    nt = ctypes.c_int64()
    _chk(lib.pcot_la_plan_query(int(kind), int(n), int(schedule), _params(params), ctypes.byref(L), ctypes.byref(b),
                                ctypes.byref(nt), None, None, 0), "pcot_la_plan_query")
    out = dict(L=L.value, b=b.value, n_tiles=nt.value)
    if with_queue:
        ncell = L.value ** 3
        cap = max(nt.value, ncell)
        qq = np.zeros(cap, dtype=np.int32)
        dd = np.zeros(cap, dtype=np.int32)
        _chk(lib.pcot_la_plan_query(int(kind), int(n), int(schedule), _params(params), None, None, None,
                                    qq.ctypes.data_as(_I32P), dd.ctypes.data_as(_I32P), cap), "pcot_la_plan_query")
        out["queue"] = qq[:nt.value].copy()
        out["deps"] = dd[:ncell].copy()
    return out


def pcot_run_host(h, host_grid, dev_grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedule,
                  params=None, stream=None):
    s, st = _i64(sizes), _i64(strides)
    _chk(_load().pcot_run_host(h, _ptr(host_grid), _ptr(dev_grid), _ptr(workspace), int(workspace_bytes), _p64(s),
                               _p64(st), int(T), int(dtype), int(schedule), _params(params), _stream(stream)),
         "pcot_run_host")


def pcot_check(h, stream=None):
    """Returns the status code (does not raise) so tests can inspect it."""
    return int(_load().pcot_check(h, _stream(stream)))


def pcot_plan_query(h, sizes, T, dtype, params=None, with_queue=True):
    s = _i64(sizes)
    lat = (ctypes.c_int32 * 4)()
    ext = (ctypes.c_int32 * 3)()
    depth = ctypes.c_int32()
    nt = ctypes.c_int64()
    tail = ctypes.c_int64()
    lib = _load()
    _chk(lib.pcot_plan_query(h, _p64(s), int(T), int(dtype), _params(params), lat, ext, ctypes.byref(depth),
                             ctypes.byref(nt), ctypes.byref(tail), None, None, 0), "pcot_plan_query")
    out = dict(lattice=list(lat), tile_ext=list(ext), depth=depth.value, n_tiles=nt.value, tail_steps=tail.value)
    if with_queue and nt.value > 0:
        q = np.zeros(nt.value, dtype=np.int32)
        d = np.zeros(nt.value, dtype=np.int32)
        _chk(lib.pcot_plan_query(h, _p64(s), int(T), int(dtype), _params(params), None, None, None, None, None,
                                 q.ctypes.data_as(_I32P), d.ctypes.data_as(_I32P), int(nt.value)), "pcot_plan_query")
        out["queue"] = q
        out["deps"] = d
    return out


def pcot_test_wait_timeout(h, workspace, timeout_ms, stream=None):
    _chk(_load().pcot_test_wait_timeout(h, _ptr(workspace), int(timeout_ms), _stream(stream)),
         "pcot_test_wait_timeout")


def pcot_grid_sum(h, grid, sizes, strides, dtype, out_device, stream=None):
    s, st = _i64(sizes), _i64(strides)
    _chk(_load().pcot_grid_sum(h, _ptr(grid), _p64(s), _p64(st), int(dtype), _ptr(out_device), _stream(stream)),
         "pcot_grid_sum")


def pcot_launch_count(h):
    n = ctypes.c_int64()
    _chk(_load().pcot_launch_count(h, ctypes.byref(n)), "pcot_launch_count")
    return int(n.value)


def _param_array(params, nb):
    if params is None:
        return None
    arr = (pcot_tile_params * nb)()
    for i, p in enumerate(params):
        arr[i] = p if isinstance(p, pcot_tile_params) else tile_params(**p)
    return arr


def _ptr_array(ptrs):
    arr = (_VP * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = _ptr(p)
    return arr


def pcot_batch_workspace_bytes(h, sizes, strides, T, dtype, params=None):
    nb = len(T)
    n = ctypes.c_size_t()
    _chk(_load().pcot_batch_workspace_bytes(h, nb, _p64(_i64(sizes)), _p64(_i64(strides)), _p64(_i64(T)), int(dtype),
                                            _param_array(params, nb), ctypes.byref(n)), "pcot_batch_workspace_bytes")
    return int(n.value)


def pcot_batch_create(h, grids, sizes, strides, T, dtype, params, workspace, workspace_bytes, done_ns=None,
                      stream=None):
    nb = len(grids)
    b = _VP()
    _chk(_load().pcot_batch_create(h, nb, _ptr_array(grids), _p64(_i64(sizes)), _p64(_i64(strides)), _p64(_i64(T)),
                                   int(dtype), _param_array(params, nb), _ptr(workspace), int(workspace_bytes),
                                   _ptr(done_ns), _stream(stream), ctypes.byref(b)), "pcot_batch_create")
    return b


def pcot_batch_launch(b, stream=None):
    _chk(_load().pcot_batch_launch(b, _stream(stream)), "pcot_batch_launch")


def pcot_batch_destroy(b):
    _chk(_load().pcot_batch_destroy(b), "pcot_batch_destroy")


def pcot_run_batched(h, grids, sizes, strides, T, dtype, params, workspace, workspace_bytes, done_ns=None,
                     stream=None):
    nb = len(grids)
    _chk(_load().pcot_run_batched(h, nb, _ptr_array(grids), _p64(_i64(sizes)), _p64(_i64(strides)), _p64(_i64(T)),
                                  int(dtype), _param_array(params, nb), _ptr(workspace), int(workspace_bytes),
                                  _ptr(done_ns), _stream(stream)), "pcot_run_batched")


def _sched_array(scheds):
    arr = (ctypes.c_int * len(scheds))()
    for i, v in enumerate(scheds):
        arr[i] = int(v)
    return arr


def pcot_autotune(h, grid, workspace, workspace_bytes, sizes, strides, T, dtype, schedules, params, reps=2,
                  stream=None):
    """Mean milliseconds per candidate (-1 where the library rejects it)."""
    n = len(schedules)
    out = (ctypes.c_float * n)()
    _chk(_load().pcot_autotune(h, _ptr(grid), _ptr(workspace), int(workspace_bytes), _p64(_i64(sizes)),
                               _p64(_i64(strides)), int(T), int(dtype), n, _sched_array(schedules),
                               _param_array(params, n), int(reps), out, _stream(stream)), "pcot_autotune")
    return [float(v) for v in out]


def pcot_mlp_param_count():
    return int(_load().pcot_mlp_param_count())


def pcot_mlp_scratch_bytes(batch):
    n = ctypes.c_size_t()
    _chk(_load().pcot_mlp_scratch_bytes(int(batch), ctypes.byref(n)), "pcot_mlp_scratch_bytes")
    return int(n.value)


def pcot_mlp_forward(params, x, batch, y, stream=None):
    _chk(_load().pcot_mlp_forward(_ptr(params), _ptr(x), int(batch), _ptr(y), _stream(stream)), "pcot_mlp_forward")


def pcot_mlp_grad(params, x, target, batch, grad, loss, scratch, scratch_bytes, stream=None):
    _chk(_load().pcot_mlp_grad(_ptr(params), _ptr(x), _ptr(target), int(batch), _ptr(grad), _ptr(loss),
                               _ptr(scratch), int(scratch_bytes), _stream(stream)), "pcot_mlp_grad")


def pcot_mlp_adam(params, grad, m, v, n, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _chk(_load().pcot_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(n), int(step), float(lr),
                               float(beta1), float(beta2), float(eps), _stream(stream)), "pcot_mlp_adam")


def pcot_mlp_argmin(y, n, stride, col, out_index, stream=None):
    _chk(_load().pcot_mlp_argmin(_ptr(y), int(n), int(stride), int(col), _ptr(out_index), _stream(stream)),
         "pcot_mlp_argmin")


def pcot_features(h, sizes, T, dtype, schedule, params=None):
    out = (ctypes.c_float * 12)()
    _chk(_load().pcot_features(h, _p64(_i64(sizes)), int(T), int(dtype), int(schedule), _params(params), out),
         "pcot_features")
    return np.array(list(out), dtype=np.float32)


def pcot_pick_among(h, sizes, T, dtype, mlp_params, feat_mean, feat_std, schedules, params, scratch, stream=None):
    """Index of the candidate with the least predicted time under an explicit
    model (device parameters) and candidate list."""
    n = len(schedules)
    mean = (ctypes.c_float * 12)(*[float(v) for v in feat_mean])
    std = (ctypes.c_float * 12)(*[float(v) for v in feat_std])
    best = ctypes.c_int(-1)
    _chk(_load().pcot_pick_among(h, _p64(_i64(sizes)), int(T), int(dtype), _ptr(mlp_params), mean, std, n,
                                 _sched_array(schedules), _param_array(params, n), _ptr(scratch), ctypes.byref(best),
                                 _stream(stream)), "pcot_pick_among")
    return int(best.value)


def params_dict(p):
    """A pcot_tile_params as the keyword dict tile_params() takes."""
    return dict(tile=tuple(int(v) for v in p.tile), time_depth=int(p.time_depth),
                cot_threshold=tuple(int(v) for v in p.cot_threshold))


def pcot_pick(h, sizes, T, dtype):
    """(schedule, tile-parameter dict) the library picks for a problem: its
    loaded model, else the autotuner."""
    sched = ctypes.c_int(-1)
    p = pcot_tile_params()
    _chk(_load().pcot_pick(h, _p64(_i64(sizes)), int(T), int(dtype), ctypes.byref(sched), ctypes.byref(p)),
         "pcot_pick")
    return int(sched.value), params_dict(p)


def pcot_picker_load(h, mlp_params=None, feat_mean=None, feat_std=None):
    """Load a model (host arrays) into the handle; no arguments unload it."""
    if mlp_params is None:
        _chk(_load().pcot_picker_load(h, None, None, None), "pcot_picker_load")
        return
    n = pcot_mlp_param_count()
    P = (ctypes.c_float * n)(*[float(v) for v in np.asarray(mlp_params, dtype=np.float32)])
    m = (ctypes.c_float * 12)(*[float(v) for v in feat_mean])
    s = (ctypes.c_float * 12)(*[float(v) for v in feat_std])
    _chk(_load().pcot_picker_load(h, P, m, s), "pcot_picker_load")


def pcot_candidates(h, dtype):
    """[(schedule, tile-parameter dict)] the picker chooses among."""
    n = ctypes.c_int(0)
    _chk(_load().pcot_candidates(h, int(dtype), 0, None, None, ctypes.byref(n)), "pcot_candidates")
    sc = (ctypes.c_int * max(n.value, 1))()
    pr = (pcot_tile_params * max(n.value, 1))()
    _chk(_load().pcot_candidates(h, int(dtype), n.value, sc, pr, ctypes.byref(n)), "pcot_candidates")
    return [(int(sc[i]), params_dict(pr[i])) for i in range(n.value)]


def library_path():
    return LIB_PATH
