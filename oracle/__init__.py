"""CPU oracle for the time-iterated stencil engine (arXiv 1802.00166, PCOT).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline / reference arm of ``bench.py``.  The CUDA library
never imports, links or calls anything here, and nothing here imports the
CUDA library.

Contents
  * ``sweep``        naive FP64 sweeps (C, ``oracle.c``): the plain definition
                     of T steps of the point update.  Pinned by closed forms.
  * ``pcot``         the paper's recursive (cache-oblivious) schedule run on
                     the CPU (C): bounding box, padding, 2^D orthant split,
                     zero/empty exits, lexicographic base loops (Sec. 4).
                     Pinned by bitwise equality with ``sweep``.
  * ``orthant_empty`` / ``padded_box``  the pieces of that recursion.
  * ``grid_sum``     correctly rounded sum of the interior (math.fsum).
  * ``max_rel_error`` / ``pointwise_rel_error`` / ``errors``  the FP32 error
                     measures against the FP64 result: normwise, and per cell
                     with a floor of 1e-3 of the grid's maximum.
  * ``mlp``          FP64 MLP forward/backward/Adam (module ``oracle.mlp``).
  * ``legality``     tile-level hazard checker for tile queues (``oracle.legality``).
  * ``gs2d`` / ``gs2d_pcot`` / ``gs2d_box_empty`` / ``gs2d_tile_order``
                     Gauss-Seidel 2-D (in place, 9-point average): the plain
                     loop nest and the recursive order over its skewed space
                     (C, ``oracle_gs.c``).
  * ``fdtd2d``       FDTD-2D (three fields, a source row): the plain loop nest
                     (C, ``oracle_fdtd.c``).
  * ``lu`` / ``cholesky`` / ``la_pcot`` / ``la_box_empty`` / ``la_tile_order``
                     LU (no pivoting) and Cholesky factorizations: the plain
                     loops and the recursive order over their (k, i, j)
                     space, whose bounding box holds empty orthants (C,
                     ``oracle_la.c``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "oracle_gs.c"), os.path.join(_HERE, "oracle_fdtd.c"),
         os.path.join(_HERE, "oracle_la.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_I64P = ctypes.POINTER(ctypes.c_int64)
_F64P = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with plain IEEE binary64 semantics."""
    if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS):
        return _LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", _LIB + ".tmp"] + _SRCS + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_sweep.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, ctypes.c_int,
                                         _F64P, ctypes.c_int64, _F64P, ctypes.c_int]
            lib.oracle_sweep.restype = ctypes.c_int
            lib.oracle_pcot.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, _F64P,
                                        ctypes.c_int64, _I64P, _F64P, _I64P]
            lib.oracle_pcot.restype = ctypes.c_int
            lib.oracle_padded_box.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, ctypes.c_int64,
                                              _I64P, _I64P, _I64P, _I32P]
            lib.oracle_padded_box.restype = ctypes.c_int
            lib.oracle_orthant_empty.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, ctypes.c_int64,
                                                 _I64P, _I64P]
            lib.oracle_orthant_empty.restype = ctypes.c_int
            lib.oracle_gs2d.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _F64P, ctypes.c_int64]
            lib.oracle_gs2d.restype = ctypes.c_int
            lib.oracle_gs2d_pcot.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _F64P, ctypes.c_int64,
                                             _I64P, _I64P]
            lib.oracle_gs2d_pcot.restype = ctypes.c_int
            lib.oracle_gs2d_box_empty.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _I64P, _I64P]
            lib.oracle_gs2d_box_empty.restype = ctypes.c_int
            lib.oracle_gs2d_tile_order.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _I64P, _I64P,
                                                   ctypes.c_int, _I64P, ctypes.c_int64]
            lib.oracle_gs2d_tile_order.restype = ctypes.c_int64
            lib.oracle_fdtd2d.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _F64P, _F64P, _F64P,
                                          _F64P, ctypes.c_int64]
            lib.oracle_fdtd2d.restype = ctypes.c_int
            lib.oracle_pcot_order.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, ctypes.c_int64, _I64P,
                                              _I64P, ctypes.c_int64]
            lib.oracle_pcot_order.restype = ctypes.c_int64
            lib.oracle_lu.argtypes = [ctypes.c_int64, ctypes.c_int64, _F64P, ctypes.c_int]
            lib.oracle_lu.restype = ctypes.c_int
            lib.oracle_cholesky.argtypes = [ctypes.c_int64, ctypes.c_int64, _F64P, ctypes.c_int]
            lib.oracle_cholesky.restype = ctypes.c_int
            lib.oracle_la_box_empty.argtypes = [ctypes.c_int, ctypes.c_int64, _I64P, _I64P]
            lib.oracle_la_box_empty.restype = ctypes.c_int
            lib.oracle_la_pcot.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _F64P, ctypes.c_int,
                                           _I64P, _I64P]
            lib.oracle_la_pcot.restype = ctypes.c_int
            lib.oracle_la_tile_order.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _I64P, ctypes.c_int,
                                                 _I64P, ctypes.c_int64]
            lib.oracle_la_tile_order.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ptr(a, t):
    return a.ctypes.data_as(t)


def storage_shape(sizes, radius=1, periodic=False):
    if periodic:
        return tuple(int(n) for n in sizes)
    return tuple(int(n) + 2 * radius for n in sizes)


def sweep(grid, sizes, coeffs, T, radius=1, periodic=False, threads=0):
    """T naive steps (Sec. 4.2 point update, t%2 storage) on a copy of ``grid``.

    ``grid`` is in storage layout; any float dtype is widened to float64
    first (the FP32 error reference of the tests).  Returns the float64 grid.
    """
    sizes = _i64(sizes)
    g = np.array(grid, dtype=np.float64, order="C", copy=True)
    if g.shape != storage_shape(sizes, radius, periodic):
        raise ValueError(f"grid shape {g.shape} does not match sizes {tuple(sizes)}")
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    if c.size != 1 + 2 * len(sizes) * radius:
        raise ValueError("wrong number of coefficients")
    rc = _load().oracle_sweep(len(sizes), radius, _ptr(sizes, _I64P), int(bool(periodic)),
                              _ptr(c, _F64P), int(T), _ptr(g, _F64P), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_sweep failed ({rc})")
    return g


def pcot(grid, sizes, coeffs, T, leaf, radius=1, return_stats=False):
    """T steps under the PCOT recursion (Sec. 4), Dirichlet boundaries.

    ``leaf`` = (time extent, skewed extent of axis 0, ...) of a leaf orthant.
    """
    sizes = _i64(sizes)
    leaf = _i64(leaf)
    if leaf.size != len(sizes) + 1:
        raise ValueError("leaf needs dims+1 entries (time first)")
    g = np.array(grid, dtype=np.float64, order="C", copy=True)
    if g.shape != storage_shape(sizes, radius, False):
        raise ValueError("grid shape does not match sizes")
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    stats = np.zeros(6, dtype=np.int64)
    rc = _load().oracle_pcot(len(sizes), radius, _ptr(sizes, _I64P), _ptr(c, _F64P), int(T),
                             _ptr(leaf, _I64P), _ptr(g, _F64P), _ptr(stats, _I64P))
    if rc != 0:
        raise RuntimeError(f"oracle_pcot failed ({rc})")
    if return_stats:
        keys = ("recursive_calls", "base_calls", "zero_exits", "empty_exits", "points", "max_depth")
        return g, dict(zip(keys, (int(v) for v in stats)))
    return g


def pcot_order(sizes, T, leaf, radius=1):
    """Points (t, i_0, ..) in the order the recursion's base function visits
    them (Sec. 4.2-4.5), as an (npoints, dims+1) int64 array."""
    sizes = _i64(sizes)
    leaf = _i64(leaf)
    d = len(sizes)
    lib = _load()
    npts = lib.oracle_pcot_order(d, radius, _ptr(sizes, _I64P), int(T), _ptr(leaf, _I64P), None, 0)
    if npts < 0:
        raise RuntimeError("oracle_pcot_order failed")
    out = np.zeros((max(npts, 1), d + 1), dtype=np.int64)
    lib.oracle_pcot_order(d, radius, _ptr(sizes, _I64P), int(T), _ptr(leaf, _I64P), _ptr(out, _I64P), int(npts))
    return out[:npts]


def padded_box(sizes, T, leaf, radius=1):
    """Bounding box of the skewed domain padded to leaf * 2^k (Sec. 4.5)."""
    sizes = _i64(sizes)
    leaf = _i64(leaf)
    d = len(sizes)
    lo = np.zeros(d + 1, dtype=np.int64)
    size = np.zeros(d + 1, dtype=np.int64)
    lev = np.zeros(d + 1, dtype=np.int32)
    rc = _load().oracle_padded_box(d, radius, _ptr(sizes, _I64P), int(T), _ptr(leaf, _I64P),
                                   _ptr(lo, _I64P), _ptr(size, _I64P), _ptr(lev, _I32P))
    if rc != 0:
        raise RuntimeError("oracle_padded_box failed")
    return lo, size, lev


def orthant_empty(sizes, T, lo, size, radius=1):
    """checkEmpty (Sec. 4.3): 1 = a zero width, 2 = no point of the domain, 0 = work."""
    sizes = _i64(sizes)
    lo = _i64(lo)
    size = _i64(size)
    rc = _load().oracle_orthant_empty(len(sizes), radius, _ptr(sizes, _I64P), int(T),
                                      _ptr(lo, _I64P), _ptr(size, _I64P))
    if rc < 0:
        raise RuntimeError("oracle_orthant_empty failed")
    return rc


# ---- Gauss-Seidel 2-D (oracle_gs.c) -------------------------------------

def gs2d(grid, T):
    """T in-place lexicographic Gauss-Seidel steps of the 9-point average on a
    (n0+2) x (n1+2) FP64 grid with a fixed ring; returns a new array."""
    u = np.ascontiguousarray(np.array(grid, dtype=np.float64))
    n0, n1 = u.shape[0] - 2, u.shape[1] - 2
    if _load().oracle_gs2d(n0, n1, u.shape[1], _ptr(u, _F64P), int(T)) != 0:
        raise ValueError("oracle_gs2d: bad arguments")
    return u


def gs2d_pcot(grid, T, leaf, return_stats=False):
    """The same steps in the paper's recursive order over the skewed space
    (t, t+i, 2t+i+j) with leaf box `leaf` (three widths)."""
    u = np.ascontiguousarray(np.array(grid, dtype=np.float64))
    n0, n1 = u.shape[0] - 2, u.shape[1] - 2
    lf = _i64(leaf)
    st = np.zeros(4, dtype=np.int64)
    if _load().oracle_gs2d_pcot(n0, n1, u.shape[1], _ptr(u, _F64P), int(T), _ptr(lf, _I64P), _ptr(st, _I64P)) != 0:
        raise ValueError("oracle_gs2d_pcot: bad arguments")
    if return_stats:
        return u, dict(leaves=int(st[0]), zero_exits=int(st[1]), empty_exits=int(st[2]), points=int(st[3]))
    return u


def gs2d_box_empty(n0, n1, T, lo, hi):
    """Exact emptiness of an inclusive box of skewed points (t, a, c)."""
    return bool(_load().oracle_gs2d_box_empty(int(n0), int(n1), int(T), _ptr(_i64(lo), _I64P), _ptr(_i64(hi), _I64P)))


def gs2d_tile_order(n0, n1, T, tile, theta, wavefront=False):
    """Non-empty tiles (b0, b1, b2) of the skewed lattice in the recursive
    order (children and leaves lexicographic, or grouped into wavefronts), as
    an (count, 3) int64 array."""
    lib = _load()
    tl, th = _i64(tile), _i64(theta)
    wf = 1 if wavefront else 0
    n = lib.oracle_gs2d_tile_order(int(n0), int(n1), int(T), _ptr(tl, _I64P), _ptr(th, _I64P), wf, None, 0)
    if n < 0:
        raise ValueError("oracle_gs2d_tile_order: bad arguments")
    out = np.zeros((max(n, 1), 3), dtype=np.int64)
    lib.oracle_gs2d_tile_order(int(n0), int(n1), int(T), _ptr(tl, _I64P), _ptr(th, _I64P), wf, _ptr(out, _I64P), n)
    return out[:n]


# ---- FDTD-2D (oracle_fdtd.c) --------------------------------------------

def fdtd2d(ex, ey, hz, fict, T):
    """T steps of FDTD-2D on nx x ny FP64 fields (fict: at least T source
    values); returns new (ex, ey, hz)."""
    ex, ey, hz = (np.ascontiguousarray(np.array(a, dtype=np.float64)) for a in (ex, ey, hz))
    f = np.ascontiguousarray(np.array(fict, dtype=np.float64).reshape(-1))
    if not (ex.shape == ey.shape == hz.shape) or (T > 0 and f.size < T):
        raise ValueError("fdtd2d: field shapes differ or fict too short")
    nx, ny = ex.shape
    fp = _ptr(f, _F64P) if f.size else None
    if _load().oracle_fdtd2d(nx, ny, ny, _ptr(ex, _F64P), _ptr(ey, _F64P), _ptr(hz, _F64P), fp, int(T)) != 0:
        raise ValueError("oracle_fdtd2d: bad arguments")
    return ex, ey, hz


# ---- LU and Cholesky (oracle_la.c) --------------------------------------

LA_KINDS = {"lu": 0, "cholesky": 1}


def _square(A):
    a = np.ascontiguousarray(np.array(A, dtype=np.float64))
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected a square matrix")
    return a


def lu(A, fused=False):
    """In-place LU without pivoting of a square FP64 matrix (unit lower L
    below the diagonal, U on and above it); returns a new array."""
    a = _square(A)
    n = a.shape[0]
    if _load().oracle_lu(n, n, _ptr(a, _F64P), int(bool(fused))) != 0:
        raise ValueError("oracle_lu: bad arguments")
    return a


def cholesky(A, fused=False):
    """In-place lower Cholesky factor of a square FP64 matrix (the strict
    upper triangle is returned unchanged); returns a new array."""
    a = _square(A)
    n = a.shape[0]
    if _load().oracle_cholesky(n, n, _ptr(a, _F64P), int(bool(fused))) != 0:
        raise ValueError("oracle_cholesky: bad arguments")
    return a


def la_pcot(kind, A, leaf, fused=False, return_stats=False):
    """The factorization `kind` ("lu" or "cholesky") in the recursive order
    over its (k, i, j) space with leaf box `leaf` (three widths)."""
    a = _square(A)
    n = a.shape[0]
    lf = _i64(leaf)
    st = np.zeros(4, dtype=np.int64)
    if _load().oracle_la_pcot(LA_KINDS[kind], n, n, _ptr(a, _F64P), int(bool(fused)), _ptr(lf, _I64P),
                              _ptr(st, _I64P)) != 0:
        raise ValueError("oracle_la_pcot: bad arguments")
    if return_stats:
        return a, dict(leaves=int(st[0]), zero_exits=int(st[1]), empty_exits=int(st[2]), points=int(st[3]))
    return a


def la_box_empty(kind, n, lo, hi):
    """Exact emptiness of an inclusive box of (k, i, j) points."""
    return bool(_load().oracle_la_box_empty(LA_KINDS[kind], int(n), _ptr(_i64(lo), _I64P), _ptr(_i64(hi), _I64P)))


def la_tile_order(kind, n, b, theta=(1, 1, 1), recursive=True):
    """Non-empty tiles (kb, ib, jb) of b x b x b tiles in execution order, as
    a (count, 3) int64 array."""
    lib = _load()
    th = _i64(theta)
    r = 1 if recursive else 0
    cnt = lib.oracle_la_tile_order(LA_KINDS[kind], int(n), int(b), _ptr(th, _I64P), r, None, 0)
    if cnt < 0:
        raise ValueError("oracle_la_tile_order: bad arguments")
    out = np.zeros((max(cnt, 1), 3), dtype=np.int64)
    lib.oracle_la_tile_order(LA_KINDS[kind], int(n), int(b), _ptr(th, _I64P), r, _ptr(out, _I64P), cnt)
    return out[:cnt]


def interior(grid, sizes, radius=1, periodic=False):
    """View of the interior points of a storage-layout grid."""
    if periodic:
        return grid
    return grid[tuple(slice(radius, radius + int(n)) for n in sizes)]


def grid_sum(grid, sizes, radius=1, periodic=False):
    """Correctly rounded FP64 sum of the interior values (math.fsum)."""
    return math.fsum(np.asarray(interior(grid, sizes, radius, periodic), dtype=np.float64).ravel().tolist())


def max_rel_error(u, ref):
    """Normwise error max|u - ref| / max|ref| of the FP32 results."""
    u = np.asarray(u, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref))) if ref.size else 0.0
    num = float(np.max(np.abs(u - ref))) if ref.size else 0.0
    return num / den if den > 0 else num


POINTWISE_FLOOR = 1e-3


def pointwise_rel_error(u, ref, floor=POINTWISE_FLOOR):
    """Pointwise error max_x |u(x) - ref(x)| / max(|ref(x)|, floor * max|ref|).

    The normwise error divides every difference by the largest value of the
    grid, so a wrong value in a cell far below that maximum can hide under
    it; this measure divides each cell's difference by the cell's own
    magnitude, floored at `floor` times the maximum so that cells at or near
    zero do not divide by zero."""
    u = np.asarray(u, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    a = np.abs(ref)
    top = float(np.max(a))
    if top == 0.0:
        return float(np.max(np.abs(u - ref)))
    den = np.maximum(a, floor * top)
    return float(np.max(np.abs(u - ref) / den))


def errors(u, ref, floor=POINTWISE_FLOOR):
    """Both error measures of a result against the FP64 reference."""
    return {"normwise": max_rel_error(u, ref), "pointwise": pointwise_rel_error(u, ref, floor),
            "pointwise_floor": floor}
