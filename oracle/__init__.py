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
  * ``mlp``          FP64 MLP forward/backward/Adam (module ``oracle.mlp``).
  * ``legality``     tile-level hazard checker for tile queues (``oracle.legality``).
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
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_I64P = ctypes.POINTER(ctypes.c_int64)
_F64P = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with plain IEEE binary64 semantics."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC]
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
            lib.oracle_pcot_order.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, ctypes.c_int64, _I64P,
                                              _I64P, ctypes.c_int64]
            lib.oracle_pcot_order.restype = ctypes.c_int64
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
