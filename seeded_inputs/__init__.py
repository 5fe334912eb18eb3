"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and lays them out in the grid storage
format; it contains none of the stencil arithmetic.  Both the CPU oracle and
the CUDA path receive the arrays built here, so the two sides never share any
code that computes the method.

Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Output i of the stream seeded
with ``s`` is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``; a double in [0, 1) is
``(z >> 11) * 2**-53``.  FP32 grids are the round-to-nearest of those doubles.

Storage layout (shared convention of the library and the oracle):
  * row-major, last axis contiguous;
  * Dirichlet: every axis is stored with ``n_a + 2r`` entries, the outer ring of
    width r holds fixed boundary values that are never written;
  * periodic: every axis is stored with ``n_a`` entries.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream ``seed``."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the SplitMix64 stream (53 high bits)."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def storage_shape(sizes, radius: int = 1, periodic: bool = False) -> tuple:
    """Stored extent of every axis for interior sizes ``sizes``."""
    if periodic:
        return tuple(int(n) for n in sizes)
    return tuple(int(n) + 2 * radius for n in sizes)


def uniform_grid(sizes, seed: int, radius: int = 1, periodic: bool = False,
                 ring: str = "zero", dtype=np.float64) -> np.ndarray:
    """Grid of U[0,1) values in storage layout, one draw per stored element.

    ``ring`` (Dirichlet only): ``"zero"`` overwrites the boundary ring with 0
    (the heat configuration), ``"random"`` keeps the drawn values (the
    Jacobi-1D configuration with two seeded boundary values).
    """
    shape = storage_shape(sizes, radius, periodic)
    g = uniform01(seed, int(np.prod(shape))).reshape(shape)
    if not periodic and ring == "zero":
        inner = tuple(slice(radius, radius + int(n)) for n in sizes)
        z = np.zeros_like(g)
        z[inner] = g[inner]
        g = z
    elif not periodic and ring != "random":
        raise ValueError(f"unknown ring mode {ring!r}")
    return np.ascontiguousarray(g.astype(dtype))


def fourier_modes(dims: int, seed: int, nmodes: int = 8, kmax: int = 8):
    """Amplitudes, integer wave vectors and phases of the Fourier initial field.

    Draw order per mode m: A_m = 0.5 + 0.5 u, then one integer component per
    axis k = floor(17 u) - 8 (uniform on [-kmax, kmax] for kmax = 8), then the
    phase 2 pi u.
    """
    per = 2 + dims
    u = uniform01(seed, nmodes * per)
    amps = np.empty(nmodes)
    ks = np.empty((nmodes, dims), dtype=np.int64)
    phases = np.empty(nmodes)
    span = 2 * kmax + 1
    for m in range(nmodes):
        row = u[m * per:(m + 1) * per]
        amps[m] = 0.5 + 0.5 * row[0]
        for a in range(dims):
            ks[m, a] = min(int(math.floor(span * row[1 + a])), span - 1) - kmax
        phases[m] = 2.0 * math.pi * row[1 + dims]
    return amps, ks, phases


def fourier_grid(sizes, seed: int, nmodes: int = 8, dtype=np.float64):
    """Periodic grid u0(x) = sum_m A_m cos(2 pi sum_a k_ma x_a / n_a + phi_m).

    Returns ``(grid, (amps, ks, phases))`` so that a test can evaluate the
    closed-form decay of the same modes.
    """
    dims = len(sizes)
    amps, ks, phases = fourier_modes(dims, seed, nmodes)
    axes = np.meshgrid(*[np.arange(int(n), dtype=np.float64) for n in sizes],
                       indexing="ij", sparse=True)
    g = np.zeros(tuple(int(n) for n in sizes))
    for m in range(nmodes):
        arg = phases[m]
        for a in range(dims):
            arg = arg + 2.0 * math.pi * ks[m, a] * axes[a] / float(sizes[a])
        g = g + amps[m] * np.cos(arg)
    return np.ascontiguousarray(g.astype(dtype)), (amps, ks, phases)


def batched_problem_set(seed: int = 4, count: int = 256, side_lo: int = 256,
                        side_hi: int = 2048, t_lo: int = 64, t_hi: int = 1024):
    """Sides log-uniform in [side_lo, side_hi] and step counts uniform in
    [t_lo, t_hi] for a batch of independent square grids.

    Draws per grid g: u_side, u_T.  side = round(side_lo * (side_hi/side_lo)**u),
    T = t_lo + floor(u * (t_hi - t_lo + 1)).  Grid g's values use the seed
    ``seed * 1_000_003 + g + 1``.
    """
    u = uniform01(seed, 2 * count)
    ratio = side_hi / side_lo
    out = []
    for g in range(count):
        side = int(round(side_lo * ratio ** u[2 * g]))
        side = max(side_lo, min(side_hi, side))
        T = t_lo + min(int(math.floor(u[2 * g + 1] * (t_hi - t_lo + 1))), t_hi - t_lo)
        out.append((side, T, seed * 1_000_003 + g + 1))
    return out


def random_coefficients(dims: int, radius: int, seed: int) -> np.ndarray:
    """Distinct coefficients in [-1, 1) (tests of operand order and signs)."""
    k = 1 + 2 * dims * radius
    return 2.0 * uniform01(seed, k) - 1.0


def dominant_matrix(n: int, seed: int, symmetric: bool = False) -> np.ndarray:
    """n x n FP64 matrix with off-diagonal entries U[0, 1) and diagonal
    entries n + U[0, 1): strictly diagonally dominant, so elimination without
    pivoting is stable; with ``symmetric`` the strict lower triangle's draws
    are mirrored above the diagonal (then the matrix is also positive
    definite, by Gershgorin's theorem).  Draws in row-major order."""
    a = uniform01(seed, n * n).reshape(n, n).copy()
    if symmetric:
        lower = np.tril(a, -1)
        a = lower + lower.T + np.diag(np.diag(a))
    a[np.diag_indices(n)] += float(n)
    return a
