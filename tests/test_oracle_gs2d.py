"""Pins of the Gauss-Seidel 2-D oracle (GS-2D of the benchmark suite,
Sec. 5.1.2) and of its recursive schedule (Sec. 4 applied to the skewed
iteration space).  CPU only."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _grid_3x4():
    return np.array([[1, 2, 3, 4], [5, 9, 0, 6], [7, 8, 1, 8]], dtype=np.float64)


def test_hand_derived_steps():
    """tests/golden/gs2d_steps.txt: values derived by hand, including the
    point whose result depends on the in-place order."""
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "gs2d_steps.txt"))
            if ln.strip() and not ln.startswith("#")]
    for T, r, c, num, den in ((int(a), int(b), int(c_), int(d), int(e)) for a, b, c_, d, e in rows):
        got = oracle.gs2d(_grid_3x4(), T)
        assert got[r, c] == float(Fraction(num, den)), (T, r, c)


@pytest.mark.parametrize("shape", [(3, 3), (5, 8), (9, 6), (17, 23)])
def test_harmonic_quadratics_are_fixed_points(shape):
    """a + b i + c j + d i j + e (i^2 - j^2) averages to itself over every
    3 x 3 neighbourhood; with small integers all sums are exact, so every
    step reproduces the field bitwise."""
    i, j = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    for a, b, c, d, e in ((3, 2, -1, 0, 0), (-7, 0, 5, 1, 0), (1, 1, 1, 1, 1), (0, -3, 2, -2, 1)):
        u = (a + b * i + c * j + d * i * j + e * (i * i - j * j)).astype(np.float64)
        assert np.array_equal(oracle.gs2d(u, 6), u)


def test_in_place_order_differs_from_two_buffer_update():
    """The oracle updates in place: on random data one step differs from the
    two-buffer (Jacobi-style) 9-point average, except in the first point."""
    u = np.random.default_rng(1).random((8, 11))
    gs = oracle.gs2d(u, 1)
    jac = u.copy()
    box = sum(u[1 + di:u.shape[0] - 1 + di, 1 + dj:u.shape[1] - 1 + dj]
              for di in (-1, 0, 1) for dj in (-1, 0, 1))
    jac[1:-1, 1:-1] = box / 9.0
    assert abs(gs[1, 1] - jac[1, 1]) < 1e-15
    assert np.max(np.abs(gs - jac)) > 1e-3


def test_maximum_principle_error_never_grows():
    """The update is an average, so with a harmonic boundary the interior
    error max|u - h| cannot grow from one step to the next (discrete maximum
    principle), and it shrinks towards 0."""
    n0, n1 = 14, 19
    i, j = np.meshgrid(np.arange(n0 + 2), np.arange(n1 + 2), indexing="ij")
    h = 0.25 + 0.5 * i - 0.125 * j
    u = h.copy()
    u[1:-1, 1:-1] += np.random.default_rng(2).random((n0, n1)) - 0.5
    err = [np.max(np.abs(u - h))]
    for _ in range(40):
        u = oracle.gs2d(u, 1)
        err.append(np.max(np.abs(u - h)))
    assert all(b <= a + 1e-15 for a, b in zip(err, err[1:]))
    assert err[-1] < 0.5 * err[0]


def _tiny_cases():
    rng = np.random.default_rng(3)
    for n0, n1 in ((1, 1), (1, 5), (4, 1), (3, 7), (6, 5)):
        for T in (0, 1, 2, 5):
            for leaf in ((1, 1, 1), (2, 3, 5), (3, 2, 1), (4, 4, 4)):
                yield n0, n1, T, leaf, rng.random((n0 + 2, n1 + 2))


def test_recursive_order_equals_plain_loops_bitwise():
    """The recursion over the skewed space (bounding box, padding, orthants,
    zero/empty exits, lexicographic leaves) reproduces the plain loop nest bit
    for bit on brute-forced tiny problems, leaves of width 1 and non-powers
    of two included, and actually takes both kinds of exit."""
    exits = [0, 0]
    for n0, n1, T, leaf, g in _tiny_cases():
        ref = oracle.gs2d(g, T)
        got, st = oracle.gs2d_pcot(g, T, leaf, return_stats=True)
        assert np.array_equal(got, ref), (n0, n1, T, leaf)
        assert st["points"] == n0 * n1 * T
        exits[0] += st["zero_exits"]
        exits[1] += st["empty_exits"]
    assert exits[0] > 0 and exits[1] > 0


def test_box_emptiness_against_enumeration():
    rng = np.random.default_rng(4)
    for _ in range(500):
        n0, n1, T = (int(v) for v in rng.integers(1, 6, size=3))
        lo = rng.integers(-3, 12, size=3)
        hi = lo + rng.integers(-1, 6, size=3)
        pts = any(1 <= a - t <= n0 and 1 <= c - a - t <= n1 and 0 <= t < T
                  for t in range(lo[0], hi[0] + 1) for a in range(lo[1], hi[1] + 1)
                  for c in range(lo[2], hi[2] + 1))
        assert oracle.gs2d_box_empty(n0, n1, T, lo, hi) == (not pts), (n0, n1, T, lo, hi)


def _tile_points(n0, n1, T, tile, b):
    """Domain points of tile b, as (t, i, j)."""
    out = []
    for t in range(b[0] * tile[0], (b[0] + 1) * tile[0]):
        for a in range(1 + b[1] * tile[1], 1 + (b[1] + 1) * tile[1]):
            for c in range(2 + b[2] * tile[2], 2 + (b[2] + 1) * tile[2]):
                i, j = a - t, c - a - t
                if 0 <= t < T and 1 <= i <= n0 and 1 <= j <= n1:
                    out.append((t, i, j, t + a + c))
    return out


@pytest.mark.parametrize("n0,n1,T,tile,theta", [(5, 7, 4, (2, 2, 3), (1, 2, 2)), (6, 4, 6, (2, 3, 2), (2, 1, 4)),
                                                (3, 9, 5, (3, 2, 4), (1, 1, 1)), (7, 7, 3, (1, 4, 4), (2, 2, 2))])
def test_tile_order_and_wavefronts_reproduce_the_loop_nest(n0, n1, T, tile, theta):
    """Tiled execution as the GPU runs it: tiles in the recursive order, each
    tile's points by wavefront t + a + c with the points of one wavefront in
    random order (they must be independent).  Every non-empty tile appears
    once and the result equals the plain loop nest bitwise; each tile comes
    after its (up to) seven lower lattice neighbours."""
    rng = np.random.default_rng(5)
    g = rng.random((n0 + 2, n1 + 2))
    ref = oracle.gs2d(g, T)
    order = [tuple(b) for b in oracle.gs2d_tile_order(n0, n1, T, tile, theta)]
    assert len(order) == len(set(order))
    lat = [(T + tile[0] - 1) // tile[0], (T - 1 + n0 + tile[1] - 1) // tile[1],
           (2 * T - 3 + n0 + n1 + tile[2] - 1) // tile[2]]
    nonempty = {b for b in itertools.product(*(range(L) for L in lat)) if _tile_points(n0, n1, T, tile, b)}
    assert set(order) == nonempty
    pos = {b: k for k, b in enumerate(order)}
    for b in order:
        for d in itertools.product((0, 1), repeat=3):
            p = (b[0] - d[0], b[1] - d[1], b[2] - d[2])
            if d != (0, 0, 0) and p in pos:
                assert pos[p] < pos[b], (p, b)
    u = g.copy()
    for b in order:
        pts = _tile_points(n0, n1, T, tile, b)
        for tau in sorted({p[3] for p in pts}):
            level = [p for p in pts if p[3] == tau]
            rng.shuffle(level)
            for t, i, j, _ in level:
                s = u[i - 1, j - 1] + u[i - 1, j] + u[i - 1, j + 1]
                s = s + u[i, j - 1] + u[i, j] + u[i, j + 1]
                s = s + u[i + 1, j - 1] + u[i + 1, j] + u[i + 1, j + 1]
                u[i, j] = s / 9.0
    assert np.array_equal(u, ref)
