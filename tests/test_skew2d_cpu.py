"""Skewed-tile schedule (PCOT_SKEW) through the C ABI, without a GPU: the
non-empty tiles against an enumeration of the skewed points, the queue as a
topological order of the seven-neighbour dependences with the right
predecessor counts, and an emulation of the tile kernel's two-buffer window
(the same window, step rectangles and write-back of the updated cells) under an
adversarial interleaving of concurrently running tiles, whose result must
equal the oracle's loop nest bit for bit."""
import itertools

import numpy as np
import pytest

import oracle
from gpu_util import HEAT2D

pcot = pytest.importorskip("paper_1802_00166_gb300")

# (sizes, T, (kt, ha, wc)), ragged against every tile extent
CASES = [((5, 7), 4, (2, 2, 3)), ((9, 6), 6, (3, 3, 4)), ((3, 11), 5, (1, 2, 5)), ((12, 12), 3, (4, 4, 4)),
         ((1, 1), 1, (2, 2, 2)), ((20, 17), 9, (4, 5, 6)), ((7, 30), 13, (5, 2, 7)), ((16, 16), 8, (8, 8, 8))]


def _params(tile, theta=None):
    return pcot.tile_params(tile=(tile[1], tile[2]), time_depth=tile[0], cot_threshold=theta or (0, 0, 0))


def _decode(ids, lat):
    return [(int(k) // (lat[1] * lat[2]), (int(k) // lat[2]) % lat[1], int(k) % lat[2]) for k in ids]


def _tiles_of_points(sizes, T, tile):
    """Tile of every point (t, i, j) after the skew (t, t + i, t + j); a and c
    start at 1, tiles are numbered from there."""
    kt, ha, wc = tile
    out = set()
    for t in range(T):
        for i in range(1, sizes[0] + 1):
            for j in range(1, sizes[1] + 1):
                out.add((t // kt, (t + i - 1) // ha, (t + j - 1) // wc))
    return out


def _lower(b):
    for d in itertools.product((0, 1), repeat=3):
        if d != (0, 0, 0):
            yield tuple(x - y for x, y in zip(b, d))


@pytest.mark.parametrize("recursive", [False, True])
@pytest.mark.parametrize("sizes,T,tile", CASES)
def test_queue_is_a_topological_order_of_the_nonempty_tiles(sizes, T, tile, recursive):
    theta = (1, 2, 2) if recursive else None
    q = pcot.pcot_skew_plan_query(sizes, T, _params(tile, theta))
    lat = q["lattice"]
    assert q["tile"] == list(tile)
    assert lat == [-(-T // tile[0]), -(-(T - 1 + sizes[0]) // tile[1]), -(-(T - 1 + sizes[1]) // tile[2])]
    tiles = _decode(q["queue"], lat)
    ne = _tiles_of_points(sizes, T, tile)
    assert len(tiles) == len(set(tiles)) == q["n_tiles"]
    assert set(tiles) == ne
    seen = set()
    for b, deps in zip(tiles, q["deps"]):
        preds = [p for p in _lower(b) if p in ne]
        assert all(p in seen for p in preds), b
        assert deps == len(preds), b
        seen.add(b)
    if not recursive:
        assert tiles == sorted(ne, key=lambda b: (sum(b), b))


def test_recursive_order_differs_from_the_wavefront():
    sizes, T, tile = (40, 40), 16, (2, 4, 4)
    wf = pcot.pcot_skew_plan_query(sizes, T, _params(tile))["queue"]
    rc = pcot.pcot_skew_plan_query(sizes, T, _params(tile, (2, 2, 2)))["queue"]
    assert sorted(wf.tolist()) == sorted(rc.tolist())
    assert wf.tolist() != rc.tolist()


def test_dependences_stay_within_one_tile_step():
    """Every read of a point (t, i, j) -- its five operands at level t, and the
    level t - 1 values its write overwrites -- maps, after the skew, to a
    point whose skewed coordinates are lower by 0..2 per axis (time by 0 or
    1); with tiles at least 1 x 2 x 2 that is the tile itself or one of its
    seven lower neighbours."""
    for di, dj in [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]:
        # producer of the operand at (i + di, j + dj): point (t - 1, i + di, j + dj)
        d = (1, 1 - di, 1 - dj)
        assert all(0 <= x <= 2 for x in d) and d[0] == 1
        # readers of level t - 1 at (i, j): points (t - 1, i - di, j - dj); the
        # writer of level t + 1 there must follow them
        d = (1, 1 + di, 1 + dj)
        assert all(0 <= x <= 2 for x in d)
    with pytest.raises(RuntimeError):
        pcot.pcot_skew_plan_query((8, 8), 4, _params((2, 1, 4)))
    with pytest.raises(RuntimeError):
        pcot.pcot_skew_plan_query((8, 8), 4, _params((2, 4, 1)))


class _Tile:
    """The tile kernel's work on one tile, split where concurrency matters:
    load() copies the window of both buffers, finish() runs the steps on the
    copy and writes back the touched cells."""

    def __init__(self, b, sizes, T, tile, coeffs):
        self.b = b
        self.n0, self.n1 = sizes
        kt, self.ha, self.wc = tile
        self.t_lo = b[0] * kt
        self.t_hi = min(self.t_lo + kt, T) - 1
        self.a_lo = 1 + b[1] * self.ha
        self.c_lo = 1 + b[2] * self.wc
        self.rows = self.ha + kt + 1
        self.cols = self.wc + kt + 1
        self.i_lo = self.a_lo - self.t_hi - 1
        self.j_lo = self.c_lo - self.t_hi - 1
        self.c = coeffs

    def load(self, bufs):
        self.win = [np.full((self.rows, self.cols), np.nan) for _ in range(2)]
        for lr in range(self.rows):
            i = self.i_lo + lr
            if not 0 <= i <= self.n0 + 1:
                continue
            for lc in range(self.cols):
                j = self.j_lo + lc
                if 0 <= j <= self.n1 + 1:
                    for x in range(2):
                        self.win[x][lr, lc] = bufs[x][i, j]

    def finish(self, bufs):
        c = self.c
        for t in range(self.t_lo, self.t_hi + 1):
            src, dst = self.win[t % 2], self.win[(t + 1) % 2]
            ia, ib = max(self.a_lo - t, 1), min(self.a_lo + self.ha - 1 - t, self.n0)
            ja, jb = max(self.c_lo - t, 1), min(self.c_lo + self.wc - 1 - t, self.n1)
            if ia > ib or ja > jb:
                continue
            r0, r1 = ia - self.i_lo, ib - self.i_lo + 1
            q0, q1 = ja - self.j_lo, jb - self.j_lo + 1
            assert r0 >= 1 and q0 >= 1 and r1 + 1 <= self.rows and q1 + 1 <= self.cols
            C = src[r0:r1, q0:q1]
            acc = c[0] * C
            acc = acc + c[1] * src[r0 - 1:r1 - 1, q0:q1]
            acc = acc + c[2] * src[r0 + 1:r1 + 1, q0:q1]
            acc = acc + c[3] * src[r0:r1, q0 - 1:q1 - 1]
            acc = acc + c[4] * src[r0:r1, q0 + 1:q1 + 1]
            dst[r0:r1, q0:q1] = acc
        # write-back: cell (i, j) was updated at the tile's steps t with
        # i + t in [a_lo, a_lo + ha) and j + t in [c_lo, c_lo + wc); step t
        # wrote buffer (t + 1) % 2
        for lr in range(self.rows):
            i = self.i_lo + lr
            for lc in range(self.cols):
                j = self.j_lo + lc
                if not (1 <= i <= self.n0 and 1 <= j <= self.n1):
                    continue
                lo = max(self.t_lo, self.a_lo - i, self.c_lo - j)
                hi = min(self.t_hi, self.a_lo + self.ha - 1 - i, self.c_lo + self.wc - 1 - j)
                for x in range(2):
                    if lo <= hi and (hi > lo or (lo + 1) % 2 == x):
                        bufs[x][i, j] = self.win[x][lr, lc]


def _emulate(grid, sizes, T, tile, coeffs, queue, lat, rng, max_running):
    """Pop tiles in queue order; a popped tile loads its window once its
    predecessors have finished; running tiles finish in random order."""
    bufs = [grid.copy(), grid.copy()]
    bufs[1][1:-1, 1:-1] = np.nan  # the twin's interior starts stale
    tiles = _decode(queue, lat)
    ne = set(tiles)
    done, running, pos = set(), [], 0
    while pos < len(tiles) or running:
        can_pop = pos < len(tiles) and len(running) < max_running and all(
            p in done for p in _lower(tiles[pos]) if p in ne)
        if can_pop and (not running or rng.random() < 0.6):
            t = _Tile(tiles[pos], sizes, T, tile, coeffs)
            t.load(bufs)
            running.append(t)
            pos += 1
        else:
            assert running, "queue stalled: the next tile waits on a tile that never ran"
            t = running.pop(int(rng.integers(len(running))))
            t.finish(bufs)
            done.add(t.b)
    return bufs[T % 2]


@pytest.mark.parametrize("recursive", [False, True])
@pytest.mark.parametrize("sizes,T,tile", CASES)
def test_window_emulation_equals_the_loop_nest(sizes, T, tile, recursive):
    rng = np.random.default_rng(sum(sizes) * 131 + T * 7 + tile[0])
    coeffs = np.asarray(HEAT2D, dtype=np.float64) * (1 + 0.1 * rng.standard_normal(5))
    grid = rng.standard_normal(oracle.storage_shape(sizes))
    q = pcot.pcot_skew_plan_query(sizes, T, _params(tile, (1, 2, 2) if recursive else None))
    ref = oracle.sweep(grid, sizes, coeffs, T)
    for max_running in (1, 3, 8):
        got = _emulate(grid, sizes, T, tile, coeffs, q["queue"], q["lattice"], rng, max_running)
        assert np.array_equal(got, ref), max_running
