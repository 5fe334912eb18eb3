"""Tile-level legality checker for persistent-kernel tile queues.

TEST INFRASTRUCTURE ONLY.  Tiling is legal when every tile is atomic and the
dependences between tiles form no cycle (Sec. 3.1); the persistent executor
replaces the paper's task waits (Sec. 4.2) by per-tile dependency counters.
This module checks a queue produced by the library against first principles,
with its own model of what each tile touches:

  tile (b, I) of time block b reads buffer b % 2 on its output box widened by
  the halo (k cells per side, clipped to the stored grid) and writes buffer
  (b + 1) % 2 on its output box.

The sequential meaning is block-by-block execution.  A pair of tiles has a
hazard when one writes cells the other reads or writes in the same buffer;
the earlier one in the sequential meaning must then finish first.  The
executor lets a tile start once every tile of block b-1 at lattice distance
<= 1 has finished (their count is the tile's initial counter).  The checker
verifies that (1) the queue lists every tile once, (2) the initial counters
equal the number of those predecessors, (3) every predecessor is earlier in
the queue (in-order popping cannot deadlock), and (4) every hazardous pair is
ordered by the transitive closure of the predecessor relation.
"""
from __future__ import annotations

import itertools

import numpy as np


def decode(tile_id, lattice):
    """Lattice id ((b*L0 + i0)*L1 + i1)*L2 + i2 -> (b, (i0, i1, i2))."""
    L0, L1, L2 = lattice[1], lattice[2], lattice[3]
    i2 = tile_id % L2
    r = tile_id // L2
    i1 = r % L1
    r //= L1
    i0 = r % L0
    b = r // L0
    return int(b), (int(i0), int(i1), int(i2))


def encode(b, I, lattice):
    L0, L1, L2 = lattice[1], lattice[2], lattice[3]
    return ((b * L0 + I[0]) * L1 + I[1]) * L2 + I[2]


def _box(I, ext, extent, dims, halo):
    lo, hi = [], []
    for a in range(3):
        if a < dims:
            l = I[a] * ext[a] - halo
            h = min((I[a] + 1) * ext[a], extent[a]) + halo
            lo.append(max(l, 0))
            hi.append(min(h, extent[a]))
        else:
            lo.append(0)
            hi.append(1)
    return lo, hi


def _overlap(a, b):
    (alo, ahi), (blo, bhi) = a, b
    return all(max(alo[i], blo[i]) < min(ahi[i], bhi[i]) for i in range(3))


def check(lattice, tile_ext, depth, storage_extent, dims, queue, deps):
    """Raise AssertionError describing the first violation; return stats."""
    P = lattice[0]
    L = [lattice[1], lattice[2], lattice[3]]
    ntiles = P * L[0] * L[1] * L[2]
    queue = [int(q) for q in queue]
    assert len(queue) == ntiles, f"queue has {len(queue)} entries, lattice has {ntiles}"
    assert sorted(queue) == list(range(ntiles)), "queue is not a permutation of the lattice"
    pos = {t: i for i, t in enumerate(queue)}

    def preds(t):
        b, I = decode(t, lattice)
        if b == 0:
            return []
        out = []
        rng = [range(max(0, I[a] - 1), min(L[a], I[a] + 2)) if a < dims else range(1) for a in range(3)]
        for J in itertools.product(*rng):
            out.append(encode(b - 1, J, lattice))
        return out

    for i, t in enumerate(queue):
        p = preds(t)
        assert int(deps[i]) == len(p), f"tile {t}: initial count {deps[i]} != {len(p)} predecessors"
        for u in p:
            assert pos[u] < i, f"tile {t} at {i} waits on tile {u} queued later at {pos[u]}"

    # Transitive predecessors as bitsets, in queue (topological) order.
    anc = {}
    for t in queue:
        m = 0
        for u in preds(t):
            m |= anc[u] | (1 << u)
        anc[t] = m

    ext = list(tile_ext) + [1] * (3 - len(tile_ext))
    extent = list(storage_extent) + [1] * (3 - len(storage_extent))
    reads, writes = {}, {}
    for t in range(ntiles):
        b, I = decode(t, lattice)
        reads[t] = (b % 2, _box(I, ext, extent, dims, depth))
        writes[t] = ((b + 1) % 2, _box(I, ext, extent, dims, 0))
    hazards = 0
    tiles = list(range(ntiles))
    for u in tiles:
        bu, _ = decode(u, lattice)
        for v in tiles:
            bv, _ = decode(v, lattice)
            if bv <= bu:
                continue
            h = False
            if writes[u][0] == reads[v][0] and _overlap(writes[u][1], reads[v][1]):
                h = True   # v reads what u wrote, or a later version must not be overwritten early
            if writes[v][0] == reads[u][0] and _overlap(writes[v][1], reads[u][1]):
                h = True   # v overwrites cells u still has to read
            if writes[v][0] == writes[u][0] and _overlap(writes[v][1], writes[u][1]):
                h = True
            if h:
                hazards += 1
                assert (anc[v] >> u) & 1, f"hazard between tile {u} (block {bu}) and {v} (block {bv}) is unordered"
    return {"tiles": ntiles, "hazards": hazards}
