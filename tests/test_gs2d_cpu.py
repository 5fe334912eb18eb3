"""Gauss-Seidel 2-D planner through the C ABI, without a GPU: the tile
queues against the oracle's independent orders, the dependency counts, and
an emulation of the tile kernel's shared-memory window (bounds of every
access, result equal to the plain loop nest)."""
import itertools

import numpy as np
import pytest

import oracle

pcot = pytest.importorskip("paper_1802_00166_gb300")

CASES = [((5, 7), 4, (2, 2, 3), (1, 2, 2)), ((9, 6), 6, (2, 3, 4), (2, 1, 4)), ((3, 11), 5, (3, 2, 5), (1, 1, 1)),
         ((12, 12), 3, (1, 4, 4), (2, 2, 2)), ((1, 1), 1, (2, 2, 2), (1, 1, 1)), ((20, 17), 9, (4, 5, 6), (2, 2, 3))]


def _params(tile, theta):
    return pcot.tile_params(tile=(tile[1], tile[2]), time_depth=tile[0], cot_threshold=theta)


def _decode(ids, lat):
    return [(int(k) // (lat[1] * lat[2]), (int(k) // lat[2]) % lat[1], int(k) % lat[2]) for k in ids]


def _nonempty(sizes, T, tile, lat):
    out = set()
    for b in itertools.product(*(range(L) for L in lat)):
        lo = [b[0] * tile[0], 1 + b[1] * tile[1], 2 + b[2] * tile[2]]
        hi = [lo[d] + tile[d] - 1 for d in range(3)]
        if not oracle.gs2d_box_empty(sizes[0], sizes[1], T, lo, hi):
            out.add(b)
    return out


@pytest.mark.parametrize("sizes,T,tile,theta", CASES)
def test_wavefront_queue_and_dependency_counts(sizes, T, tile, theta):
    q = pcot.pcot_gs2d_plan_query(sizes, T, pcot.PCOT_SLT, _params(tile, theta))
    lat = q["lattice"]
    assert q["tile"] == list(tile)
    tiles = _decode(q["queue"], lat)
    ne = _nonempty(sizes, T, tile, lat)
    assert tiles == sorted(ne, key=lambda b: (sum(b), b))
    deps = q["deps"].reshape(lat)
    for b in itertools.product(*(range(L) for L in lat)):
        want = 0
        if b in ne:
            want = sum(1 for d in itertools.product((0, 1), repeat=3)
                       if d != (0, 0, 0) and tuple(x - y for x, y in zip(b, d)) in ne)
        assert deps[b] == want, b


@pytest.mark.parametrize("sizes,T,tile,theta", CASES)
def test_recursive_queue_equals_oracle_order(sizes, T, tile, theta):
    """The planner's recursive order (C++) equals the oracle's (C), written
    separately from the paper's description."""
    q = pcot.pcot_gs2d_plan_query(sizes, T, pcot.PCOT_COT, _params(tile, theta))
    ref = [tuple(int(v) for v in b) for b in oracle.gs2d_tile_order(sizes[0], sizes[1], T, tile, theta, wavefront=True)]
    assert _decode(q["queue"], q["lattice"]) == ref


def _emulate(u, sizes, T, tile, order, lat):
    """The tile kernel's steps in numpy: window load, wavefront levels, write
    back of the updated cells.  Asserts every shared-memory index."""
    n0, n1 = sizes
    kt, ha, wc = tile
    R, C = ha + kt + 1, wc + ha + kt
    if (C - 2) % 2 == 0:
        C += 1
    for b0, b1, b2 in order:
        t0, a0, c0 = b0 * kt, 1 + b1 * ha, 2 + b2 * wc
        i_lo = a0 - (t0 + kt - 1) - 1
        j_lo = c0 - (a0 + ha - 1) - (t0 + kt - 1) - 1
        sm = np.full(R * C, np.nan)
        touched = np.zeros(R * C, dtype=bool)
        for k in range(R * C):
            i, j = i_lo + k // C, j_lo + k % C
            if 0 <= i <= n0 + 1 and 0 <= j <= n1 + 1:
                sm[k] = u[i, j]
        for lev in range(kt + ha + wc - 2):
            level = []
            for dt in range(kt):
                for da in range(ha):
                    t, a = t0 + dt, a0 + da
                    i = a - t
                    dc = lev - dt - da
                    j = c0 - a - t + dc
                    if not (t < T and 1 <= i <= n0 and 0 <= dc < wc and 1 <= j <= n1):
                        continue
                    k = (i - i_lo) * C + (c0 - a - t - j_lo) + dc
                    assert 0 <= k - C - 1 and k + C + 1 < R * C
                    level.append(k)
            for k in level:   # independent within a level
                nb = [sm[k - C - 1], sm[k - C], sm[k - C + 1], sm[k - 1], sm[k], sm[k + 1],
                      sm[k + C - 1], sm[k + C], sm[k + C + 1]]
                assert not any(np.isnan(nb))
                s = nb[0]
                for v in nb[1:]:
                    s = s + v
                sm[k] = s / 9.0
                touched[k] = True
        for k in np.nonzero(touched)[0]:
            u[i_lo + k // C, j_lo + k % C] = sm[k]
    return u


@pytest.mark.parametrize("sched", ["slt", "cot"])
@pytest.mark.parametrize("sizes,T,tile,theta", CASES[:4])
def test_kernel_emulation_matches_loop_nest(sched, sizes, T, tile, theta):
    s = pcot.PCOT_SLT if sched == "slt" else pcot.PCOT_COT
    q = pcot.pcot_gs2d_plan_query(sizes, T, s, _params(tile, theta))
    g = np.random.default_rng(7).random((sizes[0] + 2, sizes[1] + 2))
    got = _emulate(g.copy(), sizes, T, tile, _decode(q["queue"], q["lattice"]), q["lattice"])
    assert np.array_equal(got, oracle.gs2d(g, T))


def test_invalid_arguments():
    with pytest.raises(pcot.PcotError):
        pcot.pcot_gs2d_plan_query((0, 5), 3, pcot.PCOT_SLT)
    with pytest.raises(pcot.PcotError):   # a sweep is one step deep
        pcot.pcot_gs2d_plan_query((5, 5), 3, pcot.PCOT_SWEEP, pcot.tile_params(tile=(4, 8), time_depth=2))
    with pytest.raises(pcot.PcotError):   # 64 x 32 threads per tile is above 1024
        pcot.pcot_gs2d_plan_query((5, 5), 3, pcot.PCOT_SLT, pcot.tile_params(tile=(32, 8), time_depth=64))
    assert pcot.pcot_gs2d_workspace_bytes((5, 5), 0, pcot.PCOT_SLT) == 0
