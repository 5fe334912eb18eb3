"""Pins of the FDTD-2D oracle (the FDTD-2D kernel of the benchmark suite,
Sec. 5.1.2).  CPU only."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _fields():
    ex = np.array([[1, 2, 3], [4, 5, 6]], dtype=np.float64)
    ey = np.array([[0, 1, 0], [2, 2, 2]], dtype=np.float64)
    hz = np.array([[4, 2, 6], [8, 0, 2]], dtype=np.float64)
    return ex, ey, hz


def _value(tok):
    if "+" in tok:
        a, b = tok.split("+")
        return float(a) + float(b.split("*")[0]) * 0.7
    return float(tok)


def test_hand_derived_step():
    """tests/golden/fdtd2d_steps.txt: one step on a 2 x 3 grid derived by hand."""
    ex, ey, hz = oracle.fdtd2d(*_fields(), [3.0], 1)
    got = {"ex": ex, "ey": ey, "hz": hz}
    n = 0
    for ln in open(os.path.join(HERE, "golden", "fdtd2d_steps.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        name, i, j, tok = ln.split()
        assert got[name][int(i), int(j)] == _value(tok), (name, i, j)
        n += 1
    assert n == 18


def _changed(a, b):
    return {tuple(int(v) for v in x) for x in np.argwhere(a != b)}


@pytest.mark.parametrize("i0,j0", [(4, 5), (1, 1), (6, 3)])
def test_one_step_influence_of_each_field(i0, j0):
    """The exact set of cells that a change in one input cell reaches in one
    step (random data, so no accidental cancellation): it fixes every offset
    and direction of the three updates."""
    rng = np.random.default_rng(8)
    nx, ny = 9, 10
    base = [rng.random((nx, ny)) for _ in range(3)]
    fict = [0.25]
    ref = oracle.fdtd2d(*base, fict, 1)
    inside = lambda s: {(i, j) for i, j in s if 0 <= i < nx and 0 <= j < ny}
    hz_rows = lambda s: {(i, j) for i, j in s if i <= nx - 2 and j <= ny - 2}
    # a perturbed hz[i0][j0]
    p = [a.copy() for a in base]
    p[2][i0, j0] += 1.0
    out = oracle.fdtd2d(*p, fict, 1)
    ey_set = inside({(i0, j0), (i0 + 1, j0)}) - {(0, j) for j in range(ny)}
    ex_set = inside({(i0, j0), (i0, j0 + 1)}) - {(i, 0) for i in range(nx)}
    hz_set = hz_rows(inside({(i0, j0), (i0, j0 - 1), (i0, j0 + 1), (i0 - 1, j0), (i0 + 1, j0)})) | {(i0, j0)}
    assert _changed(out[1], ref[1]) == ey_set
    assert _changed(out[0], ref[0]) == ex_set
    assert _changed(out[2], ref[2]) == hz_set
    # a perturbed ex[i0][j0] (j0 >= 1): itself, and hz to its west and at it
    p = [a.copy() for a in base]
    p[0][i0, j0] += 1.0
    out = oracle.fdtd2d(*p, fict, 1)
    assert _changed(out[0], ref[0]) == {(i0, j0)}
    assert _changed(out[1], ref[1]) == set()
    assert _changed(out[2], ref[2]) == hz_rows({(i0, j0), (i0, j0 - 1)})
    # a perturbed ey[i0][j0] (i0 >= 1): itself, and hz above it and at it
    p = [a.copy() for a in base]
    p[1][i0, j0] += 1.0
    out = oracle.fdtd2d(*p, fict, 1)
    assert _changed(out[1], ref[1]) == {(i0, j0)}
    assert _changed(out[2], ref[2]) == hz_rows({(i0, j0), (i0 - 1, j0)})


def test_fields_constant_along_j_follow_the_1d_yee_scheme():
    """With ex = 0 and ey, hz constant along j, columns far enough from the
    right edge (which hz never updates) evolve by the 1-D Yee recurrence
    ey_i <- ey_i - 0.5 (h_i - h_{i-1}), h_i <- h_i - 0.7 (ey_{i+1} - ey_i),
    ey_0 = source; a disturbance from the edge moves one column per step."""
    rng = np.random.default_rng(9)
    nx, ny, T = 12, 40, 9
    e1 = rng.random(nx)
    h1 = rng.random(nx)
    fict = rng.random(T)
    ex = np.zeros((nx, ny))
    ey = np.repeat(e1[:, None], ny, axis=1)
    hz = np.repeat(h1[:, None], ny, axis=1)
    out = oracle.fdtd2d(ex, ey, hz, fict, T)
    e, h = e1.copy(), h1.copy()
    for t in range(T):
        e[0] = fict[t]
        e[1:] = e[1:] - 0.5 * (h[1:] - h[:-1])
        h[:-1] = h[:-1] - 0.7 * (((0.0 - 0.0) + e[1:]) - e[:-1])
    cols = ny - 2 - 2 * T
    assert cols > 0
    assert np.array_equal(out[1][:, :cols], np.repeat(e[:, None], cols, axis=1))
    assert np.array_equal(out[2][:, :cols], np.repeat(h[:, None], cols, axis=1))
    assert np.array_equal(out[0][:, :cols], np.zeros((nx, cols)))


def test_zero_fields_and_source_stay_zero():
    z = np.zeros((7, 5))
    out = oracle.fdtd2d(z, z, z, np.zeros(6), 6)
    assert all(not np.any(a) for a in out)
