"""Pins of the CPU PCOT executor (Sec. 4) by brute force.

Tiling only reorders legal computations (Sec. 3.1), so the recursive schedule
must reproduce the naive sweep bitwise; checkEmpty must agree with an
enumeration of the orthant's points; the padding must be the least b*2^k.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests import golden
import seeded_inputs as si

HEAT2D = [0.5, 0.125, 0.125, 0.125, 0.125]
JAC3D = [0.4] + [0.1] * 6


def _coeffs(d, seed):
    return si.random_coefficients(d, 1, seed)


@pytest.mark.parametrize("n", list(range(1, 41, 3)))
@pytest.mark.parametrize("T", [0, 1, 2, 3, 7, 16])
def test_pcot_equals_naive_1d(oracle_lib, n, T):
    c = _coeffs(1, n + T)
    g = si.uniform_grid((n,), 100 + n, ring="random")
    ref = oracle.sweep(g, (n,), c, T)
    for leaf in [(1, 1), (2, 3), (3, 5), (4, 4), (T + 1, n + 2 * T)]:
        got, st = oracle.pcot(g, (n,), c, T, leaf, return_stats=True)
        assert np.array_equal(got, ref), (n, T, leaf)
        assert st["points"] == n * T


@pytest.mark.parametrize("sizes", [(1, 1), (2, 5), (7, 3), (11, 13), (23, 29)])
@pytest.mark.parametrize("T", [1, 3, 7])
def test_pcot_equals_naive_2d(oracle_lib, sizes, T):
    c = _coeffs(2, sum(sizes) + T)
    g = si.uniform_grid(sizes, 7 + T, ring="random")
    ref = oracle.sweep(g, sizes, c, T)
    for leaf in [(1, 1, 1), (2, 3, 5), (4, 8, 2), (3, 7, 7)]:
        got, st = oracle.pcot(g, sizes, c, T, leaf, return_stats=True)
        assert np.array_equal(got, ref), (sizes, T, leaf)
        assert st["points"] == sizes[0] * sizes[1] * T


def test_pcot_equals_naive_2d_long(oracle_lib):
    sizes, T = (10, 9), 16
    g = si.uniform_grid(sizes, 3)
    ref = oracle.sweep(g, sizes, HEAT2D, T)
    for leaf in [(2, 2, 2), (5, 3, 6), (16, 40, 40)]:
        assert np.array_equal(oracle.pcot(g, sizes, HEAT2D, T, leaf), ref)


@pytest.mark.parametrize("sizes,T", [((3, 4, 5), 3), ((9, 11, 13), 4), ((5, 2, 7), 7)])
def test_pcot_equals_naive_3d(oracle_lib, sizes, T):
    c = _coeffs(3, sum(sizes))
    g = si.uniform_grid(sizes, 11, ring="random")
    ref = oracle.sweep(g, sizes, c, T)
    for leaf in [(1, 2, 3, 4), (2, 4, 4, 4), (3, 5, 3, 6)]:
        got = oracle.pcot(g, sizes, c, T, leaf)
        assert np.array_equal(got, ref), (sizes, T, leaf)


def test_pcot_radius_two(oracle_lib):
    sizes, T = (13, 9), 5
    c = si.random_coefficients(2, 2, 21)
    g = si.uniform_grid(sizes, 21, radius=2, ring="random")
    ref = oracle.sweep(g, sizes, c, T, radius=2)
    got = oracle.pcot(g, sizes, c, T, (2, 3, 4), radius=2)
    assert np.array_equal(got, ref)


def test_padding_is_least_b_times_power_of_two(oracle_lib):
    for sizes, T, leaf in [((10,), 5, (2, 3)), ((23, 29), 7, (3, 7, 7)), ((5, 6, 7), 4, (1, 2, 3, 4))]:
        lo, size, lev = oracle.padded_box(sizes, T, leaf)
        # bounding box of the skewed domain: t in [1, T], x'_a in [1, T + n_a - 1]
        N = [T] + [T + n - 1 for n in sizes]
        assert lo[0] == 1 and all(lo[1:] == 1)
        for i in range(len(N)):
            assert size[i] == leaf[i] * 2 ** lev[i]
            assert size[i] >= N[i]
            assert lev[i] == 0 or leaf[i] * 2 ** (lev[i] - 1) < N[i]


def _brute_nonempty(sizes, T, lo, size, r=1):
    ranges = [range(lo[i], lo[i] + size[i]) for i in range(len(lo))]
    for p in itertools.product(*ranges):
        t = p[0]
        if not (1 <= t <= T):
            continue
        if all(r * t <= p[1 + a] <= r * t + sizes[a] - 1 for a in range(len(sizes))):
            return True
    return False


def test_check_empty_exact_by_enumeration(oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(600):
        d = int(rng.integers(1, 4))
        sizes = tuple(int(v) for v in rng.integers(1, 6, size=d))
        T = int(rng.integers(1, 6))
        lo = [int(rng.integers(-2, T + 2))] + [int(rng.integers(-2, T + 8)) for _ in range(d)]
        size = [int(rng.integers(0, 5)) for _ in range(d + 1)]
        e = oracle.orthant_empty(sizes, T, lo, size)
        if min(size) == 0:
            assert e == 1
        else:
            assert (e == 0) == _brute_nonempty(sizes, T, lo, size), (sizes, T, lo, size)


def test_early_exits_taken(oracle_lib):
    """Non-cubic leaves produce zero orthants (Sec. 4.3.1) and the skewed box
    produces empty orthants (Sec. 4.3.2)."""
    sizes, T = (20, 20), 12
    g = si.uniform_grid(sizes, 1)
    _, st = oracle.pcot(g, sizes, HEAT2D, T, (12, 2, 2), return_stats=True)
    assert st["zero_exits"] > 0
    assert st["empty_exits"] > 0
    assert st["points"] == 20 * 20 * 12


def _run_points(init, sizes, coeffs, T, order):
    """Execute the points (t, i...) in the given order with the two-buffer
    t%2 storage; returns the grid after T steps (Dirichlet ring kept)."""
    X = [init.copy(), init.copy()]
    d = len(sizes)
    for rec in order:
        t, i = int(rec[0]), [int(v) + 1 for v in rec[1:]]
        src, dst = X[(t - 1) % 2], X[t % 2]
        v = coeffs[0] * src[tuple(i)]
        for a in range(d):
            for k, o in enumerate((-1, 1)):
                j = list(i)
                j[a] += o
                v = v + coeffs[1 + 2 * a + k] * src[tuple(j)]
        dst[tuple(i)] = v
    return X[T % 2]


@pytest.mark.parametrize("case", golden.pcot_orders(), ids=lambda c: c["name"])
def test_pcot_order_hand_derived(oracle_lib, case):
    """The recursion's visit order equals the hand-derived one (Sec. 4.2:
    lexicographic children, time bit most significant, zero and empty
    orthants skipped, lexicographic leaves)."""
    got = oracle.pcot_order(case["sizes"], case["T"], case["leaf"])
    assert np.array_equal(got, case["order"])


def test_pcot_order_pin_catches_a_legal_sibling_swap(oracle_lib):
    """Plant a wrong order on the CPU: run the two independent spatial
    siblings B and C of the 2-D case in swapped order.  The values do not
    change (the swap is legal), so only the order pin can catch it."""
    case = [c for c in golden.pcot_orders() if c["name"] == "order_2d_n3x3_T2"][0]
    order = case["order"]
    b_lo, c_lo, d_lo = 5, 9, 13           # leaves B = rows 5..8, C = rows 9..12
    swapped = np.concatenate([order[:b_lo], order[c_lo:d_lo], order[b_lo:c_lo], order[d_lo:]])
    sizes, T = case["sizes"], case["T"]
    g = si.uniform_grid(sizes, 5, ring="random")
    ref = oracle.sweep(g, sizes, HEAT2D, T)
    assert np.array_equal(_run_points(g, sizes, HEAT2D, T, order), ref)
    assert np.array_equal(_run_points(g, sizes, HEAT2D, T, swapped), ref)   # legal: same values
    assert not np.array_equal(swapped, case["order"])                       # ... but the pin fails
    assert np.array_equal(oracle.pcot_order(sizes, T, case["leaf"]), case["order"])
