"""Pins of the LU and Cholesky oracles (the linear-algebra kernels of the
benchmark suite, Sec. 5.1.2) and of their recursive order over the (k, i, j)
space, whose bounding box holds empty orthants (Sec. 4.3).  CPU only."""
import itertools
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN_A = {"lu": [[2, 4, -2], [4, 9, -3], [-2, -3, 7]], "cholesky": [[4, 2, -2], [2, 10, 2], [-2, 2, 6]]}


@pytest.mark.parametrize("fused", [False, True])
def test_hand_derived_factorizations(fused):
    """tests/golden/la_steps.txt: both factorizations of a 3 x 3 matrix by hand."""
    got = {k: getattr(oracle, k)(np.array(a, dtype=np.float64), fused=fused) for k, a in GOLDEN_A.items()}
    n = 0
    for ln in open(os.path.join(HERE, "golden", "la_steps.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        kind, i, j, v = ln.split()
        assert got[kind][int(i), int(j)] == float(v), (kind, i, j)
        n += 1
    assert n == 18


def _int_lu(n, seed):
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-3, 4, (n, n)), -1) + np.eye(n)
    U = np.triu(rng.integers(-3, 4, (n, n)), 1) + np.diag(rng.choice([1.0, 2.0, 4.0, -1.0, -2.0, 0.5], n))
    return L.astype(np.float64), U.astype(np.float64)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (12, 3), (20, 4)])
@pytest.mark.parametrize("fused", [False, True])
def test_lu_recovers_integer_factors(n, seed, fused):
    """A = L U with small integer L (unit diagonal) and power-of-two pivots:
    every intermediate value is a small dyadic number, so elimination is exact
    and must return L below the diagonal and U on and above it."""
    L, U = _int_lu(n, seed)
    F = oracle.lu(L @ U, fused=fused)
    assert np.array_equal(np.tril(F, -1), np.tril(L, -1))
    assert np.array_equal(np.triu(F), U)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (6, 2), (13, 3), (20, 4)])
@pytest.mark.parametrize("fused", [False, True])
def test_cholesky_recovers_integer_factor(n, seed, fused):
    """A = L L^T with small integer L and a positive integer diagonal: every
    square root is of a perfect square and every quotient is exact, so the
    lower triangle must equal L and the strict upper triangle stays as it
    was."""
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.diag(rng.integers(1, 4, n))
    A = (L @ L.T).astype(np.float64)
    A[np.triu_indices(n, 1)] = rng.integers(-9, 9, n * (n - 1) // 2)  # the unread upper triangle
    F = oracle.cholesky(A, fused=fused)
    assert np.array_equal(np.tril(F), L.astype(np.float64))
    assert np.array_equal(np.triu(F, 1), np.triu(A, 1))


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.random((n, n))
    return M @ M.T + n * np.eye(n)


@pytest.mark.parametrize("n", [8, 33, 64])
@pytest.mark.parametrize("fused", [False, True])
def test_lu_matches_library_within_backward_error(n, fused):
    """A diagonally dominant matrix needs no row exchange under partial
    pivoting, so LAPACK's getrf (scipy.linalg.lu_factor) computes the same
    factors up to rounding: both agree to a few ulps of |L||U|."""
    sla = pytest.importorskip("scipy.linalg")
    A = _spd(n, 5) + np.diag(np.full(n, 2.0 * n))
    lu, piv = sla.lu_factor(A)
    assert np.array_equal(piv, np.arange(n))
    F = oracle.lu(A, fused=fused)
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    scale = np.abs(L) @ np.abs(U)
    eps = np.finfo(np.float64).eps
    assert np.all(np.abs(F - lu) <= 4 * n * eps * scale)
    assert np.all(np.abs(L @ U - A) <= 4 * n * eps * scale)


@pytest.mark.parametrize("n", [8, 33, 64])
@pytest.mark.parametrize("fused", [False, True])
def test_cholesky_matches_library_within_backward_error(n, fused):
    """numpy.linalg.cholesky (LAPACK potrf) on a symmetric positive definite
    matrix: the same lower factor up to a few ulps of |L||L^T|."""
    A = _spd(n, 6)
    ref = np.linalg.cholesky(A)
    F = np.tril(oracle.cholesky(A, fused=fused))
    eps = np.finfo(np.float64).eps
    scale = np.abs(ref) @ np.abs(ref.T)
    assert np.all(np.abs(F - ref) <= 4 * n * eps * np.sqrt(np.diag(scale))[:, None])
    assert np.all(np.abs(F @ F.T - A) <= 4 * n * eps * scale)


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
def test_fused_flag_changes_rounding(kind):
    """On random data the fused and unfused updates round differently (so the
    flag reaches the arithmetic) but agree to rounding."""
    A = _spd(40, 7) + np.diag(np.full(40, 80.0))
    a = getattr(oracle, kind)(A, fused=False)
    b = getattr(oracle, kind)(A, fused=True)
    assert not np.array_equal(a, b)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def _domain(kind, n):
    pts = set()
    for k, i, j in itertools.product(range(n), repeat=3):
        if (kind == "lu" and k < i and k <= j) or (kind == "cholesky" and k <= j <= i):
            pts.add((k, i, j))
    return pts


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
def test_box_empty_matches_enumeration(kind):
    """The closed-form emptiness test against point enumeration on random
    boxes (including boxes reaching outside [0, n)^3)."""
    rng = np.random.default_rng(11)
    for n in (1, 2, 5, 9):
        pts = _domain(kind, n)
        for _ in range(400):
            lo = rng.integers(-3, n + 2, 3)
            hi = lo + rng.integers(-1, n + 2, 3)
            inside = any(all(lo[d] <= p[d] <= hi[d] for d in range(3)) for p in pts)
            assert oracle.la_box_empty(kind, n, lo, hi) == (not inside), (n, lo, hi)


def _points(kind, n):
    return n * (n - 1) * (n + 1) // 3 if kind == "lu" else n * (n + 1) * (n + 2) // 6


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("n,leaf", [(1, (1, 1, 1)), (2, (1, 1, 1)), (7, (1, 1, 1)), (11, (2, 3, 5)),
                                    (16, (4, 4, 4)), (23, (3, 8, 2)), (30, (64, 64, 64))])
def test_recursive_order_equals_plain_loops(kind, fused, n, leaf):
    """The recursive order (bounding box, padding, orthants, zero and empty
    exits, lexicographic leaves) applies every statement once and bitwise
    reproduces the plain loops; the triangular domains produce empty exits."""
    A = _spd(n, 9) + np.diag(np.full(n, 2.0 * n))
    ref = getattr(oracle, kind)(A, fused=fused)
    got, st = oracle.la_pcot(kind, A, leaf, fused=fused, return_stats=True)
    assert np.array_equal(got, ref)
    # LU: points (k, i, j) with k < i, k <= j; Cholesky: k <= j <= i
    assert st["points"] == _points(kind, n) == len(_domain(kind, n))
    if n >= 7 and max(leaf) < n:
        assert st["empty_exits"] > 0


def _run_tiles(kind, A, order, b, fused):
    """Apply the statements tile by tile in the given order (points of a tile
    lexicographically): a check that the order respects every dependence."""
    a = A.copy()
    n = a.shape[0]
    upd = (lambda c, x, y: np.fma(-x, y, c)) if fused else (lambda c, x, y: c - x * y)
    for kb, ib, jb in order:
        for k in range(kb * b, min(n, (kb + 1) * b)):
            for i in range(ib * b, min(n, (ib + 1) * b)):
                for j in range(jb * b, min(n, (jb + 1) * b)):
                    if kind == "lu" and k < i and k <= j:
                        if j == k:
                            a[i, k] = a[i, k] / a[k, k]
                        else:
                            a[i, j] = upd(a[i, j], a[i, k], a[k, j])
                    elif kind == "cholesky" and k <= j <= i:
                        if j == k and i == k:
                            a[k, k] = np.sqrt(a[k, k])
                        elif j == k:
                            a[i, k] = a[i, k] / a[k, k]
                        else:
                            a[i, j] = upd(a[i, j], a[i, k], a[j, k])
    return a


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
@pytest.mark.parametrize("n,b,theta", [(9, 2, (1, 1, 1)), (13, 3, (2, 1, 2)), (16, 4, (1, 2, 1)), (10, 4, (2, 2, 2))])
def test_tile_orders_are_legal(kind, n, b, theta):
    """Both tile orders list every non-empty tile once and, executed tile by
    tile, reproduce the plain loops bitwise."""
    if not hasattr(np, "fma"):
        fused_cases = [False]
    else:
        fused_cases = [False, True]
    A = _spd(n, 10) + np.diag(np.full(n, 2.0 * n))
    L = -(-n // b)
    tiles = {(k // b, i // b, j // b) for k, i, j in _domain(kind, n)}
    for recursive in (False, True):
        order = [tuple(int(v) for v in t) for t in oracle.la_tile_order(kind, n, b, theta, recursive)]
        assert len(order) == len(set(order)) and set(order) == tiles
        if not recursive:
            assert order == sorted(order)
        for fused in fused_cases:
            assert np.array_equal(_run_tiles(kind, A, order, b, fused), getattr(oracle, kind)(A, fused=fused))
    assert all(0 <= c < L for t in tiles for c in t)
