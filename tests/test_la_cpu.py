"""Host side of the LU / Cholesky path (the linear-algebra kernels of the
benchmark suite, Sec. 5.1.2): the tile planner behind the C ABI against the
oracle's tile orders, its dependency counts against a tile graph that is
checked here against every point dependence, and argument handling.  CPU
only (no kernel runs)."""
import itertools

import numpy as np
import pytest

import oracle
import paper_1802_00166_gb300 as pcot

KINDS = {"lu": pcot.PCOT_LA_LU, "cholesky": pcot.PCOT_LA_CHOLESKY}


def _in_domain(kind, k, i, j):
    return (k < i and k <= j) if kind == "lu" else (k <= j <= i)


def _tile_nonempty(kind, n, b, kb, ib, jb):
    for k in range(kb * b, min(n, (kb + 1) * b)):
        for i in range(ib * b, min(n, (ib + 1) * b)):
            for j in range(jb * b, min(n, (jb + 1) * b)):
                if _in_domain(kind, k, i, j):
                    return True
    return False


def _rule_edges(kind, n, b, ne=None):
    """Edges of the blocked algorithm's tile graph: a block's next update
    waits for its previous one, a panel for its diagonal block, an update for
    the panels it reads (Cholesky reads column block ib and column block jb).
    `ne`: the non-empty tiles (found point by point when not given)."""
    L = -(-n // b)
    if ne is None:
        ne = {t for t in itertools.product(range(L), repeat=3) if _tile_nonempty(kind, n, b, *t)}
    edges = set()
    for kb, ib, jb in ne:
        preds = [(kb - 1, ib, jb)]
        if kind == "lu":
            if (ib, jb) != (kb, kb) and (ib == kb or jb == kb):
                preds.append((kb, kb, kb))
            if ib > kb and jb > kb:
                preds += [(kb, ib, kb), (kb, kb, jb)]
        else:
            if jb == kb and ib > kb:
                preds.append((kb, kb, kb))
            if jb > kb:
                preds += [(kb, ib, kb), (kb, jb, kb)]
        for p in preds:
            if p in ne:
                edges.add((p, (kb, ib, jb)))
    return ne, edges


def _point_deps(kind, n):
    """Every dependence (flow, anti, output) between statement instances of
    the plain loops, found by replaying them and tracking accesses."""
    last_w, readers = {}, {}
    deps = set()

    def access(p, reads, write):
        for e in reads:
            if e in last_w:
                deps.add((last_w[e], p))
        if write in last_w:
            deps.add((last_w[write], p))
        for r in readers.get(write, ()):
            if r != p:
                deps.add((r, p))
        for e in reads:
            readers.setdefault(e, set()).add(p)
        readers[write] = set()
        last_w[write] = p

    for k in range(n):
        if kind == "cholesky":
            access((k, k, k), [(k, k)], (k, k))
        for i in range(k + 1, n):
            access((k, i, k), [(i, k), (k, k)], (i, k))
        for i in range(k + 1, n):
            for j in range(k + 1, n if kind == "lu" else i + 1):
                access((k, i, j), [(i, j), (i, k), (k, j) if kind == "lu" else (j, k)], (i, j))
    return deps


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
@pytest.mark.parametrize("n,b", [(7, 2), (9, 3), (10, 4), (8, 8), (11, 2), (13, 5)])
def test_tile_graph_covers_every_point_dependence(kind, n, b):
    """For each point dependence between two different tiles, the source tile
    reaches the target tile in the graph the executor releases along.  (The
    LU graph routes a block's pivot through its diagonal tile, which holds a
    point whenever the block has two rows or more: b >= 2; the library's
    tiles are 32 or 64 wide.)"""
    ne, edges = _rule_edges(kind, n, b)
    succ = {}
    for a, c in edges:
        succ.setdefault(a, set()).add(c)
    reach = {}

    def reachable(t):
        if t not in reach:
            r = set()
            for c in succ.get(t, ()):
                r.add(c)
                r |= reachable(c)
            reach[t] = r
        return reach[t]

    T = lambda p: (p[0] // b, p[1] // b, p[2] // b)
    for q, p in _point_deps(kind, n):
        assert _in_domain(kind, *q) and _in_domain(kind, *p)
        tq, tp = T(q), T(p)
        if tq != tp:
            assert tp in reachable(tq), (q, p)
    # every edge has non-negative components (so any order respecting them
    # and the lexicographic / recursive orders are compatible)
    assert all(all(c[d] >= a[d] for d in range(3)) for a, c in edges)


def _ids(order, L):
    return [int((k * L + i) * L + j) for k, i, j in order]


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
@pytest.mark.parametrize("n,b,theta", [(1, 32, (2, 2, 2)), (33, 32, (1, 1, 1)), (100, 32, (2, 2, 2)),
                                       (200, 32, (1, 2, 4)), (257, 64, (2, 2, 2)), (300, 32, (4, 4, 4)),
                                       (129, 64, (1, 1, 1)), (480, 32, (2, 4, 1))])
def test_planner_orders_match_oracle(kind, n, b, theta):
    p = pcot.tile_params(tile=(b, 0, 0), cot_threshold=theta)
    for sched, rec in ((pcot.PCOT_SLT, False), (pcot.PCOT_COT, True)):
        q = pcot.pcot_la_plan_query(KINDS[kind], n, sched, p)
        L = q["L"]
        assert L == -(-n // b) and q["b"] == b
        ref = oracle.la_tile_order(kind, n, b, theta, recursive=rec)
        assert list(q["queue"]) == _ids(ref, L)


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
@pytest.mark.parametrize("n,b", [(1, 32), (33, 32), (97, 32), (200, 64), (300, 32)])
def test_planner_dependency_counts(kind, n, b):
    """Per tile, the planner's counter equals its in-degree in the tile graph
    (whose coverage of the point dependences is checked above)."""
    q = pcot.pcot_la_plan_query(KINDS[kind], n, pcot.PCOT_COT, pcot.tile_params(tile=(b, 0, 0)))
    L = q["L"]
    if n <= 97:
        ne, edges = _rule_edges(kind, n, b)
    else:
        # larger n: non-emptiness in closed form (every tile of the pyramid holds
        # points except an LU diagonal tile of a one-row last block)
        ne = set()
        for kb, ib, jb in itertools.product(range(L), repeat=3):
            if kind == "lu":
                ok = ib >= kb and jb >= kb and not (ib == kb and min(n, (kb + 1) * b) - kb * b < 2)
            else:
                ok = kb <= jb <= ib
            if ok:
                ne.add((kb, ib, jb))
        ne, edges = _rule_edges(kind, n, b, ne)
    indeg = np.zeros(L ** 3, dtype=np.int64)
    for _, c in edges:
        indeg[(c[0] * L + c[1]) * L + c[2]] += 1
    assert sorted(_ids(sorted(ne), L)) == sorted(int(x) for x in q["queue"])
    assert np.array_equal(q["deps"].astype(np.int64), indeg)


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
def test_recursive_order_exits_empty_orthants(kind):
    """The pyramid fills about a third (LU) or a sixth (Cholesky) of the
    lattice cube, so the recursive plan lists far fewer tiles than L^3."""
    q = pcot.pcot_la_plan_query(KINDS[kind], 4000, pcot.PCOT_COT, pcot.tile_params(tile=(64, 0, 0)))
    L = q["L"]
    frac = q["n_tiles"] / L ** 3
    assert (0.3 < frac < 0.36) if kind == "lu" else (0.15 < frac < 0.19)


def test_workspace_and_arguments():
    for k in KINDS.values():
        assert pcot.pcot_la_workspace_bytes(k, 3000, pcot.PCOT_SWEEP) == 0
        assert pcot.pcot_la_workspace_bytes(k, 3000, pcot.PCOT_SLT) == 0
        L = -(-3000 // 64)
        assert pcot.pcot_la_workspace_bytes(k, 3000, pcot.PCOT_COT) >= 2 * 4 * L ** 3
        assert pcot.pcot_la_workspace_bytes(k, 0, pcot.PCOT_COT) == 0
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_la_workspace_bytes(pcot.PCOT_LA_LU, 100, pcot.PCOT_COT, pcot.tile_params(tile=(48, 0, 0)))
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_la_workspace_bytes(7, 100, pcot.PCOT_COT)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_la_workspace_bytes(pcot.PCOT_LA_LU, 100, pcot.PCOT_AUTO)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_la_plan_query(pcot.PCOT_LA_LU, 0, pcot.PCOT_COT)
    assert e.value.status == pcot.PCOT_ERR_INVALID_ARG
