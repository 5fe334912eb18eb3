"""CPU-side checks of the C ABI: the library loads, exports every declared
symbol, validates arguments, and plans legal recursive tile queues.  No GPU
is touched (planning calls need none)."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import legality

pcot = pytest.importorskip("paper_1802_00166_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEAT2D = [0.5, 0.125, 0.125, 0.125, 0.125]
JAC3D = [0.4] + [0.1] * 6
JAC1D = [1 / 3] * 3


@pytest.fixture(scope="module")
def lib():
    from paper_1802_00166_gb300 import build
    build.build()
    return pcot._load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pcot_\w+)\s*\(", txt, re.M))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"libpcot.so does not export {n}"
    assert set(pcot.exported_symbols()) <= names


def test_status_strings(lib):
    for s in range(8):
        assert pcot.status_string(s)
    assert pcot.status_string(6) == "device dependency wait timed out"


def test_create_validation(lib):
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_create(4, 1, [0.0] * 9, pcot.PCOT_DIRICHLET)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_create(2, 2, [0.0] * 9, pcot.PCOT_DIRICHLET)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_create(2, 1, [0.0] * 4, pcot.PCOT_DIRICHLET)
    assert e.value.status == pcot.PCOT_ERR_INVALID_ARG
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    pcot.pcot_destroy(h)


def test_workspace_size_is_a_grid_twin(lib):
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    n = pcot.pcot_workspace_bytes(h, (100, 60), None, 10, pcot.PCOT_F32, pcot.PCOT_SLT)
    assert n >= 102 * 62 * 4 and n % 256 == 0
    n2 = pcot.pcot_workspace_bytes(h, (100, 60), (64, 1), 10, pcot.PCOT_F64, pcot.PCOT_SLT)
    assert n2 >= (101 * 64 + 62) * 8
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_workspace_bytes(h, (100, 60), (50, 1), 10, pcot.PCOT_F32, pcot.PCOT_SLT)
    assert e.value.status == pcot.PCOT_ERR_INVALID_ARG
    pcot.pcot_destroy(h)


def _storage_extent(sizes, periodic=False):
    return [n if periodic else n + 2 for n in sizes]


@pytest.mark.parametrize("dims,sizes,T,params", [
    (1, (50,), 40, dict(tile=(8,), time_depth=4, cot_threshold=(1, 1))),
    (1, (37,), 33, dict(tile=(5,), time_depth=3, cot_threshold=(2, 2))),
    (2, (20, 300), 16, dict(tile=(8, 0), time_depth=2, cot_threshold=(1, 1, 1))),
    (2, (30, 260), 24, dict(tile=(6, 120), time_depth=4, cot_threshold=(2, 2, 1))),
    (2, (17, 130), 12, dict(tile=(4, 0), time_depth=3, cot_threshold=(4, 8, 8))),
    (3, (9, 10, 70), 8, dict(tile=(4, 4, 0), time_depth=2, cot_threshold=(1, 1, 1, 1))),
])
def test_cot_queue_matches_oracle_recursion_and_is_legal(lib, dims, sizes, T, params):
    coeffs = {1: JAC1D, 2: HEAT2D, 3: JAC3D}[dims]
    h = pcot.pcot_create(dims, 1, coeffs, pcot.PCOT_DIRICHLET)
    p = pcot.tile_params(**params)
    q = pcot.pcot_plan_query(h, sizes, T, pcot.PCOT_F32, p)
    lat, ext, k = q["lattice"], q["tile_ext"][:dims], q["depth"]
    assert lat[0] * k + q["tail_steps"] == T
    assert lat[0] % 2 == 0
    assert q["tail_steps"] >= 0
    # Independent derivation: the oracle's point-level recursion on the lattice
    # domain {1 <= t <= P, t <= x'_a <= t + L_a - 1} visits (t, i) in the order
    # the queue must list tiles (t = b + 1, i = tile index).
    if lat[0] > 0:
        theta = list(params["cot_threshold"])[:dims + 1]
        theta = [max(1, v) for v in theta]
        order = oracle.pcot_order(lat[1:1 + dims], lat[0], theta)
        expect = []
        for row in order:
            b = int(row[0]) - 1
            I = [int(v) for v in row[1:]] + [0] * (3 - dims)
            expect.append(legality.encode(b, I, lat))
        assert list(q["queue"]) == expect
        st = legality.check(lat, ext, k, _storage_extent(sizes), dims, q["queue"], q["deps"])
        assert st["hazards"] > 0
    pcot.pcot_destroy(h)


def test_legality_checker_rejects_bad_orders(lib):
    """Planted mistakes: a swapped pair, a wrong counter, a too-small halo."""
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    p = pcot.tile_params(tile=(6, 120), time_depth=4, cot_threshold=(1, 1, 1))
    sizes = (20, 240)
    q = pcot.pcot_plan_query(h, sizes, 16, pcot.PCOT_F32, p)
    lat, ext, k = q["lattice"], q["tile_ext"][:2], q["depth"]
    queue, deps = list(q["queue"]), list(q["deps"])
    legality.check(lat, ext, k, _storage_extent(sizes), 2, queue, deps)
    # a successor moved before its predecessor
    bad = queue[:]
    j = next(i for i, t in enumerate(bad) if legality.decode(t, lat)[0] == 1)
    bad.insert(0, bad.pop(j))
    bad_deps = [deps[queue.index(t)] for t in bad]
    with pytest.raises(AssertionError):
        legality.check(lat, ext, k, _storage_extent(sizes), 2, bad, bad_deps)
    # a counter one too small (the tile could start early)
    d2 = deps[:]
    j = next(i for i, v in enumerate(d2) if v > 0)
    d2[j] -= 1
    with pytest.raises(AssertionError):
        legality.check(lat, ext, k, _storage_extent(sizes), 2, queue, d2)
    # a halo wider than a tile reaches tiles the counters do not cover
    with pytest.raises(AssertionError):
        legality.check(lat, ext, ext[0] + 1, _storage_extent(sizes), 2, queue, deps)
    pcot.pcot_destroy(h)


def test_cot_unsupported_on_periodic(lib):
    h = pcot.pcot_create(3, 1, JAC3D, pcot.PCOT_PERIODIC)
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_plan_query(h, (16, 16, 16), 8, pcot.PCOT_F32)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    pcot.pcot_destroy(h)


def test_odd_block_counts_leave_even_tail(lib):
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    for T in (1, 3, 5, 7, 9, 13, 17, 31):
        q = pcot.pcot_plan_query(h, (40, 200), T, pcot.PCOT_F32, pcot.tile_params(time_depth=4), with_queue=False)
        assert q["lattice"][0] % 2 == 0
        assert q["lattice"][0] * q["depth"] + q["tail_steps"] == T
    pcot.pcot_destroy(h)


def test_undersized_workspace_rejected_before_launch(lib):
    """The size check happens on the host before any device work, so fake
    (never dereferenced) 256-byte-aligned addresses are enough here."""
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    sizes = (64, 240)
    for sched in (pcot.PCOT_SWEEP, pcot.PCOT_SLT, pcot.PCOT_COT):
        need = pcot.pcot_workspace_bytes(h, sizes, None, 20, pcot.PCOT_F32, sched)
        with pytest.raises(pcot.PcotError) as e:
            pcot.pcot_run(h, 1 << 20, 1 << 24, need - 256, sizes, None, 20, pcot.PCOT_F32, sched, None, 0)
        assert e.value.status == pcot.PCOT_ERR_OOM
    cot = pcot.pcot_workspace_bytes(h, sizes, None, 20, pcot.PCOT_F32, pcot.PCOT_COT)
    slt = pcot.pcot_workspace_bytes(h, sizes, None, 20, pcot.PCOT_F32, pcot.PCOT_SLT)
    assert cot > slt  # the queue image of the recursive schedule lives in the workspace
    pcot.pcot_destroy(h)


def test_candidates_list_host_logic():
    """The picker's candidates (a planning call, no GPU): the sweep first,
    depths the kernels compile, recursive-order candidates only for Dirichlet
    grids, every candidate's feature vector computable."""
    import paper_1802_00166_gb300 as pcot
    for dims, periodic in ((1, False), (2, False), (2, True), (3, True), (3, False)):
        coeffs = {1: [1 / 3] * 3, 2: [0.5] + [0.125] * 4, 3: [0.4] + [0.1] * 6}[dims]
        h = pcot.pcot_create(dims, 1, coeffs, pcot.PCOT_PERIODIC if periodic else pcot.PCOT_DIRICHLET)
        for dt in (pcot.PCOT_F32, pcot.PCOT_F64_EXACT):
            c = pcot.pcot_candidates(h, dt)
            assert c[0][0] == pcot.PCOT_SWEEP and len(c) > 8
            assert len(set((s, tuple(p["tile"]), p["time_depth"], tuple(p["cot_threshold"])) for s, p in c)) == len(c)
            assert all(s in (pcot.PCOT_SWEEP, pcot.PCOT_SLT, pcot.PCOT_COT) for s, _ in c)
            assert any(s == pcot.PCOT_COT for s, _ in c) == (not periodic and dims > 1)
            sizes = {1: (1000,), 2: (300, 500), 3: (40, 50, 64)}[dims]
            for s, p in c:
                f = pcot.pcot_features(h, sizes, 33, dt, s, pcot.tile_params(**p))
                assert f.shape == (12,) and np.all(np.isfinite(f))
        pcot.pcot_destroy(h)


def test_noalloc_limit_parsed_from_the_header():
    import paper_1802_00166_gb300 as pcot
    assert pcot.NOALLOC_MAX_BYTES == 32 * 1024 * 1024


def test_schedule_values_outside_the_enum_are_rejected():
    """Planning calls reject a schedule value that is not one of the enum's,
    and the picker's feature vector is defined only for its own candidates'
    schedules (sweep, single-level, recursive)."""
    h = pcot.pcot_create(2, 1, [0.5, 0.125, 0.125, 0.125, 0.125], pcot.PCOT_DIRICHLET)
    try:
        for bad in (-1, 5, 99):
            with pytest.raises(pcot.PcotError) as e:
                pcot.pcot_workspace_bytes(h, (64, 64), None, 8, pcot.PCOT_F64_EXACT, bad)
            assert e.value.status == pcot.PCOT_ERR_INVALID_ARG
            with pytest.raises(pcot.PcotError) as e:
                pcot.pcot_features(h, (64, 64), 8, pcot.PCOT_F32, bad)
            assert e.value.status == pcot.PCOT_ERR_INVALID_ARG
        for unsupported in (pcot.PCOT_AUTO, pcot.PCOT_SKEW):
            with pytest.raises(pcot.PcotError) as e:
                pcot.pcot_features(h, (64, 64), 8, pcot.PCOT_F32, unsupported)
            assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
        # the skewed schedule's workspace: the twin plus its queue bound
        twin = pcot.pcot_workspace_bytes(h, (64, 64), None, 8, pcot.PCOT_F64_EXACT, pcot.PCOT_SWEEP)
        assert pcot.pcot_workspace_bytes(h, (64, 64), None, 8, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW) > twin
    finally:
        pcot.pcot_destroy(h)
