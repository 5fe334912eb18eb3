"""Parity at the full workload sizes, in the launch configurations the
benchmark times.  The oracle (FP64 naive sweeps, all host cores) computes the
whole grid; FP64 exact mode must match bitwise, FP32 within 1e-5 of the oracle
run on the widened FP32 inputs (normwise, and cell by cell for the positive
Heat-2D fields), the FP64 FMA mode within its rounding bound.  The periodic
Jacobi-3D case is also checked against the closed-form decay of its Fourier
modes.  Every configuration the benchmark reports is covered here: the
headline recursive-order run, the single-level and sweep schedules beside it,
the FP64 schedules at the same size, Jacobi-3D at the depths it scans, and the
256-grid batch under every tile shape its autotuner tries."""
import math
import os

import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from paper_1802_00166_gb300 import tuner  # noqa: E402
from tests.gpu_util import (F32_POINTWISE_TOL_SIGNED, HEAT2D, JAC1D, JAC3D,  # noqa: E402
                            assert_f32_close, fma_mode_f64_bound, run_gpu)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = os.cpu_count() or 1
# The benchmark's timed configuration (bench.py BEST): recursive-order
# persistent executor, tiles of depth 8, 80 rows x one warp, leaf orthants of
# 2 blocks x 256 x 256 tiles, rows padded to 128 bytes.
BENCH_PARAMS = dict(tile=(80, 112), time_depth=8, cot_threshold=(2, 256, 256))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()
    oracle.build()


def _padded_strides(shape, elem):
    step = 128 // elem
    inner = ((shape[-1] + step - 1) // step) * step
    st = [1] * len(shape)
    acc = inner
    for a in range(len(shape) - 2, -1, -1):
        st[a] = acc
        acc *= shape[a]
    return st


def test_jacobi1d_config_bit_exact():
    """Jacobi-1D 3-point FP64, n = 4096, T = 1024, weights 1/3, seeded ring."""
    n, T = 4096, 1024
    h = pcot.pcot_create(1, 1, JAC1D, pcot.PCOT_DIRICHLET)
    g = si.uniform_grid((n,), 1, ring="random")
    ref = oracle.sweep(g, (n,), JAC1D, T)
    for sched, p in ((pcot.PCOT_SWEEP, None), (pcot.PCOT_SLT, pcot.tile_params(tile=(32,), time_depth=32)),
                     (pcot.PCOT_COT, pcot.tile_params(tile=(64,), time_depth=16, cot_threshold=(4, 4)))):
        got = run_gpu(h, g, (n,), T, pcot.PCOT_F64_EXACT, sched, p)
        assert np.array_equal(got, ref), sched
    pcot.pcot_destroy(h)


@pytest.fixture(scope="module")
def heat2d_full():
    n, T = 8192, 512
    g32 = si.uniform_grid((n, n), 2, dtype=np.float32)
    ref = oracle.sweep(g32, (n, n), HEAT2D, T, threads=THREADS)
    return n, T, g32, ref


# Schedules the benchmark times at 8192^2 beside the headline (FP32), with the
# tile shapes it uses: the single-level schedule at its best depth and the
# recursive order at the depths of its depth scan.
FP32_RUNS = [
    ("cot-k8-headline", "cot", dict(BENCH_PARAMS)),
    ("slt-k8", "slt", dict(BENCH_PARAMS)),
    ("slt-k4", "slt", dict(tile=(40, 112), time_depth=4, cot_threshold=(2, 256, 256))),
    ("cot-k2", "cot", dict(tile=(80, 112), time_depth=2, cot_threshold=(2, 256, 256))),
    ("cot-k4", "cot", dict(tile=(80, 112), time_depth=4, cot_threshold=(2, 256, 256))),
    ("cot-k6", "cot", dict(tile=(96, 112), time_depth=6, cot_threshold=(2, 256, 256))),
    ("cot-l2-leaves", "cot", dict(tile=(32, 112), time_depth=8, cot_threshold=(8, 8, 8))),
    ("sweep", "sweep", None),
]
SCHED = {"sweep": pcot.PCOT_SWEEP, "slt": pcot.PCOT_SLT, "cot": pcot.PCOT_COT, "skew": pcot.PCOT_SKEW}


@pytest.mark.parametrize("name,sched,prm", FP32_RUNS, ids=[r[0] for r in FP32_RUNS])
def test_heat2d_8192_fp32_bench_configs(heat2d_full, name, sched, prm):
    n, T, g32, ref = heat2d_full
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    st = _padded_strides(g32.shape, 4)
    p = pcot.tile_params(**prm) if prm else None
    got = run_gpu(h, g32, (n, n), T, pcot.PCOT_F32, SCHED[sched], p, strides=st)
    assert_f32_close(got, ref, (n, n), what=name)
    assert np.array_equal(got[0], g32[0]) and np.array_equal(got[-1], g32[-1])
    assert np.array_equal(got[:, 0], g32[:, 0]) and np.array_equal(got[:, -1], g32[:, -1])
    pcot.pcot_destroy(h)


FP64_RUNS = [
    ("slt-k2", "slt", dict(tile=(128, 0), time_depth=2)),
    ("slt-k4", "slt", dict(tile=(64, 56), time_depth=4)),
    ("cot-k4", "cot", dict(tile=(64, 56), time_depth=4, cot_threshold=(2, 256, 256))),
    ("sweep", "sweep", None),
    ("skew-k4", "skew", dict(tile=(32, 64), time_depth=4)),
    ("slt-k1", "slt", dict(tile=(64, 0), time_depth=1)),
]


@pytest.mark.parametrize("name,sched,prm", FP64_RUNS, ids=[r[0] for r in FP64_RUNS])
def test_heat2d_8192_fp64_exact_bitwise(heat2d_full, name, sched, prm):
    """The same inputs widened to FP64, FP64 exact mode: bitwise equal."""
    n, T, g32, ref = heat2d_full
    g64 = g32.astype(np.float64)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    st = _padded_strides(g64.shape, 8)
    got = run_gpu(h, g64, (n, n), T, pcot.PCOT_F64_EXACT, SCHED[sched],
                  pcot.tile_params(**prm) if prm else None, strides=st)
    assert np.array_equal(got, ref), name
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("name,sched,prm", [FP64_RUNS[2], FP64_RUNS[3], FP64_RUNS[4]],
                         ids=["cot-k4", "sweep", "skew-k4"])
def test_heat2d_8192_fp64_fma_mode(heat2d_full, name, sched, prm):
    """PCOT_F64 (FMA) against the FP64 oracle: within the rounding bound of
    five roundings per term and step on each side (positive fields)."""
    n, T, g32, ref = heat2d_full
    g64 = g32.astype(np.float64)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    st = _padded_strides(g64.shape, 8)
    got = run_gpu(h, g64, (n, n), T, pcot.PCOT_F64, SCHED[sched],
                  pcot.tile_params(**prm) if prm else None, strides=st)
    err = oracle.pointwise_rel_error(oracle.interior(got, (n, n)), oracle.interior(ref, (n, n)))
    assert err <= fma_mode_f64_bound(T), (name, err)
    pcot.pcot_destroy(h)


# Jacobi-3D 512^3 at the depths the benchmark scans (its line reports k = 4),
# 64-plane z-tiles and CTAs of up to 56 rows (as many warps as the register
# budget allows), and with the default extents.
J3D_DEPTHS = [2, 3, 4]


@pytest.fixture(scope="module")
def jacobi3d_full():
    n, T = 512, 128
    sizes = (n, n, n)
    g, modes = si.fourier_grid(sizes, 3)
    g32 = g.astype(np.float32)
    ref32 = oracle.sweep(g32, sizes, JAC3D, T, periodic=True, threads=THREADS)
    return n, T, g, g32, modes, ref32


@pytest.mark.parametrize("tile", [(64, 56, 0), (64, 0, 0)])
@pytest.mark.parametrize("k", J3D_DEPTHS)
def test_jacobi3d_512_fp32(jacobi3d_full, k, tile):
    """Jacobi-3D 7-point, 512^3 periodic, T = 128, 8 seeded Fourier modes, at
    the single-level depths the benchmark scans."""
    n, T, g, g32, modes, ref32 = jacobi3d_full
    sizes = (n, n, n)
    h = pcot.pcot_create(3, 1, JAC3D, pcot.PCOT_PERIODIC)
    got = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, pcot.PCOT_SLT, pcot.tile_params(tile=tile, time_depth=k))
    pcot.pcot_destroy(h)
    assert_f32_close(got, ref32, periodic=True, pointwise_tol=F32_POINTWISE_TOL_SIGNED, what=(k, tile))


def test_jacobi3d_512_closed_form(jacobi3d_full):
    """The FP64 oracle and the FP32 result at depth 4 against the closed-form
    decay of the Fourier modes (exact arithmetic), sampled."""
    n, T, g, g32, (amps, ks, phases), ref32 = jacobi3d_full
    sizes = (n, n, n)
    h = pcot.pcot_create(3, 1, JAC3D, pcot.PCOT_PERIODIC)
    got = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, pcot.PCOT_SLT, pcot.tile_params(tile=(64, 56, 0), time_depth=4))
    pcot.pcot_destroy(h)
    rng = np.random.default_rng(3)
    pts = rng.integers(0, n, size=(2000, 3))
    exp = np.zeros(len(pts))
    for m in range(len(amps)):
        lam = 0.4 + 2 * 0.1 * sum(math.cos(2 * math.pi * ks[m, a] / n) for a in range(3))
        arg = phases[m] + sum(2 * math.pi * ks[m, a] * pts[:, a] / n for a in range(3))
        exp += amps[m] * lam ** T * np.cos(arg)
    ref64 = oracle.sweep(g, sizes, JAC3D, T, periodic=True, threads=THREADS)
    assert np.max(np.abs(ref64[pts[:, 0], pts[:, 1], pts[:, 2]] - exp)) <= 1e-11 * float(np.sum(amps))
    samp = got[pts[:, 0], pts[:, 1], pts[:, 2]]
    assert np.max(np.abs(samp - exp)) <= 1e-5 * float(np.max(np.abs(ref64)))


@pytest.fixture(scope="module")
def batch_full():
    """The 256-grid batch (sides log-uniform in [256, 2048], T in [64, 1024])
    and the oracle's results for its two smallest and two largest problems."""
    probs = si.batched_problem_set(seed=4, count=256)
    inits = [si.uniform_grid((side, side), seed, dtype=np.float32) for side, _, seed in probs]
    order = np.argsort([s * s * T for s, T, _ in probs])
    check = [int(order[0]), int(order[1]), int(order[-2]), int(order[-1])]
    refs = {i: oracle.sweep(inits[i], (probs[i][0],) * 2, HEAT2D, probs[i][1], threads=THREADS) for i in check}
    return probs, inits, check, refs


def _cand_id(c):
    return f"k{c['time_depth']}-h{c['tile'][0]}"


@pytest.mark.parametrize("cand", tuner.batch_candidates(), ids=_cand_id)
def test_batched_256_every_tuner_candidate(batch_full, cand):
    """One persistent launch over all 256 grids for each tile shape the
    batch autotuner times (the benchmark reports the fastest of them); the
    smallest and largest problems are checked against the oracle."""
    probs, inits, check, refs = batch_full
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    grids, views, sizes, strides, Ts = [], [], [], [], []
    for (side, T, _), g in zip(probs, inits):
        shape = (side + 2, side + 2)
        st = _padded_strides(shape, 4)
        base = torch.empty(st[0] * shape[0], dtype=torch.float32, device="cuda")
        v = torch.as_strided(base, shape, st)
        v.copy_(torch.from_numpy(g).cuda())
        grids.append(base)
        views.append(v)
        sizes += [side, side]
        strides += st
        Ts.append(T)
    params = [pcot.tile_params(**cand)] * len(probs)
    nb = pcot.pcot_batch_workspace_bytes(h, sizes, strides, Ts, pcot.PCOT_F32, params)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    done = torch.zeros(len(probs) + 1, dtype=torch.int64, device="cuda")
    pcot.pcot_run_batched(h, grids, sizes, strides, Ts, pcot.PCOT_F32, params, ws, nb, done)
    d = done.cpu().numpy()
    assert np.all(d[1:] >= d[0]) and d[0] > 0
    for i in check:
        side = probs[i][0]
        assert_f32_close(views[i].cpu().numpy(), refs[i], (side, side), what=(i, side, probs[i][1]))
    pcot.pcot_destroy(h)
