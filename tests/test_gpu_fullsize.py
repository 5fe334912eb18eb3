"""Parity at the full workload sizes, in the launch configurations the
benchmark times.  The oracle (FP64 naive sweeps, all host cores) computes the
whole grid; FP64 exact mode must match bitwise, FP32 within 1e-5 normwise of
the oracle run on the widened FP32 inputs.  The periodic Jacobi-3D case is also
checked against the closed-form decay of its Fourier modes."""
import math
import os

import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from tests.gpu_util import HEAT2D, JAC1D, JAC3D, run_gpu  # noqa: E402

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


def test_heat2d_8192_fp32_bench_config(heat2d_full):
    n, T, g32, ref = heat2d_full
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    st = _padded_strides(g32.shape, 4)
    for sched in (pcot.PCOT_SLT, pcot.PCOT_COT):
        got = run_gpu(h, g32, (n, n), T, pcot.PCOT_F32, sched, pcot.tile_params(**BENCH_PARAMS), strides=st)
        err = oracle.max_rel_error(oracle.interior(got, (n, n)), oracle.interior(ref, (n, n)))
        assert err <= 1e-5, (sched, err)
        assert np.array_equal(got[0], g32[0]) and np.array_equal(got[-1], g32[-1])
    pcot.pcot_destroy(h)


def test_heat2d_8192_fp64_exact_bitwise(heat2d_full):
    """The same inputs widened to FP64, FP64 exact mode: bitwise equal."""
    n, T, g32, ref = heat2d_full
    g64 = g32.astype(np.float64)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    st = _padded_strides(g64.shape, 8)
    got = run_gpu(h, g64, (n, n), T, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT,
                  pcot.tile_params(tile=(128, 0), time_depth=2), strides=st)
    assert np.array_equal(got, ref)
    pcot.pcot_destroy(h)


def test_jacobi3d_512_fp32_error_and_closed_form():
    """Jacobi-3D 7-point, 512^3 periodic, T = 128, 8 seeded Fourier modes."""
    n, T = 512, 128
    sizes = (n, n, n)
    g, (amps, ks, phases) = si.fourier_grid(sizes, 3)
    g32 = g.astype(np.float32)
    h = pcot.pcot_create(3, 1, JAC3D, pcot.PCOT_PERIODIC)
    got = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, pcot.PCOT_SLT, pcot.tile_params(tile=(64, 0, 0), time_depth=2))
    pcot.pcot_destroy(h)
    ref = oracle.sweep(g32, sizes, JAC3D, T, periodic=True, threads=THREADS)
    err = oracle.max_rel_error(got, ref)
    assert err <= 1e-5, err
    # Closed form of the exact-arithmetic evolution of the FP64 modes, sampled.
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


def test_batched_256_grid_sample():
    """The 256-grid batch (sides log-uniform in [256, 2048], T in [64, 1024]):
    one persistent launch over every grid, 12 grids checked against the oracle."""
    probs = si.batched_problem_set(seed=4, count=256)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    grids, views, sizes, strides, Ts = [], [], [], [], []
    for side, T, seed in probs:
        shape = (side + 2, side + 2)
        st = _padded_strides(shape, 4)
        base = torch.empty(st[0] * shape[0], dtype=torch.float32, device="cuda")
        v = torch.as_strided(base, shape, st)
        v.copy_(torch.from_numpy(si.uniform_grid((side, side), seed, dtype=np.float32)).cuda())
        grids.append(base)
        views.append(v)
        sizes += [side, side]
        strides += st
        Ts.append(T)
    params = [pcot.tile_params(tile=(64, 0), time_depth=8, cot_threshold=(2, 8, 8))] * len(probs)
    nb = pcot.pcot_batch_workspace_bytes(h, sizes, strides, Ts, pcot.PCOT_F32, params)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    done = torch.zeros(len(probs) + 1, dtype=torch.int64, device="cuda")
    pcot.pcot_run_batched(h, grids, sizes, strides, Ts, pcot.PCOT_F32, params, ws, nb, done)
    d = done.cpu().numpy()
    assert np.all(d[1:] >= d[0]) and d[0] > 0
    order = np.argsort([s * s * T for s, T, _ in probs])
    check = list(order[:6]) + list(order[-6:])          # the smallest and the largest problems
    for i in check:
        side, T, seed = probs[i]
        g = si.uniform_grid((side, side), seed, dtype=np.float32)
        ref = oracle.sweep(g, (side, side), HEAT2D, T, threads=THREADS)
        got = views[i].cpu().numpy()
        err = oracle.max_rel_error(oracle.interior(got, (side, side)), oracle.interior(ref, (side, side)))
        assert err <= 1e-5, (i, side, T, err)
    pcot.pcot_destroy(h)
