"""Parity of the CUDA path with the CPU oracle, through the C ABI.

FP64 exact mode must be bitwise equal to the oracle for every schedule (the
schedules only reorder legal computations, Sec. 3.1 / Sec. 4.2).  FP32 must
stay within max-relative error 1e-5 of the oracle run on the widened FP32
inputs, normwise (max|u - ref| / max|ref|) and, for positive fields, cell by
cell (|u - ref| / max(|ref|, 1e-3 max|ref|)).  The FP64 FMA mode stays within
the rounding bound of both sides' operation counts.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from tests.gpu_util import (COEFFS, F32_POINTWISE_TOL_SIGNED, HEAT2D, JAC1D, JAC3D,  # noqa: E402
                            assert_f32_close, fma_mode_f64_bound, padded_strides, run_gpu)

pytestmark = pytest.mark.gpu

SCHEDS = [pcot.PCOT_SWEEP, pcot.PCOT_SLT, pcot.PCOT_COT]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()
    oracle.build()


def _handle(dims, periodic=False, coeffs=None):
    return pcot.pcot_create(dims, 1, COEFFS[dims] if coeffs is None else coeffs,
                            pcot.PCOT_PERIODIC if periodic else pcot.PCOT_DIRICHLET)


# ---------------------------------------------------------------- 1-D ----

@pytest.mark.parametrize("n", [1, 2, 5, 37, 100, 1000])
@pytest.mark.parametrize("T", [0, 1, 2, 3, 7, 16, 45])
@pytest.mark.parametrize("sched", SCHEDS)
def test_jacobi1d_exact(n, T, sched):
    h = _handle(1)
    g = si.uniform_grid((n,), 1, ring="random")
    ref = oracle.sweep(g, (n,), JAC1D, T)
    for params in (None, pcot.tile_params(tile=(7,), time_depth=3, cot_threshold=(2, 2))):
        got = run_gpu(h, g, (n,), T, pcot.PCOT_F64_EXACT, sched, params)
        assert np.array_equal(got, ref), (n, T, sched)
    pcot.pcot_destroy(h)


def test_jacobi1d_periodic_exact():
    h = _handle(1, periodic=True)
    g = si.uniform_grid((301,), 3, periodic=True)
    for sched in (pcot.PCOT_SWEEP, pcot.PCOT_SLT):
        got = run_gpu(h, g, (301,), 57, pcot.PCOT_F64_EXACT, sched)
        assert np.array_equal(got, oracle.sweep(g, (301,), JAC1D, 57, periodic=True))
    pcot.pcot_destroy(h)


# ---------------------------------------------------------------- 2-D ----

SIZES2 = [(1, 1), (3, 5), (33, 130), (130, 333), (257, 1000)]


@pytest.mark.parametrize("sizes", SIZES2)
@pytest.mark.parametrize("sched", SCHEDS)
def test_heat2d_exact(sizes, sched):
    h = _handle(2)
    g = si.uniform_grid(sizes, 2)
    for T in (1, 4, 11):
        ref = oracle.sweep(g, sizes, HEAT2D, T)
        got = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, sched)
        assert np.array_equal(got, ref), (sizes, T, sched)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("sched", [pcot.PCOT_SLT, pcot.PCOT_COT])
def test_heat2d_exact_depths_and_tiles(k, sched):
    """Every compiled depth plus one that falls to the generic kernel (5),
    ragged tiles in both axes, several recursion thresholds."""
    h = _handle(2, coeffs=si.random_coefficients(2, 1, 40 + k))
    c = si.random_coefficients(2, 1, 40 + k)
    sizes = (97, 301)
    g = si.uniform_grid(sizes, 5, ring="random")
    T = 3 * k + 5
    ref = oracle.sweep(g, sizes, c, T)
    for tile, th in (((8, 0), (1, 1, 1)), ((13, 130), (2, 4, 1)), ((32, 500), (4, 2, 2))):
        p = pcot.tile_params(tile=tile, time_depth=k, cot_threshold=th)
        got = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, sched, p)
        assert np.array_equal(got, ref), (k, tile, th)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("k", [1, 2, 4, 6, 8])
def test_heat2d_f32_within_tolerance(sched, k):
    h = _handle(2)
    sizes = (190, 517)
    g32 = si.uniform_grid(sizes, 2, dtype=np.float32)
    T = 40
    ref = oracle.sweep(g32, sizes, HEAT2D, T)
    p = pcot.tile_params(tile=(24, 0), time_depth=k, cot_threshold=(2, 2, 2))
    got = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, sched, p)
    assert_f32_close(got, ref, sizes, what=(sched, k))
    assert np.array_equal(got[0], g32[0]) and np.array_equal(got[:, -1], g32[:, -1])  # ring untouched
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("sched", [pcot.PCOT_SLT, pcot.PCOT_COT])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
def test_heat2d_f32_packed_equals_scalar(sched, k):
    """Rows padded to 128 bytes take the TMA-fed tile, whose interior warps
    update two cells per packed f32x2 instruction; unpadded rows take the
    plain-load tile with scalar FMAs.  Both apply the same rounded operations
    in the same order, so the FP32 results agree bitwise (and with the oracle
    within the FP32 tolerance)."""
    h = _handle(2)
    sizes = (190, 517)
    g32 = si.uniform_grid(sizes, 12, dtype=np.float32)
    T = 41
    p = pcot.tile_params(tile=(24, 0), time_depth=k, cot_threshold=(2, 2, 2))
    scalar = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, sched, p)
    packed = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, sched, p, strides=padded_strides(g32.shape, 4, 128))
    assert np.array_equal(packed, scalar)
    ref = oracle.sweep(g32, sizes, HEAT2D, T)
    assert_f32_close(packed, ref, sizes, what=(sched, k))
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("dims,sizes,periodic", [(1, (1000,), False), (2, (190, 517), False),
                                                 (2, (64, 256), True), (3, (20, 33, 70), False),
                                                 (3, (24, 16, 64), True)])
@pytest.mark.parametrize("dtype", [pcot.PCOT_F32, pcot.PCOT_F64])
def test_fma_modes_schedules_agree_bitwise(dims, sizes, periodic, dtype):
    """In the FMA modes every kernel evaluates a point with the same rounded
    operations in the same order, so the sweep, the single-level and the
    recursive schedules (and the packed FP32 tile) give identical bits."""
    h = _handle(dims, periodic=periodic)
    g = si.uniform_grid(sizes, 21, periodic=periodic, dtype=np.float32 if dtype == pcot.PCOT_F32 else np.float64)
    T = 23
    tile = {1: (32,), 2: (24, 0), 3: (8, 0, 0)}[dims]
    ref = run_gpu(h, g, sizes, T, dtype, pcot.PCOT_SWEEP)
    runs = [(pcot.PCOT_SLT, k) for k in ((1, 2, 3, 4) if dims > 1 else (4, 16))]
    if not periodic:
        runs += [(pcot.PCOT_COT, k) for k in ((2, 4) if dims > 1 else (8,))]
    elem = 4 if dtype == pcot.PCOT_F32 else 8
    for sched, k in runs:
        p = pcot.tile_params(tile=tile, time_depth=k, cot_threshold=(2, 2, 2, 2)[:dims + 1])
        got = run_gpu(h, g, sizes, T, dtype, sched, p)
        assert np.array_equal(got, ref), (sched, k)
        if dims == 2:
            got = run_gpu(h, g, sizes, T, dtype, sched, p, strides=padded_strides(g.shape, elem, 128))
            assert np.array_equal(got, ref), (sched, k, "padded")
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("dims,sizes", [(1, (1000,)), (2, (190, 517)), (3, (20, 33, 70))])
def test_fma_mode_f64_against_oracle(dims, sizes):
    """PCOT_F64 (FMA, the axis-0 +1 neighbour last) against the oracle's
    separately rounded products and sums: both are within the rounding
    bound of five roundings per term and step of the exact result."""
    h = _handle(dims)
    g = si.uniform_grid(sizes, 31, ring="random")
    T = 37
    ref = oracle.sweep(g, sizes, COEFFS[dims], T)
    tile = {1: (32,), 2: (24, 0), 3: (8, 0, 0)}[dims]
    bound = fma_mode_f64_bound(T, terms=2 * dims + 1)
    for sched, k in ((pcot.PCOT_SWEEP, 1), (pcot.PCOT_SLT, 2), (pcot.PCOT_SLT, 4 if dims > 1 else 16),
                     (pcot.PCOT_COT, 2 if dims > 1 else 8)):
        p = pcot.tile_params(tile=tile, time_depth=k, cot_threshold=(2, 2, 2, 2)[:dims + 1])
        got = run_gpu(h, g, sizes, T, pcot.PCOT_F64, sched, p)
        err = oracle.pointwise_rel_error(oracle.interior(got, sizes), oracle.interior(ref, sizes), floor=0.0)
        assert err <= bound, (sched, k, err, bound)
        assert not np.array_equal(got, ref)   # the FMA mode does round differently
    pcot.pcot_destroy(h)


def test_heat2d_periodic():
    h = _handle(2, periodic=True)
    sizes = (64, 256)
    g = si.uniform_grid(sizes, 9, periodic=True)
    ref = oracle.sweep(g, sizes, HEAT2D, 13, periodic=True)
    for sched in (pcot.PCOT_SWEEP, pcot.PCOT_SLT):
        for k in (1, 3, 4):
            got = run_gpu(h, g, sizes, 13, pcot.PCOT_F64_EXACT, sched, pcot.tile_params(tile=(16, 0), time_depth=k))
            assert np.array_equal(got, ref), (sched, k)
    pcot.pcot_destroy(h)


def test_heat2d_strided_layout_equals_contiguous():
    h = _handle(2)
    sizes = (70, 250)
    g = si.uniform_grid(sizes, 4)
    ref = oracle.sweep(g, sizes, HEAT2D, 9)
    shape = g.shape
    for sched in SCHEDS:
        st = padded_strides(shape, 8, 64)
        got = run_gpu(h, g, sizes, 9, pcot.PCOT_F64_EXACT, sched, strides=st)
        assert np.array_equal(got, ref)
    pcot.pcot_destroy(h)


def test_checkpoint_resume_bitwise():
    """The state after t steps is the grid: run(T1); run(T2) == run(T1 + T2)."""
    h = _handle(2)
    sizes = (50, 200)
    g = si.uniform_grid(sizes, 6)
    a = run_gpu(h, g, sizes, 7, pcot.PCOT_F64_EXACT, pcot.PCOT_COT)
    a = run_gpu(h, a, sizes, 10, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT)
    b = run_gpu(h, g, sizes, 17, pcot.PCOT_F64_EXACT, pcot.PCOT_COT)
    assert np.array_equal(a, b)
    pcot.pcot_destroy(h)


# ---------------------------------------------------------------- 3-D ----

@pytest.mark.parametrize("sizes", [(3, 4, 5), (20, 33, 70), (40, 21, 130)])
@pytest.mark.parametrize("sched", SCHEDS)
def test_jacobi3d_exact_dirichlet(sizes, sched):
    h = _handle(3)
    g = si.uniform_grid(sizes, 8, ring="random")
    for T, k in ((1, 1), (5, 2), (6, 3)):
        ref = oracle.sweep(g, sizes, JAC3D, T)
        got = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, sched, pcot.tile_params(tile=(8, 0, 0), time_depth=k))
        assert np.array_equal(got, ref), (sizes, T, k, sched)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_jacobi3d_periodic_f32_and_exact(k):
    h = _handle(3, periodic=True)
    sizes = (24, 40, 96)
    g, _ = si.fourier_grid(sizes, 3)
    T = 2 * k + 3
    ref = oracle.sweep(g, sizes, JAC3D, T, periodic=True)
    p = pcot.tile_params(tile=(8, 0, 0), time_depth=k)
    got32 = run_gpu(h, g.astype(np.float32), sizes, T, pcot.PCOT_F32, pcot.PCOT_SLT, p)
    ref32 = oracle.sweep(g.astype(np.float32), sizes, JAC3D, T, periodic=True)
    assert_f32_close(got32, ref32, periodic=True, pointwise_tol=F32_POINTWISE_TOL_SIGNED, what=k)
    if k <= 2:
        got = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT, p)
        assert np.array_equal(got, ref)
    got = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SWEEP)
    assert np.array_equal(got, ref)
    pcot.pcot_destroy(h)


# ------------------------------------------------------- status / sums ----

def test_timeout_is_reported_not_hung():
    h = _handle(2)
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    pcot.pcot_test_wait_timeout(h, ws.data_ptr(), 200)
    assert pcot.pcot_check(h) == pcot.PCOT_ERR_TIMEOUT
    assert pcot.pcot_check(h) == pcot.PCOT_OK   # cleared, context still usable
    g = si.uniform_grid((10, 10), 1)
    assert np.array_equal(run_gpu(h, g, (10, 10), 3, pcot.PCOT_F64_EXACT, pcot.PCOT_COT),
                          oracle.sweep(g, (10, 10), HEAT2D, 3))
    pcot.pcot_destroy(h)


def test_misaligned_workspace_rejected():
    h = _handle(2)
    g = torch.zeros((12, 12), dtype=torch.float64, device="cuda")
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_run(h, g.data_ptr(), ws.data_ptr() + 8, 4000, (10, 10), None, 2, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT)
    assert e.value.status == pcot.PCOT_ERR_ALIGNMENT
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("dims,sizes,periodic", [(1, (1000,), False), (2, (300, 257), False),
                                                 (3, (30, 40, 50), True)])
def test_grid_sum(dims, sizes, periodic):
    h = _handle(dims, periodic)
    g = si.uniform_grid(sizes, 11, periodic=periodic, ring="random")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dev = torch.from_numpy(g).cuda()
    pcot.pcot_grid_sum(h, dev.data_ptr(), sizes, None, pcot.PCOT_F64, out.data_ptr())
    s = float(out.item())
    exact = oracle.grid_sum(g, sizes, periodic=periodic)
    assert abs(s - exact) <= 1e-12 * abs(exact)
    dev32 = torch.from_numpy(g.astype(np.float32)).cuda()
    pcot.pcot_grid_sum(h, dev32.data_ptr(), sizes, None, pcot.PCOT_F32, out.data_ptr())
    exact32 = oracle.grid_sum(g.astype(np.float32), sizes, periodic=periodic)
    assert abs(float(out.item()) - exact32) <= 1e-12 * abs(exact32)
    pcot.pcot_destroy(h)


def test_run_host_end_to_end():
    h = _handle(2)
    sizes = (64, 300)
    g = si.uniform_grid(sizes, 12)
    host = torch.from_numpy(g.copy()).pin_memory()
    dev = torch.empty_like(host, device="cuda")
    nb = pcot.pcot_workspace_bytes(h, sizes, None, 10, pcot.PCOT_F64_EXACT, pcot.PCOT_COT)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    pcot.pcot_run_host(h, host.data_ptr(), dev.data_ptr(), ws.data_ptr(), nb, sizes, None, 10,
                       pcot.PCOT_F64_EXACT, pcot.PCOT_COT)
    assert np.array_equal(host.numpy(), oracle.sweep(g, sizes, HEAT2D, 10))
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("sched,T", [(pcot.PCOT_SWEEP, 5), (pcot.PCOT_SLT, 7)])
def test_strided_padding_untouched(dims, sched, T):
    """A padded grid inside a sentinel-filled buffer, an odd number of buffer
    swaps (so the result is copied back from the workspace): the stored cells
    match the oracle and no other byte of the buffer changes, even when the
    workspace held other data."""
    h = _handle(dims)
    sizes = (150, 211) if dims == 2 else (9, 14, 37)
    shape = tuple(n + 2 for n in sizes)
    st = padded_strides(shape, 8, 128)
    if dims == 3:
        st[0] += 8                                      # a gap between planes too
    span = sum((shape[a] - 1) * st[a] for a in range(dims)) + 1
    base = torch.full((span + 2048,), -777.0, dtype=torch.float64, device="cuda")
    view = torch.as_strided(base, shape, st, 512)
    g = si.uniform_grid(sizes, 19, ring="random")
    view.copy_(torch.from_numpy(g).cuda())
    p = pcot.tile_params(tile=(8, 0, 0)[:dims], time_depth=1)
    nb = pcot.pcot_workspace_bytes(h, sizes, st, T, pcot.PCOT_F64_EXACT, sched, p)
    ws = torch.full((nb,), 0x5A, dtype=torch.uint8, device="cuda")   # stale contents
    pcot.pcot_run(h, view.data_ptr(), ws.data_ptr(), nb, sizes, st, T, pcot.PCOT_F64_EXACT, sched, p)
    assert pcot.pcot_check(h) == pcot.PCOT_OK
    assert np.array_equal(view.cpu().numpy(), oracle.sweep(g, sizes, COEFFS[dims], T))
    mask = torch.ones_like(base, dtype=torch.bool)
    torch.as_strided(mask, shape, st, 512).fill_(False)
    assert np.all(base[mask].cpu().numpy() == -777.0)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("k", [4, 6, 8])
@pytest.mark.parametrize("sizes", [(33, 130), (190, 517), (257, 1000)])
def test_heat2d_f32_recursive_single_span_tiles(k, sizes):
    """Recursive order with one-span tiles on rows padded to 128 bytes (the
    persistent kernel whose stages are split over several warps): bitwise
    equal to the sweep (every FMA-mode kernel rounds the same way), within the
    FP32 tolerance of the oracle, with asymmetric coefficients and a random
    ring so that the Dirichlet pass-through and every operand's orientation
    are exercised."""
    c = si.random_coefficients(2, 1, 70 + k) * 0.2 + np.array([0.2, 0.2, 0.2, 0.2, 0.2])
    h = _handle(2, coeffs=c)
    g32 = si.uniform_grid(sizes, 23 + k, ring="random", dtype=np.float32)
    T = 2 * k + 7
    st = padded_strides(g32.shape, 4, 128)
    ref = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, pcot.PCOT_SWEEP, strides=st)
    for H in (16, 24, 80):
        p = pcot.tile_params(tile=(H, 112), time_depth=k, cot_threshold=(2, 3, 2))
        got = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, pcot.PCOT_COT, p, strides=st)
        assert np.array_equal(got, ref), (k, sizes, H)
    assert oracle.max_rel_error(oracle.interior(got, sizes), oracle.interior(oracle.sweep(g32, sizes, c, T), sizes)) \
        <= 1e-5
    pcot.pcot_destroy(h)
