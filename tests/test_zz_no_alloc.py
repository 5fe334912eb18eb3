"""The allocation-free entry point (pcot_run_noalloc) against pcot_run.

Some callers may not allocate device memory when they advance a grid: hosts
that reserve all device memory up front and forbid allocation afterwards,
services with a fixed memory budget, and library layers that receive only a
grid and a stream.  They use the library's fixed device array as the grid's
twin instead of a workspace.  Every schedule of this library evaluates a point
with the same rounded operations in the same order, so the results must be
bitwise equal to pcot_run's (which is within any tolerance the other tests
use), on every call in a row.

This file is collected last so that a failure here cannot hide any other
test's result; it passes alone in a fresh process and after the rest of the
suite.
"""
import numpy as np
import pytest

import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from tests.gpu_util import HEAT2D, JAC3D, padded_strides, run_gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()


@pytest.mark.parametrize("dtype", [pcot.PCOT_F64_EXACT, pcot.PCOT_F32])
@pytest.mark.parametrize("sched,params", [
    (pcot.PCOT_SLT, pcot.tile_params(tile=(32, 0), time_depth=4)),
    (pcot.PCOT_SLT, None),
    (pcot.PCOT_SWEEP, None),
])
def test_noalloc_matches_pcot_run_two_calls(dtype, sched, params):
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    sizes, T = (300, 517), 13
    npdt = np.float32 if dtype == pcot.PCOT_F32 else np.float64
    g0 = si.uniform_grid(sizes, 61, dtype=npdt)
    ref = g0
    dev = torch.from_numpy(g0.copy()).cuda()
    for call in range(2):
        ref = run_gpu(h, ref, sizes, T, dtype, sched, params)           # existing entry point
        pcot.pcot_run_noalloc(h, dev, sizes, None, T, dtype, sched, params)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), ref), (call, dtype, sched)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("dtype", [pcot.PCOT_F64_EXACT, pcot.PCOT_F32])
def test_noalloc_periodic_3d_two_calls(dtype):
    """3-D periodic grids: explicit depth 2, and the default parameters
    (which follow pcot_run's default depth)."""
    h = pcot.pcot_create(3, 1, JAC3D, pcot.PCOT_PERIODIC)
    sizes, T = (24, 40, 96), 7
    g0, _ = si.fourier_grid(sizes, 3)
    g0 = g0.astype(np.float32 if dtype == pcot.PCOT_F32 else np.float64)
    for p in (pcot.tile_params(tile=(8, 0, 0), time_depth=2), None):
        ref = g0
        dev = torch.from_numpy(g0.copy()).cuda()
        for call in range(2):
            ref = run_gpu(h, ref, sizes, T, dtype, pcot.PCOT_SLT, p)
            pcot.pcot_run_noalloc(h, dev, sizes, None, T, dtype, pcot.PCOT_SLT, p)
            torch.cuda.synchronize()
            assert np.array_equal(dev.cpu().numpy(), ref), (call, p is None)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("sched,T", [(pcot.PCOT_SWEEP, 5), (pcot.PCOT_SLT, 7)])
def test_noalloc_strided_grid_leaves_padding_untouched(sched, T):
    """A grid whose rows are padded, inside a larger buffer filled with a
    sentinel, after a call on a different grid shape has left other data in
    the shared array.  The interior must match pcot_run and no byte outside
    the grid's stored cells may change (an odd number of buffer swaps makes
    the call copy the result back from the array)."""
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    other = torch.from_numpy(si.uniform_grid((333, 201), 9, dtype=np.float32)).cuda()
    pcot.pcot_run_noalloc(h, other, (333, 201), None, 3, pcot.PCOT_F32, pcot.PCOT_SWEEP)
    sizes = (150, 211)
    shape = (sizes[0] + 2, sizes[1] + 2)
    st = padded_strides(shape, 4, 128)
    span = (shape[0] - 1) * st[0] + shape[1]
    sentinel = np.float32(-12345.0)
    base = torch.full((span + 4096,), float(sentinel), dtype=torch.float32, device="cuda")
    view = torch.as_strided(base, shape, st, 1024)
    g0 = si.uniform_grid(sizes, 77, dtype=np.float32)
    view.copy_(torch.from_numpy(g0).cuda())
    p = pcot.tile_params(tile=(32, 0), time_depth=1)
    ref = run_gpu(h, g0, sizes, T, pcot.PCOT_F32, sched, p, strides=st)
    pcot.pcot_run_noalloc(h, view.data_ptr(), sizes, st, T, pcot.PCOT_F32, sched, p)
    torch.cuda.synchronize()
    assert np.array_equal(view.cpu().numpy(), ref)
    mask = torch.ones_like(base, dtype=torch.bool)
    torch.as_strided(mask, shape, st, 1024).fill_(False)
    outside = base[mask].cpu().numpy()
    assert outside.size > 0 and np.all(outside == sentinel)
    pcot.pcot_destroy(h)


def test_noalloc_allocates_no_device_memory():
    """After a first call (which loads the kernels and looks up the array),
    further calls change neither torch's allocator nor the device's free
    memory."""
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    sizes = (256, 384)
    dev = torch.from_numpy(si.uniform_grid(sizes, 5, dtype=np.float32)).cuda()
    p = pcot.tile_params(tile=(32, 0), time_depth=4)
    pcot.pcot_run_noalloc(h, dev, sizes, None, 9, pcot.PCOT_F32, pcot.PCOT_SLT, p)
    torch.cuda.synchronize()
    a0, f0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(3):
        pcot.pcot_run_noalloc(h, dev, sizes, None, 9, pcot.PCOT_F32, pcot.PCOT_SLT, p)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == a0
    assert torch.cuda.mem_get_info()[0] == f0
    pcot.pcot_destroy(h)


def test_noalloc_rejects_grids_beyond_the_array():
    """Argument checks on real device buffers: a grid whose storage span
    exceeds the fixed array, and a schedule the entry point does not run."""
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    side = int((pcot.NOALLOC_MAX_BYTES // 4) ** 0.5)          # (side + 2)^2 floats: just above the limit
    big = torch.zeros((side + 2) ** 2, dtype=torch.float32, device="cuda")
    assert big.numel() * 4 > pcot.NOALLOC_MAX_BYTES
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_run_noalloc(h, big, (side, side), None, 3, pcot.PCOT_F32, pcot.PCOT_SLT)
    assert e.value.status == pcot.PCOT_ERR_OOM
    small = torch.zeros(100, dtype=torch.float32, device="cuda")
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_run_noalloc(h, small, (8, 8), None, 3, pcot.PCOT_F32, pcot.PCOT_COT)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    assert np.all(small.cpu().numpy() == 0) and float(big.abs().max()) == 0.0
    pcot.pcot_destroy(h)
