"""The allocation-free entry point (pcot_run_noalloc) against pcot_run.

Callers that may not allocate device memory when they advance a grid (code
inside a CUDA-graph capture, hosts that reserve all device memory up front)
use the library's fixed device array as the grid's twin.  This file is
collected last so that a failure here cannot hide any other test's result;
it passes alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from tests.gpu_util import HEAT2D, JAC3D, run_gpu  # noqa: E402

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()


def _same(a, b, dtype, sizes):
    if dtype == pcot.PCOT_F64_EXACT:
        return np.array_equal(a, b)
    return oracle.max_rel_error(oracle.interior(a, sizes), oracle.interior(b, sizes)) <= F32_TOL


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
        got = dev.cpu().numpy()
        assert _same(got, ref, dtype, sizes), (call, dtype, sched)
    pcot.pcot_destroy(h)


def test_noalloc_periodic_3d_two_calls():
    h = pcot.pcot_create(3, 1, JAC3D, pcot.PCOT_PERIODIC)
    sizes, T = (24, 40, 96), 7
    g0, _ = si.fourier_grid(sizes, 3)
    ref = g0
    dev = torch.from_numpy(g0.copy()).cuda()
    p = pcot.tile_params(tile=(8, 0, 0), time_depth=2)
    for call in range(2):
        ref = run_gpu(h, ref, sizes, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT, p)
        pcot.pcot_run_noalloc(h, dev, sizes, None, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT, p)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), ref), call
    pcot.pcot_destroy(h)


def test_noalloc_rejects_grids_beyond_the_array():
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    side = int((pcot.NOALLOC_MAX_BYTES // 4) ** 0.5) + 8      # span just above the limit in fp32
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_run_noalloc(h, 1 << 20, (side, side), None, 3, pcot.PCOT_F32, pcot.PCOT_SLT)
    assert e.value.status == pcot.PCOT_ERR_OOM
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_run_noalloc(h, 1 << 20, (8, 8), None, 3, pcot.PCOT_F32, pcot.PCOT_COT)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    pcot.pcot_destroy(h)
