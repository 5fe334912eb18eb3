"""FDTD-2D on the GPU against the oracle's loop nest: FP64 bitwise for every
schedule (ragged tiles, tail blocks, padded rows), FP32 within tolerance."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")

pytestmark = pytest.mark.gpu
F32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def handle():
    h = pcot.pcot_create(2, 1, [0.5, 0.125, 0.125, 0.125, 0.125], pcot.PCOT_DIRICHLET)
    yield h
    pcot.pcot_destroy(h)


def fields(nx, ny, T, seed, dtype=np.float64):
    u = si.uniform01(seed, 3 * nx * ny + T)
    ex, ey, hz = (u[k * nx * ny:(k + 1) * nx * ny].reshape(nx, ny).astype(dtype) for k in range(3))
    return ex, ey, hz, u[3 * nx * ny:].astype(dtype)


def run_fd(h, ex, ey, hz, fict, T, dtype, sched, params=None, pitch=None):
    nx, ny = ex.shape
    tdt = torch.float32 if dtype == pcot.PCOT_F32 else torch.float64
    P = pitch or ny
    dev = []
    for a in (ex, ey, hz):
        base = torch.zeros(nx * P + 16, dtype=tdt, device="cuda")
        torch.as_strided(base, (nx, ny), (P, 1)).copy_(torch.from_numpy(np.ascontiguousarray(a)).to(tdt).cuda())
        dev.append(base)
    f = torch.from_numpy(np.ascontiguousarray(fict)).to(tdt).cuda()
    st = (P, 1) if pitch else None
    nb = pcot.pcot_fdtd2d_workspace_bytes((nx, ny), st, T, dtype, sched, params)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) // 256 * 256
    pcot.pcot_fdtd2d_run(h, dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr(), f.data_ptr(), wp, nb, (nx, ny),
                         st, T, dtype, sched, params)
    s = pcot.pcot_check(h)
    if s != pcot.PCOT_OK:
        raise pcot.PcotError(s, "fdtd2d")
    return [torch.as_strided(d, (nx, ny), (P, 1)).cpu().numpy() for d in dev]


SCHEDS = [(pcot.PCOT_SWEEP, None),
          (pcot.PCOT_SLT, None),
          (pcot.PCOT_SLT, dict(tile=(5, 7), time_depth=3)),
          (pcot.PCOT_COT, dict(tile=(8, 8), time_depth=4, cot_threshold=(1, 1, 1))),
          (pcot.PCOT_COT, dict(tile=(16, 24), time_depth=5, cot_threshold=(2, 4, 4))),
          (pcot.PCOT_COT, None)]


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (17, 23), (70, 131)])
@pytest.mark.parametrize("T", [1, 3, 11])
@pytest.mark.parametrize("k", range(len(SCHEDS)))
def test_fdtd2d_fp64_bitwise(handle, shape, T, k):
    sched, p = SCHEDS[k]
    ex, ey, hz, fict = fields(*shape, T, 41)
    ref = oracle.fdtd2d(ex, ey, hz, fict, T)
    params = pcot.tile_params(**p) if p else None
    for dtype in (pcot.PCOT_F64_EXACT, pcot.PCOT_F64):
        got = run_fd(handle, ex, ey, hz, fict, T, dtype, sched, params)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), (dtype, sched, p)


@pytest.mark.parametrize("k", range(len(SCHEDS)))
def test_fdtd2d_fp32_within_tolerance(handle, k):
    sched, p = SCHEDS[k]
    T = 24
    ex, ey, hz, fict = fields(90, 150, T, 42, np.float32)
    ref = oracle.fdtd2d(*(a.astype(np.float64) for a in (ex, ey, hz)), fict.astype(np.float64), T)
    got = run_fd(handle, ex, ey, hz, fict, T, pcot.PCOT_F32, sched, pcot.tile_params(**p) if p else None)
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= F32_TOL


def test_fdtd2d_padded_rows_and_checkpoint(handle):
    ex, ey, hz, fict = fields(40, 57, 13, 43)
    ref = oracle.fdtd2d(ex, ey, hz, fict, 13)
    p = pcot.tile_params(tile=(12, 16), time_depth=4, cot_threshold=(1, 2, 2))
    got = run_fd(handle, ex, ey, hz, fict, 13, pcot.PCOT_F64_EXACT, pcot.PCOT_COT, p, pitch=64)
    assert all(np.array_equal(a, b) for a, b in zip(got, ref))
    mid = run_fd(handle, ex, ey, hz, fict[:5], 5, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT, p)
    got = run_fd(handle, *mid, fict[5:], 8, pcot.PCOT_F64_EXACT, pcot.PCOT_COT, p)
    assert all(np.array_equal(a, b) for a, b in zip(got, ref))


@pytest.mark.slow
def test_fdtd2d_paper_size(handle):
    """The paper's FDTD-2D size (2000 x 2000, T = 500; Table 2), FP64, against
    the full oracle run."""
    T = 500
    ex, ey, hz, fict = fields(2000, 2000, T, 44)
    ref = oracle.fdtd2d(ex, ey, hz, fict, T)
    got = run_fd(handle, ex, ey, hz, fict, T, pcot.PCOT_F64, pcot.PCOT_COT)
    assert all(np.array_equal(a, b) for a, b in zip(got, ref))
