"""Gauss-Seidel 2-D on the GPU against the oracle's plain loop nest: FP64
(exact and FMA modes evaluate the same operations) bitwise, FP32 within the
FP32 tolerance, every schedule, ragged tiles, padded rows."""
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


def run_gs(h, g, T, dtype, sched, params=None, pitch=None):
    n0, n1 = g.shape[0] - 2, g.shape[1] - 2
    tdt = torch.float32 if dtype == pcot.PCOT_F32 else torch.float64
    P = pitch or g.shape[1]
    base = torch.zeros(g.shape[0] * P + 32, dtype=tdt, device="cuda")
    view = torch.as_strided(base, g.shape, (P, 1))
    view.copy_(torch.from_numpy(g).to(tdt).cuda())
    nb = pcot.pcot_gs2d_workspace_bytes((n0, n1), T, sched, params)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) // 256 * 256
    pcot.pcot_gs2d_run(h, base.data_ptr(), wp, nb, (n0, n1), (P, 1) if pitch else None, T, dtype, sched, params)
    st = pcot.pcot_check(h)
    if st != pcot.PCOT_OK:
        raise pcot.PcotError(st, "gs2d")
    return torch.as_strided(base, g.shape, (P, 1)).cpu().numpy()


SCHEDS = [(pcot.PCOT_SWEEP, None),
          (pcot.PCOT_SLT, None),
          (pcot.PCOT_SLT, dict(tile=(8, 16), time_depth=4)),
          (pcot.PCOT_SLT, dict(tile=(5, 7), time_depth=3)),
          (pcot.PCOT_COT, dict(tile=(8, 16), time_depth=4, cot_threshold=(1, 1, 1))),
          (pcot.PCOT_COT, dict(tile=(16, 64), time_depth=8, cot_threshold=(2, 2, 2))),
          (pcot.PCOT_COT, None)]


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (37, 29), (70, 131)])
@pytest.mark.parametrize("T", [1, 2, 9])
@pytest.mark.parametrize("k", range(len(SCHEDS)))
def test_gs2d_fp64_bitwise(handle, shape, T, k):
    sched, p = SCHEDS[k]
    g = si.uniform_grid(shape, 31, ring="random")
    ref = oracle.gs2d(g, T)
    params = pcot.tile_params(**p) if p else None
    for dtype in (pcot.PCOT_F64_EXACT, pcot.PCOT_F64):
        got = run_gs(handle, g, T, dtype, sched, params)
        assert np.array_equal(got, ref), (dtype, sched, p)


@pytest.mark.parametrize("k", range(len(SCHEDS)))
def test_gs2d_fp32_within_tolerance(handle, k):
    sched, p = SCHEDS[k]
    g = si.uniform_grid((90, 150), 32, ring="random", dtype=np.float32)
    T = 20
    ref = oracle.gs2d(g.astype(np.float64), T)
    got = run_gs(handle, g, T, pcot.PCOT_F32, sched, pcot.tile_params(**p) if p else None)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= F32_TOL, err
    assert np.array_equal(got[0], g[0]) and np.array_equal(got[:, -1], g[:, -1])


def test_gs2d_padded_rows_and_checkpoint(handle):
    """A padded row stride gives the same bits; run(T1) then run(T2) equals
    run(T1 + T2)."""
    g = si.uniform_grid((60, 77), 33, ring="random")
    ref = oracle.gs2d(g, 11)
    p = pcot.tile_params(tile=(16, 32), time_depth=4, cot_threshold=(1, 2, 2))
    assert np.array_equal(run_gs(handle, g, 11, pcot.PCOT_F64_EXACT, pcot.PCOT_COT, p, pitch=96), ref)
    mid = run_gs(handle, g, 4, pcot.PCOT_F64_EXACT, pcot.PCOT_SLT, p)
    assert np.array_equal(run_gs(handle, mid, 7, pcot.PCOT_F64_EXACT, pcot.PCOT_COT, p), ref)


@pytest.mark.slow
def test_gs2d_paper_size_sampled(handle):
    """The paper's GS-2D size (2000 x 2000 interior, T = 500; Table 2), FP64,
    against the full oracle run."""
    g = si.uniform_grid((2000, 2000), 34, ring="random")
    T = 500
    ref = oracle.gs2d(g, T)
    got = run_gs(handle, g, T, pcot.PCOT_F64, pcot.PCOT_SLT)
    assert np.array_equal(got, ref)
