"""Batched persistent launch: many uneven grids in one kernel, each result
equal to the oracle's (bitwise in FP64 exact mode), per-grid completion
stamps recorded, graph replay advancing every grid again."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from tests.gpu_util import HEAT2D, assert_f32_close, padded_strides  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()


def _batch(sides, Ts, dtype, depth, padded, seed=30):
    tdt = torch.float32 if dtype == pcot.PCOT_F32 else torch.float64
    npdt = np.float32 if dtype == pcot.PCOT_F32 else np.float64
    elem = 4 if dtype == pcot.PCOT_F32 else 8
    grids, views, inits, sizes, strides = [], [], [], [], []
    for i, (n0, n1) in enumerate(sides):
        g = si.uniform_grid((n0, n1), seed + i, dtype=npdt)
        inits.append(g)
        shape = g.shape
        if padded:
            st = padded_strides(shape, elem, 64)
            base = torch.zeros(st[0] * shape[0] + 64, dtype=tdt, device="cuda")
            v = torch.as_strided(base, shape, st)
            v.copy_(torch.from_numpy(g).cuda())
            strides += st
            grids.append(base)
            views.append(v)
        else:
            t = torch.from_numpy(g.copy()).cuda()
            strides += [shape[1], 1]
            grids.append(t)
            views.append(t)
        sizes += [n0, n1]
    return grids, views, inits, sizes, strides


@pytest.mark.parametrize("dtype,depth", [(pcot.PCOT_F64_EXACT, 1), (pcot.PCOT_F64_EXACT, 2), (pcot.PCOT_F64_EXACT, 4),
                                         (pcot.PCOT_F32, 4), (pcot.PCOT_F32, 6), (pcot.PCOT_F32, 8)])
@pytest.mark.parametrize("padded", [True, False])
def test_batched_matches_oracle(dtype, depth, padded):
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    sides = [(5, 7), (40, 300), (130, 130), (64, 900), (1, 1), (33, 257), (200, 61)]
    Ts = [3, 9, 17, 0, 5, 26, 12]
    if dtype == pcot.PCOT_F32:
        Ts = [16, 9, 24, 0, 33, 40, 18]
    grids, views, inits, sizes, strides = _batch(sides, Ts, dtype, depth, padded)
    params = [pcot.tile_params(tile=(16 + 8 * i, 0), time_depth=depth, cot_threshold=(1 + i % 3, 2, 2))
              for i in range(len(sides))]
    nb = pcot.pcot_batch_workspace_bytes(h, sizes, strides, Ts, dtype, params)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    done = torch.zeros(len(sides) + 1, dtype=torch.int64, device="cuda")
    pcot.pcot_run_batched(h, grids, sizes, strides, Ts, dtype, params, ws, nb, done)
    for i, (v, g, T) in enumerate(zip(views, inits, Ts)):
        ref = oracle.sweep(g, sides[i], HEAT2D, T)
        got = v.cpu().numpy()
        if dtype == pcot.PCOT_F64_EXACT:
            assert np.array_equal(got, ref), (i, sides[i], T)
        else:
            assert_f32_close(got, ref, sides[i], what=(i, sides[i], T))
    d = done.cpu().numpy()
    for i, T in enumerate(Ts):
        if T > 0:
            assert d[1 + i] >= d[0] > 0
    pcot.pcot_destroy(h)


def test_batch_graph_replay_advances_again():
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    sides = [(50, 200), (77, 129), (128, 64)]
    Ts = [6, 10, 14]
    grids, views, inits, sizes, strides = _batch(sides, Ts, pcot.PCOT_F64_EXACT, 2, True, seed=50)
    params = [pcot.tile_params(tile=(12, 0), time_depth=2, cot_threshold=(1, 1, 1))] * 3
    nb = pcot.pcot_batch_workspace_bytes(h, sizes, strides, Ts, pcot.PCOT_F64_EXACT, params)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    b = pcot.pcot_batch_create(h, grids, sizes, strides, Ts, pcot.PCOT_F64_EXACT, params, ws, nb)
    for _ in range(3):
        pcot.pcot_batch_launch(b)
    assert pcot.pcot_check(h) == pcot.PCOT_OK
    pcot.pcot_batch_destroy(b)
    for i, (v, g, T) in enumerate(zip(views, inits, Ts)):
        assert np.array_equal(v.cpu().numpy(), oracle.sweep(g, sides[i], HEAT2D, 3 * T))
    pcot.pcot_destroy(h)


def test_batch_config4_shape_sample():
    """A seeded sample of the 256-grid workload (sides log-uniform in
    [256, 2048], T uniform in [64, 1024]): 6 grids, FP32, tolerance 1e-5."""
    probs = si.batched_problem_set(seed=4, count=256)
    pick = [probs[i] for i in (0, 17, 42, 99, 150, 255)]
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    sides = [(p[0] // 4, p[0] // 4) for p in pick]   # quarter sides keep the oracle quick
    Ts = [p[1] // 8 for p in pick]
    grids, views, inits, sizes, strides = _batch(sides, Ts, pcot.PCOT_F32, 8, True, seed=70)
    params = [pcot.tile_params(tile=(64, 0), time_depth=8, cot_threshold=(2, 8, 8))] * len(sides)
    nb = pcot.pcot_batch_workspace_bytes(h, sizes, strides, Ts, pcot.PCOT_F32, params)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    pcot.pcot_run_batched(h, grids, sizes, strides, Ts, pcot.PCOT_F32, params, ws, nb)
    for i, (v, g, T) in enumerate(zip(views, inits, Ts)):
        ref = oracle.sweep(g, sides[i], HEAT2D, T)
        assert_f32_close(v.cpu().numpy(), ref, sides[i], what=(i, sides[i], T))
    pcot.pcot_destroy(h)
