"""PCOT_SKEW -- parallelogram tiles of the skewed space (t, t+i, t+j) run by
the persistent executor -- on the GPU through the C ABI, against the
oracle's loop nest: FP64 exact mode bit for bit, the FP64 FMA mode within
its rounding bound, FP32 within the FP32 tolerance; ragged sizes, odd and
even T, wavefront and recursive orders, rows padded inside a sentinel-filled
buffer with a stale workspace."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from tests.gpu_util import HEAT2D, assert_f32_close, fma_mode_f64_bound, padded_strides, run_gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()
    oracle.build()


# (sizes, T, (kt, ha, wc) or None for the defaults, recursive leaf or None)
CASES = [
    ((1, 1), 1, (2, 2, 2), None),
    ((1, 1), 2, None, None),
    ((37, 53), 7, (3, 4, 6), None),
    ((37, 53), 7, (3, 4, 6), (2, 2, 2)),
    ((100, 130), 20, None, None),
    ((257, 300), 33, None, (2, 4, 4)),
    ((64, 2000), 16, (5, 8, 128), None),
    ((1000, 7), 40, (8, 16, 32), None),
    ((300, 300), 64, (16, 64, 64), (1, 2, 2)),
    ((129, 513), 9, (1, 2, 2), None),
]


def _params(tile, theta):
    if tile is None and theta is None:
        return None
    tile = tile or (0, 0, 0)
    return pcot.tile_params(tile=(tile[1], tile[2]), time_depth=tile[0], cot_threshold=theta or (0, 0, 0))


def _coeffs(seed):
    return si.random_coefficients(2, 1, seed) * 0.2 + np.array([0.2, 0.2, 0.2, 0.2, 0.2])


@pytest.mark.parametrize("sizes,T,tile,theta", CASES)
def test_fp64_exact_bitwise(sizes, T, tile, theta):
    c = _coeffs(sum(sizes) + T)
    h = pcot.pcot_create(2, 1, c, pcot.PCOT_DIRICHLET)
    g = si.uniform_grid(sizes, 31 + T, ring="random")
    got = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW, _params(tile, theta))
    assert np.array_equal(got, oracle.sweep(g, sizes, c, T))
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("sizes,T,tile,theta", CASES[2:7])
def test_fp64_fma_mode_within_bound(sizes, T, tile, theta):
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    g = si.uniform_grid(sizes, 41 + T)
    got = run_gpu(h, g, sizes, T, pcot.PCOT_F64, pcot.PCOT_SKEW, _params(tile, theta))
    ref = oracle.sweep(g, sizes, HEAT2D, T)
    err = oracle.pointwise_rel_error(oracle.interior(got, sizes), oracle.interior(ref, sizes))
    assert err <= fma_mode_f64_bound(T), err
    # the FMA-mode kernels all round alike: bitwise equal to the FP64 sweep
    same = run_gpu(h, g, sizes, T, pcot.PCOT_F64, pcot.PCOT_SWEEP)
    assert np.array_equal(got, same)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("sizes,T,tile,theta", CASES[2:7])
def test_fp32_within_tolerance(sizes, T, tile, theta):
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    g32 = si.uniform_grid(sizes, 51 + T, dtype=np.float32)
    got = run_gpu(h, g32, sizes, T, pcot.PCOT_F32, pcot.PCOT_SKEW, _params(tile, theta))
    assert_f32_close(got, oracle.sweep(g32, sizes, HEAT2D, T), sizes, what="skew")
    assert np.array_equal(got, run_gpu(h, g32, sizes, T, pcot.PCOT_F32, pcot.PCOT_SWEEP))
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("T", [6, 7])
def test_padding_and_stale_workspace(T):
    """Padded rows inside a sentinel-filled buffer, a workspace full of stale
    bytes, odd and even T (an odd T ends with the copy back from the twin):
    the stored cells equal the oracle and no other byte changes."""
    c = _coeffs(90 + T)
    h = pcot.pcot_create(2, 1, c, pcot.PCOT_DIRICHLET)
    sizes = (150, 211)
    shape = tuple(n + 2 for n in sizes)
    st = padded_strides(shape, 8, 128)
    span = (shape[0] - 1) * st[0] + shape[1]
    base = torch.full((span + 2048,), -777.0, dtype=torch.float64, device="cuda")
    view = torch.as_strided(base, shape, st, 512)
    g = si.uniform_grid(sizes, 19, ring="random")
    view.copy_(torch.from_numpy(g).cuda())
    p = _params((4, 16, 32), None)
    nb = pcot.pcot_workspace_bytes(h, sizes, st, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW, p)
    ws = torch.full((nb,), 0x5A, dtype=torch.uint8, device="cuda")
    pcot.pcot_run(h, view.data_ptr(), ws.data_ptr(), nb, sizes, st, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW, p)
    assert pcot.pcot_check(h) == pcot.PCOT_OK
    assert np.array_equal(view.cpu().numpy(), oracle.sweep(g, sizes, c, T))
    mask = torch.ones_like(base, dtype=torch.bool)
    torch.as_strided(mask, shape, st, 512).fill_(False)
    assert np.all(base[mask].cpu().numpy() == -777.0)
    pcot.pcot_destroy(h)


def test_repeated_calls_reuse_the_plan():
    """Two calls on one handle (the second reuses the cached plan and its
    upload image) give the same bits, and T = 0 leaves the grid alone."""
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    sizes, T = (200, 333), 19
    g = si.uniform_grid(sizes, 7)
    a = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW)
    b = run_gpu(h, g, sizes, T, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW)
    assert np.array_equal(a, b) and np.array_equal(a, oracle.sweep(g, sizes, HEAT2D, T))
    assert np.array_equal(run_gpu(h, g, sizes, 0, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW), g)
    pcot.pcot_destroy(h)


def test_unsupported_shapes_are_rejected():
    h3 = pcot.pcot_create(3, 1, [0.4, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1], pcot.PCOT_DIRICHLET)
    hp = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_PERIODIC)
    h = pcot.pcot_create(2, 1, HEAT2D, pcot.PCOT_DIRICHLET)
    with pytest.raises(pcot.PcotError):
        pcot.pcot_workspace_bytes(h3, (8, 8, 8), None, 4, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW, None)
    with pytest.raises(pcot.PcotError):
        pcot.pcot_workspace_bytes(hp, (8, 8), None, 4, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW, None)
    with pytest.raises(pcot.PcotError):   # window larger than shared memory
        run_gpu(h, np.zeros((66, 66)), (64, 64), 4, pcot.PCOT_F64_EXACT, pcot.PCOT_SKEW,
                _params((16, 256, 256), None))
    for x in (h3, hp, h):
        pcot.pcot_destroy(x)
