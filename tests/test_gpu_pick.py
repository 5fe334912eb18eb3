"""pcot_pick: the library's own picker (its built-in model, a loaded one, or
the exhaustive autotuner when none is loaded), and PCOT_AUTO runs through it.
The paper explores tile sizes by timing each (Sec. 5.1.5); the picker is the
GPU counterpart that predicts instead of timing every candidate."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")
from paper_1802_00166_gb300 import tuner  # noqa: E402
from tests.gpu_util import HEAT2D, JAC3D, assert_f32_close, run_gpu  # noqa: E402

pytestmark = pytest.mark.gpu

PROBLEMS = [(2, (1500, 1700), 96, False), (2, (4000, 3000), 200, False), (3, (160, 160, 160), 40, True),
            (3, (256, 256, 256), 64, True)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00166_gb300 import build
    build.build()


def _handle(dims, periodic):
    return pcot.pcot_create(dims, 1, HEAT2D if dims == 2 else JAC3D,
                            pcot.PCOT_PERIODIC if periodic else pcot.PCOT_DIRICHLET)


@pytest.mark.parametrize("dims,sizes,T,periodic", PROBLEMS)
def test_pick_with_model_equals_the_python_picker(dims, sizes, T, periodic):
    """With the committed model loaded, the library's pick is the candidate
    the explicit-model call (the tuner's Picker) chooses."""
    picker = tuner.Picker.load()
    h = _handle(dims, periodic)
    pcot.pcot_picker_load(h, picker.params, picker.feat_mean, picker.feat_std)
    sched, prm = pcot.pcot_pick(h, sizes, T, pcot.PCOT_F32)
    cands = tuner.candidates(dims, pcot.PCOT_F32, periodic)
    i = picker.pick(h, sizes, T, pcot.PCOT_F32, cands)
    full = pcot.pcot_candidates(h, pcot.PCOT_F32)
    assert (sched, prm) == full[i]
    assert pcot.pcot_pick(h, sizes, T, pcot.PCOT_F32) == (sched, prm)     # cached
    pcot.pcot_destroy(h)


def test_builtin_model_is_the_committed_one():
    picker = tuner.Picker.load()
    a = _handle(2, False)
    b = _handle(2, False)
    pcot.pcot_picker_load(b, picker.params, picker.feat_mean, picker.feat_std)
    for sizes, T in (((2048, 2048), 128), ((6000, 5000), 300)):
        assert pcot.pcot_pick(a, sizes, T, pcot.PCOT_F32) == pcot.pcot_pick(b, sizes, T, pcot.PCOT_F32)
    pcot.pcot_destroy(a)
    pcot.pcot_destroy(b)


def test_pick_without_model_falls_back_to_the_autotuner():
    """No model: the pick is the autotuner's fastest candidate; re-timed, it
    is within timing noise of the best re-timed candidate."""
    dims, sizes, T, periodic = 2, (2000, 2000), 64, False
    h = _handle(dims, periodic)
    pcot.pcot_picker_load(h)
    sched, prm = pcot.pcot_pick(h, sizes, T, pcot.PCOT_F32)
    cands = pcot.pcot_candidates(h, pcot.PCOT_F32)
    assert (sched, prm) in cands and sched != pcot.PCOT_SWEEP
    _, ms, _ = tuner.tune_problem(dict(dims=dims, sizes=sizes, T=T, periodic=periodic), reps=3,
                                  cands=tuner.candidates(dims, pcot.PCOT_F32, periodic))
    i = cands.index((sched, prm))
    best = min(t for t in ms if t > 0)
    assert ms[i] <= 1.15 * best, (ms[i], best)
    pcot.pcot_destroy(h)


@pytest.mark.parametrize("dims,sizes,T,periodic", [(2, (700, 900), 40, False), (3, (48, 40, 96), 9, True)])
@pytest.mark.parametrize("model", [True, False])
def test_auto_schedule_runs_the_pick(dims, sizes, T, periodic, model):
    """PCOT_AUTO runs the picked schedule: the result equals an explicit run
    of it bitwise (every FP32 schedule rounds the same way) and the oracle
    within the FP32 tolerance; the AUTO workspace size covers the pick."""
    h = _handle(dims, periodic)
    if not model:
        pcot.pcot_picker_load(h)
    g = si.uniform_grid(sizes, 17, periodic=periodic, dtype=np.float32) if dims == 2 else \
        si.fourier_grid(sizes, 3)[0].astype(np.float32)
    got = run_gpu(h, g, sizes, T, pcot.PCOT_F32, pcot.PCOT_AUTO)
    sched, prm = pcot.pcot_pick(h, sizes, T, pcot.PCOT_F32)
    ref = run_gpu(h, g, sizes, T, pcot.PCOT_F32, sched, pcot.tile_params(**prm))
    assert np.array_equal(got, ref)
    auto = pcot.pcot_workspace_bytes(h, sizes, None, T, pcot.PCOT_F32, pcot.PCOT_AUTO)
    assert auto >= pcot.pcot_workspace_bytes(h, sizes, None, T, pcot.PCOT_F32, sched, pcot.tile_params(**prm))
    want = oracle.sweep(g, sizes, HEAT2D if dims == 2 else JAC3D, T, periodic=periodic)
    if dims == 2:
        assert_f32_close(got, want, sizes)
    else:
        assert oracle.max_rel_error(got, want) <= 1e-5
    pcot.pcot_destroy(h)
