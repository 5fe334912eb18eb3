"""LU and Cholesky on the GPU against the oracle's plain loops (the
linear-algebra kernels of the benchmark suite, Sec. 5.1.2): every schedule,
both tile sides, ragged last blocks, padded rows, fused and unfused updates,
all bitwise."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

torch = pytest.importorskip("torch")
pcot = pytest.importorskip("paper_1802_00166_gb300")

pytestmark = pytest.mark.gpu
KINDS = {"lu": pcot.PCOT_LA_LU, "cholesky": pcot.PCOT_LA_CHOLESKY}
SENTINEL = 12345.5


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


def matrix(kind, n, seed):
    return si.dominant_matrix(n, seed, symmetric=(kind == "cholesky"))


def run_la(h, kind, A, dtype, sched, params=None, lda=None):
    n = A.shape[0]
    ld = lda or n
    base = torch.full((max(n * ld, 1) + 16,), SENTINEL, dtype=torch.float64, device="cuda")
    view = torch.as_strided(base, (n, n), (ld, 1))
    view.copy_(torch.from_numpy(A).cuda())
    nb = pcot.pcot_la_workspace_bytes(KINDS[kind], n, sched, params)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) // 256 * 256
    pcot.pcot_la_run(h, KINDS[kind], base.data_ptr(), wp, nb, n, ld, dtype, sched, params)
    st = pcot.pcot_check(h)
    if st != pcot.PCOT_OK:
        raise pcot.PcotError(st, "la")
    out = torch.as_strided(base, (n, n), (ld, 1)).cpu().numpy()
    full = base.cpu().numpy()
    for r in range(n):  # the padding of every row is untouched
        assert np.all(full[r * ld + n:(r + 1) * ld] == SENTINEL)
    assert np.all(full[n * ld:] == SENTINEL)
    return out


SCHEDS = [
    ("sweep", pcot.PCOT_SWEEP, None),
    ("slt32", pcot.PCOT_SLT, dict(tile=(32, 0, 0))),
    ("slt64", pcot.PCOT_SLT, dict(tile=(64, 0, 0))),
    ("cot32_111", pcot.PCOT_COT, dict(tile=(32, 0, 0), cot_threshold=(1, 1, 1))),
    ("cot64_222", pcot.PCOT_COT, dict(tile=(64, 0, 0), cot_threshold=(2, 2, 2))),
    ("cot32_421", pcot.PCOT_COT, dict(tile=(32, 0, 0), cot_threshold=(4, 2, 1))),
]
DTYPES = [("fma", pcot.PCOT_F64, True), ("exact", pcot.PCOT_F64_EXACT, False)]


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
@pytest.mark.parametrize("dname,dtype,fused", DTYPES)
@pytest.mark.parametrize("sname,sched,params", SCHEDS)
@pytest.mark.parametrize("n", [1, 2, 33, 64, 65, 100, 200, 257])
def test_bitwise_equal_to_plain_loops(handle, kind, dname, dtype, fused, sname, sched, params, n):
    A = matrix(kind, n, 20 + n)
    ref = getattr(oracle, kind)(A, fused=fused)
    got = run_la(handle, kind, A, dtype, sched, params)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
@pytest.mark.parametrize("sname,sched,params", SCHEDS[1:])
def test_padded_rows(handle, kind, sname, sched, params):
    """Row stride above n: the padding stays untouched and the result is the
    same."""
    n = 97
    A = matrix(kind, n, 31)
    got = run_la(handle, kind, A, pcot.PCOT_F64, sched, params, lda=n + 13)
    assert np.array_equal(got, getattr(oracle, kind)(A, fused=True))


@pytest.mark.parametrize("kind", ["lu", "cholesky"])
def test_upper_triangle_untouched_by_cholesky_and_sweeps_agree(handle, kind):
    """Cholesky leaves the strict upper triangle as it was (the oracle does
    too); every schedule gives the same bits on a larger problem."""
    n = 700
    A = matrix(kind, n, 41)
    if kind == "cholesky":
        A[np.triu_indices(n, 1)] = -7.25
    ref = getattr(oracle, kind)(A, fused=True)
    for _, sched, params in SCHEDS:
        got = run_la(handle, kind, A, pcot.PCOT_F64, sched, params)
        assert np.array_equal(got, ref)
    if kind == "cholesky":
        assert np.all(got[np.triu_indices(n, 1)] == -7.25)


def test_launch_counts(handle):
    """Sweep: two launches per k; single-level: panels and updates per block
    step (plus the first diagonal tile); recursive: one persistent launch."""
    n = 130
    A = matrix("lu", n, 5)
    c0 = pcot.pcot_launch_count(handle)
    run_la(handle, "lu", A, pcot.PCOT_F64, pcot.PCOT_COT, dict(tile=(64, 0, 0)))
    c1 = pcot.pcot_launch_count(handle)
    assert c1 - c0 == 1
    run_la(handle, "lu", A, pcot.PCOT_F64, pcot.PCOT_SLT, dict(tile=(64, 0, 0)))
    c2 = pcot.pcot_launch_count(handle)
    assert c2 - c1 == 3 + 2  # L = 3: diagonal, panels, updates; then panels, updates (the next
    # diagonal tiles are factored inside the update launches)
    run_la(handle, "lu", A, pcot.PCOT_F64, pcot.PCOT_SWEEP)
    c3 = pcot.pcot_launch_count(handle)
    assert c3 - c2 == 2 * (n - 1)


def test_unsupported_and_invalid(handle):
    A = torch.zeros(16 * 16, dtype=torch.float64, device="cuda")
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_la_run(handle, pcot.PCOT_LA_LU, A.data_ptr(), None, 0, 16, 16, pcot.PCOT_F32, pcot.PCOT_SLT)
    assert e.value.status == pcot.PCOT_ERR_UNSUPPORTED
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_la_run(handle, pcot.PCOT_LA_LU, A.data_ptr(), None, 0, 16, 15, pcot.PCOT_F64, pcot.PCOT_SLT)
    assert e.value.status == pcot.PCOT_ERR_INVALID_ARG
    with pytest.raises(pcot.PcotError) as e:
        pcot.pcot_la_run(handle, pcot.PCOT_LA_LU, A.data_ptr() + 4, None, 0, 8, 8, pcot.PCOT_F64, pcot.PCOT_SLT)
    assert e.value.status == pcot.PCOT_ERR_ALIGNMENT
    with pytest.raises(pcot.PcotError) as e:  # the recursive schedule needs its workspace
        pcot.pcot_la_run(handle, pcot.PCOT_LA_LU, A.data_ptr(), None, 0, 16, 16, pcot.PCOT_F64, pcot.PCOT_COT)
    assert e.value.status == pcot.PCOT_ERR_OOM
    pcot.pcot_la_run(handle, pcot.PCOT_LA_CHOLESKY, A.data_ptr(), None, 0, 0, 0, pcot.PCOT_F64, pcot.PCOT_COT)
    assert pcot.pcot_check(handle) == pcot.PCOT_OK


@pytest.mark.slow
@pytest.mark.parametrize("kind,n", [("lu", 3000), ("cholesky", 4000)])
def test_paper_sizes_bitwise(handle, kind, n):
    """The paper's problem sizes (Table 2: LUD 3000^2, Cholesky 4000^2) in the
    benchmark's configuration, against the full oracle."""
    A = matrix(kind, n, 7)
    ref = getattr(oracle, kind)(A, fused=False)
    got = run_la(handle, kind, A, pcot.PCOT_F64_EXACT, pcot.PCOT_COT, dict(tile=(64, 0, 0)))
    assert np.array_equal(got, ref)
