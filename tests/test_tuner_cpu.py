"""Host-side pieces of the autotuner: candidate sets, problem sets, layouts."""
import numpy as np
import pytest

pcot = pytest.importorskip("paper_1802_00166_gb300")
from paper_1802_00166_gb300 import tuner  # noqa: E402


def test_candidate_sets():
    c2 = tuner.candidates(2, pcot.PCOT_F32, False)
    assert c2[0][0] == pcot.PCOT_SWEEP
    assert any(s == pcot.PCOT_COT for s, _ in c2)
    assert not any(s == pcot.PCOT_COT for s, _ in tuner.candidates(3, pcot.PCOT_F32, True))
    d = tuner.default_candidate(2, pcot.PCOT_F32)
    assert d in c2


def test_problem_sets_are_seeded_and_in_range():
    a = tuner.problem_set(4, 10, 5)
    b = tuner.problem_set(4, 10, 5)
    assert a == b
    for p in a:
        if p["dims"] == 2:
            assert 1024 <= p["sizes"][0] <= 8192 and 64 <= p["T"] <= 512 and not p["periodic"]
        else:
            assert 120 <= p["sizes"][0] <= 512 and 16 <= p["T"] <= 128 and p["periodic"]
    assert tuner.problem_set(5, 10, 5) != a


def test_padded_layout_rows_are_128_byte_multiples():
    shape, st, span = tuner.padded_layout((100, 250), False)
    assert shape == (102, 252) and st[1] == 1 and (st[0] * 4) % 128 == 0
    assert span == 101 * st[0] + 252


def test_features_via_abi_without_gpu():
    h = pcot.pcot_create(2, 1, tuner.HEAT2D, pcot.PCOT_DIRICHLET)
    f_sweep = pcot.pcot_features(h, (1000, 2000), 64, pcot.PCOT_F32, pcot.PCOT_SWEEP)
    f_cot = pcot.pcot_features(h, (1000, 2000), 64, pcot.PCOT_F32, pcot.PCOT_COT,
                               pcot.tile_params(tile=(64, 0), time_depth=8, cot_threshold=(2, 4, 8)))
    assert f_sweep[0] == 2 and f_sweep[10] == -1 and f_sweep[9] == 0
    assert np.isclose(f_cot[2], np.log2(1000)) and np.isclose(f_cot[3], np.log2(2000))
    assert np.isclose(f_cot[9], 3.0) and np.isclose(f_cot[10], 6.0) and np.isclose(f_cot[6], 6.0)
    q = pcot.pcot_plan_query(h, (1000, 2000), 64, pcot.PCOT_F32,
                             pcot.tile_params(tile=(64, 0), time_depth=8, cot_threshold=(2, 4, 8)), with_queue=False)
    assert f_sweep[1] == 0 and np.isclose(f_cot[1], np.log2(q["lattice"][1] * q["lattice"][2]))
    pcot.pcot_destroy(h)


def test_modelled_bytes():
    assert tuner.modelled_bytes((10, 10), 8, pcot.PCOT_SWEEP, 1) == 2 * 8 * 100 * 4
    assert tuner.modelled_bytes((10, 10), 9, pcot.PCOT_SLT, 4) == 2 * 3 * 100 * 4


def test_records_targets_are_measured_time_and_slowdown():
    """Targets of the picker's records: log ms and the capped log slowdown
    against the problem's fastest candidate (0 for the fastest)."""
    prob = dict(dims=2, sizes=(64, 64), T=8, periodic=False)
    cands = [(pcot.PCOT_SWEEP, {}), (pcot.PCOT_SLT, dict(tile=(0, 0), time_depth=2)),
             (pcot.PCOT_SLT, dict(tile=(0, 0), time_depth=4)), (pcot.PCOT_SLT, dict(tile=(0, 0), time_depth=8))]
    ms = [4.0, 1.0, -1.0, 10.0]
    feats = np.zeros((4, 12), dtype=np.float32)
    x, y = tuner.records_for(prob, cands, ms, feats)
    assert len(x) == 3
    assert np.allclose([r[0] for r in y], np.log([4.0, 1.0, 10.0]))
    assert np.allclose([r[1] for r in y], [np.log(3.0), 0.0, np.log(3.0)])   # 4x and 10x slower: capped


def test_committed_picker_report_meets_the_bar():
    """The held-out evaluation recorded when the committed model was trained
    (64 problems re-tuned exhaustively): time-weighted regret <= 10%, no pick
    more than 25% off, at least 90% of picks within 10%, better than the
    fixed default tile."""
    import json
    import os
    path = os.path.join(tuner.DATA_DIR, "report.json")
    r = json.load(open(path))["heldout"]
    assert r["regret_time_weighted"] <= 0.10, r
    assert r["regret_max"] <= 0.25, r
    assert r["frac_within_10pct"] >= 0.90, r
    assert r["regret_mean"] < r["default_regret_mean"], r
