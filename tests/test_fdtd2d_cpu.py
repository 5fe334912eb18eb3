"""FDTD-2D entry points without a GPU: argument checks and workspace sizes."""
import pytest

pcot = pytest.importorskip("paper_1802_00166_gb300")


def test_workspace_holds_a_second_copy_and_the_queue():
    # three twins of a 100 x 60 FP64 field (256-byte aligned) ...
    twin = ((99 * 60 + 60) * 8 + 255) // 256 * 256
    assert pcot.pcot_fdtd2d_workspace_bytes((100, 60), None, 10, pcot.PCOT_F64, pcot.PCOT_SLT) == 3 * twin
    assert pcot.pcot_fdtd2d_workspace_bytes((100, 60), None, 10, pcot.PCOT_F64, pcot.PCOT_SWEEP) == 3 * twin
    # ... plus, for the recursive order, a head block, the counters and the queue
    # of 2 blocks x 4 x 2 tiles (32 x 32 tiles, depth 4)
    cot = pcot.pcot_fdtd2d_workspace_bytes((100, 60), None, 10, pcot.PCOT_F64, pcot.PCOT_COT)
    assert cot == 3 * twin + 256 + 2 * 256
    # padded rows
    tw2 = ((99 * 64 + 60) * 4 + 255) // 256 * 256
    assert pcot.pcot_fdtd2d_workspace_bytes((100, 60), (64, 1), 3, pcot.PCOT_F32, pcot.PCOT_SWEEP) == 3 * tw2


@pytest.mark.parametrize("kwargs", [dict(tile=(4, 32), time_depth=8),      # tile narrower than the halo
                                    dict(tile=(32, 32), time_depth=80)])   # depth above 64
def test_unsupported_tiles(kwargs):
    with pytest.raises(pcot.PcotError):
        pcot.pcot_fdtd2d_workspace_bytes((100, 60), None, 10, pcot.PCOT_F64, pcot.PCOT_SLT,
                                         pcot.tile_params(**kwargs))


def test_invalid_arguments():
    with pytest.raises(pcot.PcotError):
        pcot.pcot_fdtd2d_workspace_bytes((0, 5), None, 3, pcot.PCOT_F64, pcot.PCOT_SLT)
    with pytest.raises(pcot.PcotError):   # row stride below the row length
        pcot.pcot_fdtd2d_workspace_bytes((5, 9), (8, 1), 3, pcot.PCOT_F64, pcot.PCOT_SLT)
