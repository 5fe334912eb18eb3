"""Helpers of the GPU tests: run a problem through the C ABI on torch memory."""
import numpy as np

import paper_1802_00166_gb300 as pcot

HEAT2D = [0.5, 0.125, 0.125, 0.125, 0.125]
JAC3D = [0.4] + [0.1] * 6
JAC1D = [1.0 / 3.0] * 3
COEFFS = {1: JAC1D, 2: HEAT2D, 3: JAC3D}


def torch_dtype(dt):
    import torch
    return torch.float32 if dt == pcot.PCOT_F32 else torch.float64


def np_dtype(dt):
    return np.float32 if dt == pcot.PCOT_F32 else np.float64


def padded_strides(shape, elem, align_bytes=16):
    """Row-major strides with every row padded to a multiple of align_bytes."""
    d = len(shape)
    st = [1] * d
    step = max(1, align_bytes // elem)
    inner = ((shape[-1] + step - 1) // step) * step
    acc = inner
    for a in range(d - 2, -1, -1):
        st[a] = acc
        acc *= shape[a]
    return st


def run_gpu(h, grid_np, sizes, T, dtype, schedule, params=None, strides=None, stream=None, ws_extra=0):
    """Copy grid to the device (optionally into a strided layout), run, copy back."""
    import torch
    shape = grid_np.shape
    tdt = torch_dtype(dtype)
    elem = 4 if dtype == pcot.PCOT_F32 else 8
    if strides is None:
        dev = torch.from_numpy(np.ascontiguousarray(grid_np.astype(np_dtype(dtype)))).cuda()
        base = dev
    else:
        span = sum((shape[a] - 1) * strides[a] for a in range(len(shape))) + 1
        base = torch.zeros(span + 64, dtype=tdt, device="cuda")
        view = torch.as_strided(base, shape, strides)
        view.copy_(torch.from_numpy(np.ascontiguousarray(grid_np.astype(np_dtype(dtype)))).cuda())
        dev = view
    nbytes = pcot.pcot_workspace_bytes(h, sizes, strides, T, dtype, schedule, params)
    ws = torch.empty(nbytes + ws_extra + 256, dtype=torch.uint8, device="cuda")
    ws_ptr = (ws.data_ptr() + 255) // 256 * 256
    pcot.pcot_run(h, dev.data_ptr(), ws_ptr, nbytes, sizes, strides, T, dtype, schedule, params, stream)
    st = pcot.pcot_check(h, stream)
    if st != pcot.PCOT_OK:
        raise pcot.PcotError(st, "pcot_check")
    out = dev.cpu().numpy() if strides is None else torch.as_strided(base, shape, strides).cpu().numpy()
    return out
