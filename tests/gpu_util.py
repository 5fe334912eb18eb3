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


# FP32 results against the FP64 oracle run on the widened FP32 inputs.
# Normwise (max|u - ref| / max|ref|): the accuracy bound of the FP32 mode.
F32_TOL = 1e-5
# Pointwise (each cell's difference over max(|ref(x)|, 1e-3 max|ref|)) for
# fields that stay positive (U[0,1) inputs, positive weights): every value is
# a positive combination of the inputs, so its rounding error is relative to
# its own size and the same 1e-5 holds cell by cell.
F32_POINTWISE_TOL = 1e-5
# Sign-changing fields (the Fourier-mode Jacobi-3D inputs): near a zero
# crossing a cell is much smaller than the terms it is summed from, so its
# error is set by those terms; the floored measure then reaches up to about
# (normwise error) / 1e-3.  The FP32 coefficients 0.4 and 0.1 are not exact
# in binary32, which makes each mode decay about 1.5e-8 per step slower
# than in FP64 (1.9e-6 relative after 128 steps): that alone gives ~2e-3.
F32_POINTWISE_TOL_SIGNED = 1e-2


def f32_errors(got, ref, sizes=None, periodic=False):
    """Normwise and floored pointwise errors of the interior."""
    import oracle
    if sizes is not None and not periodic:
        got = oracle.interior(got, sizes)
        ref = oracle.interior(ref, sizes)
    return oracle.errors(got, ref)


def assert_f32_close(got, ref, sizes=None, periodic=False, pointwise_tol=F32_POINTWISE_TOL, what=""):
    e = f32_errors(got, ref, sizes, periodic)
    assert e["normwise"] <= F32_TOL, (what, e)
    assert e["pointwise"] <= pointwise_tol, (what, e)
    return e


def fma_mode_f64_bound(T, terms=5):
    """Pointwise bound of the FP64 FMA mode against the FP64 oracle for
    positive fields: each side rounds every term of an update at most
    `terms` times (centre product plus one rounding per added neighbour), so
    after T steps each is within gamma_(terms T) = n u / (1 - n u), n = terms
    T, u = 2^-53, of the exact result (relative, cell by cell)."""
    u = 2.0 ** -53
    n = terms * max(T, 1)
    return 2.0 * n * u / (1.0 - n * u) * 1.001
