"""Torch-tensor front end of the C ABI (device memory and streams only).

``beamform`` calls ``pa_beamform`` on CUDA tensors; ``beamform_host`` calls
``pa_beamform_host`` on host tensors or numpy arrays.  Shapes follow the
ABI: RF ``[frames][N][Ns]``, output ``[frames][stages][outputs][nx][nz]``.
"""

from __future__ import annotations

import ctypes

import numpy as np

from ._native import (
    PA_RF_BF16,
    PA_RF_F16,
    PA_RF_F32,
    Metrics,
    Plan,
    Roi,
    check,
    load,
    make_grid,
    make_region,
)


def _torch():
    import torch

    return torch


def _rf_torch_dtype(code):
    torch = _torch()
    return {PA_RF_F32: torch.float32, PA_RF_BF16: torch.bfloat16, PA_RF_F16: torch.float16}[code]


def _check_rf(plan: Plan, rf, device: bool):
    torch = _torch()
    d = plan.desc
    if rf.dim() != 3 or rf.shape[1] != d.n_elem or rf.shape[2] != d.n_samples:
        raise ValueError(f"rf must be [frames][{d.n_elem}][{d.n_samples}], got {tuple(rf.shape)}")
    want = _rf_torch_dtype(d.rf_dtype)
    if rf.dtype != want and not (rf.dtype == torch.int16 and d.rf_dtype != PA_RF_F32):
        raise ValueError(f"rf dtype {rf.dtype} does not match the plan ({want})")
    if not rf.is_contiguous():
        raise ValueError("rf must be contiguous")
    if device and not rf.is_cuda:
        raise ValueError("rf must be a CUDA tensor")


def beamform(plan: Plan, rf, stages: int, out=None, stream=None):
    """Run the hot path on device-resident frames; asynchronous on ``stream``
    (default: torch's current stream)."""
    torch = _torch()
    _check_rf(plan, rf, device=True)
    shape = plan.out_shape(rf.shape[0], stages)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=rf.device)
    elif tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError(f"out must be contiguous float32 {shape}")
    if stream is None:
        stream = torch.cuda.current_stream(rf.device)
    plan.beamform(rf.data_ptr(), rf.shape[0], out.data_ptr(), stages, stream)
    return out


def beamform_host(plan: Plan, rf, stages: int, out=None, stream=None):
    """Host buffers in, host buffers out (copies inside the call).  ``rf`` is
    a host torch tensor (pinned for full copy speed) or a numpy array (BF16
    as uint16 bit patterns)."""
    torch = _torch()
    if isinstance(rf, np.ndarray):
        rf = np.ascontiguousarray(rf)
        n = rf.shape[0]
        ptr = rf.ctypes.data
        d = plan.desc
        if rf.shape[1:] != (d.n_elem, d.n_samples):
            raise ValueError("rf shape does not match the plan")
        if rf.dtype.itemsize != (4 if d.rf_dtype == PA_RF_F32 else 2):
            raise ValueError("rf element size does not match the plan")
    else:
        _check_rf(plan, rf, device=False)
        n = rf.shape[0]
        ptr = rf.data_ptr()
    shape = plan.out_shape(n, stages)
    if out is None:
        out = np.empty(shape, dtype=np.float32)
    if isinstance(out, np.ndarray):
        if out.shape != shape or out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError(f"out must be contiguous float32 {shape}")
        optr = out.ctypes.data
    else:
        if tuple(out.shape) != shape or out.dtype != torch.float32:
            raise ValueError(f"out must be float32 {shape}")
        optr = out.data_ptr()
    plan.beamform_host(ptr, n, optr, stages, stream)
    return out


METRIC_FIELDS = tuple(name for name, _ in Metrics._fields_)


def image_metrics(images, grid, rois, stream=None, out=None):
    """SNR, CR, gCNR and lateral FWHM (Eqs. 10-12) of every ROI pair on every
    image, computed on the device by ``pa_image_metrics``.

    ``images``: CUDA float32 tensor ``[..., nx, nz]`` (leading dims are
    flattened into the image count); ``grid``: workload dict or PlanDesc;
    ``rois``: list of (target, background) region dicts.  Returns a dict of
    numpy arrays shaped ``[n_images, n_roi]`` (synchronises ``stream``), or,
    with ``out`` (a CUDA uint8 tensor of n_images * n_roi * sizeof(Metrics)
    bytes), leaves the raw records there without synchronising."""
    torch = _torch()
    g = make_grid(grid)
    if not (images.is_cuda and images.dtype == torch.float32 and images.is_contiguous()):
        raise ValueError("images must be a contiguous CUDA float32 tensor")
    if tuple(images.shape[-2:]) != (g.nx, g.nz):
        raise ValueError(f"images must end in [{g.nx}][{g.nz}]")
    n_img = int(np.prod(images.shape[:-2])) if images.dim() > 2 else 1
    arr = (Roi * len(rois))(*[Roi(make_region(t), make_region(b)) for t, b in rois])
    nbytes = n_img * len(rois) * ctypes.sizeof(Metrics)
    if out is None:
        dev = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=images.device)
    else:
        dev = out
        if dev.numel() < nbytes or not dev.is_cuda:
            raise ValueError("out is too small")
    if stream is None:
        stream = torch.cuda.current_stream(images.device)
    L = load()
    check(L, L.pa_image_metrics(ctypes.byref(g), images.data_ptr(), n_img, arr, len(rois),
                                dev.data_ptr(), stream.cuda_stream))
    if out is not None:
        return out
    stream.synchronize()
    host = dev[:nbytes].cpu().numpy()
    rec = np.frombuffer(host.tobytes(), dtype=_metrics_dtype()).reshape(n_img, len(rois))
    return {name: rec[name].copy() for name in METRIC_FIELDS}


def _metrics_dtype():
    fmt = {ctypes.c_double: "f8", ctypes.c_int64: "i8", ctypes.c_int32: "i4"}
    return np.dtype({"names": list(METRIC_FIELDS),
                     "formats": [fmt[t] for _, t in Metrics._fields_],
                     "offsets": [getattr(Metrics, n).offset for n in METRIC_FIELDS],
                     "itemsize": ctypes.sizeof(Metrics)})
