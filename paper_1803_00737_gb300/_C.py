"""ctypes binding of libdwtfuse (include/dwtfuse.h): argument marshalling only.

Every function here checks that tensors live on a CUDA device and are dense,
turns them into pointers, sizes and the current torch stream, and calls the C
entry point of the same name.  There is no CPU path: if the library is not
built, or a tensor is not on the GPU, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from .build import LIB

OK, EINVAL, ESHAPE, EALIGN, ENOMEM, ECUDA, ETIMEOUT, EDEVICE = range(8)
HAAR, D4 = 0, 1
U8, F32 = 0, 1
MAX_BANDS = 16
MAX_SCENES = 128

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t


class DwtfuseError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = lib().dwtfuse_status_string(status).decode()
        if status == ECUDA:
            msg += f" (cudaError {lib().dwtfuse_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [status {status}]")


class Scene(ctypes.Structure):
    """dwtfuse_scene of include/dwtfuse.h."""
    _fields_ = [
        ("pan", _vp),
        ("ms", _vp * MAX_BANDS),
        ("out_f32", _vp),
        ("out_u8", _vp),
        ("H", _i64),
        ("W", _i64),
        ("bands", ctypes.c_int32),
        ("wavelet", ctypes.c_int32),
        ("in_dtype", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class GradScene(ctypes.Structure):
    """dwtfuse_grad_scene of include/dwtfuse.h."""
    _fields_ = [
        ("grad_out", _vp),
        ("grad_pan", _vp),
        ("grad_ms", _vp * MAX_BANDS),
        ("H", _i64),
        ("W", _i64),
        ("bands", ctypes.c_int32),
        ("wavelet", ctypes.c_int32),
    ]


_SIGS = {
    "dwtfuse_status_string": (ctypes.c_char_p, [_i]),
    "dwtfuse_version": (_i, []),
    "dwtfuse_last_cuda_error": (_i, []),
    "dwtfuse_fuse": (_i, [_vp, ctypes.POINTER(_vp), _i, _i64, _i64, _i, _i, _vp, _vp, _vp]),
    "dwtfuse_fuse_ex": (_i, [_vp, ctypes.POINTER(_vp), _i, _i64, _i64, _i, _i, ctypes.c_float, _vp, _vp,
                             _vp]),
    "dwtfuse_fuse_rows": (_i, [_vp, ctypes.POINTER(_vp), _i, _i64, _i64, _i64, _i64, _i, _i, _vp, _vp,
                               _vp]),
    "dwtfuse_dwt2": (_i, [_vp, _i, _i64, _i64, _i, _vp, _vp]),
    "dwtfuse_idwt2": (_i, [_vp, _i64, _i64, _i, _vp, _vp, _vp]),
    "dwtfuse_fuse_backward": (_i, [_vp, _i, _i64, _i64, _i, _vp, ctypes.POINTER(_vp), _vp]),
    "dwtfuse_fuse_backward_batched": (_i, [ctypes.POINTER(GradScene), _i, _vp, _sz, _vp]),
    "dwtfuse_batched_workspace_size": (_sz, []),
    "dwtfuse_fuse_batched": (_i, [ctypes.POINTER(Scene), _i, _vp, _sz, _i, _i, _vp]),
    "dwtfuse_get_last_device_status": (_i, [_vp, _vp]),
    "dwtfuse_set_rows_per_item": (_i, [_i]),
    "dwtfuse_set_band_chunks": (_i, [_i, _i]),
    "dwtfuse_set_fuse_staging": (_i, [_i]),
    "dwtfuse_set_metric_wait_test": (_i, [_i]),
    "dwtfuse_fuse_batched_noalloc": (_i, [ctypes.POINTER(Scene), _i, _i, _i, _vp]),
    "dwtfuse_metrics_workspace_size": (_sz, []),
    "dwtfuse_metrics": (_i, [_vp, _i, ctypes.POINTER(_vp), _vp, _i, _i, _i64, _i64, _i, _vp, _sz,
                             _vp, _vp]),
    "dwtfuse_fuse_metrics": (_i, [_vp, ctypes.POINTER(_vp), _i, _i64, _i64, _i, _i, _vp, _vp, _vp, _sz,
                                  _vp, _vp]),
    "dwtfuse_fuse_and_score": (_i, [_vp, ctypes.POINTER(_vp), _i, _i64, _i64, _i, _i, _vp, _vp, _vp, _sz,
                                    _vp]),
    "dwtfuse_score_finish": (_i, [ctypes.POINTER(_vp), _vp, _i, _i, _i64, _i64, _vp, _vp, _sz, _vp, _vp]),
    "dwtfuse_ergas": (_i, [_vp, _i, ctypes.POINTER(_vp), _i, _i, _i64, _i64, _vp, _sz,
                           ctypes.POINTER(ctypes.c_double), _vp]),
    "dwtfuse_qnr": (_i, [_vp, _i, ctypes.POINTER(_vp), _vp, _i, _i, _i64, _i64, _i, _vp, _sz,
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double), _vp]),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libdwtfuse.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(
                    f"{LIB} is missing: build it with paper_1803_00737_gb300.build.build() "
                    "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue  # reported by the symbol test, raised on use
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, what: str) -> None:
    if status != OK:
        raise DwtfuseError(status, what)


def _dev(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (libdwtfuse has no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _dtype_code(t: torch.Tensor, name: str) -> int:
    if t.dtype == torch.uint8:
        return U8
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"{name} must be uint8 or float32, got {t.dtype}")


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _need(t: torch.Tensor | None, n: int, dtype: torch.dtype | None, name: str) -> None:
    """The library reads or writes n elements of t's dtype at t's address: refuse
    a smaller buffer or another element type (it would run past the buffer)."""
    if t is None:
        return
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {n}")


def _bands(ms) -> list[torch.Tensor]:
    if isinstance(ms, torch.Tensor):
        return [ms[b] for b in range(ms.shape[0])] if ms.dim() == 3 else [ms]
    return list(ms)


def dwtfuse_fuse(pan: torch.Tensor, ms, wavelet: int, out_f32: torch.Tensor | None = None,
                 out_u8: torch.Tensor | None = None, stream=None) -> None:
    """Fused forward into caller-provided outputs (see dwtfuse_fuse in dwtfuse.h)."""
    bands = _bands(ms)
    H, W = pan.shape
    code = _dtype_code(pan, "pan")
    ptrs = (_vp * len(bands))(*[_dev(m, f"ms[{b}]") for b, m in enumerate(bands)])
    for b, m in enumerate(bands):
        if m.dtype != pan.dtype or tuple(m.shape) != (H // 2, W // 2):
            raise ValueError(f"ms[{b}] must be {pan.dtype} of shape ({H // 2}, {W // 2})")
    for name, o, dt in (("out_f32", out_f32, torch.float32), ("out_u8", out_u8, torch.uint8)):
        if o is not None and (o.dtype != dt or tuple(o.shape) != (len(bands), H, W)):
            raise ValueError(f"{name} must be {dt} of shape ({len(bands)}, {H}, {W})")
    st = lib().dwtfuse_fuse(_dev(pan, "pan"), ptrs, len(bands), H, W, int(wavelet), code,
                            _dev(out_f32, "out_f32") if out_f32 is not None else None,
                            _dev(out_u8, "out_u8") if out_u8 is not None else None,
                            _stream(stream))
    _check(st, "dwtfuse_fuse")


def dwtfuse_fuse_ex(pan: torch.Tensor, ms, wavelet: int, ll_gain: float,
                    out_f32: torch.Tensor | None = None, out_u8: torch.Tensor | None = None,
                    stream=None) -> None:
    """dwtfuse_fuse with an explicit LL replacement gain."""
    bands = _bands(ms)
    H, W = pan.shape
    for b, m in enumerate(bands):
        _need(m, (H // 2) * (W // 2), pan.dtype, f"ms[{b}]")
    _need(out_f32, len(bands) * H * W, torch.float32, "out_f32")
    _need(out_u8, len(bands) * H * W, torch.uint8, "out_u8")
    ptrs = (_vp * len(bands))(*[_dev(m, f"ms[{b}]") for b, m in enumerate(bands)])
    st = lib().dwtfuse_fuse_ex(_dev(pan, "pan"), ptrs, len(bands), H, W, int(wavelet),
                               _dtype_code(pan, "pan"), float(ll_gain),
                               _dev(out_f32, "out_f32") if out_f32 is not None else None,
                               _dev(out_u8, "out_u8") if out_u8 is not None else None,
                               _stream(stream))
    _check(st, "dwtfuse_fuse_ex")


def row_halo(wavelet: int) -> tuple[int, int]:
    """(PAN rows, MS rows) of halo above a row band's slab (the PAN halo is
    also taken below): 2 and 1 for D4, none for Haar."""
    return (2, 1) if int(wavelet) == D4 else (0, 0)


def dwtfuse_fuse_rows(pan_slab: torch.Tensor, ms_slab, wavelet: int, H: int, y0: int, y1: int,
                      out_f32: torch.Tensor | None = None, out_u8: torch.Tensor | None = None,
                      stream=None) -> None:
    """Fused rows [y0, y1) of an H x W scene from a slab with halo rows (see
    dwtfuse_fuse_rows in dwtfuse.h): pan_slab (y1 - y0 + 2h, W), ms_slab
    (B, (y1 - y0)/2 + hm, W/2), outputs (B, y1 - y0, W)."""
    bands = _bands(ms_slab)
    h, hm = row_halo(wavelet)
    n_rows = y1 - y0
    Hs, W = pan_slab.shape
    if Hs != n_rows + 2 * h:
        raise ValueError(f"pan_slab must hold {n_rows + 2 * h} rows (band plus halo), got {Hs}")
    code = _dtype_code(pan_slab, "pan_slab")
    for b, m in enumerate(bands):
        if m.dtype != pan_slab.dtype or tuple(m.shape) != (n_rows // 2 + hm, W // 2):
            raise ValueError(f"ms_slab[{b}] must be {pan_slab.dtype} of shape ({n_rows // 2 + hm}, {W // 2})")
    for name, o, dt in (("out_f32", out_f32, torch.float32), ("out_u8", out_u8, torch.uint8)):
        if o is not None and (o.dtype != dt or tuple(o.shape) != (len(bands), n_rows, W)):
            raise ValueError(f"{name} must be {dt} of shape ({len(bands)}, {n_rows}, {W})")
    ptrs = (_vp * len(bands))(*[_dev(m, f"ms_slab[{b}]") for b, m in enumerate(bands)])
    st = lib().dwtfuse_fuse_rows(_dev(pan_slab, "pan_slab"), ptrs, len(bands), int(H), W, int(y0), int(y1),
                                 int(wavelet), code,
                                 _dev(out_f32, "out_f32") if out_f32 is not None else None,
                                 _dev(out_u8, "out_u8") if out_u8 is not None else None,
                                 _stream(stream))
    _check(st, "dwtfuse_fuse_rows")


def dwtfuse_dwt2(img: torch.Tensor, wavelet: int, coeffs: torch.Tensor, stream=None) -> None:
    """One-level 2D DWT (rows, then columns) into a float coefficient image."""
    H, W = img.shape
    if coeffs.dtype != torch.float32 or tuple(coeffs.shape) != (H, W):
        raise ValueError(f"coeffs must be float32 of shape ({H}, {W})")
    _check(lib().dwtfuse_dwt2(_dev(img, "img"), _dtype_code(img, "img"), H, W, int(wavelet),
                              _dev(coeffs, "coeffs"), _stream(stream)), "dwtfuse_dwt2")


def dwtfuse_idwt2(coeffs: torch.Tensor, wavelet: int, out_f32: torch.Tensor | None = None,
                  out_u8: torch.Tensor | None = None, stream=None) -> None:
    """Inverse one-level 2D DWT (columns, then rows) into float and/or uint8 images."""
    H, W = coeffs.shape
    if coeffs.dtype != torch.float32:
        raise TypeError("coeffs must be float32")
    _need(out_f32, H * W, torch.float32, "out_f32")
    _need(out_u8, H * W, torch.uint8, "out_u8")
    _check(lib().dwtfuse_idwt2(_dev(coeffs, "coeffs"), H, W, int(wavelet),
                               _dev(out_f32, "out_f32") if out_f32 is not None else None,
                               _dev(out_u8, "out_u8") if out_u8 is not None else None,
                               _stream(stream)), "dwtfuse_idwt2")


def dwtfuse_fuse_backward(grad_out: torch.Tensor, wavelet: int, grad_pan: torch.Tensor,
                          grad_ms, stream=None) -> None:
    """Adjoint of the fusion into caller-provided gradient buffers."""
    B, H, W = grad_out.shape
    if grad_out.dtype != torch.float32 or grad_pan.dtype != torch.float32:
        raise TypeError("gradients must be float32")
    gms = _bands(grad_ms)
    if len(gms) != B:
        raise ValueError("one grad_ms buffer per band")
    _need(grad_pan, H * W, torch.float32, "grad_pan")
    for b, g in enumerate(gms):
        _need(g, (H // 2) * (W // 2), torch.float32, f"grad_ms[{b}]")
    ptrs = (_vp * B)(*[_dev(g, f"grad_ms[{b}]") for b, g in enumerate(gms)])
    st = lib().dwtfuse_fuse_backward(_dev(grad_out, "grad_out"), B, H, W, int(wavelet),
                                     _dev(grad_pan, "grad_pan"), ptrs, _stream(stream))
    _check(st, "dwtfuse_fuse_backward")


def make_grad_scene(grad_out: torch.Tensor, wavelet: int, grad_pan: torch.Tensor, grad_ms) -> GradScene:
    B, H, W = grad_out.shape
    if grad_out.dtype != torch.float32 or grad_pan.dtype != torch.float32:
        raise TypeError("gradients must be float32")
    gms = _bands(grad_ms)
    if len(gms) != B:
        raise ValueError("one grad_ms buffer per band")
    _need(grad_pan, H * W, torch.float32, "grad_pan")
    for b, g in enumerate(gms):
        _need(g, (H // 2) * (W // 2), torch.float32, f"grad_ms[{b}]")
    s = GradScene()
    s.grad_out = _dev(grad_out, "grad_out")
    s.grad_pan = _dev(grad_pan, "grad_pan")
    for b, g in enumerate(gms):
        s.grad_ms[b] = _dev(g, f"grad_ms[{b}]")
    s.H, s.W, s.bands, s.wavelet = H, W, B, int(wavelet)
    return s


def dwtfuse_fuse_backward_batched(scenes: list[GradScene], workspace: torch.Tensor, stream=None) -> None:
    """The adjoint of every scene: per chunk of 8 bands, one persistent launch per
    wavelet and chunk width (see dwtfuse.h)."""
    arr = (GradScene * len(scenes))(*scenes)
    st = lib().dwtfuse_fuse_backward_batched(arr, len(scenes), _dev(workspace, "workspace"),
                                             workspace.numel() * workspace.element_size(),
                                             _stream(stream))
    _check(st, "dwtfuse_fuse_backward_batched")


def dwtfuse_batched_workspace_size() -> int:
    return int(lib().dwtfuse_batched_workspace_size())


def make_scene(pan: torch.Tensor, ms, wavelet: int, out_f32: torch.Tensor | None,
               out_u8: torch.Tensor | None = None) -> Scene:
    bands = _bands(ms)
    H, W = pan.shape
    for b, m in enumerate(bands):
        _need(m, (H // 2) * (W // 2), pan.dtype, f"ms[{b}]")
    _need(out_f32, len(bands) * H * W, torch.float32, "out_f32")
    _need(out_u8, len(bands) * H * W, torch.uint8, "out_u8")
    s = Scene()
    s.pan = _dev(pan, "pan")
    for b, m in enumerate(bands):
        s.ms[b] = _dev(m, f"ms[{b}]")
    s.out_f32 = _dev(out_f32, "out_f32") if out_f32 is not None else None
    s.out_u8 = _dev(out_u8, "out_u8") if out_u8 is not None else None
    s.H, s.W = pan.shape
    s.bands = len(bands)
    s.wavelet = int(wavelet)
    s.in_dtype = _dtype_code(pan, "pan")
    s.reserved = 0
    return s


def dwtfuse_fuse_batched(scenes: list[Scene], workspace: torch.Tensor, rows_per_item: int = 0,
                         blocks_per_sm: int = 0, stream=None) -> None:
    """One persistent launch over all scenes (capturable in a CUDA graph)."""
    arr = (Scene * len(scenes))(*scenes)
    st = lib().dwtfuse_fuse_batched(arr, len(scenes), _dev(workspace, "workspace"),
                                    workspace.numel() * workspace.element_size(),
                                    int(rows_per_item), int(blocks_per_sm), _stream(stream))
    _check(st, "dwtfuse_fuse_batched")


def dwtfuse_fuse_batched_noalloc(scenes: list[Scene], rows_per_item: int = 0,
                                 blocks_per_sm: int = 0, stream=None) -> None:
    """Batched launch for callers that cannot allocate device memory: the queue
    counter lives in the library's own static device array (see dwtfuse.h)."""
    arr = (Scene * len(scenes))(*scenes)
    st = lib().dwtfuse_fuse_batched_noalloc(arr, len(scenes), int(rows_per_item),
                                            int(blocks_per_sm), _stream(stream))
    _check(st, "dwtfuse_fuse_batched_noalloc")


def dwtfuse_metrics_workspace_size() -> int:
    return int(lib().dwtfuse_metrics_workspace_size())


def _metric_args(fused: torch.Tensor, ms):
    bands = _bands(ms)
    B, H, W = fused.shape
    if len(bands) != B:
        raise ValueError("one MS band per fused band")
    for b, m in enumerate(bands):
        _need(m, (H // 2) * (W // 2), bands[0].dtype, f"ms[{b}]")
    ptrs = (_vp * B)(*[_dev(m, f"ms[{b}]") for b, m in enumerate(bands)])
    return bands, B, H, W, ptrs


def dwtfuse_metrics(fused: torch.Tensor, ms, pan: torch.Tensor, workspace: torch.Tensor,
                    out_device: torch.Tensor, window: int = 32, stream=None) -> None:
    """ERGAS, QNR, D_lambda, D_s into the float64 CUDA tensor out_device[0:4] (async)."""
    bands, B, H, W, ptrs = _metric_args(fused, ms)
    if out_device.dtype != torch.float64 or out_device.numel() < 4:
        raise ValueError("out_device must be a float64 CUDA tensor with >= 4 elements")
    _need(pan, H * W, bands[0].dtype, "pan")
    st = lib().dwtfuse_metrics(_dev(fused, "fused"), _dtype_code(fused, "fused"), ptrs,
                               _dev(pan, "pan"), _dtype_code(pan, "pan"), B, H, W, int(window),
                               _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                               _dev(out_device, "out_device"), _stream(stream))
    _check(st, "dwtfuse_metrics")


def _fuse_score_args(pan: torch.Tensor, ms, out_f32, out_u8):
    bands = _bands(ms)
    H, W = pan.shape
    ptrs = (_vp * len(bands))(*[_dev(m, f"ms[{b}]") for b, m in enumerate(bands)])
    for b, m in enumerate(bands):
        if m.dtype != pan.dtype or tuple(m.shape) != (H // 2, W // 2):
            raise ValueError(f"ms[{b}] must be {pan.dtype} of shape ({H // 2}, {W // 2})")
    for name, o, dt in (("out_f32", out_f32, torch.float32), ("out_u8", out_u8, torch.uint8)):
        if o is not None and (o.dtype != dt or tuple(o.shape) != (len(bands), H, W)):
            raise ValueError(f"{name} must be {dt} of shape ({len(bands)}, {H}, {W})")
    return bands, H, W, ptrs


def _out_device(out_device: torch.Tensor):
    if out_device.dtype != torch.float64 or out_device.numel() < 4:
        raise ValueError("out_device must be a float64 CUDA tensor with >= 4 elements")
    return _dev(out_device, "out_device")


def dwtfuse_fuse_metrics(pan: torch.Tensor, ms, wavelet: int, out_f32: torch.Tensor | None,
                         out_u8: torch.Tensor, workspace: torch.Tensor, out_device: torch.Tensor,
                         stream=None) -> None:
    """Fused forward into the caller's outputs, then ERGAS, QNR, D_lambda, D_s
    of the uint8 product into out_device[0:4] (async; see dwtfuse.h)."""
    bands, H, W, ptrs = _fuse_score_args(pan, ms, out_f32, out_u8)
    st = lib().dwtfuse_fuse_metrics(_dev(pan, "pan"), ptrs, len(bands), H, W, int(wavelet),
                                    _dtype_code(pan, "pan"),
                                    _dev(out_f32, "out_f32") if out_f32 is not None else None,
                                    _dev(out_u8, "out_u8"), _dev(workspace, "workspace"),
                                    workspace.numel() * workspace.element_size(),
                                    _out_device(out_device), _stream(stream))
    _check(st, "dwtfuse_fuse_metrics")


def dwtfuse_fuse_and_score(pan: torch.Tensor, ms, wavelet: int, out_f32: torch.Tensor | None,
                           out_u8: torch.Tensor, workspace: torch.Tensor, stream=None) -> None:
    """First half of dwtfuse_fuse_metrics: the forward that scores its product."""
    bands, H, W, ptrs = _fuse_score_args(pan, ms, out_f32, out_u8)
    st = lib().dwtfuse_fuse_and_score(_dev(pan, "pan"), ptrs, len(bands), H, W, int(wavelet),
                                      _dtype_code(pan, "pan"),
                                      _dev(out_f32, "out_f32") if out_f32 is not None else None,
                                      _dev(out_u8, "out_u8"), _dev(workspace, "workspace"),
                                      workspace.numel() * workspace.element_size(), _stream(stream))
    _check(st, "dwtfuse_fuse_and_score")


def dwtfuse_score_finish(ms, pan: torch.Tensor, out_u8: torch.Tensor, workspace: torch.Tensor,
                         out_device: torch.Tensor, stream=None) -> None:
    """Second half of dwtfuse_fuse_metrics: MS-resolution pass and reduction."""
    bands, H, W, ptrs = _fuse_score_args(pan, ms, None, out_u8)
    st = lib().dwtfuse_score_finish(ptrs, _dev(pan, "pan"), _dtype_code(pan, "pan"), len(bands), H, W,
                                    _dev(out_u8, "out_u8"), _dev(workspace, "workspace"),
                                    workspace.numel() * workspace.element_size(),
                                    _out_device(out_device), _stream(stream))
    _check(st, "dwtfuse_score_finish")


def dwtfuse_ergas(fused: torch.Tensor, ms, workspace: torch.Tensor, stream=None) -> float:
    bands, B, H, W, ptrs = _metric_args(fused, ms)
    out = ctypes.c_double()
    st = lib().dwtfuse_ergas(_dev(fused, "fused"), _dtype_code(fused, "fused"), ptrs,
                             _dtype_code(bands[0], "ms"), B, H, W, _dev(workspace, "workspace"),
                             workspace.numel() * workspace.element_size(), ctypes.byref(out),
                             _stream(stream))
    _check(st, "dwtfuse_ergas")
    return out.value


def dwtfuse_qnr(fused: torch.Tensor, ms, pan: torch.Tensor, workspace: torch.Tensor,
                window: int = 32, stream=None) -> tuple[float, float, float]:
    bands, B, H, W, ptrs = _metric_args(fused, ms)
    _need(pan, H * W, bands[0].dtype, "pan")
    q, dl, ds = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().dwtfuse_qnr(_dev(fused, "fused"), _dtype_code(fused, "fused"), ptrs, _dev(pan, "pan"),
                           _dtype_code(pan, "pan"), B, H, W, int(window), _dev(workspace, "workspace"),
                           workspace.numel() * workspace.element_size(), ctypes.byref(q),
                           ctypes.byref(dl), ctypes.byref(ds), _stream(stream))
    _check(st, "dwtfuse_qnr")
    return q.value, dl.value, ds.value


def dwtfuse_get_last_device_status(workspace: torch.Tensor | None, stream=None) -> int:
    """Status word of a batched workspace; None: of the last no-alloc batched call."""
    ws = None if workspace is None else _dev(workspace, "workspace")
    return int(lib().dwtfuse_get_last_device_status(ws, _stream(stream)))


def dwtfuse_set_rows_per_item(rows: int) -> None:
    _check(lib().dwtfuse_set_rows_per_item(int(rows)), "dwtfuse_set_rows_per_item")


def dwtfuse_set_band_chunks(fwd: int, bwd: int) -> None:
    """Most bands per forward / adjoint launch (0 = library default; see dwtfuse.h)."""
    _check(lib().dwtfuse_set_band_chunks(int(fwd), int(bwd)), "dwtfuse_set_band_chunks")


def dwtfuse_set_fuse_staging(on: bool) -> None:
    """Let the single-scene forward take the staged kernel where it applies (default on; see dwtfuse.h)."""
    _check(lib().dwtfuse_set_fuse_staging(int(bool(on))), "dwtfuse_set_fuse_staging")


def dwtfuse_set_metric_wait_test(on: bool) -> None:
    """Test hook: make the unaligned metric pass's bounded wait give up (see dwtfuse.h)."""
    _check(lib().dwtfuse_set_metric_wait_test(int(bool(on))), "dwtfuse_set_metric_wait_test")
