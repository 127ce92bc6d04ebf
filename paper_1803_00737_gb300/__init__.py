"""libdwtfuse: one-level 2D DWT pansharpening (arXiv:1803.00737, Sec. 2) on one
GPU, as hand-written CUDA for sm_103a behind a C ABI (include/dwtfuse.h).

PyTorch supplies device memory and streams; every step of the fusion runs in
the library's kernels.  ``fuse`` allocates outputs and calls the C ABI;
``_C`` exposes the entry points under their C names.
"""
from __future__ import annotations

import torch

from . import _C
from ._C import D4, F32, HAAR, U8, DwtfuseError  # noqa: F401


def fuse(pan: torch.Tensor, ms, wavelet: int, f32: bool = True, u8: bool = False, stream=None):
    """Fused bands of one scene.

    pan: (H, W) uint8 or float32 CUDA tensor; ms: (B, H/2, W/2) tensor or list
    of (H/2, W/2) tensors of the same dtype.  Returns (out_f32, out_u8), each a
    (B, H, W) tensor or None.  Runs in the launch shape the autotuner cached
    for this scene class (tune.tune_fuse), if there is one.
    """
    from . import tune
    bands = _C._bands(ms)
    H, W = pan.shape
    out_f = torch.empty((len(bands), H, W), dtype=torch.float32, device=pan.device) if f32 else None
    out_u = torch.empty((len(bands), H, W), dtype=torch.uint8, device=pan.device) if u8 else None
    # The launch shape tune.tune_fuse cached for this scene class, if any (no tuning here).
    key = tune.current_device_key() + "|" + tune.fuse_class(
        H, W, len(bands), wavelet, _C._dtype_code(pan, "pan"), ("f" if f32 else "") + ("u" if u8 else ""))
    with tune.using(tune.cached(key)):
        _C.dwtfuse_fuse(pan, bands, wavelet, out_f, out_u, stream)
    return out_f, out_u
