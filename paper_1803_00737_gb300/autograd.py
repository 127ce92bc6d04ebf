"""Differentiable fusion: torch.autograd.Function over the forward and adjoint
kernels of libdwtfuse.

The fusion is linear in (PAN, MS), so the backward needs no saved
activations: it applies the transpose of the fused map (dwtfuse_fuse_backward)
to the incoming gradient.  Only shapes and the wavelet are kept in ctx.
"""
from __future__ import annotations

import torch

from . import _C, tune


def _shape(key: str, run_tuner) -> "tune.LaunchShape | None":
    """The tuned launch shape for a key: from the cache, else tuned now (once
    per machine and shape class), else None when tuning is not allowed (inside
    a graph capture, or DWTFUSE_AUTOTUNE=0)."""
    got = tune.cached(key)
    if got is None and tune.tuning_allowed():
        got = run_tuner()
    return got


def fuse_batch(P: torch.Tensor, M: torch.Tensor, wavelet: int, out: torch.Tensor) -> None:
    """Float forward of a batch: P (N, H, W), M (N, B, H/2, W/2), out (N, B, H, W).
    Batches go through the batched persistent kernel (one launch per up to
    DWTFUSE_MAX_SCENES scenes, its workspace from torch's allocator) in the
    launch shape the autotuner picked for this batch shape; a single scene, or
    more than 8 bands, through dwtfuse_fuse."""
    N, B = M.shape[0], M.shape[1]
    if N == 1 or B > 8:
        for i in range(N):
            _C.dwtfuse_fuse(P[i], M[i], wavelet, out[i], None)
        return
    ws = torch.empty(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=P.device)
    for i0 in range(0, N, _C.MAX_SCENES):
        idx = range(i0, min(N, i0 + _C.MAX_SCENES))
        scenes = [_C.make_scene(P[i], M[i], wavelet, out[i], None) for i in idx]
        specs = [(P.shape[1], P.shape[2], B, wavelet)] * len(idx)
        shape = _shape(tune.current_device_key() + "|" + tune.batched_class(specs),
                       lambda: tune.tune_batched(scenes, specs, ws))
        rows, blocks = (shape.rows_per_item, shape.blocks_per_sm) if shape else (0, 0)
        with tune.using(tune.LaunchShape(0, 0, shape.fwd_chunk, 0) if shape else None):
            _C.dwtfuse_fuse_batched(scenes, ws, rows, blocks)


def fuse_batch_backward(g: torch.Tensor, wavelet: int, gp: torch.Tensor, gm: torch.Tensor) -> None:
    """Adjoint of a batch: g (N, B, H, W) into gp (N, H, W) and gm (N, B, H/2, W/2).
    Batches go through the batched adjoint (one persistent launch per band
    chunk over up to DWTFUSE_MAX_SCENES scenes) in the launch shape the
    autotuner picked for this batch shape; a single scene through
    dwtfuse_fuse_backward."""
    N = g.shape[0]
    if N == 1:
        _C.dwtfuse_fuse_backward(g[0], wavelet, gp[0], gm[0])
        return
    N_, B, H, W = g.shape
    shape = _shape(tune.current_device_key() + "|" + tune.backward_class(N, H, W, B, wavelet),
                   lambda: tune.tune_backward(g, wavelet, gp, gm))
    ws = torch.empty(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=g.device)
    with tune.using(shape):
        for i0 in range(0, N, _C.MAX_SCENES):
            scenes = [_C.make_grad_scene(g[i], wavelet, gp[i], gm[i])
                      for i in range(i0, min(N, i0 + _C.MAX_SCENES))]
            _C.dwtfuse_fuse_backward_batched(scenes, ws)


class DWTFuseFn(torch.autograd.Function):
    """fused = DWTFuseFn.apply(pan, ms, wavelet)

    pan: (N, H, W) or (H, W) float32 CUDA; ms: (N, B, H/2, W/2) or (B, H/2, W/2)
    float32 CUDA.  Returns (N, B, H, W) or (B, H, W) float32.
    """

    @staticmethod
    def forward(ctx, pan: torch.Tensor, ms: torch.Tensor, wavelet: int):
        batched = pan.dim() == 3
        P = pan if batched else pan.unsqueeze(0)
        M = ms if batched else ms.unsqueeze(0)
        P = P.contiguous()
        M = M.contiguous()
        N, H, W = P.shape
        B = M.shape[1]
        if M.shape != (N, B, H // 2, W // 2):
            raise ValueError("ms must be (N, B, H/2, W/2) matching pan (N, H, W)")
        out = torch.empty((N, B, H, W), dtype=torch.float32, device=P.device)
        fuse_batch(P, M, wavelet, out)
        ctx.wavelet = int(wavelet)
        ctx.batched = batched
        ctx.shape = (N, B, H, W)
        return out if batched else out[0]

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        N, B, H, W = ctx.shape
        g = (grad if ctx.batched else grad.unsqueeze(0)).contiguous().float()
        gp = torch.empty((N, H, W), dtype=torch.float32, device=g.device)
        gm = torch.empty((N, B, H // 2, W // 2), dtype=torch.float32, device=g.device)
        fuse_batch_backward(g, ctx.wavelet, gp, gm)
        if not ctx.batched:
            gp, gm = gp[0], gm[0]
        return gp, gm, None


def dwt_fuse(pan: torch.Tensor, ms: torch.Tensor, wavelet: int) -> torch.Tensor:
    return DWTFuseFn.apply(pan, ms, wavelet)
