"""Seeded synthetic Landsat-7-shaped scenes (8-bit PAN and half-resolution MS).

Shared input generator: the tests, the smoke check and the benchmark use it to
feed both the CUDA path and the oracle.  It holds none of the fusion method's
arithmetic (no wavelet, no LL replacement); the 2 x 2 block mean below only
simulates a sensor of half the PAN resolution.

Recipe (stand-in for the paper's Landsat 7 scenes, which are not available):
  PAN  = clip(round(128 + 40 * F + 30 * sum_k a_k G_k), 0, 255), uint8, where
         F is a Gaussian random field with power spectrum ~ f^-1.8 (DC removed,
         unit std) and G_k are 20 Gaussian blobs with centres uniform over the
         image, sigma ~ U(8, 40) * blob_scale px and amplitude a_k = +-1.
  MS_b = clip(round(g_b * blockmean2x2(PAN) + 6 * N_b), 0, 255), uint8, where
         g_b ~ U(0.6, 1.2) and N_b is white noise blurred by a periodic
         Gaussian of sigma 16 MS px, renormalised to unit std.
  round() is half to even.  Randomness comes from a torch.Generator seeded with
  `seed` on the target device (CPU and CUDA streams differ, so a scene is
  reproducible per device).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

HAAR = 0
D4 = 1


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _pink_field(h: int, w: int, gen, device, beta: float = 1.8) -> torch.Tensor:
    white = torch.randn((h, w), generator=gen, device=device, dtype=torch.float32)
    spec = torch.fft.rfft2(white)
    del white
    fy = torch.fft.fftfreq(h, device=device).view(h, 1)
    fx = torch.fft.rfftfreq(w, device=device).view(1, w // 2 + 1)
    f2 = fy * fy + fx * fx
    f2[0, 0] = 1.0
    amp = f2.pow_(-beta / 4.0)  # |F| ~ f^(-beta/2), power ~ f^-beta
    amp[0, 0] = 0.0
    spec.mul_(amp)
    del amp
    field = torch.fft.irfft2(spec, s=(h, w))
    del spec
    field.sub_(field.mean())
    field.div_(field.std().clamp_min(1e-12))
    return field


def _blobs(h: int, w: int, gen, device, n: int, scale: float) -> torch.Tensor:
    p = torch.rand((n, 4), generator=gen, device=device, dtype=torch.float64).cpu()
    ys = torch.arange(h, device=device, dtype=torch.float32)
    xs = torch.arange(w, device=device, dtype=torch.float32)
    out = torch.zeros((h, w), device=device, dtype=torch.float32)
    for k in range(n):
        cy, cx = float(p[k, 0]) * h, float(p[k, 1]) * w
        sig = (8.0 + 32.0 * float(p[k, 2])) * scale
        amp = 1.0 if float(p[k, 3]) < 0.5 else -1.0
        gy = torch.exp(-((ys - cy) ** 2) / (2 * sig * sig))
        gx = torch.exp(-((xs - cx) ** 2) / (2 * sig * sig))
        out.addr_(gy, gx, alpha=amp)
    return out


def _smooth_noise(h: int, w: int, gen, device, sigma: float = 16.0) -> torch.Tensor:
    white = torch.randn((h, w), generator=gen, device=device, dtype=torch.float32)
    spec = torch.fft.rfft2(white)
    fy = torch.fft.fftfreq(h, device=device).view(h, 1)
    fx = torch.fft.rfftfreq(w, device=device).view(1, w // 2 + 1)
    spec.mul_(torch.exp(-2.0 * math.pi ** 2 * sigma ** 2 * (fy * fy + fx * fx)))
    out = torch.fft.irfft2(spec, s=(h, w))
    out.sub_(out.mean())
    out.div_(out.std().clamp_min(1e-12))
    return out


def make_pan(H: int, W: int, seed: int, blob_scale: float = 1.0, device="cpu",
             n_blobs: int = 20) -> torch.Tensor:
    """uint8 PAN image (H, W)."""
    gen = _gen(seed, device)
    img = _pink_field(H, W, gen, device).mul_(40.0)
    img.add_(_blobs(H, W, gen, device, n_blobs, blob_scale), alpha=30.0)
    img.add_(128.0)
    return img.round_().clamp_(0, 255).to(torch.uint8)


def make_ms(pan: torch.Tensor, bands: int, seed: int) -> torch.Tensor:
    """uint8 MS bands (B, H/2, W/2) simulated from a PAN image."""
    device = pan.device
    H, W = pan.shape
    gen = _gen(seed + 7919, device)
    gains = 0.6 + 0.6 * torch.rand((bands,), generator=gen, device=device, dtype=torch.float64)
    base = torch.nn.functional.avg_pool2d(pan.float().view(1, 1, H, W), 2).view(H // 2, W // 2)
    out = torch.empty((bands, H // 2, W // 2), dtype=torch.uint8, device=device)
    for b in range(bands):
        v = base * float(gains[b]) + 6.0 * _smooth_noise(H // 2, W // 2, gen, device)
        out[b] = v.round_().clamp_(0, 255).to(torch.uint8)
    return out


def make_scene(H: int, W: int, bands: int, seed: int, blob_scale: float = 1.0, device="cpu"):
    """(pan uint8 (H, W), ms uint8 (B, H/2, W/2)) on `device`."""
    if H % 2 or W % 2:
        raise ValueError("PAN sides must be even")
    pan = make_pan(H, W, seed, blob_scale, device)
    return pan, make_ms(pan, bands, seed)


@dataclass(frozen=True)
class SceneSpec:
    H: int
    W: int
    bands: int
    wavelet: int
    seed: int


def batch_specs(n: int = 96, seed: int = 0, lo: int = 256, hi: int = 8192, bands=(3, 8),
                wavelets=(HAAR, D4), square: bool = False) -> list[SceneSpec]:
    """Scene shapes of an uneven batch: even sides U[lo, hi] (independent H, W
    unless square), band counts U[bands], wavelet drawn from `wavelets`; scene i
    gets seed 1000 * seed + i."""
    g = _gen(seed, "cpu")
    specs = []
    for i in range(n):
        r = torch.randint(0, 1 << 30, (4,), generator=g).tolist()
        H = lo + 2 * (r[0] % ((hi - lo) // 2 + 1))
        W = H if square else lo + 2 * (r[1] % ((hi - lo) // 2 + 1))
        B = bands[0] + r[2] % (bands[1] - bands[0] + 1)
        wav = wavelets[r[3] % len(wavelets)]
        specs.append(SceneSpec(H, W, B, wav, 1000 * seed + i))
    return specs


def target_like(shape, seed: int, device="cpu") -> torch.Tensor:
    """Seeded float32 noise of a given shape (regression targets, gradients)."""
    gen = _gen(seed, device)
    return torch.randn(shape, generator=gen, device=device, dtype=torch.float32)
