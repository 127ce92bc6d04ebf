"""Element-wise parity on windows of images too large for the whole-image
oracle: seeded square windows plus the rows and columns where the periodic
wrap of Eq. 5-6 and 13-14 acts (the first and last two of each), compared
pixel by pixel with the oracle's point-wise evaluators.

A region is (y0, h, x0, w) in PAN pixels: rows (y0 + r) % H, r < h, and
columns (x0 + s) % W, s < w, with y0, x0, h, w even.  Gradients and images
are gathered from the device by index, so only the windows (plus a 4-pixel
margin, the reach of a D4 tap chain) travel to the host.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle as O

MARGIN = 4


def regions(H: int, W: int, seed: int, n_windows: int = 2, side: int = 256):
    """Seeded side x side windows, the wrap rows H-2..1 over the whole width,
    and the wrap columns W-2..1 over the whole height."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_windows):
        y0 = 2 * int(rng.integers(0, H // 2))
        x0 = 2 * int(rng.integers(0, W // 2))
        out.append((y0, min(side, H), x0, min(side, W)))
    out.append((H - 2, 4, 0, W))
    out.append((0, H, W - 2, 4))
    return out


def _idx(start: int, n: int, N: int, device) -> torch.Tensor:
    return torch.from_numpy((start + np.arange(n)) % N).to(device)


def gather(t: torch.Tensor, y0: int, h: int, x0: int, w: int) -> np.ndarray:
    """Rows (y0 + r) % H and columns (x0 + s) % W of the last two dimensions
    of a device tensor, as a float64 (or uint8) host array."""
    H, W = t.shape[-2:]
    sub = t.index_select(-2, _idx(y0, h, H, t.device)).index_select(-1, _idx(x0, w, W, t.device))
    a = sub.cpu().numpy()
    return a if a.dtype == np.uint8 else a.astype(np.float64)


def _padded(y0, h, N):
    """A span widened by MARGIN on both sides, or the whole axis if that covers it."""
    if h + 2 * MARGIN >= N:
        return 0, N
    return y0 - MARGIN, h + 2 * MARGIN


def adjoint_region_error(G: torch.Tensor, gp: torch.Tensor, gm: torch.Tensor, wavelet: int, region) -> float:
    """max |GPU - oracle| over a region of grad_PAN (every pixel) and of every
    band's grad_MS (the region halved), relative to max(1, max |oracle|).
    G (B, H, W) is the output gradient, gp (H, W) and gm (B, H/2, W/2) the
    GPU's gradients."""
    B, H, W = G.shape
    y0, h, x0, w = region
    gy0, hg = _padded(y0, h, H)
    gx0, wg = _padded(x0, w, W)
    gwin = gather(G, gy0, hg, gx0, wg)
    ys = (y0 + np.arange(h)) % H
    xs = (x0 + np.arange(w)) % W
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    iis = (y0 // 2 + np.arange(h // 2)) % (H // 2)
    jjs = (x0 // 2 + np.arange(w // 2)) % (W // 2)
    ii, jj = np.meshgrid(iis, jjs, indexing="ij")
    rp, rm = O.fuse_adjoint_points(gwin, wavelet, H, W, yy.ravel(), xx.ravel(), ii.ravel(), jj.ravel(),
                                   gy0=gy0 % H, gx0=gx0 % W)
    got_p = gather(gp, y0, h, x0, w).ravel()
    got_m = gather(gm, y0 // 2, h // 2, x0 // 2, w // 2).reshape(B, -1)
    scale = max(1.0, float(np.abs(rp).max()), float(np.abs(rm).max()))
    return max(float(np.abs(got_p - rp).max()), float(np.abs(got_m - rm).max())) / scale


def forward_region_error(pan_h: np.ndarray, ms_h: np.ndarray, out: torch.Tensor, wavelet: int, region,
                         bands) -> float:
    """max |GPU - oracle| of the fused float32 bands `bands` over a region
    (pan_h, ms_h: the whole inputs on the host)."""
    H, W = pan_h.shape
    y0, h, x0, w = region
    ys = (y0 + np.arange(h)) % H
    xs = (x0 + np.arange(w)) % W
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    err = 0.0
    for b in bands:
        ref = O.fuse_points(pan_h, ms_h[b], wavelet, yy.ravel(), xx.ravel())
        got = gather(out[b], y0, h, x0, w).ravel()
        err = max(err, float(np.abs(got - ref).max()))
    return err
