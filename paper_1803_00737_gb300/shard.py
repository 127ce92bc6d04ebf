"""Row-band split of one scene: each part fuses its own PAN rows after
receiving its halo rows from its neighbours.

The paper (Sec. 3) splits the source image among the nodes of a cluster and
merges separately fused parts.  With the periodic wrap of Eq. 5-6 and 13-14
a Daubechies-4 part needs rows of its neighbours (2 PAN rows above and below,
1 MS row above; the first and last parts are neighbours through the wrap),
so a plain merge of parts is wrong at the seams.  Here a part's slab carries
those rows, and dwtfuse_fuse_rows turns it into exactly the part's rows of
the whole-scene result.  Haar needs no halo.

Three pieces, all host-side bookkeeping (every pixel is computed by the
library's kernel):
  row_bands    splits the H/2 MS rows of a scene evenly into parts;
  make_slab    gathers a part's slab from a whole scene held on one device
               (parts fused one after another to bound memory, or tests);
  exchange_halo  builds a part's slab from its own rows when the parts live
               on different ranks of a torch.distributed group: each rank
               sends its first PAN rows up the ring and its last PAN and MS
               rows down it (point-to-point, gloo or NCCL).
"""
from __future__ import annotations

import torch

from . import _C


def row_bands(H: int, parts: int) -> list[tuple[int, int]]:
    """PAN row ranges [y0, y1) of `parts` bands covering an H-row scene: the
    H/2 MS rows split as evenly as possible, so every band has an even number
    of at least 2 rows."""
    H2 = H // 2
    if H % 2 or parts < 1 or parts > H2:
        raise ValueError(f"cannot split {H} rows into {parts} even bands")
    return [(2 * (k * H2 // parts), 2 * ((k + 1) * H2 // parts)) for k in range(parts)]


def slab_rows(H: int, y0: int, y1: int, wavelet: int) -> tuple[list[int], list[int]]:
    """Whole-scene indices of a band's slab rows: PAN rows y0 - h .. y1 + h - 1
    and MS rows y0/2 - hm .. y1/2 - 1, each taken mod the scene's height."""
    h, hm = _C.row_halo(wavelet)
    H2 = H // 2
    pan = [(y % H) for y in range(y0 - h, y1 + h)]
    ms = [(m % H2) for m in range(y0 // 2 - hm, y1 // 2)]
    return pan, ms


def make_slab(pan: torch.Tensor, ms: torch.Tensor, y0: int, y1: int, wavelet: int):
    """(pan_slab, ms_slab) of band [y0, y1) from a whole scene pan (H, W) and
    ms (B, H/2, W/2) on one device."""
    H = pan.shape[0]
    pr, mr = slab_rows(H, y0, y1, wavelet)
    pi = torch.tensor(pr, dtype=torch.long, device=pan.device)
    mi = torch.tensor(mr, dtype=torch.long, device=ms.device)
    return pan.index_select(0, pi).contiguous(), ms.index_select(1, mi).contiguous()


# Message tags of the two halos (gloo matches on them; NCCL matches the
# point-to-point operations between two ranks in the order they are posted,
# which is the same order on every rank).
_TAG_DOWN, _TAG_UP = 17, 18


def exchange_halo(pan_band: torch.Tensor, ms_band: torch.Tensor, wavelet: int, group=None):
    """Slab of this rank's band from its own rows: pan_band (y1 - y0, W) and
    ms_band (B, (y1 - y0)/2, W/2), rank r holding the r-th band of
    row_bands(H, world) (the ring wraps from the last rank to the first, as
    the image does).  Returns (pan_slab, ms_slab) for dwtfuse_fuse_rows."""
    import torch.distributed as dist
    h, hm = _C.row_halo(wavelet)
    if h == 0:
        return pan_band.contiguous(), ms_band.contiguous()
    n, W = pan_band.shape
    B, n2, W2 = ms_band.shape
    if n < h or n2 < hm or n2 * 2 != n:
        raise ValueError("a band needs at least 2 PAN rows and matching MS rows")
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        top = pan_band[n - h:]
        bottom = pan_band[:h]
        ms_top = ms_band[:, n2 - hm:]
    else:
        rank = dist.get_rank(group)
        up = dist.get_global_rank(group, (rank - 1) % world) if group is not None else (rank - 1) % world
        down = dist.get_global_rank(group, (rank + 1) % world) if group is not None else (rank + 1) % world
        # To the rank below: this band's last PAN rows and last MS row (its top halo).
        send_down = torch.cat([pan_band[n - h:].reshape(-1), ms_band[:, n2 - hm:].reshape(-1)])
        # To the rank above: this band's first PAN rows (its bottom halo).
        send_up = pan_band[:h].reshape(-1).contiguous()
        recv_top = torch.empty(h * W + B * hm * W2, dtype=pan_band.dtype, device=pan_band.device)
        recv_bottom = torch.empty(h * W, dtype=pan_band.dtype, device=pan_band.device)
        ops = [dist.P2POp(dist.isend, send_down, down, group, _TAG_DOWN),
               dist.P2POp(dist.isend, send_up, up, group, _TAG_UP),
               dist.P2POp(dist.irecv, recv_top, up, group, _TAG_DOWN),
               dist.P2POp(dist.irecv, recv_bottom, down, group, _TAG_UP)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        top = recv_top[:h * W].view(h, W)
        ms_top = recv_top[h * W:].view(B, hm, W2)
        bottom = recv_bottom.view(h, W)
    pan_slab = torch.cat([top, pan_band, bottom], dim=0).contiguous()
    ms_slab = torch.cat([ms_top, ms_band], dim=1).contiguous()
    return pan_slab, ms_slab


def fuse_band(pan_slab: torch.Tensor, ms_slab: torch.Tensor, wavelet: int, H: int, y0: int, y1: int,
              f32: bool = True, u8: bool = False, stream=None):
    """Fused rows [y0, y1) of an H-row scene from its slab: (out_f32, out_u8),
    each (B, y1 - y0, W) or None."""
    B, W = ms_slab.shape[0], pan_slab.shape[1]
    n = y1 - y0
    out_f = torch.empty((B, n, W), dtype=torch.float32, device=pan_slab.device) if f32 else None
    out_u = torch.empty((B, n, W), dtype=torch.uint8, device=pan_slab.device) if u8 else None
    _C.dwtfuse_fuse_rows(pan_slab, ms_slab, wavelet, H, y0, y1, out_f, out_u, stream)
    return out_f, out_u
