"""dwtfuse_fuse_rows: a scene fused as row bands, each from a slab carrying
its halo rows, against the whole-scene call (bit for bit: the same kernel
arithmetic on the same values) and against the FP64 oracle (Haar exact, D4
5e-4 max-abs).  Splits into 1 to 5 bands of uneven heights, bands of a
single MS row, both wavelets, widths W = 0 and 2 mod 4 and off the strip
grid, 1 to 9 MS bands (two band chunks), uint8 and float inputs."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from paper_1803_00737_gb300 import _C, fuse, shard

pytestmark = pytest.mark.gpu
DEV = "cuda"


def fused_by_bands(pan, ms, wav, parts, f32=True, u8=True):
    H, W = pan.shape
    B = ms.shape[0]
    of = torch.empty((B, H, W), device=DEV) if f32 else None
    ou = torch.empty((B, H, W), dtype=torch.uint8, device=DEV) if u8 else None
    for y0, y1 in shard.row_bands(H, parts):
        ps, mss = shard.make_slab(pan, ms, y0, y1, wav)
        bf, bu = shard.fuse_band(ps, mss, wav, H, y0, y1, f32=f32, u8=u8)
        if f32:
            of[:, y0:y1] = bf
        if u8:
            ou[:, y0:y1] = bu
    return of, ou


CASES = [((64, 136), 3, 2), ((66, 258), 4, 3), ((130, 250), 9, 5), ((12, 814), 1, 6), ((4, 4), 2, 2),
         ((200, 384), 6, 4), ((1030, 196), 8, 3)]


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape,B,parts", CASES)
def test_bands_equal_whole_scene_and_oracle(wav, shape, B, parts):
    H, W = shape
    pan, ms = scenegen.make_scene(H, W, B, seed=H + W)
    pd, md = pan.to(DEV), ms.to(DEV)
    of, ou = fused_by_bands(pd, md, wav, parts)
    wf, wu = fuse(pd, md, wav, f32=True, u8=True)
    torch.cuda.synchronize()
    assert torch.equal(of, wf) and torch.equal(ou, wu)
    ref = O.fuse(pan.numpy().astype(np.float64), ms.numpy().astype(np.float64), wav)
    err = np.abs(of.cpu().numpy().astype(np.float64) - ref).max()
    assert err <= (0.0 if wav == O.HAAR else 5e-4), err


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_float_inputs_and_single_output(wav):
    H, W = 96, 130
    rng = np.random.default_rng(3)
    pan = torch.from_numpy(rng.uniform(0, 255, (H, W)).astype(np.float32)).to(DEV)
    ms = torch.from_numpy(rng.uniform(0, 255, (5, H // 2, W // 2)).astype(np.float32)).to(DEV)
    of, _ = fused_by_bands(pan, ms, wav, 4, u8=False)
    _, ou = fused_by_bands(pan, ms, wav, 3, f32=False)
    wf, wu = fuse(pan, ms, wav, f32=True, u8=True)
    torch.cuda.synchronize()
    assert torch.equal(of, wf) and torch.equal(ou, wu)


def test_full_size_four_bands():
    """The benchmark scene (D4, 16384^2, 6 bands) fused as 4 row bands equals
    the whole-scene call bit for bit."""
    H = W = 16384
    pan, ms = scenegen.make_scene(H, W, 6, seed=0, blob_scale=16.0, device=DEV)
    wf, _ = fuse(pan, ms, O.D4)
    for y0, y1 in shard.row_bands(H, 4):
        ps, mss = shard.make_slab(pan, ms, y0, y1, O.D4)
        bf, _ = shard.fuse_band(ps, mss, O.D4, H, y0, y1)
        assert torch.equal(bf, wf[:, y0:y1]), (y0, y1)


def test_rejects_bad_row_ranges():
    pan = torch.zeros((10, 8), dtype=torch.uint8, device=DEV)
    ms = torch.zeros((1, 5, 4), dtype=torch.uint8, device=DEV)
    out = torch.empty((1, 6, 8), device=DEV)
    L = _C.lib()
    import ctypes
    ptrs = (ctypes.c_void_p * 1)(ms.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for y0, y1 in [(1, 7), (0, 7), (4, 2), (-2, 4), (16, 22)]:
        st = L.dwtfuse_fuse_rows(ctypes.c_void_p(pan.data_ptr()), ptrs, 1, 16, 8, y0, y1, O.D4, _C.U8,
                                 ctypes.c_void_p(out.data_ptr()), None, s)
        assert st == _C.ESHAPE, (y0, y1, st)
    with pytest.raises(ValueError):
        _C.dwtfuse_fuse_rows(pan[:8], ms, O.D4, 16, 0, 6, out, None)
