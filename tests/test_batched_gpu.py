"""Batched persistent fusion: one launch over scenes of uneven sizes, band
counts, wavelets and input types equals the single-scene path bit for bit, and
the oracle within the single-scene bars; it replays from a captured CUDA graph
deterministically."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from paper_1803_00737_gb300 import _C, fuse

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _make(specs, f32_every=0):
    scenes, keep = [], []
    for i, sp in enumerate(specs):
        rng = np.random.default_rng(sp.seed)
        pan = torch.from_numpy(rng.integers(0, 256, (sp.H, sp.W)).astype(np.uint8)).to(DEV)
        ms = torch.from_numpy(rng.integers(0, 256, (sp.bands, sp.H // 2, sp.W // 2))
                              .astype(np.uint8)).to(DEV)
        if f32_every and i % f32_every == 0:
            pan, ms = pan.float(), ms.float()
        out = torch.full((sp.bands, sp.H, sp.W), float("nan"), device=DEV)
        out8 = torch.zeros((sp.bands, sp.H, sp.W), dtype=torch.uint8, device=DEV)
        scenes.append(_C.make_scene(pan, ms, sp.wavelet, out, out8))
        keep.append((sp, pan, ms, out, out8))
    return scenes, keep


def _workspace():
    return torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=DEV)


def test_batched_equals_single_scene_and_oracle():
    specs = scenegen.batch_specs(n=14, seed=3, lo=4, hi=300)
    scenes, keep = _make(specs, f32_every=3)
    ws = _workspace()
    _C.dwtfuse_fuse_batched(scenes, ws)
    torch.cuda.synchronize()
    assert _C.dwtfuse_get_last_device_status(ws) == _C.OK
    for sp, pan, ms, out, out8 in keep:
        f, u = fuse(pan, ms, sp.wavelet, f32=True, u8=True)
        torch.cuda.synchronize()
        assert torch.equal(out, f), sp
        assert torch.equal(out8, u), sp
        ref = O.fuse(pan.cpu().numpy().astype(np.float64), ms.cpu().numpy().astype(np.float64),
                     sp.wavelet)
        err = np.abs(out.cpu().numpy() - ref).max()
        assert err <= (0 if sp.wavelet == O.HAAR else 5e-4), (sp, err)


@pytest.mark.parametrize("rows,bps", [(1, 1), (8, 0), (64, 2)])
def test_batched_launch_shapes(rows, bps):
    specs = scenegen.batch_specs(n=6, seed=5, lo=8, hi=200)
    scenes, keep = _make(specs)
    ws = _workspace()
    _C.dwtfuse_fuse_batched(scenes, ws, rows_per_item=rows, blocks_per_sm=bps)
    torch.cuda.synchronize()
    for sp, pan, ms, out, _ in keep:
        f, _ = fuse(pan, ms, sp.wavelet)
        assert torch.equal(out, f)


def test_batched_graph_capture_and_replay():
    specs = scenegen.batch_specs(n=9, seed=8, lo=16, hi=400)
    scenes, keep = _make(specs)
    ws = _workspace()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        _C.dwtfuse_fuse_batched(scenes, ws, stream=s)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = [k[3].clone() for k in keep]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        _C.dwtfuse_fuse_batched(scenes, ws)
    for _ in range(3):
        for k in keep:
            k[3].fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for k, f0 in zip(keep, first):
            assert torch.equal(k[3], f0)
    assert _C.dwtfuse_get_last_device_status(ws) == _C.OK


def test_batched_uneven_config_full_size():
    """96 scenes, independent even sides U[256, 8192], 3-8 bands, Haar/D4 mixed,
    uint8 inputs generated by the scene recipe, one persistent launch: every
    scene equals the single-scene kernel bit for bit; sampled pixels of every
    scene match the point-wise oracle."""
    specs = scenegen.batch_specs(n=96, seed=0)
    scenes, keep = [], []
    for sp in specs:
        pan, ms = scenegen.make_scene(sp.H, sp.W, sp.bands, seed=sp.seed, device=DEV)
        out = torch.empty((sp.bands, sp.H, sp.W), device=DEV)
        scenes.append(_C.make_scene(pan, ms, sp.wavelet, out, None))
        keep.append((sp, pan, ms, out))
    ws = _workspace()
    _C.dwtfuse_fuse_batched(scenes, ws)
    torch.cuda.synchronize()
    assert _C.dwtfuse_get_last_device_status(ws) == _C.OK
    rng = np.random.default_rng(0)
    for sp, pan, ms, out in keep:
        f, _ = fuse(pan, ms, sp.wavelet)
        assert torch.equal(out, f), sp
        del f
        ys = rng.integers(0, sp.H, 40)
        xs = rng.integers(0, sp.W, 40)
        yt, xt = torch.from_numpy(ys).to(DEV), torch.from_numpy(xs).to(DEV)
        pan_h = pan.cpu().numpy()
        b = int(rng.integers(0, sp.bands))
        ref = O.fuse_points(pan_h, ms[b].cpu().numpy(), sp.wavelet, ys, xs)
        got = out[b][yt, xt].cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= (0 if sp.wavelet == O.HAAR else 5e-4), sp


def test_batched_band_groups_and_table_capacity():
    """Scenes with W = 2 mod 4 and 7-8 bands run as two band groups (two
    table entries) while the table has room; at DWTFUSE_MAX_SCENES such
    scenes, the ones that no longer fit take the pixel-pair body.  Results
    equal the single-scene path either way."""
    specs = [scenegen.SceneSpec(6 + 2 * (i % 5), 10 + 4 * (i % 7), 7 + (i % 2), O.D4 if i % 3 else O.HAAR, 100 + i)
             for i in range(_C.MAX_SCENES)]
    assert all(sp.W % 4 == 2 for sp in specs)
    for n in (3, _C.MAX_SCENES):
        scenes, keep = _make(specs[:n])
        ws = _workspace()
        _C.dwtfuse_fuse_batched(scenes, ws)
        torch.cuda.synchronize()
        assert _C.dwtfuse_get_last_device_status(ws) == _C.OK
        for sp, pan, ms, out, out8 in keep:
            f, u = fuse(pan, ms, sp.wavelet, f32=True, u8=True)
            torch.cuda.synchronize()
            assert torch.equal(out, f), sp
            assert torch.equal(out8, u), sp


def test_batched_equals_staged_single_scene_and_capacity():
    """The batched launch (warp items) against the single-scene path, which
    takes the staged kernel (1024-column CTA items, float rows written by bulk
    copies) for scenes on the 16-byte grid with a float output and at most 6
    bands: the two different kernels agree bit for bit, on scenes of 1-8
    bands, W = 0 and 2 mod 4, several 1024-column strips and ragged ones, a
    uint8-only output, and a full table of 8-band scenes."""
    mix = [scenegen.SceneSpec(64, 1028, 8, O.D4, 1), scenegen.SceneSpec(66, 2052, 3, O.HAAR, 2),
           scenegen.SceneSpec(34, 1030, 7, O.D4, 3), scenegen.SceneSpec(8, 4, 1, O.D4, 4),
           scenegen.SceneSpec(130, 516, 6, O.D4, 5), scenegen.SceneSpec(12, 3000, 2, O.HAAR, 6)]
    full = [scenegen.SceneSpec(6 + 2 * (i % 4), 8 + 4 * (i % 9), 8, O.D4 if i % 3 else O.HAAR, 200 + i)
            for i in range(_C.MAX_SCENES)]
    assert all(sp.W % 4 == 0 for sp in full)
    for specs in (mix, full):
        scenes, keep = _make(specs)
        if specs is mix:  # a uint8-only scene
            sp, pan, ms, out, out8 = keep[1]
            scenes[1] = _C.make_scene(pan, ms, sp.wavelet, None, out8)
        ws = _workspace()
        _C.dwtfuse_fuse_batched(scenes, ws)
        torch.cuda.synchronize()
        assert _C.dwtfuse_get_last_device_status(ws) == _C.OK
        for i, (sp, pan, ms, out, out8) in enumerate(keep):
            f, u = fuse(pan, ms, sp.wavelet, f32=True, u8=True)
            torch.cuda.synchronize()
            if not (specs is mix and i == 1):
                assert torch.equal(out, f), sp
            assert torch.equal(out8, u), sp
