"""Host side of the row-band split (paper_1803_00737_gb300.shard): the band
plan, the slab reading (checked with the FP64 oracle: a band's slab fused as
a scene of its own and cropped equals the band's rows of the whole-scene
fusion), and the halo exchange between ranks (gloo, world size 2 and 3, on
CPU).  No GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
from paper_1803_00737_gb300 import shard


@pytest.mark.parametrize("H,parts", [(2, 1), (16, 3), (34, 4), (100, 50), (4096, 7)])
def test_row_bands_cover_the_scene_in_even_bands(H, parts):
    b = shard.row_bands(H, parts)
    assert b[0][0] == 0 and b[-1][1] == H and len(b) == parts
    assert all(y1 == b[k + 1][0] for k, (_, y1) in enumerate(b[:-1]))
    sizes = [y1 - y0 for y0, y1 in b]
    assert all(s >= 2 and s % 2 == 0 for s in sizes) and max(sizes) - min(sizes) <= 2


def test_row_bands_rejects_impossible_splits():
    for H, parts in [(15, 2), (8, 5), (8, 0)]:
        with pytest.raises(ValueError):
            shard.row_bands(H, parts)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape,parts", [((16, 20), 3), ((34, 18), 4), ((12, 10), 6), ((8, 12), 1)])
def test_slab_fused_as_a_scene_gives_the_band_rows(wav, shape, parts):
    """The reading dwtfuse_fuse_rows relies on: with 2 PAN rows and 1 MS row
    of halo above and 2 PAN rows below (D4), the slab fused as a scene of its
    own (one more MS row of any value appended, which only touches rows that
    are cropped) has, past its halo, the band's rows of the whole-scene
    fusion; the periodic wrap of Eq. 5-6 and 13-14 enters through the halo
    rows taken mod H."""
    H, W = shape
    rng = np.random.default_rng(H * W + parts)
    pan = rng.integers(0, 256, (H, W)).astype(float)
    ms = rng.integers(0, 256, (2, H // 2, W // 2)).astype(float)
    whole = O.fuse(pan, ms, wav)
    h, _ = (2, 1) if wav == O.D4 else (0, 0)
    for y0, y1 in shard.row_bands(H, parts):
        pr, mr = shard.slab_rows(H, y0, y1, wav)
        ps, mss = pan[pr], ms[:, mr]
        if wav == O.D4:
            mss = np.concatenate([mss, rng.integers(0, 256, (2, 1, W // 2)).astype(float)], axis=1)
        got = O.fuse(ps, mss, wav)[:, h:h + (y1 - y0)]
        assert np.abs(got - whole[:, y0:y1]).max() < 1e-11, (y0, y1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene(H, W, B, seed):
    g = torch.Generator().manual_seed(seed)
    pan = torch.randint(0, 256, (H, W), generator=g, dtype=torch.uint8)
    ms = torch.randint(0, 256, (B, H // 2, W // 2), generator=g, dtype=torch.uint8)
    return pan, ms


def _rank(rank, world, port, q, H, W, B, wav):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pan, ms = _scene(H, W, B, seed=5)
        y0, y1 = shard.row_bands(H, world)[rank]
        ps, mss = shard.exchange_halo(pan[y0:y1].clone(), ms[:, y0 // 2:y1 // 2].clone(), wav)
        rp, rm = shard.make_slab(pan, ms, y0, y1, wav)
        q.put((rank, bool(torch.equal(ps, rp)), bool(torch.equal(mss, rm))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_halo_exchange_builds_the_slabs_gloo(world, wav):
    """Each rank holds only its band's rows; after exchange_halo its slab
    equals the one gathered from the whole scene (wrap seam included)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    H, W, B = 22, 18, 3
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, H, W, B, wav)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert got == [(r, True, True) for r in range(world)]


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_single_part_slab_wraps_onto_itself(wav):
    pan, ms = _scene(10, 14, 2, seed=1)
    ps, mss = shard.exchange_halo(pan, ms, wav)
    rp, rm = shard.make_slab(pan, ms, 0, 10, wav)
    assert torch.equal(ps, rp) and torch.equal(mss, rm)
