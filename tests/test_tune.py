"""Autotuner: cache keys, cache persistence and recovery, candidate choice
(host logic, no GPU), and on the GPU a tuned batched launch that reproduces
the default launch's output."""
import json

import numpy as np
import pytest

from paper_1803_00737_gb300 import tune


def test_pick_fastest_and_ties():
    c = [tune.LaunchShape(r, 0, f) for r in (8, 16, 32) for f in (0, 4)]
    t = {(8, 0): 3.0, (16, 0): 1.0, (32, 0): 1.0, (8, 4): 2.0, (16, 4): 1.5, (32, 4): 1.0}
    best, table = tune.pick(c, lambda s: t[(s.rows_per_item, s.fwd_chunk)])
    assert best == tune.LaunchShape(16, 0)
    assert table["r16b0f0g0"] == 1.0 and table["r8b0f4g0"] == 2.0 and len(table) == 6
    with pytest.raises(ValueError):
        tune.pick([], lambda s: 0.0)


def test_keys_separate_devices_and_shape_classes():
    a = tune.device_key("GB300", 152, (10, 3), 13000)
    b = tune.device_key("GB300", 148, (10, 3), 13000)
    assert a != b
    s1 = tune.batched_class([(1024, 1024, 4, 1)] * 10)
    s2 = tune.batched_class([(1024, 1024, 4, 1)] * 100)
    s3 = tune.batched_class([(1024, 1024, 4, 0)] * 10)
    assert len({s1, s2, s3}) == 3
    assert tune.fuse_class(512, 512, 3, 0, 0, "fu") != tune.fuse_class(512, 512, 3, 1, 0, "fu")


def test_cache_round_trip_and_reuse(tmp_path):
    path = str(tmp_path / "t.json")
    calls = []

    def run():
        calls.append(1)
        return tune.LaunchShape(24, 0, 6, 4), {"r24b0f6g4": 0.5}

    assert tune.cached("k", path) is None
    assert tune.cached_or_tune("k", run, path) == tune.LaunchShape(24, 0, 6, 4)
    assert tune.cached_or_tune("k", run, path) == tune.LaunchShape(24, 0, 6, 4)
    assert tune.cached("k", path) == tune.LaunchShape(24, 0, 6, 4)
    assert len(calls) == 1
    data = json.load(open(path))
    assert data["entries"]["k"]["times_ms"] == {"r24b0f6g4": 0.5}
    assert tune.cached_or_tune("k", run, path, retune=True) == tune.LaunchShape(24, 0, 6, 4)
    assert len(calls) == 2


@pytest.mark.parametrize("content", ["{not json", "[]", '{"version": 1, "entries": {}}',
                                     '{"version": %d, "entries": {"k": {"rows_per_item": "x"}}}'
                                     % tune.CACHE_VERSION])
def test_corrupt_cache_is_rebuilt(tmp_path, content):
    path = tmp_path / "t.json"
    path.write_text(content)
    got = tune.cached_or_tune("k", lambda: (tune.LaunchShape(8, 0), {}), str(path))
    assert got == tune.LaunchShape(8, 0)
    assert json.load(open(path))["entries"]["k"]["rows_per_item"] == 8


def test_cache_path_env(monkeypatch, tmp_path):
    monkeypatch.setenv("DWTFUSE_TUNE_CACHE", str(tmp_path / "x.json"))
    assert tune.cache_path() == str(tmp_path / "x.json")


@pytest.mark.gpu
def test_tuned_batched_launch_matches_default(tmp_path):
    import torch

    import scenegen
    from paper_1803_00737_gb300 import _C
    specs = scenegen.batch_specs(n=6, seed=2, lo=64, hi=700)
    scenes, outs, keep = [], [], []
    for sp in specs:
        rng = np.random.default_rng(sp.seed)
        p = torch.from_numpy(rng.integers(0, 256, (sp.H, sp.W)).astype(np.uint8)).cuda()
        m = torch.from_numpy(rng.integers(0, 256, (sp.bands, sp.H // 2, sp.W // 2)).astype(np.uint8)).cuda()
        o = torch.empty((sp.bands, sp.H, sp.W), device="cuda")
        keep.append((p, m))
        outs.append(o)
        scenes.append(_C.make_scene(p, m, sp.wavelet, o, None))
    ws = torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device="cuda")
    _C.dwtfuse_fuse_batched(scenes, ws)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    shape = tune.tune_batched(scenes, [(s.H, s.W, s.bands, s.wavelet) for s in specs], ws, reps=1,
                              path=str(tmp_path / "t.json"))
    assert shape.rows_per_item in tune.ROWS and shape.blocks_per_sm in tune.BLOCKS
    assert shape.fwd_chunk in tune.FWD_CHUNKS
    # every candidate band chunk gives the default launch's bits
    for f in tune.FWD_CHUNKS:
        for o in outs:
            o.fill_(float("nan"))
        with tune.using(tune.LaunchShape(0, 0, f, 0)):
            _C.dwtfuse_fuse_batched(scenes, ws, shape.rows_per_item, shape.blocks_per_sm)
        torch.cuda.synchronize()
        for a, b in zip(outs, ref):
            assert torch.equal(a, b), f


@pytest.mark.gpu
@pytest.mark.parametrize("f,g", [(4, 4), (6, 0), (3, 2)])
def test_band_chunk_knobs_keep_results(f, g):
    """The forward is bit-identical for any band chunk; the adjoint's grad_MS
    too, and grad_PAN (chunks added in order) within FP32 rounding."""
    import torch

    import scenegen
    from paper_1803_00737_gb300 import _C
    # (the 2048-wide scenes run the staged single-scene kernel, chunked by the knob)
    for wav, (H, W), B in [(1, (64, 136), 8), (0, (66, 258), 7), (1, (130, 250), 6), (1, (34, 2048), 6),
                           (0, (20, 2048), 5)]:
        pan, ms = scenegen.make_scene(H, W, B, seed=H)
        pan, ms = pan.cuda(), ms.cuda()
        ref = torch.empty((B, H, W), device="cuda")
        _C.dwtfuse_fuse(pan, ms, wav, ref, None)
        G = scenegen.target_like((B, H, W), seed=3, device="cuda")
        gp0, gm0 = torch.empty((H, W), device="cuda"), torch.empty((B, H // 2, W // 2), device="cuda")
        _C.dwtfuse_fuse_backward(G, wav, gp0, gm0)
        with tune.using(tune.LaunchShape(0, 0, f, g)):
            got = torch.empty_like(ref)
            _C.dwtfuse_fuse(pan, ms, wav, got, None)
            gp, gm = torch.empty_like(gp0), torch.empty_like(gm0)
            _C.dwtfuse_fuse_backward(G, wav, gp, gm)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        assert torch.equal(gm, gm0)
        assert (gp - gp0).abs().max().item() <= 1e-5 * max(1.0, gp0.abs().max().item())


@pytest.mark.gpu
@pytest.mark.parametrize("g", [3, 4, 6])
def test_batched_adjoint_with_band_chunk_knob(g):
    """The batched adjoint under an adjoint band-chunk knob equals the
    single-scene adjoint under the same knob bit for bit (scenes of 1-9
    bands, chunk widths that do and do not divide them)."""
    import torch

    import scenegen
    from paper_1803_00737_gb300 import _C
    rows = []
    for i, ((H, W), B, wav) in enumerate([((64, 136), 8, 1), ((66, 258), 7, 0), ((130, 250), 9, 1),
                                          ((12, 814), 5, 1), ((96, 96), 3, 0)]):
        G = scenegen.target_like((B, H, W), seed=10 + i, device="cuda")
        rows.append((G, wav, torch.full((H, W), float("nan"), device="cuda"),
                     torch.full((B, H // 2, W // 2), float("nan"), device="cuda")))
    ws = torch.empty(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device="cuda")
    with tune.using(tune.LaunchShape(0, 0, 0, g)):
        _C.dwtfuse_fuse_backward_batched([_C.make_grad_scene(*r) for r in rows], ws)
        refs = []
        for G, wav, gp, gm in rows:
            rp, rm = torch.empty_like(gp), torch.empty_like(gm)
            _C.dwtfuse_fuse_backward(G, wav, rp, rm)
            refs.append((rp, rm))
    torch.cuda.synchronize()
    for (G, wav, gp, gm), (rp, rm) in zip(rows, refs):
        assert torch.equal(gp, rp) and torch.equal(gm, rm), (tuple(G.shape), wav)


def test_knob_validation():
    pytest.importorskip("torch")
    from paper_1803_00737_gb300 import _C
    L = _C.lib()
    assert L.dwtfuse_set_band_chunks(0, 0) == _C.OK
    for f, g in [(-1, 0), (0, 9), (9, 0)]:
        assert L.dwtfuse_set_band_chunks(f, g) == _C.EINVAL
    assert L.dwtfuse_set_band_chunks(0, 0) == _C.OK
