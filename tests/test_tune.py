"""Autotuner: cache keys, cache persistence and recovery, candidate choice
(host logic, no GPU), and on the GPU a tuned batched launch that reproduces
the default launch's output."""
import json

import numpy as np
import pytest

from paper_1803_00737_gb300 import tune


def test_pick_fastest_and_ties():
    c = [tune.LaunchShape(r, 0) for r in (8, 16, 32)]
    t = {8: 3.0, 16: 1.0, 32: 1.0}
    best, table = tune.pick(c, lambda s: t[s.rows_per_item])
    assert best == tune.LaunchShape(16, 0)
    assert table == {"8x0": 3.0, "16x0": 1.0, "32x0": 1.0}
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
        return tune.LaunchShape(24, 1), {"24x1": 0.5}

    assert tune.cached_or_tune("k", run, path) == tune.LaunchShape(24, 1)
    assert tune.cached_or_tune("k", run, path) == tune.LaunchShape(24, 1)
    assert len(calls) == 1
    data = json.load(open(path))
    assert data["entries"]["k"]["times_ms"] == {"24x1": 0.5}
    assert tune.cached_or_tune("k", run, path, retune=True) == tune.LaunchShape(24, 1)
    assert len(calls) == 2


@pytest.mark.parametrize("content", ["{not json", "[]", '{"version": 2, "entries": {}}',
                                     '{"version": 1, "entries": {"k": {"rows_per_item": "x"}}}'])
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
    for o in outs:
        o.fill_(float("nan"))
    _C.dwtfuse_fuse_batched(scenes, ws, shape.rows_per_item, shape.blocks_per_sm)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
