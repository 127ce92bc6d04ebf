"""Launch-shape autotuner with a JSON cache.

The fused kernels have two launch knobs: the number of MS rows per warp work
item (the tile height of a 128-column strip: taller items amortise the D4
prologue row, shorter ones balance the last wave) and the resident CTAs per SM
of the persistent grid.  `tune_batched` times every candidate of a batched
launch with CUDA events on the given scenes and keeps the fastest;
`tune_fuse` does the same for the single-scene forward.  Results are cached in
a JSON file keyed by GPU (name, SM count, compute capability, driver) and a
shape class, so a process pays for tuning once per machine and workload kind.

Cache location: $DWTFUSE_TUNE_CACHE, else ~/.cache/dwtfuse/tune.json.  A
missing or corrupt cache is rebuilt.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
import threading
from dataclasses import dataclass
from typing import Callable, Iterable

ROWS = (8, 16, 24, 32, 48, 64)
BLOCKS = (0, 1)  # 0 = as many CTAs per SM as fit

_lock = threading.Lock()


@dataclass(frozen=True)
class LaunchShape:
    rows_per_item: int
    blocks_per_sm: int


def cache_path() -> str:
    return os.environ.get("DWTFUSE_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "dwtfuse", "tune.json")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        if not isinstance(data, dict) or data.get("version") != 1 or not isinstance(data.get("entries"), dict):
            return {"version": 1, "entries": {}}
        return data
    except (OSError, ValueError):
        return {"version": 1, "entries": {}}


def save_cache(data: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", prefix=".tune", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def device_key(name: str, sms: int, cc: tuple[int, int], driver: int) -> str:
    return f"{name}|sm{sms}|cc{cc[0]}{cc[1]}|drv{driver}"


def current_device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    drv = torch.cuda.driver_version() if hasattr(torch.cuda, "driver_version") else 0
    return device_key(p.name, p.multi_processor_count, (p.major, p.minor), int(drv or 0))


def batched_class(specs: Iterable[tuple[int, int, int, int]]) -> str:
    """Shape class of a batched launch from (H, W, bands, wavelet) per scene:
    scene count and total fused pixels, both bucketed by powers of two, and the
    wavelet mix."""
    specs = list(specs)
    px = sum(h * w * b for h, w, b, _ in specs)
    wavs = sorted({w for *_, w in specs})
    return (f"batched|n{2 ** math.ceil(math.log2(max(1, len(specs))))}"
            f"|px2^{round(math.log2(max(1, px)))}|wav{''.join(map(str, wavs))}")


def fuse_class(H: int, W: int, bands: int, wavelet: int, in_dtype: int, outputs: str) -> str:
    return (f"fuse|wav{wavelet}|in{in_dtype}|b{bands}|{outputs}"
            f"|px2^{round(math.log2(max(1, H * W)))}")


def pick(candidates: Iterable[LaunchShape], time_ms: Callable[[LaunchShape], float]) -> tuple[LaunchShape, dict]:
    """Fastest candidate by time_ms (ties go to the earlier candidate)."""
    best, best_t, table = None, float("inf"), {}
    for c in candidates:
        t = float(time_ms(c))
        table[f"{c.rows_per_item}x{c.blocks_per_sm}"] = t
        if t < best_t:
            best, best_t = c, t
    if best is None:
        raise ValueError("no candidates")
    return best, table


def cached_or_tune(key: str, tune: Callable[[], tuple[LaunchShape, dict]], path: str | None = None,
                   retune: bool = False) -> LaunchShape:
    with _lock:
        data = load_cache(path)
        e = data["entries"].get(key)
        if e is not None and not retune:
            try:
                return LaunchShape(int(e["rows_per_item"]), int(e["blocks_per_sm"]))
            except (KeyError, TypeError, ValueError):
                pass
    best, table = tune()
    with _lock:
        data = load_cache(path)
        data["entries"][key] = {"rows_per_item": best.rows_per_item,
                                "blocks_per_sm": best.blocks_per_sm, "times_ms": table}
        save_cache(data, path)
    return best


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_batched(scenes, specs, workspace, reps: int = 3, path: str | None = None,
                 retune: bool = False) -> LaunchShape:
    """Launch shape for dwtfuse_fuse_batched over `scenes` (dwtfuse_scene
    structs); specs gives (H, W, bands, wavelet) per scene for the cache key."""
    from . import _C
    key = current_device_key() + "|" + batched_class(specs)

    def run():
        cands = [LaunchShape(r, b) for r in ROWS for b in BLOCKS]
        return pick(cands, lambda c: _time(
            lambda: _C.dwtfuse_fuse_batched(scenes, workspace, c.rows_per_item, c.blocks_per_sm), reps))

    return cached_or_tune(key, run, path, retune)


def tune_fuse(pan, ms, wavelet: int, out_f32, out_u8, reps: int = 3, path: str | None = None,
              retune: bool = False) -> LaunchShape:
    """Rows per item for dwtfuse_fuse on this scene shape; leaves the library
    knob set to the chosen value."""
    from . import _C
    bands = ms.shape[0] if hasattr(ms, "shape") else len(ms)
    outs = ("f" if out_f32 is not None else "") + ("u" if out_u8 is not None else "")
    key = current_device_key() + "|" + fuse_class(pan.shape[0], pan.shape[1], bands, wavelet,
                                                  _C._dtype_code(pan, "pan"), outs)

    def timed(c):
        _C.dwtfuse_set_rows_per_item(c.rows_per_item)
        return _time(lambda: _C.dwtfuse_fuse(pan, ms, wavelet, out_f32, out_u8), reps)

    def run():
        try:
            return pick([LaunchShape(r, 0) for r in ROWS], timed)
        finally:
            _C.dwtfuse_set_rows_per_item(0)

    best = cached_or_tune(key, run, path, retune)
    _C.dwtfuse_set_rows_per_item(best.rows_per_item)
    return best
