"""Launch-shape autotuner with a JSON cache.

Knobs of the fused kernels: the number of MS rows per warp work item (the
tile height of a 128-column strip: taller items amortise the D4 prologue row,
shorter ones balance the last wave), the most bands one forward launch or
batched table entry handles (fewer bands per launch hold fewer registers per
lane but read PAN once per chunk), the same for the adjoint (chunks after the
first add into grad_PAN), and the resident CTAs per SM of the persistent grid
(kept at the maximum: one CTA per SM measured about 45 % slower on every
workload tried).  `tune_batched`, `tune_fuse` and `tune_backward` time every
candidate of a launch with CUDA events on the given data and keep the
fastest.  Results are cached in a JSON file keyed by GPU (name, SM count,
compute capability, driver) and a shape class, so a process pays for tuning
once per machine and workload kind; `cached` looks a shape up without tuning
and `using` applies one around a call (the knobs are process-wide).

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
BLOCKS = (0,)  # 0 = as many CTAs per SM as fit
FWD_CHUNKS = (0, 6, 4)  # 0 = library default (8 bands per launch, 6 on shifted rows)
BWD_CHUNKS = (0, 4)     # 0 = library default (8)
# Bumped when the kernels behind the knobs change enough that cached choices
# may no longer be the fastest (3: TMEM scoring kernel, narrow batched
# instance).
CACHE_VERSION = 3

_lock = threading.Lock()


@dataclass(frozen=True)
class LaunchShape:
    rows_per_item: int
    blocks_per_sm: int
    fwd_chunk: int = 0
    bwd_chunk: int = 0

    def label(self) -> str:
        return f"r{self.rows_per_item}b{self.blocks_per_sm}f{self.fwd_chunk}g{self.bwd_chunk}"


DEFAULT = LaunchShape(0, 0, 0, 0)
_applied = DEFAULT  # the knob values this module last set in the library


def apply(shape: LaunchShape) -> None:
    """Set the library's process-wide knobs (rows per item, band chunks)."""
    global _applied
    from . import _C
    _C.dwtfuse_set_rows_per_item(shape.rows_per_item)
    _C.dwtfuse_set_band_chunks(shape.fwd_chunk, shape.bwd_chunk)
    _applied = shape


class using:
    """Context manager: the knobs of `shape` around a call, the previous ones after."""

    def __init__(self, shape: LaunchShape | None):
        self.shape = shape

    def __enter__(self):
        self.prev = _applied
        if self.shape is not None:
            apply(self.shape)
        return self.shape

    def __exit__(self, *exc):
        if self.shape is not None:
            apply(self.prev)
        return False


def cache_path() -> str:
    return os.environ.get("DWTFUSE_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "dwtfuse", "tune.json")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        if (not isinstance(data, dict) or data.get("version") != CACHE_VERSION
                or not isinstance(data.get("entries"), dict)):
            return {"version": CACHE_VERSION, "entries": {}}
        return data
    except (OSError, ValueError):
        return {"version": CACHE_VERSION, "entries": {}}


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


def backward_class(N: int, H: int, W: int, bands: int, wavelet: int) -> str:
    return f"bwd|wav{wavelet}|n{N}|b{bands}|px2^{round(math.log2(max(1, H * W)))}"


def pick(candidates: Iterable[LaunchShape], time_ms: Callable[[LaunchShape], float]) -> tuple[LaunchShape, dict]:
    """Fastest candidate by time_ms (ties go to the earlier candidate)."""
    best, best_t, table = None, float("inf"), {}
    for c in candidates:
        t = float(time_ms(c))
        table[c.label()] = t
        if t < best_t:
            best, best_t = c, t
    if best is None:
        raise ValueError("no candidates")
    return best, table


def _entry_shape(e) -> LaunchShape | None:
    try:
        return LaunchShape(int(e["rows_per_item"]), int(e["blocks_per_sm"]), int(e.get("fwd_chunk", 0)),
                           int(e.get("bwd_chunk", 0)))
    except (KeyError, TypeError, ValueError, AttributeError):
        return None


def cached(key: str, path: str | None = None) -> LaunchShape | None:
    """The cached shape for a key, or None (no tuning)."""
    with _lock:
        e = load_cache(path)["entries"].get(key)
    return _entry_shape(e) if e is not None else None


def cached_or_tune(key: str, tune: Callable[[], tuple[LaunchShape, dict]], path: str | None = None,
                   retune: bool = False) -> LaunchShape:
    with _lock:
        data = load_cache(path)
        e = data["entries"].get(key)
        if e is not None and not retune:
            got = _entry_shape(e)
            if got is not None:
                return got
    best, table = tune()
    with _lock:
        data = load_cache(path)
        data["entries"][key] = {"rows_per_item": best.rows_per_item, "blocks_per_sm": best.blocks_per_sm,
                                "fwd_chunk": best.fwd_chunk, "bwd_chunk": best.bwd_chunk, "times_ms": table}
        save_cache(data, path)
    return best


def tuning_allowed() -> bool:
    """False while a CUDA graph is being captured on the current stream, or
    with DWTFUSE_AUTOTUNE=0 (then only cached shapes are used)."""
    if os.environ.get("DWTFUSE_AUTOTUNE", "1") == "0":
        return False
    import torch
    return not torch.cuda.is_current_stream_capturing()


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

    def timed(c):
        with using(LaunchShape(0, 0, c.fwd_chunk, 0)):
            return _time(lambda: _C.dwtfuse_fuse_batched(scenes, workspace, c.rows_per_item, c.blocks_per_sm),
                         reps)

    def run():
        cands = [LaunchShape(r, b, f) for f in FWD_CHUNKS for r in ROWS for b in BLOCKS]
        return pick(cands, timed)

    return cached_or_tune(key, run, path, retune)


def tune_backward(g, wavelet: int, gp, gm, reps: int = 3, path: str | None = None,
                  retune: bool = False) -> LaunchShape:
    """Rows per item and adjoint band chunk for the batched adjoint of g
    (N, B, H, W) into gp (N, H, W) and gm (N, B, H/2, W/2) (the autograd
    backward's launch)."""
    from . import _C
    N, B, H, W = g.shape
    key = current_device_key() + "|" + backward_class(N, H, W, B, wavelet)
    import torch
    ws = torch.empty(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=g.device)
    scenes = [_C.make_grad_scene(g[i], wavelet, gp[i], gm[i]) for i in range(min(N, _C.MAX_SCENES))]

    def timed(c):
        with using(c):
            return _time(lambda: _C.dwtfuse_fuse_backward_batched(scenes, ws), reps)

    def run():
        cands = [LaunchShape(r, 0, 0, k) for k in BWD_CHUNKS for r in (0, 16, 48, 64)]
        return pick(cands, timed)

    return cached_or_tune(key, run, path, retune)


def tune_fuse(pan, ms, wavelet: int, out_f32, out_u8, reps: int = 3, path: str | None = None,
              retune: bool = False) -> LaunchShape:
    """Rows per item and forward band chunk for dwtfuse_fuse on this scene
    shape; leaves the library knobs set to the chosen values."""
    from . import _C
    bands = ms.shape[0] if hasattr(ms, "shape") else len(ms)
    outs = ("f" if out_f32 is not None else "") + ("u" if out_u8 is not None else "")
    key = current_device_key() + "|" + fuse_class(pan.shape[0], pan.shape[1], bands, wavelet,
                                                  _C._dtype_code(pan, "pan"), outs)

    def timed(c):
        with using(c):
            return _time(lambda: _C.dwtfuse_fuse(pan, ms, wavelet, out_f32, out_u8), reps)

    def run():
        return pick([LaunchShape(r, 0, f) for f in FWD_CHUNKS for r in (0, 16, 32, 48, 64)], timed)

    best = cached_or_tune(key, run, path, retune)
    apply(best)
    return best
