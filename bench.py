#!/usr/bin/env python
"""Benchmark of the fused DWT pansharpening hot path on one GB300 per rank.

Workload (one step): Daubechies-4 fusion of a Landsat-7-shaped synthetic scene,
PAN 16384 x 16384 uint8 with 6 MS bands 8192 x 8192 uint8 (periodic wrap, LL
gain 2), writing every fused band both as float32 and as rounded uint8 in one
pass, then ERGAS and QNR of the uint8 product on the GPU.  Inputs are
generated on the device from a seed (scenegen).  The step is one call of the
library's fused form, dwtfuse_fuse_metrics: the forward, scoring its uint8
product on chip, then the MS-resolution pass (started as the forward drains)
and the reduction.

  value     fused Gpx/s = PAN pixels x bands per second, inputs resident in HBM
  e2e       the same metric with the inputs copied host -> device from pinned
            memory and the uint8 fused bands and quality figures copied back
            every step (copies and compute of neighbouring steps overlap); the
            float32 bands stay on the device, so seen from the host this is a
            uint8-out pipeline
  roofline  the forward-and-score kernel (the step's dominant kernel, ~89 % of
            it): algorithmic bytes per launch (inputs read once, both outputs
            written once) / mean launch time, from CUDA events on the launch
            stream around each of K launches of dwtfuse_fuse_and_score (the
            same kernel alone) right after the main timed region, against the
            measured HBM copy bandwidth
  separate  the same step as two separate calls (dwtfuse_fuse, then
            dwtfuse_metrics reading the product back), with the plain
            forward's roofline
  forms     the other forms of the path, timed after the main region on their
            own workloads: 96 uneven scenes through one captured batched launch;
            forward + backward of a batch of 8 float32 4096^2 scenes (4 bands)
            next to the plain forward of the same batch; and 12 scenes of
            8192^2 .. 32768^2 x 8 bands through one graph of forward, metrics and
            backward (outputs streamed through one slot)

Multi-GPU: the path does not shard here (replicas only): each rank fuses its
own scene, timing is the max over ranks, value sums every rank's pixels.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused Gpx/s (PAN px × bands) and % HBM roofline; fwd+bwd Gpx/s vs plain fwd"
UNIT = "Gpx/s"
H = W = 16384  # overridden by --side (profiling cases only)
BANDS = 6
WAVELET = 1  # Daubechies-4
BLOB_SCALE = 16.0
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, vendor figure (context; the measured copy peak is the denominator)

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the
# forward-and-score kernel at this workload, keyed by the hash of the kernel
# sources it was taken on.
KNOWN_TRAFFIC: dict[str, float] = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum (one pass) on the
    # default workload at full size, captured with the step's launch list:
    # read 689,832,448 + write 7,991,618,304
    "88490acee432": 8681450752.0,
    # the same capture after the row-band fields joined the tile header:
    # read 689,828,693 + write 7,989,620,992 (mean of 3 launches)
    "3c44d97b0575": 8679449685.0,
    # after the scoring emitter took 7-8 bands (the 6-band body unchanged):
    # read 689,794,219 + write 7,989,526,784 (mean of 3 launches)
    "af32194f41e5": 8679321003.0,
    # the window sums in TMEM (16-warp CTAs), items round the CTAs first:
    # read 689,499,904 + write 7,989,635,328 (mean of 3 launches)
    "6b8106a5e69f": 8679135232.0,
    # the same 6-band body after 7 bands joined the TMEM kernel:
    # read 689,457,322 + write 7,989,600,853 (mean of 3 launches)
    "9f3157beffa0": 8679058175.0,
    # the same 6-band body after 8 bands joined the TMEM kernel (12-warp CTAs):
    # read 689,428,992 + write 7,989,767,594 (mean of 3 launches)
    "117fcefd467f": 8679196586.0,
    # the same kernel waiting for its TMEM stores before every scoring:
    # read 689,644,885 + write 7,989,676,288 (mean of 3 launches)
    "22e4d6d25dce": 8679321173.0,
}
KERNEL_SOURCES = ("fuse_tile.cuh", "fuse_metrics.cu", "metric_q.cuh", "tmem.cuh")


def kernel_hash() -> str:
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1803_00737_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def workload_config() -> dict:
    return {
        "workload": f"D4 DWT fusion, PAN {H}x{W} uint8, {BANDS} MS bands {H // 2}x{W // 2} uint8, "
                    "float32 + uint8 fused output in one pass, then ERGAS + QNR (32x32 windows) "
                    "of the uint8 product",
        "wavelet": "daubechies4_periodic",
        "pan": [H, W],
        "bands": BANDS,
        "outputs": ["float32", "uint8"],
        "metrics": ["ERGAS", "QNR", "D_lambda", "D_s"],
        "l2": "inputs and outputs (8.7 GB per step) exceed L2; no flush needed",
        "parallelism": "replicas",
    }


def fwd_bytes_per_launch() -> float:
    # PAN u8 (1 B/px) + per band: MS u8 (0.25 B/px) + f32 out (4) + u8 out (1)
    return H * W * (1.0 + BANDS * (0.25 + 4.0 + 1.0))


def measured_hbm() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks (NVML, read-only)

class ClockSampler:
    """Samples SM clock and clock-event reasons through NVML (read-only) in a
    background thread while the timed region runs."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid: str | None, interval_s: float = 0.002):
        self.samples: list[tuple[int, int]] = []
        self.max_mhz = None
        self.ok = False
        self._stop = threading.Event()
        self._t = None
        self.interval = interval_s
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            rc = 1
            if uuid:
                rc = self.nvml.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h))
            if rc != 0:
                return
            self._reason_fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self.ok = True
        except Exception:
            self.ok = False

    def _sample(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0 and \
                self._reason_fn(self.h, ctypes.byref(rs)) == 0:
            self.samples.append((clk.value, rs.value))

    def _run(self):
        while not self._stop.is_set():
            self._sample()
            time.sleep(self.interval)

    def start(self):
        if self.ok:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()

    def stop(self) -> dict:
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "NVML unavailable"}
        self._stop.set()
        self._t.join()
        if not self.samples:
            self._sample()
        mhz = [s[0] for s in self.samples]
        bits = 0
        for s in self.samples:
            bits |= s[1]
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": self.max_mhz,
                "reasons": [n for b, n in self.REASONS.items() if bits & b],
                "samples": len(self.samples)}


# ------------------------------------------------------------------ distributed helpers

def dist_env() -> tuple[int, int, int]:
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def aggregate(elapsed_s: float, units: float, world: int, device=None) -> tuple[float, float]:
    """(max elapsed over ranks, sum of units over ranks); identity at world 1."""
    if world == 1:
        return elapsed_s, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ CPU oracle (baseline only)

def oracle_step(pan, ms, pan_u8, ms_u8) -> None:
    """One step of the path in the oracle: FP64 fusion, the uint8 product, and
    ERGAS + QNR of that product."""
    import oracle as O
    fused = O.fuse(pan, ms, WAVELET)
    u8 = O.to_u8(fused)
    del fused
    O.ergas(u8, list(ms_u8))
    O.qnr(u8, list(ms_u8), pan_u8)


def oracle_rate(pan_u8, ms_u8, min_seconds: float, max_reps: int) -> tuple[float, int, float, int]:
    """Oracle rate of the whole step on a host sample: (Gpx/s, threads, seconds, reps)."""
    import numpy as np

    import oracle as O
    pan = pan_u8.astype(np.float64)
    ms = ms_u8.astype(np.float64)
    units = pan.size * ms.shape[0]
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle_step(pan, ms, pan_u8, ms_u8)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            break
    return units * reps / el / 1e9, O.num_threads(), el, reps


def run_reference(args) -> None:
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import scenegen
    side = args.ref_side
    pan, ms = scenegen.make_scene(side, side, BANDS, seed=0, blob_scale=BLOB_SCALE)
    pan, ms = pan.numpy(), ms.numpy()
    import numpy as np

    import oracle as O
    pf, mf = pan.astype(np.float64), ms.astype(np.float64)
    for _ in range(args.warmup):
        oracle_step(pf, mf, pan, ms)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(pf, mf, pan, ms)
    el = time.perf_counter() - t0
    value = side * side * BANDS * args.steps / el / 1e9
    sample = (f"FP64 oracle, D4 fusion of a {side}x{side} PAN scene with {BANDS} bands (same "
              f"generator) + ERGAS/QNR of the uint8 product, per step")
    cpu = {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle", "sample": sample}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(), "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm

def measure_e2e(args, pan, ms, out_f, mws, stream, world, dev) -> dict:
    """End to end through the public API: every step copies its inputs from
    pinned host memory to the device, fuses, computes ERGAS/QNR, and copies the
    uint8 fused bands and the four quality figures back to pinned host memory.
    Steps are pipelined over three streams (host->device, compute,
    device->host) with two buffer sets, so one step's copies overlap its
    neighbours' compute; the timed region spans the first upload to the last
    download."""
    import torch

    from paper_1803_00737_gb300 import _C
    Ke = max(1, min(args.steps, args.e2e_steps))
    pan_h = [pan.cpu().pin_memory() for _ in range(2)]
    ms_h = [ms.cpu().pin_memory() for _ in range(2)]
    out_h = [torch.empty((BANDS, H, W), dtype=torch.uint8).pin_memory() for _ in range(2)]
    res_h = [torch.empty(4, dtype=torch.float64).pin_memory() for _ in range(2)]
    pan_d = [pan, torch.empty_like(pan)]
    ms_d = [ms, torch.empty_like(ms)]
    out_u = [torch.empty((BANDS, H, W), dtype=torch.uint8, device=dev) for _ in range(2)]
    res_d = [torch.zeros(4, dtype=torch.float64, device=dev) for _ in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=False)  # noqa: E731
    uploaded = [ev() for _ in range(2)]
    computed = [ev() for _ in range(2)]
    downloaded = [ev() for _ in range(2)]
    for e in downloaded + computed:
        e.record(stream)

    def one(k):
        i = k % 2
        with torch.cuda.stream(s_in):
            s_in.wait_event(computed[i])          # compute k-2 is done with this input set
            pan_d[i].copy_(pan_h[i], non_blocking=True)
            ms_d[i].copy_(ms_h[i], non_blocking=True)
            uploaded[i].record(s_in)
        with torch.cuda.stream(s_cmp):
            s_cmp.wait_event(uploaded[i])
            s_cmp.wait_event(downloaded[i])       # download k-2 is done with this output set
            _C.dwtfuse_fuse_metrics(pan_d[i], ms_d[i], WAVELET, out_f, out_u[i], mws, res_d[i], stream=s_cmp)
            computed[i].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(computed[i])
            out_h[i].copy_(out_u[i], non_blocking=True)
            res_h[i].copy_(res_d[i], non_blocking=True)
            downloaded[i].record(s_out)

    # Warm-up: pipelined steps (first touches of the pinned buffers), then one
    # untimed run of Ke steps (the first run over a cold host link measured
    # about half the rate of the runs after it).
    warm = max(2, args.warmup) + Ke
    for k in range(warm):
        one(k)
    torch.cuda.synchronize()
    # Three timed runs of Ke steps each; the value is their median (the host
    # link's rate varies from run to run), every run's rate is listed.
    trials = []
    k0 = warm
    for _ in range(3):
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        for k in range(k0, k0 + Ke):
            one(k)
        e1.record(s_out)
        torch.cuda.synchronize()
        barrier(world)
        k0 += Ke
        e_el, e_units = aggregate(e0.elapsed_time(e1) / 1e3, float(H * W * BANDS * Ke), world, dev)
        trials.append(e_units / e_el / 1e9)
    return {"value": statistics.median(trials), "unit": UNIT,
            "h2d_bytes_per_step": pan.numel() + ms.numel(),
            "d2h_bytes_per_step": out_u[0].numel() + 4 * 8,
            "steps": Ke, "runs": [round(t, 2) for t in trials], "statistic": "median of 3 runs",
            "pipelined": "3 streams, 2 buffer sets",
            "returned": "the uint8 fused bands and the four quality figures; the float32 fused "
                        "bands the step also writes stay in device memory (a uint8-out pipeline "
                        "seen from the host)"}


def _time_ms(fn, reps: int, stream) -> float:
    """Mean milliseconds of fn() over reps runs (CUDA events on `stream`)."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_forms(args, dev, peak: float, world: int) -> dict:
    """Batched (96 uneven scenes, one captured persistent launch) and autograd
    (batch 8 x 4096^2 float32, 4 bands: forward + backward vs plain forward)."""
    import torch

    import scenegen
    from paper_1803_00737_gb300 import _C
    out = {}
    stream = torch.cuda.current_stream()
    reps = max(1, args.form_reps)

    # -- batched: 96 scenes, sides U[256, 8192], 3-8 bands, Haar/D4, float32 out
    # (--forms-small: 24 scenes up to 4096, for profiling only)
    specs = scenegen.batch_specs(n=24, seed=0, hi=4096) if args.forms_small else scenegen.batch_specs(n=96, seed=0)
    keep, scenes = [], []
    px_bands = 0.0
    nbytes = 0.0
    for sp in specs:
        p, m = scenegen.make_scene(sp.H, sp.W, sp.bands, seed=sp.seed, device=dev)
        o = torch.empty((sp.bands, sp.H, sp.W), dtype=torch.float32, device=dev)
        keep.append((p, m, o))
        scenes.append(_C.make_scene(p, m, sp.wavelet, o, None))
        px_bands += sp.H * sp.W * sp.bands
        nbytes += sp.H * sp.W * (1.0 + sp.bands * (0.25 + 4.0))
    ws = torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=dev)
    from paper_1803_00737_gb300 import tune
    shape = tune.tune_batched(scenes, [(sp.H, sp.W, sp.bands, sp.wavelet) for sp in specs], ws)
    _C.dwtfuse_fuse_batched(scenes, ws, shape.rows_per_item, shape.blocks_per_sm)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        _C.dwtfuse_fuse_batched(scenes, ws, shape.rows_per_item, shape.blocks_per_sm)
    g.replay()
    ms_b = _time_ms(g.replay, reps, stream)
    out["batched"] = {
        "workload": "96 scenes, PAN sides even U[256, 8192] (independent H, W), 3-8 bands, "
                    "Haar/D4 mixed, uint8 in, float32 out, persistent launches in a CUDA graph (one per "
                    "kernel instance: entries of at most 4 bands, wider ones)",
        "value": px_bands / (ms_b / 1e3) / 1e9, "unit": UNIT, "ms": ms_b,
        "roofline": {"achieved": nbytes / (ms_b / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": nbytes / (ms_b / 1e3) / 1e9 / peak},
        "gpu_launches_per_replay": 2 if (any(sp.bands <= 4 for sp in specs) and any(sp.bands > 4 for sp in specs))
        else 1,
        "launch_shape": {"rows_per_item": shape.rows_per_item, "blocks_per_sm": shape.blocks_per_sm,
                         "chosen_by": "autotuner (paper_1803_00737_gb300.tune)",
                         "candidates_ms": tune.load_cache()["entries"].get(
                             tune.current_device_key() + "|" + tune.batched_class(
                                 [(sp.H, sp.W, sp.bands, sp.wavelet) for sp in specs]), {}).get("times_ms")},
    }
    del keep, scenes, g
    torch.cuda.empty_cache()

    # -- autograd: batch 8 of PAN 4096^2 float32 with 4 MS bands (--forms-small: 2 x 4096^2)
    N, B, S = (2, 4, 4096) if args.forms_small else (8, 4, 4096)
    pans, mss = [], []
    for i in range(N):
        p, m = scenegen.make_scene(S, S, B, seed=i, device=dev)
        pans.append(p.float())
        mss.append(m.float())
    P = torch.stack(pans)
    M = torch.stack(mss)
    del pans, mss
    F = torch.empty((N, B, S, S), dtype=torch.float32, device=dev)
    G = scenegen.target_like((N, B, S, S), seed=1000, device=dev)
    gp = torch.empty((N, S, S), dtype=torch.float32, device=dev)
    gm = torch.empty((N, B, S // 2, S // 2), dtype=torch.float32, device=dev)

    from paper_1803_00737_gb300.autograd import fuse_batch, fuse_batch_backward

    def fwd_all():  # the autograd forward: one batched launch for the batch
        fuse_batch(P, M, WAVELET, F)

    def bwd_all():  # the autograd backward: one batched launch (4 bands: one chunk)
        fuse_batch_backward(G, WAVELET, gp, gm)

    def fwd_bwd():
        fwd_all()
        bwd_all()

    for f in (fwd_all, bwd_all):
        f()
    ms_f = _time_ms(fwd_all, reps, stream)
    ms_bw = _time_ms(bwd_all, reps, stream)
    ms_fb = _time_ms(fwd_bwd, reps, stream)
    units = N * B * S * S
    fbytes = N * S * S * (4.0 + B * (1.0 + 4.0))
    bbytes = N * S * S * (4.0 * B + 4.0 + B)
    out["autograd"] = {
        "workload": "D4, batch 8 x PAN 4096^2 float32, 4 MS bands 2048^2 float32; forward "
                    "(float32 out) + adjoint backward (grad PAN, grad MS)",
        "fwd_bwd": units / (ms_fb / 1e3) / 1e9, "plain_fwd": units / (ms_f / 1e3) / 1e9,
        "unit": UNIT, "ratio_fwd_bwd_to_fwd": ms_f / ms_fb,
        "fwd_ms": ms_f, "bwd_ms": ms_bw, "fwd_bwd_ms": ms_fb,
        "roofline_fwd": {"achieved": fbytes / (ms_f / 1e3) / 1e9, "frac": fbytes / (ms_f / 1e3) / 1e9 / peak},
        "roofline_bwd": {"achieved": bbytes / (ms_bw / 1e3) / 1e9, "frac": bbytes / (ms_bw / 1e3) / 1e9 / peak},
        "gpu_launches_per_pass": 2,
    }
    return out


def measure_config4(args, dev, peak: float) -> dict:
    """12 square scenes, sides even U[8192, 32768], 8 MS bands, D4: per scene the
    batched forward (float32 + uint8), ERGAS/QNR of the uint8 product and the
    adjoint with grad_out = F (loss 1/2 ||F||^2), all in one captured CUDA graph.
    Inputs of every scene stay resident (~17 GB); the outputs and gradients
    stream through one slot sized for the largest scene (~60 GB), so the whole
    workload (~445 GB if everything were resident) runs in a bounded pool."""
    import torch

    import scenegen
    from paper_1803_00737_gb300 import _C
    specs = scenegen.batch_specs(n=12, seed=0, lo=8192, hi=32768, bands=(8, 8),
                                 wavelets=(scenegen.D4,), square=True)
    if args.forms_small:
        specs = [scenegen.SceneSpec(s.H // 4, s.W // 4, s.bands, s.wavelet, s.seed) for s in specs[:3]]
    B = 8
    inputs = [scenegen.make_scene(sp.H, sp.W, B, seed=sp.seed, blob_scale=16.0, device=dev) for sp in specs]
    torch.cuda.empty_cache()
    n_max = max(sp.H * sp.W for sp in specs)
    out_f = torch.empty(B * n_max, dtype=torch.float32, device=dev)
    out_u = torch.empty(B * n_max, dtype=torch.uint8, device=dev)
    gp_s = torch.empty(n_max, dtype=torch.float32, device=dev)
    gm_s = torch.empty(B * n_max // 4, dtype=torch.float32, device=dev)
    ws = torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=dev)
    mws = torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=dev)
    res = torch.zeros((len(specs), 4), dtype=torch.float64, device=dev)
    views = []
    for sp, (p, m) in zip(specs, inputs):
        n = sp.H * sp.W
        f = out_f[:B * n].view(B, sp.H, sp.W)
        u = out_u[:B * n].view(B, sp.H, sp.W)
        views.append((sp, p, m, f, u, gp_s[:n].view(sp.H, sp.W),
                      gm_s[:B * n // 4].view(B, sp.H // 2, sp.W // 2), _C.make_scene(p, m, sp.wavelet, f, u)))

    def run():  # per scene: forward scoring its uint8 product on chip, MS pass, finalize; adjoint
        for k, (sp, p, m, f, u, gp, gm, scene) in enumerate(views):
            _C.dwtfuse_fuse_metrics(p, m, sp.wavelet, f, u, mws, res[k])
            _C.dwtfuse_fuse_backward(f, sp.wavelet, gp, gm)

    def run_phases(ev):  # the same work with the two halves of the metrics call apart, for timing
        for k, (sp, p, m, f, u, gp, gm, scene) in enumerate(views):
            ev[k][0].record()
            _C.dwtfuse_fuse_and_score(p, m, sp.wavelet, f, u, mws)
            ev[k][1].record()
            _C.dwtfuse_score_finish(m, p, u, mws, res[k])
            ev[k][2].record()
            _C.dwtfuse_fuse_backward(f, sp.wavelet, gp, gm)
            ev[k][3].record()

    run()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in views]
    run_phases(ev)
    torch.cuda.synchronize()
    t_f = sum(e[0].elapsed_time(e[1]) for e in ev) / 1e3
    t_m = sum(e[1].elapsed_time(e[2]) for e in ev) / 1e3
    t_b = sum(e[2].elapsed_time(e[3]) for e in ev) / 1e3
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        run()
    g.replay()
    torch.cuda.synchronize()
    ms_graph = _time_ms(g.replay, max(1, min(3, args.form_reps)), torch.cuda.current_stream())
    px = sum(sp.H * sp.W for sp in specs)
    units = px * B
    fb = px * (1.0 + B * (0.25 + 4.0 + 1.0))  # the forward's bytes; its scoring reads nothing more
    mb = px * (B * 0.25 + 1.0)  # MS-resolution pass: MS and PAN read once
    bb = px * (4.0 * B + 4.0 + B)
    rf = lambda nbytes, t: {"achieved": nbytes / t / 1e9, "frac": nbytes / t / 1e9 / peak}  # noqa: E731
    q = res.cpu().numpy()
    del views, inputs, out_f, out_u, gp_s, gm_s, g
    torch.cuda.empty_cache()
    return {
        "workload": "12 square scenes, PAN sides even U[8192, 32768] uint8, 8 MS bands, D4: forward "
                    "(float32 + uint8) scoring its uint8 product on chip + MS-resolution pass and "
                    "finalize of ERGAS/QNR + adjoint with grad_out = F, one CUDA graph, outputs "
                    "streamed through one slot"
                    + (" [reduced: --forms-small]" if args.forms_small else ""),
        "scenes": [sp.H for sp in specs], "pan_gpx": px / 1e9,
        "fwd_bwd_metrics_gpxs": units / (ms_graph / 1e3) / 1e9, "unit": UNIT, "graph_ms": ms_graph,
        "per_kernel": {"fused_forward": {"ms": t_f * 1e3, **rf(fb, t_f),
                                         "note": "forward + PAN-resolution scoring on chip"},
                       "metrics": {"ms": t_m * 1e3, **rf(mb, t_m),
                                   "note": "MS-resolution pass + finalize (the PAN-resolution sums "
                                           "come from the forward, no read-back of the product)"},
                       "adjoint": {"ms": t_b * 1e3, **rf(bb, t_b)}},
        "qnr_range": [float(q[:, 1].min()), float(q[:, 1].max())],
        "gpu_launches_per_replay": len(specs) * (3 + 2),
    }


def measure_transforms(args, dev, peak: float) -> dict:
    """Standalone one-level 2D DWT and inverse at the benchmark size (D4 and Haar)."""
    import torch

    from paper_1803_00737_gb300 import _C
    S = 4096 if args.forms_small else 16384
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    img = torch.randint(0, 256, (S, S), generator=g, device=dev, dtype=torch.uint8)
    Z = torch.empty((S, S), dtype=torch.float32, device=dev)
    out = torch.empty((S, S), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {"workload": f"PAN {S}x{S}: uint8 image -> float coefficients (dwt2), float coefficients "
                       "-> float image (idwt2)"}
    for wav, name in ((1, "d4"), (0, "haar")):
        _C.dwtfuse_dwt2(img, wav, Z)  # first launches (module load, occupancy query) stay untimed
        _C.dwtfuse_idwt2(Z, wav, out)
        t_f = _time_ms(lambda: _C.dwtfuse_dwt2(img, wav, Z), max(3, args.form_reps), stream) / 1e3
        t_i = _time_ms(lambda: _C.dwtfuse_idwt2(Z, wav, out), max(3, args.form_reps), stream) / 1e3
        px = S * S
        res[name] = {
            "dwt2_gpxs": px / t_f / 1e9, "idwt2_gpxs": px / t_i / 1e9,
            "dwt2_roofline": {"achieved": 5.0 * px / t_f / 1e9, "frac": 5.0 * px / t_f / 1e9 / peak},
            "idwt2_roofline": {"achieved": 8.0 * px / t_i / 1e9, "frac": 8.0 * px / t_i / 1e9 / peak},
        }
    del img, Z, out
    torch.cuda.empty_cache()
    return res


def run_ours(args) -> None:
    import torch

    global H, W
    H = W = args.side

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import scenegen
    from paper_1803_00737_gb300 import _C
    from paper_1803_00737_gb300.build import build
    build()
    _C.lib()

    pan, ms = scenegen.make_scene(H, W, BANDS, seed=rank, blob_scale=BLOB_SCALE, device=dev)
    out_f = torch.empty((BANDS, H, W), dtype=torch.float32, device=dev)
    out_u = torch.empty((BANDS, H, W), dtype=torch.uint8, device=dev)
    mws = torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=dev)
    res = torch.zeros(4, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():  # forward + on-chip scoring, MS-resolution pass, finalize: 3 kernels
        _C.dwtfuse_fuse_metrics(pan, ms, WAVELET, out_f, out_u, mws, res)

    def fused_kernel():  # the step's first kernel alone
        _C.dwtfuse_fuse_and_score(pan, ms, WAVELET, out_f, out_u, mws)

    launches_per_step = 3
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid is not None else None)
    K = args.steps
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(2)) for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    torch.cuda.nvtx.range_push("timed")
    t_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    # The dominant kernel alone, K launches, CUDA events around each.
    kev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(2)) for _ in range(K)]
    torch.cuda.nvtx.range_push("kernel")
    for k in range(K):
        kev[k][0].record(stream)
        fused_kernel()
        kev[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    elapsed = t_start.elapsed_time(t_end) / 1e3
    step_ms = [a.elapsed_time(b) for a, b in ev]
    fwd_ms = [a.elapsed_time(b) for a, b in kev]
    quality = res.cpu().tolist()
    units = float(H * W * BANDS * K)
    max_el, total_units = aggregate(elapsed, units, world, dev)
    value = total_units / max_el / 1e9

    # The same step as separate calls, for comparison (not the headline).
    res_sep = torch.zeros(4, dtype=torch.float64, device=dev)
    f_sep = _time_ms(lambda: _C.dwtfuse_fuse(pan, ms, WAVELET, out_f, out_u), K, stream)
    m_sep = _time_ms(lambda: _C.dwtfuse_metrics(out_u, ms, pan, mws, res_sep), K, stream)
    separate = {"fwd_ms": f_sep, "metrics_ms": m_sep, "step_ms": f_sep + m_sep,
                "fwd_roofline_frac": fwd_bytes_per_launch() / (f_sep / 1e3) / 1e9 / measured_hbm()[0],
                "quality_equal_to_fused": bool(torch.allclose(res_sep, res, rtol=0, atol=1e-6))}

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, pan, ms, out_f, mws, stream, world, dev)

    peak, peak_kind = measured_hbm()
    mean_fwd_s = statistics.mean(fwd_ms) / 1e3
    achieved = fwd_bytes_per_launch() / mean_fwd_s / 1e9
    kh = kernel_hash()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": KNOWN_TRAFFIC.get(kh),
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "peak_source": f"{peak_kind} (copy bandwidth)",
                "kernel": "fuse_metrics_kernel<uint8, D4, 6> (forward + on-chip scoring)", "kernel_hash": kh,
                "algorithmic_bytes_per_launch": fwd_bytes_per_launch(),
                "mean_launch_ms": mean_fwd_s * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        side = min(args.cpu_side, H)
        pan_c = pan[:side, :side].cpu().numpy()
        ms_c = ms[:, :side // 2, :side // 2].cpu().numpy()
        rate, cores, secs, reps = oracle_rate(pan_c, ms_c, args.cpu_seconds, 20)
        # The same oracle on one thread, on a quarter-side crop (about as long).
        import oracle as O
        side1 = max(64, side // 4)
        O.set_threads(1)
        try:
            rate1, _, secs1, reps1 = oracle_rate(pan_c[:side1, :side1], ms_c[:, :side1 // 2, :side1 // 2],
                                                 args.cpu_seconds, 20)
        finally:
            O.set_threads(cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle step (D4 fusion + ERGAS/QNR of the uint8 product) on the "
                         f"top-left {side}x{side} PAN crop with its {BANDS} MS crops (periodic "
                         f"wrap at the crop), {reps} rep(s), {secs:.1f} s",
               "one_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"the same step on the top-left {side1}x{side1} crop, "
                                        f"{reps1} rep(s), {secs1:.1f} s"}}

    forms = None
    if not args.no_forms:
        del out_f
        torch.cuda.empty_cache()
        forms = measure_forms(args, dev, peak, world)
        forms["config4"] = measure_config4(args, dev, peak)
        forms["transforms"] = measure_transforms(args, dev, peak)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": max_el / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * K, "clocks": clocks,
            "step_ms": {"mean": statistics.mean(step_ms), "min": min(step_ms), "max": max(step_ms)},
            "fused_kernel_ms": {"mean": statistics.mean(fwd_ms), "min": min(fwd_ms), "max": max(fwd_ms)},
            "fwd_only_gpxs": H * W * BANDS / (statistics.mean(fwd_ms) / 1e3) / 1e9,
            "separate": separate,
            "quality": dict(zip(["ERGAS", "QNR", "D_lambda", "D_s"], quality)),
            "forms": forms,
        }))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_case(args) -> None:
    """One library call on a seeded synthetic scene, timed alone (for profiling
    a single kernel family at a chosen size; not the benchmark line).  Prints
    one JSON line: mean milliseconds per call and its algorithmic bytes / s."""
    import torch

    import scenegen
    from paper_1803_00737_gb300 import _C, build as bld

    bld.build()
    dev = "cuda"
    H, W, B = args.side, args.width or args.side, args.bands
    if args.rows or args.fwd_chunk or args.bwd_chunk:  # launch-shape knobs for this case
        from paper_1803_00737_gb300 import tune
        tune.apply(tune.LaunchShape(args.rows, 0, args.fwd_chunk, args.bwd_chunk))
    if args.no_staging:  # the warp-strip forward instead of the staged one
        _C.dwtfuse_set_fuse_staging(False)
    pan, ms = scenegen.make_scene(H, W, B, seed=0, blob_scale=BLOB_SCALE, device=dev)
    extra = {}
    if args.case == "metrics":
        fused = torch.empty((B, H, W), dtype=torch.uint8, device=dev)
        _C.dwtfuse_fuse(pan, ms, WAVELET, None, fused)
        ws = torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=dev)
        res = torch.zeros(4, dtype=torch.float64, device=dev)
        call = lambda: _C.dwtfuse_metrics(fused, ms, pan, ws, res)  # noqa: E731
        nbytes = H * W * (B + 1 + B * 0.25) + H * W * (B * 0.25 + 1)
    elif args.case == "fuse":
        of = torch.empty((B, H, W), dtype=torch.float32, device=dev)
        ou = torch.empty((B, H, W), dtype=torch.uint8, device=dev)
        call = lambda: _C.dwtfuse_fuse(pan, ms, WAVELET, of, ou)  # noqa: E731
        nbytes = H * W * (1.0 + B * (0.25 + 4.0 + 1.0))
    elif args.case == "fuse_score":  # the forward that scores its uint8 product on chip
        of = torch.empty((B, H, W), dtype=torch.float32, device=dev)
        ou = torch.empty((B, H, W), dtype=torch.uint8, device=dev)
        ws = torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=dev)
        call = lambda: _C.dwtfuse_fuse_and_score(pan, ms, WAVELET, of, ou, ws)  # noqa: E731
        nbytes = H * W * (1.0 + B * (0.25 + 4.0 + 1.0))
    elif args.case == "score_finish":  # the MS-resolution pass and the finalize of the fused form
        of = torch.empty((B, H, W), dtype=torch.float32, device=dev)
        ou = torch.empty((B, H, W), dtype=torch.uint8, device=dev)
        ws = torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=dev)
        res = torch.zeros(4, dtype=torch.float64, device=dev)
        _C.dwtfuse_fuse_and_score(pan, ms, WAVELET, of, ou, ws)
        call = lambda: _C.dwtfuse_score_finish(ms, pan, ou, ws, res)  # noqa: E731
        nbytes = H * W * (B * 0.25 + 1.0)  # MS bands and PAN read once
    elif args.case == "batched_f32":  # the autograd form's forward: float inputs, one batched launch
        P = torch.stack([pan.float() for _ in range(args.scenes)])
        M = torch.stack([ms.float() for _ in range(args.scenes)])
        of = torch.empty((args.scenes, B, H, W), dtype=torch.float32, device=dev)
        ws = torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=dev)
        scenes = [_C.make_scene(P[i], M[i], WAVELET, of[i], None) for i in range(args.scenes)]
        call = lambda: _C.dwtfuse_fuse_batched(scenes, ws)  # noqa: E731
        nbytes = args.scenes * H * W * (4.0 + B * (1.0 + 4.0))
    elif args.case in ("dwt2", "idwt2"):
        Z = torch.empty((H, W), dtype=torch.float32, device=dev)
        _C.dwtfuse_dwt2(pan, WAVELET, Z)
        if args.case == "dwt2":
            call = lambda: _C.dwtfuse_dwt2(pan, WAVELET, Z)  # noqa: E731
            nbytes = H * W * 5.0  # uint8 image in, float coefficients out
        else:
            img = torch.empty((H, W), dtype=torch.float32, device=dev)
            call = lambda: _C.dwtfuse_idwt2(Z, WAVELET, img)  # noqa: E731
            nbytes = H * W * 8.0  # float coefficients in, float image out
    elif args.case == "rows":
        from paper_1803_00737_gb300 import shard
        parts = shard.row_bands(H, 4)
        slabs = [(y0, y1, *shard.make_slab(pan, ms, y0, y1, WAVELET)) for y0, y1 in parts]
        outs = [torch.empty((B, y1 - y0, W), dtype=torch.float32, device=dev) for y0, y1 in parts]

        def call():  # the scene as 4 row bands, each from its slab
            for (y0, y1, ps, mss), o in zip(slabs, outs):
                _C.dwtfuse_fuse_rows(ps, mss, WAVELET, H, y0, y1, o, None)
        nbytes = H * W * (1.0 + B * (0.25 + 4.0))
        whole = torch.empty((B, H, W), dtype=torch.float32, device=dev)
        _C.dwtfuse_fuse(pan, ms, WAVELET, whole, None)
        extra["whole_scene_ms"] = _time_ms(lambda: _C.dwtfuse_fuse(pan, ms, WAVELET, whole, None),
                                           args.steps, torch.cuda.current_stream())
    else:  # backward
        g = scenegen.target_like((B, H, W), seed=1000, device=dev)
        gp = torch.empty((H, W), dtype=torch.float32, device=dev)
        gm = torch.empty((B, H // 2, W // 2), dtype=torch.float32, device=dev)
        call = lambda: _C.dwtfuse_fuse_backward(g, WAVELET, gp, gm)  # noqa: E731
        nbytes = H * W * (4.0 * B + 4.0 + B)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms_call = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"case": args.case, "H": H, "W": W, "bands": B, "calls": args.steps, "ms": ms_call,
                      "knobs": {"rows": args.rows, "fwd_chunk": args.fwd_chunk, "bwd_chunk": args.bwd_chunk, "staging": not args.no_staging},
                      "algorithmic_GBps": nbytes / (ms_call / 1e3) / 1e9, **extra}))


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-side", type=int, default=8192, help="PAN side of the CPU-baseline sample")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-side", type=int, default=4096, help="PAN side of a reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--form-reps", type=int, default=10)
    ap.add_argument("--forms-small", action="store_true",
                    help="shrink the batched and autograd workloads (profiling only)")
    ap.add_argument("--side", type=int, default=16384,
                    help="PAN side (default: the benchmark workload; smaller only for profiling)")
    ap.add_argument("--case", choices=["metrics", "fuse", "fuse_score", "score_finish", "batched_f32", "backward",
                                       "dwt2", "idwt2", "rows"],
                    help="time one library call alone at --side x --width with --bands (profiling aid)")
    ap.add_argument("--width", type=int, default=0, help="PAN width of a --case run (default: --side)")
    ap.add_argument("--bands", type=int, default=BANDS, help="MS bands of a --case run")
    ap.add_argument("--scenes", type=int, default=8, help="scenes of a --case batched_f32 run")
    ap.add_argument("--rows", type=int, default=0, help="rows-per-item knob of a --case run (0: default)")
    ap.add_argument("--fwd-chunk", type=int, default=0, help="forward band-chunk knob of a --case run")
    ap.add_argument("--bwd-chunk", type=int, default=0, help="adjoint band-chunk knob of a --case run")
    ap.add_argument("--no-staging", action="store_true",
                    help="a --case run on the warp-strip forward kernel (dwtfuse_set_fuse_staging(0))")
    args = ap.parse_args()
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
