#!/usr/bin/env python
"""Benchmark of the fused DWT pansharpening hot path on one GB300 per rank.

Workload (one step): Daubechies-4 fusion of a Landsat-7-shaped synthetic scene,
PAN 16384 x 16384 uint8 with 6 MS bands 8192 x 8192 uint8 (periodic wrap, LL
gain 2), writing every fused band both as float32 and as rounded uint8 in one
pass.  Inputs are generated on the device from a seed (scenegen).

  value     fused Gpx/s = PAN pixels x bands per second, inputs resident in HBM
  e2e       the same metric with the inputs copied host -> device from pinned
            memory and the uint8 fused bands copied back every step
  roofline  fused-forward kernel: algorithmic bytes per launch / mean launch
            time (CUDA events on the launch stream) against the measured HBM
            copy bandwidth

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
H = W = 16384
BANDS = 6
WAVELET = 1  # Daubechies-4
BLOB_SCALE = 16.0
FALLBACK_HBM_GBS = 6800.0

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the fused forward
# at this workload, keyed by the hash of the kernel sources it was taken on.
KNOWN_TRAFFIC: dict[str, float] = {}


def kernel_hash() -> str:
    h = hashlib.sha1()
    for f in ("fuse_tile.cuh", "fuse_fwd.cu"):
        with open(os.path.join(ROOT, "paper_1803_00737_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def workload_config() -> dict:
    return {
        "workload": f"D4 DWT fusion, PAN {H}x{W} uint8, {BANDS} MS bands {H // 2}x{W // 2} uint8, "
                    "float32 + uint8 fused output in one pass",
        "wavelet": "daubechies4_periodic",
        "pan": [H, W],
        "bands": BANDS,
        "outputs": ["float32", "uint8"],
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

def oracle_rate(pan_u8, ms_u8, min_seconds: float, max_reps: int) -> tuple[float, int, float, int]:
    """Oracle FP64 fusion rate on a host sample: (Gpx/s, threads, seconds, reps)."""
    import numpy as np

    import oracle as O
    pan = pan_u8.astype(np.float64)
    ms = ms_u8.astype(np.float64)
    units = pan.size * ms.shape[0]
    reps, t0 = 0, time.perf_counter()
    while True:
        O.fuse(pan, ms, WAVELET)
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
        O.fuse(pf, mf, WAVELET)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.fuse(pf, mf, WAVELET)
    el = time.perf_counter() - t0
    value = side * side * BANDS * args.steps / el / 1e9
    sample = (f"FP64 oracle, D4 fusion of a {side}x{side} PAN crop-size scene with {BANDS} "
              f"bands (same generator), per step")
    cpu = {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle", "sample": sample}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(), "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm

def run_ours(args) -> None:
    import torch

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
    stream = torch.cuda.current_stream()

    def step():
        _C.dwtfuse_fuse(pan, ms, WAVELET, out_f, out_u)

    launches_per_step = (BANDS + 7) // 8
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid is not None else None)
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    t_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    elapsed = t_start.elapsed_time(t_end) / 1e3
    fwd_ms = [a.elapsed_time(b) for a, b in ev]
    units = float(H * W * BANDS * K)
    max_el, total_units = aggregate(elapsed, units, world, dev)
    value = total_units / max_el / 1e9

    # end to end: pinned host inputs in, uint8 fused bands out, every step
    pan_h = pan.cpu().pin_memory()
    ms_h = ms.cpu().pin_memory()
    out_h = torch.empty((BANDS, H, W), dtype=torch.uint8).pin_memory()
    Ke = max(1, min(K, args.e2e_steps))
    for _ in range(2):
        pan.copy_(pan_h, non_blocking=True)
        ms.copy_(ms_h, non_blocking=True)
        step()
        out_h.copy_(out_u, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        pan.copy_(pan_h, non_blocking=True)
        ms.copy_(ms_h, non_blocking=True)
        step()
        out_h.copy_(out_u, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e_el, e_units = aggregate(e0.elapsed_time(e1) / 1e3, float(H * W * BANDS * Ke), world, dev)
    e2e = {"value": e_units / e_el / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": pan.numel() + ms.numel(),
           "d2h_bytes_per_step": out_u.numel(),
           "steps": Ke}

    peak, peak_kind = measured_hbm()
    mean_fwd_s = statistics.mean(fwd_ms) / 1e3 / launches_per_step
    achieved = fwd_bytes_per_launch() / mean_fwd_s / 1e9
    kh = kernel_hash()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": KNOWN_TRAFFIC.get(kh),
                "peak_source": f"{peak_kind} (copy bandwidth)",
                "kernel": "fuse_fwd_kernel<uint8, D4, 6>", "kernel_hash": kh,
                "algorithmic_bytes_per_launch": fwd_bytes_per_launch(),
                "mean_launch_ms": mean_fwd_s * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        side = args.cpu_side
        pan_c = pan[:side, :side].cpu().numpy()
        ms_c = ms[:, :side // 2, :side // 2].cpu().numpy()
        rate, cores, secs, reps = oracle_rate(pan_c, ms_c, args.cpu_seconds, 5)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle D4 fusion of the top-left {side}x{side} PAN crop with its "
                         f"{BANDS} MS crops (periodic wrap at the crop), {reps} rep(s), "
                         f"{secs:.1f} s"}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": max_el / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * K, "clocks": clocks,
            "fwd_ms": {"mean": statistics.mean(fwd_ms), "min": min(fwd_ms), "max": max(fwd_ms)},
        }))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
