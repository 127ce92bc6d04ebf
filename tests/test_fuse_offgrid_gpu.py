"""Parity of the fused forward with the FP64 oracle on output rows off the
16-byte and 32-byte grids.

Widths W = 2 mod 4 (odd rows 2 pixels past a 16-byte boundary: the
shifted-row instance), W = 0 mod 4 not a multiple of 32, several 128-column
strips with a ragged last one, and output planes at offsets from their
allocation (every band plane and row then has its own phase; a float offset
of 8 bytes leaves the 16-byte grid and takes the pixel-pair path).  Guard
regions around the outputs check that nothing is written outside them.
Bars as in test_fuse_gpu: Haar bit-exact, D4 max-abs 5e-4, uint8 = clamp +
round-half-even (D4: off by one only at a tie).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1803_00737_gb300 import _C

from test_fuse_gpu import D4_TOL, check, rand_scene

pytestmark = pytest.mark.gpu
DEV = "cuda"


def run(pan, ms, wav, f32=True, u8=True, f_off=0, u_off=0, guard=256):
    """Fused outputs written into flat buffers at element offsets f_off / u_off
    past a guard region; returns the outputs and whether the guards held."""
    B, H, W = ms.shape[0], pan.shape[0], pan.shape[1]
    n = B * H * W
    p = torch.from_numpy(np.ascontiguousarray(pan)).to(DEV)
    m = torch.from_numpy(np.ascontiguousarray(ms)).to(DEV)
    fbuf = torch.full((n + 2 * guard + f_off,), -7.0, device=DEV) if f32 else None
    ubuf = torch.full((n + 2 * guard + u_off,), 77, dtype=torch.uint8, device=DEV) if u8 else None
    of = fbuf[guard + f_off: guard + f_off + n].view(B, H, W) if f32 else None
    ou = ubuf[guard + u_off: guard + u_off + n].view(B, H, W) if u8 else None
    _C.dwtfuse_fuse(p, m, wav, of, ou)
    torch.cuda.synchronize()
    ok = True
    if f32:
        ok &= bool((fbuf[:guard + f_off] == -7).all()) and bool((fbuf[guard + f_off + n:] == -7).all())
    if u8:
        ok &= bool((ubuf[:guard + u_off] == 77).all()) and bool((ubuf[guard + u_off + n:] == 77).all())
    return (of.cpu().numpy() if f32 else None), (ou.cpu().numpy() if u8 else None), ok


# Widths: W = 2 mod 4 and W = 0 mod 4 off the sector grid; one strip, a
# strip boundary exactly at W, and many strips with a ragged last one.
WIDTHS = [6, 94, 100, 130, 256 + 2, 1030, 1092, 2050, 3000, 4092, 4094]


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("W", WIDTHS)
def test_offgrid_widths(wav, W):
    pan, ms = rand_scene(10, W, 3, seed=W)
    f, u, ok = run(pan, ms, wav)
    assert ok
    check(pan, ms, wav, f, u)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("B", [1, 2, 5, 6, 7, 8, 11])
def test_offgrid_band_counts(wav, B):
    """W = 2 mod 4 for every band count (the shifted-row instance takes
    balanced chunks of at most 6 bands: 7 = 4 + 3, 8 = 4 + 4, 11 = 6 + 5)."""
    pan, ms = rand_scene(6, 2050, B, seed=B)
    f, u, ok = run(pan, ms, wav)
    assert ok
    check(pan, ms, wav, f, u)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("outs", ["f", "u"])
def test_offgrid_single_output(wav, outs):
    pan, ms = rand_scene(8, 1030, 4, seed=3)
    f, u, ok = run(pan, ms, wav, f32=outs == "f", u8=outs == "u")
    assert ok
    check(pan, ms, wav, f, u)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("f_off,u_off", [(4, 4), (4, 0), (0, 68), (36, 12), (2, 2)])
def test_offgrid_plane_offsets(wav, f_off, u_off):
    """Aligned width, planes moved off their allocation's alignment."""
    pan, ms = rand_scene(8, 2048, 3, seed=f_off + u_off)
    f, u, ok = run(pan, ms, wav, f_off=f_off, u_off=u_off)
    assert ok
    check(pan, ms, wav, f, u)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_offgrid_f32_inputs(wav):
    rng = np.random.default_rng(11)
    pan = (rng.random((12, 2050)) * 255).astype(np.float32)
    ms = (rng.random((5, 6, 1025)) * 255).astype(np.float32)
    f, u, ok = run(pan, ms, wav)
    assert ok
    ref = O.fuse(pan.astype(np.float64), ms.astype(np.float64), wav)
    tol = 2e-4 if wav == O.HAAR else D4_TOL
    assert np.abs(f.astype(np.float64) - ref).max() <= tol


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("rows", [1, 3, 64])
def test_offgrid_rows_per_item(wav, rows):
    """Item heights down to one MS row (D4: every item has its own prologue)
    give the same result as the default on a W = 2 mod 4 scene."""
    pan, ms = rand_scene(70, 1030, 3, seed=9)
    base, _, _ = run(pan, ms, wav, u8=False)
    _C.dwtfuse_set_rows_per_item(rows)
    try:
        got, _, ok = run(pan, ms, wav, u8=False)
    finally:
        _C.dwtfuse_set_rows_per_item(0)
    assert ok
    np.testing.assert_array_equal(got, base)


def test_offgrid_equals_aligned():
    """The same scene written to planes on and off the sector grid gives
    identical bits."""
    pan, ms = rand_scene(16, 2048, 6, seed=5)
    a, ua, _ = run(pan, ms, O.D4)
    b, ub, ok = run(pan, ms, O.D4, f_off=4, u_off=4)
    assert ok
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ua, ub)


def test_shifted_row_instance_is_launched():
    """Kernel names seen by the profiler: a 1030-wide scene (W = 2 mod 4) runs
    the shifted-row instance, a 1024-wide one (rows on the 16-byte grid, float
    output) the staged kernel."""
    prof = pytest.importorskip("torch.profiler")
    names = {}
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]):  # the first session can miss kernels
        torch.zeros(1, device=DEV).add_(1)
        torch.cuda.synchronize()
    for W in (1024, 1030):
        pan, ms = rand_scene(8, W, 2, seed=1)
        p, m = torch.from_numpy(pan).to(DEV), torch.from_numpy(ms).to(DEV)
        of = torch.empty((2, 8, W), device=DEV)
        ou = torch.empty((2, 8, W), dtype=torch.uint8, device=DEV)
        torch.cuda.synchronize()
        with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as pr:
            _C.dwtfuse_fuse(p, m, O.D4, of, ou)
            torch.cuda.synchronize()
        names[W] = {e.name for e in pr.events() if "fuse" in e.name}
    if not names[1024] and not names[1030]:
        pytest.skip("profiler recorded no kernels")
    assert any("fuse_staged_kernel" in n for n in names[1024]), names
    assert any("fuse_fwd_kernel" in n and "true>" in n for n in names[1030]), names


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape,B", [((64, 1024), 6), ((34, 2048), 4), ((66, 1920), 3), ((40, 4092), 5)])
def test_staging_knob_gives_the_same_bits(wav, shape, B):
    """dwtfuse_set_fuse_staging(0) runs the warp-strip kernel on scenes the
    staged kernel takes; the outputs are the same bits, and the staged run
    matches the oracle."""
    pan, ms = rand_scene(*shape, B, seed=sum(shape) + B)
    try:
        a, ua, ok_a = run(pan, ms, wav)
        _C.dwtfuse_set_fuse_staging(False)
        b, ub, ok_b = run(pan, ms, wav)
    finally:
        _C.dwtfuse_set_fuse_staging(True)
    assert ok_a and ok_b
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ua, ub)
    check(pan, ms, wav, a, ua)
