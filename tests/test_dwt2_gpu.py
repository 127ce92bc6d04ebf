"""Standalone 2D DWT and inverse on the GPU against the oracle's literal
Eq. 1-16 transforms (whose matrices are pinned to the textbook filter bank).
Haar on 8-bit images is exact (multiples of 1/4); D4 coefficients of 0-255
images are within 5e-4, and so is the inverse of 0-255-scale coefficients;
inverse(forward(x)) = x."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1803_00737_gb300 import _C

pytestmark = pytest.mark.gpu
DEV = "cuda"
SHAPES = [(4, 4), (6, 18), (10, 6), (64, 128), (66, 258), (130, 250), (34, 814), (200, 384)]


@pytest.mark.parametrize("wav", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_dwt2_matches_oracle(wav, shape):
    rng = np.random.default_rng(hash(shape) % 1000)
    img = rng.integers(0, 256, shape).astype(np.uint8)
    Z = torch.empty(shape, device=DEV)
    _C.dwtfuse_dwt2(torch.from_numpy(img).to(DEV), wav, Z)
    torch.cuda.synchronize()
    ref = O.dwt2(img.astype(np.float64), wav)
    got = Z.cpu().numpy()
    if wav == 0:
        np.testing.assert_array_equal(got, ref.astype(np.float32))
    else:
        assert np.abs(got - ref).max() <= 5e-4


@pytest.mark.parametrize("wav", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_idwt2_matches_oracle(wav, shape):
    """Coefficients on the 0-255 scale (the oracle's transform of an 8-bit
    image, every coefficient moved by N(0, 8) so the inverse is not the image)
    invert to within the D4 bar of 5e-4 (max-abs); Haar of quarter-integer
    coefficients is exact."""
    rng = np.random.default_rng(7 + hash(shape) % 1000)
    img = rng.integers(0, 256, shape).astype(np.float64)
    Z = O.dwt2(img, wav) + rng.normal(0, 8, shape)
    if wav == 0:
        Z = np.round(Z * 4) / 4
    Z = Z.astype(np.float32)
    out = torch.empty(shape, device=DEV)
    _C.dwtfuse_idwt2(torch.from_numpy(Z).to(DEV), wav, out)
    torch.cuda.synchronize()
    ref = O.idwt2(Z.astype(np.float64), wav)
    if wav == 0:
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), ref)
    else:
        assert np.abs(out.cpu().numpy() - ref).max() <= 5e-4


@pytest.mark.parametrize("wav", [0, 1])
def test_round_trip_and_u8_output(wav):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (96, 136)).astype(np.uint8)
    x = torch.from_numpy(img).to(DEV)
    Z = torch.empty((96, 136), device=DEV)
    _C.dwtfuse_dwt2(x, wav, Z)
    f = torch.empty((96, 136), device=DEV)
    u = torch.empty((96, 136), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_idwt2(Z, wav, f, u)
    torch.cuda.synchronize()
    assert (f.cpu() - x.cpu().float()).abs().max().item() <= (0 if wav == 0 else 1e-3)
    assert torch.equal(u.cpu(), x.cpu())


def test_dwt2_float_input_and_fusion_consistency():
    """Fusing = replacing the LL quadrant of dwtfuse_dwt2's output and inverting."""
    rng = np.random.default_rng(4)
    H, W = 64, 96
    pan = rng.integers(0, 256, (H, W)).astype(np.uint8)
    ms = rng.integers(0, 256, (1, H // 2, W // 2)).astype(np.uint8)
    Z = torch.empty((H, W), device=DEV)
    _C.dwtfuse_dwt2(torch.from_numpy(pan).float().to(DEV), 1, Z)
    Z[: H // 2, : W // 2] = 2.0 * torch.from_numpy(ms[0]).float().to(DEV)
    out = torch.empty((H, W), device=DEV)
    _C.dwtfuse_idwt2(Z, 1, out)
    fused = torch.empty((1, H, W), device=DEV)
    _C.dwtfuse_fuse(torch.from_numpy(pan).to(DEV), torch.from_numpy(ms).to(DEV), 1, fused, None)
    torch.cuda.synchronize()
    assert (out - fused[0]).abs().max().item() <= 5e-4


def test_dwt2_full_size_sampled_and_round_trip():
    """16384^2 uint8 image, D4: sampled coefficients of every quadrant against
    the point-wise oracle, and inverse(forward(x)) = x at full size."""
    H = W = 16384
    g = torch.Generator(device=DEV)
    g.manual_seed(0)
    img = torch.randint(0, 256, (H, W), generator=g, device=DEV, dtype=torch.uint8)
    Z = torch.empty((H, W), device=DEV)
    _C.dwtfuse_dwt2(img, 1, Z)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    ii = np.concatenate([[0, H // 2 - 1, H // 2, H - 1], rng.integers(0, H, 400)])
    jj = np.concatenate([[W - 1, 0, W // 2, W // 2 - 1], rng.integers(0, W, 400)])
    ref = O.dwt2_points(img.cpu().numpy(), 1, ii, jj)
    got = Z[torch.from_numpy(ii).to(DEV), torch.from_numpy(jj).to(DEV)].cpu().numpy()
    assert np.abs(got - ref).max() <= 5e-4
    back = torch.empty((H, W), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_idwt2(Z, 1, None, back)
    torch.cuda.synchronize()
    assert torch.equal(back, img)


# Widths the staged forward takes for D4 (W % 8 == 0, a 16-byte-aligned
# coefficient plane and a last 1024-column strip at least 7/8 full; Haar runs
# warp items there):
# one and several strips, a ragged last strip, odd H/2, both step parities.
STAGED = [(34, 1024), (66, 2048), (130, 1976), (20, 3064), (6, 4096)]


@pytest.mark.parametrize("wav", [0, 1])
@pytest.mark.parametrize("shape", STAGED)
def test_staged_transforms_match_oracle(wav, shape):
    """The staged forward (uint8 and float images) against the oracle, the
    inverse at the same widths (float and uint8 outputs), and the round
    trip."""
    rng = np.random.default_rng(sum(shape) + wav)
    img = rng.integers(0, 256, shape).astype(np.uint8)
    x = torch.from_numpy(img).to(DEV)
    Z = torch.empty(shape, device=DEV)
    Zf = torch.empty(shape, device=DEV)
    _C.dwtfuse_dwt2(x, wav, Z)
    _C.dwtfuse_dwt2(x.float(), wav, Zf)
    torch.cuda.synchronize()
    ref = O.dwt2(img.astype(np.float64), wav)
    for got in (Z, Zf):
        g = got.cpu().numpy()
        if wav == 0:
            np.testing.assert_array_equal(g, ref.astype(np.float32))
        else:
            assert np.abs(g - ref).max() <= 5e-4
    C = O.dwt2(img.astype(np.float64), wav) + rng.normal(0, 8, shape)
    if wav == 0:
        C = np.round(C * 4) / 4
    C32 = torch.from_numpy(C.astype(np.float32)).to(DEV)
    f = torch.empty(shape, device=DEV)
    u = torch.empty(shape, dtype=torch.uint8, device=DEV)
    _C.dwtfuse_idwt2(C32, wav, f, u)
    torch.cuda.synchronize()
    iref = O.idwt2(C.astype(np.float32).astype(np.float64), wav)
    if wav == 0:
        np.testing.assert_array_equal(f.cpu().numpy().astype(np.float64), iref)
        np.testing.assert_array_equal(u.cpu().numpy(), O.to_u8(iref))
    else:
        assert np.abs(f.cpu().numpy() - iref).max() <= 5e-4
        du = np.abs(u.cpu().numpy().astype(int) - O.to_u8(iref).astype(int))
        assert du.max() <= 1
    back = torch.empty(shape, dtype=torch.uint8, device=DEV)
    backf = torch.empty(shape, device=DEV)
    _C.dwtfuse_idwt2(Z, wav, backf, back)
    torch.cuda.synchronize()
    assert torch.equal(back, x)


def test_staged_transform_kernels_are_launched():
    """Kernel names seen by the profiler: a 2048-wide image runs the staged
    forward, a 1030-wide one the warp-item forward; the inverse runs warp
    items at both widths."""
    prof = pytest.importorskip("torch.profiler")
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]):  # the first session can miss kernels
        torch.zeros(1, device=DEV).add_(1)
        torch.cuda.synchronize()
    names = {}
    for W in (2048, 1030):
        x = torch.zeros((8, W), dtype=torch.uint8, device=DEV)
        Z = torch.empty((8, W), device=DEV)
        out = torch.empty((8, W), device=DEV)
        torch.cuda.synchronize()
        with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as pr:
            _C.dwtfuse_dwt2(x, 1, Z)
            _C.dwtfuse_idwt2(Z, 1, out)
            torch.cuda.synchronize()
        names[W] = {e.name for e in pr.events() if "dwt2" in e.name}
    if not names[2048] and not names[1030]:
        pytest.skip("profiler recorded no kernels")
    assert sum("dwt2_staged_kernel" in n for n in names[2048]) == 1, names
    assert not any("dwt2_staged_kernel" in n for n in names[1030]), names
