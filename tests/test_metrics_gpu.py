"""Parity of the GPU quality metrics (ERGAS, QNR, D_lambda, D_s) with the FP64
oracle on the same fused product.

Tolerances.  uint8 products: every window sum of shifted values is an exact
integer and the numerators (n Sxy - Sx Sy, n Sxx - Sx^2) are exact int64, so
the only rounding is the final FP32 ratio, <= 8 roundings ~5e-7 of |Q| <= 1 per
window; D_lambda and D_s are means of differences of such means: 2e-6
absolute; ERGAS sums are exact integers: 1e-12 relative.  float32 products:
per-lane FP32 sums of up to 128 shifted values (|v| <= 128) carry relative
error ~1e-7 of sums up to 2^21, i.e. ~1e-5 of a window's covariance for weak
texture; averaged over windows the bar is 2e-5 absolute on QNR, D_lambda, D_s
and 1e-6 relative on ERGAS.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from paper_1803_00737_gb300 import _C, fuse

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def ws():
    return torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=DEV)


def gpu_metrics(fused, ms, pan, ws):
    out = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
    _C.dwtfuse_metrics(fused, ms, pan, ws, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def ref_metrics(fused, ms, pan):
    f, m, p = fused.cpu().numpy(), ms.cpu().numpy(), pan.cpu().numpy()
    q, dl, ds = O.qnr(f, list(m), p)
    return np.array([O.ergas(f, list(m)), q, dl, ds])


def check(got, ref, f32):
    tol_q = 2e-5 if f32 else 2e-6
    assert abs(got[0] - ref[0]) <= (1e-6 if f32 else 1e-12) * max(1.0, abs(ref[0])), (got, ref)
    assert np.abs(got[1:] - ref[1:]).max() <= tol_q, (got, ref)


@pytest.mark.parametrize("wav", [0, 1])
@pytest.mark.parametrize("shape,B", [((64, 64), 3), ((128, 192), 6), ((130, 258), 4),
                                     ((200, 136), 8), ((96, 512), 1), ((66, 70), 2),
                                     ((96, 1056), 5), ((160, 528), 7), ((64, 80), 2),
                                     ((96, 610), 6), ((64, 534), 8), ((130, 4070), 3),
                                     ((72, 1048), 4)])
def test_metrics_u8_product(wav, shape, B, ws):
    H, W = shape
    pan, ms = scenegen.make_scene(H, W, B, seed=H + W + B)
    pan, ms = pan.to(DEV), ms.to(DEV)
    _, u8 = fuse(pan, ms, wav, f32=False, u8=True)
    check(gpu_metrics(u8, ms, pan, ws), ref_metrics(u8, ms, pan), False)


@pytest.mark.parametrize("shape,B", [((64, 128), 3), ((130, 258), 5), ((256, 256), 8)])
def test_metrics_f32_product(shape, B, ws):
    H, W = shape
    pan, ms = scenegen.make_scene(H, W, B, seed=7)
    pan, ms = pan.to(DEV), ms.to(DEV)
    f32, _ = fuse(pan, ms, 1, f32=True, u8=False)
    check(gpu_metrics(f32, ms, pan, ws), ref_metrics(f32, ms, pan), True)


def test_metrics_f32_inputs(ws):
    rng = np.random.default_rng(3)
    pan = torch.from_numpy(rng.uniform(0, 255, (128, 160)).astype(np.float32)).to(DEV)
    ms = torch.from_numpy(rng.uniform(0, 255, (3, 64, 80)).astype(np.float32)).to(DEV)
    f32, _ = fuse(pan, ms, 1)
    check(gpu_metrics(f32, ms, pan, ws), ref_metrics(f32, ms, pan), True)


def _offset_copy(t, off):
    buf = torch.zeros(t.numel() + off, dtype=t.dtype, device=DEV)
    buf[off:].copy_(t.reshape(-1))
    return buf[off:].view(t.shape)


@pytest.mark.parametrize("W", [544, 1056, 610])
def test_u8_aligned_and_misaligned_planes_agree(W, ws):
    """The 8-bit paths stage 16-byte chunks and shift rows into place; planes at
    odd byte offsets (MS bands starting mid-chunk, copied byte by byte at the
    plane start) give the same figures as aligned planes."""
    H, B = 96, 4
    pan, ms = scenegen.make_scene(H, W, B, seed=9)
    pan, ms = pan.to(DEV), ms.to(DEV)
    _, u8 = fuse(pan, ms, 1, f32=False, u8=True)
    fast = gpu_metrics(u8, ms, pan, ws)
    slow = gpu_metrics(_offset_copy(u8, 2), [_offset_copy(m, 1) for m in ms], pan, ws)
    np.testing.assert_allclose(fast, slow, rtol=0, atol=1e-12)


@pytest.mark.parametrize("W", [512, 614])
def test_u8_path_equals_float_path(W, ws):
    """The same integer-valued product through the 8-bit (dp4a) path and the
    float path: equal within the float path's bar."""
    H, B = 96, 5
    pan, ms = scenegen.make_scene(H, W, B, seed=12)
    pan, ms = pan.to(DEV), ms.to(DEV)
    _, u8 = fuse(pan, ms, 1, f32=False, u8=True)
    a = gpu_metrics(u8, ms, pan, ws)
    b = gpu_metrics(u8.float(), ms.float(), pan.float(), ws)
    assert abs(a[0] - b[0]) <= 1e-6 * a[0]
    assert np.abs(a[1:] - b[1:]).max() <= 2e-5


def test_sync_entry_points_agree(ws):
    pan, ms = scenegen.make_scene(128, 128, 4, seed=1)
    pan, ms = pan.to(DEV), ms.to(DEV)
    _, u8 = fuse(pan, ms, 0, f32=False, u8=True)
    m = gpu_metrics(u8, ms, pan, ws)
    e = _C.dwtfuse_ergas(u8, ms, ws)
    q, dl, ds = _C.dwtfuse_qnr(u8, ms, pan, ws)
    assert e == m[0] and q == m[1] and dl == m[2] and ds == m[3]


def test_replicated_ms_gives_zero_ergas(ws):
    H, W, B = 96, 128, 3
    pan, ms = scenegen.make_scene(H, W, B, seed=4)
    rep = ms.repeat_interleave(2, dim=1).repeat_interleave(2, dim=2).contiguous()
    got = gpu_metrics(rep.to(DEV), ms.to(DEV), pan.to(DEV), ws)
    assert got[0] == 0.0


def test_identical_bands_give_qnr_one(ws):
    """F_l = PAN and MS_l = PAN~ for every band: every Q is 1 (constant windows
    included), so D_lambda = D_s = 0 and QNR = 1 (float data: the final FP32
    ratio of each window leaves ~1e-7)."""
    H = W = 128
    pan = scenegen.make_pan(H, W, seed=5)
    pan[:32, :32] = 77  # a constant window on both sides
    lo = torch.nn.functional.avg_pool2d(pan.float().view(1, 1, H, W), 2).view(H // 2, W // 2)
    fused = torch.stack([pan.float()] * 3).to(DEV)
    ms = torch.stack([lo] * 3).to(DEV)
    got = gpu_metrics(fused, ms, pan.float().to(DEV), ws)
    np.testing.assert_allclose(got[1:], [1.0, 0.0, 0.0], atol=1e-6)


def test_metrics_deterministic(ws):
    pan, ms = scenegen.make_scene(512, 512, 6, seed=2)
    pan, ms = pan.to(DEV), ms.to(DEV)
    f32, _ = fuse(pan, ms, 1)
    a = gpu_metrics(f32, ms, pan, ws)
    b = gpu_metrics(f32, ms, pan, ws)
    assert np.array_equal(a, b)


def test_rejects_bad_window_and_sizes(ws):
    pan, ms = scenegen.make_scene(64, 64, 2, seed=0)
    pan, ms = pan.to(DEV), ms.to(DEV)
    fused = torch.zeros((2, 64, 64), dtype=torch.uint8, device=DEV)
    out = torch.zeros(4, dtype=torch.float64, device=DEV)
    with pytest.raises(_C.DwtfuseError) as e:
        _C.dwtfuse_metrics(fused, ms, pan, ws, out, window=16)
    assert e.value.status == _C.ESHAPE
    small_pan, small_ms = scenegen.make_scene(40, 64, 2, seed=0)
    with pytest.raises(_C.DwtfuseError) as e:
        _C.dwtfuse_metrics(torch.zeros((2, 40, 64), dtype=torch.uint8, device=DEV),
                           small_ms.to(DEV), small_pan.to(DEV), ws, out)
    assert e.value.status == _C.ESHAPE
    # ERGAS alone has no window requirement
    e_small = _C.dwtfuse_ergas(torch.zeros((2, 40, 64), dtype=torch.uint8, device=DEV),
                               small_ms.to(DEV), ws)
    assert np.isfinite(e_small)


def test_config1_metrics_full_size(ws):
    """The benchmark workload (D4, PAN 16384^2, 6 bands): metrics of the uint8
    product on the GPU equal the oracle's on the whole images."""
    H = W = 16384
    pan, ms = scenegen.make_scene(H, W, 6, seed=0, blob_scale=16.0, device=DEV)
    _, u8 = fuse(pan, ms, 1, f32=False, u8=True)
    got = gpu_metrics(u8, ms, pan, ws)
    ref = ref_metrics(u8, ms, pan)
    check(got, ref, False)


def test_bounded_wait_gives_up_and_the_context_survives(ws):
    """Rows off the 16-byte grid are staged by bulk copies whose mbarrier waits
    are bounded.  With the test hook one warp waits on 16 bytes that no copy
    sends: after about a second the call reports DWTFUSE_ETIMEOUT (the async
    form NaN figures), and the next call on the same context is exact again."""
    H, W, B = 64, 534, 3  # W % 16 != 0: the staged path
    pan, ms = scenegen.make_scene(H, W, B, seed=12, device=DEV)
    u8 = torch.empty((B, H, W), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_fuse(pan, ms, 1, None, u8)
    ref = _C.dwtfuse_ergas(u8, ms, ws)
    _C.dwtfuse_set_metric_wait_test(True)
    try:
        with pytest.raises(_C.DwtfuseError) as err:
            _C.dwtfuse_ergas(u8, ms, ws)
        assert err.value.status == _C.ETIMEOUT
        out = torch.zeros(4, dtype=torch.float64, device=DEV)
        _C.dwtfuse_metrics(u8, ms, pan, ws, out)
        torch.cuda.synchronize()
        assert torch.isnan(out).all()
    finally:
        _C.dwtfuse_set_metric_wait_test(False)
    assert _C.dwtfuse_ergas(u8, ms, ws) == ref
    got = gpu_metrics(u8, ms, pan, ws)
    check(got, ref_metrics(u8, ms, pan), False)
