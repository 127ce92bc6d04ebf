"""dwtfuse_fuse_metrics (fused forward scoring its uint8 product on chip) against
the two separate calls it replaces, dwtfuse_fuse then dwtfuse_metrics, and
against the FP64 oracle.

Bars.  The fused outputs are the same kernels' arithmetic: bit-identical.
ERGAS: squared errors are exact integers, summed exactly: identical.  Q
terms: every window's Q is the same FP32 value, but the sums over windows run
in another order: 1e-6 absolute between the two paths; against the oracle the
test_metrics_gpu bar for uint8 products (2e-6 absolute, ERGAS 1e-12 relative).
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from paper_1803_00737_gb300 import _C

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def ws():
    return torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=DEV)


def scene(H, W, B, seed):
    pan, ms = scenegen.make_scene(H, W, B, seed=seed)
    return pan.to(DEV), ms.to(DEV)


def fused_path(pan, ms, wav, ws, f32=True):
    B, (H, W) = ms.shape[0], pan.shape
    of = torch.full((B, H, W), -1.0, device=DEV) if f32 else None
    ou = torch.zeros((B, H, W), dtype=torch.uint8, device=DEV)
    res = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
    _C.dwtfuse_fuse_metrics(pan, ms, wav, of, ou, ws, res)
    torch.cuda.synchronize()
    return of, ou, res.cpu().numpy()


def separate_path(pan, ms, wav, ws):
    B, (H, W) = ms.shape[0], pan.shape
    of = torch.empty((B, H, W), device=DEV)
    ou = torch.empty((B, H, W), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_fuse(pan, ms, wav, of, ou)
    res = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
    _C.dwtfuse_metrics(ou, ms, pan, ws, res)
    torch.cuda.synchronize()
    return of, ou, res.cpu().numpy()


def agree(a, b):
    assert a[0] == b[0], (a, b)
    assert np.abs(a[1:] - b[1:]).max() <= 1e-6, (a, b)


# Window-aligned and ragged sizes: W off the 128-column strip grid, W = 2 mod 4,
# H/2 odd (a last two-row block of one MS row), partial window rows and columns.
SHAPES = [((64, 64), 3), ((128, 256), 6), ((96, 160), 2), ((130, 258), 4), ((200, 136), 5),
          ((66, 70), 1), ((192, 1030), 6), ((64, 534), 6), ((98, 610), 3), ((128, 256), 8),
          ((130, 258), 7), ((192, 1030), 8), ((64, 534), 7), ((98, 612), 8)]


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape,B", SHAPES)
def test_fused_metrics_equal_separate_calls(wav, shape, B, ws):
    pan, ms = scene(*shape, B, seed=sum(shape) + B)
    f1, u1, r1 = fused_path(pan, ms, wav, ws)
    f2, u2, r2 = separate_path(pan, ms, wav, ws)
    assert torch.equal(f1, f2) and torch.equal(u1, u2)
    agree(r1, r2)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape,B", [((128, 192), 6), ((130, 258), 3), ((96, 610), 5), ((128, 192), 8),
                                     ((98, 610), 7)])
def test_fused_metrics_against_oracle(wav, shape, B, ws):
    pan, ms = scene(*shape, B, seed=3 * sum(shape) + B)
    _, u, r = fused_path(pan, ms, wav, ws, f32=False)
    f, m, p = u.cpu().numpy(), ms.cpu().numpy(), pan.cpu().numpy()
    q, dl, ds = O.qnr(f, list(m), p)
    ref = np.array([O.ergas(f, list(m)), q, dl, ds])
    assert abs(r[0] - ref[0]) <= 1e-12 * ref[0], (r, ref)
    assert np.abs(r[1:] - ref[1:]).max() <= 2e-6, (r, ref)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("B", [7, 8])
def test_seven_and_eight_bands_score_on_chip(wav, B, ws):
    """7 and 8 bands (8 parks one MS row at a time, the pair sums run in two
    passes): the two-call form accepts them, and the outputs and figures
    equal the separate calls' (Q sums to 1e-6)."""
    pan, ms = scene(160, 288, B, seed=B)
    Bn, (H, W) = ms.shape[0], pan.shape
    ou = torch.empty((Bn, H, W), dtype=torch.uint8, device=DEV)
    res = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
    _C.dwtfuse_fuse_and_score(pan, ms, wav, None, ou, ws)
    _C.dwtfuse_score_finish(ms, pan, ou, ws, res)
    torch.cuda.synchronize()
    f2, u2, r2 = separate_path(pan, ms, wav, ws)
    assert torch.equal(ou, u2)
    agree(res.cpu().numpy(), r2)


def test_float_inputs_run_the_separate_kernels(ws):
    pan, ms = scene(64, 96, 3, seed=1)
    pan, ms = pan.float(), ms.float()
    f1, u1, r1 = fused_path(pan, ms, O.D4, ws)
    f2, u2, r2 = separate_path(pan, ms, O.D4, ws)
    assert torch.equal(f1, f2) and torch.equal(u1, u2)
    assert np.array_equal(r1, r2)


def test_uint8_output_only_and_offset_planes(ws):
    """Without the float output, and with the uint8 planes 4 bytes past
    their allocation."""
    pan, ms = scene(128, 384, 6, seed=9)
    B, (H, W) = ms.shape[0], pan.shape
    buf = torch.zeros(B * H * W + 4, dtype=torch.uint8, device=DEV)
    ou = buf[4:].view(B, H, W)
    res = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
    _C.dwtfuse_fuse_metrics(pan, ms, O.D4, None, ou, ws, res)
    torch.cuda.synchronize()
    _, u2, r2 = separate_path(pan, ms, O.D4, ws)
    assert torch.equal(ou, u2) and buf[:4].sum().item() == 0
    agree(res.cpu().numpy(), r2)


def test_larger_scene_and_repeat(ws):
    """2048 x 2048 x 6 (several waves of items, items of several window rows):
    equal to the separate calls, and the same bits on a second call (the
    reduction order is fixed)."""
    pan, ms = scene(2048, 2048, 6, seed=11)
    _, u1, r1 = fused_path(pan, ms, O.D4, ws, f32=False)
    _, u1b, r1b = fused_path(pan, ms, O.D4, ws, f32=False)
    _, u2, r2 = separate_path(pan, ms, O.D4, ws)
    assert torch.equal(u1, u2)
    assert np.array_equal(r1, r1b)
    agree(r1, r2)


def test_graph_capture(ws):
    pan, ms = scene(256, 512, 6, seed=4)
    B, (H, W) = ms.shape[0], pan.shape
    of = torch.empty((B, H, W), device=DEV)
    ou = torch.empty((B, H, W), dtype=torch.uint8, device=DEV)
    res = torch.zeros(4, dtype=torch.float64, device=DEV)
    _C.dwtfuse_fuse_metrics(pan, ms, O.D4, of, ou, ws, res)  # set-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            _C.dwtfuse_fuse_metrics(pan, ms, O.D4, of, ou, ws, res, stream=s)
    res.zero_()
    g.replay()
    torch.cuda.synchronize()
    _, _, r2 = separate_path(pan, ms, O.D4, ws)
    agree(res.cpu().numpy(), r2)


def test_two_call_form(ws):
    """dwtfuse_fuse_and_score then dwtfuse_score_finish = dwtfuse_fuse_metrics."""
    pan, ms = scene(192, 1030, 6, seed=21)
    B, (H, W) = ms.shape[0], pan.shape
    ou = torch.empty((B, H, W), dtype=torch.uint8, device=DEV)
    of = torch.empty((B, H, W), device=DEV)
    res = torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)
    _C.dwtfuse_fuse_and_score(pan, ms, O.D4, of, ou, ws)
    _C.dwtfuse_score_finish(ms, pan, ou, ws, res)
    torch.cuda.synchronize()
    f1, u1, r1 = fused_path(pan, ms, O.D4, ws)
    assert torch.equal(of, f1) and torch.equal(ou, u1)
    assert np.array_equal(res.cpu().numpy(), r1)


def test_two_call_form_rejects_unsupported(ws):
    pan, ms = scene(64, 96, 3, seed=2)
    ou = torch.empty((3, 64, 96), dtype=torch.uint8, device=DEV)
    with pytest.raises(_C.DwtfuseError):  # float inputs are scored by the separate passes only
        _C.dwtfuse_fuse_and_score(pan.float(), ms.float(), O.D4, None, ou, ws)
    pan9, ms9 = scene(64, 96, 9, seed=2)
    ou9 = torch.empty((9, 64, 96), dtype=torch.uint8, device=DEV)
    with pytest.raises(_C.DwtfuseError):  # the metrics take at most 8 bands
        _C.dwtfuse_fuse_and_score(pan9, ms9, O.D4, None, ou9, ws)


def test_benchmark_step_full_size(ws):
    """The benchmark step as timed (D4, PAN 16384^2 uint8, 6 MS bands 8192^2,
    float32 + uint8 outputs, one dwtfuse_fuse_metrics call): outputs equal the
    plain forward's bits; every pixel of every float32 band is within 5e-4 of
    the whole-image oracle, every uint8 pixel follows the rounding rule on the
    oracle's value (off by one only within 5e-4 of a tie); the metrics equal
    the oracle's on the whole images."""
    from tests.test_fuse_gpu import check_u8
    H = W = 16384
    pan, ms = scenegen.make_scene(H, W, 6, seed=0, blob_scale=16.0, device=DEV)
    of, ou, r = fused_path(pan, ms, O.D4, ws)
    f2 = torch.empty_like(of)
    u2 = torch.empty_like(ou)
    _C.dwtfuse_fuse(pan, ms, O.D4, f2, u2)
    torch.cuda.synchronize()
    assert torch.equal(of, f2) and torch.equal(ou, u2)
    del f2, u2
    p, m = pan.cpu().numpy(), ms.cpu().numpy()
    pf = p.astype(np.float64)
    for b in range(6):
        ref = O.fuse(pf, [m[b]], O.D4)[0]
        got = of[b].cpu().numpy()
        err = float(np.abs(got - ref).max())
        assert err <= 5e-4, (b, err)
        del got
        check_u8(ou[b].cpu().numpy(), ref, O.D4)
        del ref
    del pf
    f = ou.cpu().numpy()
    q, dl, ds = O.qnr(f, list(m), p)
    ref = np.array([O.ergas(f, list(m)), q, dl, ds])
    assert abs(r[0] - ref[0]) <= 1e-12 * ref[0], (r, ref)
    assert np.abs(r[1:] - ref[1:]).max() <= 2e-6, (r, ref)


@pytest.mark.parametrize("B", [2, 6, 8])
def test_two_streams_at_once(ws, B):
    """Two scoring calls on two streams at the same time give the results of
    the calls one after the other.  Each CTA of the scoring kernel allocates
    tensor memory (TMEM) and takes more than half of an SM's registers, so
    CTAs of the two launches never share an SM."""
    pan, ms = scene(512, 1024, B, seed=40 + B)
    ws2 = torch.empty_like(ws)
    f1, u1, r1 = fused_path(pan, ms, O.D4, ws)
    Bn, (H, W) = ms.shape[0], pan.shape
    outs = [(torch.empty((Bn, H, W), device=DEV), torch.empty((Bn, H, W), dtype=torch.uint8, device=DEV),
             torch.full((4,), float("nan"), dtype=torch.float64, device=DEV)) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for k in range(3):
        for (of, ou, res), st, w in zip(outs, streams, (ws, ws2)):
            with torch.cuda.stream(st):
                _C.dwtfuse_fuse_metrics(pan, ms, O.D4, of, ou, w, res, stream=st)
    torch.cuda.synchronize()
    for of, ou, res in outs:
        assert torch.equal(of, f1) and torch.equal(ou, u1)
        assert np.array_equal(res.cpu().numpy(), r1)
