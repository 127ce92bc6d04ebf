"""Parity of the CUDA adjoint (dwtfuse_fuse_backward) and of the autograd
Function with the oracle's transposed fusion, FP64 finite differences and the
explicit adjoint matrix.

Tolerance: gradients are sums of at most ~16 B products of FP32 values of
order |g|; the bar is max-abs <= 1e-4 * max(1, max|g_ref|) (FP32 rounding of
such sums is ~1e-6 relative)."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from paper_1803_00737_gb300 import _C
from paper_1803_00737_gb300.autograd import DWTFuseFn

pytestmark = pytest.mark.gpu
DEV = "cuda"


def gpu_backward(G, wav):
    g = torch.from_numpy(G.astype(np.float32)).to(DEV)
    B, H, W = G.shape
    gp = torch.empty((H, W), device=DEV)
    gm = torch.empty((B, H // 2, W // 2), device=DEV)
    _C.dwtfuse_fuse_backward(g, wav, gp, gm)
    torch.cuda.synchronize()
    return gp.cpu().numpy().astype(np.float64), gm.cpu().numpy().astype(np.float64)


def assert_close(got, ref):
    tol = 1e-4 * max(1.0, np.abs(ref).max())
    err = np.abs(got - ref).max()
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape", [(4, 4), (6, 18), (10, 6), (64, 64), (66, 258), (130, 250),
                                   (12, 814)])
@pytest.mark.parametrize("B", [1, 4, 6, 9])
def test_backward_matches_oracle_adjoint(wav, shape, B):
    rng = np.random.default_rng(abs(hash((wav, shape, B))) % 2**32)
    G = rng.standard_normal((B, *shape))
    gp, gm = gpu_backward(G, wav)
    rp, rm = O.fuse_adjoint(G, wav)
    assert_close(gp, rp)
    assert_close(gm, rm)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_backward_equals_explicit_adjoint_matrix_16(wav):
    """Columns of the GPU backward on unit vectors form the transposed Jacobian
    built column by column from the forward oracle (16 x 16, 1 band)."""
    H = W = 16
    n, m = H * W, (H // 2) * (W // 2)
    J = np.empty((n, n + m))
    zp, zm = np.zeros((H, W)), np.zeros((1, H // 2, W // 2))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1
        J[:, k] = O.fuse(e.reshape(H, W), zm, wav)[0].ravel()
    for k in range(m):
        e = np.zeros(m)
        e[k] = 1
        J[:, n + k] = O.fuse(zp, e.reshape(1, H // 2, W // 2), wav)[0].ravel()
    K = np.empty((n + m, n))
    for k in range(n):
        e = np.zeros((1, n))
        e[0, k] = 1
        gp, gm = gpu_backward(e.reshape(1, H, W), wav)
        K[:, k] = np.concatenate([gp.ravel(), gm.ravel()])
    assert np.abs(K - J.T).max() <= 1e-5


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_gradients_vs_fp64_finite_differences_64(wav):
    """L = <T, fuse(P, M)>: GPU gradients vs central FP64 differences of the
    oracle forward on a 64 x 64 crop with 4 bands (sampled coordinates)."""
    H = W = 64
    B = 4
    pan, ms = scenegen.make_scene(H, W, B, seed=3)
    pan = pan.numpy().astype(np.float64)
    ms = ms.numpy().astype(np.float64)
    T = np.random.default_rng(0).standard_normal((B, H, W))
    gp, gm = gpu_backward(T, wav)
    rng = np.random.default_rng(1)
    for k in rng.choice(H * W, 48, replace=False):
        d = np.zeros(H * W)
        d[k] = 1.0
        d = d.reshape(H, W)
        fd = ((O.fuse(pan + d, ms, wav) - O.fuse(pan - d, ms, wav)) * T).sum() / 2
        assert abs(fd - gp.ravel()[k]) <= 1e-4 * max(1, abs(fd))
    for k in rng.choice(B * (H // 2) * (W // 2), 48, replace=False):
        d = np.zeros(B * (H // 2) * (W // 2))
        d[k] = 1.0
        d = d.reshape(B, H // 2, W // 2)
        fd = ((O.fuse(pan, ms + d, wav) - O.fuse(pan, ms - d, wav)) * T).sum() / 2
        assert abs(fd - gm.ravel()[k]) <= 1e-4 * max(1, abs(fd))


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("N,B,H,W", [(2, 4, 64, 96), (3, 9, 66, 130)])
def test_autograd_mse_loss(wav, N, B, H, W):
    """Batches of D4/Haar scenes as float32 (the second: 9 bands, three band
    chunks in the batched adjoint, W = 2 mod 4); loss = MSE to a seeded target;
    the gradients equal the oracle adjoint of 2 (F - T) / numel."""
    pans, mss = [], []
    for i in range(N):
        p, m = scenegen.make_scene(H, W, B, seed=i)
        pans.append(p.float())
        mss.append(m.float())
    pan = torch.stack(pans).to(DEV).requires_grad_(True)
    ms = torch.stack(mss).to(DEV).requires_grad_(True)
    target = scenegen.target_like((N, B, H, W), seed=1000).to(DEV) * 20 + 120
    out = DWTFuseFn.apply(pan, ms, wav)
    loss = torch.nn.functional.mse_loss(out, target)
    loss.backward()
    F = out.detach().cpu().numpy().astype(np.float64)
    dF = 2.0 * (F - target.cpu().numpy()) / F.size
    for i in range(N):
        ref = O.fuse(pan[i].detach().cpu().numpy(), ms[i].detach().cpu().numpy(), wav)
        assert np.abs(F[i] - ref).max() <= 5e-4
        rp, rm = O.fuse_adjoint(dF[i], wav)
        assert_close(pan.grad[i].cpu().numpy().astype(np.float64), rp)
        assert_close(ms.grad[i].cpu().numpy().astype(np.float64), rm)


def test_autograd_unbatched_shapes():
    pan = torch.rand((32, 64), device=DEV, requires_grad=True)
    ms = torch.rand((3, 16, 32), device=DEV, requires_grad=True)
    out = DWTFuseFn.apply(pan, ms, O.D4)
    assert out.shape == (3, 32, 64)
    out.sum().backward()
    assert pan.grad.shape == pan.shape and ms.grad.shape == ms.shape


def test_autograd_config3_elementwise():
    """The autograd workload as timed: a batch of 8 scenes, PAN 4096^2 and 4 MS
    bands 2048^2 generated as 8-bit scenes and cast to float32, D4, through
    DWTFuseFn (batched forward and batched adjoint).  With a seeded output
    gradient, grad_PAN and every band's grad_MS equal the oracle's point-wise
    adjoint element by element on two seeded 256 x 256 windows per scene and on
    every scene's wrap rows and columns; the fused bands match the point-wise
    oracle on the same windows."""
    from tests.parity_windows import adjoint_region_error, forward_region_error, regions
    N, B, H, W = 8, 4, 4096, 4096
    pans, mss = [], []
    for i in range(N):
        p, m = scenegen.make_scene(H, W, B, seed=i, device=DEV)
        pans.append(p.float())
        mss.append(m.float())
    pan = torch.stack(pans).requires_grad_(True)
    ms = torch.stack(mss).requires_grad_(True)
    del pans, mss
    G = scenegen.target_like((N, B, H, W), seed=77, device=DEV)
    out = DWTFuseFn.apply(pan, ms, O.D4)
    out.backward(G)
    torch.cuda.synchronize()
    for i in range(N):
        pan_h = pan[i].detach().cpu().numpy().astype(np.float64)
        ms_h = ms[i].detach().cpu().numpy().astype(np.float64)
        for k, reg in enumerate(regions(H, W, seed=100 + i)):
            e = adjoint_region_error(G[i], pan.grad[i], ms.grad[i], O.D4, reg)
            assert e <= 1e-4, (i, reg, e)
            if k < 2:
                ef = forward_region_error(pan_h, ms_h, out[i].detach(), O.D4, reg, range(B))
                assert ef <= 5e-4, (i, reg, ef)


def test_dot_product_identity_config3_size():
    """<F(x), y> = <x, F^T(y)> at the autograd workload's scene size
    (PAN 4096^2, 4 MS bands 2048^2, float32), dot products in FP64."""
    H = W = 4096
    B = 4
    g = torch.Generator(device=DEV)
    g.manual_seed(0)
    pan = torch.randn((H, W), generator=g, device=DEV)
    ms = torch.randn((B, H // 2, W // 2), generator=g, device=DEV)
    y = torch.randn((B, H, W), generator=g, device=DEV)
    out = torch.empty((B, H, W), device=DEV)
    _C.dwtfuse_fuse(pan, ms, O.D4, out, None)
    gp = torch.empty((H, W), device=DEV)
    gm = torch.empty((B, H // 2, W // 2), device=DEV)
    _C.dwtfuse_fuse_backward(y, O.D4, gp, gm)
    lhs = (out.double() * y.double()).sum().item()
    rhs = (pan.double() * gp.double()).sum().item() + (ms.double() * gm.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * (out.double().abs() * y.double().abs()).sum().item()


# Mixed batch: both wavelets, W = 0 and 2 mod 4 and off the 128-column strip
# grid, odd H/2, 1 to 16 bands (one to four band chunks; scenes with fewer
# bands drop out of the later chunks).
BATCH = [((64, 64), 3, O.D4), ((66, 258), 4, O.HAAR), ((130, 250), 9, O.D4), ((12, 814), 1, O.HAAR),
         ((4, 4), 2, O.D4), ((200, 136), 6, O.HAAR), ((98, 610), 5, O.D4), ((256, 512), 16, O.D4),
         ((6, 18), 13, O.HAAR), ((1030, 196), 8, O.D4)]


def _batch(specs, seed):
    gen = torch.Generator(device=DEV)
    gen.manual_seed(seed)
    rows = []
    for (H, W), B, wav in specs:
        g = torch.randn((B, H, W), generator=gen, device=DEV)
        gp = torch.full((H, W), float("nan"), device=DEV)
        gm = torch.full((B, H // 2, W // 2), float("nan"), device=DEV)
        rows.append((g, wav, gp, gm))
    return rows


def _per_scene(rows):
    refs = []
    for g, wav, gp, gm in rows:
        rp, rm = torch.empty_like(gp), torch.empty_like(gm)
        _C.dwtfuse_fuse_backward(g, wav, rp, rm)
        refs.append((rp, rm))
    return refs


def test_batched_backward_equals_per_scene():
    """dwtfuse_fuse_backward_batched gives the per-scene adjoint's bits: the
    same item arithmetic, band chunks in the same order."""
    rows = _batch(BATCH, 7)
    ws = torch.empty(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_fuse_backward_batched([_C.make_grad_scene(*r) for r in rows], ws)
    refs = _per_scene(rows)
    torch.cuda.synchronize()
    for (g, wav, gp, gm), (rp, rm) in zip(rows, refs):
        assert torch.equal(gp, rp) and torch.equal(gm, rm), (tuple(g.shape), wav)


def test_batched_backward_against_oracle():
    rows = _batch(BATCH[:4], 8)
    ws = torch.empty(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_fuse_backward_batched([_C.make_grad_scene(*r) for r in rows], ws)
    torch.cuda.synchronize()
    for g, wav, gp, gm in rows:
        rp, rm = O.fuse_adjoint(g.cpu().numpy().astype(np.float64), wav)
        assert_close(gp.cpu().numpy().astype(np.float64), rp)
        assert_close(gm.cpu().numpy().astype(np.float64), rm)


def test_batched_backward_full_table_and_graph():
    """128 scenes (the table's capacity) captured in a CUDA graph and replayed."""
    specs = [((8 + 4 * (i % 9), 6 + 4 * (i % 11)), 1 + i % 6, O.D4 if i % 3 else O.HAAR) for i in range(128)]
    rows = _batch(specs, 9)
    ws = torch.empty(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=DEV)
    scenes = [_C.make_grad_scene(*r) for r in rows]
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            _C.dwtfuse_fuse_backward_batched(scenes, ws, stream=s)
    graph.replay()
    refs = _per_scene(rows)
    torch.cuda.synchronize()
    for (g, wav, gp, gm), (rp, rm) in zip(rows, refs):
        assert torch.equal(gp, rp) and torch.equal(gm, rm), (tuple(g.shape), wav)
