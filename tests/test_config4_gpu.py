"""Full-size batched forward + backward with metrics: scenes of the 12-scene
workload (square PAN, sides even in [8192, 32768], 8 MS bands, D4), streamed
through one output slot: batched forward (float32 + uint8), ERGAS/QNR of the
uint8 product, and the adjoint with grad_out = F (loss 1/2 ||F||^2).

Checked per scene: sampled fused pixels against the point-wise oracle (D4 bar
5e-4), the dot-product identity <F(P, M), F> = <P, grad_P> + <M, grad_M> in
FP64 (holds at any size), and, on the smallest scene, the metrics against the
oracle on the whole images (uint8 bars of test_metrics_gpu)."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from paper_1803_00737_gb300 import _C

pytestmark = pytest.mark.gpu
DEV = "cuda"


def config4_specs():
    return scenegen.batch_specs(n=12, seed=0, lo=8192, hi=32768, bands=(8, 8),
                                wavelets=(scenegen.D4,), square=True)


def test_config4_scene_shapes():
    specs = config4_specs()
    assert len(specs) == 12
    assert all(s.H == s.W and s.H % 2 == 0 and 8192 <= s.H <= 32768 and s.bands == 8 for s in specs)


def dot64(a, b):
    """<a, b> accumulated in FP64, one leading-dimension slice at a time."""
    if a.dim() == 2:
        return (a.double() * b.double()).sum().item()
    return sum((a[i].double() * b[i].double()).sum().item() for i in range(a.shape[0]))


def _run_scene(sp, ws, mws):
    H = W = sp.H
    pan, ms = scenegen.make_scene(H, W, 8, seed=sp.seed, blob_scale=16.0, device=DEV)
    out = torch.empty((8, H, W), device=DEV)
    out8 = torch.empty((8, H, W), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_fuse_batched([_C.make_scene(pan, ms, sp.wavelet, out, out8)], ws)
    res = torch.zeros(4, dtype=torch.float64, device=DEV)
    _C.dwtfuse_metrics(out8, ms, pan, mws, res)
    gp = torch.empty((H, W), device=DEV)
    gm = torch.empty((8, H // 2, W // 2), device=DEV)
    _C.dwtfuse_fuse_backward(out, sp.wavelet, gp, gm)  # grad of 1/2 ||F||^2 is F
    torch.cuda.synchronize()
    return pan, ms, out, out8, res.cpu().numpy(), gp, gm


@pytest.mark.parametrize("which", ["smallest", "largest"])
def test_config4_scene(which):
    specs = config4_specs()
    if which == "largest":
        sp = max(specs, key=lambda s: s.H)
        sp = scenegen.SceneSpec(32768, 32768, 8, sp.wavelet, sp.seed)  # the size bound itself
    else:
        sp = min(specs, key=lambda s: s.H)
    ws = torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=DEV)
    mws = torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=DEV)
    pan, ms, out, out8, res, gp, gm = _run_scene(sp, ws, mws)
    H = W = sp.H
    assert _C.dwtfuse_get_last_device_status(ws) == _C.OK
    rng = np.random.default_rng(sp.seed)
    ys = np.concatenate([[0, 1, H - 2, H - 1], rng.integers(0, H, 300)])
    xs = np.concatenate([[0, W - 1, 1, W - 2], rng.integers(0, W, 300)])
    yt, xt = torch.from_numpy(ys).to(DEV), torch.from_numpy(xs).to(DEV)
    pan_h = pan.cpu().numpy()
    for b in (0, 7):
        ref = O.fuse_points(pan_h, ms[b].cpu().numpy(), sp.wavelet, ys, xs)
        got = out[b][yt, xt].cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 5e-4
    lhs = dot64(out, out)
    rhs = dot64(pan, gp) + dot64(ms, gm)
    assert abs(lhs - rhs) <= 1e-5 * lhs
    assert np.isfinite(res).all()
    if which == "smallest":
        f = out8.cpu().numpy()
        m = list(ms.cpu().numpy())
        q, dl, ds = O.qnr(f, m, pan_h)
        ref = np.array([O.ergas(f, m), q, dl, ds])
        assert abs(res[0] - ref[0]) <= 1e-12 * ref[0]
        assert np.abs(res[1:] - ref[1:]).max() <= 2e-6
