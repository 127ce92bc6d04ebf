"""Full-size batched forward + backward with metrics: scenes of the 12-scene
workload (square PAN, sides even in [8192, 32768], 8 MS bands, D4), one at a
time: batched forward (float32 + uint8), ERGAS/QNR of the uint8 product (the
separate passes, and the forward that scores its product on chip, which
must agree), and the adjoint of a seeded output gradient G.

Checked per scene, element by element against the oracle's point-wise
evaluators: the fused bands on two seeded 256 x 256 windows and on the wrap
rows and columns (D4 bar 5e-4), grad_PAN and every band's grad_MS on the same
regions (bar 1e-4 of max(1, max |ref|)); as extra checks the dot-product
identity <F(P, M), G> = <P, grad_P> + <M, grad_M> in FP64, and, on the
smallest scene, the metrics against the oracle on the whole images (uint8
bars of test_metrics_gpu)."""
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
    # The benchmark's form: the forward scoring its uint8 product on chip.  Its
    # outputs overwrite the batched forward's with the same bits (checked).
    keep8 = out8.clone()
    res2 = torch.zeros(4, dtype=torch.float64, device=DEV)
    _C.dwtfuse_fuse_metrics(pan, ms, sp.wavelet, None, out8, mws, res2)
    torch.cuda.synchronize()
    assert torch.equal(keep8, out8)
    del keep8
    r1, r2 = res.cpu().numpy(), res2.cpu().numpy()
    assert r1[0] == r2[0] and np.abs(r1[1:] - r2[1:]).max() <= 1e-6, (r1, r2)
    G = scenegen.target_like((8, H, W), seed=sp.seed + 5, device=DEV)
    gp = torch.empty((H, W), device=DEV)
    gm = torch.empty((8, H // 2, W // 2), device=DEV)
    _C.dwtfuse_fuse_backward(G, sp.wavelet, gp, gm)
    torch.cuda.synchronize()
    return pan, ms, out, out8, res.cpu().numpy(), G, gp, gm


@pytest.mark.parametrize("which", ["smallest", "largest"])
def test_config4_scene(which):
    from tests.parity_windows import adjoint_region_error, forward_region_error, regions
    specs = config4_specs()
    if which == "largest":
        sp = max(specs, key=lambda s: s.H)
        sp = scenegen.SceneSpec(32768, 32768, 8, sp.wavelet, sp.seed)  # the size bound itself
    else:
        sp = min(specs, key=lambda s: s.H)
    ws = torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=DEV)
    mws = torch.empty(_C.dwtfuse_metrics_workspace_size(), dtype=torch.uint8, device=DEV)
    pan, ms, out, out8, res, G, gp, gm = _run_scene(sp, ws, mws)
    H = W = sp.H
    assert _C.dwtfuse_get_last_device_status(ws) == _C.OK
    pan_h, ms_h = pan.cpu().numpy(), ms.cpu().numpy()
    for reg in regions(H, W, seed=sp.seed):
        ef = forward_region_error(pan_h, ms_h, out, sp.wavelet, reg, range(8))
        assert ef <= 5e-4, (reg, ef)
        eb = adjoint_region_error(G, gp, gm, sp.wavelet, reg)
        assert eb <= 1e-4, (reg, eb)
    lhs = dot64(out, G)
    rhs = dot64(pan, gp) + dot64(ms, gm)
    assert abs(lhs - rhs) <= 1e-6 * (dot64(out, out) * dot64(G, G)) ** 0.5
    assert np.isfinite(res).all()
    if which == "smallest":
        f = out8.cpu().numpy()
        m = list(ms_h)
        q, dl, ds = O.qnr(f, m, pan_h)
        ref = np.array([O.ergas(f, m), q, dl, ds])
        assert abs(res[0] - ref[0]) <= 1e-12 * ref[0]
        assert np.abs(res[1:] - ref[1:]).max() <= 2e-6
