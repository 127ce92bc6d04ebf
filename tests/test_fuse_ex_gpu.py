"""dwtfuse_fuse_ex: the fusion with an explicit LL replacement gain (the paper
leaves it unstated) against the oracle run with the same gain."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen
from paper_1803_00737_gb300 import _C

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("wav,gain", [(0, 1.0), (0, 0.5), (1, 1.0), (1, 2.0), (1, 1.5)])
@pytest.mark.parametrize("shape", [(64, 96), (34, 614)])
def test_fuse_ex_matches_oracle_gain(wav, gain, shape):
    H, W = shape
    pan, ms = scenegen.make_scene(H, W, 3, seed=H + int(10 * gain))
    out = torch.empty((3, H, W), device=DEV)
    out8 = torch.empty((3, H, W), dtype=torch.uint8, device=DEV)
    _C.dwtfuse_fuse_ex(pan.to(DEV), ms.to(DEV), wav, gain, out, out8)
    torch.cuda.synchronize()
    ref = O.fuse(pan.numpy().astype(np.float64), ms.numpy().astype(np.float64), wav, gain=gain)
    got = out.cpu().numpy()
    if wav == 0 and gain in (1.0, 0.5):  # multiples of 1/8: exact in FP32
        np.testing.assert_array_equal(got, ref.astype(np.float32))
    else:
        assert np.abs(got - ref).max() <= 5e-4


def test_fuse_ex_default_gain_equals_fuse():
    pan, ms = scenegen.make_scene(64, 128, 4, seed=3)
    pan, ms = pan.to(DEV), ms.to(DEV)
    a = torch.empty((4, 64, 128), device=DEV)
    b = torch.empty_like(a)
    _C.dwtfuse_fuse(pan, ms, 1, a, None)
    _C.dwtfuse_fuse_ex(pan, ms, 1, 2.0, b, None)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_fuse_ex_rejects_nan_gain():
    pan, ms = scenegen.make_scene(16, 16, 1, seed=0)
    out = torch.empty((1, 16, 16), device=DEV)
    with pytest.raises(_C.DwtfuseError) as e:
        _C.dwtfuse_fuse_ex(pan.to(DEV), ms.to(DEV), 0, float("nan"), out, None)
    assert e.value.status == _C.EINVAL
