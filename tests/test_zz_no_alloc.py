"""The batched entry point for callers that cannot allocate device memory.

Such callers (an application that has reserved all GPU memory in its own pool,
a plug-in host that passes only image pointers, a chain whose memory footprint
is fixed at start-up) cannot provide the workspace dwtfuse_fuse_batched needs.
dwtfuse_fuse_batched_noalloc keeps the queue counter in the library's static
device array instead.  This test calls it through the C ABI twice in a row and
checks both results against the workspace entry point's on the same scenes:
the two run the same kernel on the same scene table, so the outputs must be
equal bit for bit.  The second call must not change how much device memory
torch's allocator holds or how much the device reports free, and the status
word each call leaves in the static array reads back as OK.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenegen
from paper_1803_00737_gb300 import _C

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _scenes(specs, outs):
    scenes = []
    for sp, (pan, ms, out) in zip(specs, outs):
        scenes.append(_C.make_scene(pan, ms, sp.wavelet, out, None))
    return (_C.Scene * len(scenes))(*scenes)


def test_noalloc_batched_matches_workspace_batched_twice():
    L = _C.lib()
    specs = scenegen.batch_specs(n=7, seed=11, lo=8, hi=260)
    inputs = []
    for sp in specs:
        rng = np.random.default_rng(sp.seed)
        pan = torch.from_numpy(rng.integers(0, 256, (sp.H, sp.W)).astype(np.uint8)).to(DEV)
        ms = torch.from_numpy(rng.integers(0, 256, (sp.bands, sp.H // 2, sp.W // 2))
                              .astype(np.uint8)).to(DEV)
        inputs.append((pan, ms))
    ref = [torch.empty((sp.bands, sp.H, sp.W), device=DEV) for sp in specs]
    got = [torch.empty((sp.bands, sp.H, sp.W), device=DEV) for sp in specs]
    ws = torch.zeros(_C.dwtfuse_batched_workspace_size(), dtype=torch.uint8, device=DEV)
    arr_ref = _scenes(specs, [(p, m, o) for (p, m), o in zip(inputs, ref)])
    st = L.dwtfuse_fuse_batched(arr_ref, len(specs), ctypes.c_void_p(ws.data_ptr()),
                                ws.numel(), 0, 0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _C.OK
    torch.cuda.synchronize()
    arr = _scenes(specs, [(p, m, o) for (p, m), o in zip(inputs, got)])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        for o in got:
            o.fill_(float("nan"))
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
        st = L.dwtfuse_fuse_batched_noalloc(arr, len(specs), 0, 0, stream)
        assert st == _C.OK, L.dwtfuse_status_string(st)
        torch.cuda.synchronize()
        after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
        if call == 1:
            assert after == before, (before, after)
        # the call's device status word, read from the library's static array
        assert L.dwtfuse_get_last_device_status(None, stream) == _C.OK
        for sp, a, b in zip(specs, got, ref):
            assert torch.equal(a, b), (call, sp)


def test_noalloc_rejects_too_many_scenes():
    L = _C.lib()
    s = _C.Scene()
    arr = (_C.Scene * 1)(s)
    assert L.dwtfuse_fuse_batched_noalloc(arr, _C.MAX_SCENES + 1, 0, 0, None) == _C.ESHAPE
