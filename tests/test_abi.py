"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and its argument validation answers before any GPU work.
No GPU needed (every call here returns from validation)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1803_00737_gb300 import _C
from paper_1803_00737_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return _C.lib()


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(dwtfuse_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("dwtfuse_fuse", "dwtfuse_fuse_batched", "dwtfuse_fuse_backward",
                 "dwtfuse_status_string", "dwtfuse_get_last_device_status"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert not [n for n in declared_symbols() if n not in _C._SIGS]


def test_status_strings(L):
    for code in range(8):
        assert L.dwtfuse_status_string(code)
    assert L.dwtfuse_status_string(99) == b"unknown status"


FAKE = 0x10000  # never dereferenced: every call below fails validation first


def _ms(n, addr=FAKE):
    return (ctypes.c_void_p * n)(*([addr] * n))


@pytest.mark.parametrize("H,W,wav,code", [
    (5, 4, 0, _C.ESHAPE), (4, 6, 1, _C.OK), (2, 2, 1, _C.ESHAPE), (0, 4, 0, _C.ESHAPE),
    (4, 3, 0, _C.ESHAPE), (4, 4, 2, _C.EINVAL), (1 << 21, 4, 0, _C.ESHAPE)])
def test_shape_validation(L, H, W, wav, code):
    if code == _C.OK:
        pytest.skip("valid shapes would launch")
    assert L.dwtfuse_fuse(FAKE, _ms(1), 1, H, W, wav, _C.U8, FAKE, None, None) == code


def test_null_and_count_validation(L):
    assert L.dwtfuse_fuse(None, _ms(1), 1, 4, 4, 0, _C.U8, FAKE, None, None) == _C.EINVAL
    assert L.dwtfuse_fuse(FAKE, None, 1, 4, 4, 0, _C.U8, FAKE, None, None) == _C.EINVAL
    assert L.dwtfuse_fuse(FAKE, _ms(1), 1, 4, 4, 0, _C.U8, None, None, None) == _C.EINVAL
    assert L.dwtfuse_fuse(FAKE, _ms(1), 0, 4, 4, 0, _C.U8, FAKE, None, None) == _C.EINVAL
    assert L.dwtfuse_fuse(FAKE, _ms(17), 17, 4, 4, 0, _C.U8, FAKE, None, None) == _C.ESHAPE
    assert L.dwtfuse_fuse(FAKE, _ms(2, 0), 2, 4, 4, 0, _C.U8, FAKE, None, None) == _C.EINVAL
    assert L.dwtfuse_fuse(FAKE, _ms(1), 1, 4, 4, 0, 7, FAKE, None, None) == _C.EINVAL


def test_alignment_validation(L):
    # float PAN must be 8-byte aligned (pixel pairs), float out 8-byte, uint8 out 2-byte
    assert L.dwtfuse_fuse(FAKE + 4, _ms(1), 1, 4, 4, 0, _C.F32, FAKE, None, None) == _C.EALIGN
    assert L.dwtfuse_fuse(FAKE + 1, _ms(1), 1, 4, 4, 0, _C.U8, FAKE, None, None) == _C.EALIGN
    assert L.dwtfuse_fuse(FAKE, _ms(1), 1, 4, 4, 0, _C.U8, FAKE + 4, None, None) == _C.EALIGN
    assert L.dwtfuse_fuse(FAKE, _ms(1), 1, 4, 4, 0, _C.U8, None, FAKE + 1, None) == _C.EALIGN
    assert L.dwtfuse_fuse(FAKE, _ms(1, FAKE + 2), 1, 4, 4, 0, _C.F32, FAKE, None, None) == _C.EALIGN


def test_backward_validation(L):
    gms = _ms(2)
    assert L.dwtfuse_fuse_backward(None, 2, 4, 4, 0, FAKE, gms, None) == _C.EINVAL
    assert L.dwtfuse_fuse_backward(FAKE, 2, 4, 5, 0, FAKE, gms, None) == _C.ESHAPE
    assert L.dwtfuse_fuse_backward(FAKE + 4, 2, 4, 4, 0, FAKE, gms, None) == _C.EALIGN
    assert L.dwtfuse_fuse_backward(FAKE, 0, 4, 4, 0, FAKE, gms, None) == _C.EINVAL


def test_batched_validation(L):
    s = _C.Scene()
    s.pan = FAKE
    s.ms[0] = FAKE
    s.out_f32 = FAKE
    s.H, s.W, s.bands, s.wavelet, s.in_dtype = 4, 4, 9, 0, 0
    arr = (_C.Scene * 1)(s)
    ws = _C.lib().dwtfuse_batched_workspace_size()
    assert ws >= 16
    assert L.dwtfuse_fuse_batched(arr, 1, FAKE, ws, 0, 0, None) == _C.ESHAPE  # 9 bands > 8
    s.bands = 1
    arr = (_C.Scene * 1)(s)
    assert L.dwtfuse_fuse_batched(arr, 1, FAKE, ws - 1, 0, 0, None) == _C.ENOMEM
    assert L.dwtfuse_fuse_batched(arr, 0, FAKE, ws, 0, 0, None) == _C.EINVAL
    assert L.dwtfuse_fuse_batched(arr, 129, FAKE, ws, 0, 0, None) == _C.ESHAPE
    s.reserved = 1
    arr = (_C.Scene * 1)(s)
    assert L.dwtfuse_fuse_batched(arr, 1, FAKE, ws, 0, 0, None) == _C.EINVAL


def test_batched_backward_validation(L):
    s = _C.GradScene()
    s.grad_out, s.grad_pan = FAKE, FAKE
    s.grad_ms[0] = s.grad_ms[1] = FAKE
    s.H, s.W, s.bands, s.wavelet = 4, 4, 2, 1
    ws = _C.lib().dwtfuse_batched_workspace_size()

    def call(n=1, w=FAKE, nbytes=ws):
        return L.dwtfuse_fuse_backward_batched((_C.GradScene * 1)(s), n, w, nbytes, None)

    assert call(n=0) == _C.EINVAL
    assert call(n=129) == _C.ESHAPE
    assert call(w=None) == _C.EINVAL
    assert call(nbytes=ws - 1) == _C.ENOMEM
    assert call(w=FAKE + 8) == _C.EALIGN
    s.W = 5
    assert call() == _C.ESHAPE
    s.W, s.bands = 4, 17
    assert call() == _C.ESHAPE
    s.bands = 0
    assert call() == _C.EINVAL
    s.bands, s.wavelet = 2, 2
    assert call() == _C.EINVAL
    s.wavelet, s.grad_out = 1, FAKE + 4
    assert call() == _C.EALIGN
    s.grad_out, s.grad_ms[1] = FAKE, None
    assert call() == _C.EINVAL
    s.grad_ms[1] = FAKE + 2
    assert call() == _C.EALIGN


def test_metric_wait_test_hook_validation(L):
    assert L.dwtfuse_set_metric_wait_test(2) == _C.EINVAL
    assert L.dwtfuse_set_metric_wait_test(-1) == _C.EINVAL
    assert L.dwtfuse_set_metric_wait_test(0) == _C.OK


def test_rows_knob(L):
    assert L.dwtfuse_set_rows_per_item(-1) == _C.EINVAL
    assert L.dwtfuse_set_rows_per_item(16) == _C.OK
    assert L.dwtfuse_set_rows_per_item(0) == _C.OK


def test_staging_knob(L):
    assert L.dwtfuse_set_fuse_staging(2) == _C.EINVAL
    assert L.dwtfuse_set_fuse_staging(-1) == _C.EINVAL
    assert L.dwtfuse_set_fuse_staging(0) == _C.OK
    assert L.dwtfuse_set_fuse_staging(1) == _C.OK


def test_cpu_tensors_are_rejected():
    torch = pytest.importorskip("torch")
    pan = torch.zeros((4, 4), dtype=torch.uint8)
    ms = torch.zeros((1, 2, 2), dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA"):
        _C.dwtfuse_fuse(pan, ms, 0, torch.zeros((1, 4, 4)), None)


def test_binding_refuses_buffers_the_call_would_overrun():
    """The binding checks every buffer the library reads or writes against the
    element count and type the call implies, before any pointer reaches C;
    right-sized CPU tensors get as far as the CUDA check."""
    torch = pytest.importorskip("torch")
    H, W, B = 8, 12, 3
    pan = torch.zeros((H, W), dtype=torch.uint8)
    ms = torch.zeros((B, H // 2, W // 2), dtype=torch.uint8)
    f32 = torch.zeros((B, H, W))
    u8 = torch.zeros((B, H, W), dtype=torch.uint8)
    g = torch.zeros((B, H, W))
    gp = torch.zeros((H, W))
    gm = torch.zeros((B, H // 2, W // 2))
    ok = [
        lambda: _C.make_scene(pan, ms, 1, f32, u8),
        lambda: _C.dwtfuse_fuse_ex(pan, ms, 1, 2.0, f32, u8),
        lambda: _C.make_grad_scene(g, 1, gp, gm),
        lambda: _C.dwtfuse_fuse_backward(g, 1, gp, gm),
        lambda: _C.dwtfuse_idwt2(gp, 1, gp.clone(), None),
    ]
    for call in ok:
        with pytest.raises(ValueError, match="CUDA"):
            call()
    short = [
        lambda: _C.make_scene(pan, ms, 1, f32[:2], None),
        lambda: _C.make_scene(pan, ms[:, :2], 1, None, u8),
        lambda: _C.dwtfuse_fuse_ex(pan, ms, 1, 2.0, None, u8[:, :4]),
        lambda: _C.make_grad_scene(g, 1, gp[:4], gm),
        lambda: _C.dwtfuse_fuse_backward(g, 1, gp, gm[:, :2]),
        lambda: _C.dwtfuse_idwt2(gp, 1, None, torch.zeros((H, W // 2), dtype=torch.uint8)),
    ]
    for call in short:
        with pytest.raises(ValueError, match="holds"):
            call()
    with pytest.raises(TypeError):
        _C.make_scene(pan, ms, 1, u8, None)  # a uint8 buffer as the float32 output
    with pytest.raises(TypeError):
        _C.dwtfuse_fuse_backward(g, 1, gp, gm.double())
