"""FP64 CPU oracle for one-level 2D DWT pansharpening (arXiv:1803.00737, Sec. 2).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product
(``paper_1803_00737_gb300``) never does, and the two share no code.

The arithmetic lives in ``dwt_oracle.c`` (plain C, FP64, OpenMP over rows);
this module compiles it with gcc on first use and wraps it with ctypes over
NumPy arrays.  ``matrices.py`` holds the textbook matrix forms used to pin it.

Wavelet codes: 0 = Haar (Eq. 1-2, 11-12), 1 = Daubechies-4 (Eq. 3-10, 13-16).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HAAR = 0
D4 = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_L = ctypes.POINTER(ctypes.c_long)
_V = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile dwt_oracle.c into liboracle.so beside it (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-Wall", "-Wextra",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


# A prebuilt oracle library to load instead of liboracle.so.  Only the
# mutation tests set it, to run the pins against a copy of dwt_oracle.c with a
# planted mistake.
_LIB_ENV = "DWTFUSE_ORACLE_LIB"


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get(_LIB_ENV)
            if not path:
                path = build()
            lib = ctypes.CDLL(path)
            i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
            sig = {
                "oracle_d4_h": (None, [_D]),
                "oracle_d4_g": (None, [_D]),
                "oracle_d4_g_printed": (None, [_D]),
                "oracle_default_gain": (d, [i]),
                "oracle_dwt1d": (i, [i, l, _D, _D]),
                "oracle_idwt1d": (i, [i, l, _D, _D]),
                "oracle_dwt1d_g": (i, [l, _D, _D, _D]),
                "oracle_idwt1d_g": (i, [l, _D, _D, _D]),
                "oracle_dwt2": (i, [i, l, l, _D, _D]),
                "oracle_idwt2": (i, [i, l, l, _D, _D]),
                "oracle_fuse": (i, [i, l, l, i, d, _D, ctypes.POINTER(_D), _D]),
                "oracle_fuse_adjoint": (i, [i, l, l, i, d, _D, _D, ctypes.POINTER(_D)]),
                "oracle_fuse_points": (i, [i, l, l, d, _D, _U8, _D, _U8, l, _L, _L, _D]),
                "oracle_fuse_adjoint_points": (i, [i, l, l, i, d, _D, l, l, l, l, l, _L, _L, _D,
                                                   l, _L, _L, _D]),
                "oracle_to_u8": (None, [l, _D, _U8]),
                "oracle_dwt2_points": (i, [i, l, l, _D, _U8, l, _L, _L, _D]),
                "oracle_ergas_t": (d, [l, l, i, _V, i, ctypes.POINTER(_V), i]),
                "oracle_q_index_t": (d, [l, l, _V, i, _V, i, l]),
                "oracle_qnr_t": (i, [l, l, i, _V, i, ctypes.POINTER(_V), i, _V, i, l,
                                     ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]),
                "oracle_num_threads": (i, []),
                "oracle_set_threads": (None, [i]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (code {rc})")


# ------------------------------------------------------------ coefficients

def d4_h() -> np.ndarray:
    """h of Eq. 7-8."""
    out = np.zeros(4)
    _load().oracle_d4_h(_p(out))
    return out


def d4_g() -> np.ndarray:
    """g used by the oracle: the quadrature mirror [h3, -h2, h1, -h0] (reading of Eq. 9-10)."""
    out = np.zeros(4)
    _load().oracle_d4_g(_p(out))
    return out


def d4_g_printed() -> np.ndarray:
    """g of Eq. 9-10 exactly as printed (fails perfect reconstruction)."""
    out = np.zeros(4)
    _load().oracle_d4_g_printed(_p(out))
    return out


def default_gain(wavelet: int) -> float:
    """LL replacement gain: 1 for Haar, 2 for D4 (DC gain of the 2D low-pass)."""
    return float(_load().oracle_default_gain(int(wavelet)))


# ------------------------------------------------------------- transforms

def dwt1d(x, wavelet: int, g=None) -> np.ndarray:
    """1D forward transform of a vector: [approximation | detail] (Eq. 1-6)."""
    x = _f64(x)
    y = np.empty_like(x)
    if g is not None:
        _check(_load().oracle_dwt1d_g(x.size, _p(_f64(g)), _p(x), _p(y)), "dwt1d")
    else:
        _check(_load().oracle_dwt1d(int(wavelet), x.size, _p(x), _p(y)), "dwt1d")
    return y


def idwt1d(c, wavelet: int, g=None) -> np.ndarray:
    """1D inverse transform (Eq. 11-16)."""
    c = _f64(c)
    y = np.empty_like(c)
    if g is not None:
        _check(_load().oracle_idwt1d_g(c.size, _p(_f64(g)), _p(c), _p(y)), "idwt1d")
    else:
        _check(_load().oracle_idwt1d(int(wavelet), c.size, _p(c), _p(y)), "idwt1d")
    return y


def dwt2(x, wavelet: int) -> np.ndarray:
    """Forward 2D transform: rows, then columns; LL is the top-left quadrant."""
    x = _f64(x)
    y = np.empty_like(x)
    _check(_load().oracle_dwt2(int(wavelet), x.shape[0], x.shape[1], _p(x), _p(y)), "dwt2")
    return y


def idwt2(c, wavelet: int) -> np.ndarray:
    """Inverse 2D transform: columns, then rows."""
    c = _f64(c)
    y = np.empty_like(c)
    _check(_load().oracle_idwt2(int(wavelet), c.shape[0], c.shape[1], _p(c), _p(y)), "idwt2")
    return y


# ----------------------------------------------------------------- fusion

def _ptr_array(arrs):
    return (_D * len(arrs))(*[_p(a) for a in arrs])


def fuse(pan, ms, wavelet: int, gain: float | None = None) -> np.ndarray:
    """Fused bands, shape (B, H, W): IDWT2(DWT2(pan) with LL <- gain * ms[b]).

    pan: (H, W); ms: (B, H/2, W/2) or a list of (H/2, W/2) arrays.
    """
    pan = _f64(pan)
    ms = [_f64(m) for m in ms]
    H, W = pan.shape
    for m in ms:
        if m.shape != (H // 2, W // 2):
            raise ValueError("each MS band must be (H/2, W/2)")
    g = default_gain(wavelet) if gain is None else float(gain)
    out = np.empty((len(ms), H, W))
    _check(_load().oracle_fuse(int(wavelet), H, W, len(ms), ctypes.c_double(g), _p(pan),
                               _ptr_array(ms), _p(out)), "fuse")
    return out


def fuse_adjoint(grad_out, wavelet: int, gain: float | None = None):
    """Transpose of the fusion map: returns (grad_pan (H, W), grad_ms (B, H/2, W/2))."""
    grad_out = _f64(grad_out)
    B, H, W = grad_out.shape
    g = default_gain(wavelet) if gain is None else float(gain)
    gp = np.empty((H, W))
    gm = [np.empty((H // 2, W // 2)) for _ in range(B)]
    _check(_load().oracle_fuse_adjoint(int(wavelet), H, W, B, ctypes.c_double(g), _p(grad_out),
                                       _p(gp), _ptr_array(gm)), "fuse_adjoint")
    return gp, np.stack(gm)


def fuse_points(pan, ms_band, wavelet: int, ys, xs, gain: float | None = None) -> np.ndarray:
    """Fused values of one band at pixels (ys[k], xs[k]), evaluated lazily from
    the same equations (for images too large for the whole-image oracle).
    pan (H, W) and ms_band (H/2, W/2) may be uint8 or float."""
    H, W = pan.shape
    if ms_band.shape != (H // 2, W // 2):
        raise ValueError("MS band must be (H/2, W/2)")
    g = default_gain(wavelet) if gain is None else float(gain)
    ys = np.ascontiguousarray(ys, dtype=np.int64)
    xs = np.ascontiguousarray(xs, dtype=np.int64)
    if ys.shape != xs.shape or ys.ndim != 1:
        raise ValueError("ys and xs must be equal-length 1D arrays")
    if ys.size and (ys.min() < 0 or ys.max() >= H or xs.min() < 0 or xs.max() >= W):
        raise ValueError("sample outside the image")
    out = np.empty(ys.size)
    keep = []

    def as_args(a):
        if a.dtype == np.uint8:
            a = np.ascontiguousarray(a)
            keep.append(a)
            return None, a.ctypes.data_as(_U8)
        a = _f64(a)
        keep.append(a)
        return _p(a), None

    pd, pu = as_args(pan)
    md, mu = as_args(ms_band)
    _check(_load().oracle_fuse_points(int(wavelet), H, W, ctypes.c_double(g), pd, pu, md, mu,
                                      ys.size, ys.ctypes.data_as(_L), xs.ctypes.data_as(_L),
                                      _p(out)), "fuse_points")
    return out


def fuse_adjoint_points(g_win, wavelet: int, H: int, W: int, ys=(), xs=(), is_=(), js=(),
                        gy0: int = 0, gx0: int = 0, gain: float | None = None):
    """The transposed fusion (fuse_adjoint) evaluated lazily at sampled outputs.

    g_win (B, hg, wg): the output gradient of every band on a periodic window of
    the H x W image, g_win[b, r, s] = grad_out[b, (gy0 + r) % H, (gx0 + s) % W]
    (the whole gradient with gy0 = gx0 = 0).  Returns (grad_pan at (ys[k], xs[k]),
    grad_ms (B, len(is_)) at MS pixels (is_[k], js[k])).  Raises if a value needs
    gradient outside the window."""
    g = _f64(g_win)
    if g.ndim != 3 or g.shape[1] > H or g.shape[2] > W:
        raise ValueError("g_win must be (B, hg <= H, wg <= W)")
    B, hg, wg = g.shape
    gn = default_gain(wavelet) if gain is None else float(gain)
    ys, xs = (np.ascontiguousarray(a, dtype=np.int64) for a in (ys, xs))
    is_, js = (np.ascontiguousarray(a, dtype=np.int64) for a in (is_, js))
    if ys.shape != xs.shape or is_.shape != js.shape or ys.ndim != 1 or is_.ndim != 1:
        raise ValueError("coordinates must be equal-length 1D arrays")
    if ys.size and (ys.min() < 0 or ys.max() >= H or xs.min() < 0 or xs.max() >= W):
        raise ValueError("PAN sample outside the image")
    if is_.size and (is_.min() < 0 or is_.max() >= H // 2 or js.min() < 0 or js.max() >= W // 2):
        raise ValueError("MS sample outside the image")
    gp = np.empty(ys.size)
    gm = np.empty((B, is_.size))
    _check(_load().oracle_fuse_adjoint_points(
        int(wavelet), int(H), int(W), B, ctypes.c_double(gn), _p(g), int(gy0) % H, int(gx0) % W, hg, wg,
        ys.size, ys.ctypes.data_as(_L), xs.ctypes.data_as(_L), _p(gp),
        is_.size, is_.ctypes.data_as(_L), js.ctypes.data_as(_L), _p(gm)), "fuse_adjoint_points")
    if np.isnan(gp).any() or np.isnan(gm).any():
        raise ValueError("a sample needs output gradient outside the given window")
    return gp, gm


def dwt2_points(img, wavelet: int, is_, js) -> np.ndarray:
    """Forward 2D transform coefficients at (is_[k], js_[k]) of an (H, W) uint8
    or float image, evaluated from the tap lists."""
    H, W = img.shape
    is_ = np.ascontiguousarray(is_, dtype=np.int64)
    js = np.ascontiguousarray(js, dtype=np.int64)
    out = np.empty(is_.size)
    if img.dtype == np.uint8:
        a = np.ascontiguousarray(img)
        rc = _load().oracle_dwt2_points(int(wavelet), H, W, None, a.ctypes.data_as(_U8), is_.size,
                                        is_.ctypes.data_as(_L), js.ctypes.data_as(_L), _p(out))
    else:
        a = _f64(img)
        rc = _load().oracle_dwt2_points(int(wavelet), H, W, _p(a), None, is_.size,
                                        is_.ctypes.data_as(_L), js.ctypes.data_as(_L), _p(out))
    _check(rc, "dwt2_points")
    return out


def to_u8(x) -> np.ndarray:
    """uint8 output rule: clamp to [0, 255], round half to even."""
    x = _f64(x)
    y = np.empty(x.shape, dtype=np.uint8)
    _load().oracle_to_u8(x.size, _p(x), y.ctypes.data_as(_U8))
    return y


# ---------------------------------------------------------------- metrics
# Metric inputs may be uint8 (the 8-bit product) or float; uint8 arrays are
# read as such, anything else is converted to float64.

def _img(a):
    a = np.asarray(a)
    if a.dtype == np.uint8:
        a = np.ascontiguousarray(a)
        return a, 1
    return _f64(a), 0


def _imgs(arrs):
    conv = [_img(a) for a in arrs]
    types = {t for _, t in conv}
    if len(types) != 1:
        raise ValueError("all MS bands must share one dtype")
    ptrs = (_V * len(conv))(*[a.ctypes.data for a, _ in conv])
    return conv, ptrs, types.pop()


def ergas(fused, ms) -> float:
    """ERGAS of fused (B, H, W) against MS (B, H/2, W/2); definition in dwt_oracle.c."""
    f, ft = _img(fused)
    B, H, W = f.shape
    keep, ptrs, mt = _imgs(list(ms))
    return float(_load().oracle_ergas_t(H, W, B, f.ctypes.data, ft, ptrs, mt))


def q_index(x, y, win: int = 32) -> float:
    """Wang-Bovik Q averaged over non-overlapping win x win windows."""
    x, xt = _img(x)
    y, yt = _img(y)
    if x.shape != y.shape:
        raise ValueError("shape mismatch")
    return float(_load().oracle_q_index_t(x.shape[0], x.shape[1], x.ctypes.data, xt, y.ctypes.data,
                                          yt, int(win)))


def qnr(fused, ms, pan, win: int = 32):
    """(QNR, D_lambda, D_s); definition in dwt_oracle.c."""
    f, ft = _img(fused)
    B, H, W = f.shape
    keep, ptrs, mt = _imgs(list(ms))
    p, pt = _img(pan)
    q = ctypes.c_double()
    dl = ctypes.c_double()
    ds = ctypes.c_double()
    _check(_load().oracle_qnr_t(H, W, B, f.ctypes.data, ft, ptrs, mt, p.ctypes.data, pt, int(win),
                                ctypes.byref(q), ctypes.byref(dl), ctypes.byref(ds)), "qnr")
    return q.value, dl.value, ds.value


# ----------------------------------------------------------------- threads

def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))
