"""CPU correctness oracle for the OpenVX-style image graph path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2008_11476_gb300``)
and never imports it.

``hvx_oracle.c`` holds one plain loop per node (Table 2 point / local
operators, Section 4 abstractions); this module compiles it with gcc, loads it
with ctypes and wraps each function for numpy arrays.  ``graph.py`` holds the
graph-level oracle: verification (Section 5.2), dead-computation elimination
(Algorithm 1) and a node-by-node graph runner.

Every function here is pinned, in ``tests/test_oracle_pins.py``, by at least
one closed form, invariant or brute-force check that does not retype it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hvx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BORDER_UNDEFINED = 0
BORDER_REPLICATE = 1
BORDER_CONSTANT = 2
BORDER_MIRROR = 3   # Hipacc MIRROR: ... c b a | a b c ... (reflect with the edge repeated)
BORDER_REPEAT = 4   # Hipacc REPEAT: periodic continuation

ROUND_ZERO = 0
ROUND_NEAREST = 1

U8, S16, S32, F32 = 1, 2, 3, 4
_NP = {U8: np.uint8, S16: np.int16, S32: np.int32, F32: np.float32}
_FMT_OF = {np.dtype(np.uint8): U8, np.dtype(np.int16): S16, np.dtype(np.int32): S32,
           np.dtype(np.float32): F32}


def build(force: bool = False) -> str:
    """Compile hvx_oracle.c into liboracle.so (plain gcc, no vector flags)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


def _declare(L):
    P = ctypes.c_void_p
    I = ctypes.c_int
    R = ctypes.POINTER(ctypes.c_int)
    L.orc_gaussian3x3.argtypes = [P, P, I, I, I, I, I, R, R]
    L.orc_box3x3.argtypes = [P, P, I, I, I, I, I, R, R]
    L.orc_sobel3x3.argtypes = [P, P, P, I, I, I, I, R, R]
    L.orc_window_sum_s32.argtypes = [P, P, I, I, I, I, I, I, R, R]
    L.orc_convolve_u8_s16.argtypes = [P, P, I, I, I, I, P, I, I, I, R, R]
    L.orc_magnitude.argtypes = [P, P, P, I, I, R, R, R]
    L.orc_phase.argtypes = [P, P, P, I, I, R, R, R]
    L.orc_threshold.argtypes = [P, I, P, I, I, I, ctypes.c_double, ctypes.c_double, I, I, R, R]
    L.orc_channel_extract_uyvy.argtypes = [P, P, I, I, I]
    L.orc_arith.argtypes = [P, I, P, I, P, I, I, I, I, I, R, R, R]
    L.orc_mul_s16_s32.argtypes = [P, P, P, I, I, R, R, R]
    L.orc_harris_response.argtypes = [P, P, P, P, I, I, ctypes.c_int64, ctypes.c_int64,
                                      R, R, R, R]
    L.orc_round_ratio.argtypes = [ctypes.c_int64, ctypes.c_int64]
    L.orc_round_ratio.restype = ctypes.c_float
    L.orc_harris_graph.argtypes = [P, P, P, I, I, I, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_double, P]
    L.orc_edge_graph.argtypes = [P, P, P, P, I, I, I, I, I, I, P]
    L.orc_morph3x3.argtypes = [P, P, I, I, I, I, I, R, R]
    L.orc_convolve_u8_u8.argtypes = [P, P, I, I, I, I, P, I, I, I, R, R]
    L.orc_tomasi_response.argtypes = [P, P, P, P, I, I, R, R, R, R]
    L.orc_bitwise.argtypes = [P, P, P, I, I, I, R, R, R]
    L.orc_multiply.argtypes = [P, I, P, I, P, I, I, I, ctypes.c_float, I, I, R, R, R]
    L.orc_mean_stddev.argtypes = [P, I, I, I, R, ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_float)]
    L.orc_minmaxloc.argtypes = [P, I, I, I, R, ctypes.POINTER(ctypes.c_int64)]
    L.orc_histogram.argtypes = [P, I, I, R, I, I, I, P]
    L.orc_equalize_hist.argtypes = [P, P, I, I, R, R]
    L.orc_convert_depth.argtypes = [P, I, P, I, I, I, I, I, R, R]
    for name in ("orc_gaussian3x3", "orc_box3x3", "orc_morph3x3", "orc_bitwise",
                 "orc_convolve_u8_u8", "orc_tomasi_response",
                 "orc_sobel3x3", "orc_window_sum_s32",
                 "orc_convolve_u8_s16", "orc_magnitude", "orc_phase", "orc_threshold",
                 "orc_channel_extract_uyvy", "orc_arith", "orc_mul_s16_s32",
                 "orc_harris_response", "orc_harris_graph", "orc_edge_graph",
                 "orc_multiply", "orc_mean_stddev", "orc_minmaxloc", "orc_histogram",
                 "orc_equalize_hist", "orc_convert_depth"):
        getattr(L, name).restype = ctypes.c_int


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _rect(r):
    return (ctypes.c_int * 4)(*r)


def full_rect(img: np.ndarray):
    h, w = img.shape[:2]
    return (0, 0, w, h)


def _check(rc):
    if rc != 0:
        raise ValueError("oracle rejected its arguments")


class Img:
    """A numpy image plus its valid rectangle (x0, y0, x1, y1), half-open."""

    def __init__(self, data: np.ndarray, rect=None):
        self.data = np.ascontiguousarray(data)
        self.rect = tuple(rect) if rect is not None else full_rect(self.data)

    @property
    def h(self):
        return self.data.shape[0]

    @property
    def w(self):
        return self.data.shape[1]


def _as_img(x) -> Img:
    return x if isinstance(x, Img) else Img(x)


# --- local operators --------------------------------------------------------

def gaussian3x3(src, border=BORDER_REPLICATE, cval=0, rounding=ROUND_ZERO) -> Img:
    s = _as_img(src)
    assert s.data.dtype == np.uint8
    out = np.empty_like(s.data)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_gaussian3x3(_p(s.data), _p(out), s.w, s.h, border, cval, rounding,
                                 _rect(s.rect), vo))
    return Img(out, tuple(vo))


def box3x3(src, border=BORDER_REPLICATE, cval=0, rounding=ROUND_ZERO) -> Img:
    s = _as_img(src)
    assert s.data.dtype == np.uint8
    out = np.empty_like(s.data)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_box3x3(_p(s.data), _p(out), s.w, s.h, border, cval, rounding,
                            _rect(s.rect), vo))
    return Img(out, tuple(vo))


MORPH_DILATE, MORPH_ERODE, MORPH_MEDIAN = 0, 1, 2
BIT_AND, BIT_OR, BIT_XOR, BIT_NOT = 0, 1, 2, 3


def morph3x3(src, op, border=BORDER_REPLICATE, cval=0) -> Img:
    """Dilate3x3 / Erode3x3 / Median3x3 (max / min / median of the 3x3 window)."""
    s = _as_img(src)
    assert s.data.dtype == np.uint8
    out = np.empty_like(s.data)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_morph3x3(_p(s.data), _p(out), s.w, s.h, border, cval, op, _rect(s.rect), vo))
    return Img(out, tuple(vo))


def bitwise(a, b, op) -> Img:
    """And / Or / Xor of two U8 images, or Not of one (b None)."""
    A = _as_img(a)
    B = _as_img(b) if b is not None else None
    assert A.data.dtype == np.uint8
    out = np.empty_like(A.data)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_bitwise(_p(A.data), _p(B.data) if B is not None else None, _p(out), A.w, A.h,
                             op, _rect(A.rect), _rect(B.rect if B is not None else A.rect), vo))
    return Img(out, tuple(vo))


def sobel3x3(src, border=BORDER_REPLICATE, cval=0):
    s = _as_img(src)
    assert s.data.dtype == np.uint8
    gx = np.empty(s.data.shape, np.int16)
    gy = np.empty(s.data.shape, np.int16)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_sobel3x3(_p(s.data), _p(gx), _p(gy), s.w, s.h, border, cval,
                              _rect(s.rect), vo))
    return Img(gx, tuple(vo)), Img(gy, tuple(vo))


def window_sum(src, kw=5, kh=5, border=BORDER_UNDEFINED, cval=0) -> Img:
    s = _as_img(src)
    assert s.data.dtype == np.int32
    out = np.empty_like(s.data)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_window_sum_s32(_p(s.data), _p(out), s.w, s.h, kw, kh, border, cval,
                                    _rect(s.rect), vo))
    return Img(out, tuple(vo))


def convolve(src, coeffs, shift=0, border=BORDER_REPLICATE, cval=0, out_dtype=np.int16) -> Img:
    s = _as_img(src)
    assert s.data.dtype == np.uint8
    c = np.ascontiguousarray(np.asarray(coeffs, np.int32))
    kh, kw = c.shape
    out = np.empty(s.data.shape, out_dtype)
    vo = (ctypes.c_int * 4)()
    fn = lib().orc_convolve_u8_u8 if np.dtype(out_dtype) == np.uint8 else lib().orc_convolve_u8_s16
    _check(fn(_p(s.data), _p(out), s.w, s.h, kw, kh, _p(c), shift, border, cval, _rect(s.rect), vo))
    return Img(out, tuple(vo))


def tomasi_response(sxx, syy, sxy) -> Img:
    """Shi-Tomasi response: smaller eigenvalue of [Sxx Sxy; Sxy Syy], F32."""
    A, B, C = _as_img(sxx), _as_img(syy), _as_img(sxy)
    out = np.empty(A.data.shape, np.float32)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_tomasi_response(_p(A.data), _p(B.data), _p(C.data), _p(out), A.w, A.h,
                                     _rect(A.rect), _rect(B.rect), _rect(C.rect), vo))
    return Img(out, tuple(vo))


# --- point operators ----------------------------------------------------------

def magnitude(gx, gy) -> Img:
    a, b = _as_img(gx), _as_img(gy)
    out = np.empty(a.data.shape, np.int16)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_magnitude(_p(a.data), _p(b.data), _p(out), a.w, a.h, _rect(a.rect),
                               _rect(b.rect), vo))
    return Img(out, tuple(vo))


def phase(gx, gy) -> Img:
    a, b = _as_img(gx), _as_img(gy)
    out = np.empty(a.data.shape, np.uint8)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_phase(_p(a.data), _p(b.data), _p(out), a.w, a.h, _rect(a.rect),
                           _rect(b.rect), vo))
    return Img(out, tuple(vo))


def threshold(src, thr, true_val=255, false_val=0) -> Img:
    s = _as_img(src)
    out = np.empty(s.data.shape, np.uint8)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_threshold(_p(s.data), _FMT_OF[s.data.dtype], _p(out), s.w, s.h, 0,
                               float(thr), 0.0, true_val, false_val, _rect(s.rect), vo))
    return Img(out, tuple(vo))


def threshold_range(src, lower, upper, true_val=255, false_val=0) -> Img:
    s = _as_img(src)
    out = np.empty(s.data.shape, np.uint8)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_threshold(_p(s.data), _FMT_OF[s.data.dtype], _p(out), s.w, s.h, 1,
                               float(lower), float(upper), true_val, false_val,
                               _rect(s.rect), vo))
    return Img(out, tuple(vo))


def channel_extract_uyvy(uyvy: np.ndarray, channel: int) -> Img:
    """uyvy: (H, 2W) uint8 rows of U0 Y0 V0 Y1 macro-pixels; channel 0=Y 1=U 2=V."""
    u = np.ascontiguousarray(uyvy)
    h, w2 = u.shape
    w = w2 // 2
    out = np.empty((h, w if channel == 0 else w // 2), np.uint8)
    _check(lib().orc_channel_extract_uyvy(_p(u), _p(out), w, h, channel))
    return Img(out)


ARITH_ADD, ARITH_SUB, ARITH_ABSDIFF = 0, 1, 2


def arith(a, b, out_dtype, op=ARITH_ADD, saturate=True) -> Img:
    A, B = _as_img(a), _as_img(b)
    out = np.empty(A.data.shape, out_dtype)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_arith(_p(A.data), _FMT_OF[A.data.dtype], _p(B.data),
                           _FMT_OF[B.data.dtype], _p(out), _FMT_OF[np.dtype(out_dtype)],
                           A.w, A.h, op, int(saturate), _rect(A.rect), _rect(B.rect), vo))
    return Img(out, tuple(vo))


def multiply(a, b, scale, out_dtype, saturate=True, nearest_even=False) -> Img:
    """Multiply node: a * b * scale (scale rounded to binary32), one rounding
    (toward zero, or to nearest with ties to even), then wrap / saturate."""
    A, B = _as_img(a), _as_img(b)
    out = np.empty(A.data.shape, out_dtype)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_multiply(_p(A.data), _FMT_OF[A.data.dtype], _p(B.data),
                              _FMT_OF[B.data.dtype], _p(out), _FMT_OF[np.dtype(out_dtype)],
                              A.w, A.h, ctypes.c_float(scale), int(saturate), int(nearest_even),
                              _rect(A.rect), _rect(B.rect), vo))
    return Img(out, tuple(vo))


def mean_stddev(src):
    """Global reduction: (mean, stddev, (S1, S2, N)) over the valid rectangle;
    mean and stddev binary32 (Python floats holding binary32 values)."""
    A = _as_img(src)
    sums = (ctypes.c_int64 * 3)()
    out = (ctypes.c_float * 2)()
    _check(lib().orc_mean_stddev(_p(A.data), _FMT_OF[A.data.dtype], A.w, A.h, _rect(A.rect),
                                 sums, out))
    return out[0], out[1], (sums[0], sums[1], sums[2])


def minmaxloc(src):
    """Global reduction: dict(min, max, min_count, max_count, min_loc, max_loc),
    locations (x, y) of the first occurrence in raster order."""
    A = _as_img(src)
    r = (ctypes.c_int64 * 8)()
    _check(lib().orc_minmaxloc(_p(A.data), _FMT_OF[A.data.dtype], A.w, A.h, _rect(A.rect), r))
    return {"min": r[0], "max": r[1], "min_count": r[2], "max_count": r[3],
            "min_loc": (r[4], r[5]), "max_loc": (r[6], r[7])}


def histogram(src, num_bins=256, offset=0, range_=256) -> np.ndarray:
    A = _as_img(src)
    assert A.data.dtype == np.uint8
    bins = np.zeros(num_bins, np.uint32)
    _check(lib().orc_histogram(_p(A.data), A.w, A.h, _rect(A.rect), num_bins, offset, range_,
                               _p(bins)))
    return bins


def equalize_hist(src) -> Img:
    A = _as_img(src)
    assert A.data.dtype == np.uint8
    out = np.empty(A.data.shape, np.uint8)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_equalize_hist(_p(A.data), _p(out), A.w, A.h, _rect(A.rect), vo))
    return Img(out, tuple(vo))


def convert_depth(src, out_dtype, shift=0, saturate=True) -> Img:
    """ConvertDepth (Copy when the formats agree): U8 -> S16 shifts left,
    S16 -> U8 shifts right (floor) then wraps or saturates."""
    A = _as_img(src)
    out = np.empty(A.data.shape, out_dtype)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_convert_depth(_p(A.data), _FMT_OF[A.data.dtype], _p(out),
                                   _FMT_OF[np.dtype(out_dtype)], A.w, A.h, shift, int(saturate),
                                   _rect(A.rect), vo))
    return Img(out, tuple(vo))


def mul_s32(a, b) -> Img:
    A, B = _as_img(a), _as_img(b)
    out = np.empty(A.data.shape, np.int32)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_mul_s16_s32(_p(A.data), _p(B.data), _p(out), A.w, A.h, _rect(A.rect),
                                 _rect(B.rect), vo))
    return Img(out, tuple(vo))


def harris_response(sxx, syy, sxy, kn=1, kd=25) -> Img:
    a, b, c = _as_img(sxx), _as_img(syy), _as_img(sxy)
    out = np.empty(a.data.shape, np.float32)
    vo = (ctypes.c_int * 4)()
    _check(lib().orc_harris_response(_p(a.data), _p(b.data), _p(c.data), _p(out), a.w, a.h,
                                     kn, kd, _rect(a.rect), _rect(b.rect), _rect(c.rect), vo))
    return Img(out, tuple(vo))


def round_ratio(num: int, den: int) -> float:
    return float(lib().orc_round_ratio(num, den))


# --- whole graphs (composed from the node functions above, in C) --------------

def edge_graph(img: np.ndarray, border=BORDER_REPLICATE, cval=0, rounding=ROUND_ZERO,
               thr=100, want_mag=False):
    """Gaussian3x3 -> Sobel3x3 -> Magnitude -> Threshold(thr) and Phase."""
    a = np.ascontiguousarray(img, np.uint8)
    h, w = a.shape
    phase_o = np.empty_like(a)
    mask_o = np.empty_like(a)
    mag = np.empty(a.shape, np.int16) if want_mag else None
    scratch = np.empty(w * h * 8 + 64, np.uint8)
    _check(lib().orc_edge_graph(_p(a), _p(phase_o), _p(mask_o),
                                _p(mag) if want_mag else None, w, h, border, cval, rounding,
                                thr, _p(scratch)))
    return (phase_o, mask_o, mag) if want_mag else (phase_o, mask_o)


def harris_graph(img: np.ndarray, border=BORDER_UNDEFINED, kn=1, kd=25, thr=1e6):
    """Sobel3x3 -> products -> 5x5 window sums -> response -> Threshold(thr)."""
    a = np.ascontiguousarray(img, np.uint8)
    h, w = a.shape
    mask_o = np.empty_like(a)
    resp = np.empty(a.shape, np.float32)
    scratch = np.empty(w * h * 32 + 64, np.uint8)
    _check(lib().orc_harris_graph(_p(a), _p(mask_o), _p(resp), w, h, border, kn, kd,
                                  float(thr), _p(scratch)))
    return mask_o, resp
