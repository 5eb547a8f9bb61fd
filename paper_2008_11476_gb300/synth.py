"""Seeded synthetic workloads for the image-graph path.

This module draws random numbers and paints test images; it holds none of the
graph arithmetic (no filter, no point operator).  Both the CPU oracle tests and
the CUDA path's tests and benchmark take their inputs from here, so each side
sees the same bytes.

The paper evaluates on unnamed camera frames (1020x1020 to 2048x2048); no
dataset is named, so every image is synthetic:

* ``uniform_u8``: independent uniform bytes 0-255.
* ``rects_noise``: a uniform background level, then max(8, W*H/20000)
  axis-aligned rectangles (sides uniform in [W/50, W/4] x [H/50, H/4],
  intensity uniform 0-255, painted in order), then additive Gaussian noise
  (sigma = 10 by default, Box-Muller), rounded half-up and clamped to 0-255.
* ``uyvy``: uniform bytes laid out as UYVY macro-pixels (2 bytes per pixel).
* ``batch_sizes``: image sizes with width uniform in {320..3840} and height
  uniform in {240..2160}.
* ``poisson_arrivals``: exponential inter-arrival times of a Poisson process.

The generator is counter based: value i of stream s under seed k is
SplitMix64's output function (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to a unique 64-bit
counter built from (k, s, i).  It is vectorised with numpy uint64 arithmetic
and gives identical bytes on every machine.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z + _GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    k = _mix(np.array([(seed & 0xFFFFFFFF) << 20 | (stream & 0xFFFFF)], np.uint64))
    return k[0]


def bits64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n independent 64-bit words of stream `stream` under `seed`."""
    with np.errstate(over="ignore"):
        idx = np.arange(start, start + n, dtype=np.uint64)
        return _mix(idx * _GOLDEN ^ _key(seed, stream))


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform in (0, 1): (top 53 bits + 0.5) / 2^53."""
    b = bits64(seed, stream, n) >> np.uint64(11)
    return (b.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def randint(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive), by multiply-shift."""
    span = np.uint64(hi - lo + 1)
    b = bits64(seed, stream, n) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return ((b * span) >> np.uint64(32)).astype(np.int64) + lo


def uniform_u8(w: int, h: int, seed: int) -> np.ndarray:
    b = bits64(seed, 0, w * h) >> np.uint64(56)
    return b.astype(np.uint8).reshape(h, w)


def rects_noise(w: int, h: int, seed: int, sigma: float = 10.0,
                n_rects: int | None = None) -> np.ndarray:
    n = n_rects if n_rects is not None else max(8, (w * h) // 20000)
    bg = int(randint(seed, 1, 1, 0, 255)[0])
    img = np.full((h, w), bg, np.float64)
    rw_lo, rw_hi = max(1, w // 50), max(1, w // 4)
    rh_lo, rh_hi = max(1, h // 50), max(1, h // 4)
    rw = randint(seed, 2, n, rw_lo, rw_hi)
    rh = randint(seed, 3, n, rh_lo, rh_hi)
    fx = uniform01(seed, 4, n)
    fy = uniform01(seed, 5, n)
    val = randint(seed, 6, n, 0, 255)
    for k in range(n):
        x0 = int(fx[k] * (w - rw[k] + 1))
        y0 = int(fy[k] * (h - rh[k] + 1))
        img[y0:y0 + rh[k], x0:x0 + rw[k]] = val[k]
    if sigma > 0:
        u1 = uniform01(seed, 7, w * h).reshape(h, w)
        u2 = uniform01(seed, 8, w * h).reshape(h, w)
        img += sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return np.clip(np.floor(img + 0.5), 0, 255).astype(np.uint8)


def uyvy(w: int, h: int, seed: int) -> np.ndarray:
    """(h, 2*w) bytes: w/2 macro-pixels U Y V Y per row (w must be even)."""
    assert w % 2 == 0
    b = bits64(seed, 9, 2 * w * h) >> np.uint64(56)
    return b.astype(np.uint8).reshape(h, 2 * w)


def batch_sizes(n: int, seed: int, wlo=320, whi=3840, hlo=240, hhi=2160):
    ws = randint(seed, 10, n, wlo, whi)
    hs = randint(seed, 11, n, hlo, hhi)
    return [(int(a), int(b)) for a, b in zip(ws, hs)]


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of the first n events at `rate_hz`."""
    u = uniform01(seed, 12, n)
    return np.cumsum(-np.log(u) / rate_hz)


def choice(seed: int, stream: int, n: int, weights) -> np.ndarray:
    """n indices drawn with the given probabilities."""
    c = np.cumsum(np.asarray(weights, np.float64))
    c /= c[-1]
    u = uniform01(seed, stream, n)
    return np.searchsorted(c, u, side="right")
