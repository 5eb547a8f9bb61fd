"""Generate the constants of the CUDA Phase evaluations (phase_table.h).

Phase (Table 2 point operator) is q = round(atan2(gy, gx) * 128 / pi) mod 256.
Both CUDA forms reduce it to the octant angle a = atan(t) * 128 / pi, t = mn / mx
in [0, 1] (mn, mx = min, max of |gx|, |gy|), in units of the 256 bins per
turn, and round a exactly.

1. phase_u8 (plain and generic kernels) evaluates a as t * P(t^2), P of degree
   6 (fit below, max error 1.4e-5 bins), and re-decides in double the pixels
   within 1e-4 of a rounding boundary against cos / sin of the boundaries
   b_j = (j + 1/2) pi / 128, j = 0..31 (kPhaseBoundCos / kPhaseBoundSin).

2. The fused edge kernel takes one cheap guess y = t (A + B t) (max error
   0.14 bins, so n = floor(y + 1) is the true rounded value or one above it;
   a round-down fma adds 1.5 * 2^23 + 1, so that n is read off the low
   mantissa bits) and always decides between n - 1 and n with one exact test
   against the boundary beta_n = (n - 1/2) pi / 128 (n = 1..33):
       a >= n - 1/2  <=>  mn - mx tan(beta_n) > 0,
   evaluated as fma(-mx, T_n, mn) with T_n = tan(beta_n) rounded to binary32
   (kPhaseTan).  Over all integer gradients (|gx|, |gy| <= 1020)
   |mn - mx tan(beta_n)| is at least 3.15e-5 while mx |tan(beta_n) - T_n| is
   at most 2.93e-5, so the exact value of the fma has the true sign, and its
   one rounding keeps that sign (it is never 0 for mx >= 1).  mx is raised
   to 1 for gx = gy = 0, which makes the test negative there (phase 0).  The
   kernel's table, indexed by octant and n, maps the octant angle to the
   phase byte.  verify_tan_test() and verify_phase_all() check every pair.

Run: python gen_phase_poly.py [path of phase_table.h to write]
"""
import sys

import numpy as np

GMAX = 1020  # largest |gx|, |gy| of Sobel3x3 on U8 input


def fit(deg=6, n=4000, iters=60):
    k = np.arange(n)
    t = np.sort(np.cos(np.pi * (k + 0.5) / n) * 0.5 + 0.5)
    y = np.arctan(t) * 128 / np.pi
    u = t * t
    V = np.stack([t * u ** j for j in range(deg + 1)], 1)
    w = np.ones(n)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
        e = V @ c - y
        w = w * (1 + np.abs(e) / np.abs(e).max())
        w /= w.mean()
    return c.astype(np.float32)


def max_error_f32(cf):
    tt = np.linspace(0, 1, 2000001).astype(np.float32)
    uu = (tt * tt).astype(np.float32)
    p = np.float32(cf[-1])
    for j in range(len(cf) - 2, -1, -1):
        p = (p * uu + cf[j]).astype(np.float32)
    a = (p * tt).astype(np.float32)
    return np.abs(a.astype(np.float64) - np.arctan(tt.astype(np.float64)) * 128 / np.pi).max()


def boundary_table():
    """cos / sin of the 32 rounding boundaries (j + 1/2) * pi / 128, j = 0..31,
    of the octant angle (used by the exact re-decision near a boundary)."""
    b = (np.arange(32) + 0.5) * np.pi / 128
    return np.cos(b), np.sin(b)


# ---- the edge kernel's guess and exact test ----------------------------------------

def fit_guess(n=20001, iters=200):
    """Minimax-weighted fit of t (A + B t) to atan(t) * 128 / pi on [0, 1]."""
    t = np.linspace(0.0, 1.0, n)
    y = np.arctan(t) * 128 / np.pi
    V = np.stack([t, t * t], 1)
    w = np.ones(n)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
        e = V @ c - y
        w = w * (1 + np.abs(e) / np.abs(e).max())
        w /= w.mean()
    return np.float32(c[0]), np.float32(c[1])


def tan_table():
    """tan((n - 1/2) pi / 128), n = 0..33, rounded to binary32, and the
    rounding error of each entry (in double)."""
    import mpmath
    mpmath.mp.prec = 200
    hi, err = [], []
    for n in range(34):
        tv = mpmath.tan((n - mpmath.mpf(1) / 2) * mpmath.pi / 128)
        h = np.float32(float(tv))
        hi.append(h)
        err.append(float(tv - mpmath.mpf(float(h))))
    return np.array(hi, np.float32), np.array(err)


def _all_pairs():
    mx, mn = np.meshgrid(np.arange(GMAX + 1), np.arange(GMAX + 1), indexing="ij")
    keep = mn <= mx
    return mn[keep].astype(np.float64), mx[keep].astype(np.float64)


def _guess_n(t, A, B):
    """n = floor(t * fma(t, B, A) + 1) as the kernel's round-down fma forms it
    (the product is exact in double, and so is adding 1)."""
    inner = np.float32(np.float64(t) * np.float64(B) + np.float64(A))
    return np.floor(np.float64(t) * np.float64(inner) + 1.0).astype(np.int64)


def _perturbed(t0, du):
    t = t0
    for _ in range(abs(du)):
        t = np.nextafter(t, np.float32(np.inf if du > 0 else -np.inf))
    return np.where(t0 == 0, t0, t).astype(np.float32)


def verify_tan_test(A=None, B=None, T=None, rcp_ulps=4):
    """Emulate the edge kernel's octant rounding on every integer pair
    0 <= mn <= mx <= 1020 and compare with round(atan(mn / mx) * 128 / pi).

    The guess is checked with t moved by +-rcp_ulps binary32 ulps (the
    hardware reciprocal is approximate); the exact test is emulated
    bit-exactly: mn - max(mx, 1) T_n is formed exactly in double (a 10-bit
    integer times a binary32 value) and rounded once to binary32, as the fma
    does.  Returns the number of mismatching pairs (0 expected) and the
    smallest |mn - mx tan(beta_n)| over the pairs with mx > 0.
    """
    if A is None:
        A, B = fit_guess()
    if T is None:
        T, _ = tan_table()
    mn, mx = _all_pairs()
    truth = np.floor(np.arctan2(mn, mx) * 128 / np.pi + 0.5).astype(np.int64)
    mx1 = np.maximum(mx, 1.0)
    bad = 0
    tmin = np.inf
    t0 = (mn / mx1).astype(np.float32)
    for du in (-rcp_ulps, 0, rcp_ulps):
        n = _guess_n(_perturbed(t0, du), A, B)
        if n.min() < 1 or n.max() > 33:
            return -1, 0.0
        h = np.float32(mn - mx1 * np.float64(T[n]))  # the fma, rounded once
        if np.any(h == 0):
            return -1, 0.0
        ra = n - (h < 0)
        bad += int(np.count_nonzero(ra != truth))
        if du == 0:
            gap = np.abs(mn - mx * np.tan((n - 0.5) * np.pi / 128))
            tmin = float(gap[mx > 0].min())
    return bad, tmin


def phase_table(T=None):
    """The kernel's (octant, n) table: octant o = 4 [gx < 0] + 2 [gy < 0] +
    [|gy| > |gx|]; entry o * 34 + n holds T_n and the phase bytes for the
    octant angle n (q_ge) and n - 1 (q_lt)."""
    if T is None:
        T, _ = tan_table()
    q_ge = np.zeros(8 * 34, np.int64)
    q_lt = np.zeros(8 * 34, np.int64)
    for o in range(8):
        sx, sy, sw = (o >> 2) & 1, (o >> 1) & 1, o & 1
        for n in range(34):
            for k, dst in ((0, q_ge), (1, q_lt)):
                ra = n - k
                q1 = 64 - ra if sw else ra
                dst[o * 34 + n] = ((128 if sx else 0) + (-q1 if sx != sy else q1)) & 255
    return np.tile(T, 8), q_ge, q_lt


def verify_phase_all(A=None, B=None, T=None, table=None):
    """Every (gx, gy) in [-1020, 1020]^2 through the emulated kernel Phase
    (guess, table, exact test) against round(atan2(gy, gx) * 128 / pi) mod
    256.  Returns the number of mismatches (0 expected)."""
    if A is None:
        A, B = fit_guess()
    tan8, q_ge, q_lt = phase_table(T) if table is None else table
    g = np.arange(-GMAX, GMAX + 1, dtype=np.float64)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    gx, gy = gx.ravel(), gy.ravel()
    ax, ay = np.abs(gx), np.abs(gy)
    mx = np.maximum(np.maximum(ax, ay), 1.0)
    mn = np.minimum(ax, ay)
    n = _guess_n((mn / mx).astype(np.float32), A, B)
    o = 136 * (gx < 0) + 68 * (gy < 0) + 34 * (ay > ax)
    idx = o + n
    h = np.float32(mn - mx * np.float64(tan8[idx]))
    q = np.where(h < 0, q_lt[idx], q_ge[idx])
    ang = np.arctan2(gy, gx)
    ang = np.where(ang < 0, ang + 2 * np.pi, ang)
    truth = np.floor(ang * 128 / np.pi + 0.5).astype(np.int64) % 256
    return int(np.count_nonzero(q != truth))


def write_table_header(path):
    c, s = boundary_table()
    A, B = fit_guess()
    T, _ = tan_table()
    fmt = lambda v: ",\n    ".join(", ".join(f"{x:.17g}" for x in v[i:i + 4]) for i in range(0, 32, 4))
    tans = ",\n    ".join(", ".join(f"{float(T[i])!r}f" for i in range(j, min(j + 4, 34)))
                          for j in range(0, 34, 4))
    with open(path, "w") as f:
        f.write("// Generated by gen_phase_poly.py (constants of the Phase evaluations).\n"
                "// Do not edit.\n#pragma once\n\n"
                "// cos / sin of the octant-angle rounding boundaries (j + 1/2) pi / 128,\n"
                "// j = 0..31 (phase_u8's exact re-decision).\n"
                f"static __constant__ double kPhaseBoundCos[32] = {{\n    {fmt(c)}}};\n\n"
                f"static __constant__ double kPhaseBoundSin[32] = {{\n    {fmt(s)}}};\n\n"
                "// tan((n - 1/2) pi / 128), n = 0..33, rounded to binary32 (the edge\n"
                "// kernel's exact test; copied to shared memory by each CTA).\n"
                f"static __device__ const float kPhaseTan[34] = {{\n    {tans}}};\n\n"
                "// Guess of the octant angle in bins: t (A + B t), |error| <= 0.14.\n"
                f"constexpr float kPhaseGuessA = {float(A)!r}f;\n"
                f"constexpr float kPhaseGuessB = {float(B)!r}f;\n")


if __name__ == "__main__":
    cf = fit()
    print("degree-6 coefficients (c0..c6):", ", ".join(f"{float(c)!r}f" for c in cf))
    print("max |error| in bins (binary32 Horner):", max_error_f32(cf))
    A, B = fit_guess()
    t = np.linspace(0, 1, 200001)
    print("guess A, B:", float(A), float(B), "max |error| in bins:",
          np.abs(t * (A + B * t) - np.arctan(t) * 128 / np.pi).max())
    T, err = tan_table()
    print("largest 1020 |tan - T_n|:", 1020 * np.abs(err).max())
    print("exact test over all integer pairs (mismatches, min gap):", verify_tan_test(A, B, T))
    print("full phase over all (gx, gy) (mismatches):", verify_phase_all(A, B, T))
    if len(sys.argv) > 1:
        write_table_header(sys.argv[1])
