"""Generate the coefficients of the Phase kernel's arctangent polynomial.

The CUDA Phase op evaluates A(t) = atan(t) * 128 / pi on t in [0, 1] (one
octant, in units of the 256 phase bins per turn) as t * P(t^2), P of degree 6.
This script fits P by iteratively re-weighted least squares towards the
minimax error on Chebyshev nodes and prints the binary32 coefficients and the
maximum error of a binary32 Horner evaluation.  The kernel's exact-rounding
fallback covers the remaining error (it re-decides every pixel whose value lies
within 1e-4 bins of a rounding boundary).

Run: python gen_phase_poly.py
"""
import numpy as np


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


if __name__ == "__main__":
    cf = fit()
    print("coefficients (c0..c6):", ", ".join(f"{float(c)!r}f" for c in cf))
    print("max |error| in bins (binary32 Horner):", max_error_f32(cf))


def boundary_table():
    """cos / sin of the 32 rounding boundaries (j + 1/2) * pi / 128, j = 0..31,
    of the octant angle (used by the exact re-decision near a boundary)."""
    b = (np.arange(32) + 0.5) * np.pi / 128
    return np.cos(b), np.sin(b)


def write_table_header(path):
    c, s = boundary_table()
    fmt = lambda v: ",\n    ".join(", ".join(f"{x:.17g}" for x in v[i:i + 4]) for i in range(0, 32, 4))
    with open(path, "w") as f:
        f.write("// Generated by gen_phase_poly.py: cos / sin of the octant-angle rounding\n"
                "// boundaries (j + 1/2) * pi / 128, j = 0..31.  Do not edit.\n#pragma once\n\n"
                f"static __constant__ double kPhaseBoundCos[32] = {{\n    {fmt(c)}}};\n\n"
                f"static __constant__ double kPhaseBoundSin[32] = {{\n    {fmt(s)}}};\n")


if __name__ == "__main__" and len(__import__("sys").argv) > 1:
    write_table_header(__import__("sys").argv[1])
