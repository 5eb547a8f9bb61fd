// Exact point-operator arithmetic of the image graphs (Table 2 point
// operators Magnitude and Phase, the Harris and Shi-Tomasi corner responses
// of the Section 6 applications) and the saturations of the arithmetic
// nodes.  Self-contained (no includes but the generated Phase constants) so
// that the library's kernels and the kernels generated at run time for fused
// groups share one definition.
#pragma once

// ---------------------------------------------------------------------------
// Magnitude: floor(sqrt(s) + 1/2) for s = gx^2 + gy^2 (s < 2^32), exact.
// sqrtf is correctly rounded; one integer correction each way removes the
// error of converting s to binary32, then the half-up rounding is decided in
// integers: sqrt(s) >= r + 1/2  <=>  s > r^2 + r.
__device__ __forceinline__ unsigned int isqrt_round(unsigned int s) {
    unsigned int r = (unsigned int)sqrtf((float)s);
    r -= (r * r > s) ? 1u : 0u;
    r += ((r + 1) * (r + 1) <= s) ? 1u : 0u;
    return r + ((s - r * r > r) ? 1u : 0u);
}

__device__ __forceinline__ int magnitude_s16(int gx, int gy) {
    unsigned int s = (unsigned int)(gx * gx) + (unsigned int)(gy * gy);
    unsigned int m = isqrt_round(s);
    return (int)(m > 32767u ? 32767u : m);
}

// ---------------------------------------------------------------------------
// Phase: q = floor(atan2(gy, gx) * 128 / pi + 1/2) mod 256, angle in [0, 2 pi).
//
// With mn = min(|gx|,|gy|), mx = max(|gx|,|gy|), the octant angle in bins
// (128 / pi units) is a = atan(mn / mx) * 128 / pi in [0, 32], and the full
// angle is B + s*a for a quadrant base B in {0, 64, 128, 256} and s = +-1.
// a is never a half-integer for integer gradients (atan of a rational is a
// rational multiple of pi only at 0 and 1), so round(B + s*a) = B + s*round(a)
// and only the octant angle has to be rounded.  It is evaluated as t * P(t^2),
// t = mn / mx, with P from gen_phase_poly.py (max error 1.4e-5 bins in
// binary32).  When a + 1/2 lies within 1e-4 of an integer (about 1.5e-4 of all
// integer pairs) the rounding is re-decided exactly: a >= j + 1/2 holds iff
// mn cos(b_j) - mx sin(b_j) >= 0 with b_j = (j + 1/2) pi / 128, evaluated in
// double (its magnitude is at least 2.9e-5 for 11-bit gradients, far above
// double rounding error).

#include "phase_table.h"

__device__ __forceinline__ int phase_octant_round(int mn, int mx) {
    float t = __fdividef((float)mn, (float)mx);
    float u = t * t;
    float p = 0.27753710746765137f;
    p = fmaf(p, u, -1.3691582679748535f);
    p = fmaf(p, u, 3.244159698486328f);
    p = fmaf(p, u, -5.391748428344727f);
    p = fmaf(p, u, 8.070429801940918f);
    p = fmaf(p, u, -13.574716567993164f);
    p = fmaf(p, u, 40.743507385253906f);
    float f = fmaf(p, t, 0.5f);
    float fl = floorf(f);
    float d = f - fl;
    int ra = (int)fl;
    if (fabsf(d - 0.5f) > 0.5f - 1e-4f) {
        int j = d < 0.5f ? ra - 1 : ra;  // the boundary a + 1/2 is close to
        if (j >= 0 && j < 32) {
            double cr = (double)mn * kPhaseBoundCos[j] - (double)mx * kPhaseBoundSin[j];
            ra = cr >= 0.0 ? j + 1 : j;
        }
    }
    return ra;
}

__device__ __forceinline__ unsigned int phase_u8(int gx, int gy) {
    int ax = abs(gx), ay = abs(gy);
    int mx = max(ax, ay), mn = min(ax, ay);
    if (mx == 0) return 0u;
    int ra = phase_octant_round(mn, mx);
    int q1 = ay > ax ? 64 - ra : ra;  // first-quadrant angle, 0 .. 64
    int q = gy >= 0 ? (gx >= 0 ? q1 : 128 - q1) : (gx >= 0 ? 256 - q1 : 128 + q1);
    return (unsigned int)q & 255u;
}

// ---------------------------------------------------------------------------
// Harris response.  Sxx, Syy, Sxy are exact integer window sums, so with
// k = kn / kd the scaled response q = kd * (Sxx Syy - Sxy^2) - kn (Sxx + Syy)^2
// is an exact 64-bit integer (|S| <= 2^25, which covers every 5x5 sum of
// Sobel3x3 products, keeps it below 2^63 for kn, kd <= 1000), and R = q / kd.

__device__ __forceinline__ long long harris_q(int a, int b, int c, long long kn, long long kd) {
    long long det = (long long)a * b - (long long)c * c;
    long long tr = (long long)a + b;
    return kd * det - kn * tr * tr;
}

// Binary32 value nearest to m / d (ties to even), m < 2^62, 1 <= d <= 1000:
// a candidate from two correctly rounded steps (m to binary32, then the
// division) is within about one unit in the last place; it is then moved to
// the correctly rounded value by exact integer comparisons against the
// midpoints to its neighbours.
__device__ __forceinline__ float ratio_to_float(long long q, long long d) {
    if (q == 0) return 0.0f;
    bool neg = q < 0;
    unsigned long long m = neg ? (unsigned long long)(-q) : (unsigned long long)q;
    float c = __fdiv_rn(__ull2float_rn(m), (float)d);
    for (int it = 0; it < 4; ++it) {
        int e;
        float fr = frexpf(c, &e);                      // c = fr * 2^e, fr in [1/2, 1)
        unsigned int M = (unsigned int)ldexpf(fr, 24); // c = M * 2^(e - 24)
        int sh = 2 - (e - 24);                         // compare m * 2^sh with (4M +- k) d
        unsigned __int128 L = m;
        unsigned __int128 Hi = (unsigned __int128)(4ull * M + 2ull) * (unsigned long long)d;
        unsigned __int128 Lo =
            (unsigned __int128)(4ull * M - (M == (1u << 23) ? 1ull : 2ull)) * (unsigned long long)d;
        if (sh >= 0) {
            L <<= sh;
        } else {
            Hi <<= -sh;
            Lo <<= -sh;
        }
        if (L > Hi || (L == Hi && (M & 1u)))
            c = nextafterf(c, 3.0e38f);
        else if (L < Lo || (L == Lo && (M & 1u)))
            c = nextafterf(c, 0.0f);
        else
            break;
    }
    return neg ? -c : c;
}

// ---------------------------------------------------------------------------
// Saturation of Add / Subtract / Convolve results.

__device__ __forceinline__ int sat_u8(int v) { return min(max(v, 0), 255); }
__device__ __forceinline__ int sat_s16(int v) { return min(max(v, -32768), 32767); }

// ---------------------------------------------------------------------------
// Multiply: a * b * scale for scale = m * 2^e (m the 24-bit significand of a
// binary32 scale <= 2^16), exact in 64-bit integers (|a b m| < 2^54), rounded
// once toward zero or to nearest with ties to even.
__device__ __forceinline__ long long multiply_scaled(int a, int b, long long m, int e,
                                                     bool nearest_even) {
    const long long p = (long long)a * b * m;
    if (e >= 0) return p << e;  // |p| 2^e <= 2^30 * 2^16
    const int k = -e;
    if (k > 62) return 0;       // |p| 2^-k < 2^54 / 2^63 < 1/2
    const unsigned long long u = p < 0 ? 0ull - (unsigned long long)p : (unsigned long long)p;
    unsigned long long q = u >> k;
    if (nearest_even) {
        const unsigned long long rem = u & ((1ull << k) - 1), half = 1ull << (k - 1);
        if (rem > half || (rem == half && (q & 1ull))) ++q;
    }
    return p < 0 ? -(long long)q : (long long)q;
}

// Saturation / wrap-around of a 64-bit result to U8 or S16.
__device__ __forceinline__ int sat64_u8(long long v) { return (int)(v < 0 ? 0 : (v > 255 ? 255 : v)); }
__device__ __forceinline__ int sat64_s16(long long v) {
    return (int)(v < -32768 ? -32768 : (v > 32767 ? 32767 : v));
}
__device__ __forceinline__ int wrap64_s16(long long v) { return (int)(short)(unsigned short)(v & 0xFFFF); }
__device__ __forceinline__ int sat64_s32(long long v) {
    return (int)(v < -2147483648ll ? -2147483648ll : (v > 2147483647ll ? 2147483647ll : v));
}

// ---------------------------------------------------------------------------
// Shi-Tomasi response: the smaller eigenvalue of the structure matrix
// [a c; c b] of exact integer window sums, (tr - s) / 2 = 2 det / (tr + s)
// with s = sqrt((a - b)^2 + 4 c^2), written without the cancellation of
// tr - s; binary32.
__device__ __forceinline__ float tomasi_response_f32(int a, int b, int c) {
    const long long det = (long long)a * b - (long long)c * c;
    const long long d = (long long)a - b;
    const long long disc = d * d + 4ll * c * c;  // < 2^53 for |a|, |b|, |c| < 2^25
    const float s = sqrtf((float)disc), tr = (float)((long long)a + b);
    const float den = tr + s;
    return den == 0.0f ? tr : 2.0f * (float)det / den;
}
