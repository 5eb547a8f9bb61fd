// Device helpers shared by the image-graph kernels: TMA / mbarrier wrappers in
// inline PTX (sm_90+ async proxy, compiled for sm_103a), bounded waits, and
// the exact point-operator arithmetic (Magnitude, Phase, Harris response).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernel_params.h"

namespace hvx {
namespace dev {

// ---------------------------------------------------------------------------
// TMA and mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Make the mbarrier initialisation visible to the async proxy (TMA).
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this CTA's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Acquire a tensor map that lives in global memory before the first TMA
// that uses it.
__device__ __forceinline__ void tensormap_acquire(const void* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 2-D tiled TMA load of box (x, y) of `map` into shared memory; completion
// is signalled on `bar` as transaction bytes.  x * element size must be a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Bulk copy (no tensor map) of `bytes` from global to shared memory,
// signalled on `bar`; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Error codes written to the context's device error word.
constexpr int ERR_TMA_TIMEOUT = 1;

// Wait for phase `parity` of `bar` for at most ~2^31 SM cycles (about a
// second).  On time-out, record the error, wait once more with the same limit
// so that a late copy does not land after the CTA has moved on, and return
// false; the caller then leaves the tile.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  long long limit = 1ll << 31) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            if (err) atomicCAS(err, 0, ERR_TMA_TIMEOUT);
            long long t1 = clock64();
            while (!mbar_try_wait(bar, parity) && clock64() - t1 < limit) {
            }
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Magnitude: floor(sqrt(s) + 1/2) for s = gx^2 + gy^2 (s < 2^32), exact.
// sqrtf is correctly rounded; one integer correction each way removes the
// error of converting s to binary32, then the half-up rounding is decided in
// integers: sqrt(s) >= r + 1/2  <=>  s > r^2 + r.
__device__ __forceinline__ uint32_t isqrt_round(uint32_t s) {
    uint32_t r = (uint32_t)sqrtf((float)s);
    r -= (r * r > s) ? 1u : 0u;
    r += ((r + 1) * (r + 1) <= s) ? 1u : 0u;
    return r + ((s - r * r > r) ? 1u : 0u);
}

__device__ __forceinline__ int magnitude_s16(int gx, int gy) {
    uint32_t s = (uint32_t)(gx * gx) + (uint32_t)(gy * gy);
    uint32_t m = isqrt_round(s);
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

__device__ __forceinline__ uint32_t phase_u8(int gx, int gy) {
    int ax = abs(gx), ay = abs(gy);
    int mx = max(ax, ay), mn = min(ax, ay);
    if (mx == 0) return 0u;
    int ra = phase_octant_round(mn, mx);
    int q1 = ay > ax ? 64 - ra : ra;  // first-quadrant angle, 0 .. 64
    int q = gy >= 0 ? (gx >= 0 ? q1 : 128 - q1) : (gx >= 0 ? 256 - q1 : 128 + q1);
    return (uint32_t)q & 255u;
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
// small helpers

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ bool rect_full(const int32_t* r, int W, int H) {
    return r[0] == 0 && r[1] == 0 && r[2] == W && r[3] == H;
}

__device__ __forceinline__ bool in_rect(const int32_t* r, int x, int y) {
    return x >= r[0] && x < r[2] && y >= r[1] && y < r[3];
}

__device__ __forceinline__ int sat_u8(int v) { return min(max(v, 0), 255); }
__device__ __forceinline__ int sat_s16(int v) { return min(max(v, -32768), 32767); }

// One point operator (Table 2 "point") on the values a, b, c of its inputs at
// one pixel.  P is GenStage or PlainParams; both carry op, i0..i3, f0, f1,
// k0, k1 with the meaning below.  Results are int32, or binary32 bits for F32.
//   Threshold: i0 type, i1 true value, i2 false value, i3 input is F32;
//              k0 / k1 integer lower(value) / upper, f0 / f1 binary32 ones.
//   Add / Subtract / AbsDiff: i0 saturate, i1 output format.
//   Harris response: k0 = kn, k1 = kd.
template <class P>
__device__ __forceinline__ int32_t eval_point(const P& st, int32_t a, int32_t b, int32_t c) {
    switch (st.op) {
        case OP_MAG: return magnitude_s16(a, b);
        case OP_PHASE: return (int32_t)phase_u8(a, b);
        case OP_THRESH: {
            bool t;
            if (st.i3) {
                float f = __int_as_float(a);
                t = st.i0 == HVX_THRESHOLD_BINARY ? f > st.f0 : !(f > st.f1 || f < st.f0);
            } else {
                long long iv = a;
                t = st.i0 == HVX_THRESHOLD_BINARY ? iv > st.k0 : !(iv > st.k1 || iv < st.k0);
            }
            return t ? st.i1 : st.i2;
        }
        case OP_CHX: return (a >> 8) & 0xFF;  // Y byte of a UYVY pixel pair
        case OP_ADD:
        case OP_SUB:
        case OP_ABSDIFF: {
            int r = st.op == OP_ADD ? a + b : (st.op == OP_SUB ? a - b : abs(a - b));
            if (st.i1 == HVX_DF_U8) return st.i0 ? sat_u8(r) : (r & 0xFF);
            return st.i0 ? sat_s16(r) : (int32_t)(int16_t)(uint16_t)(r & 0xFFFF);
        }
        case OP_MUL: return a * b;
        case OP_AND: return a & b;
        case OP_OR: return a | b;
        case OP_XOR: return a ^ b;
        case OP_NOT: return ~a & 0xFF;
        case OP_HARRIS:
            return __float_as_int(ratio_to_float(harris_q(a, b, c, st.k0, st.k1), st.k1));
        case OP_TOMASI: {
            // smaller eigenvalue of [a c; c b] = (tr - s) / 2 = 2 det / (tr + s),
            // s = sqrt((a - b)^2 + 4 c^2), without the cancellation of tr - s
            const long long det = (long long)a * b - (long long)c * c;
            const long long d = (long long)a - b;
            const long long disc = d * d + 4ll * c * c;  // < 2^53 for |a|, |b|, |c| < 2^25
            const float s = sqrtf((float)disc), tr = (float)((long long)a + b);
            const float den = tr + s;
            return __float_as_int(den == 0.0f ? tr : 2.0f * (float)det / den);
        }
    }
    return 0;
}

// Calls f(r, c) for every cell (r, c) of an R x C box whose top-left cell is
// image pixel (bx, by) and that lies outside the W x H image: the full rows
// above and below the image, then the left / right strips of the rows in
// between, spread over the CTA's threads.
template <class F>
__device__ __forceinline__ void for_each_outside(int R, int C, int bx, int by, int W, int H, F f) {
    const int cl = clampi(-bx, 0, C), cr = max(cl, clampi(W - bx, 0, C));
    const int rt = clampi(-by, 0, R), rb = max(rt, clampi(H - by, 0, R));
    const int nfull = (rt + (R - rb)) * C;
    const int side = cl + (C - cr);
    const int n = nfull + (rb - rt) * side;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int r, c;
        if (i < nfull) {
            int rr = i / C;
            c = i - rr * C;
            r = rr < rt ? rr : rb + (rr - rt);
        } else {
            int j = i - nfull;
            int rr = j / side;
            int k = j - rr * side;
            r = rt + rr;
            c = k < cl ? k : cr + (k - cl);
        }
        f(r, c);
    }
}

// ---------------------------------------------------------------------------
// 16-bit-lane (SWAR) helpers of the U8 stencil kernels: two pixels per
// 32-bit word, so that one add or shift works on both.

// 16-bit lane pairs of bytes: (b0, b1) and (b2, b3) of a word.
__device__ __forceinline__ uint32_t lo_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4140); }
__device__ __forceinline__ uint32_t hi_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4342); }

// (lane1 of a, lane0 of b): the pair starting one pixel to the right of a.
__device__ __forceinline__ uint32_t shift_pair(uint32_t a, uint32_t b) {
    return __funnelshift_r(a, b, 16);
}

// Batch tile t -> image: the last i with tile_start[i] <= t (binary search
// over the n + 1 prefix sums of per-image tile counts), in global memory or
// in a shared-memory copy.
__device__ __forceinline__ int find_image(const int* tile_start, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int find_image_smem(const int* tile_start, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_start[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace dev
}  // namespace hvx
