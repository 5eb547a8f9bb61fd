// Fused Harris-corner group (HarrisCorners row of Table 2 as point + local +
// custom abstractions; the corner-detector benchmark of Section 6):
//
//   in U8 --Sobel3x3--> gx, gy (S16) --point--> gx^2, gy^2, gx*gy (S32)
//        --local 5x5 window sums--> Sxx, Syy, Sxy (S32)
//        --point--> R = Sxx Syy - Sxy^2 - k (Sxx + Syy)^2 (F32)
//        --Threshold--> mask (U8)
//
// One CTA computes a 64 x 32 output tile from a TMA box of the input with a
// 3-pixel halo:
//   1. edge tiles apply the Sobel's border mode to the input bytes outside
//      the image;
//   2. items of 4 pixels of one row compute gx, gy with separable sums and
//      store the three exact int32 products (16-byte stores) over the tile +
//      2-pixel halo;
//   3. edge tiles apply the window sums' border mode to the product cells
//      outside the image;
//   4. vertical 5-sums, 4 columns x 8 rows per item, sliding, 16-byte loads
//      and stores;
//   5. each thread takes 8 pixels of one row: horizontal 5-sums from three
//      16-byte loads per product, the response in exact 64-bit integer form
//      q = kd * R and the threshold.  R > T on the binary32 value is decided
//      as q > q_thr, where the host computed q_thr so that this equals the
//      comparison of the correctly rounded binary32 response with T.  When R
//      is exported it is rounded once from q / kd.
//
// The Tomasi application of Section 6 is the same group with the Shi-Tomasi
// response (the smaller eigenvalue of [Sxx Sxy; Sxy Syy]) in place of R; both
// kernels below then evaluate tomasi_response_f32 on the window sums, the
// binary32 function the point operator computes, and threshold its value.
#include <atomic>

#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int TW = HARRIS_TW;     // 64
constexpr int TH = HARRIS_TH;     // 32
constexpr int LW = HARRIS_LOAD_W; // 96
constexpr int IN_ROWS = TH + 6;   // 38
constexpr int PR = TH + 4;        // product rows (y0-2 .. y0+TH+1)
constexpr int PC = TW + 4;        // product cols (x0-2 .. x0+TW+1) = 68
constexpr int PCS = TW + 8;       // product row stride (16-byte multiple)
constexpr uint32_t IN_BYTES = IN_ROWS * LW;

struct HarrisSmem {
    alignas(128) uint8_t in[IN_ROWS][LW];  // image (x0 - 16 + c, y0 - 3 + r)
    alignas(16) int32_t p[3][PR][PCS];     // products (x0 - 2 + c, y0 - 2 + r)
    alignas(16) int32_t v[3][TH][PCS];     // vertical 5-sums (x0 - 2 + c, y0 + r)
    alignas(8) uint64_t bar;
};

__device__ __forceinline__ bool interior_tile(const HarrisParams& p, int x0, int y0) {
    return x0 >= 3 && y0 >= 3 && x0 + TW + 3 <= (int)p.W && y0 + TH + 3 <= (int)p.H;
}

__device__ __forceinline__ bool full_rect(const int32_t* r, const HarrisParams& p) {
    return r[0] == 0 && r[1] == 0 && r[2] == (int)p.W && r[3] == (int)p.H;
}

__device__ __forceinline__ int4 add4(int4 a, int4 b) {
    return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ int4 sub4(int4 a, int4 b) {
    return make_int4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

__global__ void __launch_bounds__(HARRIS_THREADS, 3)
    harris_kernel(const __grid_constant__ CUtensorMap tmap, const HarrisParams p) {
    pdl_launch_dependents();  // launched by launch_pdl
    pdl_wait();
    extern __shared__ __align__(128) uint8_t smem_raw[];
    HarrisSmem& sm = *reinterpret_cast<HarrisSmem*>(smem_raw);
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int W = p.W, H = p.H;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&sm.bar, IN_BYTES);
        tma_load_2d(&sm.in[0][0], &tmap, &sm.bar, x0 - 16, y0 - 3);
    }
    // every thread leaves together when the (bounded) wait ran out
    if (__syncthreads_or(!mbar_wait_bounded(&sm.bar, 0, p.err))) return;
    const bool interior = interior_tile(p, x0, y0);

    // 1. the Sobel's border mode on input bytes outside the image
    if (!interior && p.border_s != HVX_BORDER_UNDEFINED) {
        const bool cst = p.border_s == HVX_BORDER_CONSTANT;
        const uint8_t cv = (uint8_t)p.cval_s;
        for_each_outside(IN_ROWS, LW, x0 - 16, y0 - 3, W, H, [&](int r, int c) {
            int x = x0 - 16 + c, y = y0 - 3 + r;
            sm.in[r][c] =
                cst ? cv : sm.in[clampi(y, 0, H - 1) - (y0 - 3)][clampi(x, 0, W - 1) - (x0 - 16)];
        });
        __syncthreads();
    }

    // 2. gx, gy and their products over the tile + 2-pixel halo, 4 pixels per item
    const bool pfull = interior || full_rect(p.pvalid, p);
    constexpr int CHUNKS = PC / 4;  // 17
    for (int it = threadIdx.x; it < PR * CHUNKS; it += blockDim.x) {
        const int r = it / CHUNKS, c = 4 * (it - r * CHUNKS);
        // input rows r .. r+2; columns c+13 .. c+18 hold the windows of the 4 pixels
        int vs[6], dy[6];
        uint32_t w0[3][2];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            w0[d][0] = *reinterpret_cast<const uint32_t*>(&sm.in[r + d][c + 12]);
            w0[d][1] = *reinterpret_cast<const uint32_t*>(&sm.in[r + d][c + 16]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            // byte c+13+k: word (k+1) >> 2, byte (k+1) & 3
            const int wi = (k + 1) >> 2, sh = 8 * ((k + 1) & 3);
            int a = (w0[0][wi] >> sh) & 0xFF, b = (w0[1][wi] >> sh) & 0xFF,
                e = (w0[2][wi] >> sh) & 0xFF;
            vs[k] = a + 2 * b + e;
            dy[k] = e - a;
        }
        int px[4], py[4], pxy[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gx = vs[j + 2] - vs[j];
            int gy = dy[j] + 2 * dy[j + 1] + dy[j + 2];
            if (!pfull) {
                int x = x0 - 2 + c + j, y = y0 - 2 + r;
                if (x >= 0 && x < W && y >= 0 && y < H && !in_rect(p.pvalid, x, y)) gx = gy = 0;
            }
            px[j] = gx * gx;
            py[j] = gy * gy;
            pxy[j] = gx * gy;
        }
        *reinterpret_cast<int4*>(&sm.p[0][r][c]) = make_int4(px[0], px[1], px[2], px[3]);
        *reinterpret_cast<int4*>(&sm.p[1][r][c]) = make_int4(py[0], py[1], py[2], py[3]);
        *reinterpret_cast<int4*>(&sm.p[2][r][c]) = make_int4(pxy[0], pxy[1], pxy[2], pxy[3]);
    }
    __syncthreads();

    // 3. the window sums' border mode on product cells outside the image
    if (!interior && p.border_b != HVX_BORDER_UNDEFINED) {
        const bool cst = p.border_b == HVX_BORDER_CONSTANT;
        for_each_outside(PR, PC, x0 - 2, y0 - 2, W, H, [&](int r, int c) {
            int x = x0 - 2 + c, y = y0 - 2 + r;
            if (cst) {
                sm.p[0][r][c] = sm.p[1][r][c] = sm.p[2][r][c] = p.cval_b;
            } else {
                int cr = clampi(y, 0, H - 1) - (y0 - 2), cc = clampi(x, 0, W - 1) - (x0 - 2);
                sm.p[0][r][c] = sm.p[0][cr][cc];
                sm.p[1][r][c] = sm.p[1][cr][cc];
                sm.p[2][r][c] = sm.p[2][cr][cc];
            }
        });
        __syncthreads();
    }

    // 4. vertical 5-sums: 4 columns x 8 rows per item, sliding
    for (int it = threadIdx.x; it < 3 * CHUNKS * (TH / 8); it += blockDim.x) {
        const int k = it / (CHUNKS * (TH / 8));
        const int rem = it - k * CHUNKS * (TH / 8);
        const int c = 4 * (rem % CHUNKS);
        const int r0 = 8 * (rem / CHUNKS);
        const int32_t(*P)[PCS] = sm.p[k];
        int4 s = add4(add4(*reinterpret_cast<const int4*>(&P[r0][c]),
                           *reinterpret_cast<const int4*>(&P[r0 + 1][c])),
                      add4(add4(*reinterpret_cast<const int4*>(&P[r0 + 2][c]),
                                *reinterpret_cast<const int4*>(&P[r0 + 3][c])),
                           *reinterpret_cast<const int4*>(&P[r0 + 4][c])));
        *reinterpret_cast<int4*>(&sm.v[k][r0][c]) = s;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            s = sub4(add4(s, *reinterpret_cast<const int4*>(&P[r0 + j + 4][c])),
                     *reinterpret_cast<const int4*>(&P[r0 + j - 1][c]));
            *reinterpret_cast<int4*>(&sm.v[k][r0 + j][c]) = s;
        }
    }
    __syncthreads();

    // 5. horizontal 5-sums, response, threshold: 8 pixels of one row per thread
    const int row = threadIdx.x >> 3, seg = threadIdx.x & 7;
    const int y = y0 + row, xs = x0 + seg * 8;
    if (y >= H || xs >= W) return;
    const bool full = interior || full_rect(p.valid, p);
    int S[3][8];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int4* vr = reinterpret_cast<const int4*>(&sm.v[k][row][seg * 8]);
        int4 a = vr[0], b = vr[1], c = vr[2];
        int v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
        int s = v[0] + v[1] + v[2] + v[3] + v[4];
        S[k][0] = s;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            s += v[j + 4] - v[j - 1];
            S[k][j] = s;
        }
    }
    uint32_t mk[8];
    float rv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        bool ok = full || in_rect(p.valid, xs + j, y);
        bool hit;
        float r;
        if (p.tomasi) {
            r = tomasi_response_f32(S[0][j], S[1][j], S[2][j]);
            hit = r > p.thr_f;
        } else {
            long long q = harris_q(S[0][j], S[1][j], S[2][j], p.kn, p.kd);
            hit = q > p.q_thr;
            r = p.resp ? ratio_to_float(q, p.kd) : 0.0f;
        }
        mk[j] = ok ? (hit ? (uint32_t)p.tv : (uint32_t)p.fv) : 0u;
        if (p.resp) rv[j] = ok ? r : 0.0f;
    }
    if (p.mask) {
        uint8_t* dst = p.mask + (size_t)y * p.mask_pitch;
        if (xs + 8 <= W) {
            uint2 w;
            w.x = mk[0] | (mk[1] << 8) | (mk[2] << 16) | (mk[3] << 24);
            w.y = mk[4] | (mk[5] << 8) | (mk[6] << 16) | (mk[7] << 24);
            *reinterpret_cast<uint2*>(dst + xs) = w;
        } else {
            for (int j = 0; j < 8 && xs + j < W; ++j) dst[xs + j] = (uint8_t)mk[j];
        }
    }
    if (p.resp) {
        float* dst = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(p.resp) +
                                              (size_t)y * p.resp_pitch);
        if (xs + 8 <= W) {
            float4* d4 = reinterpret_cast<float4*>(dst + xs);
            d4[0] = make_float4(rv[0], rv[1], rv[2], rv[3]);
            d4[1] = make_float4(rv[4], rv[5], rv[6], rv[7]);
        } else {
            for (int j = 0; j < 8 && xs + j < W; ++j) dst[xs + j] = rv[j];
        }
    }
}

// ---- BORDER_UNDEFINED fast path ------------------------------------------------------
// When both the Sobel and the window sums leave their border UNDEFINED, no
// valid output reads a gradient or product outside the image or outside its
// valid region, so no border fix-up is needed anywhere.  One CTA (128
// threads) computes a 112 x 8R output tile from one TMA box of 144 x (8R + 6)
// input bytes.  Thread (q, g) owns the 8 columns xs = x0 - 8 + 8q .. xs + 7
// (q = 0 .. 15) and R rows; strips 1 .. 14 produce the outputs, strips 0 and
// 15 only provide the vertical sums of the halo columns to their neighbours.
// R (8 .. 24) is chosen per image size at plan time so that the busiest SM
// walks the fewest rows (harris_fast_rows); 4 CTAs share an SM.
// Each thread walks down its rows (three per loop trip, so the input windows
// rotate by renaming):
//   * each step forms one new gradient row (gx, gy at its 8 columns) in
//     biased 16-bit lanes from a sliding 3-row window of input pixel pairs
//     and keeps it in a 5-row ring in shared memory (the thread's own slots);
//   * 24 running vertical 5-sums (8 columns x 3 products, held as pairs of
//     columns in packed binary32, where every value is an exact integer
//     below 2^23) gain the new row's products by packed fmas and, after the
//     outputs of the row, lose the row that leaves the window (its lanes
//     re-read from the ring);
//   * the vertical sums become integers through their bit patterns (v plus
//     2^23 or 1.5 * 2^23), those of columns xs - 2, xs - 1 and xs + 8, xs + 9
//     come from the neighbouring lanes by shuffles, and exact int32
//     horizontal 5-sums slide along the strip;
//   * the mask alone (the benchmark's form) is decided for two pixels per
//     packed binary32 operation between two bounds of q - q_thr (Shi-Tomasi:
//     of r - T), with the exact test only for the pixels the bounds leave
//     open; an exported response is computed exactly from the sums, as in
//     the general kernel.
// Every thread runs all R rows (rows below the image read box rows the TMA
// filled with 0 and are not stored), so the shuffles always see full warps.
constexpr int FTW = 112, FTHREADS = 128;
constexpr int FROWS_MIN = 8, FROWS_MAX = 24;  // boxes up to 144 x 198 bytes
constexpr int FLW = FTW + 32;                 // box columns x0 - 16 .. x0 + 127
constexpr int FLH_MAX = 8 * FROWS_MAX + 6;    // box rows y0 - 3 .. y0 + 8R + 2
constexpr int RING = 5;        // gradient rows of the vertical window
constexpr int RSTRIDE = 11;    // 16-byte units per thread: 5 rows x 2 + 1 (odd: no conflicts)
static_assert(FTHREADS == 16 * 8, "16 strips x 8 row groups");
static_assert(FTW % 16 == 0, "TMA boxes start on 16-byte columns");

struct FastSmem {
    alignas(128) uint8_t in[FLH_MAX][FLW];  // image (x0 - 16 + c, y0 - 3 + r)
    alignas(16) uint4 ring[FTHREADS][RSTRIDE];
    alignas(8) uint64_t bar;
    HarrisParams prm;  // batch: this tile's image parameters
};
static_assert(sizeof(HarrisParams) % 4 == 0, "parameters copied as words");

// Pixel pairs (xs - 2, xs - 1), (xs, xs + 1) .. (xs + 8, xs + 9) of one box
// row, for the strip starting at box column c (= xs - x0 + 16).
__device__ __forceinline__ void load_pairs6(const uint8_t* row, int c, uint32_t P[6]) {
    const uint32_t wl = *reinterpret_cast<const uint32_t*>(row + c - 4);
    const uint2 m = *reinterpret_cast<const uint2*>(row + c);
    const uint32_t wr = *reinterpret_cast<const uint32_t*>(row + c + 8);
    P[0] = hi_pair(wl);
    P[1] = lo_pair(m.x);
    P[2] = hi_pair(m.x);
    P[3] = lo_pair(m.y);
    P[4] = hi_pair(m.y);
    P[5] = lo_pair(wr);
}

// Gradient row from the input pair rows above (a), at (b) and below (c): word
// j holds columns (xs + 2j, xs + 2j + 1); gx + 1024 in G[j], gy + 1024 in
// G[4 + j].  Lanes: vertical sums <= 1020, differences + 255 in [0, 510], so
// every lane stays in [4, 2044] and never borrows from its neighbour.
__device__ __forceinline__ void grad_row(const uint32_t* a, const uint32_t* b, const uint32_t* c,
                                         uint32_t* G) {
    uint32_t V[6], D[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        V[k] = a[k] + 2u * b[k] + c[k];
        D[k] = c[k] + 0x00FF00FFu - a[k];
    }
    uint32_t sv[5], sd[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        sv[k] = shift_pair(V[k], V[k + 1]);  // columns (xs - 1 + 2k, xs + 2k)
        sd[k] = shift_pair(D[k], D[k + 1]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        G[j] = sv[j + 1] + 0x04000400u - sv[j];
        G[4 + j] = sd[j] + sd[j + 1] + 2u * D[j + 1] + 0x00040004u;
    }
}

// Vertical 5-sums of the three products at the strip's 8 columns, as pairs of
// columns (2j, 2j + 1) in packed binary32.  Every product is an integer with
// |gx^2|, |gy^2| <= 1020^2 and |gx gy| <= 765^2 (for the 3x3 Sobel of bytes,
// gx = 2 e1 + u + v and gy = 2 e2 + u - v with e1, e2, u, v differences of
// bytes, so |gx gy| <= 765^2 - v^2), and a sum of at most five rows stays
// below 2^23 in magnitude, so every packed fma below is exact.
struct VSums {
    float2 xx[4], yy[4], xy[4];
};

// s * gx (or s * gy) of a gradient word's two lanes (lane + 1024 each): a
// lane spliced under the exponent of 2^23 is the float 2^23 + lane, and one
// packed fma takes out the offset.
__device__ __forceinline__ float2 lanes_f32(uint32_t w, float s) {
    return __ffma2_rn(make_float2(__int_as_float(__byte_perm(w, 0x4B00u, 0x5410)),
                                  __int_as_float(__byte_perm(w, 0x4B00u, 0x5432))),
                      make_float2(s, s), make_float2(-s * 8389632.0f, -s * 8389632.0f));
}

// V += the products of gradient row G (G[j]: gx lanes, G[4 + j]: gy lanes).
__device__ __forceinline__ void add_products(const uint32_t* G, VSums& V) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 gx = lanes_f32(G[j], 1.0f), gy = lanes_f32(G[4 + j], 1.0f);
        V.xx[j] = __ffma2_rn(gx, gx, V.xx[j]);
        V.yy[j] = __ffma2_rn(gy, gy, V.yy[j]);
        V.xy[j] = __ffma2_rn(gx, gy, V.xy[j]);
    }
}

// V -= the products of gradient row G (packed operands take no negation, so
// -gx and -gy come from their own fmas).
__device__ __forceinline__ void sub_products(const uint32_t* G, VSums& V) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 gx = lanes_f32(G[j], 1.0f), ngx = lanes_f32(G[j], -1.0f);
        const float2 gy = lanes_f32(G[4 + j], 1.0f), ngy = lanes_f32(G[4 + j], -1.0f);
        V.xx[j] = __ffma2_rn(ngx, gx, V.xx[j]);
        V.yy[j] = __ffma2_rn(ngy, gy, V.yy[j]);
        V.xy[j] = __ffma2_rn(ngx, gy, V.xy[j]);
    }
}

// The vertical sums as integers: v + 2^23 (squares, v in [0, 2^23)) and
// v + 1.5 * 2^23 (cross products, |v| < 2^22) lie in [2^23, 2^24), where the
// float's bit pattern is that of 2^23 plus an integer, so the pattern is
// v + 0x4B000000 (0x4B400000) exactly; b[k][c] for product k, column c.
constexpr uint32_t kSqBits = 0x4B000000u, kXyBits = 0x4B400000u;
__device__ __forceinline__ void vsum_bits(const VSums& V, uint32_t (*b)[8]) {
    const float2 sq = make_float2(0x1p23f, 0x1p23f), xy = make_float2(0x1.8p23f, 0x1.8p23f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 a = __fadd2_rn(V.xx[j], sq), c = __fadd2_rn(V.yy[j], sq);
        const float2 e = __fadd2_rn(V.xy[j], xy);
        b[0][2 * j] = __float_as_uint(a.x);
        b[0][2 * j + 1] = __float_as_uint(a.y);
        b[1][2 * j] = __float_as_uint(c.x);
        b[1][2 * j + 1] = __float_as_uint(c.y);
        b[2][2 * j] = __float_as_uint(e.x);
        b[2][2 * j + 1] = __float_as_uint(e.y);
    }
}

// Horizontal 5-sums h[j] of the strip's columns j - 2 .. j + 2 from the bit
// patterns s (own columns), l (columns -2, -1) and r (columns 8, 9), all
// offset by the same m: five patterns carry 5 m (mod 2^32), taken out once;
// the sliding steps add one pattern and drop one, so the offsets cancel.
__device__ __forceinline__ void hsums(const uint32_t* s, const uint32_t* l, const uint32_t* r,
                                      uint32_t m, int* h) {
    uint32_t v = l[0] + l[1] + s[0] + s[1] + s[2] - 5u * m;
    h[0] = (int)v;
#pragma unroll
    for (int j = 1; j < 8; ++j) {
        v += (j + 2 < 8 ? s[j + 2] : r[j - 6]) - (j - 3 >= 0 ? s[j - 3] : l[j - 1]);
        h[j] = (int)v;
    }
}

// q = kd (a b - c^2) - kn (a + b)^2 for 0 <= a, b < 2^25 and 1 <= kn, kd <=
// 1000 (32-bit factors, 64-bit products).
__device__ __forceinline__ long long harris_q32(int a, int b, int c, int kn, int kd) {
    const long long det = (long long)a * b - (long long)c * c;
    const unsigned tr = (unsigned)(a + b);
    return det * kd - (long long)((unsigned long long)tr * tr) * kn;
}

// Hardware approximations (PTX rsqrt.approx / rcp.approx, relative error at
// most 2^-22.9 and 2^-23).
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The mask-only decision of r > T for the binary32 Shi-Tomasi response
// r = tomasi_response_f32(a, b, c) of two pixels at once (packed binary32).
// With A, B, C, E the window sums a, b, c and a - b converted (rounded),
//   h = D rcp(den) - T / 2,  D = A B - C^2,  den = S + disc rsqrt(disc),
//   S = A + B,  disc = (2C)^2 + (E^2 + 2^-100)
// (every step rounded once; rsqrt / rcp are the hardware approximations with
// relative errors of at most 2^-22.9 and 2^-23), lo = h - K S and hi = h + K S
// with K = 2^-20 bracket r / 2 - T / 2: lo > 0 implies r > T, hi < 0 implies
// r < T, otherwise the exact response decides.  With u = 2^-24: D is within
// 2u (a + b)^2 of det = a b - c^2 (c^2 <= a b <= (a + b)^2 / 4), disc and den
// (sums of non-negative terms) within a few u relatively, so D rcp(den) is
// within 3.8u (a + b) of det / (a + b + sqrt(disc)) = lambda / 2, and r within
// 5u lambda <= 2.5u (a + b) of lambda: K S = 16u (a + b) exceeds the sum 2.4
// times.  The 2^-100 keeps disc and den positive when the window is all zero
// (then D = 0 and h = -T / 2 exactly).  tests/test_tomasi_decision.py replays
// the procedure with the extreme approximation errors.
struct TomasiDecide2 {
    float2 nth, nk, k;
};

__device__ __forceinline__ TomasiDecide2 tomasi_decide_consts(float T) {
    TomasiDecide2 k;
    k.nth = make_float2(-0.5f * T, -0.5f * T);
    k.nk = make_float2(-0x1p-20f, -0x1p-20f);
    k.k = make_float2(0x1p-20f, 0x1p-20f);
    return k;
}

__device__ __forceinline__ void tomasi_bracket2(int a0, int a1, int b0, int b1, int c0, int c1,
                                                const TomasiDecide2& k, float2* lo, float2* hi) {
    const float2 A = make_float2((float)a0, (float)a1), B = make_float2((float)b0, (float)b1);
    const float2 C = make_float2((float)c0, (float)c1);
    const float2 E = make_float2((float)(a0 - b0), (float)(a1 - b1));
    const float2 D = __ffma2_rn(__fmul2_rn(C, C), make_float2(-1.0f, -1.0f), __fmul2_rn(A, B));
    const float2 S = __fadd2_rn(A, B);
    const float2 C2 = __fadd2_rn(C, C);
    const float2 disc =
        __ffma2_rn(C2, C2, __ffma2_rn(E, E, make_float2(0x1p-100f, 0x1p-100f)));
    const float2 den = __ffma2_rn(disc, make_float2(rsqrt_approx(disc.x), rsqrt_approx(disc.y)), S);
    const float2 h = __ffma2_rn(D, make_float2(rcp_approx(den.x), rcp_approx(den.y)), k.nth);
    *lo = __ffma2_rn(S, k.nk, h);
    *hi = __ffma2_rn(S, k.k, h);
}

// The mask-only decision of q > q_thr for two pixels at once (packed
// binary32).  With A, B, C the window sums converted (rounded), the values
//   lo = kd (A B - C^2) + (S^2 n1 + n2),  hi = kd (A B - C^2) + (S^2 m1 + m2),
// S = A + B, n1 = -(kn + Kb), n2 = -(q_thr + Qb), m1 = -(kn - Kb), m2 =
// -(q_thr - Qb), Kb = 2^-19 (kd + 2 kn), Qb = 2^-21 |q_thr| (every step
// rounded once), bracket q - q_thr: lo > 0 implies q > q_thr, hi < 0 implies
// q < q_thr, and otherwise the exact test decides.  With u = 2^-24 the
// computed kd (A B - C^2) - kn S^2 - q_thr is within u ((2 kd + 7 kn) (a + b)^2
// + 3 |q_thr|) of q - q_thr (up to O(u^2)), using c^2 <= a b <= (a + b)^2 / 4
// (Cauchy-Schwarz on window sums of gx^2, gy^2, gx gy), and Kb S^2 + Qb
// exceeds that with a margin above 2.5 (tests/test_harris_decision.py replays
// the procedure).  lo <= hi always (rounding is monotonic), so at most one
// decides.
struct HarrisDecide2 {
    float2 kd, n1, n2, m1, m2;
};

__device__ __forceinline__ HarrisDecide2 harris_decide_consts(int kn, int kd, long long q_thr) {
    const float kb = (float)(kd + 2 * kn) * 0x1p-19f;
    const float qt = (float)q_thr, qb = fabsf(qt) * 0x1p-21f;
    HarrisDecide2 k;
    k.kd = make_float2((float)kd, (float)kd);
    const float n1 = -((float)kn + kb), n2 = -(qt + qb);
    const float m1 = -((float)kn - kb), m2 = -(qt - qb);
    k.n1 = make_float2(n1, n1);
    k.n2 = make_float2(n2, n2);
    k.m1 = make_float2(m1, m1);
    k.m2 = make_float2(m2, m2);
    return k;
}

__device__ __forceinline__ void harris_bracket2(float2 A, float2 B, float2 C, const HarrisDecide2& k,
                                                float2* lo, float2* hi) {
    const float2 P = __fmul2_rn(A, B);
    const float2 CC = __fmul2_rn(C, C);
    const float2 D = __ffma2_rn(CC, make_float2(-1.0f, -1.0f), P);
    const float2 S = __fadd2_rn(A, B);
    const float2 S2 = __fmul2_rn(S, S);
    *lo = __ffma2_rn(k.kd, D, __ffma2_rn(S2, k.n1, k.n2));
    *hi = __ffma2_rn(k.kd, D, __ffma2_rn(S2, k.m1, k.m2));
}

// Bytes 0 and 1: the sign bits of a and b replicated over a byte (prmt with
// the sign flag of selector nibbles 0xB and 0xF; __byte_perm ignores that flag).
__device__ __forceinline__ uint32_t sign_bytes2(float a, float b) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, 0xFB;" : "=r"(r) : "r"(__float_as_uint(a)), "r"(__float_as_uint(b)));
    return r;
}

// max(a, b, c): one three-input max.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// One 112 x 8R output tile at (x0, y0) of the image that `tmap` / `p` describe.
// RESP: the launch may export the response (p.resp); without it the row loop
// holds only the mask path, which keeps the loop body small.
template <bool TOMASI, bool RESP>
__device__ __forceinline__ void harris_fast_tile(const CUtensorMap* tmap, const HarrisParams& p,
                                                 FastSmem& sm, int x0, int y0) {
    const int R = p.rows;
    const int W = p.W, H = p.H;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&sm.bar, (uint32_t)(FLW * (8 * R + 6)));
        tma_load_2d(&sm.in[0][0], tmap, &sm.bar, x0 - 16, y0 - 3);
    }
    // every thread leaves together when the (bounded) wait ran out
    if (__syncthreads_or(!mbar_wait_bounded(&sm.bar, 0, p.err))) return;

    const int q = threadIdx.x & 15, g = threadIdx.x >> 4;
    const int xs = x0 - 8 + 8 * q, yb = y0 + R * g;
    const bool producer = q >= 1 && q <= 14 && xs < W;
    const int c = 8 + 8 * q;
    const uint8_t* row = &sm.in[R * g][0];  // input row yb - 3
    uint4* ring = sm.ring[threadIdx.x];
    const bool full = xs >= p.valid[0] && xs + 8 <= p.valid[2] && yb >= p.valid[1] &&
                      yb + R <= p.valid[3];
    const int kn = (int)p.kn, kd = (int)p.kd;
    const HarrisDecide2 dk = harris_decide_consts(kn, kd, p.q_thr);
    const TomasiDecide2 tk = tomasi_decide_consts(p.thr_f);
    VSums V;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        V.xx[j] = make_float2(0.0f, 0.0f);
        V.yy[j] = make_float2(0.0f, 0.0f);
        V.xy[j] = make_float2(0.0f, 0.0f);
    }
    // prologue: gradient rows yb - 2 .. yb + 1 (input rows yb - 3 .. yb + 2)
    uint32_t A[6], B[6], C[6], G[8];
    load_pairs6(row, c, A);
    load_pairs6(row + FLW, c, B);
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
        load_pairs6(row + (r + 2) * FLW, c, C);
        grad_row(A, B, C, G);
        ring[2 * r + 0] = make_uint4(G[0], G[1], G[2], G[3]);
        ring[2 * r + 1] = make_uint4(G[4], G[5], G[6], G[7]);
        add_products(G, V);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            A[k] = B[k];
            B[k] = C[k];
        }
    }
    uint8_t* mrow = p.mask ? p.mask + (size_t)yb * p.mask_pitch : nullptr;
    float* rrow = RESP && p.resp ? reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(p.resp) +
                                                    (size_t)yb * p.resp_pitch)
                         : nullptr;
    const uint32_t fx = ((uint32_t)(p.tv ^ p.fv) & 0xFFu) * 0x01010101u;
    const uint32_t tvx = ((uint32_t)p.tv & 0xFFu) * 0x01010101u;
    // one output row y = yb + i; Pa, Pb: input rows y + 1, y + 2, Pn receives y + 3
    auto step = [&](const uint32_t* Pa, const uint32_t* Pb, uint32_t* Pn, int i) {
        const int y = yb + i;
        // new gradient row y + 2 (input rows y + 1 .. y + 3) into ring slot (i + 4) mod 5
        load_pairs6(row + (i + 6) * FLW, c, Pn);
        grad_row(Pa, Pb, Pn, G);
        const int sn = (i + 4) % RING, so = i % RING;
        ring[2 * sn + 0] = make_uint4(G[0], G[1], G[2], G[3]);
        ring[2 * sn + 1] = make_uint4(G[4], G[5], G[6], G[7]);
        add_products(G, V);
        // vertical sums as integer bit patterns; those of the halo columns
        // from the neighbouring strips
        uint32_t Sb[3][8], L[3][2], Rr[3][2];
        vsum_bits(V, Sb);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            L[k][0] = __shfl_up_sync(0xffffffffu, Sb[k][6], 1);
            L[k][1] = __shfl_up_sync(0xffffffffu, Sb[k][7], 1);
            Rr[k][0] = __shfl_down_sync(0xffffffffu, Sb[k][0], 1);
            Rr[k][1] = __shfl_down_sync(0xffffffffu, Sb[k][1], 1);
        }
        // every lane forms the sums and (mask alone) the decisions, so the
        // common path has no divergent branch; only producers of rows inside
        // the image store
        const bool out = producer && y < H;
        int ha[8], hb[8], hc[8];
        hsums(Sb[0], L[0], Rr[0], kSqBits, ha);
        hsums(Sb[1], L[1], Rr[1], kSqBits, hb);
        hsums(Sb[2], L[2], Rr[2], kXyBits, hc);
        {
            if (!RESP || !rrow) {
                // the mask alone (the benchmark's form): the bracket of every
                // pixel pair first, the exact test only in the rare row where
                // a pixel is left undecided
                float2 lo[4], hi[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (TOMASI)
                        tomasi_bracket2(ha[2 * j], ha[2 * j + 1], hb[2 * j], hb[2 * j + 1],
                                        hc[2 * j], hc[2 * j + 1], tk, &lo[j], &hi[j]);
                    else
                        harris_bracket2(make_float2((float)ha[2 * j], (float)ha[2 * j + 1]),
                                        make_float2((float)hb[2 * j], (float)hb[2 * j + 1]),
                                        make_float2((float)hc[2 * j], (float)hc[2 * j + 1]), dk,
                                        &lo[j], &hi[j]);
                }
                // undecided: lo <= 0 <= hi, i.e. min(-lo, hi) >= 0
                float un[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    un[2 * j] = fminf(-lo[j].x, hi[j].x);
                    un[2 * j + 1] = fminf(-lo[j].y, hi[j].y);
                }
                const float worst = fmaxf(fmax3(un[0], un[1], un[2]),
                                          fmax3(fmax3(un[3], un[4], un[5]), un[6], un[7]));
                // mask bytes from the sign bits of lo: 0xFF (false) where lo
                // is negative, then the true / false values
                uint32_t w0 = (__byte_perm(sign_bytes2(lo[0].x, lo[0].y),
                                           sign_bytes2(lo[1].x, lo[1].y), 0x5410) & fx) ^ tvx;
                uint32_t w1 = (__byte_perm(sign_bytes2(lo[2].x, lo[2].y),
                                           sign_bytes2(lo[3].x, lo[3].y), 0x5410) & fx) ^ tvx;
                if (worst >= 0.0f) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (un[j] >= 0.0f) {
                            const bool t =
                                TOMASI ? tomasi_response_f32(ha[j], hb[j], hc[j]) > p.thr_f
                                       : harris_q32(ha[j], hb[j], hc[j], kn, kd) > p.q_thr;
                            const uint32_t v = (uint32_t)(t ? p.tv : p.fv) & 0xFFu;
                            const int sh = 8 * (j & 3);
                            if (j < 4)
                                w0 = (w0 & ~(0xFFu << sh)) | (v << sh);
                            else
                                w1 = (w1 & ~(0xFFu << sh)) | (v << sh);
                        }
                }
                if (out && mrow) {
                    if (!full) {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (!in_rect(p.valid, xs + j, y)) {
                                if (j < 4)
                                    w0 &= ~(0xFFu << (8 * j));
                                else
                                    w1 &= ~(0xFFu << (8 * (j - 4)));
                            }
                    }
                    if (xs + 8 <= W) {
                        *reinterpret_cast<uint2*>(mrow + xs) = make_uint2(w0, w1);
                    } else {
                        for (int j = 0; j < 8 && xs + j < W; ++j)
                            mrow[xs + j] = (uint8_t)((j < 4 ? w0 : w1) >> (8 * (j & 3)));
                    }
                }
            } else if (out) {
                uint32_t mk[8];
                float rv[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const bool ok = full || in_rect(p.valid, xs + j, y);
                    bool hit;
                    if (TOMASI) {  // binary32 response, as the point operator computes it
                        const float t = tomasi_response_f32(ha[j], hb[j], hc[j]);
                        hit = t > p.thr_f;
                        rv[j] = ok ? t : 0.0f;
                    } else {  // the response is exported: exact q for both
                        const long long qv = harris_q32(ha[j], hb[j], hc[j], kn, kd);
                        hit = qv > p.q_thr;
                        rv[j] = ok ? ratio_to_float(qv, p.kd) : 0.0f;
                    }
                    mk[j] = ok ? (hit ? (uint32_t)p.tv : (uint32_t)p.fv) & 0xFFu : 0u;
                }
                if (mrow) {
                    if (xs + 8 <= W) {
                        *reinterpret_cast<uint2*>(mrow + xs) =
                            make_uint2(mk[0] | (mk[1] << 8) | (mk[2] << 16) | (mk[3] << 24),
                                       mk[4] | (mk[5] << 8) | (mk[6] << 16) | (mk[7] << 24));
                    } else {
                        for (int j = 0; j < 8 && xs + j < W; ++j) mrow[xs + j] = (uint8_t)mk[j];
                    }
                }
                if (rrow) {
                    if (xs + 8 <= W) {
                        float4* d4 = reinterpret_cast<float4*>(rrow + xs);
                        d4[0] = make_float4(rv[0], rv[1], rv[2], rv[3]);
                        d4[1] = make_float4(rv[4], rv[5], rv[6], rv[7]);
                    } else {
                        for (int j = 0; j < 8 && xs + j < W; ++j) rrow[xs + j] = rv[j];
                    }
                }
            }
        }
        if (mrow) mrow += p.mask_pitch;
        if (rrow) rrow = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(rrow) + p.resp_pitch);
        // gradient row y - 2 leaves the window
        const uint4 o0 = ring[2 * so + 0], o1 = ring[2 * so + 1];
        const uint32_t O[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
        sub_products(O, V);
    };
    // three rows per trip: the input windows rotate by renaming
#pragma unroll 1
    for (int i = 0; i < R; i += 3) {
        step(A, B, C, i);
        if (i + 1 >= R) break;
        step(B, C, A, i + 1);
        if (i + 2 >= R) break;
        step(C, A, B, i + 2);
    }
}

template <bool TOMASI, bool RESP>
__global__ void __launch_bounds__(FTHREADS, 4)
    harris_fast_kernel(const __grid_constant__ CUtensorMap tmap, const HarrisParams p) {
    pdl_launch_dependents();  // launched by launch_pdl
    pdl_wait();
    extern __shared__ __align__(128) uint8_t smem_raw[];
    FastSmem& sm = *reinterpret_cast<FastSmem*>(smem_raw);
    harris_fast_tile<TOMASI, RESP>(&tmap, p, sm, blockIdx.x * FTW, blockIdx.y * 8 * p.rows);
}

// Several images in one launch (hvxProcessGraphBatch): block t is tile
// t - tile_start[i] of the last image i with tile_start[i] <= t; tensor maps
// and parameters in global memory, all images with the same rows per thread
// and the same response (Harris or Shi-Tomasi: TOMASI); RESP: some image
// exports its response.
template <bool TOMASI, bool RESP>
__global__ void __launch_bounds__(FTHREADS, 4)
    harris_fast_batch_kernel(const CUtensorMap* __restrict__ maps,
                             const HarrisParams* __restrict__ ps, const int* __restrict__ tile_start,
                             const int* __restrict__ tiles_x, int n) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    FastSmem& sm = *reinterpret_cast<FastSmem*>(smem_raw);
    const int t = blockIdx.x;
    const int i = find_image(tile_start, n, t);
    const int local = t - __ldg(tile_start + i), tx = __ldg(tiles_x + i);
    const int ty = local / tx;
    if (threadIdx.x == 0) tensormap_acquire(maps + i);
    // the image's parameters into shared memory: the row loop reads them
    // there instead of from global memory
    constexpr int PW = (int)(sizeof(HarrisParams) / 4);
    if (threadIdx.x < PW)
        reinterpret_cast<uint32_t*>(&sm.prm)[threadIdx.x] =
            __ldg(reinterpret_cast<const uint32_t*>(ps + i) + threadIdx.x);
    __syncthreads();
    harris_fast_tile<TOMASI, RESP>(maps + i, sm.prm, sm, (local - ty * tx) * FTW,
                                   ty * 8 * sm.prm.rows);
}

}  // namespace

bool harris_fast_path(const HarrisParams& p) {
    return p.border_s == HVX_BORDER_UNDEFINED && p.border_b == HVX_BORDER_UNDEFINED && p.wr == 2 &&
           p.rows >= FROWS_MIN && p.rows <= FROWS_MAX;
}

// Rows per thread of the BORDER_UNDEFINED kernel for a W x H image on
// `num_sms` SMs: the R that minimises (waves of 4 CTAs per SM) x (rows each
// CTA walks, R plus the 4-row prologue).  Measured on 4096 x 2160: R = 17 (592
// CTAs, one full wave) 41 us; R = 20 (518) and 23 (444 CTAs, SMs left with
// fewer than 4) 49 us; R = 15 (666 CTAs, two waves) 54 us.
int harris_fast_rows(int W, int H, int num_sms) {
    const long tiles_x = (W + FTW - 1) / FTW;
    const long slots = 4L * (num_sms > 0 ? num_sms : 1);
    int best = FROWS_MAX;
    long best_cost = -1;
    for (int r = FROWS_MIN; r <= FROWS_MAX; ++r) {
        const long tiles = tiles_x * ((H + 8 * r - 1) / (8 * r));
        const long cost = (tiles + slots - 1) / slots * (r + 4);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = r;
        }
    }
    return best;
}

void harris_box(const HarrisParams& p, int* w, int* h) {
    *w = harris_fast_path(p) ? FLW : HARRIS_LOAD_W;
    *h = harris_fast_path(p) ? 8 * p.rows + 6 : HARRIS_TH + 6;
}

int harris_fast_tile_w() { return FTW; }

// Rows per thread for a batch of images in one launch: the same wave model
// as harris_fast_rows over the tiles of all images.
int harris_batch_rows(const int* W, const int* H, int n, int num_sms) {
    const long slots = 4L * (num_sms > 0 ? num_sms : 1);
    int best = FROWS_MAX;
    long best_cost = -1;
    for (int r = FROWS_MIN; r <= FROWS_MAX; ++r) {
        long tiles = 0;
        for (int i = 0; i < n; ++i)
            tiles += (long)((W[i] + FTW - 1) / FTW) * ((H[i] + 8 * r - 1) / (8 * r));
        const long cost = (tiles + slots - 1) / slots * (r + 4);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = r;
        }
    }
    return best;
}

namespace {
template <class K>
cudaError_t set_fast_smem(K kernel, std::atomic<bool>& done) {
    if (done.load(std::memory_order_acquire)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(FastSmem));
    if (e == cudaSuccess) done.store(true, std::memory_order_release);
    return e;
}
}  // namespace

template <bool TOMASI, bool RESP>
cudaError_t launch_harris_batch_t(const CUtensorMap* maps, const HarrisParams* ps,
                                  const int* tile_start, const int* tiles_x, int n, int total,
                                  cudaStream_t s) {
    static std::atomic<bool> attr{false};
    cudaError_t e = set_fast_smem(harris_fast_batch_kernel<TOMASI, RESP>, attr);
    if (e != cudaSuccess) return e;
    harris_fast_batch_kernel<TOMASI, RESP><<<total, FTHREADS, (int)sizeof(FastSmem), s>>>(
        maps, ps, tile_start, tiles_x, n);
    return cudaGetLastError();
}

template <bool TOMASI, bool RESP>
cudaError_t launch_harris_fast_t(const CUtensorMap& map, const HarrisParams& p, cudaStream_t s) {
    static std::atomic<bool> attr{false};
    cudaError_t e = set_fast_smem(harris_fast_kernel<TOMASI, RESP>, attr);
    if (e != cudaSuccess) return e;
    dim3 grid((p.W + FTW - 1) / FTW, (p.H + 8 * p.rows - 1) / (8 * p.rows));
    return launch_pdl(harris_fast_kernel<TOMASI, RESP>, grid, dim3(FTHREADS), sizeof(FastSmem), s,
                      map, p);
}

cudaError_t launch_harris_batch(const CUtensorMap* maps, const HarrisParams* ps,
                                const int* tile_start, const int* tiles_x, int n, int total,
                                bool tomasi, bool resp, cudaStream_t s) {
    if (tomasi)
        return resp ? launch_harris_batch_t<true, true>(maps, ps, tile_start, tiles_x, n, total, s)
                    : launch_harris_batch_t<true, false>(maps, ps, tile_start, tiles_x, n, total, s);
    return resp ? launch_harris_batch_t<false, true>(maps, ps, tile_start, tiles_x, n, total, s)
                : launch_harris_batch_t<false, false>(maps, ps, tile_start, tiles_x, n, total, s);
}

cudaError_t launch_harris(const CUtensorMap& map, const HarrisParams& p, cudaStream_t s) {
    if (harris_fast_path(p)) {
        if (p.tomasi)
            return p.resp ? launch_harris_fast_t<true, true>(map, p, s)
                          : launch_harris_fast_t<true, false>(map, p, s);
        return p.resp ? launch_harris_fast_t<false, true>(map, p, s)
                      : launch_harris_fast_t<false, false>(map, p, s);
    }
    static bool attr_set = false;
    const int smem = (int)sizeof(HarrisSmem);
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(harris_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((p.W + TW - 1) / TW, (p.H + TH - 1) / TH);
    return launch_pdl(harris_kernel, grid, dim3(HARRIS_THREADS), smem, s, map, p);
}

}  // namespace hvx
