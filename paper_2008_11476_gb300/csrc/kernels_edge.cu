// Fused edge-detection group (Table 2 local and point operators; the edge
// graph of Listing 1 / the Section 6 benchmarks):
//
//   in U8 --Gaussian3x3--> G (on chip) --Sobel3x3--> gx, gy (registers)
//        --Magnitude--> m --Threshold--> mask (U8)      --Phase--> phase (U8)
//
// One CTA (256 threads) computes a 128 x 30 output tile:
//   1. one TMA 2-D load brings the 160 x 34 input box (tile + 2-pixel halo,
//      widened to 16-byte-aligned columns) into shared memory; the hardware
//      fills out-of-image bytes with 0, and edge tiles then apply the
//      Gaussian's border mode to them;
//   2. G over the tile + 1-pixel halo (130 x 32) is computed in SWAR form: each
//      32-bit word holds two adjacent pixels as 16-bit lanes, so every add,
//      shift and funnel shift works on two pixels; G stays in shared memory as
//      16-bit pixels.  Edge tiles then apply the Sobel's border mode to the G
//      cells outside the image (REPLICATE reads the replicated *Gaussian*
//      output, as the node-by-node definition requires);
//   3. each item is 8 pixels of one row: gx and gy are formed in the same
//      16-bit-lane form (biased so that no lane goes negative), unpacked to
//      binary32 by exponent splicing, and the point operators run in binary32
//      (every value involved is an integer below 2^24, so the float arithmetic
//      is exact); the U8 results are written with 8-byte stores.
// Magnitude followed by a binary threshold T is evaluated as
// gx^2 + gy^2 > T^2 + T, which equals round(sqrt(gx^2 + gy^2)) > T exactly.
//
// The batch kernel runs the same tile code persistently over the tiles of
// many images (one tensor map per image, in global memory), and issues the
// TMA load of its next tile as soon as the current input box has been read.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int TW = EDGE_TW;          // 128
constexpr int TH = EDGE_TH;          // 30
constexpr int LW = EDGE_LOAD_W;      // 160
constexpr int IN_ROWS = TH + 4;      // 34
constexpr int G_ROWS = TH + 2;       // 32
constexpr int GW = TW + 16;          // G columns x0 - 8 .. x0 + 135
constexpr uint32_t IN_BYTES = IN_ROWS * LW;

// Kernel modes (template parameter).
constexpr int M_GAUSS = EDGE_MODE_GAUSS;  // Gaussian3x3 alone (kernels_gauss.cu)
constexpr int M_MASK_PHASE = 1; // binary threshold mask + phase
constexpr int M_MASK = 2;       // binary threshold mask only
constexpr int M_PHASE = 3;      // phase only
constexpr int M_GENERAL = 4;    // any outputs (magnitude export, range threshold)

constexpr int STAGES = EDGE_STAGES;     // input boxes in flight per CTA (batch kernel)

using InTile = uint8_t[IN_ROWS][LW];    // image (x0 - 16 + c, y0 - 2 + r)
using GTile = uint16_t[G_ROWS][GW];     // Gaussian (x0 - 8 + k, y0 - 1 + r)

struct alignas(128) InStage {
    InTile b;
};

template <int NS>
struct EdgeSmem {
    InStage in[NS];                     // ring of TMA destinations
    alignas(16) GTile g;
    alignas(8) uint64_t bar[NS];
    // batch: parameters and origin of the tiles in flight, in a ring one longer
    // than the input ring (tile k uses slot k mod (NS + 1), so the slot that
    // tile k + NS fills belongs to tile k - 1, which is finished)
    EdgeParams prm[NS + 1];
    int tx0[NS + 1], ty0[NS + 1];
    float tanb[36];                     // Phase boundary tangents (kPhaseTan)
};

// Lane values of a 16-bit-lane word as binary32, minus a bias, exactly.
__device__ __forceinline__ float lane_lo_f(uint32_t w, float bias) {
    return __int_as_float(__byte_perm(w, 0x4B00u, 0x5410)) - (8388608.0f + bias);
}
__device__ __forceinline__ float lane_hi_f(uint32_t w, float bias) {
    return __int_as_float(__byte_perm(w, 0x4B00u, 0x5432)) - (8388608.0f + bias);
}

__device__ __forceinline__ uint32_t pack4(uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
    return __byte_perm(__byte_perm(b0, b1, 0x0040), __byte_perm(b2, b3, 0x0040), 0x5410);
}

__device__ __forceinline__ bool tile_is_interior(const EdgeParams& p, int x0, int y0) {
    return x0 >= 2 && y0 >= 2 && x0 + TW + 2 <= (int)p.W && y0 + TH + 2 <= (int)p.H;
}

__device__ __forceinline__ bool rect_is_full(const int32_t* r, const EdgeParams& p) {
    return r[0] == 0 && r[1] == 0 && r[2] == (int)p.W && r[3] == (int)p.H;
}

// Hardware reciprocal approximation (rcp.approx.ftz.f32, at most 1 ulp off).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Phase from exact integer gradients held in binary32 (gen_phase_poly.py
// derives and checks every step over all integer gradient pairs): with
// mn, mx = min, max of |gx|, |gy| and t = mn / mx, the rounded octant angle
// is n or n - 1 for n = floor(1 + t (A + B t)), and it is n exactly when
// mn - mx tan((n - 1/2) pi / 128) > 0.  tanb holds those tangents (n = 0..33)
// in shared memory.  The octant angle then maps to the full turn by the
// signs of gx, gy and the swap of |gx|, |gy|; the low byte is the phase.
__device__ __forceinline__ uint32_t phase_from_float(float gx, float gy, const float* tanb) {
    const float ax = fabsf(gx), ay = fabsf(gy);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mn * rcp_approx(fmaxf(mx, 1.0f));  // integers: mx = 0 only when mn = 0
    const int n = __float2int_rd(fmaf(t, fmaf(t, kPhaseGuessB, kPhaseGuessA), 1.0f));  // 1..33
    const int ra = fmaf(-mx, tanb[n], mn) > 0.0f ? n : n - 1;
    const int q1 = ay > ax ? 64 - ra : ra;
    const bool sx = gx < 0.0f, sy = gy < 0.0f;
    return (uint32_t)((sx ? 128 : 0) + ((sx != sy) ? -q1 : q1));
}

__device__ __forceinline__ void store8_u8(uint8_t* row, int x, int W, const uint32_t* b) {
    if (x + 8 <= W) {
        *reinterpret_cast<uint2*>(row + x) =
            make_uint2(pack4(b[0], b[1], b[2], b[3]), pack4(b[4], b[5], b[6], b[7]));
    } else {
        for (int j = 0; j < 8 && x + j < W; ++j) row[x + j] = (uint8_t)b[j];
    }
}

// ---- stage 1: input border -------------------------------------------------------

__device__ void fix_input_border(InTile& in, const EdgeParams& p, int x0, int y0) {
    const int W = p.W, H = p.H;
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    const bool cst = p.border_g == HVX_BORDER_CONSTANT;
    const uint8_t cv = (uint8_t)p.cval_g;
    for_each_outside(IN_ROWS, LW, x0 - 16, y0 - 2, W, H, [&](int r, int c) {
        int x = x0 - 16 + c, y = y0 - 2 + r;
        in[r][c] = cst ? cv : in[clampi(y, 0, H - 1) - (y0 - 2)][clampi(x, 0, W - 1) - (x0 - 16)];
    });
}

// ---- stage 2: Gaussian in 16-bit lanes ---------------------------------------------
// Item (r, q): G row r (y = y0 - 1 + r), pixels x = x0 + 8q .. x0 + 8q + 7;
// group 0 also produces x0 - 1 and group 15 also x0 + 128.
__device__ void gaussian_stage(const InTile& in, GTile& g, const EdgeParams& p) {
    const uint32_t rnd = p.rounding == HVX_ROUND_TO_NEAREST ? 0x00080008u : 0u;
    for (int it = threadIdx.x; it < G_ROWS * 16; it += blockDim.x) {
        const int r = it >> 4, q = it & 15;
        const int c = 16 + 8 * q;
        uint32_t V[6];  // vertical sums of pixel pairs (x-2,x-1), (x,x+1) .. (x+8,x+9)
#pragma unroll
        for (int dr = 0; dr < 3; ++dr) {
            const uint8_t* row = in[r + dr];
            uint2 m = *reinterpret_cast<const uint2*>(row + c);
            uint32_t wl = *reinterpret_cast<const uint32_t*>(row + c - 4);
            uint32_t wr = *reinterpret_cast<const uint32_t*>(row + c + 8);
            uint32_t P[6] = {hi_pair(wl), lo_pair(m.x), hi_pair(m.x),
                             lo_pair(m.y), hi_pair(m.y), lo_pair(wr)};
#pragma unroll
            for (int k = 0; k < 6; ++k) V[k] = dr == 0 ? P[k] : V[k] + (dr == 1 ? 2u : 1u) * P[k];
        }
        uint32_t Gp[4];
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            uint32_t s = shift_pair(V[j - 1], V[j]) + shift_pair(V[j], V[j + 1]) + 2u * V[j] + rnd;
            Gp[j - 1] = (s >> 4) & 0x00FF00FFu;
        }
        *reinterpret_cast<uint4*>(&g[r][8 + 8 * q]) = make_uint4(Gp[0], Gp[1], Gp[2], Gp[3]);
    }
    // The two halo columns x0 - 1 and x0 + 128, one scalar item per row and
    // side on the first 64 threads (kept out of the loop above, where they
    // would make every warp diverge).  Each is written as a word together
    // with the column beyond it set to 0: stage 3 reads those outer lanes
    // (cols 6, 137) as part of its pair loads, and a zero lane cannot carry
    // into its neighbour in the 16-bit-lane arithmetic.
    if (threadIdx.x < 2 * G_ROWS) {
        const int r = threadIdx.x >> 1, side = threadIdx.x & 1;
        const int c = side ? 16 + TW : 15;  // input column of the halo pixel
        uint32_t s = rnd & 0xFFFFu;
#pragma unroll
        for (int dr = 0; dr < 3; ++dr) {
            const uint32_t w = dr == 1 ? 2u : 1u;
            s += w * (in[r + dr][c - 1] + 2u * in[r + dr][c] + in[r + dr][c + 1]);
        }
        if (side)
            *reinterpret_cast<uint32_t*>(&g[r][136]) = s >> 4;
        else
            *reinterpret_cast<uint32_t*>(&g[r][6]) = (s >> 4) << 16;
    }
}

// G cells: zero inside the image but outside the Gaussian's valid region; the
// Sobel's border mode outside the image.  Edge tiles only.
__device__ void fix_g_border(GTile& g, const EdgeParams& p, int x0, int y0) {
    const int W = p.W, H = p.H;
    constexpr int COLS = TW + 2;  // k = 7 .. 136, x = x0 - 1 .. x0 + 128
    if (!rect_is_full(p.gvalid, p)) {
        for (int i = threadIdx.x; i < G_ROWS * COLS; i += blockDim.x) {
            int r = i / COLS, k = 7 + (i - r * COLS);
            int x = x0 - 8 + k, y = y0 - 1 + r;
            if (x >= 0 && x < W && y >= 0 && y < H && !in_rect(p.gvalid, x, y)) g[r][k] = 0;
        }
        __syncthreads();
    }
    if (p.border_s == HVX_BORDER_UNDEFINED) return;
    const bool cst = p.border_s == HVX_BORDER_CONSTANT;
    const uint16_t cv = (uint16_t)(p.cval_s & 0xFF);
    for_each_outside(G_ROWS, COLS, x0 - 1, y0 - 1, W, H, [&](int r, int c) {
        int x = x0 - 1 + c, y = y0 - 1 + r;
        g[r][7 + c] =
            cst ? cv : g[clampi(y, 0, H - 1) - (y0 - 1)][clampi(x, 0, W - 1) - (x0 - 8)];
    });
}

// ---- stage 3: Sobel + point operators ------------------------------------------------

__device__ __forceinline__ void load_g_row(const uint16_t* row, int k, uint32_t P[6]) {
    uint4 m = *reinterpret_cast<const uint4*>(row + k);
    P[0] = *reinterpret_cast<const uint32_t*>(row + k - 2);
    P[1] = m.x;
    P[2] = m.y;
    P[3] = m.z;
    P[4] = m.w;
    P[5] = *reinterpret_cast<const uint32_t*>(row + k + 8);
}

// All-ones when a > b, else 0 (one instruction).
__device__ __forceinline__ uint32_t set_gt(float a, float b) {
    uint32_t r;
    asm("set.gt.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void store8_words(uint8_t* row, int x, int W, uint32_t lo, uint32_t hi) {
    if (x + 8 <= W) {
        *reinterpret_cast<uint2*>(row + x) = make_uint2(lo, hi);
    } else {
        for (int j = 0; j < 8 && x + j < W; ++j) row[x + j] = (uint8_t)((j < 4 ? lo : hi) >> (8 * (j & 3)));
    }
}

template <int MODE>
__device__ void sobel_point_stage(const GTile& g, const EdgeParams& p, int x0, int y0,
                                  bool interior, const float* tanb) {
    const float s_thr = (float)p.s_thr;
    const bool full = interior || rect_is_full(p.valid, p);
    const int W = p.W, H = p.H;
    // mask bytes from all-ones / zero compare results: (c & (tv ^ fv)) ^ fv
    const uint32_t tvx = ((uint32_t)(p.tv ^ p.fv) & 0xFFu) * 0x01010101u;
    const uint32_t fvx = ((uint32_t)p.fv & 0xFFu) * 0x01010101u;
    constexpr bool kMask = MODE == M_MASK_PHASE || MODE == M_MASK;
    constexpr bool kPhase = MODE == M_MASK_PHASE || MODE == M_PHASE;
    uint8_t* const mask = p.mask;
    uint8_t* const phase = p.phase;
    const size_t mask_pitch = p.mask_pitch, phase_pitch = p.phase_pitch;
#pragma unroll 1
    for (int it = threadIdx.x; it < TH * 16; it += blockDim.x) {
        const int r = it >> 4, s8 = it & 15;
        const int y = y0 + r, x = x0 + 8 * s8;
        if (y >= H || x >= W) continue;
        const int k = 8 + 8 * s8;
        uint32_t A[6], B[6], C[6];
        load_g_row(g[r], k, A);
        load_g_row(g[r + 1], k, B);
        load_g_row(g[r + 2], k, C);
        uint32_t vs[6], dy[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            vs[j] = A[j] + 2u * B[j] + C[j];          // <= 1020 per lane
            dy[j] = C[j] + 0x00FF00FFu - A[j];        // gy part + 255 per lane
        }
        float gx[8], gy[8];
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            uint32_t gxp = shift_pair(vs[j], vs[j + 1]) + 0x04000400u - shift_pair(vs[j - 1], vs[j]);
            uint32_t gyp = shift_pair(dy[j - 1], dy[j]) + 2u * dy[j] + shift_pair(dy[j], dy[j + 1]);
            gx[2 * j - 2] = lane_lo_f(gxp, 1024.0f);
            gx[2 * j - 1] = lane_hi_f(gxp, 1024.0f);
            gy[2 * j - 2] = lane_lo_f(gyp, 1020.0f);
            gy[2 * j - 1] = lane_hi_f(gyp, 1020.0f);
        }
        uint32_t mk[8], ph[8];
        int mg[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            mk[i] = ph[i] = 0u;
            mg[i] = 0;
            if (kMask) mk[i] = set_gt(fmaf(gx[i], gx[i], gy[i] * gy[i]), s_thr);
            if (kPhase) ph[i] = phase_from_float(gx[i], gy[i], tanb);
            if (MODE == M_GENERAL) {
                int ix = (int)gx[i], iy = (int)gy[i];
                mg[i] = magnitude_s16(ix, iy);
                if (mask) {
                    bool t;
                    if (!p.thr_general)
                        t = ix * ix + iy * iy > p.s_thr;
                    else
                        t = p.thr_type == HVX_THRESHOLD_BINARY
                                ? mg[i] > p.thr_lo
                                : !(mg[i] > p.thr_hi || mg[i] < p.thr_lo);
                    mk[i] = t ? 0xFFFFFFFFu : 0u;
                }
                if (phase) ph[i] = phase_from_float(gx[i], gy[i], tanb);
            }
        }
        const bool want_mask = kMask || (MODE == M_GENERAL && mask);
        const bool want_phase = kPhase || (MODE == M_GENERAL && phase);
        if (full) {
            if (want_mask)
                store8_words(mask + (size_t)y * mask_pitch, x, W,
                             (pack4(mk[0], mk[1], mk[2], mk[3]) & tvx) ^ fvx,
                             (pack4(mk[4], mk[5], mk[6], mk[7]) & tvx) ^ fvx);
            if (want_phase)
                store8_words(phase + (size_t)y * phase_pitch, x, W,
                             pack4(ph[0], ph[1], ph[2], ph[3]), pack4(ph[4], ph[5], ph[6], ph[7]));
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                mk[i] = (mk[i] & tvx) ^ fvx;
                if (!in_rect(p.valid, x + i, y)) {
                    mk[i] = 0u;
                    ph[i] = 0u;
                    mg[i] = 0;
                }
            }
            if (want_mask) store8_u8(mask + (size_t)y * mask_pitch, x, W, mk);
            if (want_phase) store8_u8(phase + (size_t)y * phase_pitch, x, W, ph);
        }
        if (MODE == M_GENERAL && p.mag) {
            int16_t* row = reinterpret_cast<int16_t*>(reinterpret_cast<uint8_t*>(p.mag) +
                                                      (size_t)y * p.mag_pitch);
            if (x + 8 <= W) {
                *reinterpret_cast<uint4*>(row + x) =
                    make_uint4((mg[0] & 0xFFFF) | ((uint32_t)mg[1] << 16),
                               (mg[2] & 0xFFFF) | ((uint32_t)mg[3] << 16),
                               (mg[4] & 0xFFFF) | ((uint32_t)mg[5] << 16),
                               (mg[6] & 0xFFFF) | ((uint32_t)mg[7] << 16));
            } else {
                for (int j = 0; j < 8 && x + j < W; ++j) row[x + j] = (int16_t)mg[j];
            }
        }
    }
}

// One tile after its input box has landed in `in`.  `prefetch` runs on warp
// 0 as soon as `in` is no longer read (after the Gaussian stage), so that the
// box can be refilled while the rest of the tile is computed.
template <int MODE, class Prefetch>
__device__ void edge_tile_body(InTile& in, GTile& g, const EdgeParams& p, int x0, int y0,
                               const float* tanb, Prefetch prefetch) {
    const bool interior = tile_is_interior(p, x0, y0);
    if (!interior) {
        fix_input_border(in, p, x0, y0);
        __syncthreads();
    }
    gaussian_stage(in, g, p);
    __syncthreads();
    if (threadIdx.x < 32) prefetch();
    if (!interior) {
        fix_g_border(g, p, x0, y0);
        __syncthreads();
    }
    sobel_point_stage<MODE>(g, p, x0, y0, interior, tanb);
    __syncthreads();
}

__device__ __forceinline__ void issue_box(InTile& in, uint64_t* bar, const CUtensorMap* map, int x0,
                                          int y0) {
    mbar_arrive_expect_tx(bar, IN_BYTES);
    tma_load_2d(&in[0][0], map, bar, x0 - 16, y0 - 2);
}

template <int MODE>
__global__ void __launch_bounds__(EDGE_THREADS, 4)
    edge_kernel(const __grid_constant__ CUtensorMap tmap, const EdgeParams p) {
    __shared__ EdgeSmem<1> sm;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        fence_barrier_init();
    }
    if (threadIdx.x < 34) sm.tanb[threadIdx.x] = kPhaseTan[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) issue_box(sm.in[0].b, &sm.bar[0], &tmap, x0, y0);
    if (!mbar_wait_bounded(&sm.bar[0], 0, p.err)) return;
    edge_tile_body<MODE>(sm.in[0].b, sm.g, p, x0, y0, sm.tanb, [] {});
}

__device__ __forceinline__ void tile_origin(const EdgeParams& p, int t, int& x0, int& y0) {
    int tiles_x = (p.W + TW - 1) / TW;
    int ty = t / tiles_x;
    x0 = (t - ty * tiles_x) * TW;
    y0 = ty * TH;
}

// Warp 0: stage the parameters and origin of batch tile t in parameter slot
// ps and start the TMA load of its input box into ring stage s.
__device__ __forceinline__ void issue_tile(EdgeSmem<STAGES>& sm, const EdgeBatchDesc& d, int s,
                                           int ps, int t) {
    const int lane = threadIdx.x & 31;
    int img = 0;
    if (lane == 0) img = find_image(d.tile_start, d.n_img, t);
    img = __shfl_sync(0xffffffffu, img, 0);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&d.params[img]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sm.prm[ps]);
    for (int i = lane; i < (int)(sizeof(EdgeParams) / 4); i += 32) dst[i] = __ldg(src + i);
    __syncwarp();
    if (lane == 0) {
        int x0, y0;
        tile_origin(sm.prm[ps], t - __ldg(d.tile_start + img), x0, y0);
        sm.tx0[ps] = x0;
        sm.ty0[ps] = y0;
        tensormap_acquire(&d.maps[img]);
        fence_proxy_async_smem();
        issue_box(sm.in[s].b, &sm.bar[s], &d.maps[img], x0, y0);
    }
}

// Persistent: CTA b takes tiles b, b + grid, b + 2 grid, ...; tile k of the
// CTA lives in ring stage k mod STAGES, so STAGES input boxes are in flight
// while one is computed.  Each tile's parameters come from shared memory.
template <int MODE>
__global__ void __launch_bounds__(EDGE_THREADS, 4) edge_batch_kernel(const EdgeBatchDesc d) {
    __shared__ EdgeSmem<STAGES> sm;
    const int first = blockIdx.x;
    if (first >= d.total_tiles) return;
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < STAGES; ++s) mbar_init(&sm.bar[s], 1);
            fence_barrier_init();
        }
        __syncwarp();
        for (int s = 0; s < STAGES; ++s) {
            const int t = first + s * (int)gridDim.x;
            if (t < d.total_tiles) issue_tile(sm, d, s, s, t);
        }
    } else if (threadIdx.x < 32 + 34) {
        sm.tanb[threadIdx.x - 32] = kPhaseTan[threadIdx.x - 32];
    }
    __syncthreads();
    int k = 0;
    for (int t = first; t < d.total_tiles; t += gridDim.x, ++k) {
        const int s = k % STAGES;
        const int ps = k % (STAGES + 1);
        const uint32_t parity = (uint32_t)(k / STAGES) & 1u;
        const bool ok = mbar_wait_bounded(&sm.bar[s], parity, d.err);
        if (__syncthreads_or(!ok)) return;
        const EdgeParams& p = sm.prm[ps];
        const int x0 = sm.tx0[ps], y0 = sm.ty0[ps];
        const int tn = t + STAGES * (int)gridDim.x;  // the next tile of this stage
        const int pn = (k + STAGES) % (STAGES + 1);
        edge_tile_body<MODE>(sm.in[s].b, sm.g, p, x0, y0, sm.tanb, [&] {
            if (tn < d.total_tiles) issue_tile(sm, d, s, pn, tn);
        });
    }
}

template <int MODE>
cudaError_t launch_mode(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s) {
    dim3 grid((p.W + TW - 1) / TW, (p.H + TH - 1) / TH);
    edge_kernel<MODE><<<grid, EDGE_THREADS, 0, s>>>(map, p);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_batch_mode(const EdgeBatchDesc& d, int grid, cudaStream_t s) {
    edge_batch_kernel<MODE><<<grid, EDGE_THREADS, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace

int edge_mode(const EdgeParams& p) {
    if (p.gout) return M_GAUSS;
    if (p.mag || p.thr_general) return M_GENERAL;
    if (p.mask && p.phase) return M_MASK_PHASE;
    if (p.mask) return M_MASK;
    return M_PHASE;
}

void edge_tile_dims(int mode, int* tw, int* th) {
    *tw = mode == M_GAUSS ? GAUSS_TW : EDGE_TW;
    *th = mode == M_GAUSS ? GAUSS_TH : EDGE_TH;
}

cudaError_t launch_edge(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s) {
    switch (edge_mode(p)) {
        case M_GAUSS: return launch_gauss(map, p, s);
        case M_MASK_PHASE: return launch_mode<M_MASK_PHASE>(map, p, s);
        case M_MASK: return launch_mode<M_MASK>(map, p, s);
        case M_PHASE: return launch_mode<M_PHASE>(map, p, s);
        default: return launch_mode<M_GENERAL>(map, p, s);
    }
}

cudaError_t launch_edge_batch(const EdgeBatchDesc& d, int mode, int grid, cudaStream_t s) {
    switch (mode) {
        case M_GAUSS: return launch_gauss_batch(d, grid, s);
        case M_MASK_PHASE: return launch_batch_mode<M_MASK_PHASE>(d, grid, s);
        case M_MASK: return launch_batch_mode<M_MASK>(d, grid, s);
        case M_PHASE: return launch_batch_mode<M_PHASE>(d, grid, s);
        default: return launch_batch_mode<M_GENERAL>(d, grid, s);
    }
}

int edge_batch_blocks_per_sm(int mode) {
    if (mode == M_GAUSS) return gauss_batch_blocks_per_sm();
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, edge_batch_kernel<M_MASK_PHASE>,
                                                  EDGE_THREADS, 0);
    return n;
}

}  // namespace hvx
