// Fused Harris-corner group (HarrisCorners row of Table 2 as point + local +
// custom abstractions; the corner-detector benchmark of Section 6):
//
//   in U8 --Sobel3x3--> gx, gy (S16) --point--> gx^2, gy^2, gx*gy (S32)
//        --local 5x5 window sums--> Sxx, Syy, Sxy (S32)
//        --point--> R = Sxx Syy - Sxy^2 - k (Sxx + Syy)^2 (F32)
//        --Threshold--> mask (U8)
//
// One CTA computes a 64 x 32 output tile: a TMA box of the input with a
// 3-pixel halo, the three products over the tile + 2-pixel halo into shared
// memory (exact int32), their vertical 5-sums into shared memory, then per
// thread 8 pixels of horizontal 5-sums, the response in exact 64-bit integer
// form q = kd * R and the threshold.  R > T on the binary32 value is decided
// as q > q_thr, where the host computed q_thr so that this equals the
// comparison of the correctly rounded binary32 response with T.  When R is
// exported it is rounded once from q / kd.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int TW = HARRIS_TW;
constexpr int TH = HARRIS_TH;
constexpr int LW = HARRIS_LOAD_W;     // 96
constexpr int IN_ROWS = TH + 6;       // 38
constexpr int PR = TH + 4;            // product rows (y0-2 .. y0+TH+1)
constexpr int PC = TW + 4;            // product cols (x0-2 .. x0+TW+1)
constexpr uint32_t IN_BYTES = IN_ROWS * LW;

struct HarrisSmem {
    alignas(128) uint8_t in[IN_ROWS][LW];  // image (x0 - 16 + c, y0 - 3 + r)
    alignas(16) int32_t p[3][PR][PC];      // products (x0 - 2 + c, y0 - 2 + r)
    alignas(16) int32_t v[3][TH][PC];      // vertical 5-sums (x0 - 2 + c, y0 + r)
    alignas(8) uint64_t bar;
};

__device__ __forceinline__ bool interior_tile(const HarrisParams& p, int x0, int y0) {
    return x0 >= 3 && y0 >= 3 && x0 + TW + 3 <= (int)p.W && y0 + TH + 3 <= (int)p.H;
}

__device__ __forceinline__ bool full_rect(const int32_t* r, const HarrisParams& p) {
    return r[0] == 0 && r[1] == 0 && r[2] == (int)p.W && r[3] == (int)p.H;
}

__global__ void __launch_bounds__(HARRIS_THREADS, 3)
    harris_kernel(const __grid_constant__ CUtensorMap tmap, const HarrisParams p) {
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
    if (!mbar_wait_bounded(&sm.bar, 0, p.err)) return;
    const bool interior = interior_tile(p, x0, y0);

    // 1. the Sobel's border mode on input bytes outside the image
    if (!interior && p.border_s != HVX_BORDER_UNDEFINED) {
        for (int i = threadIdx.x; i < IN_ROWS * LW; i += blockDim.x) {
            int r = i / LW, c = i - r * LW;
            int x = x0 - 16 + c, y = y0 - 3 + r;
            if (x >= 0 && x < W && y >= 0 && y < H) continue;
            uint8_t val;
            if (p.border_s == HVX_BORDER_CONSTANT)
                val = (uint8_t)p.cval_s;
            else
                val = sm.in[clampi(y, 0, H - 1) - (y0 - 3)][clampi(x, 0, W - 1) - (x0 - 16)];
            sm.in[r][c] = val;
        }
        __syncthreads();
    }

    // 2. gx, gy and their products over the tile + 2-pixel halo
    const bool pfull = interior || full_rect(p.pvalid, p);
    for (int i = threadIdx.x; i < PR * PC; i += blockDim.x) {
        int r = i / PC, c = i - r * PC;
        // input rows r .. r+2, columns c+13 .. c+15 hold the 3x3 window
        const uint8_t* a = &sm.in[r][c + 13];
        const uint8_t* b = &sm.in[r + 1][c + 13];
        const uint8_t* d = &sm.in[r + 2][c + 13];
        int gx = (a[2] - a[0]) + 2 * (b[2] - b[0]) + (d[2] - d[0]);
        int gy = (d[0] + 2 * d[1] + d[2]) - (a[0] + 2 * a[1] + a[2]);
        if (!pfull) {
            int x = x0 - 2 + c, y = y0 - 2 + r;
            if (x >= 0 && x < W && y >= 0 && y < H && !in_rect(p.pvalid, x, y)) gx = gy = 0;
        }
        sm.p[0][r][c] = gx * gx;
        sm.p[1][r][c] = gy * gy;
        sm.p[2][r][c] = gx * gy;
    }
    __syncthreads();

    // 3. the window sums' border mode on product cells outside the image
    if (!interior && p.border_b != HVX_BORDER_UNDEFINED) {
        for (int i = threadIdx.x; i < PR * PC; i += blockDim.x) {
            int r = i / PC, c = i - r * PC;
            int x = x0 - 2 + c, y = y0 - 2 + r;
            if (x >= 0 && x < W && y >= 0 && y < H) continue;
            if (p.border_b == HVX_BORDER_CONSTANT) {
                sm.p[0][r][c] = sm.p[1][r][c] = sm.p[2][r][c] = p.cval_b;
            } else {
                int cr = clampi(y, 0, H - 1) - (y0 - 2), cc = clampi(x, 0, W - 1) - (x0 - 2);
                sm.p[0][r][c] = sm.p[0][cr][cc];
                sm.p[1][r][c] = sm.p[1][cr][cc];
                sm.p[2][r][c] = sm.p[2][cr][cc];
            }
        }
        __syncthreads();
    }

    // 4. vertical 5-sums: one column of 8 rows per item
    for (int i = threadIdx.x; i < 3 * PC * (TH / 8); i += blockDim.x) {
        int k = i / (PC * (TH / 8));
        int rem = i - k * PC * (TH / 8);
        int c = rem % PC;
        int r0 = (rem / PC) * 8;
        int s = sm.p[k][r0][c] + sm.p[k][r0 + 1][c] + sm.p[k][r0 + 2][c] + sm.p[k][r0 + 3][c] +
                sm.p[k][r0 + 4][c];
        sm.v[k][r0][c] = s;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            s += sm.p[k][r0 + j + 4][c] - sm.p[k][r0 + j - 1][c];
            sm.v[k][r0 + j][c] = s;
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
        const int32_t* vr = &sm.v[k][row][seg * 8];
        int s = vr[0] + vr[1] + vr[2] + vr[3] + vr[4];
        S[k][0] = s;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            s += vr[j + 4] - vr[j - 1];
            S[k][j] = s;
        }
    }
    uint32_t mk[8];
    float rv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        bool ok = full || in_rect(p.valid, xs + j, y);
        long long q = harris_q(S[0][j], S[1][j], S[2][j], p.kn, p.kd);
        mk[j] = ok ? (q > p.q_thr ? (uint32_t)p.tv : (uint32_t)p.fv) : 0u;
        if (p.resp) rv[j] = ok ? ratio_to_float(q, p.kd) : 0.0f;
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

}  // namespace

cudaError_t launch_harris(const CUtensorMap& map, const HarrisParams& p, cudaStream_t s) {
    static bool attr_set = false;
    const int smem = (int)sizeof(HarrisSmem);
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(harris_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((p.W + TW - 1) / TW, (p.H + TH - 1) / TH);
    harris_kernel<<<grid, HARRIS_THREADS, smem, s>>>(map, p);
    return cudaGetLastError();
}

}  // namespace hvx
