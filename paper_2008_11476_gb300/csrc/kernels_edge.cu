// Fused edge-detection group and the Gaussian3x3 kernel (Table 2 local and
// point operators; the edge graph of Listing 1 / Section 6 benchmarks):
//
//   in U8 --Gaussian3x3--> G (U8, on chip) --Sobel3x3--> gx, gy (S16, registers)
//        --Magnitude--> m (S16) --Threshold--> mask (U8)
//        --Phase--> phase (U8)
//
// One CTA computes a 128 x 32 output tile:
//   1. one TMA 2-D load brings the 160 x 36 input box (tile + 2-pixel halo,
//      widened to 16-byte-aligned columns) into shared memory; the hardware
//      fills out-of-image bytes with 0, and edge tiles then apply the
//      Gaussian's border mode to those bytes;
//   2. G is computed over the tile + 1-pixel halo (130 x 34) into a shared
//      line buffer; edge tiles then apply the Sobel's border mode to the G
//      cells outside the image (REPLICATE reads the replicated *Gaussian*
//      output, as the node-by-node definition requires);
//   3. each thread takes 16 consecutive pixels of one row, forms gx, gy with
//      separable sums, and produces mask / phase / magnitude, written with
//      16-byte stores.
// Magnitude followed by a binary threshold T is evaluated as
// gx^2 + gy^2 > T^2 + T, which equals round(sqrt(gx^2 + gy^2)) > T exactly.
//
// The batch kernel runs the same tile code persistently over the tiles of
// many images (one tensor map per image, kept in global memory), and issues
// the TMA load of its next tile while it computes the current one.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int TW = EDGE_TW;
constexpr int TH = EDGE_TH;
constexpr int LW = EDGE_LOAD_W;
constexpr int IN_ROWS = TH + 4;
constexpr int G_ROWS = TH + 2;
constexpr uint32_t IN_BYTES = IN_ROWS * LW;

struct EdgeSmem {
    alignas(128) uint8_t in[IN_ROWS][LW];  // image (x0 - 16 + c, y0 - 2 + r)
    alignas(16) uint8_t g[G_ROWS][LW];     // Gaussian (x0 - 16 + c, y0 - 1 + r)
    alignas(8) uint64_t bar;
    int img;                               // batch: image of the current tile
    int next_img;
};

__device__ __forceinline__ void load18(const uint8_t* row, int c, int v[18]) {
    v[0] = row[c - 1];
    uint4 q = *reinterpret_cast<const uint4*>(row + c);
    uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) v[1 + j] = (w[j >> 2] >> (8 * (j & 3))) & 0xFF;
    v[17] = row[c + 16];
}

__device__ __forceinline__ uint32_t pack4(const uint32_t* b) {
    return b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
}

__device__ __forceinline__ void store16_u8(uint8_t* row, int x, int W, const uint32_t b[16]) {
    if (x + 16 <= W) {
        uint4 q;
        q.x = pack4(b);
        q.y = pack4(b + 4);
        q.z = pack4(b + 8);
        q.w = pack4(b + 12);
        *reinterpret_cast<uint4*>(row + x) = q;
    } else {
        for (int j = 0; j < 16 && x + j < W; ++j) row[x + j] = (uint8_t)b[j];
    }
}

__device__ __forceinline__ void store16_s16(int16_t* row, int x, int W, const int v[16]) {
    if (x + 16 <= W) {
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            w[j] = ((uint32_t)v[2 * j] & 0xFFFFu) | ((uint32_t)v[2 * j + 1] << 16);
        uint4* d = reinterpret_cast<uint4*>(row + x);
        d[0] = make_uint4(w[0], w[1], w[2], w[3]);
        d[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
        for (int j = 0; j < 16 && x + j < W; ++j) row[x + j] = (int16_t)v[j];
    }
}

__device__ __forceinline__ bool tile_is_interior(const EdgeParams& p, int x0, int y0) {
    return x0 >= 2 && y0 >= 2 && x0 + TW + 2 <= (int)p.W && y0 + TH + 2 <= (int)p.H;
}

__device__ __forceinline__ bool rect_is_full(const int32_t* r, const EdgeParams& p) {
    return r[0] == 0 && r[1] == 0 && r[2] == (int)p.W && r[3] == (int)p.H;
}

// Apply the Gaussian's border mode to the input bytes outside the image.
__device__ void fix_input_border(EdgeSmem& sm, const EdgeParams& p, int x0, int y0) {
    const int W = p.W, H = p.H;
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    for (int i = threadIdx.x; i < IN_ROWS * LW; i += blockDim.x) {
        int r = i / LW, c = i - r * LW;
        int x = x0 - 16 + c, y = y0 - 2 + r;
        if (x >= 0 && x < W && y >= 0 && y < H) continue;
        uint8_t v;
        if (p.border_g == HVX_BORDER_CONSTANT) {
            v = (uint8_t)p.cval_g;
        } else {
            int cy = clampi(y, 0, H - 1) - (y0 - 2);
            int cx = clampi(x, 0, W - 1) - (x0 - 16);
            v = sm.in[cy][cx];
        }
        sm.in[r][c] = v;
    }
}

// G over rows y0-1 .. y0+TH, columns x0-4 .. x0+TW+3 (4-pixel chunks).
__device__ void compute_gaussian(EdgeSmem& sm, const EdgeParams& p, int x0, int y0,
                                 bool interior) {
    const int rnd = p.rounding == HVX_ROUND_TO_NEAREST ? 8 : 0;
    constexpr int CHUNKS = (TW + 8) / 4;  // 34 chunks of 4 columns, c = 12 .. 144
    const bool full = interior || rect_is_full(p.gvalid, p);
    for (int it = threadIdx.x; it < G_ROWS * CHUNKS; it += blockDim.x) {
        int r = it / CHUNKS;
        int c = 12 + 4 * (it - r * CHUNKS);
        int v[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            int cc = c - 1 + j;
            v[j] = sm.in[r][cc] + 2 * sm.in[r + 1][cc] + sm.in[r + 2][cc];
        }
        uint32_t b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = (uint32_t)((v[i] + 2 * v[i + 1] + v[i + 2] + rnd) >> 4);
        if (!full) {
            int y = y0 - 1 + r;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int x = x0 - 16 + c + i;
                if (x >= 0 && x < (int)p.W && y >= 0 && y < (int)p.H && !in_rect(p.gvalid, x, y))
                    b[i] = 0;
            }
        }
        *reinterpret_cast<uint32_t*>(&sm.g[r][c]) = pack4(b);
    }
}

// Apply the Sobel's border mode to the G cells outside the image.
__device__ void fix_g_border(EdgeSmem& sm, const EdgeParams& p, int x0, int y0) {
    const int W = p.W, H = p.H;
    if (p.border_s == HVX_BORDER_UNDEFINED) return;
    constexpr int COLS = TW + 8;  // c = 12 .. 147
    for (int i = threadIdx.x; i < G_ROWS * COLS; i += blockDim.x) {
        int r = i / COLS, c = 12 + (i - r * COLS);
        int x = x0 - 16 + c, y = y0 - 1 + r;
        if (x >= 0 && x < W && y >= 0 && y < H) continue;
        uint8_t v;
        if (p.border_s == HVX_BORDER_CONSTANT) {
            v = (uint8_t)p.cval_s;
        } else {
            int cy = clampi(y, 0, H - 1) - (y0 - 1);
            int cx = clampi(x, 0, W - 1) - (x0 - 16);
            v = sm.g[cy][cx];
        }
        sm.g[r][c] = v;
    }
}

// Sobel + point operators for 16 pixels of one row, stores to global.
__device__ void sobel_point_stage(EdgeSmem& sm, const EdgeParams& p, int x0, int y0,
                                  bool interior) {
    const int row = threadIdx.x >> 3, seg = threadIdx.x & 7;
    const int y = y0 + row, x = x0 + seg * 16;
    if (y >= (int)p.H || x >= (int)p.W) return;
    const int c = 16 + seg * 16;
    int g0[18], g1[18], g2[18];
    load18(sm.g[row], c, g0);
    load18(sm.g[row + 1], c, g1);
    load18(sm.g[row + 2], c, g2);
    int vs[18], dy[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
        vs[k] = g0[k] + 2 * g1[k] + g2[k];
        dy[k] = g2[k] - g0[k];
    }
    const bool full = interior || rect_is_full(p.valid, p);
    uint32_t mk[16], ph[16];
    int mg[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        int gx = vs[i + 2] - vs[i];
        int gy = dy[i] + 2 * dy[i + 1] + dy[i + 2];
        bool ok = full || in_rect(p.valid, x + i, y);
        if (p.mask) {
            uint32_t m;
            if (!p.thr_general) {
                long long s = (long long)gx * gx + (long long)gy * gy;
                m = s > p.s_thr ? (uint32_t)p.tv : (uint32_t)p.fv;
            } else {
                int mv = magnitude_s16(gx, gy);
                bool t = p.thr_type == HVX_THRESHOLD_BINARY ? mv > p.thr_lo
                                                             : !(mv > p.thr_hi || mv < p.thr_lo);
                m = t ? (uint32_t)p.tv : (uint32_t)p.fv;
            }
            mk[i] = ok ? m : 0u;
        }
        if (p.phase) ph[i] = ok ? phase_u8(gx, gy) : 0u;
        if (p.mag) mg[i] = ok ? magnitude_s16(gx, gy) : 0;
    }
    if (p.mask) store16_u8(p.mask + (size_t)y * p.mask_pitch, x, p.W, mk);
    if (p.phase) store16_u8(p.phase + (size_t)y * p.phase_pitch, x, p.W, ph);
    if (p.mag)
        store16_s16(reinterpret_cast<int16_t*>(reinterpret_cast<uint8_t*>(p.mag) +
                                               (size_t)y * p.mag_pitch),
                    x, p.W, mg);
}

// Gaussian3x3 alone: 16 pixels of one row straight from the input box.
__device__ void gaussian_only_stage(EdgeSmem& sm, const EdgeParams& p, int x0, int y0,
                                    bool interior) {
    const int row = threadIdx.x >> 3, seg = threadIdx.x & 7;
    const int y = y0 + row, x = x0 + seg * 16;
    if (y >= (int)p.H || x >= (int)p.W) return;
    const int c = 16 + seg * 16;
    const int rnd = p.rounding == HVX_ROUND_TO_NEAREST ? 8 : 0;
    int a[18], b[18], d[18];
    load18(sm.in[row + 1], c, a);
    load18(sm.in[row + 2], c, b);
    load18(sm.in[row + 3], c, d);
    int v[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) v[k] = a[k] + 2 * b[k] + d[k];
    const bool full = interior || rect_is_full(p.gvalid, p);
    uint32_t o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        uint32_t g = (uint32_t)((v[i] + 2 * v[i + 1] + v[i + 2] + rnd) >> 4);
        o[i] = (full || in_rect(p.gvalid, x + i, y)) ? g : 0u;
    }
    store16_u8(p.gout + (size_t)y * p.gout_pitch, x, p.W, o);
}

__device__ __forceinline__ void issue_load(EdgeSmem& sm, const CUtensorMap* map, int x0, int y0) {
    mbar_arrive_expect_tx(&sm.bar, IN_BYTES);
    tma_load_2d(&sm.in[0][0], map, &sm.bar, x0 - 16, y0 - 2);
}

// One tile after its input box has landed in sm.in.
__device__ void edge_tile_body(EdgeSmem& sm, const EdgeParams& p, int x0, int y0, bool gauss_only,
                               const CUtensorMap* next_map, int nx0, int ny0) {
    const bool interior = tile_is_interior(p, x0, y0);
    if (!interior) {
        fix_input_border(sm, p, x0, y0);
        __syncthreads();
    }
    if (gauss_only) {
        gaussian_only_stage(sm, p, x0, y0, interior);
        __syncthreads();
        if (next_map && threadIdx.x == 0) {
            fence_proxy_async_smem();
            issue_load(sm, next_map, nx0, ny0);
        }
        return;
    }
    compute_gaussian(sm, p, x0, y0, interior);
    __syncthreads();
    // the input box is no longer read: start the next tile's load now
    if (next_map && threadIdx.x == 0) {
        fence_proxy_async_smem();
        issue_load(sm, next_map, nx0, ny0);
    }
    if (!interior) {
        fix_g_border(sm, p, x0, y0);
        __syncthreads();
    }
    sobel_point_stage(sm, p, x0, y0, interior);
    __syncthreads();
}

__global__ void __launch_bounds__(EDGE_THREADS, 3)
    edge_kernel(const __grid_constant__ CUtensorMap tmap, const EdgeParams p, int gauss_only) {
    __shared__ EdgeSmem sm;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) issue_load(sm, &tmap, x0, y0);
    if (!mbar_wait_bounded(&sm.bar, 0, p.err)) return;
    edge_tile_body(sm, p, x0, y0, gauss_only != 0, nullptr, 0, 0);
}

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

__device__ __forceinline__ void tile_origin(const EdgeParams& p, int t, int& x0, int& y0) {
    int tiles_x = (p.W + TW - 1) / TW;
    int ty = t / tiles_x;
    x0 = (t - ty * tiles_x) * TW;
    y0 = ty * TH;
}

__global__ void __launch_bounds__(EDGE_THREADS, 3) edge_batch_kernel(const EdgeBatchDesc d) {
    __shared__ EdgeSmem sm;
    int t = blockIdx.x;
    if (t >= d.total_tiles) return;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        fence_barrier_init();
        int img = find_image(d.tile_start, d.n_img, t);
        sm.img = img;
        tensormap_acquire(&d.maps[img]);
        EdgeParams p = d.params[img];
        int x0, y0;
        tile_origin(p, t - d.tile_start[img], x0, y0);
        issue_load(sm, &d.maps[img], x0, y0);
    }
    __syncthreads();
    uint32_t parity = 0;
    for (; t < d.total_tiles; t += gridDim.x) {
        const int img = sm.img;
        const EdgeParams& p = d.params[img];
        int x0, y0;
        tile_origin(p, t - __ldg(d.tile_start + img), x0, y0);
        // next tile of this CTA: its image and origin (thread 0 issues the load)
        int tn = t + gridDim.x;
        const CUtensorMap* next_map = nullptr;
        int nx0 = 0, ny0 = 0;
        if (tn < d.total_tiles && threadIdx.x == 0) {
            int ni = find_image(d.tile_start, d.n_img, tn);
            sm.next_img = ni;
            tensormap_acquire(&d.maps[ni]);
            tile_origin(d.params[ni], tn - d.tile_start[ni], nx0, ny0);
            next_map = &d.maps[ni];
        }
        bool ok = mbar_wait_bounded(&sm.bar, parity, d.err);
        if (__syncthreads_or(!ok)) return;
        parity ^= 1u;
        edge_tile_body(sm, p, x0, y0, d.gauss_only != 0, next_map, nx0, ny0);
        if (threadIdx.x == 0) sm.img = sm.next_img;
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_edge(const CUtensorMap& map, const EdgeParams& p, bool gauss_only,
                        cudaStream_t s) {
    dim3 grid((p.W + TW - 1) / TW, (p.H + TH - 1) / TH);
    edge_kernel<<<grid, EDGE_THREADS, 0, s>>>(map, p, gauss_only ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_edge_batch(const EdgeBatchDesc& d, int grid, cudaStream_t s) {
    edge_batch_kernel<<<grid, EDGE_THREADS, 0, s>>>(d);
    return cudaGetLastError();
}

int edge_batch_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, edge_batch_kernel, EDGE_THREADS, 0);
    return n;
}

}  // namespace hvx
