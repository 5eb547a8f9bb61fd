// Gaussian3x3 node alone (Table 2 local operator): the plain Gaussian graph
// and the Gaussian requests of a serving mix.
//
// One CTA (128 threads) computes a 128 x 120 output tile from one TMA box of
// 160 x 122 input bytes (the tile plus one halo row above and below; the
// columns widened to 16-byte boundaries, x0 - 16 .. x0 + 143).  Thread (q, g)
// owns the 8-pixel column strip x0 + 8q .. x0 + 8q + 7 and the 15 rows
// y0 + 15g .. y0 + 15g + 14, and walks down them with a 3-row window: each
// input row is read from shared memory once (three loads), split once into
// 16-bit lanes of pixel pairs, and serves three output rows.  The vertical and
// horizontal 1-2-1 sums, the rounding term and the shift by 4 all work on two
// pixels per 32-bit add; the 8 output bytes are gathered by two byte permutes
// and written with one 8-byte store (a half-warp writes 128 contiguous bytes).
//
// Edge tiles first apply the node's border mode to the box cells outside the
// image (the TMA load fills them with 0); pixels outside the output's valid
// region (BORDER_UNDEFINED) are written as 0.
//
// The batch kernel runs persistently over the tiles of many images (one
// tensor map and parameter block per image), with two boxes in flight per
// CTA: the next tile's box is loading while the current one is computed.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int TW = GAUSS_TW;          // 128
constexpr int TH = GAUSS_TH;          // 120
constexpr int LW = GAUSS_LOAD_W;      // 160
constexpr int LH = GAUSS_LOAD_H;      // 122
constexpr int ROWS = GAUSS_ROWS;      // 15 output rows per thread
constexpr int STAGES = GAUSS_STAGES;  // 2
constexpr uint32_t BOX_BYTES = LW * LH;
static_assert(GAUSS_THREADS == 16 * (TH / ROWS), "16 strips x row groups");

using Box = uint8_t[LH][LW];  // image (x0 - 16 + c, y0 - 1 + r)

struct alignas(128) BoxStage {
    Box b;
};

template <int NS>
struct GaussSmem {
    BoxStage in[NS];
    alignas(8) uint64_t bar[NS];
    // batch: parameters and origin of the tiles in flight (slot k mod (NS + 1))
    EdgeParams prm[NS + 1];
    int tx0[NS + 1], ty0[NS + 1];
    // batch of at most BATCH_SMEM_IMAGES images: its tile tables
    int ts[BATCH_SMEM_IMAGES + 1], tx[BATCH_SMEM_IMAGES];
    // batch: warps that finished with each box stage (the last of a tile
    // issues the stage's next load) and the last tile index loaded into it
    unsigned released[NS];
    int last_k[NS];
};

__device__ __forceinline__ bool tile_is_interior(const EdgeParams& p, int x0, int y0, int th) {
    return x0 >= 1 && y0 >= 1 && x0 + TW + 1 <= (int)p.W && y0 + th + 1 <= (int)p.H;
}

// Box cells outside the image under REPLICATE / CONSTANT (edge tiles only);
// lh: the box rows the TMA filled.
__device__ void fix_box_border(Box& in, const EdgeParams& p, int x0, int y0, int lh) {
    const int W = p.W, H = p.H;
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    const bool cst = p.border_g == HVX_BORDER_CONSTANT;
    const uint8_t cv = (uint8_t)p.cval_g;
    for_each_outside(lh, LW, x0 - 16, y0 - 1, W, H, [&](int r, int c) {
        const int x = x0 - 16 + c, y = y0 - 1 + r;
        in[r][c] = cst ? cv : in[clampi(y, 0, H - 1) - (y0 - 1)][clampi(x, 0, W - 1) - (x0 - 16)];
    });
}

// fix_box_border restricted to box rows r0 .. r1 - 1 and the columns the
// strips read (12 .. 147), for the batch kernel, whose warps run ahead of
// each other without a block barrier: each warp fixes the rows its two row
// groups read, lanes striding over the cells, then syncs.  Neighbouring
// warps share halo rows; both write the same values, each taken from a cell
// inside the image (which no thread writes).
__device__ void fix_box_border_warp(Box& in, const EdgeParams& p, int x0, int y0, int r0,
                                    int r1) {
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    const int W = p.W, H = p.H, bx = x0 - 16, by = y0 - 1;
    const bool cst = p.border_g == HVX_BORDER_CONSTANT;
    const uint8_t cv = (uint8_t)p.cval_g;
    const int lane = threadIdx.x & 31;
    auto put = [&](int r, int c) {
        in[r][c] = cst ? cv : in[clampi(by + r, 0, H - 1) - by][clampi(bx + c, 0, W - 1) - bx];
    };
    constexpr int C0 = 12, C1 = 148;
    const int ra = max(r0, -by), rb = min(r1, H - by);  // rows inside the image
    // rows outside the image: every column
    for (int r = r0; r < r1; ++r)
        if (r < ra || r >= rb)
            for (int c = C0 + lane; c < C1; c += 32) put(r, c);
    // rows inside: the columns left and right of the image
    const int la = C0, lb = min(C1, -bx), rca = max(C0, W - bx), rcb = C1;
    const int nl = max(lb - la, 0), nr = max(rcb - rca, 0), n = nl + nr;
    if (n > 0)
        for (int i = lane; i < (rb - ra) * n; i += 32) {
            const int r = ra + i / n, j = i - (i / n) * n;
            put(r, j < nl ? la + j : rca + j - nl);
        }
    __syncwarp();
}

// Pixel pairs (x - 2, x - 1), (x, x + 1) .. (x + 8, x + 9) of one box row as
// 16-bit lanes, for the strip starting at box column c (= x - x0 + 16).
__device__ __forceinline__ void load_pairs(const uint8_t* row, int c, uint32_t P[6]) {
    const uint2 m = *reinterpret_cast<const uint2*>(row + c);
    const uint32_t wl = *reinterpret_cast<const uint32_t*>(row + c - 4);
    const uint32_t wr = *reinterpret_cast<const uint32_t*>(row + c + 8);
    P[0] = hi_pair(wl);
    P[1] = lo_pair(m.x);
    P[2] = hi_pair(m.x);
    P[3] = lo_pair(m.y);
    P[4] = hi_pair(m.y);
    P[5] = lo_pair(wr);
}

// Gaussian outputs x .. x + 7 of one row from the pair words of the input rows
// above (a), at (b) and below (c); bytes packed into two words.  Each lane
// sum is at most 16 * 255 + 8 < 2^12, so lanes never carry into each other;
// after the shift by 4 the results sit in bytes 0 and 2 of each word.
__device__ __forceinline__ uint2 gauss8(const uint32_t* a, const uint32_t* b, const uint32_t* c,
                                        uint32_t rnd) {
    uint32_t V[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) V[k] = a[k] + 2u * b[k] + c[k];
    uint32_t o[4];
#pragma unroll
    for (int j = 1; j <= 4; ++j)
        o[j - 1] = (shift_pair(V[j - 1], V[j]) + shift_pair(V[j], V[j + 1]) + 2u * V[j] + rnd) >> 4;
    return make_uint2(__byte_perm(o[0], o[1], 0x6420), __byte_perm(o[2], o[3], 0x6420));
}

// Store of a strip row that is cut by the right image edge or crosses the
// output's valid region.
__device__ __noinline__ void store_edge(uint8_t* dst, int x, int y, const EdgeParams& p, uint2 o) {
    const bool full = rect_full(p.gvalid, p.W, p.H);
    for (int j = 0; j < 8 && x + j < (int)p.W; ++j) {
        uint8_t v = (uint8_t)((j < 4 ? o.x : o.y) >> (8 * (j & 3)));
        if (!full && !in_rect(p.gvalid, x + j, y)) v = 0;
        dst[x + j] = v;
    }
}

// One 128 x 8R tile after its box has landed (and, on edge tiles, been
// border-fixed); R output rows per thread.
template <int R>
__device__ __forceinline__ void gauss_tile(const Box& in, const EdgeParams& p, int x0, int y0,
                                           bool interior) {
    const int q = threadIdx.x & 15, g = threadIdx.x >> 4;
    const int W = p.W, H = p.H;
    const int x = x0 + 8 * q, yb = y0 + R * g;
    if (x >= W || yb >= H) return;
    const uint32_t rnd = p.rounding == HVX_ROUND_TO_NEAREST ? 0x00080008u : 0u;
    const size_t pitch = p.gout_pitch;
    uint8_t* dst = p.gout + (size_t)yb * pitch;
    const uint8_t* row = &in[R * g][0];  // input row yb - 1
    const int c = 16 + 8 * q;
    uint32_t P[3][6];
    load_pairs(row, c, P[0]);
    load_pairs(row + LW, c, P[1]);
    const bool fast = (interior || rect_full(p.gvalid, W, H)) && x + 8 <= W && yb + R <= H;
    if (fast) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            load_pairs(row + (i + 2) * LW, c, P[(i + 2) % 3]);
            *reinterpret_cast<uint2*>(dst + x) = gauss8(P[i % 3], P[(i + 1) % 3], P[(i + 2) % 3], rnd);
            dst += pitch;
        }
    } else {
        const int n = min(R, H - yb);
#pragma unroll 1
        for (int i = 0; i < n; ++i) {
            uint32_t* a = P[0];
            uint32_t* b = P[1];
            uint32_t c2[6];
            load_pairs(row + (i + 2) * LW, c, c2);
            store_edge(dst, x, yb + i, p, gauss8(a, b, c2, rnd));
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                a[k] = b[k];
                b[k] = c2[k];
            }
            dst += pitch;
        }
    }
}

// One image: one CTA per 128 x 8R tile (R rows per thread, chosen per image
// size by gauss_single_rows; the tensor map's box is 160 x (8R + 2)).
template <int R>
__global__ void __launch_bounds__(GAUSS_THREADS)
    gauss_kernel(const __grid_constant__ CUtensorMap tmap, const EdgeParams p) {
    static_assert(R >= 1 && R <= ROWS, "the box holds at most 8 ROWS + 2 rows");
    __shared__ GaussSmem<1> sm;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * 8 * R;
    // a programmatic dependent launch (launch_pdl): no global-memory access
    // before the previous grid on the stream has completed
    pdl_launch_dependents();
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        fence_barrier_init();
    }
    pdl_wait();
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&sm.bar[0], (uint32_t)(LW * (8 * R + 2)));
        tma_load_2d(&sm.in[0].b[0][0], &tmap, &sm.bar[0], x0 - 16, y0 - 1);
    }
    // every thread leaves together when the (bounded) wait ran out
    if (__syncthreads_or(!mbar_wait_bounded(&sm.bar[0], 0, p.err))) return;
    const bool interior = tile_is_interior(p, x0, y0, 8 * R);
    if (!interior) {
        fix_box_border(sm.in[0].b, p, x0, y0, 8 * R + 2);
        __syncthreads();
    }
    gauss_tile<R>(sm.in[0].b, p, x0, y0, interior);
}

// Thread 0: the origin of batch tile t into slot ps, then one bulk copy of
// its image's parameter block into slot ps and the TMA load of its box into
// stage s, both completing on the stage's barrier.  `tab`: the tile tables
// are in shared memory.
__device__ __forceinline__ void issue_tile(GaussSmem<STAGES>& sm, const EdgeBatchDesc& d, bool tab,
                                           int s, int ps, int t) {
    int img, t0, tiles_x;
    if (tab) {
        img = find_image_smem(sm.ts, d.n_img, t);
        t0 = sm.ts[img];
        tiles_x = sm.tx[img];
    } else {
        img = find_image(d.tile_start, d.n_img, t);
        t0 = __ldg(d.tile_start + img);
        tiles_x = __ldg(d.tiles_x + img);
    }
    const int local = t - t0, ty = local / tiles_x;
    const int x0 = (local - ty * tiles_x) * TW, y0 = ty * TH;
    sm.tx0[ps] = x0;
    sm.ty0[ps] = y0;
    tensormap_acquire(&d.maps[img]);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&sm.bar[s], BOX_BYTES + (uint32_t)sizeof(EdgeParams));
    bulk_copy_g2s(&sm.prm[ps], &d.params[img], (uint32_t)sizeof(EdgeParams), &sm.bar[s]);
    tma_load_2d(&sm.in[s].b[0][0], &d.maps[img], &sm.bar[s], x0 - 16, y0 - 1);
}

// Persistent: CTA b takes tiles b, b + grid, b + 2 grid, ...; tile k of the
// CTA lives in box stage k mod STAGES.  No block barrier in the tile loop:
// each warp waits for its tile's box on the stage's mbarrier, fixes the
// border cells of its own rows (edge tiles), computes, and counts itself out
// of the stage; the last warp out of tile k issues tile k + STAGES into it.
// A wait that runs out (bounded, about a second) records the error and ends
// the warp's loop; after the loop thread 0 waits (bounded) for any load still
// in flight.
__global__ void __launch_bounds__(GAUSS_THREADS) gauss_batch_kernel(const EdgeBatchDesc d) {
    constexpr unsigned NWARPS = GAUSS_THREADS / 32;
    __shared__ GaussSmem<STAGES> sm;
    const int first = blockIdx.x;
    if (first >= d.total_tiles) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sm.bar[s], 1);
            sm.released[s] = 0u;
            sm.last_k[s] = -1;
        }
        fence_barrier_init();
    }
    const bool tab = d.n_img <= BATCH_SMEM_IMAGES;
    if (tab)
        for (int i = threadIdx.x; i <= d.n_img; i += blockDim.x) {
            sm.ts[i] = __ldg(d.tile_start + i);
            if (i < d.n_img) sm.tx[i] = __ldg(d.tiles_x + i);
        }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < STAGES; ++s) {
            const int t = first + s * (int)gridDim.x;
            if (t < d.total_tiles) {
                sm.last_k[s] = s;
                issue_tile(sm, d, tab, s, s, t);
            }
        }
    const int r0 = 2 * ROWS * (threadIdx.x >> 5);  // first box row of this warp's row groups
    bool failed = false;
    int k = 0;
    for (int t = first; t < d.total_tiles; t += gridDim.x, ++k) {
        const int s = k % STAGES;
        const int ps = k % (STAGES + 1);
        const uint32_t parity = (uint32_t)(k / STAGES) & 1u;
        if (!mbar_wait_bounded(&sm.bar[s], parity, d.err)) {
            failed = true;
            break;
        }
        const EdgeParams& p = sm.prm[ps];
        const int x0 = sm.tx0[ps], y0 = sm.ty0[ps];
        const bool interior = tile_is_interior(p, x0, y0, TH);
        if (!interior) fix_box_border_warp(sm.in[s].b, p, x0, y0, r0, r0 + 2 * ROWS + 2);
        gauss_tile<ROWS>(sm.in[s].b, p, x0, y0, interior);
        // this warp is done with box s: count it out, the last one loads the next tile
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            __threadfence_block();
            const unsigned prev = atomicAdd(&sm.released[s], 1u);
            if (prev % NWARPS == NWARPS - 1) {
                __threadfence_block();
                const int tn = t + STAGES * (int)gridDim.x;
                if (tn < d.total_tiles) {
                    sm.last_k[s] = k + STAGES;
                    issue_tile(sm, d, tab, s, (k + STAGES) % (STAGES + 1), tn);
                }
            }
        }
    }
    // a wait that ran out: no load may still be writing shared memory when the CTA ends
    if (__syncthreads_or(failed) && threadIdx.x == 0)
        for (int s = 0; s < STAGES; ++s)
            if (sm.last_k[s] >= 0)
                mbar_wait_bounded(&sm.bar[s], (uint32_t)(sm.last_k[s] / STAGES) & 1u, nullptr);
}

}  // namespace

cudaError_t launch_gauss(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s) {
    const int R = p.rows == 2 || p.rows == 5 ? p.rows : ROWS;
    dim3 grid((p.W + TW - 1) / TW, (p.H + 8 * R - 1) / (8 * R));
    switch (R) {
        case 2: return launch_pdl(gauss_kernel<2>, grid, dim3(GAUSS_THREADS), 0, s, map, p);
        case 5: return launch_pdl(gauss_kernel<5>, grid, dim3(GAUSS_THREADS), 0, s, map, p);
        default: return launch_pdl(gauss_kernel<ROWS>, grid, dim3(GAUSS_THREADS), 0, s, map, p);
    }
}

// Rows per thread of the single-image Gaussian kernel (tiles of 128 x 8R):
// as for the edge kernel, R = 5, or R = 2 when the image has fewer 128 x 40
// tiles than SMs (a small image then still spreads over the GPU), so that a
// launch's latency is a few rows of work per thread.
int gauss_single_rows(int W, int H, int num_sms) {
    const long long tiles5 = (long long)((W + TW - 1) / TW) * ((H + 39) / 40);
    return tiles5 >= (num_sms > 0 ? num_sms : 152) ? 5 : 2;
}

cudaError_t launch_gauss_batch(const EdgeBatchDesc& d, int grid, cudaStream_t s) {
    gauss_batch_kernel<<<grid, GAUSS_THREADS, 0, s>>>(d);
    return cudaGetLastError();
}

int gauss_batch_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gauss_batch_kernel, GAUSS_THREADS, 0);
    return n;
}

}  // namespace hvx
