// 5x5 binomial Convolve (Table 2 local operator; the Gauss application of
// the Section 6 evaluation): out = floor(sum_{5x5} w I / 256) with
// w = [1 4 6 4 1]^T [1 4 6 4 1], U8 in and out.
//
// Same tiles, threads, boxes and batch machinery as the fused edge kernel:
// one CTA (128 threads) computes a 128 x 8R tile from one TMA box of
// 160 x (8R + 4) input bytes (the tile plus a 2-pixel halo, columns widened
// to 16-byte boundaries).  Thread (q, g) owns the strip x0 + 8q .. + 7 and R
// rows and walks down them with a 5-row window of input pixel pairs in
// registers (each input row read from shared memory once).  The vertical
// 1-4-6-4-1 sums of a row and then the horizontal ones run in 16-bit lanes,
// two pixels per 32-bit operation: vertical sums are at most 16 * 255, the
// full sums at most 256 * 255 = 65280, so no lane ever carries; the shift by
// 8 leaves the output bytes in bytes 0 and 2 of each word.  The 8 bytes of
// a strip row leave in one 8-byte store.
//
// Edge tiles first give the box cells outside the image the node's border
// mode (the TMA load fills them with 0); outputs outside the valid region
// (BORDER_UNDEFINED: 2 pixels in from every edge) are written as 0.  The
// batch kernel is persistent with a 2-stage box ring and, like the edge
// batch kernel, no block barrier in its tile loop.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int TW = EDGE_TW;          // 128
constexpr int LW = EDGE_LOAD_W;      // 160
constexpr int LH = EDGE_LOAD_H;      // 124: 8 * 15 rows + the halo
constexpr int MAXR = EDGE_ROWS;      // 15
constexpr int STAGES = EDGE_STAGES;  // 2
constexpr int THREADS = EDGE_THREADS;  // 128: 16 strips x 8 row groups

using Box = uint8_t[LH][LW];  // image (x0 - 16 + c, y0 - 2 + r)

struct alignas(128) BoxStage {
    Box b;
};

template <int NS>
struct G5Smem {
    BoxStage in[NS];
    alignas(8) uint64_t bar[NS];
    // batch: parameters and origin of the tiles in flight (slot k mod (NS + 1))
    EdgeParams prm[NS + 1];
    int tx0[NS + 1], ty0[NS + 1];
    int ts[BATCH_SMEM_IMAGES + 1], tx[BATCH_SMEM_IMAGES];
    unsigned released[NS];
    int last_k[NS];
};

__device__ __forceinline__ bool interior5(const EdgeParams& p, int x0, int y0, int th) {
    return x0 >= 2 && y0 >= 2 && x0 + TW + 2 <= (int)p.W && y0 + th + 2 <= (int)p.H;
}

// The border value of box cell (r, c) outside the image (REPLICATE: the
// nearest pixel, CONSTANT: the constant); reads only cells inside the image.
__device__ __forceinline__ uint8_t border_cell(const Box& in, const EdgeParams& p, int bx, int by,
                                               int r, int c) {
    if (p.border_g == HVX_BORDER_CONSTANT) return (uint8_t)p.cval_g;
    return in[clampi(by + r, 0, (int)p.H - 1) - by][clampi(bx + c, 0, (int)p.W - 1) - bx];
}

// Every box cell outside the image, rows 0 .. lh - 1 (single-image kernel:
// the whole CTA, then a barrier).
__device__ void fix_border5(Box& in, const EdgeParams& p, int x0, int y0, int lh) {
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    const int W = p.W, H = p.H, bx = x0 - 16, by = y0 - 2;
    for_each_outside(lh, LW, bx, by, W, H,
                     [&](int r, int c) { in[r][c] = border_cell(in, p, bx, by, r, c); });
}

// The same for box rows r0 .. r1 - 1 and the columns the strips read
// (12 .. 147), by one warp, lanes striding over the cells (batch kernel:
// each warp fixes the rows its two row groups read; neighbouring warps write
// the same values into their shared halo rows).
__device__ void fix_border5_warp(Box& in, const EdgeParams& p, int x0, int y0, int r0, int r1) {
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    const int W = p.W, H = p.H, bx = x0 - 16, by = y0 - 2;
    const int lane = threadIdx.x & 31;
    constexpr int C0 = 12, C1 = 148;
    const int ra = max(r0, -by), rb = min(r1, H - by);  // rows inside the image
    for (int r = r0; r < r1; ++r)
        if (r < ra || r >= rb)
            for (int c = C0 + lane; c < C1; c += 32) in[r][c] = border_cell(in, p, bx, by, r, c);
    const int la = C0, lb = min(C1, -bx), rca = max(C0, W - bx);
    const int nl = max(lb - la, 0), nr = max(C1 - rca, 0), n = nl + nr;
    if (n > 0)
        for (int i = lane; i < (rb - ra) * n; i += 32) {
            const int r = ra + i / n, j = i - (i / n) * n;
            const int c = j < nl ? la + j : rca + j - nl;
            in[r][c] = border_cell(in, p, bx, by, r, c);
        }
    __syncwarp();
}

// Pixel pairs (x - 2, x - 1), (x, x + 1) .. (x + 8, x + 9) of one box row as
// 16-bit lanes, for the strip starting at box column c (= x - x0 + 16).
__device__ __forceinline__ void load_pairs5(const uint8_t* row, int c, uint32_t P[6]) {
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

// Outputs x .. x + 7 of one row from the pair words of the input rows
// y - 2 .. y + 2 (a .. e); bytes packed into two words.  Word k of V holds
// the vertical sums at (x - 2 + 2k, x - 1 + 2k); output word j (pixels
// x + 2j, x + 2j + 1) is V[j] + 4 S[j] + 6 V[j + 1] + 4 S[j + 1] + V[j + 2]
// with S[k] the pair one pixel to the right of V[k].
__device__ __forceinline__ uint2 binom5_row(const uint32_t* a, const uint32_t* b,
                                            const uint32_t* c, const uint32_t* d,
                                            const uint32_t* e) {
    uint32_t V[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) V[k] = (a[k] + e[k]) + 4u * (b[k] + d[k]) + 6u * c[k];
    uint32_t S[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) S[k] = shift_pair(V[k], V[k + 1]);
    uint32_t o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = ((V[j] + V[j + 2]) + 4u * (S[j] + S[j + 1]) + 6u * V[j + 1]) >> 8;
    return make_uint2(__byte_perm(o[0], o[1], 0x6420), __byte_perm(o[2], o[3], 0x6420));
}

// Store of a strip row that is cut by the right image edge or crosses the
// output's valid region.
__device__ __noinline__ void store_edge5(uint8_t* dst, int x, int y, const EdgeParams& p, uint2 o) {
    const bool full = rect_full(p.gvalid, p.W, p.H);
    for (int j = 0; j < 8 && x + j < (int)p.W; ++j) {
        uint8_t v = (uint8_t)((j < 4 ? o.x : o.y) >> (8 * (j & 3)));
        if (!full && !in_rect(p.gvalid, x + j, y)) v = 0;
        dst[x + j] = v;
    }
}

// One 128 x 8R tile after its box has landed (and, on edge tiles, been
// border-filled); R output rows per thread.  The 5-row window rotates by
// renaming (the row loop is unrolled).
template <int R>
__device__ __forceinline__ void binom5_tile(const Box& in, const EdgeParams& p, int x0, int y0,
                                            bool interior) {
    const int q = threadIdx.x & 15, g = threadIdx.x >> 4;
    const int W = p.W, H = p.H;
    const int x = x0 + 8 * q, yb = y0 + R * g;
    if (x >= W || yb >= H) return;
    const size_t pitch = p.gout_pitch;
    uint8_t* dst = p.gout + (size_t)yb * pitch;
    const uint8_t* row = &in[R * g][0];  // input row yb - 2
    const int c = 16 + 8 * q;
    uint32_t P[5][6];
#pragma unroll
    for (int k = 0; k < 4; ++k) load_pairs5(row + k * LW, c, P[k]);
    const bool fast = (interior || rect_full(p.gvalid, W, H)) && x + 8 <= W && yb + R <= H;
    const int n = min(R, H - yb);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        if (!fast && i >= n) break;
        load_pairs5(row + (i + 4) * LW, c, P[(i + 4) % 5]);
        const uint2 o = binom5_row(P[i % 5], P[(i + 1) % 5], P[(i + 2) % 5], P[(i + 3) % 5],
                                   P[(i + 4) % 5]);
        if (fast)
            *reinterpret_cast<uint2*>(dst + x) = o;
        else
            store_edge5(dst, x, yb + i, p, o);
        dst += pitch;
    }
}

// One image: one CTA per 128 x 8R tile (R = p.rows, 2 or 5 by image size;
// the tensor map's box is 160 x (8R + 4)); a programmatic dependent launch.
template <int R>
__global__ void __launch_bounds__(THREADS) binom5_kernel(const __grid_constant__ CUtensorMap tmap,
                                                         const EdgeParams p) {
    __shared__ G5Smem<1> sm;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * 8 * R;
    pdl_launch_dependents();
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        fence_barrier_init();
    }
    pdl_wait();
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&sm.bar[0], (uint32_t)(LW * (8 * R + 4)));
        tma_load_2d(&sm.in[0].b[0][0], &tmap, &sm.bar[0], x0 - 16, y0 - 2);
    }
    // every thread leaves together when the (bounded) wait ran out
    if (__syncthreads_or(!mbar_wait_bounded(&sm.bar[0], 0, p.err))) return;
    const bool interior = interior5(p, x0, y0, 8 * R);
    if (!interior) {
        fix_border5(sm.in[0].b, p, x0, y0, 8 * R + 4);
        __syncthreads();
    }
    binom5_tile<R>(sm.in[0].b, p, x0, y0, interior);
}

// Thread 0 / the last warp out of a stage: the origin of batch tile t into
// slot ps, one bulk copy of its image's parameter block into slot ps and the
// TMA load of its box into stage s, both completing on the stage's barrier.
template <int R>
__device__ __forceinline__ void issue5(G5Smem<STAGES>& sm, const EdgeBatchDesc& d, bool tab, int s,
                                       int ps, int t) {
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
    const int x0 = (local - ty * tiles_x) * TW, y0 = ty * 8 * R;
    sm.tx0[ps] = x0;
    sm.ty0[ps] = y0;
    tensormap_acquire(&d.maps[img]);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&sm.bar[s], (uint32_t)(LW * (8 * R + 4)) + (uint32_t)sizeof(EdgeParams));
    bulk_copy_g2s(&sm.prm[ps], &d.params[img], (uint32_t)sizeof(EdgeParams), &sm.bar[s]);
    tma_load_2d(&sm.in[s].b[0][0], &d.maps[img], &sm.bar[s], x0 - 16, y0 - 2);
}

// Persistent over the tiles of many images (tile k of a CTA in box stage k
// mod STAGES), without a block barrier in the tile loop: each warp waits for
// its tile's box, fills the border cells of its own rows (edge tiles),
// computes, and counts itself out of the stage; the last warp out issues
// tile k + STAGES.  A wait that runs out (bounded) records the error and
// ends the warp's loop; thread 0 then waits (bounded) for loads in flight.
template <int R>
__global__ void __launch_bounds__(THREADS) binom5_batch_kernel(const EdgeBatchDesc d) {
    static_assert(R >= 3 && R <= MAXR, "box ring holds at most 8 MAXR + 4 rows");
    constexpr unsigned NWARPS = THREADS / 32;
    __shared__ G5Smem<STAGES> sm;
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
                issue5<R>(sm, d, tab, s, s, t);
            }
        }
    const int r0 = 2 * R * (threadIdx.x >> 5);  // first box row of this warp's row groups
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
        const bool interior = interior5(p, x0, y0, 8 * R);
        if (!interior) fix_border5_warp(sm.in[s].b, p, x0, y0, r0, r0 + 2 * R + 4);
        binom5_tile<R>(sm.in[s].b, p, x0, y0, interior);
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            __threadfence_block();
            const unsigned prev = atomicAdd(&sm.released[s], 1u);
            if (prev % NWARPS == NWARPS - 1) {
                __threadfence_block();
                const int tn = t + STAGES * (int)gridDim.x;
                if (tn < d.total_tiles) {
                    sm.last_k[s] = k + STAGES;
                    issue5<R>(sm, d, tab, s, (k + STAGES) % (STAGES + 1), tn);
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

cudaError_t launch_binom5(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s) {
    const int R = p.rows == 2 ? 2 : 5;
    dim3 grid((p.W + TW - 1) / TW, (p.H + 8 * R - 1) / (8 * R));
    if (R == 2) return launch_pdl(binom5_kernel<2>, grid, dim3(THREADS), 0, s, map, p);
    return launch_pdl(binom5_kernel<5>, grid, dim3(THREADS), 0, s, map, p);
}

cudaError_t launch_binom5_batch(const EdgeBatchDesc& d, int grid, int rows, cudaStream_t s) {
    switch (rows) {
        case 5: binom5_batch_kernel<5><<<grid, THREADS, 0, s>>>(d); break;
        case 10: binom5_batch_kernel<10><<<grid, THREADS, 0, s>>>(d); break;
        default: binom5_batch_kernel<MAXR><<<grid, THREADS, 0, s>>>(d); break;
    }
    return cudaGetLastError();
}

int binom5_batch_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, binom5_batch_kernel<MAXR>, THREADS, 0);
    return n;
}

}  // namespace hvx
