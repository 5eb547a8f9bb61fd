// Fused edge-detection group (Table 2 local and point operators; the edge
// graph of Listing 1 / the Section 6 benchmarks):
//
//   in U8 --Gaussian3x3--> G --Sobel3x3--> gx, gy
//        --Magnitude--> m --Threshold--> mask (U8)      --Phase--> phase (U8)
//
// G, gx, gy and m never leave the SM.  One CTA (128 threads) computes a
// 128 x 120 output tile from one TMA box of 160 x 124 input bytes (the tile
// plus a 2-pixel halo, columns widened to 16-byte boundaries).  Thread (q, g)
// owns the 8-pixel column strip x = x0 + 8q .. x + 7 and the 15 output rows
// y0 + 15g .. y0 + 15g + 14, and walks down them with two sliding 3-row
// windows held in registers:
//   * input rows, each read from shared memory once (three loads) and split
//     once into 16-bit lanes of pixel pairs;
//   * Gaussian rows: each G row (the 10 values x - 1 .. x + 8 the Sobel needs,
//     in five words of pairs (x - 1 + 2j, x + 2j)) is computed once from three
//     input rows and enters three Sobel rows.
// Gaussian and Sobel sums run in 16-bit lanes (two pixels per 32-bit add,
// biased so that no lane goes negative).  A Gaussian lane holds 16 G, the
// weighted sum with its low four bits cleared (one mask instead of a shift
// and a mask), and the Sobel sums run on those lanes; gx and gy are unpacked
// to binary32 by exponent splicing and one packed fma that also takes out the
// factor 16, and the point operators run in binary32, where every value is an
// exact integer.  Magnitude followed by a binary threshold T is evaluated as
// gx^2 + gy^2 > T^2 + T, which equals round(sqrt(gx^2 + gy^2)) > T, two
// pixels per packed fma; the mask bytes come from the sign bits of those
// values by sign-replicating byte permutes.  The mask and phase bytes of a
// strip row leave in one 8-byte store each (a half-warp writes 128
// contiguous bytes).  Interior tiles run a copy of the row loop with no
// border, validity or bounds tests.
//
// Borders.  The TMA load fills the box cells outside the image with 0; edge
// tiles then apply the Gaussian's border mode to them.  G rows and columns
// outside the image take the Sobel's border mode (REPLICATE reads the
// replicated *Gaussian output*, as the node-by-node definition requires), and
// G inside the image but outside the Gaussian's valid region is 0; those G
// rows are rebuilt lane by lane on a slow path that only the threads whose
// window touches the image edge take.  Outputs outside their valid region
// are written as 0.
//
// The batch kernel runs the same tile code persistently over the tiles of
// many images (one tensor map and parameter block per image) with two boxes
// in flight per CTA.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int TW = EDGE_TW;          // 128
constexpr int TH = EDGE_TH;          // 120
constexpr int LW = EDGE_LOAD_W;      // 160
constexpr int LH = EDGE_LOAD_H;      // 124
constexpr int ROWS = EDGE_ROWS;      // 15
constexpr int STAGES = EDGE_STAGES;  // 2
constexpr uint32_t BOX_BYTES = LW * LH;
static_assert(EDGE_THREADS == 16 * (TH / ROWS), "16 strips x row groups");

// Kernel modes (template parameter).
constexpr int M_GAUSS = EDGE_MODE_GAUSS;  // Gaussian3x3 alone (kernels_gauss.cu)
constexpr int M_MASK_PHASE = 1;  // binary threshold mask + phase
constexpr int M_MASK = 2;        // binary threshold mask only
constexpr int M_PHASE = 3;       // phase only
constexpr int M_GENERAL = 4;     // any outputs (magnitude export, range threshold)
constexpr int M_MASK_YY = 5;     // binary threshold mask of Magnitude(gy, gy) (gx dead)
constexpr int M_SOBEL_MASK = 6;  // no Gaussian: the mask of Sobel -> Magnitude -> Threshold
constexpr int M_BINOM5 = EDGE_MODE_BINOM5;  // 5x5 binomial Convolve alone (kernels_gauss5.cu)
constexpr int M_SOBEL_GX = 8;    // no Gaussian: the Sobel's gx alone, stored as S16

using Box = uint8_t[LH][LW];  // image (x0 - 16 + c, y0 - 2 + r)

struct alignas(128) BoxStage {
    Box b;
};

// Phase table entry for octant o = 4 [gx < 0] + 2 [gy < 0] + [|gy| > |gx|]
// and guess n (entry o * 34 + n): tan((n - 1/2) pi / 128), and the phase byte
// for the octant angle n (byte 0) and n - 1 (byte 1).
struct PhaseEntry {
    float tan;
    uint32_t q;
};

template <int NS>
struct EdgeSmem {
    BoxStage in[NS];                    // ring of TMA destinations
    alignas(8) uint64_t bar[NS];
    // batch: parameters and origin of the tiles in flight, in a ring one longer
    // than the box ring (tile k uses slot k mod (NS + 1), so the slot that
    // tile k + NS fills belongs to tile k - 1, which is finished)
    EdgeParams prm[NS + 1];
    int tx0[NS + 1], ty0[NS + 1];
    PhaseEntry plut[8 * 34];            // Phase table (build_phase_lut)
    uint32_t gslow[EDGE_THREADS][5];    // per-thread result of the slow G path
    // batch of at most BATCH_SMEM_IMAGES images: its tile tables
    int ts[BATCH_SMEM_IMAGES + 1], tx[BATCH_SMEM_IMAGES];
    // batch: warps that finished with each box stage (the last of a tile
    // issues the stage's next load) and the last tile index loaded into it
    unsigned released[NS];
    int last_k[NS];
};

__device__ __forceinline__ uint32_t pack4(uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
    return __byte_perm(__byte_perm(b0, b1, 0x0040), __byte_perm(b2, b3, 0x0040), 0x5410);
}

// Hardware reciprocal approximation (rcp.approx.ftz.f32, at most 1 ulp off).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Fill the Phase table (once per CTA).
__device__ void build_phase_lut(PhaseEntry* lut) {
    for (int i = threadIdx.x; i < 8 * 34; i += blockDim.x) {
        const int o = i / 34, n = i - o * 34;
        const bool sx = (o >> 2) & 1, sy = (o >> 1) & 1, sw = o & 1;
        uint32_t q[2];
        for (int k = 0; k < 2; ++k) {
            const int ra = n - k;                 // octant angle in bins, 0 .. 32
            const int q1 = sw ? 64 - ra : ra;     // first-quadrant angle
            q[k] = (uint32_t)((sx ? 128 : 0) + ((sx != sy) ? -q1 : q1)) & 0xFFu;
        }
        lut[i].tan = kPhaseTan[n];
        lut[i].q = q[0] | (q[1] << 8);
    }
}

// Phase from exact integer gradients held in binary32 (gen_phase_poly.py
// derives and checks every step over all integer gradient pairs): with
// mn, mx = min, max of |gx|, |gy| and t = mn / mx, the rounded octant angle
// is n or n - 1 for n = floor(1 + t (A + B t)), and it is n exactly when
// mn - mx tan((n - 1/2) pi / 128) > 0.  n comes out of a round-down fma as
// the low mantissa bits of a number in [1.5 * 2^23, 2^24); the table entry of
// (octant, n) holds tan((n - 1/2) pi / 128) and the final phase byte for both
// outcomes (byte 0: n, byte 1: n - 1), and the sign of the test picks the
// byte.  The octant's sign bits as 0 / 1 floats come from saturating
// operations on exact integers (sat(-gx) = [gx < 0], sat(|gy| - |gx|) =
// [|gy| > |gx|]), and the table index is added to the guess with exact fmas
// (the guess has unit spacing in [1.5 * 2^23, 2^24)), so the index costs
// floating-point operations only.  gx = gy = 0 gives t = 0, n = 1 and a
// negative test (mx is raised to 1 there), so phase 0.

// max(|a|, |b|, 1): one three-input max.
__device__ __forceinline__ float max_abs_1(float a, float b) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(fabsf(a)), "f"(fabsf(b)), "f"(1.0f));
    return r;
}

// The Phase bytes of a pixel pair (lanes x, y of gx and gy) in bytes 0 and 1:
// the steps above for both pixels, with the guess and the octant index
// formed by packed f32x2 instructions (every lane rounds as a scalar step
// would), then one byte permute whose selector takes byte 0 or 1 of the
// first entry word and byte 4 or 5 (bytes 0, 1 of the second) by the signs
// of the two tests.  The pair works with
// -mn (a max of negated magnitudes), so that no packed operand needs a
// negation: t' = -t, the inner term -(A + B t) = B t' - A, and the guess
// t' (B t' - A) = t (A + B t); the tests are h' = mx tan - mn = -h
// (round-to-nearest is symmetric, so |h'| = |h| >= 2^-40 and
// sat(2^40 h') = [h < 0]).  The selector is formed in the low bits of
// 2^23 + 0x40 + [ha < 0] + 16 [hb < 0] (the byte permute reads only the low
// 16 bits of its selector).  The tests and the selector stay scalar: a
// packed test needs the two entries' tangents moved into a register pair,
// and a selector from one packed round-up fma puts two dependent adds after
// it; both measured slower.
__device__ __forceinline__ uint32_t phase_pair2(float2 gx, float2 gy, const PhaseEntry* lut) {
    const float2 mx = make_float2(max_abs_1(gx.x, gy.x), max_abs_1(gx.y, gy.y));
    const float2 nmn = make_float2(fmaxf(-fabsf(gx.x), -fabsf(gy.x)),
                                   fmaxf(-fabsf(gx.y), -fabsf(gy.y)));
    const float2 t = __fmul2_rn(nmn, make_float2(rcp_approx(mx.x), rcp_approx(mx.y)));
    const float2 in = __ffma2_rn(t, make_float2(kPhaseGuessB, kPhaseGuessB),
                                 make_float2(-kPhaseGuessA, -kPhaseGuessA));
    float2 y = __ffma2_rd(t, in, make_float2(12582913.0f, 12582913.0f));  // 1.5*2^23 + 1
    // octant o = 4 [gx < 0] + 2 [gy < 0] + [|gy| > |gx|], then + 34 o
    const float2 two = make_float2(2.0f, 2.0f);
    float2 o = __ffma2_rn(make_float2(__saturatef(-gx.x), __saturatef(-gx.y)), two,
                          make_float2(__saturatef(-gy.x), __saturatef(-gy.y)));
    o = __ffma2_rn(o, two, make_float2(__saturatef(fabsf(gy.x) - fabsf(gx.x)),
                                       __saturatef(fabsf(gy.y) - fabsf(gx.y))));
    y = __ffma2_rn(o, make_float2(34.0f, 34.0f), y);
    const PhaseEntry ea = lut[__float_as_int(y.x) - 0x4B400000];
    const PhaseEntry eb = lut[__float_as_int(y.y) - 0x4B400000];
    const float na = __saturatef(fmaf(mx.x, ea.tan, nmn.x) * 1099511627776.0f);
    const float nb = __saturatef(fmaf(mx.y, eb.tan, nmn.y) * 1099511627776.0f);
    const float sel = fmaf(nb, 16.0f, na + 8388672.0f);  // 2^23 + 0x40
    return __byte_perm(ea.q, eb.q, __float_as_uint(sel));
}

// One pixel's Phase byte (the general output path): the pair routine with
// the pixel in both lanes, so that every Phase byte of the edge kernel comes
// from phase_pair2.
__device__ __forceinline__ uint32_t phase_from_float(float gx, float gy, const PhaseEntry* lut) {
    return phase_pair2(make_float2(gx, gx), make_float2(gy, gy), lut) & 0xFFu;
}

__device__ __forceinline__ void store8_u8(uint8_t* row, int x, int W, const uint32_t* b) {
    if (x + 8 <= W) {
        *reinterpret_cast<uint2*>(row + x) =
            make_uint2(pack4(b[0], b[1], b[2], b[3]), pack4(b[4], b[5], b[6], b[7]));
    } else {
        for (int j = 0; j < 8 && x + j < W; ++j) row[x + j] = (uint8_t)b[j];
    }
}

__device__ __forceinline__ bool tile_is_interior(const EdgeParams& p, int x0, int y0,
                                                 int th = TH) {
    return x0 >= 2 && y0 >= 2 && x0 + TW + 2 <= (int)p.W && y0 + th + 2 <= (int)p.H;
}

// ---- input box border ------------------------------------------------------------

// Both borders REPLICATE: every tile runs the plain row loop (see
// fix_input_border).
__device__ __forceinline__ bool rep2_borders(const EdgeParams& p) {
    return p.border_g == HVX_BORDER_REPLICATE && p.border_s == HVX_BORDER_REPLICATE;
}

// Whether every G row of a tile is the plain one of its (border-filled) box,
// so that the tile runs the unrolled loop: interior tiles; every tile when
// both borders replicate (fix_input_border); and every tile without a
// Gaussian node whose Sobel border is REPLICATE or CONSTANT (the box then
// holds exactly the values the Sobel reads).
__device__ __forceinline__ bool plain_g_rows(const EdgeParams& p, bool interior) {
    return interior || rep2_borders(p) || (p.g_op == 1 && p.border_s != HVX_BORDER_UNDEFINED);
}

// Box cells outside the image that a G value inside the image, or the plain
// G of the row / column just outside it, reads: the two rows above and below
// the image and the two columns left and right of it.  They take the
// Gaussian's border mode (CONSTANT: the constant; REPLICATE: the nearest
// pixel).  When the Sobel replicates too (rep2), the second cell repeats the
// pixel one further in (-2 -> 1, W + 1 -> W - 2): the plain Gaussian of row
// (column) -1 then equals the Gaussian of row (column) 0, which is exactly
// the value Sobel REPLICATE reads there, and the same at the far edges, so
// no G row or lane needs a fix.  Cells further out are never read for a
// stored output.  lh: box rows the TMA filled (LH, or 8R + 4 in the
// single-image kernel).  Reads only cells inside the image, writes only
// cells outside it, so threads never race.
__device__ void fix_input_border(Box& in, const EdgeParams& p, int x0, int y0, int lh = LH) {
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    const int W = p.W, H = p.H, bx = x0 - 16, by = y0 - 2;
    const bool cst = p.border_g == HVX_BORDER_CONSTANT;
    const bool rep2 = rep2_borders(p);
    const uint8_t cv = (uint8_t)p.cval_g;
    auto src = [&](int v, int n) {  // source coordinate of v in [-2, n + 1]
        if (v >= 0 && v < n) return v;
        if (v < 0) return (rep2 && v == -2) ? min(1, n - 1) : 0;
        return (rep2 && v == n + 1) ? max(n - 2, 0) : n - 1;
    };
    auto put = [&](int r, int c) {
        in[r][c] = cst ? cv : in[src(by + r, H) - by][src(bx + c, W) - bx];
    };
    // rows -2, -1, H, H + 1 that the box holds, every column
    for (int k = threadIdx.x; k < 4 * LW; k += blockDim.x) {
        const int j = k / LW, c = k - j * LW;
        const int r = (j < 2 ? j - 2 : H + j - 2) - by;
        if (r >= 0 && r < lh) put(r, c);
    }
    // columns -2, -1, W, W + 1 of the box rows inside the image
    for (int k = threadIdx.x; k < 4 * lh; k += blockDim.x) {
        const int r = k >> 2, j = k & 3;
        const int c = (j < 2 ? j - 2 : W + j - 2) - bx;
        if (by + r >= 0 && by + r < H && c >= 0 && c < LW) put(r, c);
    }
}

// The cells of fix_input_border in box rows r0 .. r1 - 1 (every column the
// strips read, 12 .. 147), for the batch kernel, whose warps run ahead of
// each other without a block barrier: each warp fixes the rows its two row
// groups read, its lanes striding over the cells, then syncs.  Windows of
// neighbouring warps overlap in their halo rows; both write the same values,
// each taken from a cell inside the image (which no thread writes).
__device__ void fix_input_border_warp(Box& in, const EdgeParams& p, int x0, int y0, int r0,
                                      int r1) {
    if (p.border_g == HVX_BORDER_UNDEFINED) return;
    const int W = p.W, H = p.H, bx = x0 - 16, by = y0 - 2;
    const bool cst = p.border_g == HVX_BORDER_CONSTANT;
    const bool rep2 = rep2_borders(p);
    const uint8_t cv = (uint8_t)p.cval_g;
    const int lane = threadIdx.x & 31;
    auto src = [&](int v, int n) {  // source coordinate of v in [-2, n + 1]
        if (v >= 0 && v < n) return v;
        if (v < 0) return (rep2 && v == -2) ? min(1, n - 1) : 0;
        return (rep2 && v == n + 1) ? max(n - 2, 0) : n - 1;
    };
    auto put = [&](int r, int cc) {
        in[r][cc] = cst ? cv : in[src(by + r, H) - by][src(bx + cc, W) - bx];
    };
    constexpr int C0 = 12, NC = 136;  // columns 12 .. 147
    // rows -2, -1, H, H + 1 among r0 .. r1 - 1: every column
    for (int j = 0; j < 4; ++j) {
        const int r = (j < 2 ? j - 2 : H + j - 2) - by;
        if (r >= r0 && r < r1)
            for (int cc = C0 + lane; cc < C0 + NC; cc += 32) put(r, cc);
    }
    // columns -2, -1, W, W + 1: the rows inside the image
    const int ra = max(r0, -by), rb = min(r1, H - by);
    for (int j = 0; j < 4; ++j) {
        const int cc = (j < 2 ? j - 2 : W + j - 2) - bx;
        if (cc >= C0 && cc < C0 + NC)
            for (int r = ra + lane; r < rb; r += 32) put(r, cc);
    }
    __syncwarp();
}

// ---- Gaussian rows ---------------------------------------------------------------

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

// 16 G at x - 1 .. x + 8 of one row from the pair words of the input rows
// above (a), at (b) and below (c): word j holds (x - 1 + 2j, x + 2j) in
// 16-bit lanes.  Lane sums stay below 16 * 255 + 8 < 2^12, so lanes never
// carry; clearing the low four bits of a lane leaves 16 floor(sum / 16).
__device__ __forceinline__ void g_row(const uint32_t* a, const uint32_t* b, const uint32_t* c,
                                      uint32_t rnd, uint32_t* G) {
    uint32_t V[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) V[k] = a[k] + 2u * b[k] + c[k];
#pragma unroll
    for (int j = 0; j < 5; ++j)
        G[j] = (V[j] + V[j + 1] + rnd + 2u * shift_pair(V[j], V[j + 1])) & 0xFFF0FFF0u;
}

// The input row b itself in place of a Gaussian row (no Gaussian node): the
// pixels x - 1 .. x + 8 as pairs (x - 1 + 2j, x + 2j), times 16 like the
// Gaussian lanes (at most 4080, so lanes never carry).  When the box cells
// outside the image hold the Sobel's border values, these rows are exactly
// what the Sobel reads, on every tile.
__device__ __forceinline__ void input_row16(const uint32_t* b, uint32_t* G) {
#pragma unroll
    for (int j = 0; j < 5; ++j) G[j] = shift_pair(b[j], b[j + 1]) << 4;
}

// G row yq (x - 1 .. x + 8, as 16 G) as the Sobel reads it, for a strip whose window
// leaves the Gaussian's valid region: outside the image the Sobel's border
// mode (REPLICATE: the Gaussian output at the clamped position; CONSTANT: the
// constant; UNDEFINED: 0, read by no valid output), inside the image but
// outside the valid region 0, else the Gaussian of the border-fixed box.
// The result goes to the thread's slot G in shared memory (the caller copies
// it into registers), so the call needs no local-memory array.
__device__ __noinline__ void g_row_edge(const Box& in, const EdgeParams& p, int x, int x0, int y0,
                                        int yq, uint32_t rnd, uint32_t* G) {
    const int W = p.W, H = p.H;
    const uint32_t cv = 16u * (uint32_t)(p.cval_s & 0xFF);
    int yy = yq;
    if (yy < 0 || yy >= H) {
        if (p.border_s != HVX_BORDER_REPLICATE) {
            const uint32_t v = p.border_s == HVX_BORDER_CONSTANT ? cv * 0x00010001u : 0u;
            for (int j = 0; j < 5; ++j) G[j] = v;
            return;
        }
        yy = clampi(yy, 0, H - 1);
    }
    const bool row_ok = yy >= p.gvalid[1] && yy < p.gvalid[3];
    const uint8_t* r0 = in[yy - y0 + 1];  // image rows yy - 1, yy, yy + 1
    const uint8_t* r1 = in[yy - y0 + 2];
    const uint8_t* r2 = in[yy - y0 + 3];
    uint32_t g[10];
    for (int l = 0; l < 10; ++l) {
        int xs = x - 1 + l;
        if (xs < 0 || xs >= W) {
            if (p.border_s != HVX_BORDER_REPLICATE) {
                g[l] = p.border_s == HVX_BORDER_CONSTANT ? cv : 0u;
                continue;
            }
            xs = clampi(xs, 0, W - 1);
        }
        if (!row_ok || xs < p.gvalid[0] || xs >= p.gvalid[2]) {
            g[l] = 0;
            continue;
        }
        const int c = xs - x0 + 16;
        const uint32_t s = (r0[c - 1] + 2u * r0[c] + r0[c + 1]) +
                           2u * (r1[c - 1] + 2u * r1[c] + r1[c + 1]) +
                           (r2[c - 1] + 2u * r2[c] + r2[c + 1]) + (rnd & 0xFFFFu);
        g[l] = s & ~15u;
    }
    for (int j = 0; j < 5; ++j) G[j] = g[2 * j] | (g[2 * j + 1] << 16);
}

// How a strip forms its G rows (fixed for a tile).  When the Sobel's border is
// UNDEFINED no valid output reads G outside the Gaussian's valid region, so
// every row is formed the fast way.  Otherwise rows outside the valid rows
// take the scalar path, and so do rows of strips whose columns leave the valid
// columns -- except when the valid region is the whole image: then only lanes
// outside the image differ, and they are patched in registers.
struct GPolicy {
    int gv1, gv3;      // valid rows of G
    bool sobel_undef;
    int colmode;       // 0: no column fix, 1: patch lanes outside the image, 2: scalar path
    bool rep;          // Sobel border REPLICATE (else CONSTANT)
    bool left;         // x == 0: lane 0 (x - 1) is outside the image
    int L;             // lanes 0 .. L - 1 are inside the image
    uint32_t cv;       // Sobel border constant, times 16
};

__device__ __forceinline__ void patch_cols(const GPolicy& gp, uint32_t* G) {
    if (gp.left) G[0] = (G[0] & 0xFFFF0000u) | (gp.rep ? (G[0] >> 16) : gp.cv);
    if (gp.L < 10) {
        uint32_t v = gp.cv;
        if (gp.rep) {  // the last lane inside the image
            const int k = gp.L - 1;
            uint32_t w = G[0];
#pragma unroll
            for (int j = 1; j < 5; ++j) w = (k >> 1) == j ? G[j] : w;
            v = (k & 1) ? (w >> 16) : (w & 0xFFFFu);
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            if (2 * j >= gp.L)
                G[j] = v * 0x00010001u;
            else if (2 * j + 1 >= gp.L)
                G[j] = (G[j] & 0xFFFFu) | (v << 16);
        }
    }
}

// G row yg from the input pair rows a, b, c (the rows yg - 1, yg, yg + 1).
__device__ __forceinline__ void g_row_any(const GPolicy& gp, const Box& in, const EdgeParams& p,
                                          int x, int x0, int y0, int yg, uint32_t rnd,
                                          uint32_t* gslow, const uint32_t* a, const uint32_t* b,
                                          const uint32_t* c, uint32_t* G) {
    const bool row_slow = !gp.sobel_undef && (yg < gp.gv1 || yg >= gp.gv3);
    if (!row_slow && gp.colmode < 2) {
        g_row(a, b, c, rnd, G);
        if (gp.colmode == 1) patch_cols(gp, G);
    } else {
        g_row_edge(in, p, x, x0, y0, yg, rnd, gslow);
#pragma unroll
        for (int j = 0; j < 5; ++j) G[j] = gslow[j];
    }
}

// ---- Sobel + point operators of one output row --------------------------------------

// gx, gy at x .. x + 7 from the 16 G rows above (a), at (b) and below (c),
// as pairs (x + 2j, x + 2j + 1).  Lanes: vs <= 16320, dy = c - a + 4096 in
// [16, 8176]; 16 gx + 16384 and 16 gy + 16384 are in [64, 32704].  A lane
// spliced under the exponent of 2^19 is 2^19 + lane / 16 (the mantissa's
// unit there is 1/16), and one packed add takes out the common offset,
// exactly.
__device__ __forceinline__ void sobel8(const uint32_t* a, const uint32_t* b, const uint32_t* c,
                                       float2* gx, float2* gy) {
    uint32_t vs[5], dy[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        vs[j] = a[j] + 2u * b[j] + c[j];
        dy[j] = c[j] + 0x10001000u - a[j];
    }
    const float2 off = make_float2(-(524288.0f + 1024.0f), -(524288.0f + 1024.0f));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t gxp = vs[j + 1] + 0x40004000u - vs[j];
        const uint32_t gyp = dy[j] + dy[j + 1] + 2u * shift_pair(dy[j], dy[j + 1]);
        gx[j] = __fadd2_rn(make_float2(__int_as_float(__byte_perm(gxp, 0x4900u, 0x5410)),
                                       __int_as_float(__byte_perm(gxp, 0x4900u, 0x5432))),
                           off);
        gy[j] = __fadd2_rn(make_float2(__int_as_float(__byte_perm(gyp, 0x4900u, 0x5410)),
                                       __int_as_float(__byte_perm(gyp, 0x4900u, 0x5432))),
                           off);
    }
}

// Per-thread view of a tile's parameters, held in registers.
struct RowCtx {
    const PhaseEntry* plut;
    uint32_t* gslow;    // this thread's slow-path slot in shared memory
    uint8_t* mask;
    uint8_t* phase;
    size_t mask_pitch, phase_pitch;
    float nthr;         // -(min(s_thr, 2^22) + 1/2): gx^2 + gy^2 + nthr > 0 <=> mask true
    uint32_t fx, tvx;   // mask bytes: (c & fx) ^ tvx from all-ones (false) / zero (true)
    int W, x;
    bool full;          // every output of the strip is inside its valid region
    bool fast;          // whole 8-byte stores: a fast tile and the strip inside the image
};

__device__ __forceinline__ void store8_words(uint8_t* row, int x, int W, uint32_t lo, uint32_t hi) {
    if (x + 8 <= W) {
        *reinterpret_cast<uint2*>(row + x) = make_uint2(lo, hi);
    } else {
        for (int j = 0; j < 8 && x + j < W; ++j)
            row[x + j] = (uint8_t)((j < 4 ? lo : hi) >> (8 * (j & 3)));
    }
}

// gx^2 + gy^2 + nthr for a pixel pair: every term is an integer or a half
// below 2^23, so the packed fmas are exact and the value is never 0; it is
// negative exactly when the mask is false.
__device__ __forceinline__ float2 mask_value2(float2 gx, float2 gy, float nthr) {
    return __ffma2_rn(gx, gx, __ffma2_rn(gy, gy, make_float2(nthr, nthr)));
}

// Bytes 0 and 1: the sign bits of a and b replicated over a byte (prmt with
// the sign flag of selector nibbles 0xB and 0xF; __byte_perm ignores that flag).
__device__ __forceinline__ uint32_t sign_bytes2(float a, float b) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, 0xFB;" : "=r"(r) : "r"(__float_as_uint(a)), "r"(__float_as_uint(b)));
    return r;
}

// Mask bytes of four pixels from the sign bits of their values: 0xFF where
// the mask is false, then true / false values applied.
__device__ __forceinline__ uint32_t mask4(const RowCtx& cx, float2 a, float2 b) {
    return (__byte_perm(sign_bytes2(a.x, a.y), sign_bytes2(b.x, b.y), 0x5410) & cx.fx) ^ cx.tvx;
}

__device__ __forceinline__ void point_row_general(const RowCtx& cx, const EdgeParams& p,
                                                  const float2* gx2, const float2* gy2, int y);

template <int MODE>
__device__ __forceinline__ void point_row(const RowCtx& cx, const EdgeParams& p, const float2* gx2,
                                          const float2* gy2, int y) {
    constexpr bool kMask =
        MODE == M_MASK_PHASE || MODE == M_MASK || MODE == M_MASK_YY || MODE == M_SOBEL_MASK;
    constexpr bool kPhase = MODE == M_MASK_PHASE || MODE == M_PHASE;
    const int x = cx.x;
    if constexpr (MODE != M_GENERAL) {
        uint32_t mw[2] = {0u, 0u}, pw[2] = {0u, 0u};
        if (kMask) {
            float2 mv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                mv[j] = mask_value2(MODE == M_MASK_YY ? gy2[j] : gx2[j], gy2[j], cx.nthr);
            mw[0] = mask4(cx, mv[0], mv[1]);
            mw[1] = mask4(cx, mv[2], mv[3]);
        }
        if (kPhase) {
            uint32_t pp[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                pp[j] = phase_pair2(gx2[j], gy2[j], cx.plut);
            pw[0] = __byte_perm(pp[0], pp[1], 0x5410);
            pw[1] = __byte_perm(pp[2], pp[3], 0x5410);
        }
        if (cx.fast) {
            if (kMask)
                *reinterpret_cast<uint2*>(cx.mask + (size_t)y * cx.mask_pitch + x) =
                    make_uint2(mw[0], mw[1]);
            if (kPhase)
                *reinterpret_cast<uint2*>(cx.phase + (size_t)y * cx.phase_pitch + x) =
                    make_uint2(pw[0], pw[1]);
            return;
        }
        if (!cx.full) {  // zero outside the valid region, byte by byte
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (!in_rect(p.valid, x + i, y)) {
                    const uint32_t keep = ~(0xFFu << (8 * (i & 3)));
                    mw[i >> 2] &= keep;
                    pw[i >> 2] &= keep;
                }
        }
        if (kMask) store8_words(cx.mask + (size_t)y * cx.mask_pitch, x, cx.W, mw[0], mw[1]);
        if (kPhase) store8_words(cx.phase + (size_t)y * cx.phase_pitch, x, cx.W, pw[0], pw[1]);
    } else {
        point_row_general(cx, p, gx2, gy2, y);
    }
}

// Any outputs: magnitude export, range threshold, mask and / or phase.
__device__ __forceinline__ void point_row_general(const RowCtx& cx, const EdgeParams& p,
                                                  const float2* gx2, const float2* gy2, int y) {
    const int x = cx.x;
    uint32_t mk[8], ph[8];
    int mg[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float gx = (i & 1) ? gx2[i >> 1].y : gx2[i >> 1].x;
        const float gy = (i & 1) ? gy2[i >> 1].y : gy2[i >> 1].x;
        const int ix = (int)gx, iy = (int)gy;
        mg[i] = magnitude_s16(ix, iy);
        mk[i] = 0u;
        if (cx.mask) {
            bool t;
            if (!p.thr_general)
                t = ix * ix + iy * iy > p.s_thr;
            else
                t = p.thr_type == HVX_THRESHOLD_BINARY ? mg[i] > p.thr_lo
                                                       : !(mg[i] > p.thr_hi || mg[i] < p.thr_lo);
            mk[i] = (uint32_t)(t ? p.tv : p.fv) & 0xFFu;
        }
        ph[i] = cx.phase ? phase_from_float(gx, gy, cx.plut) : 0u;
        if (!cx.full && !in_rect(p.valid, x + i, y)) {
            mk[i] = 0u;
            ph[i] = 0u;
            mg[i] = 0;
        }
    }
    if (cx.mask) store8_u8(cx.mask + (size_t)y * cx.mask_pitch, x, cx.W, mk);
    if (cx.phase) store8_u8(cx.phase + (size_t)y * cx.phase_pitch, x, cx.W, ph);
    if (p.mag) {
        int16_t* row = reinterpret_cast<int16_t*>(reinterpret_cast<uint8_t*>(p.mag) +
                                                  (size_t)y * p.mag_pitch);
        if (x + 8 <= cx.W) {
            *reinterpret_cast<uint4*>(row + x) =
                make_uint4((mg[0] & 0xFFFF) | ((uint32_t)mg[1] << 16),
                           (mg[2] & 0xFFFF) | ((uint32_t)mg[3] << 16),
                           (mg[4] & 0xFFFF) | ((uint32_t)mg[5] << 16),
                           (mg[6] & 0xFFFF) | ((uint32_t)mg[7] << 16));
        } else {
            for (int j = 0; j < 8 && x + j < cx.W; ++j) row[x + j] = (int16_t)mg[j];
        }
    }
}

// ---- one tile ------------------------------------------------------------------------

// gx of a pixel pair as two's-complement S16 lanes from its (16 gx + 16384)
// lanes: (lane >> 4) - 1024 in each lane, without a borrow between lanes
// (the top bit of each lane is set before the subtraction and flipped after).
__device__ __forceinline__ uint32_t gx_s16_pair(uint32_t gxp) {
    return ((((gxp >> 4) & 0x0FFF0FFFu) | 0x80008000u) - 0x04000400u) ^ 0x80008000u;
}

// Store of a gx strip row that is cut by the right image edge or crosses the
// valid region.
__device__ __noinline__ void store_gx_edge(int16_t* row, int x, int y, const EdgeParams& p,
                                           const uint32_t* w, bool full) {
    for (int j = 0; j < 8 && x + j < (int)p.W; ++j) {
        int16_t v = (int16_t)(w[j >> 1] >> (16 * (j & 1)));
        if (!full && !in_rect(p.valid, x + j, y)) v = 0;
        row[x + j] = v;
    }
}

// The Sobel's gx at x .. x + 7 of row y from the rows above (a), at (b) and
// below (c), stored as S16 (one 16-byte store on whole strips).
__device__ __forceinline__ void sobel_gx_row(const RowCtx& cx, const EdgeParams& p,
                                             const uint32_t* a, const uint32_t* b,
                                             const uint32_t* c, int y) {
    uint32_t vs[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) vs[j] = a[j] + 2u * b[j] + c[j];
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = gx_s16_pair(vs[j + 1] + 0x40004000u - vs[j]);
    int16_t* row = reinterpret_cast<int16_t*>(reinterpret_cast<uint8_t*>(p.mag) +
                                              (size_t)y * p.mag_pitch);
    if (cx.fast)
        *reinterpret_cast<uint4*>(row + cx.x) = make_uint4(w[0], w[1], w[2], w[3]);
    else
        store_gx_edge(row, cx.x, y, p, w, cx.full);
}

// One output row y of the strip: load input row y + 2 into Pn, form G row y + 1
// into Gc from (Pa, Pb, Pn), then Sobel over (Ga, Gb, Gc) and the point ops.
// FAST: the plain G row (no border fix-ups) and whole stores where the strip
// lies inside the image.
template <int MODE, bool FAST>
__device__ __forceinline__ void edge_row(const RowCtx& cx, const GPolicy& gp, const EdgeParams& p,
                                         const Box& in, const uint8_t* in_row, int c, int x0,
                                         int y0, uint32_t rnd, const uint32_t* Pa,
                                         const uint32_t* Pb, uint32_t* Pn, const uint32_t* Ga,
                                         const uint32_t* Gb, uint32_t* Gc, int y) {
    load_pairs(in_row, c, Pn);
    if constexpr (MODE == M_SOBEL_MASK || MODE == M_SOBEL_GX)
        input_row16(Pb, Gc);
    else if (FAST)
        g_row(Pa, Pb, Pn, rnd, Gc);
    else
        g_row_any(gp, in, p, cx.x, x0, y0, y + 1, rnd, cx.gslow, Pa, Pb, Pn, Gc);
    if constexpr (MODE == M_SOBEL_GX) {
        sobel_gx_row(cx, p, Ga, Gb, Gc, y);
    } else {
        float2 gx[4], gy[4];
        sobel8(Ga, Gb, Gc, gx, gy);
        point_row<MODE>(cx, p, gx, gy, y);
    }
}

// One tile after its box has landed (and, on edge tiles, been border-fixed):
// 128 x 8 rows output pixels, `rows` per thread.  `fast`: every G row of the
// tile is the plain Gaussian of the box and every output is valid -- interior
// tiles, and every tile when both borders replicate (fix_input_border).  Those
// run the row loop unrolled three times (the sliding windows rotate by
// renaming); the others run the general loop, one row per trip with the
// windows moved, which keeps the code small.
template <int MODE>
__device__ __forceinline__ void edge_tile(const Box& in, const EdgeParams& p, int x0, int y0,
                                          bool fast, const PhaseEntry* plut,
                                          uint32_t (*gslow)[5], int rows = ROWS) {
    const int q = threadIdx.x & 15, gi = threadIdx.x >> 4;
    const int W = p.W, H = p.H;
    const int x = x0 + 8 * q, yb = y0 + rows * gi;
    if (x >= W || yb >= H) return;
    RowCtx cx;
    cx.plut = plut;
    cx.gslow = gslow[threadIdx.x];
    cx.mask = p.mask;
    cx.phase = p.phase;
    cx.mask_pitch = p.mask_pitch;
    cx.phase_pitch = p.phase_pitch;
    cx.nthr = -((float)min(p.s_thr, 1 << 22) + 0.5f);
    cx.fx = ((uint32_t)(p.tv ^ p.fv) & 0xFFu) * 0x01010101u;
    cx.tvx = ((uint32_t)p.tv & 0xFFu) * 0x01010101u;
    cx.W = W;
    cx.x = x;
    cx.full = fast || rect_full(p.valid, W, H);
    cx.fast = fast && x + 8 <= W;  // whole 8-byte stores
    const uint32_t rnd = p.rounding == HVX_ROUND_TO_NEAREST ? 0x00080008u : 0u;
    const int c = 16 + 8 * q;
    const uint8_t* row = &in[rows * gi][0];  // input row yb - 2
    const int n = min(rows, H - yb);
    uint32_t P0[6], P1[6], P2[6], G0[5], G1[5], G2[5];
    load_pairs(row, c, P1);           // yb - 2
    load_pairs(row + 2 * LW, c, P0);  // yb
    GPolicy gp;
    if (fast) {
        load_pairs(row + LW, c, P2);      // yb - 1
        if constexpr (MODE == M_SOBEL_MASK || MODE == M_SOBEL_GX)
            input_row16(P2, G0);          // input row yb - 1 in place of G(yb - 1)
        else
            g_row(P1, P2, P0, rnd, G0);   // G(yb - 1)
        load_pairs(row + 3 * LW, c, P1);  // yb + 1
        if constexpr (MODE == M_SOBEL_MASK || MODE == M_SOBEL_GX)
            input_row16(P0, G1);          // input row yb in place of G(yb)
        else
            g_row(P2, P0, P1, rnd, G1);   // G(yb)
        // rows: P0 = input y, P1 = input y + 1, G0 = G(y - 1), G1 = G(y); the
        // windows rotate with period 3, so three rows per trip keep them in place
        const uint8_t* r = row + 4 * LW;  // input row yb + 2
#pragma unroll 1
        for (int i = 0; i < n; i += 3) {
            edge_row<MODE, true>(cx, gp, p, in, r, c, x0, y0, rnd, P0, P1, P2, G0, G1, G2, yb + i);
            if (i + 1 >= n) break;
            edge_row<MODE, true>(cx, gp, p, in, r + LW, c, x0, y0, rnd, P1, P2, P0, G1, G2, G0,
                                 yb + i + 1);
            if (i + 2 >= n) break;
            edge_row<MODE, true>(cx, gp, p, in, r + 2 * LW, c, x0, y0, rnd, P2, P0, P1, G2, G0,
                                 G1, yb + i + 2);
            r += 3 * LW;
        }
        return;
    }
    gp.gv1 = p.gvalid[1];
    gp.gv3 = p.gvalid[3];
    gp.sobel_undef = p.border_s == HVX_BORDER_UNDEFINED;
    const bool cols_ok = x - 1 >= p.gvalid[0] && x + 8 < p.gvalid[2];
    gp.colmode = (gp.sobel_undef || cols_ok) ? 0 : rect_full(p.gvalid, W, H) ? 1 : 2;
    gp.rep = p.border_s == HVX_BORDER_REPLICATE;
    gp.left = x == 0;
    gp.L = min(10, W - x + 1);
    gp.cv = 16u * (uint32_t)(p.cval_s & 0xFF);
    load_pairs(row + LW, c, P2);  // yb - 1
    if constexpr (MODE == M_SOBEL_MASK || MODE == M_SOBEL_GX)
        input_row16(P2, G0);
    else
        g_row_any(gp, in, p, x, x0, y0, yb - 1, rnd, cx.gslow, P1, P2, P0, G0);
    load_pairs(row + 3 * LW, c, P1);  // yb + 1
    if constexpr (MODE == M_SOBEL_MASK || MODE == M_SOBEL_GX)
        input_row16(P0, G1);
    else
        g_row_any(gp, in, p, x, x0, y0, yb, rnd, cx.gslow, P2, P0, P1, G1);
    // P0 = input y, P1 = input y + 1, G0 = G(y - 1), G1 = G(y): one row per
    // trip, then the windows move up by one
    const uint8_t* r = row + 4 * LW;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        edge_row<MODE, false>(cx, gp, p, in, r, c, x0, y0, rnd, P0, P1, P2, G0, G1, G2, yb + i);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            P0[k] = P1[k];
            P1[k] = P2[k];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            G0[k] = G1[k];
            G1[k] = G2[k];
        }
        r += LW;
    }
}

// ---- kernels -------------------------------------------------------------------------

__device__ __forceinline__ void issue_box(Box& in, uint64_t* bar, const CUtensorMap* map, int x0,
                                          int y0, uint32_t bytes = BOX_BYTES) {
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_2d(&in[0][0], map, bar, x0 - 16, y0 - 2);
}

template <int MODE>
// One image: one CTA per 128 x 8R tile, R = p.rows output rows per thread
// (chosen per image size so that a single image still spreads over every SM;
// the tensor map's box is 160 x (8R + 4) bytes).
__global__ void __launch_bounds__(EDGE_THREADS)
    edge_kernel(const __grid_constant__ CUtensorMap tmap, const EdgeParams p) {
    __shared__ EdgeSmem<1> sm;
    const int rows = p.rows, th = 8 * rows;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * th;
    // a programmatic dependent launch (launch_pdl): the table is built while
    // the previous grid on the stream finishes, global memory only after it
    pdl_launch_dependents();
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        fence_barrier_init();
    }
    build_phase_lut(sm.plut);
    pdl_wait();
    __syncthreads();
    if (threadIdx.x == 0)
        issue_box(sm.in[0].b, &sm.bar[0], &tmap, x0, y0, (uint32_t)(LW * (th + 4)));
    // every thread leaves together when the (bounded) wait ran out
    if (__syncthreads_or(!mbar_wait_bounded(&sm.bar[0], 0, p.err))) return;
    const bool interior = tile_is_interior(p, x0, y0, th);
    if (!interior) {
        fix_input_border(sm.in[0].b, p, x0, y0, th + 4);
        __syncthreads();
    }
    edge_tile<MODE>(sm.in[0].b, p, x0, y0, plain_g_rows(p, interior), sm.plut, sm.gslow, rows);
}

// Thread 0: the origin of batch tile t into slot ps, then one bulk copy of
// its image's parameter block into slot ps and the TMA load of its box into
// stage s, both completing on the stage's barrier (so the issuing thread never
// waits on global memory).  `tab`: the tile tables are in shared memory.
// Tiles are 128 x 8R, boxes 160 x (8R + 4).
template <int R>
__device__ __forceinline__ void issue_tile(EdgeSmem<STAGES>& sm, const EdgeBatchDesc& d, bool tab,
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
    const int x0 = (local - ty * tiles_x) * TW, y0 = ty * 8 * R;
    sm.tx0[ps] = x0;
    sm.ty0[ps] = y0;
    tensormap_acquire(&d.maps[img]);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&sm.bar[s], (uint32_t)(LW * (8 * R + 4)) + (uint32_t)sizeof(EdgeParams));
    bulk_copy_g2s(&sm.prm[ps], &d.params[img], (uint32_t)sizeof(EdgeParams), &sm.bar[s]);
    tma_load_2d(&sm.in[s].b[0][0], &d.maps[img], &sm.bar[s], x0 - 16, y0 - 2);
}

// Persistent: CTA b takes tiles b, b + grid, b + 2 grid, ...; tile k of the
// CTA lives in box stage k mod STAGES, so the next box loads while one is
// computed.  Each tile's parameters come from shared memory.  The warps run
// ahead of each other without a block barrier in the tile loop: each waits
// for its tile's box on the stage's mbarrier, fixes the border cells its own
// rows read (edge tiles), computes, and then counts itself out of the
// stage; the last warp out of tile k issues tile k + STAGES into the stage
// (every warp is then done with tile k and with the parameter slot of tile
// k - 1 that the load reuses).  A wait that runs out (bounded, about a
// second) records the error and ends the warp's loop; after the loop thread
// 0 waits (bounded) for any load still in flight.  R: output rows per thread
// (tiles of 128 x 8R; a compile-time constant, so the row loop's bounds and
// box offsets fold; the autotuner picks one per image size class and
// launches each class with its own R).
template <int MODE, int R>
__global__ void __launch_bounds__(EDGE_THREADS) edge_batch_kernel(const EdgeBatchDesc d) {
    static_assert(R >= 3 && R <= ROWS, "box ring holds at most 8 ROWS + 4 rows");
    constexpr unsigned NWARPS = EDGE_THREADS / 32;
    __shared__ EdgeSmem<STAGES> sm;
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
    build_phase_lut(sm.plut);
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < STAGES; ++s) {
            const int t = first + s * (int)gridDim.x;
            if (t < d.total_tiles) {
                sm.last_k[s] = s;
                issue_tile<R>(sm, d, tab, s, s, t);
            }
        }
    const int r0 = 2 * R * (threadIdx.x >> 5);  // first box row of this warp's two row groups
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
        const bool interior = tile_is_interior(p, x0, y0, 8 * R);
        if (!interior) fix_input_border_warp(sm.in[s].b, p, x0, y0, r0, r0 + 2 * R + 4);
        edge_tile<MODE>(sm.in[s].b, p, x0, y0, plain_g_rows(p, interior), sm.plut, sm.gslow, R);
        // this warp is done with box s: count it out (release: its reads of
        // the box happen before the count), the last one loads the next tile
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            __threadfence_block();
            const unsigned prev = atomicAdd(&sm.released[s], 1u);
            if (prev % NWARPS == NWARPS - 1) {
                __threadfence_block();
                const int tn = t + STAGES * (int)gridDim.x;
                if (tn < d.total_tiles) {
                    sm.last_k[s] = k + STAGES;
                    issue_tile<R>(sm, d, tab, s, (k + STAGES) % (STAGES + 1), tn);
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

template <int MODE>
cudaError_t launch_mode(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s) {
    const int th = 8 * p.rows;
    dim3 grid((p.W + TW - 1) / TW, (p.H + th - 1) / th);
    return launch_pdl(edge_kernel<MODE>, grid, dim3(EDGE_THREADS), 0, s, map, p);
}

template <int MODE>
cudaError_t launch_batch_mode(const EdgeBatchDesc& d, int grid, int rows, cudaStream_t s) {
    switch (rows) {
        case 5: edge_batch_kernel<MODE, 5><<<grid, EDGE_THREADS, 0, s>>>(d); break;
        case 10: edge_batch_kernel<MODE, 10><<<grid, EDGE_THREADS, 0, s>>>(d); break;
        default: edge_batch_kernel<MODE, ROWS><<<grid, EDGE_THREADS, 0, s>>>(d); break;
    }
    return cudaGetLastError();
}

// Point operators of the fused edge kernel over every integer gradient pair
// (gx, gy) in [-gmax, gmax]^2, element i = (gy + gmax) (2 gmax + 1) + gx + gmax:
// the Phase byte through phase_pair2 (two elements per call, as the kernel
// pairs neighbouring pixels) and the mask byte (255 / 0) through
// mask_value2 / sign_bytes2 for gx^2 + gy^2 > s_thr.  Same device code and
// shared-memory table as edge_batch_kernel; a self-test, not a hot path.
__global__ void __launch_bounds__(256) edge_point_selftest_kernel(int gmax, int s_thr,
                                                                  uint8_t* phase, uint8_t* mask) {
    __shared__ PhaseEntry lut[8 * 34];
    build_phase_lut(lut);
    __syncthreads();
    const int N = 2 * gmax + 1;
    const long long n = (long long)N * N;
    const float nthr = -((float)min(s_thr, 1 << 22) + 0.5f);
    for (long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x); i < n;
         i += 2ll * gridDim.x * blockDim.x) {
        const long long j = i + 1 < n ? i + 1 : i;  // an odd count pairs the last with itself
        const float gxa = (float)(int)(i % N - gmax), gya = (float)(int)(i / N - gmax);
        const float gxb = (float)(int)(j % N - gmax), gyb = (float)(int)(j / N - gmax);
        const uint32_t pp = phase_pair2(make_float2(gxa, gxb), make_float2(gya, gyb), lut);
        const float2 mv = mask_value2(make_float2(gxa, gxb), make_float2(gya, gyb), nthr);
        const uint32_t mb = ~sign_bytes2(mv.x, mv.y);  // 0xFF where the mask is true
        phase[i] = (uint8_t)pp;
        mask[i] = (uint8_t)mb;
        if (j != i) {
            phase[j] = (uint8_t)(pp >> 8);
            mask[j] = (uint8_t)(mb >> 8);
        }
    }
}

}  // namespace

int edge_mode(const EdgeParams& p) {
    if (p.g_op == 2) return M_BINOM5;
    if (p.gout) return M_GAUSS;
    if (p.mag_yy) return M_MASK_YY;  // the planner admits only the binary mask there
    if (p.g_op == 1) return p.mask ? M_SOBEL_MASK : M_SOBEL_GX;  // likewise
    if (p.mag || p.thr_general) return M_GENERAL;
    if (p.mask && p.phase) return M_MASK_PHASE;
    if (p.mask) return M_MASK;
    return M_PHASE;
}

// Rows per thread of the single-image kernel: R = 5 (2 Gaussian halo rows per
// 5 output rows; 405 CTAs on 1920 x 1080, 1620 on 3840 x 2160), or R = 2 when
// an image has fewer 128 x 40 tiles than SMs (the most CTAs for a small
// image).  Measured per launch, back to back, on 640x480 / 1920x1080 /
// 3840x2160: R = 2 8.2 / 12.8 / 26.6 us, R = 5 12.3 / 12.3 / 24.6 us, R = 15
// 20.6 / 20.5 / 26.7 us (timer steps of 2.05 us).
int edge_single_rows(int W, int H, int num_sms) {
    const long long tiles5 = (long long)((W + TW - 1) / TW) * ((H + 39) / 40);
    return tiles5 >= (num_sms > 0 ? num_sms : 152) ? 5 : 2;
}

void edge_tile_dims(int mode, int* tw, int* th) {
    *tw = mode == M_GAUSS ? GAUSS_TW : EDGE_TW;
    *th = mode == M_GAUSS ? GAUSS_TH : EDGE_TH;
}

cudaError_t launch_edge(const CUtensorMap& map, const EdgeParams& p, cudaStream_t s) {
    switch (edge_mode(p)) {
        case M_GAUSS: return launch_gauss(map, p, s);
        case M_BINOM5: return launch_binom5(map, p, s);
        case M_MASK_PHASE: return launch_mode<M_MASK_PHASE>(map, p, s);
        case M_MASK: return launch_mode<M_MASK>(map, p, s);
        case M_PHASE: return launch_mode<M_PHASE>(map, p, s);
        case M_MASK_YY: return launch_mode<M_MASK_YY>(map, p, s);
        case M_SOBEL_MASK: return launch_mode<M_SOBEL_MASK>(map, p, s);
        case M_SOBEL_GX: return launch_mode<M_SOBEL_GX>(map, p, s);
        default: return launch_mode<M_GENERAL>(map, p, s);
    }
}

cudaError_t launch_edge_batch(const EdgeBatchDesc& d, int mode, int grid, cudaStream_t s,
                              int rows) {
    switch (mode) {
        case M_GAUSS: return launch_gauss_batch(d, grid, s);
        case M_BINOM5: return launch_binom5_batch(d, grid, rows, s);
        case M_MASK_PHASE: return launch_batch_mode<M_MASK_PHASE>(d, grid, rows, s);
        case M_MASK: return launch_batch_mode<M_MASK>(d, grid, rows, s);
        case M_PHASE: return launch_batch_mode<M_PHASE>(d, grid, rows, s);
        case M_MASK_YY: return launch_batch_mode<M_MASK_YY>(d, grid, rows, s);
        case M_SOBEL_MASK: return launch_batch_mode<M_SOBEL_MASK>(d, grid, rows, s);
        case M_SOBEL_GX: return launch_batch_mode<M_SOBEL_GX>(d, grid, rows, s);
        default: return launch_batch_mode<M_GENERAL>(d, grid, rows, s);
    }
}

cudaError_t launch_edge_point_selftest(int gmax, int s_thr, uint8_t* phase, uint8_t* mask,
                                       cudaStream_t s) {
    edge_point_selftest_kernel<<<1216, 256, 0, s>>>(gmax, s_thr, phase, mask);
    return cudaGetLastError();
}

int edge_batch_blocks_per_sm(int mode) {
    if (mode == M_GAUSS) return gauss_batch_blocks_per_sm();
    if (mode == M_BINOM5) return binom5_batch_blocks_per_sm();
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, edge_batch_kernel<M_MASK_PHASE, ROWS>,
                                                  EDGE_THREADS, 0);
    return n;
}

}  // namespace hvx
