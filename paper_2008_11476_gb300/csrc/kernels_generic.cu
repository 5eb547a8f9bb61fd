// Generic staged tile executor: runs any fused group of point and local ops
// (Section 4 abstractions) that has no dedicated kernel, and every plain
// local node when fusion is off.
//
// One CTA owns a 64 x 16 output tile.  Every image the group touches gets a
// shared-memory buffer covering the tile grown by that image's halo (the sum
// of the window radii of the in-group ops downstream of it).  External inputs
// are loaded with their border mode applied; each op then computes its buffer
// cells that lie in the image (0 outside the image's valid region), and cells
// outside the image are filled the way the op's local consumers read them
// (REPLICATE from the nearest image cell, CONSTANT with the constant; MIRROR
// and REPEAT only occur on external inputs, read at the reflected or
// periodic pixel).  Group
// outputs are written from the buffers' central 64 x 16 region.  Cells hold
// int32 (U8 / S16 / S32 / UYVY pairs) or binary32 (F32).
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

__device__ __forceinline__ int buf_w(const GenBuf& b) { return GEN_TW + 2 * b.halo; }
__device__ __forceinline__ int buf_h(const GenBuf& b) { return GEN_TH + 2 * b.halo; }

__device__ __forceinline__ int32_t load_pixel(const GenExt& e, int x, int y) {
    const uint8_t* row = reinterpret_cast<const uint8_t*>(e.ptr) + (size_t)y * e.pitch;
    switch (e.fmt) {
        case HVX_DF_U8: return row[x];
        case HVX_DF_S16: return reinterpret_cast<const int16_t*>(row)[x];
        case HVX_DF_S32: return reinterpret_cast<const int32_t*>(row)[x];
        case HVX_DF_F32: return reinterpret_cast<const int32_t*>(row)[x];
        case HVX_DF_UYVY: return reinterpret_cast<const uint16_t*>(row)[x];
    }
    return 0;
}

__device__ __forceinline__ void store_pixel(const GenExt& e, int x, int y, int32_t v) {
    uint8_t* row = reinterpret_cast<uint8_t*>(e.ptr) + (size_t)y * e.pitch;
    switch (e.fmt) {
        case HVX_DF_U8: row[x] = (uint8_t)v; break;
        case HVX_DF_S16: reinterpret_cast<int16_t*>(row)[x] = (int16_t)v; break;
        case HVX_DF_S32:
        case HVX_DF_F32: reinterpret_cast<int32_t*>(row)[x] = v; break;
    }
}

// Image coordinate read by coordinate v (extent n) under MIRROR: reflection
// about the edge with the edge pixel repeated has period 2n; under REPEAT the
// period is n.
__device__ __forceinline__ int mirror_coord(int v, int n) {
    const int p = 2 * n;
    int m = v % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}
__device__ __forceinline__ int repeat_coord(int v, int n) {
    const int m = v % n;
    return m < 0 ? m + n : m;
}

// A buffer seen from the cells of another (output) buffer: element (c, r) of
// the output buffer sits at p[r * w + c] of the input buffer (the output's
// halo never exceeds its inputs' halos).
struct View {
    const int32_t* p;
    int w;
};

__device__ __forceinline__ View view_of(const GenericDesc& d, const int32_t* s, int bi, int out_halo) {
    const GenBuf& b = d.buf[bi];
    const int w = buf_w(b), dh = b.halo - out_halo;
    return View{s + b.smem_off + dh * w + dh, w};
}

// Calls f(c, r) for every cell of a bw x bh buffer: warps take rows, lanes
// consecutive columns (conflict-free shared-memory rows, no divisions).
template <class F>
__device__ __forceinline__ void for_cells(int bw, int bh, F f) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < bh; r += nw)
        for (int c = lane; c < bw; c += 32) f(c, r);
}

// Writes one stage's buffer: every cell inside the image gets v(c, r, q0, ..)
// when it lies in the op's valid region, else 0; returns whether some cell lies
// outside the image (the caller fills those).  The op is uniform, so each
// instantiation is one tight loop.
template <class V>
__device__ __forceinline__ bool stage_cells(const GenBuf& ob, int32_t* out, int ox, int oy, int W,
                                            int H, V v) {
    const int bw = buf_w(ob), bh = buf_h(ob);
    bool edge = false;
    for_cells(bw, bh, [&](int c, int r) {
        const int x = ox + c, y = oy + r;
        if (x < 0 || x >= W || y < 0 || y >= H) {
            edge = true;
            return;
        }
        out[r * bw + c] = in_rect(ob.valid, x, y) ? v(c, r) : 0;
    });
    return edge;
}

// A global operator over the tile's cells of its input that lie in the
// image and in the input's valid rectangle: per-thread partial results,
// combined per warp and added to the result block.
__device__ void run_global(const GenericDesc& d, int32_t* s, const GenStage& st, int x0, int y0) {
    const View a = view_of(d, s, st.in[0], 0);
    const int32_t* vr = d.buf[st.in[0]].valid;
    const int W = d.W;
    long long s1 = 0;
    unsigned long long s2 = 0;
    unsigned n = 0;
    HvxMinMaxAcc mm;
    hvx_mm_init(mm);
    uint32_t* bins = reinterpret_cast<uint32_t*>(s + st.i3);
    for_cells(GEN_TW, GEN_TH, [&](int c, int r) {
        const int x = x0 + c, y = y0 + r;
        if (x >= W || y >= d.H || !in_rect(vr, x, y)) return;
        const int v = a.p[r * a.w + c];
        if (st.op == OP_MEANSTD) {
            s1 += v;
            s2 += (unsigned long long)((long long)v * v);
            ++n;
        } else if (st.op == OP_MINMAX) {
            hvx_mm_add(mm, v, (unsigned)y * (unsigned)W + (unsigned)x);
        } else if (v >= st.i1 && v < st.i1 + st.i2) {
            atomicAdd(&bins[(v - st.i1) * st.i0 / st.i2], 1u);
        }
    });
    if (st.op == OP_MEANSTD) {
        hvx_ms_commit(st.res, s1, s2, n);
    } else if (st.op == OP_MINMAX) {
        hvx_mm_commit_warp(st.res, mm);
    } else {
        __syncthreads();
        uint32_t* g = static_cast<uint32_t*>(st.res);
        for (int i = threadIdx.x; i < st.i0; i += blockDim.x)
            if (bins[i]) atomicAdd(&g[i], bins[i]);
    }
}

__device__ bool run_stage(const GenericDesc& d, int32_t* s, const GenStage& st, int x0, int y0) {
    if (op_is_global(st.op)) {
        run_global(d, s, st, x0, y0);
        return false;
    }
    const GenBuf& ob = d.buf[st.out];
    int32_t* out = s + ob.smem_off;
    const int ox = x0 - ob.halo, oy = y0 - ob.halo;
    const int W = d.W, H = d.H;
    const View a = view_of(d, s, st.in[0], ob.halo);
    switch (st.op) {
        case OP_GAUSS:
        case OP_BOX: {
            const bool gauss = st.op == OP_GAUSS, near = st.rounding == HVX_ROUND_TO_NEAREST;
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                const int32_t* q = a.p + r * a.w + c;
                const int32_t* u = q - a.w;
                const int32_t* l = q + a.w;
                if (gauss) {
                    const int t = (u[-1] + 2 * u[0] + u[1]) + 2 * (q[-1] + 2 * q[0] + q[1]) +
                                  (l[-1] + 2 * l[0] + l[1]);
                    return near ? (t + 8) >> 4 : t >> 4;
                }
                const int t = u[-1] + u[0] + u[1] + q[-1] + q[0] + q[1] + l[-1] + l[0] + l[1];
                return near ? (t + 4) / 9 : t / 9;
            });
        }
        case OP_SOBEL_X:
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                const int32_t* q = a.p + r * a.w + c;
                return (q[1 - a.w] - q[-1 - a.w]) + 2 * (q[1] - q[-1]) + (q[1 + a.w] - q[-1 + a.w]);
            });
        case OP_SOBEL_Y:
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                const int32_t* q = a.p + r * a.w + c;
                return (q[a.w - 1] - q[-a.w - 1]) + 2 * (q[a.w] - q[-a.w]) + (q[a.w + 1] - q[-a.w + 1]);
            });
        case OP_DILATE:
        case OP_ERODE: {
            const bool dil = st.op == OP_DILATE;
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                const int32_t* q = a.p + (r - 1) * a.w + c;
                int m = q[-1];
#pragma unroll
                for (int k = 1; k < 9; ++k) {
                    const int v = q[(k / 3) * a.w + k % 3 - 1];
                    m = dil ? max(m, v) : min(m, v);
                }
                return m;
            });
        }
        case OP_MEDIAN:
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                const int32_t* q = a.p + (r - 1) * a.w + c;
                int v[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = q[(k / 3) * a.w + k % 3 - 1];
                // median of nine by the exchange network of Paeth (Graphics Gems)
                auto cx = [&](int i, int j) {
                    const int lo = min(v[i], v[j]), hi = max(v[i], v[j]);
                    v[i] = lo;
                    v[j] = hi;
                };
                cx(1, 2); cx(4, 5); cx(7, 8); cx(0, 1); cx(3, 4); cx(6, 7);
                cx(1, 2); cx(4, 5); cx(7, 8); cx(0, 3); cx(5, 8); cx(4, 7);
                cx(3, 6); cx(1, 4); cx(2, 5); cx(4, 7); cx(4, 2); cx(6, 4);
                cx(4, 2);
                return v[4];
            });
        case OP_CONV:
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                long long t = 0;
                const int kw = 2 * st.rx + 1;
                const int32_t* q = a.p + (r - st.ry) * a.w + (c - st.rx);
                for (int dy = 0; dy <= 2 * st.ry; ++dy)
                    for (int dx = 0; dx < kw; ++dx)
                        t += (long long)d.coeff[st.coeff_off + dy * kw + dx] * q[dy * a.w + dx];
                const long long v = t >> st.shift;  // arithmetic shift: floor division
                if (st.i0 == HVX_DF_U8) return (int32_t)(v > 255 ? 255 : (v < 0 ? 0 : v));
                return (int32_t)(v > 32767 ? 32767 : (v < -32768 ? -32768 : v));
            });
        case OP_LSUM:
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                long long t = 0;
                const int32_t* q = a.p + (r - st.ry) * a.w + (c - st.rx);
                for (int dy = 0; dy <= 2 * st.ry; ++dy)
                    for (int dx = 0; dx <= 2 * st.rx; ++dx) t += q[dy * a.w + dx];
                return (int32_t)t;
            });
        default: {
            const View b = st.in[1] >= 0 ? view_of(d, s, st.in[1], ob.halo) : a;
            const View e = st.in[2] >= 0 ? view_of(d, s, st.in[2], ob.halo) : a;
            return stage_cells(ob, out, ox, oy, W, H, [&](int c, int r) {
                return eval_point(st, a.p[r * a.w + c], b.p[r * b.w + c], e.p[r * e.w + c]);
            });
        }
    }
}

// Value of buffer bi at image pixel (x, y) (inside the buffer).
__device__ __forceinline__ int32_t buf_at(const GenericDesc& d, const int32_t* s, int bi, int x0,
                                          int y0, int x, int y) {
    const GenBuf& b = d.buf[bi];
    return s[b.smem_off + (y - (y0 - b.halo)) * buf_w(b) + (x - (x0 - b.halo))];
}

__global__ void __launch_bounds__(GEN_THREADS) generic_kernel(const GenericDesc d) {
    pdl_launch_dependents();  // launched by launch_pdl
    pdl_wait();
    extern __shared__ int32_t s[];
    const int x0 = blockIdx.x * GEN_TW, y0 = blockIdx.y * GEN_TH;
    const int W = d.W, H = d.H;

    // the tile's histograms of global operators start empty
    for (int k = 0; k < d.n_stage; ++k)
        if (d.st[k].op == OP_HIST)
            for (int i = threadIdx.x; i < d.st[k].i0; i += blockDim.x) s[d.st[k].i3 + i] = 0;

    // external inputs, border applied
    for (int e = 0; e < d.n_in; ++e) {
        const GenExt& ex = d.in[e];
        const GenBuf& b = d.buf[ex.buf];
        const int bw = buf_w(b);
        int32_t* dst = s + b.smem_off;
        for_cells(bw, buf_h(b), [&](int c, int r) {
            const int x = x0 - b.halo + c, y = y0 - b.halo + r;
            int32_t v;
            if (x >= 0 && x < W && y >= 0 && y < H)
                v = load_pixel(ex, x, y);
            else if (b.fill == FILL_CONSTANT)
                v = b.cval;
            else if (b.fill == FILL_REPLICATE)
                v = load_pixel(ex, clampi(x, 0, W - 1), clampi(y, 0, H - 1));
            else if (b.fill == FILL_MIRROR)
                v = load_pixel(ex, mirror_coord(x, W), mirror_coord(y, H));
            else if (b.fill == FILL_REPEAT)
                v = load_pixel(ex, repeat_coord(x, W), repeat_coord(y, H));
            else
                v = 0;
            dst[r * bw + c] = v;
        });
    }
    __syncthreads();

    for (int k = 0; k < d.n_stage; ++k) {
        const GenStage& st = d.st[k];
        const bool edge = run_stage(d, s, st, x0, y0);
        if (__syncthreads_or(edge)) {
            // cells outside the image, the way the op's local consumers read them
            const GenBuf& b = d.buf[st.out];
            const int bw = buf_w(b);
            int32_t* out = s + b.smem_off;
            for_cells(bw, buf_h(b), [&](int c, int r) {
                const int x = x0 - b.halo + c, y = y0 - b.halo + r;
                if (x >= 0 && x < W && y >= 0 && y < H) return;
                int32_t v;
                if (b.fill == FILL_CONSTANT)
                    v = b.cval;
                else if (b.fill == FILL_REPLICATE)
                    v = buf_at(d, s, st.out, x0, y0, clampi(x, 0, W - 1), clampi(y, 0, H - 1));
                else
                    v = 0;
                out[r * bw + c] = v;
            });
            __syncthreads();
        }
    }

    for (int e = 0; e < d.n_out; ++e) {
        const GenExt& ex = d.out[e];
        for_cells(GEN_TW, GEN_TH, [&](int c, int r) {
            const int x = x0 + c, y = y0 + r;
            if (x < W && y < H) store_pixel(ex, x, y, buf_at(d, s, ex.buf, x0, y0, x, y));
        });
    }
}

}  // namespace

cudaError_t launch_generic(const GenericDesc& d, cudaStream_t s) {
    static int attr_bytes = 0;
    const int smem = d.smem_words * 4;
    if (smem > 48 * 1024 && smem > attr_bytes) {
        cudaError_t e =
            cudaFuncSetAttribute(generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    dim3 grid((d.W + GEN_TW - 1) / GEN_TW, (d.H + GEN_TH - 1) / GEN_TH);
    return launch_pdl(generic_kernel, grid, dim3(GEN_THREADS), (size_t)smem, s, d);
}

}  // namespace hvx
