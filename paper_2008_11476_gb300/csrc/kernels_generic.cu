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
// (REPLICATE from the nearest image cell, CONSTANT with the constant).  Group
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

struct Ctx {
    const GenericDesc& d;
    int32_t* s;
    int x0, y0;
    __device__ __forceinline__ int32_t at(int bi, int x, int y) const {
        const GenBuf& b = d.buf[bi];
        int i = x - (x0 - b.halo), j = y - (y0 - b.halo);
        return s[b.smem_off + j * buf_w(b) + i];
    }
};

__device__ int32_t eval_op(const Ctx& c, const GenStage& st, int x, int y) {
    switch (st.op) {
        case OP_GAUSS: {
            int s = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    s += (2 - dx * dx) * (2 - dy * dy) * c.at(st.in[0], x + dx, y + dy);
            return st.rounding == HVX_ROUND_TO_NEAREST ? (s + 8) >> 4 : s >> 4;
        }
        case OP_BOX: {
            int s = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) s += c.at(st.in[0], x + dx, y + dy);
            return st.rounding == HVX_ROUND_TO_NEAREST ? (s + 4) / 9 : s / 9;
        }
        case OP_SOBEL_X: {
            int s = 0;
            for (int dy = -1; dy <= 1; ++dy) {
                int w = 2 - dy * dy;
                s += w * (c.at(st.in[0], x + 1, y + dy) - c.at(st.in[0], x - 1, y + dy));
            }
            return s;
        }
        case OP_SOBEL_Y: {
            int s = 0;
            for (int dx = -1; dx <= 1; ++dx) {
                int w = 2 - dx * dx;
                s += w * (c.at(st.in[0], x + dx, y + 1) - c.at(st.in[0], x + dx, y - 1));
            }
            return s;
        }
        case OP_CONV: {
            long long s = 0;
            const int kw = 2 * st.rx + 1;
            for (int dy = -st.ry; dy <= st.ry; ++dy)
                for (int dx = -st.rx; dx <= st.rx; ++dx)
                    s += (long long)c.d.coeff[st.coeff_off + (dy + st.ry) * kw + (dx + st.rx)] *
                         c.at(st.in[0], x + dx, y + dy);
            long long q = s >> st.shift;  // arithmetic shift: floor division
            return (int32_t)(q > 32767 ? 32767 : (q < -32768 ? -32768 : q));
        }
        case OP_DILATE:
        case OP_ERODE: {
            int m = c.at(st.in[0], x - 1, y - 1);
            for (int k = 1; k < 9; ++k) {
                const int v = c.at(st.in[0], x + k % 3 - 1, y + k / 3 - 1);
                m = st.op == OP_DILATE ? max(m, v) : min(m, v);
            }
            return m;
        }
        case OP_MEDIAN: {
            int v[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] = c.at(st.in[0], x + k % 3 - 1, y + k / 3 - 1);
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
        }
        case OP_LSUM: {
            long long s = 0;
            for (int dy = -st.ry; dy <= st.ry; ++dy)
                for (int dx = -st.rx; dx <= st.rx; ++dx) s += c.at(st.in[0], x + dx, y + dy);
            return (int32_t)s;
        }
        default: {
            int32_t a = c.at(st.in[0], x, y);
            int32_t b = st.in[1] >= 0 ? c.at(st.in[1], x, y) : 0;
            int32_t cc = st.in[2] >= 0 ? c.at(st.in[2], x, y) : 0;
            return eval_point(st, a, b, cc);
        }
    }
    return 0;
}

__global__ void __launch_bounds__(GEN_THREADS) generic_kernel(const GenericDesc d) {
    extern __shared__ int32_t s[];
    const int x0 = blockIdx.x * GEN_TW, y0 = blockIdx.y * GEN_TH;
    const int W = d.W, H = d.H;
    Ctx c{d, s, x0, y0};

    // external inputs, border applied
    for (int e = 0; e < d.n_in; ++e) {
        const GenExt& ex = d.in[e];
        const GenBuf& b = d.buf[ex.buf];
        const int bw = buf_w(b), n = bw * buf_h(b);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int j = i / bw;
            int x = x0 - b.halo + (i - j * bw), y = y0 - b.halo + j;
            int32_t v;
            if (x >= 0 && x < W && y >= 0 && y < H)
                v = load_pixel(ex, x, y);
            else if (b.fill == FILL_CONSTANT)
                v = b.cval;
            else if (b.fill == FILL_REPLICATE)
                v = load_pixel(ex, clampi(x, 0, W - 1), clampi(y, 0, H - 1));
            else
                v = 0;
            s[b.smem_off + i] = v;
        }
    }
    __syncthreads();

    for (int k = 0; k < d.n_stage; ++k) {
        const GenStage& st = d.st[k];
        const GenBuf& b = d.buf[st.out];
        const int bw = buf_w(b), n = bw * buf_h(b);
        bool edge = false;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int j = i / bw;
            int x = x0 - b.halo + (i - j * bw), y = y0 - b.halo + j;
            if (x >= 0 && x < W && y >= 0 && y < H) {
                s[b.smem_off + i] = in_rect(b.valid, x, y) ? eval_op(c, st, x, y) : 0;
            } else {
                edge = true;
            }
        }
        if (__syncthreads_or(edge)) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int j = i / bw;
                int x = x0 - b.halo + (i - j * bw), y = y0 - b.halo + j;
                if (x >= 0 && x < W && y >= 0 && y < H) continue;
                int32_t v;
                if (b.fill == FILL_CONSTANT)
                    v = b.cval;
                else if (b.fill == FILL_REPLICATE)
                    v = c.at(st.out, clampi(x, 0, W - 1), clampi(y, 0, H - 1));
                else
                    v = 0;
                s[b.smem_off + i] = v;
            }
            __syncthreads();
        }
    }

    for (int e = 0; e < d.n_out; ++e) {
        const GenExt& ex = d.out[e];
        for (int i = threadIdx.x; i < GEN_TW * GEN_TH; i += blockDim.x) {
            int j = i / GEN_TW;
            int x = x0 + (i - j * GEN_TW), y = y0 + j;
            if (x < W && y < H) store_pixel(ex, x, y, c.at(ex.buf, x, y));
        }
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
    generic_kernel<<<grid, GEN_THREADS, smem, s>>>(d);
    return cudaGetLastError();
}

}  // namespace hvx
