// Plain one-node point kernels (the unfused, one-launch-per-node form of
// Table 2 point operators) and ChannelExtract of U / V from UYVY.
//
// Each thread handles 4 consecutive pixels of one row with one vector load
// per input (4 x U8 = 4 B, 4 x S16 / UYVY = 8 B, 4 x S32 / F32 = 16 B) and
// one vector store; a warp covers 128 consecutive pixels, so every access is
// coalesced.  Pixels outside the output's valid region are written as 0.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

using namespace dev;

constexpr int PT_THREADS = 256;

__device__ __forceinline__ void load4(const PlainImg& im, int x, int y, int W, int32_t v[4]) {
    const uint8_t* row = reinterpret_cast<const uint8_t*>(im.ptr) + (size_t)y * im.pitch;
    if (x + 4 <= W) {
        switch (im.fmt) {
            case HVX_DF_U8: {
                uint32_t w = *reinterpret_cast<const uint32_t*>(row + x);
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = (w >> (8 * j)) & 0xFF;
                return;
            }
            case HVX_DF_S16: {
                uint2 w = *reinterpret_cast<const uint2*>(row + 2 * x);
                v[0] = (int16_t)(w.x & 0xFFFF);
                v[1] = (int16_t)(w.x >> 16);
                v[2] = (int16_t)(w.y & 0xFFFF);
                v[3] = (int16_t)(w.y >> 16);
                return;
            }
            case HVX_DF_UYVY: {
                uint2 w = *reinterpret_cast<const uint2*>(row + 2 * x);
                v[0] = w.x & 0xFFFF;
                v[1] = w.x >> 16;
                v[2] = w.y & 0xFFFF;
                v[3] = w.y >> 16;
                return;
            }
            default: {
                int4 w = *reinterpret_cast<const int4*>(row + 4 * x);
                v[0] = w.x;
                v[1] = w.y;
                v[2] = w.z;
                v[3] = w.w;
                return;
            }
        }
    }
    for (int j = 0; j < 4; ++j) {
        int xx = x + j;
        if (xx >= W) {
            v[j] = 0;
            continue;
        }
        switch (im.fmt) {
            case HVX_DF_U8: v[j] = row[xx]; break;
            case HVX_DF_S16: v[j] = reinterpret_cast<const int16_t*>(row)[xx]; break;
            case HVX_DF_UYVY: v[j] = reinterpret_cast<const uint16_t*>(row)[xx]; break;
            default: v[j] = reinterpret_cast<const int32_t*>(row)[xx]; break;
        }
    }
}

__device__ __forceinline__ void store4(const PlainImg& im, int x, int y, int W, const int32_t v[4]) {
    uint8_t* row = reinterpret_cast<uint8_t*>(im.ptr) + (size_t)y * im.pitch;
    if (x + 4 <= W) {
        switch (im.fmt) {
            case HVX_DF_U8:
                *reinterpret_cast<uint32_t*>(row + x) = (v[0] & 0xFF) | ((v[1] & 0xFF) << 8) |
                                                        ((v[2] & 0xFF) << 16) |
                                                        ((uint32_t)(v[3] & 0xFF) << 24);
                return;
            case HVX_DF_S16:
                *reinterpret_cast<uint2*>(row + 2 * x) =
                    make_uint2((v[0] & 0xFFFF) | ((uint32_t)v[1] << 16),
                               (v[2] & 0xFFFF) | ((uint32_t)v[3] << 16));
                return;
            default:
                *reinterpret_cast<int4*>(row + 4 * x) = make_int4(v[0], v[1], v[2], v[3]);
                return;
        }
    }
    for (int j = 0; j < 4 && x + j < W; ++j) {
        switch (im.fmt) {
            case HVX_DF_U8: row[x + j] = (uint8_t)v[j]; break;
            case HVX_DF_S16: reinterpret_cast<int16_t*>(row)[x + j] = (int16_t)v[j]; break;
            default: reinterpret_cast<int32_t*>(row)[x + j] = v[j]; break;
        }
    }
}

__global__ void __launch_bounds__(PT_THREADS) point_kernel(const PlainParams p) {
    pdl_launch_dependents();  // launched by launch_pdl
    pdl_wait();
    const int x = (blockIdx.x * PT_THREADS + threadIdx.x) * 4;
    const int y = blockIdx.y;
    const int W = p.W;
    if (x >= W) return;
    int32_t a[4], b[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0}, o[4];
    load4(p.in[0], x, y, W, a);
    if (p.n_in > 1) load4(p.in[1], x, y, W, b);
    if (p.n_in > 2) load4(p.in[2], x, y, W, c);
    const bool rowv = y >= p.valid[1] && y < p.valid[3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        bool ok = rowv && x + j >= p.valid[0] && x + j < p.valid[2];
        o[j] = ok ? eval_point(p, a[j], b[j], c[j]) : 0;
    }
    store4(p.out[0], x, y, W, o);
}

// U (i0 = 1) or V (i0 = 2) plane of a UYVY image: output pixel x is byte
// 4x (U) or 4x + 2 (V) of the input row.
__global__ void __launch_bounds__(PT_THREADS) chx_uv_kernel(const PlainParams p) {
    pdl_launch_dependents();  // launched by launch_pdl
    pdl_wait();
    const int x = blockIdx.x * PT_THREADS + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= (int)p.W) return;
    const uint8_t* row = reinterpret_cast<const uint8_t*>(p.in[0].ptr) + (size_t)y * p.in[0].pitch;
    uint32_t w = *reinterpret_cast<const uint32_t*>(row + 4 * x);
    uint8_t v = (uint8_t)(p.i0 == HVX_CHANNEL_U ? (w & 0xFF) : ((w >> 16) & 0xFF));
    reinterpret_cast<uint8_t*>(p.out[0].ptr)[(size_t)y * p.out[0].pitch + x] = v;
}

}  // namespace

cudaError_t launch_plain(const PlainParams& p, cudaStream_t s) {
    if (p.op == OP_CHX && p.i0 != HVX_CHANNEL_Y) {
        dim3 grid((p.W + PT_THREADS - 1) / PT_THREADS, p.H);
        return launch_pdl(chx_uv_kernel, grid, dim3(PT_THREADS), 0, s, p);
    }
    dim3 grid((p.W + 4 * PT_THREADS - 1) / (4 * PT_THREADS), p.H);
    return launch_pdl(point_kernel, grid, dim3(PT_THREADS), 0, s, p);
}

}  // namespace hvx
