// Device helpers shared by the image-graph kernels: TMA / mbarrier wrappers in
// inline PTX (sm_90+ async proxy, compiled for sm_103a), bounded waits, and
// the exact point-operator arithmetic (Magnitude, Phase, Harris response).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernel_params.h"

namespace hvx {
namespace dev {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Single-image kernels are launched with
// programmatic stream serialisation (launch_pdl): a launch may begin while
// the previous kernel on its stream is still running, so such a kernel lets
// the next launch begin (pdl_launch_dependents) and waits for the previous
// grid to complete and its memory to be visible (pdl_wait) before its first
// global-memory access.  In a launch without the attribute both are no-ops.

__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;");
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// ---------------------------------------------------------------------------
// TMA and mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Make the mbarrier initialisation visible to the async proxy (TMA).
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this CTA's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Acquire a tensor map that lives in global memory before the first TMA
// that uses it.
__device__ __forceinline__ void tensormap_acquire(const void* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 2-D tiled TMA load of box (x, y) of `map` into shared memory; completion
// is signalled on `bar` as transaction bytes.  x * element size must be a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Bulk copy (no tensor map) of `bytes` from global to shared memory,
// signalled on `bar`; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Error codes written to the context's device error word.
constexpr int ERR_TMA_TIMEOUT = 1;

// Wait for phase `parity` of `bar` for at most ~2^31 SM cycles (about a
// second).  On time-out, record the error, wait once more with the same limit
// so that a late copy does not land after the CTA has moved on, and return
// false; the caller then leaves the tile.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  long long limit = 1ll << 31) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            if (err) atomicCAS(err, 0, ERR_TMA_TIMEOUT);
            long long t1 = clock64();
            while (!mbar_try_wait(bar, parity) && clock64() - t1 < limit) {
            }
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Exact point arithmetic (Magnitude, Phase, Harris and Shi-Tomasi responses):
// a self-contained header that generated kernels include too.
#include "point_math.cuh"
#include "reduce_math.cuh"

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ bool rect_full(const int32_t* r, int W, int H) {
    return r[0] == 0 && r[1] == 0 && r[2] == W && r[3] == H;
}

__device__ __forceinline__ bool in_rect(const int32_t* r, int x, int y) {
    return x >= r[0] && x < r[2] && y >= r[1] && y < r[3];
}


// One point operator (Table 2 "point") on the values a, b, c of its inputs at
// one pixel.  P is GenStage or PlainParams; both carry op, i0..i3, f0, f1,
// k0, k1 with the meaning below.  Results are int32, or binary32 bits for F32.
//   Threshold: i0 type, i1 true value, i2 false value, i3 input is F32;
//              k0 / k1 integer lower(value) / upper, f0 / f1 binary32 ones.
//   Add / Subtract / AbsDiff: i0 saturate, i1 output format.
//   Harris response: k0 = kn, k1 = kd.
template <class P>
__device__ __forceinline__ int32_t eval_point(const P& st, int32_t a, int32_t b, int32_t c) {
    switch (st.op) {
        case OP_MAG: return magnitude_s16(a, b);
        case OP_PHASE: return (int32_t)phase_u8(a, b);
        case OP_THRESH: {
            bool t;
            if (st.i3) {
                float f = __int_as_float(a);
                t = st.i0 == HVX_THRESHOLD_BINARY ? f > st.f0 : !(f > st.f1 || f < st.f0);
            } else {
                long long iv = a;
                t = st.i0 == HVX_THRESHOLD_BINARY ? iv > st.k0 : !(iv > st.k1 || iv < st.k0);
            }
            return t ? st.i1 : st.i2;
        }
        case OP_CHX: return (a >> 8) & 0xFF;  // Y byte of a UYVY pixel pair
        case OP_ADD:
        case OP_SUB:
        case OP_ABSDIFF: {
            int r = st.op == OP_ADD ? a + b : (st.op == OP_SUB ? a - b : abs(a - b));
            if (st.i1 == HVX_DF_U8) return st.i0 ? sat_u8(r) : (r & 0xFF);
            return st.i0 ? sat_s16(r) : (int32_t)(int16_t)(uint16_t)(r & 0xFFFF);
        }
        case OP_MUL: return a * b;
        case OP_AND: return a & b;
        case OP_OR: return a | b;
        case OP_XOR: return a ^ b;
        case OP_NOT: return ~a & 0xFF;
        case OP_HARRIS:
            return __float_as_int(ratio_to_float(harris_q(a, b, c, st.k0, st.k1), st.k1));
        case OP_TOMASI: return __float_as_int(tomasi_response_f32(a, b, c));
        case OP_CONVDEPTH:
            if (st.i1 == st.i3) return a;                    // Copy
            if (st.i1 == HVX_DF_S16) return (int32_t)((uint32_t)a << st.i0);  // U8 -> S16
            return st.i2 ? sat_u8(a >> st.i0) : ((a >> st.i0) & 0xFF);    // S16 -> U8
        case OP_MULTIPLY: {
            const long long v = multiply_scaled(a, b, st.k0, st.i3, st.i2 != 0);
            if (st.i1 == HVX_DF_U8) return st.i0 ? sat64_u8(v) : (int32_t)(v & 0xFF);
            return st.i0 ? sat64_s16(v) : wrap64_s16(v);
        }
    }
    return 0;
}

// Calls f(r, c) for every cell (r, c) of an R x C box whose top-left cell is
// image pixel (bx, by) and that lies outside the W x H image: the full rows
// above and below the image, then the left / right strips of the rows in
// between, spread over the CTA's threads.
template <class F>
__device__ __forceinline__ void for_each_outside(int R, int C, int bx, int by, int W, int H, F f) {
    const int cl = clampi(-bx, 0, C), cr = max(cl, clampi(W - bx, 0, C));
    const int rt = clampi(-by, 0, R), rb = max(rt, clampi(H - by, 0, R));
    const int nfull = (rt + (R - rb)) * C;
    const int side = cl + (C - cr);
    const int n = nfull + (rb - rt) * side;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int r, c;
        if (i < nfull) {
            int rr = i / C;
            c = i - rr * C;
            r = rr < rt ? rr : rb + (rr - rt);
        } else {
            int j = i - nfull;
            int rr = j / side;
            int k = j - rr * side;
            r = rt + rr;
            c = k < cl ? k : cr + (k - cl);
        }
        f(r, c);
    }
}

// ---------------------------------------------------------------------------
// 16-bit-lane (SWAR) helpers of the U8 stencil kernels: two pixels per
// 32-bit word, so that one add or shift works on both.

// 16-bit lane pairs of bytes: (b0, b1) and (b2, b3) of a word.
__device__ __forceinline__ uint32_t lo_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4140); }
__device__ __forceinline__ uint32_t hi_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4342); }

// (lane1 of a, lane0 of b): the pair starting one pixel to the right of a.
__device__ __forceinline__ uint32_t shift_pair(uint32_t a, uint32_t b) {
    return __funnelshift_r(a, b, 16);
}

// Batch tile t -> image: the last i with tile_start[i] <= t (binary search
// over the n + 1 prefix sums of per-image tile counts), in global memory or
// in a shared-memory copy.
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
__device__ __forceinline__ int find_image_smem(const int* tile_start, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_start[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace dev
}  // namespace hvx
