// Self-test of the device-side failure path: a kernel waits on an mbarrier
// that nothing ever completes.  Its bounded wait (the same routine every TMA
// consumer uses) must run out, record ERR_TMA_TIMEOUT in the context's error
// word and return, leaving the context usable; the host then reports
// HVX_ERROR_TIMEOUT.  No fault, trap or unbounded spin is involved.
#include "device_common.cuh"
#include "hvx_internal.h"
#include "launchers.h"

namespace hvx {
namespace {

__global__ void bounded_wait_probe(int* err, long long limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_barrier_init();
    }
    __syncthreads();
    // no thread arrives and no copy signals the barrier
    dev::mbar_wait_bounded(&bar, 0, err, limit);
}

}  // namespace
}  // namespace hvx

using namespace hvx;

extern "C" hvx_status hvxSelfTestBoundedWait(hvx_context hc) {
    Context* ctx = reinterpret_cast<Context*>(hc);
    if (!ctx || ctx->magic != kMagicContext) return HVX_ERROR_INVALID_REFERENCE;
    if (ctx->plan_only) return HVX_ERROR_NOT_SUPPORTED;
    hvx_status st = check_device_error(ctx);  // start from a clear error word
    if (st != HVX_SUCCESS && st != HVX_ERROR_TIMEOUT) return st;
    bounded_wait_probe<<<1, 32>>>(ctx->d_error, 1ll << 24);  // ~10 ms per wait
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e);
    return check_device_error(ctx);
}

extern "C" hvx_status hvxSelfTestEdgePoint(hvx_context hc, int32_t gmax, int32_t s_thr,
                                           uint8_t* phase_out, uint8_t* mask_out) {
    Context* ctx = reinterpret_cast<Context*>(hc);
    if (!ctx || ctx->magic != kMagicContext) return HVX_ERROR_INVALID_REFERENCE;
    if (ctx->plan_only) return HVX_ERROR_NOT_SUPPORTED;
    if (gmax < 0 || gmax > 4096 || !phase_out || !mask_out) return HVX_ERROR_INVALID_PARAMETERS;
    bind_device(ctx);
    const size_t n = (size_t)(2 * gmax + 1) * (size_t)(2 * gmax + 1);
    uint8_t* d = nullptr;
    if (cudaMalloc(&d, 2 * n) != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_NO_MEMORY;
    }
    cudaError_t e = launch_edge_point_selftest(gmax, s_thr, d, d + n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(phase_out, d, n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(mask_out, d + n, n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? HVX_SUCCESS : cuda_status(e);
}
