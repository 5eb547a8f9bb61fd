// EqualizeHist (Table 2: histogram + point).  The mapping of every pixel
// needs the histogram of the whole image, so it takes two launches: a
// histogram of the input's valid rectangle (per-CTA shared-memory bins added
// to the global ones), then the mapping, where every CTA forms the 256-entry
// table from the cumulative histogram before mapping its pixels.
#include "device_common.cuh"
#include "launchers.h"

namespace hvx {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) eqhist_count_kernel(const EqHistParams p) {
    __shared__ uint32_t bins[256];
    bins[threadIdx.x] = 0;
    __syncthreads();
    const int x0 = p.valid[0], y0 = p.valid[1], w = p.valid[2] - x0, h = p.valid[3] - y0;
    // rows of the valid rectangle
    for (int y = blockIdx.x; y < h; y += gridDim.x) {
        const uint8_t* row = p.in + (size_t)(y0 + y) * p.in_pitch + x0;
        for (int x = threadIdx.x; x < w; x += kThreads) atomicAdd(&bins[row[x]], 1u);
    }
    __syncthreads();
    if (bins[threadIdx.x]) atomicAdd(&p.hist[threadIdx.x], bins[threadIdx.x]);
}

__global__ void __launch_bounds__(kThreads) eqhist_map_kernel(const EqHistParams p) {
    __shared__ uint32_t c[256];
    __shared__ uint8_t lut[256];
    c[threadIdx.x] = __ldg(p.hist + threadIdx.x);
    __syncthreads();
    // inclusive prefix sum of the 256 bins (Hillis-Steele, 8 steps)
    for (int o = 1; o < 256; o <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)o ? c[threadIdx.x - o] : 0u;
        __syncthreads();
        c[threadIdx.x] += v;
        __syncthreads();
    }
    const unsigned long long n = c[255];
    // cmin: the cumulative count at the smallest value present = the
    // smallest nonzero prefix
    __shared__ uint32_t cmin;
    if (threadIdx.x == 0) cmin = 0xFFFFFFFFu;
    __syncthreads();
    if (c[threadIdx.x]) atomicMin(&cmin, c[threadIdx.x]);
    __syncthreads();
    const unsigned long long den = n - cmin;
    const unsigned v = threadIdx.x;
    if (den == 0) {
        lut[v] = (uint8_t)v;  // constant image: unchanged
    } else {
        const unsigned long long cv = c[v] > cmin ? c[v] - cmin : 0ull;
        lut[v] = (uint8_t)((2ull * cv * 255ull + den) / (2ull * den));  // halves rounded up
    }
    __syncthreads();
    for (int y = blockIdx.x; y < (int)p.H; y += gridDim.x) {
        const uint8_t* in = p.in + (size_t)y * p.in_pitch;
        uint8_t* out = p.out + (size_t)y * p.out_pitch;
        const bool yin = y >= p.valid[1] && y < p.valid[3];
        for (int x = threadIdx.x; x < (int)p.W; x += kThreads)
            out[x] = yin && x >= p.valid[0] && x < p.valid[2] ? lut[in[x]] : 0;
    }
}

}  // namespace

cudaError_t launch_eqhist(const EqHistParams& p, cudaStream_t s) {
    const int rows = (int)p.H;
    const int grid = rows < 1 ? 1 : (rows < 2048 ? rows : 2048);
    eqhist_count_kernel<<<grid, kThreads, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    eqhist_map_kernel<<<grid, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace hvx
