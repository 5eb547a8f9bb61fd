// Global reductions of the image graphs (Table 2 "reduce": MeanStdDev,
// MinMaxLoc; "histogram"): per-warp combination by shuffles and the global
// combination by atomics, shared by the library's staged-tile interpreter and
// the kernels generated for fused groups (self-contained, like
// point_math.cuh).
//
// Device result blocks (zeroed / set to all ones before each launch):
//   MeanStdDev: long long S1; unsigned long long S2, N       (zeroed)
//   MinMaxLoc:  unsigned long long min_key, max_key,           (all ones)
//               min_pack, max_pack
// A key is (biased value << 32 | raster index): the atomic minimum keeps the
// smallest value and, among equal values, its first pixel in raster order.
// A pack is (biased value << 40 | count): the smallest value with the number
// of pixels taking it.  Maxima are stored as minima of 65535 - (v + 32768).
#pragma once

struct HvxMinMaxAcc {
    int minv, maxv;          // 32767 / -32768 when empty
    unsigned mini, maxi;     // raster index of the first occurrence
    unsigned minc, maxc;     // number of pixels taking the value
};

__device__ __forceinline__ void hvx_mm_init(HvxMinMaxAcc& a) {
    a.minv = 32767;
    a.maxv = -32768;
    a.mini = a.maxi = 0xFFFFFFFFu;
    a.minc = a.maxc = 0;
}

__device__ __forceinline__ void hvx_mm_add(HvxMinMaxAcc& a, int v, unsigned idx) {
    if (v < a.minv || (v == a.minv && a.minc == 0)) {
        a.minv = v;
        a.mini = idx;
        a.minc = 1;
    } else if (v == a.minv) {
        a.mini = min(a.mini, idx);
        ++a.minc;
    }
    if (v > a.maxv || (v == a.maxv && a.maxc == 0)) {
        a.maxv = v;
        a.maxi = idx;
        a.maxc = 1;
    } else if (v == a.maxv) {
        a.maxi = min(a.maxi, idx);
        ++a.maxc;
    }
}

__device__ __forceinline__ void hvx_mm_merge(HvxMinMaxAcc& a, int v, unsigned i, unsigned c,
                                             int w, unsigned j, unsigned d) {
    // (v, i, c): another minimum candidate; (w, j, d): another maximum
    if (c) {
        if (a.minc == 0 || v < a.minv) {
            a.minv = v;
            a.mini = i;
            a.minc = c;
        } else if (v == a.minv) {
            a.mini = min(a.mini, i);
            a.minc += c;
        }
    }
    if (d) {
        if (a.maxc == 0 || w > a.maxv) {
            a.maxv = w;
            a.maxi = j;
            a.maxc = d;
        } else if (w == a.maxv) {
            a.maxi = min(a.maxi, j);
            a.maxc += d;
        }
    }
}

__device__ __forceinline__ void hvx_mm_warp(HvxMinMaxAcc& a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int v = __shfl_xor_sync(0xFFFFFFFFu, a.minv, o);
        const unsigned i = __shfl_xor_sync(0xFFFFFFFFu, a.mini, o);
        const unsigned c = __shfl_xor_sync(0xFFFFFFFFu, a.minc, o);
        const int w = __shfl_xor_sync(0xFFFFFFFFu, a.maxv, o);
        const unsigned j = __shfl_xor_sync(0xFFFFFFFFu, a.maxi, o);
        const unsigned d = __shfl_xor_sync(0xFFFFFFFFu, a.maxc, o);
        hvx_mm_merge(a, v, i, c, w, j, d);
    }
}

// Keeps the smallest biased value of a (value << 40 | count) word, adding
// counts of equal values.  Lock-free: every failed exchange means another
// thread's update succeeded; the loop is still bounded.
__device__ __forceinline__ void hvx_pack_min(unsigned long long* p, unsigned bv, unsigned cnt) {
    unsigned long long old = *(volatile unsigned long long*)p;
    for (int it = 0; it < (1 << 20); ++it) {
        const unsigned ov = (unsigned)(old >> 40);
        unsigned long long nw;
        if (bv < ov)
            nw = ((unsigned long long)bv << 40) | cnt;
        else if (bv == ov)
            nw = old + cnt;
        else
            return;
        const unsigned long long seen = atomicCAS(p, old, nw);
        if (seen == old) return;
        old = seen;
    }
}

// Combines one warp's accumulator (lane 0 calls this) into the result block.
__device__ __forceinline__ void hvx_mm_commit(unsigned long long* res, const HvxMinMaxAcc& a) {
    if (a.minc) {
        const unsigned bv = (unsigned)(a.minv + 32768);
        atomicMin(res + 0, ((unsigned long long)bv << 32) | a.mini);
        hvx_pack_min(res + 2, bv, a.minc);
    }
    if (a.maxc) {
        const unsigned bv = 65535u - (unsigned)(a.maxv + 32768);
        atomicMin(res + 1, ((unsigned long long)bv << 32) | a.maxi);
        hvx_pack_min(res + 3, bv, a.maxc);
    }
}

// MeanStdDev: one warp's sums into the result block (lane 0 adds).
__device__ __forceinline__ void hvx_ms_commit(void* res, long long s1, unsigned long long s2,
                                              unsigned n) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
        s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
        n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
    }
    if ((threadIdx.x & 31) == 0 && n) {
        unsigned long long* r = (unsigned long long*)res;
        atomicAdd(r + 0, (unsigned long long)s1);  // two's complement sum
        atomicAdd(r + 1, s2);
        atomicAdd(r + 2, (unsigned long long)n);
    }
}

__device__ __forceinline__ void hvx_mm_commit_warp(void* res, HvxMinMaxAcc& a) {
    hvx_mm_warp(a);
    if ((threadIdx.x & 31) == 0) hvx_mm_commit((unsigned long long*)res, a);
}
