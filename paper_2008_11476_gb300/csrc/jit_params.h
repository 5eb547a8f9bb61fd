// Launch parameters of the kernels generated at verify time for fused groups
// (codegen.cpp).  Self-contained plain C so that the host and the generated
// source share this one definition: everything that depends on the image
// size or on device memory is here; the group's structure and constants are
// compiled into the kernel.
#pragma once

#define HVX_JIT_MAX_BUF 12
#define HVX_JIT_MAX_EXT 6
#define HVX_JIT_MAX_RES 4

/* A CUDA tensor map (CUtensorMap: 128 bytes, 64-byte aligned) as plain data. */
typedef struct __attribute__((aligned(64))) {
    unsigned long long opaque[16];
} HvxTensorMap;

struct HvxJitParams {
    int W, H;                       // size of every image of the group
    int ix0, ix1, iy0, iy1;         // interior tiles (inclusive; none when ix0 > ix1):
                                    // every image's cells needed by the tile lie
                                    // inside that image's valid region
    int valid[HVX_JIT_MAX_BUF][4];  // valid rectangle of each image (x0, y0, x1, y1)
    void* in[HVX_JIT_MAX_EXT];      // external inputs, row-major, pitch in bytes
    unsigned long long in_pitch[HVX_JIT_MAX_EXT];
    void* out[HVX_JIT_MAX_EXT];     // external outputs
    unsigned long long out_pitch[HVX_JIT_MAX_EXT];
    void* res[HVX_JIT_MAX_RES];     // result blocks of the group's global operators
    int* err;                       // device error word (a bounded wait that ran out)
    HvxTensorMap tmap[HVX_JIT_MAX_EXT];  // U8 inputs staged by TMA: box = the staged slot
};
