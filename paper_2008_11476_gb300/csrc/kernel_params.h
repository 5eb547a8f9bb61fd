// Plain-old-data kernel parameter blocks, shared by the host planner and the
// CUDA kernels.  Everything here is passed by value as a kernel argument.
#pragma once

#include <cstdint>

#include "../../include/hvx.h"

namespace hvx {

// Point / local abstraction ops of the implementation graph (Section 4).
enum OpKind : int {
    OP_GAUSS = 1,
    OP_BOX,
    OP_SOBEL_X,
    OP_SOBEL_Y,
    OP_MAG,
    OP_PHASE,
    OP_THRESH,
    OP_CHX,
    OP_ADD,
    OP_SUB,
    OP_ABSDIFF,
    OP_MUL,
    OP_HARRIS,
    OP_LSUM,
    OP_CONV,
    OP_DILATE,
    OP_ERODE,
    OP_MEDIAN,
    OP_AND,
    OP_OR,
    OP_XOR,
    OP_NOT,
    OP_TOMASI,
    OP_MULTIPLY,
    // global operators (Table 2 "reduce" / "histogram"): no image output
    OP_MEANSTD,
    OP_MINMAX,
    OP_HIST,
    // EqualizeHist (histogram + point): its own two launches
    OP_EQHIST,
    OP_CONVDEPTH,  // ConvertDepth / Copy
    // user-defined operators (generated kernels only): i0 = expression index
    OP_USER_POINT,
    OP_USER_LOCAL,
};

#ifdef __CUDACC__
#define HVX_HD __host__ __device__
#else
#define HVX_HD
#endif

HVX_HD inline bool op_is_global(int kind) {
    return kind == OP_MEANSTD || kind == OP_MINMAX || kind == OP_HIST;
}

// Bytes of a global operator's device result block, and the byte every
// byte of it is set to before a launch.
HVX_HD inline unsigned long long global_result_bytes(int kind, int bins) {
    return kind == OP_MEANSTD ? 24ull : kind == OP_MINMAX ? 32ull : 4ull * (unsigned long long)bins;
}
HVX_HD inline int global_result_fill(int kind) { return kind == OP_MINMAX ? 0xFF : 0; }

// ---------------------------------------------------------------------------
// Generic staged tile executor (any fused group of point / local ops).
constexpr int GEN_MAX_BUF = 12;
constexpr int GEN_MAX_STAGE = 12;
constexpr int GEN_MAX_EXT = 6;
constexpr int GEN_MAX_COEFF = 128;
constexpr int GEN_MAX_HALO = 8;
constexpr int GEN_TW = 64;   // output tile width of the generic executor
constexpr int GEN_TH = 16;   // output tile height
constexpr int GEN_THREADS = 256;

enum GenFill : int32_t {
    FILL_NONE = 0,
    FILL_REPLICATE = 1,
    FILL_CONSTANT = 2,
    FILL_MIRROR = 3,  // external inputs only
    FILL_REPEAT = 4,  // external inputs only
};

struct GenBuf {
    int32_t halo;      // the buffer holds the output tile grown by `halo` pixels
    int32_t fill;      // how cells outside the image are filled (GenFill)
    int32_t cval;      // constant for FILL_CONSTANT (float bits when is_float)
    int32_t is_float;  // cells hold binary32 (else int32)
    int32_t smem_off;  // offset in 4-byte words
    int32_t valid[4];  // valid rectangle of the image held (x0, y0, x1, y1)
    int32_t fmt;       // HVX_DF_* of the image held
};

struct GenStage {
    int32_t op;        // OpKind
    int32_t in[3];     // buffer ids
    int32_t out;       // buffer id
    int32_t rx, ry;    // window radius of a local op
    int32_t rounding;
    int32_t i0, i1, i2, i3;
    int32_t coeff_off, shift;
    float f0, f1;      // F32 thresholds
    int64_t k0, k1;    // integer thresholds, or kn / kd of the Harris response
    void* res;         // global operators: device result block (out is -1)
};

struct GenExt {
    void* ptr;
    uint64_t pitch;
    int32_t fmt;       // HVX_DF_*
    int32_t buf;
};

// EqualizeHist: histogram of the input's valid rectangle, then the mapping
// through the normalised cumulative histogram.
struct EqHistParams {
    uint32_t W, H;
    const uint8_t* in;
    uint64_t in_pitch;
    uint8_t* out;
    uint64_t out_pitch;
    uint32_t* hist;    // 256 bins, zeroed before the first launch
    int32_t valid[4];  // the input's valid rectangle (= the output's)
};

struct GenericDesc {
    int32_t W, H;
    int32_t n_buf, n_stage, n_in, n_out;
    int32_t smem_words;
    int32_t pad;
    GenBuf buf[GEN_MAX_BUF];
    GenStage st[GEN_MAX_STAGE];
    GenExt in[GEN_MAX_EXT];
    GenExt out[GEN_MAX_EXT];
    int32_t coeff[GEN_MAX_COEFF];
};

// ---------------------------------------------------------------------------
// Fused edge group: Gaussian3x3 -> Sobel3x3 -> {Magnitude -> Threshold, Phase}.
// Tall tiles; each thread slides a 3-row window of input rows and of Gaussian
// rows down one 8-pixel column strip.
constexpr int EDGE_TW = 128;               // output tile width (bytes of U8)
constexpr int EDGE_TH = 120;               // 1080 = 9 x 120, 2160 = 18 x 120, 480 = 4 x 120
constexpr int EDGE_THREADS = 128;          // 16 column strips x 8 row groups
constexpr int EDGE_ROWS = EDGE_TH / 8;     // output rows per thread (15)
constexpr int EDGE_LOAD_W = EDGE_TW + 32;  // TMA box width: 16 B aligned both sides
constexpr int EDGE_LOAD_H = EDGE_TH + 4;   // two halo rows above and below
constexpr int EDGE_STAGES = 2;             // input boxes per persistent CTA

// Gaussian3x3 group alone (its own kernel, same parameter block): tall tiles,
// each thread slides a 3-row window down one 8-pixel column strip.
constexpr int GAUSS_TW = 128;
constexpr int GAUSS_TH = 120;              // 1080 = 9 x 120, 2160 = 18 x 120, 480 = 4 x 120
constexpr int GAUSS_THREADS = 128;         // 16 column strips x 8 row groups
constexpr int GAUSS_ROWS = GAUSS_TH / 8;   // output rows per thread (15)
constexpr int GAUSS_LOAD_W = GAUSS_TW + 32;
constexpr int GAUSS_LOAD_H = GAUSS_TH + 2;
constexpr int GAUSS_STAGES = 2;            // input boxes per persistent CTA

// Persistent batch kernels keep the per-image tile tables of batches of at
// most this many images in shared memory (larger batches search them in
// global memory).
constexpr int BATCH_SMEM_IMAGES = 256;

// 16-byte aligned and sized: the batch kernels fetch it with one bulk copy.
struct alignas(16) EdgeParams {
    uint32_t W, H;
    const uint8_t* in;
    uint64_t in_pitch;
    uint8_t* phase;    // null: not produced
    uint64_t phase_pitch;
    uint8_t* mask;     // null: not produced
    uint64_t mask_pitch;
    int16_t* mag;      // null: not exported
    uint64_t mag_pitch;
    uint8_t* gout;     // Gaussian-only group: the Gaussian image
    uint64_t gout_pitch;
    int32_t border_g, cval_g;  // how the Gaussian reads the input outside the image
    int32_t border_s, cval_s;  // how the Sobel reads the Gaussian image outside the image
    int32_t rounding;
    int32_t thr_general;       // 0: mask = gx^2 + gy^2 > s_thr; 1: threshold on magnitude
    int32_t thr_type, tv, fv;
    int32_t thr_lo, thr_hi;
    int32_t s_thr;     // mask = gx^2 + gy^2 > s_thr (clamped to int32)
    int32_t rows;      // single-image kernel: output rows per thread (2 .. EDGE_ROWS)
    int32_t mag_yy;    // 1: Magnitude(gy, gy) (the Sobel's gx dead): mask = 2 gy^2 > s_thr
    int32_t g_op;      // the local op of the group's first stage: 0 Gaussian3x3 (before the
                       // Sobel, or alone into gout); 1 none, the Sobel reads the input
                       // (the mask only, or gx alone into mag as S16); 2 a 5x5 binomial
                       // Convolve alone (into gout)
    int32_t gvalid[4];  // valid rectangle of the Gaussian image
    int32_t valid[4];   // valid rectangle of the outputs
    int* err;
};

// ---------------------------------------------------------------------------
// Fused corner group: Sobel3x3 -> gx^2, gy^2, gx*gy -> 5x5 window sums ->
// Harris or Shi-Tomasi response -> binary threshold.
constexpr int HARRIS_TW = 64;
constexpr int HARRIS_TH = 32;
constexpr int HARRIS_THREADS = 256;
constexpr int HARRIS_LOAD_W = HARRIS_TW + 32;

struct HarrisParams {
    uint32_t W, H;
    const uint8_t* in;
    uint64_t in_pitch;
    uint8_t* mask;     // null: not produced
    uint64_t mask_pitch;
    float* resp;       // null: not exported
    uint64_t resp_pitch;
    int32_t border_s, cval_s;  // how the Sobel reads the input
    int32_t border_b, cval_b;  // how the window sums read the products
    int32_t wr;                // window radius (2 for 5x5)
    int32_t tv, fv;
    int32_t rows;              // BORDER_UNDEFINED kernel: output rows per thread
    int32_t tomasi;            // 1: Shi-Tomasi response instead of Harris's
    float thr_f;               // Shi-Tomasi: mask = (binary32 response > thr_f)
    int64_t kn, kd;
    int64_t q_thr;     // mask = kd * R > q_thr, exact integer form of R_f32 > T
    int32_t pvalid[4]; // valid rectangle of gx, gy and the products
    int32_t valid[4];  // valid rectangle of the sums, response and mask
    int* err;
};

// ---------------------------------------------------------------------------
// Plain one-node kernels (the unfused per-node form).
constexpr int PLAIN_TW = 64;
constexpr int PLAIN_TH = 16;

struct PlainImg {
    void* ptr;
    uint64_t pitch;
    int32_t fmt;
    int32_t pad;
};

struct PlainParams {
    uint32_t W, H;     // output size
    int32_t op;        // OpKind (OP_SOBEL_X with n_out 2 = both derivatives)
    int32_t n_in, n_out;
    int32_t border, cval, rounding, rx, ry;
    int32_t i0, i1, i2, i3, shift;
    float f0, f1;
    int64_t k0, k1;
    PlainImg in[3];
    PlainImg out[2];
    int32_t valid[4];  // output valid rectangle
    int32_t coeff[81];
};

}  // namespace hvx
