/*
 * hvx_oracle.c -- CPU correctness oracle for the OpenVX-style image graph path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library; neither includes
 * the other.
 *
 * Every function is a plain, single-threaded loop over pixels that writes out
 * the definition of one node (one "CV function" of the paper's Table 2, or one
 * point / local abstraction of Section 4) with int64 / double arithmetic.
 * No blocking, no fusion, no reordering: a reader can check each loop against
 * the node's definition by eye.
 *
 * Conventions shared by every function here:
 *   - images are dense row-major arrays, row stride == width (in elements);
 *   - a "valid rectangle" vr = {x0, y0, x1, y1} (half-open) travels with every
 *     image.  A local operator under BORDER_UNDEFINED only produces pixels
 *     whose whole window lies inside its input's valid rectangle, so its
 *     output rectangle is the input's shrunk by the window radius.  A point
 *     operator's output rectangle is the intersection of its inputs'.  Every
 *     function writes 0 to each output pixel outside its output rectangle.
 *   - BORDER_REPLICATE reads the nearest pixel of the image (coordinates
 *     clamped to [0,W-1]x[0,H-1]); BORDER_CONSTANT reads a constant.  Both
 *     apply at the image edge (the paper's Hipacc listing selects clamping
 *     as its boundary condition, Section 3.2).  BORDER_MIRROR and
 *     BORDER_REPEAT are the other boundary conditions the Hipacc DSL of
 *     Section 3.2 names (MIRROR, REPEAT); the paper does not define them.
 *     Reading: MIRROR reflects a coordinate about the image edge with the
 *     edge pixel repeated (... c b a | a b c ...), again and again until it
 *     lies inside; REPEAT continues the image periodically.  Like
 *     REPLICATE, neither shrinks the valid rectangle.
 *
 * The OpenVX per-node arithmetic (saturation, rounding) is not printed in the
 * paper; the readings taken here are listed at each function.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

#define ORC_BORDER_UNDEFINED 0
#define ORC_BORDER_REPLICATE 1
#define ORC_BORDER_CONSTANT 2
#define ORC_BORDER_MIRROR 3
#define ORC_BORDER_REPEAT 4

#define ORC_ROUND_ZERO 0
#define ORC_ROUND_NEAREST 1

/* Element formats of the oracle's own numbering. */
#define ORC_U8 1
#define ORC_S16 2
#define ORC_S32 3
#define ORC_F32 4

#define ORC_OK 0
#define ORC_ERR (-1)

/* ------------------------------------------------------------------------ */
/* valid rectangles                                                           */

static void rect_copy(int dst[4], const int src[4]) {
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
}

static void rect_intersect(int dst[4], const int a[4], const int b[4]) {
    dst[0] = a[0] > b[0] ? a[0] : b[0];
    dst[1] = a[1] > b[1] ? a[1] : b[1];
    dst[2] = a[2] < b[2] ? a[2] : b[2];
    dst[3] = a[3] < b[3] ? a[3] : b[3];
    if (dst[2] < dst[0]) dst[2] = dst[0];
    if (dst[3] < dst[1]) dst[3] = dst[1];
}

/* Output rectangle of a local operator with radii (rx, ry). */
static void rect_local(int dst[4], const int src[4], int rx, int ry, int border) {
    rect_copy(dst, src);
    if (border == ORC_BORDER_UNDEFINED) {
        dst[0] += rx; dst[1] += ry; dst[2] -= rx; dst[3] -= ry;
        if (dst[2] < dst[0]) dst[2] = dst[0];
        if (dst[3] < dst[1]) dst[3] = dst[1];
    }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* The coordinate inside [0, n) that coordinate v reads under MIRROR (reflect
 * about the edge it crossed, repeating the edge sample, until inside) or
 * REPEAT (shift by the extent n until inside). */
static int wrap_coord(int v, int n, int border) {
    while (v < 0 || v >= n) {
        if (border == ORC_BORDER_REPEAT)
            v = v < 0 ? v + n : v - n;
        else
            v = v < 0 ? -v - 1 : 2 * n - 1 - v;
    }
    return v;
}

/* Read one input sample of a local operator at (x, y), which may lie outside
 * the image.  Under UNDEFINED the caller never asks for such a sample. */
static int64_t read_u8(const uint8_t* p, int w, int h, int x, int y, int border, int cval) {
    if (x >= 0 && x < w && y >= 0 && y < h) return p[(size_t)y * w + x];
    if (border == ORC_BORDER_CONSTANT) return (uint8_t)cval;
    if (border == ORC_BORDER_MIRROR || border == ORC_BORDER_REPEAT)
        return p[(size_t)wrap_coord(y, h, border) * w + wrap_coord(x, w, border)];
    return p[(size_t)clampi(y, 0, h - 1) * w + clampi(x, 0, w - 1)];
}

static int64_t read_s32(const int32_t* p, int w, int h, int x, int y, int border, int cval) {
    if (x >= 0 && x < w && y >= 0 && y < h) return p[(size_t)y * w + x];
    if (border == ORC_BORDER_CONSTANT) return cval;
    if (border == ORC_BORDER_MIRROR || border == ORC_BORDER_REPEAT)
        return p[(size_t)wrap_coord(y, h, border) * w + wrap_coord(x, w, border)];
    return p[(size_t)clampi(y, 0, h - 1) * w + clampi(x, 0, w - 1)];
}

/* ------------------------------------------------------------------------ */
/* Local operators (Table 2 "local"; Section 4)                               */

/* Gaussian3x3 (Table 2; Listing 1 applies it to the extracted luma).
 * Weights [1 2 1; 2 4 2; 1 2 1], sum 16.  Reading: the weighted integer sum
 * is divided by 16 with truncation (ORC_ROUND_ZERO, the default) or with
 * round-half-up (ORC_ROUND_NEAREST).  The result always fits U8. */
int orc_gaussian3x3(const uint8_t* in, uint8_t* out, int w, int h, int border, int cval,
                    int rounding, const int vin[4], int vout[4]) {
    static const int wt[3][3] = {{1, 2, 1}, {2, 4, 2}, {1, 2, 1}};
    int r[4];
    if (w <= 0 || h <= 0) return ORC_ERR;
    rect_local(r, vin, 1, 1, border);
    memset(out, 0, (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            int64_t s = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    s += wt[dy + 1][dx + 1] * read_u8(in, w, h, x + dx, y + dy, border, cval);
            int64_t v = rounding == ORC_ROUND_NEAREST ? (s + 8) / 16 : s / 16;
            out[(size_t)y * w + x] = (uint8_t)v;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Box3x3 (Table 2): unweighted 3x3 sum divided by 9 (truncation, or
 * round-half-up with ORC_ROUND_NEAREST). */
int orc_box3x3(const uint8_t* in, uint8_t* out, int w, int h, int border, int cval,
               int rounding, const int vin[4], int vout[4]) {
    int r[4];
    if (w <= 0 || h <= 0) return ORC_ERR;
    rect_local(r, vin, 1, 1, border);
    memset(out, 0, (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            int64_t s = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    s += read_u8(in, w, h, x + dx, y + dy, border, cval);
            int64_t v = rounding == ORC_ROUND_NEAREST ? (s + 4) / 9 : s / 9;
            out[(size_t)y * w + x] = (uint8_t)v;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Dilate3x3, Erode3x3, Median3x3 (Table 2 local operators on U8): the
 * maximum (op 0), minimum (op 1) or median (op 2) of the nine samples of the
 * 3x3 window, read under the node's border mode.  The median sorts the nine
 * values (insertion sort) and takes the fifth. */
int orc_morph3x3(const uint8_t* in, uint8_t* out, int w, int h, int border, int cval, int op,
                 const int vin[4], int vout[4]) {
    int r[4];
    if (w <= 0 || h <= 0 || op < 0 || op > 2) return ORC_ERR;
    rect_local(r, vin, 1, 1, border);
    memset(out, 0, (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            int v[9], n = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    v[n++] = (int)read_u8(in, w, h, x + dx, y + dy, border, cval);
            int res;
            if (op == 0) {
                res = v[0];
                for (int i = 1; i < 9; ++i) res = v[i] > res ? v[i] : res;
            } else if (op == 1) {
                res = v[0];
                for (int i = 1; i < 9; ++i) res = v[i] < res ? v[i] : res;
            } else {
                for (int i = 1; i < 9; ++i) {
                    int t = v[i], j = i - 1;
                    while (j >= 0 && v[j] > t) {
                        v[j + 1] = v[j];
                        --j;
                    }
                    v[j + 1] = t;
                }
                res = v[4];
            }
            out[(size_t)y * w + x] = (uint8_t)res;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Sobel3x3 (Table 2; Listing 1, and the dead-output example of Section 5.2.2).
 * gx with [-1 0 1; -2 0 2; -1 0 1], gy with [-1 -2 -1; 0 0 0; 1 2 1], no
 * scaling: |g| <= 1020 fits S16.  Either output may be NULL. */
int orc_sobel3x3(const uint8_t* in, int16_t* gx, int16_t* gy, int w, int h, int border,
                 int cval, const int vin[4], int vout[4]) {
    static const int kx[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
    static const int ky[3][3] = {{-1, -2, -1}, {0, 0, 0}, {1, 2, 1}};
    int r[4];
    if (w <= 0 || h <= 0) return ORC_ERR;
    rect_local(r, vin, 1, 1, border);
    if (gx) memset(gx, 0, sizeof(int16_t) * (size_t)w * h);
    if (gy) memset(gy, 0, sizeof(int16_t) * (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            int64_t sx = 0, sy = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t v = read_u8(in, w, h, x + dx, y + dy, border, cval);
                    sx += kx[dy + 1][dx + 1] * v;
                    sy += ky[dy + 1][dx + 1] * v;
                }
            if (gx) gx[(size_t)y * w + x] = (int16_t)sx;
            if (gy) gy[(size_t)y * w + x] = (int16_t)sy;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Custom local operator SUM (the user-defined local nodes of Section 5.1,
 * used for the 5x5 window of the Harris graph): out = sum over the kw x kh
 * window of S32 input samples, exact in int64, stored as S32.  Returns
 * ORC_ERR if a sum does not fit S32 (it cannot for the Harris products:
 * 25 * 1020^2 * 2 < 2^31). */
int orc_window_sum_s32(const int32_t* in, int32_t* out, int w, int h, int kw, int kh,
                       int border, int cval, const int vin[4], int vout[4]) {
    int r[4];
    int rx = kw / 2, ry = kh / 2;
    if (w <= 0 || h <= 0 || kw <= 0 || kh <= 0 || !(kw & 1) || !(kh & 1)) return ORC_ERR;
    rect_local(r, vin, rx, ry, border);
    memset(out, 0, sizeof(int32_t) * (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            int64_t s = 0;
            for (int dy = -ry; dy <= ry; ++dy)
                for (int dx = -rx; dx <= rx; ++dx)
                    s += read_s32(in, w, h, x + dx, y + dy, border, cval);
            if (s > INT32_MAX || s < INT32_MIN) return ORC_ERR;
            out[(size_t)y * w + x] = (int32_t)s;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Custom local operator WEIGHTED_SUM on U8 (the paper's Listing 2/3 style
 * convolve(): a mask times the input window, summed).  Integer coefficients
 * coeffs[kh][kw] (row-major, applied without flipping), then an arithmetic
 * right shift by `shift` (floor division by 2^shift) and saturation to S16. */
int orc_convolve_u8_s16(const uint8_t* in, int16_t* out, int w, int h, int kw, int kh,
                        const int32_t* coeffs, int shift, int border, int cval,
                        const int vin[4], int vout[4]) {
    int r[4];
    int rx = kw / 2, ry = kh / 2;
    if (w <= 0 || h <= 0 || kw <= 0 || kh <= 0 || !(kw & 1) || !(kh & 1) || shift < 0 ||
        shift > 30)
        return ORC_ERR;
    rect_local(r, vin, rx, ry, border);
    memset(out, 0, sizeof(int16_t) * (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            int64_t s = 0;
            for (int dy = -ry; dy <= ry; ++dy)
                for (int dx = -rx; dx <= rx; ++dx)
                    s += (int64_t)coeffs[(dy + ry) * kw + (dx + rx)] *
                         read_u8(in, w, h, x + dx, y + dy, border, cval);
            /* floor division by 2^shift (s may be negative) */
            int64_t d = (int64_t)1 << shift;
            int64_t q = s >= 0 ? s / d : -((-s + d - 1) / d);
            if (q > 32767) q = 32767;
            if (q < -32768) q = -32768;
            out[(size_t)y * w + x] = (int16_t)q;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Convolve with a U8 output (the OpenVX Convolve output may be U8): the same
 * floor-divided sum, saturated to 0 .. 255. */
int orc_convolve_u8_u8(const uint8_t* in, uint8_t* out, int w, int h, int kw, int kh,
                       const int32_t* coeffs, int shift, int border, int cval,
                       const int vin[4], int vout[4]) {
    int r[4];
    int rx = kw / 2, ry = kh / 2;
    if (w <= 0 || h <= 0 || kw <= 0 || kh <= 0 || !(kw & 1) || !(kh & 1) || shift < 0 ||
        shift > 30)
        return ORC_ERR;
    rect_local(r, vin, rx, ry, border);
    memset(out, 0, (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            int64_t s = 0;
            for (int dy = -ry; dy <= ry; ++dy)
                for (int dx = -rx; dx <= rx; ++dx)
                    s += (int64_t)coeffs[(dy + ry) * kw + (dx + rx)] *
                         read_u8(in, w, h, x + dx, y + dy, border, cval);
            int64_t d = (int64_t)1 << shift;
            int64_t q = s >= 0 ? s / d : -((-s + d - 1) / d);
            if (q > 255) q = 255;
            if (q < 0) q = 0;
            out[(size_t)y * w + x] = (uint8_t)q;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Point operators (Table 2 "point"; Section 4)                               */

/* Magnitude (Table 2): m = floor(sqrt(gx^2 + gy^2) + 0.5) in double,
 * saturated to 32767, S16 output. */
int orc_magnitude(const int16_t* gx, const int16_t* gy, int16_t* out, int w, int h,
                  const int va[4], const int vb[4], int vout[4]) {
    int r[4];
    rect_intersect(r, va, vb);
    memset(out, 0, sizeof(int16_t) * (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            double s = (double)gx[i] * gx[i] + (double)gy[i] * gy[i];
            double m = floor(sqrt(s) + 0.5);
            if (m > 32767.0) m = 32767.0;
            out[i] = (int16_t)m;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Phase (Table 2): phi = atan2(gy, gx) in double, moved into [0, 2*pi);
 * q = floor(phi * 256 / (2*pi) + 0.5) mod 256, U8 output.  atan2(0, 0) = 0. */
int orc_phase(const int16_t* gx, const int16_t* gy, uint8_t* out, int w, int h,
              const int va[4], const int vb[4], int vout[4]) {
    int r[4];
    const double two_pi = 2.0 * 3.14159265358979323846;
    rect_intersect(r, va, vb);
    memset(out, 0, (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            double phi = atan2((double)gy[i], (double)gx[i]);
            if (phi < 0) phi += two_pi;
            int64_t q = (int64_t)floor(phi * 256.0 / two_pi + 0.5);
            out[i] = (uint8_t)(q % 256);
        }
    rect_copy(vout, r);
    return ORC_OK;
}

static double load_as_double(const void* p, int fmt, size_t i) {
    switch (fmt) {
        case ORC_U8: return ((const uint8_t*)p)[i];
        case ORC_S16: return ((const int16_t*)p)[i];
        case ORC_S32: return ((const int32_t*)p)[i];
        case ORC_F32: return ((const float*)p)[i];
    }
    return 0.0;
}

/* Threshold (Table 2; Listing 1).  Binary: out = in > thr ? tv : fv (strict).
 * Range: out = (in > upper || in < lower) ? fv : tv.  Input U8, S16, S32 or
 * F32.  Reading: the threshold values carry the input's type, so for F32
 * input they are first rounded to binary32; the comparison itself is done in
 * double, which is exact for every one of these formats.  U8 out. */
int orc_threshold(const void* in, int fmt, uint8_t* out, int w, int h, int range,
                  double thr_or_lower, double upper, int tv, int fv, const int vin[4],
                  int vout[4]) {
    int r[4];
    if (fmt == ORC_F32) {
        thr_or_lower = (double)(float)thr_or_lower;
        upper = (double)(float)upper;
    }
    rect_copy(r, vin);
    memset(out, 0, (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            double v = load_as_double(in, fmt, i);
            int t;
            if (range)
                t = (v > upper || v < thr_or_lower) ? 0 : 1;
            else
                t = v > thr_or_lower;
            out[i] = (uint8_t)(t ? tv : fv);
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* ChannelExtract from UYVY (Table 2; Listing 1 takes the Y channel).  A UYVY
 * row of width W (even) holds W/2 macro-pixels of bytes U0 Y0 V0 Y1.
 * channel 0 = Y (W x H out), 1 = U, 2 = V ((W/2) x H out). */
int orc_channel_extract_uyvy(const uint8_t* in, uint8_t* out, int w, int h, int channel) {
    if (w <= 0 || h <= 0 || (w & 1)) return ORC_ERR;
    for (int y = 0; y < h; ++y) {
        const uint8_t* row = in + (size_t)y * 2 * w;
        if (channel == 0) {
            for (int x = 0; x < w; ++x) out[(size_t)y * w + x] = row[2 * x + 1];
        } else {
            int off = channel == 1 ? 0 : 2;
            for (int x = 0; x < w / 2; ++x) out[(size_t)y * (w / 2) + x] = row[4 * x + off];
        }
    }
    return ORC_OK;
}

static int64_t sat_or_wrap(int64_t v, int fmt, int saturate) {
    if (fmt == ORC_U8) {
        if (saturate) return v < 0 ? 0 : (v > 255 ? 255 : v);
        return (int64_t)(uint8_t)(v & 0xFF);
    }
    /* S16 */
    if (saturate) return v < -32768 ? -32768 : (v > 32767 ? 32767 : v);
    return (int64_t)(int16_t)(uint16_t)(v & 0xFFFF);
}

static void store_int(void* p, int fmt, size_t i, int64_t v) {
    if (fmt == ORC_U8) ((uint8_t*)p)[i] = (uint8_t)v;
    else ((int16_t*)p)[i] = (int16_t)v;
}

/* Arithmetic point operators on U8/S16 (Table 2: Add, Subtract, AbsDiff).
 * op 0 = add, 1 = subtract (a - b), 2 = absdiff |a - b|.  The exact integer
 * result is wrapped (two's complement) or saturated to the output format. */
int orc_arith(const void* a, int fa, const void* b, int fb, void* out, int fo, int w, int h,
              int op, int saturate, const int va[4], const int vb[4], int vout[4]) {
    int r[4];
    rect_intersect(r, va, vb);
    memset(out, 0, (size_t)w * h * (fo == ORC_U8 ? 1 : 2));
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            int64_t av = (int64_t)load_as_double(a, fa, i);
            int64_t bv = (int64_t)load_as_double(b, fb, i);
            int64_t v = op == 0 ? av + bv : (op == 1 ? av - bv : (av > bv ? av - bv : bv - av));
            store_int(out, fo, i, sat_or_wrap(v, fo, saturate));
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Multiply (Table 2 point operator): a * b * scale on U8/S16, scale a
 * binary32 value.  Reading (the paper prints no arithmetic; these are the
 * OpenVX policies): the product is taken exactly (a long double holds it:
 * |a * b| <= 2^30 times a 24-bit significand), rounded once toward zero
 * (nearest_even 0) or to the nearest integer with ties to even (1), then
 * wrapped or saturated to the output format. */
int orc_multiply(const void* a, int fa, const void* b, int fb, void* out, int fo, int w, int h,
                 float scale, int saturate, int nearest_even, const int va[4], const int vb[4],
                 int vout[4]) {
    int r[4];
    if (!(scale >= 0.0f) || scale > 65536.0f) return ORC_ERR;
    rect_intersect(r, va, vb);
    memset(out, 0, (size_t)w * h * (fo == ORC_U8 ? 1 : 2));
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            long double exact = (long double)load_as_double(a, fa, i) *
                                (long double)load_as_double(b, fb, i) * (long double)scale;
            long double rounded = nearest_even ? nearbyintl(exact) : truncl(exact);
            store_int(out, fo, i, sat_or_wrap((int64_t)rounded, fo, saturate));
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* ConvertDepth (Table 2 point operator; OpenVX semantics, which the paper
 * does not print): U8 -> S16 is v << shift (exact); S16 -> U8 is v >> shift
 * (arithmetic, i.e. floor division by 2^shift), then wrapped to the low 8
 * bits or saturated to 0..255.  Same format in and out is Copy (shift 0).
 * 0 <= shift < 8. */
int orc_convert_depth(const void* in, int fi, void* out, int fo, int w, int h, int shift,
                      int saturate, const int vin[4], int vout[4]) {
    if (shift < 0 || shift > 7) return ORC_ERR;
    memset(out, 0, (size_t)w * h * (fo == ORC_U8 ? 1 : 2));
    for (int y = vin[1]; y < vin[3]; ++y)
        for (int x = vin[0]; x < vin[2]; ++x) {
            size_t i = (size_t)y * w + x;
            int64_t v = (int64_t)load_as_double(in, fi, i);
            int64_t r;
            if (fi == fo)
                r = v;
            else if (fo == ORC_S16)
                r = v * (1 << shift);
            else
                r = (int64_t)floor((double)v / (double)(1 << shift));
            store_int(out, fo, i, sat_or_wrap(r, fo, saturate));
        }
    rect_copy(vout, vin);
    return ORC_OK;
}

/* Bitwise point operators on U8 (Table 2: And, Or, Xor, Not): op 0 = a & b,
 * 1 = a | b, 2 = a ^ b, 3 = ~a (b unused, may be NULL). */
int orc_bitwise(const uint8_t* a, const uint8_t* b, uint8_t* out, int w, int h, int op,
                const int va[4], const int vb[4], int vout[4]) {
    int r[4];
    if (op < 0 || op > 3 || (op < 3 && !b)) return ORC_ERR;
    if (op == 3) rect_copy(r, va);
    else rect_intersect(r, va, vb);
    memset(out, 0, (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            int v = op == 0 ? (a[i] & b[i]) : op == 1 ? (a[i] | b[i]) : op == 2 ? (a[i] ^ b[i])
                                                                         : (~a[i] & 0xFF);
            out[i] = (uint8_t)v;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Custom point operator MUL (Harris products gx^2, gy^2, gx*gy): the exact
 * integer product of two S16 samples, stored as S32. */
int orc_mul_s16_s32(const int16_t* a, const int16_t* b, int32_t* out, int w, int h,
                    const int va[4], const int vb[4], int vout[4]) {
    int r[4];
    rect_intersect(r, va, vb);
    memset(out, 0, sizeof(int32_t) * (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            out[i] = (int32_t)((int64_t)a[i] * b[i]);
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Round the rational m / d (m >= 0, d > 0) to the nearest binary32 value,
 * ties to even, by exact integer arithmetic.  Used to give the F32 Harris
 * response a single rounding. */
static float round_ratio_to_float(unsigned __int128 m, uint64_t d) {
    if (m == 0) return 0.0f;
    /* find e so that 2^23 <= m / (d * 2^e) < 2^24 */
    int e = 0;
    unsigned __int128 num = m, den = d;
    while (num < (den << 23)) { num <<= 1; --e; }
    while (num >= (den << 24)) { den <<= 1; ++e; }
    unsigned __int128 t = num / den;
    unsigned __int128 rem = num - t * den;
    /* compare rem / den with 1/2 */
    if (2 * rem > den || (2 * rem == den && (t & 1))) ++t;
    return ldexpf((float)(uint32_t)t, e); /* t <= 2^24: exact in float */
}

/* Custom point operator: the Harris corner response (HarrisCorners row of
 * Table 2; the corner-detector benchmark of Section 6) from the three window
 * sums Sxx, Syy, Sxy:
 *     R = Sxx*Syy - Sxy^2 - k * (Sxx + Syy)^2,   k = kn / kd.
 * Sxx, Syy, Sxy are exact integers, so kd*R is an exact integer (int128
 * here); R is returned as the binary32 value nearest to the exact rational. */
int orc_harris_response(const int32_t* sxx, const int32_t* syy, const int32_t* sxy, float* out,
                        int w, int h, int64_t kn, int64_t kd, const int va[4], const int vb[4],
                        const int vc[4], int vout[4]) {
    int r[4], t[4];
    if (kd <= 0 || kn < 0) return ORC_ERR;
    rect_intersect(t, va, vb);
    rect_intersect(r, t, vc);
    memset(out, 0, sizeof(float) * (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            __int128 a = sxx[i], b = syy[i], c = sxy[i];
            __int128 det = a * b - c * c;
            __int128 tr = a + b;
            __int128 q = (__int128)kd * det - (__int128)kn * tr * tr; /* = kd * R */
            float v = q >= 0 ? round_ratio_to_float((unsigned __int128)q, (uint64_t)kd)
                             : -round_ratio_to_float((unsigned __int128)(-q), (uint64_t)kd);
            out[i] = v;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

/* Exposed for the oracle's own pins: the correctly rounded float of m/d. */
float orc_round_ratio(int64_t num, int64_t den) {
    if (den <= 0) return 0.0f;
    if (num >= 0) return round_ratio_to_float((unsigned __int128)num, (uint64_t)den);
    return -round_ratio_to_float((unsigned __int128)(-(__int128)num), (uint64_t)den);
}

/* Harris-corner graph of the 4096x2160 workload, composed node by node from
 * the functions above (Sobel3x3 -> gx^2, gy^2, gx*gy -> 5x5 window sums ->
 * response -> binary threshold), for the cpu_baseline timing and smoke check.
 * scratch must hold 2*w*h int16 + 6*w*h int32 + w*h float. */
/* Shi-Tomasi response (the Tomasi application of Section 6: the smaller
 * eigenvalue of the structure tensor [Sxx Sxy; Sxy Syy]):
 *   lambda_min = (Sxx + Syy - sqrt((Sxx - Syy)^2 + 4 Sxy^2)) / 2,
 * evaluated in long double from the exact integer discriminant and rounded
 * once to binary32. */
int orc_tomasi_response(const int32_t* sxx, const int32_t* syy, const int32_t* sxy, float* out,
                        int w, int h, const int va[4], const int vb[4], const int vc[4],
                        int vout[4]) {
    int r[4], t[4];
    rect_intersect(t, va, vb);
    rect_intersect(r, t, vc);
    memset(out, 0, sizeof(float) * (size_t)w * h);
    for (int y = r[1]; y < r[3]; ++y)
        for (int x = r[0]; x < r[2]; ++x) {
            size_t i = (size_t)y * w + x;
            int64_t a = sxx[i], b = syy[i], c = sxy[i];
            int64_t disc = (a - b) * (a - b) + 4 * c * c;
            long double lam = ((long double)(a + b) - sqrtl((long double)disc)) / 2.0L;
            out[i] = (float)lam;
        }
    rect_copy(vout, r);
    return ORC_OK;
}

int orc_harris_graph(const uint8_t* in, uint8_t* mask, float* resp, int w, int h, int border,
                     int64_t kn, int64_t kd, double thr, void* scratch) {
    size_t n = (size_t)w * h;
    int16_t* gx = (int16_t*)scratch;
    int16_t* gy = gx + n;
    int32_t* p = (int32_t*)(gy + n);
    int32_t *ixx = p, *iyy = p + n, *ixy = p + 2 * n, *sxx = p + 3 * n, *syy = p + 4 * n,
            *sxy = p + 5 * n;
    float* rr = resp ? resp : (float*)(p + 6 * n);
    int full[4] = {0, 0, w, h}, vs[4], vp[4], vq[4], vw[4], vr[4], vm[4];
    if (orc_sobel3x3(in, gx, gy, w, h, border, 0, full, vs)) return ORC_ERR;
    orc_mul_s16_s32(gx, gx, ixx, w, h, vs, vs, vp);
    orc_mul_s16_s32(gy, gy, iyy, w, h, vs, vs, vq);
    orc_mul_s16_s32(gx, gy, ixy, w, h, vs, vs, vq);
    if (orc_window_sum_s32(ixx, sxx, w, h, 5, 5, border, 0, vp, vw)) return ORC_ERR;
    if (orc_window_sum_s32(iyy, syy, w, h, 5, 5, border, 0, vq, vw)) return ORC_ERR;
    if (orc_window_sum_s32(ixy, sxy, w, h, 5, 5, border, 0, vq, vw)) return ORC_ERR;
    if (orc_harris_response(sxx, syy, sxy, rr, w, h, kn, kd, vw, vw, vw, vr)) return ORC_ERR;
    return orc_threshold(rr, ORC_F32, mask, w, h, 0, thr, 0.0, 255, 0, vr, vm);
}

/* Edge graph of the 1920x1080 workload, composed node by node: Gaussian3x3 ->
 * Sobel3x3 -> Magnitude -> binary Threshold (mask) and Phase (phase).
 * scratch must hold w*h bytes + 3*w*h int16. */
int orc_edge_graph(const uint8_t* in, uint8_t* phase, uint8_t* mask, int16_t* mag_out, int w,
                   int h, int border, int cval, int rounding, int thr, void* scratch) {
    size_t n = (size_t)w * h;
    uint8_t* g = (uint8_t*)scratch;
    int16_t* gx = (int16_t*)(g + n + ((16 - (n & 15)) & 15));
    int16_t* gy = gx + n;
    int16_t* mag = mag_out ? mag_out : gy + n;
    int full[4] = {0, 0, w, h}, vg[4], vs[4], vm[4], vp[4], vt[4];
    if (orc_gaussian3x3(in, g, w, h, border, cval, rounding, full, vg)) return ORC_ERR;
    if (orc_sobel3x3(g, gx, gy, w, h, border, cval, vg, vs)) return ORC_ERR;
    orc_magnitude(gx, gy, mag, w, h, vs, vs, vm);
    orc_phase(gx, gy, phase, w, h, vs, vs, vp);
    return orc_threshold(mag, ORC_S16, mask, w, h, 0, (double)thr, 0.0, 255, 0, vm, vt);
}

/* ------------------------------------------------------------------------ */
/* Global operators (Table 2 "reduce" and "histogram"; Section 4: the output
 * depends on the whole input image).  Each traverses the input's valid
 * rectangle in raster order.                                                 */

/* MeanStdDev (reduction): the exact sums S1 = sum v, S2 = sum v^2 and the
 * count N (sums[0..2]); mean = S1 / N and stddev = sqrt(N S2 - S1^2) / N.
 * Reading (OpenVX gives no formula for the rounding): the population
 * standard deviation; mean and stddev are the binary32 roundings of the
 * double results of these expressions, with N S2 - S1^2 exact (128-bit) and
 * converted to double once.  N = 0 gives mean = stddev = 0. */
int orc_mean_stddev(const void* in, int fmt, int w, int h, const int vin[4], int64_t sums[3],
                    float out[2]) {
    int64_t s1 = 0, s2 = 0, n = 0;
    (void)w;
    (void)h;
    if (fmt != ORC_U8 && fmt != ORC_S16) return ORC_ERR;
    for (int y = vin[1]; y < vin[3]; ++y)
        for (int x = vin[0]; x < vin[2]; ++x) {
            int64_t v = (int64_t)load_as_double(in, fmt, (size_t)y * w + x);
            s1 += v;
            s2 += v * v;
            n += 1;
        }
    sums[0] = s1;
    sums[1] = s2;
    sums[2] = n;
    if (n == 0) {
        out[0] = out[1] = 0.0f;
        return ORC_OK;
    }
    __int128 var_n2 = (__int128)n * s2 - (__int128)s1 * s1;
    out[0] = (float)((double)s1 / (double)n);
    out[1] = (float)(sqrt((double)var_n2) / (double)n);
    return ORC_OK;
}

/* MinMaxLoc (reduction): the minimum and maximum, how many pixels take each,
 * and the first pixel (raster order) where each occurs.  res = {min, max,
 * min_count, max_count, min_x, min_y, max_x, max_y}; an empty rectangle gives
 * counts 0 and locations -1. */
int orc_minmaxloc(const void* in, int fmt, int w, int h, const int vin[4], int64_t res[8]) {
    (void)h;
    if (fmt != ORC_U8 && fmt != ORC_S16) return ORC_ERR;
    int64_t mn = 0, mx = 0, cmn = 0, cmx = 0;
    int64_t mnx = -1, mny = -1, mxx = -1, mxy = -1;
    for (int y = vin[1]; y < vin[3]; ++y)
        for (int x = vin[0]; x < vin[2]; ++x) {
            int64_t v = (int64_t)load_as_double(in, fmt, (size_t)y * w + x);
            if (cmn == 0 || v < mn) {
                mn = v;
                cmn = 0;
                mnx = x;
                mny = y;
            }
            if (v == mn) cmn += 1;
            if (cmx == 0 || v > mx) {
                mx = v;
                cmx = 0;
                mxx = x;
                mxy = y;
            }
            if (v == mx) cmx += 1;
        }
    res[0] = mn;
    res[1] = mx;
    res[2] = cmn;
    res[3] = cmx;
    res[4] = mnx;
    res[5] = mny;
    res[6] = mxx;
    res[7] = mxy;
    return ORC_OK;
}

/* Histogram (Table 2 "histogram"): num_bins bins over [offset, offset +
 * range) of a U8 image; value v falls in bin (v - offset) * num_bins / range
 * (integer division, the OpenVX distribution); values outside are not
 * counted.  1 <= num_bins <= 256, offset >= 0, range >= 1, offset + range <=
 * 256. */
int orc_histogram(const uint8_t* in, int w, int h, const int vin[4], int num_bins, int offset,
                  int range, uint32_t* bins) {
    (void)h;
    if (num_bins < 1 || num_bins > 256 || offset < 0 || range < 1 || offset + range > 256)
        return ORC_ERR;
    memset(bins, 0, (size_t)num_bins * sizeof(uint32_t));
    for (int y = vin[1]; y < vin[3]; ++y)
        for (int x = vin[0]; x < vin[2]; ++x) {
            int v = in[(size_t)y * w + x];
            if (v >= offset && v < offset + range) bins[(v - offset) * num_bins / range] += 1;
        }
    return ORC_OK;
}

/* EqualizeHist (Table 2: histogram + point): with the 256-bin histogram of
 * the input's valid rectangle, its cumulative sum c, cmin = c at the smallest
 * value present and N the pixel count, each pixel v becomes
 * round((c[v] - cmin) * 255 / (N - cmin)) with halves rounded up.  Reading:
 * OpenVX leaves the formula open; this is the usual normalised cumulative
 * histogram.  A constant image (N == cmin) is left unchanged.  0 outside the
 * valid rectangle, like every point operator. */
int orc_equalize_hist(const uint8_t* in, uint8_t* out, int w, int h, const int vin[4],
                      int vout[4]) {
    uint32_t hist[256];
    int64_t c[256], n = 0, cmin = -1;
    int full[4];
    orc_histogram(in, w, h, vin, 256, 0, 256, hist);
    for (int v = 0; v < 256; ++v) {
        n += hist[v];
        c[v] = n;
        if (cmin < 0 && hist[v] > 0) cmin = c[v];
    }
    memset(out, 0, (size_t)w * h);
    for (int y = vin[1]; y < vin[3]; ++y)
        for (int x = vin[0]; x < vin[2]; ++x) {
            size_t i = (size_t)y * w + x;
            if (n == cmin) {
                out[i] = in[i];
            } else {
                int64_t num = (c[in[i]] - cmin) * 255;
                int64_t den = n - cmin;
                out[i] = (uint8_t)((2 * num + den) / (2 * den));
            }
        }
    rect_copy(full, vin);
    rect_copy(vout, full);
    return ORC_OK;
}
