// Execution runtime: per-group kernel selection and launch parameters (TMA
// descriptors included), plan launch, the device error word, and the batched
// persistent launch replayed from captured CUDA graphs.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <unordered_map>

#include "hvx_internal.h"
#include "launchers.h"

namespace hvx {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
std::atomic<uint64_t> g_plan_counter{0};

hvx_status get_encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        cudaGetLastError();
    });
    return g_encode ? HVX_SUCCESS : HVX_ERROR_DEVICE;
}

hvx_status encode_u8_map_at(CUtensorMap* map, const void* ptr, uint64_t pitch, uint32_t w,
                            uint32_t h, uint32_t box_w, uint32_t box_h);

// 2-D U8 tensor map of an image with a (box_w x box_h) box; out-of-image
// elements of a box read as 0.
hvx_status encode_u8_map(CUtensorMap* map, const Image* im, uint32_t box_w, uint32_t box_h) {
    if (im->ctx->plan_only) {
        std::memset(map, 0, sizeof(*map));
        return HVX_SUCCESS;
    }
    return encode_u8_map_at(map, im->dev, im->pitch, im->w, im->h, box_w, box_h);
}

hvx_status encode_u8_map_at(CUtensorMap* map, const void* ptr, uint64_t pitch, uint32_t w,
                            uint32_t h, uint32_t box_w, uint32_t box_h) {
    hvx_status st = get_encoder();
    if (st != HVX_SUCCESS) return st;
    if (((uintptr_t)ptr & 15) || (pitch & 15)) return HVX_ERROR_INVALID_PARAMETERS;
    void* const dev = const_cast<void*>(ptr);
    cuuint64_t dims[2] = {w, h};
    cuuint64_t strides[1] = {pitch};
    cuuint32_t box[2] = {box_w, box_h};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, dev, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HVX_SUCCESS : HVX_ERROR_DEVICE;
}

void set_rect(int32_t* d, const Rect& r) {
    d[0] = r.x0;
    d[1] = r.y0;
    d[2] = r.x1;
    d[3] = r.y1;
}

uint64_t image_bytes(const Image* im) { return (uint64_t)im->w * im->h * bytes_per_pixel(im->fmt); }

// Point-operator parameters shared by GenStage and PlainParams.
template <class T>
void fill_point_params(T& st, const Op& op) {
    const NodeParams& p = op.node->p;
    st.i0 = st.i1 = st.i2 = st.i3 = 0;
    st.f0 = st.f1 = 0.f;
    st.k0 = st.k1 = 0;
    switch (op.kind) {
        case OP_THRESH:
            st.i0 = p.thr_type;
            st.i1 = p.true_value;
            st.i2 = p.false_value;
            st.i3 = op.in[0]->fmt == HVX_DF_F32;
            st.k0 = (int64_t)p.thr_value;
            st.k1 = (int64_t)p.thr_upper;
            st.f0 = (float)p.thr_value;
            st.f1 = (float)p.thr_upper;
            break;
        case OP_ADD:
        case OP_SUB:
        case OP_ABSDIFF:
            st.i0 = p.policy == HVX_POLICY_SATURATE;
            st.i1 = op.out->fmt;
            break;
        case OP_HARRIS:
            st.k0 = p.kn;
            st.k1 = p.kd;
            break;
        case OP_MULTIPLY: {
            // scale = k0 * 2^i3 exactly (k0 the 24-bit significand)
            int ex = 0;
            const float fr = std::frexp(p.scale, &ex);
            st.k0 = (int64_t)std::ldexp((double)fr, 24);
            st.i3 = p.scale == 0.0f ? 0 : ex - 24;
            st.i0 = p.policy == HVX_POLICY_SATURATE;
            st.i1 = op.out->fmt;
            st.i2 = p.mul_rounding == HVX_ROUND_TO_NEAREST_EVEN;
            break;
        }
        case OP_CHX: st.i0 = p.channel; break;
        case OP_CONVDEPTH:
            st.i0 = p.shift;
            st.i1 = op.out->fmt;
            st.i2 = p.policy == HVX_POLICY_SATURATE;
            st.i3 = op.in[0]->fmt;
            break;
        default: break;
    }
}

// ---- edge group ---------------------------------------------------------------

struct EdgeMatch {
    int gauss = -1, sx = -1, sy = -1, mag = -1, thr = -1, ph = -1;
};

bool match_edge(const Plan& P, const Group& G, EdgeMatch& m) {
    for (int i : G.ops) {
        int* slot = nullptr;
        switch (P.ops[i].kind) {
            case OP_GAUSS: slot = &m.gauss; break;
            case OP_SOBEL_X: slot = &m.sx; break;
            case OP_SOBEL_Y: slot = &m.sy; break;
            case OP_MAG: slot = &m.mag; break;
            case OP_THRESH: slot = &m.thr; break;
            case OP_PHASE: slot = &m.ph; break;
            default: return false;
        }
        if (*slot >= 0) return false;
        *slot = i;
    }
    if (m.gauss < 0 && m.sy < 0) {
        // Sobel3x3 with only gx alive, exported as S16 (the SobelX application):
        // the kernel's input-row mode, storing gx
        if (m.sx < 0 || m.mag >= 0 || m.thr >= 0 || m.ph >= 0) return false;
        const Op& sx = P.ops[m.sx];
        if (border_wraps(sx.node->border)) return false;
        if (G.inputs.size() != 1 || G.inputs[0] != sx.in[0] || sx.in[0]->fmt != HVX_DF_U8)
            return false;
        return G.outputs.size() == 1 && G.outputs[0] == sx.out && sx.out->fmt == HVX_DF_S16;
    }
    if (m.sy < 0) return false;
    if (m.gauss < 0) {
        // no Gaussian: Sobel3x3 -> Magnitude(gx, gy) -> binary Threshold on
        // the group's U8 input (the Sobel application) runs on the kernel with
        // the input itself in place of the Gaussian image
        if (m.sx < 0 || m.mag < 0 || m.thr < 0 || m.ph >= 0) return false;
        const Op &sx = P.ops[m.sx], &sy = P.ops[m.sy], &mg = P.ops[m.mag], &t = P.ops[m.thr];
        if (sx.node != sy.node || border_wraps(sx.node->border)) return false;
        if (G.inputs.size() != 1 || G.inputs[0] != sx.in[0] || sx.in[0]->fmt != HVX_DF_U8)
            return false;
        if (mg.in[0] != sx.out || mg.in[1] != sy.out || t.in[0] != mg.out) return false;
        if (t.node->p.thr_type != HVX_THRESHOLD_BINARY) return false;
        return G.outputs.size() == 1 && G.outputs[0] == t.out;
    }
    const Op &g = P.ops[m.gauss], &sy = P.ops[m.sy];
    if (m.sx < 0) {
        // the Sobel's gx is dead (Algorithm 1 removed it): only Magnitude(gy, gy)
        // -> binary Threshold, the graph of Listing 1, maps onto the kernel
        if (m.mag < 0 || m.thr < 0 || m.ph >= 0) return false;
        const Op& mg = P.ops[m.mag];
        if (mg.in[0] != sy.out || mg.in[1] != sy.out) return false;
        if (P.ops[m.thr].node->p.thr_type != HVX_THRESHOLD_BINARY) return false;
        if (G.outputs.size() != 1 || G.outputs[0] != P.ops[m.thr].out) return false;
    }
    const Op& sx = P.ops[m.sx >= 0 ? m.sx : m.sy];
    if (border_wraps(g.node->border) || border_wraps(sx.node->border)) return false;
    if (G.inputs.size() != 1 || G.inputs[0] != g.in[0] || g.in[0]->fmt != HVX_DF_U8) return false;
    if (sx.in[0] != g.out || sy.in[0] != g.out || sx.node != sy.node) return false;
    if (m.sx >= 0 && m.mag >= 0 &&
        (P.ops[m.mag].in[0] != sx.out || P.ops[m.mag].in[1] != sy.out))
        return false;
    if (m.ph >= 0 && (P.ops[m.ph].in[0] != sx.out || P.ops[m.ph].in[1] != sy.out)) return false;
    if (m.thr >= 0 && (m.mag < 0 || P.ops[m.thr].in[0] != P.ops[m.mag].out)) return false;
    if (G.outputs.empty()) return false;
    for (Image* o : G.outputs) {
        bool ok = (m.thr >= 0 && o == P.ops[m.thr].out) || (m.ph >= 0 && o == P.ops[m.ph].out) ||
                  (m.mag >= 0 && o == P.ops[m.mag].out);
        if (!ok) return false;
    }
    return true;
}

void base_edge_params(EdgeParams& e, const Group& G, const Image* in, Context* ctx) {
    std::memset(&e, 0, sizeof(e));
    e.W = G.W;
    e.H = G.H;
    e.in = static_cast<const uint8_t*>(in->dev);
    e.in_pitch = in->pitch;
    e.err = ctx->d_error;
    e.valid[0] = e.valid[1] = 0;
    e.valid[2] = G.W;
    e.valid[3] = G.H;
}

hvx_status build_edge(Plan& P, Group& G, const EdgeMatch& m, Context* ctx) {
    const Op& sx = P.ops[m.sx >= 0 ? m.sx : m.sy];
    const Op& sy = P.ops[m.sy >= 0 ? m.sy : m.sx];
    Image* const input = m.gauss >= 0 ? P.ops[m.gauss].in[0] : sx.in[0];
    EdgeParams& e = G.edge;
    base_edge_params(e, G, input, ctx);
    e.mag_yy = m.sx < 0 ? 1 : 0;
    e.border_s = sx.node->border;
    e.cval_s = sx.node->cval & 0xFF;
    if (m.gauss >= 0) {
        const Op& g = P.ops[m.gauss];
        e.border_g = g.node->border;
        e.cval_g = g.node->cval & 0xFF;
        e.rounding = g.node->rounding;
        set_rect(e.gvalid, g.out->valid);
    } else {
        // the input stands in for the Gaussian image: its cells outside the
        // image take the Sobel's border, and all of it is valid
        e.g_op = 1;
        e.border_g = e.border_s;
        e.cval_g = e.cval_s;
        e.gvalid[0] = e.gvalid[1] = 0;
        e.gvalid[2] = (int32_t)G.W;
        e.gvalid[3] = (int32_t)G.H;
    }
    set_rect(e.valid, rect_intersect(sx.out->valid, sy.out->valid));
    if (m.sy < 0) {  // gx alone, exported as S16 (it uses the magnitude's slot)
        e.mag = static_cast<int16_t*>(sx.out->dev);
        e.mag_pitch = sx.out->pitch;
    }
    auto is_out = [&](const Image* im) {
        return std::find(G.outputs.begin(), G.outputs.end(), im) != G.outputs.end();
    };
    if (m.ph >= 0) {
        e.phase = static_cast<uint8_t*>(P.ops[m.ph].out->dev);
        e.phase_pitch = P.ops[m.ph].out->pitch;
    }
    if (m.mag >= 0 && is_out(P.ops[m.mag].out)) {
        e.mag = static_cast<int16_t*>(P.ops[m.mag].out->dev);
        e.mag_pitch = P.ops[m.mag].out->pitch;
    }
    if (m.thr >= 0) {
        const Op& t = P.ops[m.thr];
        const NodeParams& tp = t.node->p;
        e.mask = static_cast<uint8_t*>(t.out->dev);
        e.mask_pitch = t.out->pitch;
        e.tv = tp.true_value;
        e.fv = tp.false_value;
        e.thr_type = tp.thr_type;
        e.thr_lo = (int32_t)std::max<int64_t>(-40000, std::min<int64_t>(40000, (int64_t)tp.thr_value));
        e.thr_hi = (int32_t)std::max<int64_t>(-40000, std::min<int64_t>(40000, (int64_t)tp.thr_upper));
        if (tp.thr_type == HVX_THRESHOLD_BINARY) {
            // round(sqrt(s)) > T  <=>  s > T^2 + T  (T >= 0), always true for T < 0;
            // s = gx^2 + gy^2, or 2 gy^2 for Magnitude(gy, gy)
            int64_t T = (int64_t)tp.thr_value;
            e.thr_general = 0;
            if (T < 0)
                e.s_thr = -1;
            else if (T >= 32767)
                e.s_thr = std::numeric_limits<int32_t>::max();
            else
                e.s_thr = (int32_t)(T * T + T);
        } else {
            e.thr_general = 1;
        }
    }
    // one image per launch: R rows per thread, a 160 x (8R + 4) box (the
    // batch kernel encodes its own 160 x EDGE_LOAD_H maps)
    e.rows = edge_single_rows((int)G.W, (int)G.H, ctx->num_sms);
    if (const char* env = getenv("HVX_EDGE_ROWS")) {  // tuning knob: 2 .. EDGE_ROWS
        const int r = atoi(env);
        static bool said = false;
        if (!said) {
            said = true;
            if (r >= 2 && r <= EDGE_ROWS)
                fprintf(stderr, "hvx: HVX_EDGE_ROWS=%d replaces the rows per thread of every "
                                "single-image edge kernel\n", r);
            else
                fprintf(stderr, "hvx: HVX_EDGE_ROWS=%s ignored (not in 2..%d)\n", env, EDGE_ROWS);
        }
        if (r >= 2 && r <= EDGE_ROWS) e.rows = r;
    }
    return encode_u8_map(&G.tmap, input, EDGE_LOAD_W, (uint32_t)(8 * e.rows + 4));
}

// A Convolve node that is the 5x5 binomial filter [1 4 6 4 1]^T [1 4 6 4 1]
// divided by 256 (shift 8), U8 to U8, with a border the kernel's box fill
// implements (every sum is non-negative and at most 255 * 256, so the floor
// division is a shift and no output saturates).
bool is_binomial5(const Op& op) {
    if (op.kind != OP_CONV || border_wraps(op.node->border)) return false;
    const NodeParams& p = op.node->p;
    if (p.kw != 5 || p.kh != 5 || p.shift != 8 || p.coeffs.size() != 25) return false;
    if (op.in[0]->fmt != HVX_DF_U8 || op.out->fmt != HVX_DF_U8) return false;
    static const int32_t b[5] = {1, 4, 6, 4, 1};
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c)
            if (p.coeffs[r * 5 + c] != b[r] * b[c]) return false;
    return true;
}

hvx_status build_binom5(Plan& P, Group& G, Context* ctx) {
    const Op& op = P.ops[G.ops[0]];
    EdgeParams& e = G.edge;
    base_edge_params(e, G, op.in[0], ctx);
    e.g_op = 2;
    e.border_g = op.node->border;
    e.cval_g = op.node->cval & 0xFF;
    e.border_s = HVX_BORDER_UNDEFINED;
    e.gout = static_cast<uint8_t*>(op.out->dev);
    e.gout_pitch = op.out->pitch;
    set_rect(e.gvalid, op.out->valid);
    set_rect(e.valid, op.out->valid);
    // one image per launch: R rows per thread, a 160 x (8R + 4) box (the batch
    // kernel encodes its own 160 x (8R + 4) maps for the R it runs)
    e.rows = edge_single_rows((int)G.W, (int)G.H, ctx->num_sms);
    return encode_u8_map(&G.tmap, op.in[0], EDGE_LOAD_W, (uint32_t)(8 * e.rows + 4));
}

hvx_status build_gauss(Plan& P, Group& G, Context* ctx) {
    const Op& g = P.ops[G.ops[0]];
    EdgeParams& e = G.edge;
    base_edge_params(e, G, g.in[0], ctx);
    e.border_g = g.node->border;
    e.cval_g = g.node->cval & 0xFF;
    e.border_s = HVX_BORDER_UNDEFINED;
    e.rounding = g.node->rounding;
    e.gout = static_cast<uint8_t*>(g.out->dev);
    e.gout_pitch = g.out->pitch;
    set_rect(e.gvalid, g.out->valid);
    // one image per launch: R rows per thread, a 160 x (8R + 2) box (the
    // batch kernel encodes its own 160 x GAUSS_LOAD_H maps)
    e.rows = gauss_single_rows((int)G.W, (int)G.H, ctx->num_sms);
    return encode_u8_map(&G.tmap, g.in[0], GAUSS_LOAD_W, (uint32_t)(8 * e.rows + 2));
}

// ---- Harris group -------------------------------------------------------------

struct HarrisMatch {
    int sx = -1, sy = -1, pxx = -1, pyy = -1, pxy = -1, sxx = -1, syy = -1, sxy = -1, resp = -1,
        thr = -1;
    bool tomasi = false;  // Shi-Tomasi response in place of Harris's
};

bool match_harris(const Plan& P, const Group& G, HarrisMatch& m) {
    std::vector<int> muls, sums;
    for (int i : G.ops) {
        const Op& o = P.ops[i];
        switch (o.kind) {
            case OP_SOBEL_X:
                if (m.sx >= 0) return false;
                m.sx = i;
                break;
            case OP_SOBEL_Y:
                if (m.sy >= 0) return false;
                m.sy = i;
                break;
            case OP_MUL: muls.push_back(i); break;
            case OP_LSUM: sums.push_back(i); break;
            case OP_HARRIS:
            case OP_TOMASI:
                if (m.resp >= 0) return false;
                m.resp = i;
                m.tomasi = o.kind == OP_TOMASI;
                break;
            case OP_THRESH:
                if (m.thr >= 0) return false;
                m.thr = i;
                break;
            default: return false;
        }
    }
    if (m.sx < 0 || m.sy < 0 || muls.size() != 3 || sums.size() != 3 || m.resp < 0) return false;
    const Op &sx = P.ops[m.sx], &sy = P.ops[m.sy];
    if (sx.node != sy.node || G.inputs.size() != 1 || G.inputs[0] != sx.in[0]) return false;
    if (border_wraps(sx.node->border)) return false;
    Image *X = sx.out, *Y = sy.out;
    for (int i : muls) {
        const Op& o = P.ops[i];
        if (o.in[0] == X && o.in[1] == X)
            m.pxx = i;
        else if (o.in[0] == Y && o.in[1] == Y)
            m.pyy = i;
        else if ((o.in[0] == X && o.in[1] == Y) || (o.in[0] == Y && o.in[1] == X))
            m.pxy = i;
        else
            return false;
    }
    if (m.pxx < 0 || m.pyy < 0 || m.pxy < 0) return false;
    const Op& s0 = P.ops[sums[0]];
    for (int i : sums) {
        const Op& o = P.ops[i];
        if (o.rx != 2 || o.ry != 2 || o.node->border != s0.node->border ||
            border_wraps(o.node->border) ||
            o.node->cval != s0.node->cval)
            return false;
        if (o.in[0] == P.ops[m.pxx].out)
            m.sxx = i;
        else if (o.in[0] == P.ops[m.pyy].out)
            m.syy = i;
        else if (o.in[0] == P.ops[m.pxy].out)
            m.sxy = i;
        else
            return false;
    }
    if (m.sxx < 0 || m.syy < 0 || m.sxy < 0) return false;
    const Op& r = P.ops[m.resp];
    if (r.in[0] != P.ops[m.sxx].out || r.in[1] != P.ops[m.syy].out || r.in[2] != P.ops[m.sxy].out)
        return false;
    if (m.thr >= 0) {
        const Op& t = P.ops[m.thr];
        if (t.in[0] != r.out || t.node->p.thr_type != HVX_THRESHOLD_BINARY) return false;
    }
    for (Image* o : G.outputs)
        if (!(o == r.out || (m.thr >= 0 && o == P.ops[m.thr].out))) return false;
    return !G.outputs.empty();
}

// Largest q with round_to_binary32(q / kd) <= T, so that a binary32 response
// exceeds T exactly when q > q_thr.  With m the midpoint between T and the
// next binary32 value above it, round(v) <= T holds for v < m, and at v = m
// when T's significand is even (ties to even).  kd * m is exact in double.
int64_t harris_q_threshold(float T, int64_t kd) {
    const double lim = 4611686018427387904.0;  // 2^62, beyond any |q| of 5x5 sums
    if (std::isnan(T)) return std::numeric_limits<int64_t>::max();
    float up = std::nextafter(T, std::numeric_limits<float>::infinity());
    if (std::isinf(T) && T > 0) return std::numeric_limits<int64_t>::max();
    double m = ((double)T + (double)up) * 0.5;
    double B = (double)kd * m;
    if (B >= lim) return (int64_t)lim;
    if (B <= -lim) return -(int64_t)lim;
    uint32_t bits;
    std::memcpy(&bits, &T, 4);
    bool tie_down = (bits & 1u) == 0;
    double fl = std::floor(B);
    if (fl == B) return tie_down ? (int64_t)B : (int64_t)B - 1;
    return (int64_t)fl;
}

hvx_status build_harris(Plan& P, Group& G, const HarrisMatch& m, Context* ctx) {
    const Op &sx = P.ops[m.sx], &s0 = P.ops[m.sxx], &r = P.ops[m.resp];
    HarrisParams& h = G.harris;
    std::memset(&h, 0, sizeof(h));
    h.W = G.W;
    h.H = G.H;
    h.in = static_cast<const uint8_t*>(sx.in[0]->dev);
    h.in_pitch = sx.in[0]->pitch;
    h.border_s = sx.node->border;
    h.cval_s = sx.node->cval & 0xFF;
    h.border_b = s0.node->border;
    h.cval_b = s0.node->cval;
    h.wr = 2;
    h.rows = harris_fast_rows((int)G.W, (int)G.H, ctx->num_sms > 0 ? ctx->num_sms : 152);
    h.tomasi = m.tomasi ? 1 : 0;
    h.kn = m.tomasi ? 0 : r.node->p.kn;
    h.kd = m.tomasi ? 1 : r.node->p.kd;
    set_rect(h.pvalid, P.ops[m.pxy].out->valid);
    set_rect(h.valid, r.out->valid);
    h.err = ctx->d_error;
    bool resp_out = std::find(G.outputs.begin(), G.outputs.end(), r.out) != G.outputs.end();
    if (resp_out) {
        h.resp = static_cast<float*>(r.out->dev);
        h.resp_pitch = r.out->pitch;
    }
    if (m.thr >= 0) {
        const Op& t = P.ops[m.thr];
        h.mask = static_cast<uint8_t*>(t.out->dev);
        h.mask_pitch = t.out->pitch;
        h.tv = t.node->p.true_value;
        h.fv = t.node->p.false_value;
        h.thr_f = (float)t.node->p.thr_value;
        if (!m.tomasi) h.q_thr = harris_q_threshold(h.thr_f, h.kd);
    }
    int bw = 0, bh = 0;
    harris_box(h, &bw, &bh);
    return encode_u8_map(&G.tmap, sx.in[0], bw, bh);
}

// ---- plain point / generic ------------------------------------------------------

void plain_img(PlainImg& d, const Image* im) {
    d.ptr = im->dev;
    d.pitch = im->pitch;
    d.fmt = im->fmt;
    d.pad = 0;
}

hvx_status build_point(Plan& P, Group& G) {
    const Op& op = P.ops[G.ops[0]];
    PlainParams& pp = G.plain;
    std::memset(&pp, 0, sizeof(pp));
    pp.W = op.out->w;
    pp.H = op.out->h;
    pp.op = op.kind;
    pp.n_in = op.n_in;
    pp.n_out = 1;
    for (int k = 0; k < op.n_in; ++k) plain_img(pp.in[k], op.in[k]);
    plain_img(pp.out[0], op.out);
    set_rect(pp.valid, op.out->valid);
    fill_point_params(pp, op);
    if (op.out->ctx->plan_only) return HVX_SUCCESS;
    for (int k = 0; k < op.n_in; ++k)
        if (!op.in[k]->dev) return HVX_ERROR_INVALID_GRAPH;
    return op.out->dev ? HVX_SUCCESS : HVX_ERROR_INVALID_GRAPH;
}

hvx_status build_eqhist(Plan& P, Group& G) {
    const Op& op = P.ops[G.ops[0]];
    EqHistParams& q = G.eqh;
    std::memset(&q, 0, sizeof(q));
    q.W = op.out->w;
    q.H = op.out->h;
    q.in = static_cast<const uint8_t*>(op.in[0]->dev);
    q.in_pitch = op.in[0]->pitch;
    q.out = static_cast<uint8_t*>(op.out->dev);
    q.out_pitch = op.out->pitch;
    q.hist = static_cast<uint32_t*>(op.node->d_aux);
    set_rect(q.valid, op.in[0]->valid);
    if (op.out->ctx->plan_only) return HVX_SUCCESS;
    return q.in && q.out && q.hist ? HVX_SUCCESS : HVX_ERROR_INVALID_GRAPH;
}

hvx_status build_generic(Plan& P, Group& G) {
    GenericDesc& d = G.gdesc;
    std::memset(&d, 0, sizeof(d));
    G.user_code.clear();
    d.W = G.W;
    d.H = G.H;
    // halo of every image: sum of the window radii of in-group ops downstream
    std::unordered_map<const Image*, int> halo, buf;
    std::unordered_map<int, int> h_out;
    for (auto it = G.ops.rbegin(); it != G.ops.rend(); ++it) {
        const Op& op = P.ops[*it];
        int h = 0;
        for (int j : G.ops) {
            const Op& c = P.ops[j];
            for (int k = 0; k < c.n_in; ++k)
                if (c.in[k] == op.out) h = std::max(h, h_out[j] + std::max(c.rx, c.ry));
        }
        h_out[*it] = h;
        halo[op.out] = std::max(halo[op.out], h);
    }
    for (int j : G.ops) {
        const Op& c = P.ops[j];
        for (int k = 0; k < c.n_in; ++k)
            if (std::find(G.inputs.begin(), G.inputs.end(), c.in[k]) != G.inputs.end())
                halo[c.in[k]] = std::max(halo[c.in[k]], h_out[j] + std::max(c.rx, c.ry));
    }
    std::vector<const Image*> images(G.inputs.begin(), G.inputs.end());
    for (int i : G.ops)
        if (!P.ops[i].out->is_result) images.push_back(P.ops[i].out);
    if ((int)images.size() > GEN_MAX_BUF || (int)G.ops.size() > GEN_MAX_STAGE ||
        (int)G.inputs.size() > GEN_MAX_EXT || (int)G.outputs.size() > GEN_MAX_EXT)
        return HVX_ERROR_NOT_SUPPORTED;
    int words = 0;
    for (const Image* im : images) {
        int b = d.n_buf++;
        buf[im] = b;
        GenBuf& gb = d.buf[b];
        gb.halo = halo[im];
        if (gb.halo > GEN_MAX_HALO) return HVX_ERROR_NOT_SUPPORTED;
        gb.is_float = im->fmt == HVX_DF_F32;
        gb.fmt = im->fmt;
        gb.fill = FILL_NONE;
        gb.cval = 0;
        for (int j : G.ops) {
            const Op& c = P.ops[j];
            if (!op_is_local(c.kind)) continue;
            for (int k = 0; k < c.n_in; ++k)
                if (c.in[k] == im) {
                    if (c.node->border == HVX_BORDER_REPLICATE) gb.fill = FILL_REPLICATE;
                    if (c.node->border == HVX_BORDER_MIRROR) gb.fill = FILL_MIRROR;
                    if (c.node->border == HVX_BORDER_REPEAT) gb.fill = FILL_REPEAT;
                    if (c.node->border == HVX_BORDER_CONSTANT) {
                        gb.fill = FILL_CONSTANT;
                        gb.cval = im->fmt == HVX_DF_U8 ? (c.node->cval & 0xFF) : c.node->cval;
                    }
                }
        }
        // MIRROR / REPEAT fills read anywhere in the image: only external
        // inputs, loaded from memory, can take them (the planner keeps such
        // consumers out of their producer's group)
        if ((gb.fill == FILL_MIRROR || gb.fill == FILL_REPEAT) &&
            std::find(G.inputs.begin(), G.inputs.end(), im) == G.inputs.end())
            return HVX_ERROR_NOT_SUPPORTED;
        set_rect(gb.valid, im->valid);
        gb.smem_off = words;
        words += (GEN_TW + 2 * gb.halo) * (GEN_TH + 2 * gb.halo);
    }
    d.smem_words = words;
    if (words * 4 > 220 * 1024) return HVX_ERROR_NOT_SUPPORTED;
    int coeffs = 0;
    for (int i : G.ops) {
        const Op& op = P.ops[i];
        GenStage& st = d.st[d.n_stage++];
        st.op = op.kind;
        st.in[0] = st.in[1] = st.in[2] = -1;
        for (int k = 0; k < op.n_in; ++k) st.in[k] = buf[op.in[k]];
        st.out = op.out->is_result ? -1 : buf[op.out];
        st.res = op.out->is_result ? op.out->dev : nullptr;
        st.rx = op.rx;
        st.ry = op.ry;
        st.rounding = op.node->rounding;
        fill_point_params(st, op);
        if (op.kind == OP_CONV) {
            const std::vector<int32_t>& c = op.node->p.coeffs;
            if (coeffs + (int)c.size() > GEN_MAX_COEFF) return HVX_ERROR_NOT_SUPPORTED;
            st.coeff_off = coeffs;
            st.shift = op.node->p.shift;
            st.i0 = op.out->fmt;  // U8 or S16: the saturation range
            for (int32_t v : c) d.coeff[coeffs++] = v;
        }
        if (op.kind == OP_USER_POINT || op.kind == OP_USER_LOCAL) {
            st.i0 = (int32_t)G.user_code.size();
            st.i1 = op.out->fmt;
            G.user_code.push_back(op.node->p.user_code);
        }
        if (op.kind == OP_HIST) {
            // bins, offset, range; shared-memory words of the tile's histogram
            st.i0 = op.node->p.hist_bins;
            st.i1 = op.node->p.hist_offset;
            st.i2 = op.node->p.hist_range;
            st.i3 = words;
            words += (st.i0 + 3) & ~3;
            d.smem_words = words;
            if (words * 4 > 220 * 1024) return HVX_ERROR_NOT_SUPPORTED;
        }
    }
    for (const Image* im : G.inputs) {
        GenExt& e = d.in[d.n_in++];
        e.ptr = im->dev;
        e.pitch = im->pitch;
        e.fmt = im->fmt;
        e.buf = buf[im];
        if (!im->dev && !im->ctx->plan_only) return HVX_ERROR_INVALID_GRAPH;
    }
    for (const Image* im : G.outputs) {
        GenExt& e = d.out[d.n_out++];
        e.ptr = im->dev;
        e.pitch = im->pitch;
        e.fmt = im->fmt;
        e.buf = buf[im];
        if (!im->dev && !im->ctx->plan_only) return HVX_ERROR_INVALID_GRAPH;
    }
    return HVX_SUCCESS;
}

}  // namespace

hvx_status ensure_context_device_state(Context* ctx) {
    if (!ctx->d_error) {
        cudaError_t e = cudaMalloc(&ctx->d_error, sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return HVX_ERROR_NO_MEMORY;
        }
        if (cudaMemset(ctx->d_error, 0, sizeof(int)) != cudaSuccess) return HVX_ERROR_DEVICE;
    }
    if (!ctx->num_sms) {
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
        if (ctx->num_sms <= 0) ctx->num_sms = 1;
    }
    return HVX_SUCCESS;
}

hvx_status check_device_error(Context* ctx) {
    int v = 0;
    if (cudaMemcpy(&v, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_DEVICE;
    }
    if (v == 0) return HVX_SUCCESS;
    cudaMemset(ctx->d_error, 0, sizeof(int));
    return HVX_ERROR_TIMEOUT;
}

// Device result blocks of global operators (kept with the result image for
// the life of the graph) and EqualizeHist's histogram.
hvx_status alloc_results(Plan& P, Context* ctx) {
    for (int i : P.order) {
        Op& op = P.ops[i];
        if (op_is_global(op.kind)) {
            const uint64_t n = global_result_bytes(op.kind, op.node->p.hist_bins);
            if (op.out->dev && op.out->bytes != n) {
                ctx->pool.free(op.out->dev);
                op.out->dev = nullptr;
            }
            if (!op.out->dev) {
                hvx_status st = ctx->pool.alloc(n, &op.out->dev);
                if (st != HVX_SUCCESS) return st;
                op.out->owns_mem = true;
                op.out->bytes = n;
                cudaMemset(op.out->dev, global_result_fill(op.kind), n);
            }
        }
        if (op.kind == OP_EQHIST && !op.node->d_aux) {
            if (cudaMalloc(&op.node->d_aux, 256 * sizeof(uint32_t)) != cudaSuccess) {
                cudaGetLastError();
                return HVX_ERROR_NO_MEMORY;
            }
        }
    }
    return HVX_SUCCESS;
}

hvx_status prepare_launches(Graph* g) {
    Plan& P = g->plan;
    Context* ctx = g->ctx;
    bind_device(ctx);
    if (!ctx->plan_only) {
        hvx_status st = alloc_results(P, ctx);
        if (st != HVX_SUCCESS) return st;
    }
    // HVX_CODEGEN_ONLY: generated kernels in place of the hand-written ones
    const bool hand = g->codegen != HVX_CODEGEN_ONLY;
    const bool must_gen = g->codegen == HVX_CODEGEN_REQUIRE || g->codegen == HVX_CODEGEN_ONLY;
    for (Group& G : P.groups) {
        G.ext_bytes = G.mem_bytes = 0;
        for (Image* im : G.inputs) {
            G.mem_bytes += image_bytes(im);
            if (!im->is_virtual) G.ext_bytes += image_bytes(im);
        }
        for (Image* im : G.outputs) {
            G.mem_bytes += image_bytes(im);
            if (!im->is_virtual) G.ext_bytes += image_bytes(im);
        }
        hvx_status st;
        EdgeMatch em;
        HarrisMatch hm;
        const Op& first = P.ops[G.ops[0]];
        G.resets.clear();
        for (int i : G.ops) {
            const Op& op = P.ops[i];
            if (op_is_global(op.kind) && op.out->dev)
                G.resets.push_back({op.out->dev, global_result_fill(op.kind), op.out->bytes});
            if (op.kind == OP_EQHIST && op.node->d_aux)
                G.resets.push_back({op.node->d_aux, 0, 256 * sizeof(uint32_t)});
        }
        if (G.ops.size() == 1 && first.kind == OP_EQHIST) {
            G.kernel = GK_EQHIST;
            st = build_eqhist(P, G);
        } else if (hand && G.ops.size() == 1 && first.kind == OP_GAUSS &&
                   !border_wraps(first.node->border)) {
            G.kernel = GK_GAUSS;
            st = build_gauss(P, G, ctx);
        } else if (hand && G.ops.size() == 1 && is_binomial5(first)) {
            G.kernel = GK_BINOM5;
            st = build_binom5(P, G, ctx);
        } else if (G.ops.size() == 1 && first.kind == OP_CHX &&
                   first.node->p.channel != HVX_CHANNEL_Y) {
            G.kernel = GK_CHX_UV;
            st = build_point(P, G);
        } else if (G.ops.size() == 1 && !op_is_local(first.kind) && !op_is_global(first.kind) &&
                   first.kind != OP_USER_POINT) {
            G.kernel = GK_POINT;
            st = build_point(P, G);
        } else if (hand && match_edge(P, G, em)) {
            G.kernel = GK_EDGE;
            st = build_edge(P, G, em, ctx);
        } else if (hand && match_harris(P, G, hm)) {
            G.kernel = GK_HARRIS;
            st = build_harris(P, G, hm, ctx);
        } else {
            G.kernel = GK_GENERIC;
            st = build_generic(P, G);
            G.jit_on = false;
            // user-defined operators exist only as generated code
            const bool user = !G.user_code.empty();
            if (st == HVX_SUCCESS && user && g->codegen == HVX_CODEGEN_OFF)
                return HVX_ERROR_NOT_SUPPORTED;
            // plan-only contexts compile generated kernels only when asked to
            const bool gen = must_gen || (g->codegen == HVX_CODEGEN_AUTO && !ctx->plan_only);
            if (st == HVX_SUCCESS && gen) {
                std::string why;
                G.jit_on = jit_prepare(G.gdesc, G.user_code, !ctx->plan_only, ctx->device, &G.jit,
                                       &why);
                G.jit.p.err = ctx->d_error;
                if (!G.jit_on && getenv("HVX_CODEGEN_VERBOSE"))
                    fprintf(stderr, "hvx: no generated kernel for a group: %s\n", why.c_str());
                if (!G.jit_on && (must_gen || user))
                    return HVX_ERROR_NOT_SUPPORTED;
            }
        }
        if (st != HVX_SUCCESS) return st;
    }
    g->plan_id = ++g_plan_counter;
    return HVX_SUCCESS;
}

hvx_status launch_plan(Graph* g, cudaStream_t s) {
    if (fault_fires(HVX_FAULT_LAUNCH)) return HVX_ERROR_DEVICE;  // injected, nothing enqueued
    bind_device(g->ctx);
    for (Group& G : g->plan.groups) {
        NvtxRange nvtx(G.jit_on ? "hvx launch generated" : group_kernel_name(G.kernel));
        cudaError_t e = cudaSuccess;
        for (const ResultReset& r : G.resets) {
            e = cudaMemsetAsync(r.p, r.byte, r.n, s);
            if (e != cudaSuccess) return cuda_status(e);
        }
        switch (G.kernel) {
            case GK_EQHIST: e = launch_eqhist(G.eqh, s); break;
            case GK_GAUSS:
            case GK_BINOM5:
            case GK_EDGE: e = launch_edge(G.tmap, G.edge, s); break;
            case GK_HARRIS: e = launch_harris(G.tmap, G.harris, s); break;
            case GK_POINT:
            case GK_CHX_UV: e = launch_plain(G.plain, s); break;
            default: e = G.jit_on ? jit_launch(G.jit, s) : launch_generic(G.gdesc, s); break;
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    return HVX_SUCCESS;
}

// ---------------------------------------------------------------------------
// Batched persistent launch

struct BatchEntry {
    std::vector<Graph*> graphs;
    std::vector<uint64_t> plan_ids;
    void* dmem = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
    int grid = 0;  // persistent CTAs chosen by the autotuner
    // generated-kernel batches: one direct launch over every image's tiles
    JitKernel* jk = nullptr;
    int n = 0, total_tiles = 0;
    bool harris = false;  // BORDER_UNDEFINED corner batch: one direct launch
    bool tomasi = false;  // ... of the Shi-Tomasi kernel
    bool resp = false;    // ... where some image exports its response
    std::vector<int> rows;  // edge batch: rows per thread of each image's tiles
    std::vector<void*> more_dmem;  // edge batch split by size class: the other tables
};

struct BatchCache {
    std::vector<BatchEntry> entries;
    cudaStream_t capture = nullptr;
    uint64_t tick = 0;
};

void destroy_batch_cache(Context* ctx) {
    BatchCache* bc = ctx->batch;
    if (!bc) return;
    for (BatchEntry& e : bc->entries) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.dmem) cudaFree(e.dmem);
        for (void* p : e.more_dmem) cudaFree(p);
    }
    if (bc->capture) cudaStreamDestroy(bc->capture);
    delete bc;
    ctx->batch = nullptr;
}

namespace {

// Persistent grid size for one batch signature: every candidate (1 .. the
// occupancy limit of CTAs per SM) runs the batch twice on the internal
// stream after the caller's stream has drained, timed with events; the
// fastest is kept.  The batch's work is idempotent (every output pixel is
// rewritten with the same value), so the trial runs are harmless.
// HVX_AUTOTUNE=0 in the environment skips the trials and takes the
// occupancy limit.
int autotune_grid(Context* ctx, BatchCache* bc, const EdgeBatchDesc& d, int mode, cudaStream_t s,
                  int rows = EDGE_ROWS) {
    const int per_sm_max = std::max(1, edge_batch_blocks_per_sm(mode));
    int best = std::min(d.total_tiles, ctx->num_sms * per_sm_max);
    const char* env = std::getenv("HVX_AUTOTUNE");
    if ((env && env[0] == '0') || per_sm_max == 1) return best;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return best;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaEventDestroy(a);
        return best;
    }
    float best_ms = 1e30f;
    for (int per = 1; per <= per_sm_max; ++per) {
        int grid = std::min(d.total_tiles, ctx->num_sms * per);
        launch_edge_batch(d, mode, grid, bc->capture, rows);  // warm-up
        cudaEventRecord(a, bc->capture);
        launch_edge_batch(d, mode, grid, bc->capture, rows);
        launch_edge_batch(d, mode, grid, bc->capture, rows);
        cudaEventRecord(b, bc->capture);
        float ms = 0;
        if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess &&
            ms < best_ms) {
            best_ms = ms;
            best = grid;
        }
        cudaGetLastError();
        if (std::getenv("HVX_AUTOTUNE_VERBOSE"))
            std::fprintf(stderr, "hvx autotune: %d tiles, grid %d (%d CTAs/SM): %.4f ms\n",
                         d.total_tiles, grid, per, ms / 2);
        if (grid == d.total_tiles) break;  // more CTAs than tiles change nothing
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Device tables of one edge / Gaussian launch: per image its tensor map, its
// parameter block and its tile counts, for `rows` rows per thread (edge
// modes: tiles of 128 x 8R and boxes of 160 x (8R + 4); the Gaussian kernel
// keeps its own tile).  One device block; *d describes it.
hvx_status make_edge_tables(Context* ctx, Graph* const* gs, int n, int mode, int rows,
                            void** dmem_out, EdgeBatchDesc* d) {
    const size_t maps_bytes = (size_t)n * sizeof(CUtensorMap);
    const size_t params_off = maps_bytes;
    const size_t tiles_off = params_off + (size_t)n * sizeof(EdgeParams);
    const size_t tx_off = tiles_off + (size_t)(n + 1) * sizeof(int);
    const size_t total = tx_off + (size_t)n * sizeof(int);
    std::vector<uint8_t> host(total);
    std::vector<int> tile_start(n + 1, 0), tiles_x(n, 0);
    int tw = 0, th = 0;
    edge_tile_dims(mode, &tw, &th);
    if (mode != EDGE_MODE_GAUSS) th = 8 * rows;
    for (int i = 0; i < n; ++i) {
        const Group& G = gs[i]->plan.groups[0];
        EdgeParams ep = G.edge;
        {  // the batch kernel's box (the single-image map may be shorter)
            CUtensorMap map;
            hvx_status st;
            if (mode == EDGE_MODE_GAUSS) {
                st = encode_u8_map(&map, G.inputs[0], GAUSS_LOAD_W, GAUSS_LOAD_H);
            } else {  // 8R rows and the halo
                ep.rows = rows;
                st = encode_u8_map(&map, G.inputs[0], EDGE_LOAD_W, (uint32_t)(th + 4));
            }
            if (st != HVX_SUCCESS) return st;
            std::memcpy(host.data() + (size_t)i * sizeof(CUtensorMap), &map, sizeof(map));
        }
        std::memcpy(host.data() + params_off + (size_t)i * sizeof(EdgeParams), &ep, sizeof(ep));
        tiles_x[i] = (int)((G.W + tw - 1) / tw);
        const long long t = (long long)tile_start[i] + (long long)tiles_x[i] * ((G.H + th - 1) / th);
        if (t > (1ll << 30)) return HVX_ERROR_NOT_SUPPORTED;
        tile_start[i + 1] = (int)t;
    }
    std::memcpy(host.data() + tiles_off, tile_start.data(), (n + 1) * sizeof(int));
    std::memcpy(host.data() + tx_off, tiles_x.data(), n * sizeof(int));
    void* dmem = nullptr;
    cudaError_t e = cudaMalloc(&dmem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_NO_MEMORY;
    }
    e = cudaMemcpy(dmem, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dmem);
        return cuda_status(e);
    }
    d->maps = static_cast<const CUtensorMap*>(dmem);
    d->params = reinterpret_cast<const EdgeParams*>(static_cast<uint8_t*>(dmem) + params_off);
    d->tile_start = reinterpret_cast<const int*>(static_cast<uint8_t*>(dmem) + tiles_off);
    d->tiles_x = reinterpret_cast<const int*>(static_cast<uint8_t*>(dmem) + tx_off);
    d->n_img = n;
    d->total_tiles = tile_start[n];
    d->err = ctx->d_error;
    *dmem_out = dmem;
    return HVX_SUCCESS;
}

// Size classes of the tile-shape tuner, by image height: under 480 rows,
// under 1080 rows, and the rest.
int shape_class(uint32_t H) { return H < 480 ? 0 : H < 1080 ? 1 : 2; }

// Milliseconds of a sequence of launches (one warm-up, the mean of two) on
// the internal stream, or a huge value when it could not be timed.
struct EdgeLaunch {
    EdgeBatchDesc d;
    int rows = EDGE_ROWS;
    int grid = 0;
};

float time_launches(BatchCache* bc, const std::vector<EdgeLaunch>& ls, int mode) {
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = 1e30f;
    if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
        for (const EdgeLaunch& l : ls) launch_edge_batch(l.d, mode, l.grid, bc->capture, l.rows);
        cudaEventRecord(a, bc->capture);
        for (int rep = 0; rep < 2; ++rep)
            for (const EdgeLaunch& l : ls) launch_edge_batch(l.d, mode, l.grid, bc->capture, l.rows);
        cudaEventRecord(b, bc->capture);
        float t = 0;
        if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess)
            ms = t / 2;
    }
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return ms;
}

// One edge batch signature, tuned: either every image in one persistent
// launch with 128 x 120 tiles (R = 15 rows per thread), or one launch per
// image size class, each class with its own tile height.  The tuner times,
// for each class present, its own launch with R = 15, 10 and 5 (128 x 120 /
// 80 / 40 tiles: shorter tiles waste fewer rows on ragged heights and spread
// small images over more SMs, taller ones recompute fewer halo rows), then
// the whole split sequence against the single launch, keeping the split only
// when it is at least 2 % faster; then the persistent grid of each launch
// (autotune_grid).  The trials run on the internal stream after the caller's
// stream has drained; the batch's work is idempotent, so they are harmless.
// HVX_AUTOTUNE=0 or =grid keeps the single launch; HVX_BATCH_ROWS=R (5, 10,
// 15) gives every image 128 x 8R tiles in a single launch, without trials.
hvx_status build_batch_entry(Context* ctx, BatchCache* bc, Graph* const* gs, int n, int mode,
                             cudaStream_t user_stream, BatchEntry& out) {
    cudaError_t e;
    if (!bc->capture) {
        e = cudaStreamCreateWithFlags(&bc->capture, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_status(e);
    }
    const int grid_max = ctx->num_sms * std::max(1, edge_batch_blocks_per_sm(mode));
    std::vector<void*> blocks;
    auto release = [&] {
        for (void* p : blocks) cudaFree(p);
        blocks.clear();
    };
    // launches for a partition of the batch: parts[k] = image indices, rows[k]
    auto build = [&](const std::vector<std::vector<int>>& parts, const std::vector<int>& rows,
                     std::vector<EdgeLaunch>& ls) -> hvx_status {
        ls.clear();
        for (size_t k = 0; k < parts.size(); ++k) {
            std::vector<Graph*> sub;
            for (int i : parts[k]) sub.push_back(gs[i]);
            EdgeLaunch l;
            l.rows = rows[k];
            void* dm = nullptr;
            hvx_status st = make_edge_tables(ctx, sub.data(), (int)sub.size(), mode, l.rows, &dm,
                                             &l.d);
            if (st != HVX_SUCCESS) return st;
            blocks.push_back(dm);
            l.grid = std::min(l.d.total_tiles, grid_max);
            ls.push_back(l);
        }
        return HVX_SUCCESS;
    };
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    std::vector<std::vector<int>> parts = {all};
    std::vector<int> rows = {EDGE_ROWS};
    const char* env = std::getenv("HVX_AUTOTUNE");
    const char* fixed = std::getenv("HVX_BATCH_ROWS");
    const int fr = fixed ? std::atoi(fixed) : 0;
    if (fixed) {  // test / tuning knob
        static bool said = false;
        if (!said) {
            said = true;
            std::fprintf(stderr, "hvx: HVX_BATCH_ROWS=%s %s\n", fixed,
                         (fr == 5 || fr == 10 || fr == 15)
                             ? "fixes the rows per thread of every batched edge tile"
                             : "ignored (not 5, 10 or 15)");
        }
    }
    const bool verbose = std::getenv("HVX_AUTOTUNE_VERBOSE") != nullptr;
    if (mode != EDGE_MODE_GAUSS && (fr == 5 || fr == 10 || fr == 15)) {
        rows[0] = fr;
    } else if (mode != EDGE_MODE_GAUSS &&
               !(env && (env[0] == '0' || std::strcmp(env, "grid") == 0))) {
        std::vector<std::vector<int>> cls(3);
        for (int i = 0; i < n; ++i) cls[shape_class(gs[i]->plan.groups[0].H)].push_back(i);
        std::vector<std::vector<int>> split;
        for (auto& c : cls)
            if (!c.empty()) split.push_back(c);
        if (cudaStreamSynchronize(user_stream) == cudaSuccess) {
            std::vector<EdgeLaunch> ls;
            float t_single = 1e30f;
            if (build(parts, rows, ls) == HVX_SUCCESS) t_single = time_launches(bc, ls, mode);
            release();
            std::vector<int> split_rows;
            for (auto& part : split) {
                int best_r = EDGE_ROWS;
                float best = 1e30f;
                for (int r : {EDGE_ROWS, 10, 5}) {
                    float ms = 1e30f;
                    if (build({part}, {r}, ls) == HVX_SUCCESS) ms = time_launches(bc, ls, mode);
                    release();
                    if (verbose)
                        std::fprintf(stderr, "hvx autotune: class of %zu images, rows %d: %.4f ms\n",
                                     part.size(), r, ms);
                    if (ms < best) {
                        best = ms;
                        best_r = r;
                    }
                }
                split_rows.push_back(best_r);
            }
            float t_split = 1e30f;
            if (build(split, split_rows, ls) == HVX_SUCCESS) t_split = time_launches(bc, ls, mode);
            release();
            if (verbose)
                std::fprintf(stderr, "hvx autotune: one launch %.4f ms, per-class launches %.4f ms\n",
                             t_single, t_split);
            if (t_split < 0.98f * t_single) {
                parts = split;
                rows = split_rows;
            }
        }
        cudaGetLastError();
    }
    std::vector<EdgeLaunch> ls;
    hvx_status st = build(parts, rows, ls);
    if (st != HVX_SUCCESS) {
        release();
        return st;
    }
    for (EdgeLaunch& l : ls) l.grid = autotune_grid(ctx, bc, l.d, mode, user_stream, l.rows);
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(bc->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        for (const EdgeLaunch& l : ls) {
            cudaError_t x = launch_edge_batch(l.d, mode, l.grid, bc->capture, l.rows);
            if (le == cudaSuccess) le = x;
        }
        e = cudaStreamEndCapture(bc->capture, &graph);
        if (le != cudaSuccess) e = le;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release();
        return cuda_status(e);
    }
    out.graphs.assign(gs, gs + n);
    out.plan_ids.resize(n);
    for (int i = 0; i < n; ++i) out.plan_ids[i] = gs[i]->plan_id;
    out.dmem = blocks[0];
    out.more_dmem.assign(blocks.begin() + 1, blocks.end());
    out.exec = exec;
    out.grid = ls[0].grid;
    out.rows.assign(n, mode == EDGE_MODE_GAUSS ? 0 : EDGE_ROWS);
    if (mode != EDGE_MODE_GAUSS)
        for (size_t k = 0; k < parts.size(); ++k)
            for (int i : parts[k]) out.rows[i] = rows[k];
    return HVX_SUCCESS;
}

}  // namespace

// Batch of graphs whose plans are one group running the same generated
// kernel: the images' launch parameters and tile prefix sums in one device
// block.
hvx_status build_jit_batch_entry(Graph* const* gs, int n, JitKernel* jk, BatchEntry& out) {
    int tw = 0, th = 0;
    jit_tile(jk, &tw, &th);
    const size_t tiles_off = (size_t)n * sizeof(HvxJitParams);
    const size_t total = tiles_off + (size_t)(n + 1) * sizeof(int);
    std::vector<uint8_t> host(total);
    std::vector<int> tile_start(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const Group& G = gs[i]->plan.groups[0];
        std::memcpy(host.data() + (size_t)i * sizeof(HvxJitParams), &G.jit.p, sizeof(HvxJitParams));
        const long long t = (long long)tile_start[i] + (long long)G.jit.gx * G.jit.gy;
        if (t > (1ll << 30)) return HVX_ERROR_NOT_SUPPORTED;
        tile_start[i + 1] = (int)t;
    }
    std::memcpy(host.data() + tiles_off, tile_start.data(), (n + 1) * sizeof(int));
    void* dmem = nullptr;
    cudaError_t e = cudaMalloc(&dmem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_NO_MEMORY;
    }
    e = cudaMemcpy(dmem, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dmem);
        return cuda_status(e);
    }
    out.graphs.assign(gs, gs + n);
    out.plan_ids.resize(n);
    for (int i = 0; i < n; ++i) out.plan_ids[i] = gs[i]->plan_id;
    out.dmem = dmem;
    out.jk = jk;
    out.n = n;
    out.total_tiles = tile_start[n];
    return HVX_SUCCESS;
}

// Batch of BORDER_UNDEFINED Harris graphs: one rows-per-thread for all of
// them, each input's tensor map boxed for it, then maps, parameters and tile
// tables in one device block.
hvx_status build_harris_batch_entry(Context* ctx, Graph* const* gs, int n, BatchEntry& out) {
    std::vector<int> ws(n), hs(n);
    for (int i = 0; i < n; ++i) {
        ws[i] = (int)gs[i]->plan.groups[0].W;
        hs[i] = (int)gs[i]->plan.groups[0].H;
    }
    const int rows = harris_batch_rows(ws.data(), hs.data(), n, ctx->num_sms);
    const int tw = harris_fast_tile_w();
    const size_t params_off = (size_t)n * sizeof(CUtensorMap);
    const size_t tiles_off = params_off + (size_t)n * sizeof(HarrisParams);
    const size_t tx_off = tiles_off + (size_t)(n + 1) * sizeof(int);
    const size_t total = tx_off + (size_t)n * sizeof(int);
    std::vector<uint8_t> host(total);
    std::vector<int> tile_start(n + 1, 0), tiles_x(n, 0);
    for (int i = 0; i < n; ++i) {
        const Group& G = gs[i]->plan.groups[0];
        HarrisParams hp = G.harris;
        hp.rows = rows;
        int bw = 0, bh = 0;
        harris_box(hp, &bw, &bh);
        CUtensorMap map;
        hvx_status st = encode_u8_map(&map, G.inputs[0], bw, bh);
        if (st != HVX_SUCCESS) return st;
        std::memcpy(host.data() + (size_t)i * sizeof(CUtensorMap), &map, sizeof(map));
        std::memcpy(host.data() + params_off + (size_t)i * sizeof(HarrisParams), &hp, sizeof(hp));
        tiles_x[i] = (ws[i] + tw - 1) / tw;
        tile_start[i + 1] = tile_start[i] + tiles_x[i] * ((hs[i] + 8 * rows - 1) / (8 * rows));
    }
    std::memcpy(host.data() + tiles_off, tile_start.data(), (n + 1) * sizeof(int));
    std::memcpy(host.data() + tx_off, tiles_x.data(), n * sizeof(int));
    void* dmem = nullptr;
    cudaError_t e = cudaMalloc(&dmem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_NO_MEMORY;
    }
    e = cudaMemcpy(dmem, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dmem);
        return cuda_status(e);
    }
    out.graphs.assign(gs, gs + n);
    out.plan_ids.resize(n);
    for (int i = 0; i < n; ++i) out.plan_ids[i] = gs[i]->plan_id;
    out.dmem = dmem;
    out.harris = true;
    out.tomasi = gs[0]->plan.groups[0].harris.tomasi != 0;
    out.resp = false;
    for (int i = 0; i < n; ++i) out.resp = out.resp || gs[i]->plan.groups[0].harris.resp != nullptr;
    out.n = n;
    out.total_tiles = tile_start[n];
    return HVX_SUCCESS;
}

hvx_status query_batch(Context* ctx, Graph* const* gs, int n, int* rows, int* grid) {
    std::lock_guard<std::mutex> lock(ctx->batch_mu);
    if (!ctx->batch) return HVX_ERROR_INVALID_PARAMETERS;
    for (const BatchEntry& e : ctx->batch->entries) {
        if ((int)e.graphs.size() != n) continue;
        bool same = true;
        for (int i = 0; i < n && same; ++i)
            same = e.graphs[i] == gs[i] && e.plan_ids[i] == gs[i]->plan_id;
        if (!same) continue;
        for (int i = 0; i < n; ++i) rows[i] = (int)e.rows.size() == n ? e.rows[i] : 0;
        *grid = e.grid;
        return HVX_SUCCESS;
    }
    return HVX_ERROR_INVALID_PARAMETERS;
}

hvx_status process_batch(Context* ctx, Graph* const* gs, int n, cudaStream_t s) {
    NvtxRange nvtx("hvx batch");
    std::lock_guard<std::mutex> lock(ctx->batch_mu);
    bind_device(ctx);
    // one launch when every plan is a single group running the same
    // generated kernel
    JitKernel* jk = nullptr;
    bool jit_same = true;
    for (int i = 0; i < n && jit_same; ++i) {
        const Plan& P = gs[i]->plan;
        jit_same = P.groups.size() == 1 && P.groups[0].kernel == GK_GENERIC &&
                   P.groups[0].jit_on && (!jk || P.groups[0].jit.k == jk);
        if (jit_same) jk = P.groups[0].jit.k;
    }
    // one launch when every plan is a single BORDER_UNDEFINED corner group
    // with the same response (Harris or Shi-Tomasi)
    bool harris_same = !jit_same;
    for (int i = 0; i < n && harris_same; ++i) {
        const Plan& P = gs[i]->plan;
        harris_same = P.groups.size() == 1 && P.groups[0].kernel == GK_HARRIS &&
                      harris_fast_path(P.groups[0].harris) &&
                      P.groups[0].harris.tomasi == gs[0]->plan.groups[0].harris.tomasi;
    }
    // one persistent launch when every plan is a single edge (or Gaussian)
    // group and all of them use the same kernel mode
    bool same = !jit_same && !harris_same;
    int mode = -1;
    for (int i = 0; i < n && same; ++i) {
        const Plan& P = gs[i]->plan;
        same = P.groups.size() == 1 &&
               (P.groups[0].kernel == GK_EDGE || P.groups[0].kernel == GK_GAUSS ||
                P.groups[0].kernel == GK_BINOM5);
        if (same) {
            int m = edge_mode(P.groups[0].edge);
            same = mode < 0 || m == mode;
            mode = m;
        }
    }
    if (!same && !jit_same && !harris_same) {
        for (int i = 0; i < n; ++i) {
            hvx_status st = launch_plan(gs[i], s);
            if (st != HVX_SUCCESS) return st;
        }
        return HVX_SUCCESS;
    }
    if (!ctx->batch) ctx->batch = new BatchCache();
    BatchCache* bc = ctx->batch;
    BatchEntry* hit = nullptr;
    for (BatchEntry& e : bc->entries) {
        if ((int)e.graphs.size() != n) continue;
        bool same = true;
        for (int i = 0; i < n && same; ++i)
            same = e.graphs[i] == gs[i] && e.plan_ids[i] == gs[i]->plan_id;
        if (same) {
            hit = &e;
            break;
        }
    }
    if (!hit) {
        if (bc->entries.size() >= 16) {
            auto oldest = std::min_element(
                bc->entries.begin(), bc->entries.end(),
                [](const BatchEntry& a, const BatchEntry& b) { return a.last_use < b.last_use; });
            cudaStreamSynchronize(s);
            if (oldest->exec) cudaGraphExecDestroy(oldest->exec);
            if (oldest->dmem) cudaFree(oldest->dmem);
            for (void* p : oldest->more_dmem) cudaFree(p);
            bc->entries.erase(oldest);
        }
        BatchEntry fresh;
        hvx_status st = jit_same      ? build_jit_batch_entry(gs, n, jk, fresh)
                        : harris_same ? build_harris_batch_entry(ctx, gs, n, fresh)
                                      : build_batch_entry(ctx, bc, gs, n, mode, s, fresh);
        if (st != HVX_SUCCESS) return st;
        bc->entries.push_back(fresh);
        hit = &bc->entries.back();
    }
    hit->last_use = ++bc->tick;
    if (hit->jk) {
        for (int i = 0; i < n; ++i)
            for (const ResultReset& rr : gs[i]->plan.groups[0].resets) {
                cudaError_t e = cudaMemsetAsync(rr.p, rr.byte, rr.n, s);
                if (e != cudaSuccess) return cuda_status(e);
            }
        const uint8_t* base = static_cast<const uint8_t*>(hit->dmem);
        return cuda_status(jit_launch_batch(
            hit->jk, reinterpret_cast<const HvxJitParams*>(base),
            reinterpret_cast<const int*>(base + (size_t)hit->n * sizeof(HvxJitParams)), hit->n,
            hit->total_tiles, s));
    }
    if (hit->harris) {
        const uint8_t* base = static_cast<const uint8_t*>(hit->dmem);
        const size_t params_off = (size_t)hit->n * sizeof(CUtensorMap);
        const size_t tiles_off = params_off + (size_t)hit->n * sizeof(HarrisParams);
        const size_t tx_off = tiles_off + (size_t)(hit->n + 1) * sizeof(int);
        return cuda_status(launch_harris_batch(
            reinterpret_cast<const CUtensorMap*>(base),
            reinterpret_cast<const HarrisParams*>(base + params_off),
            reinterpret_cast<const int*>(base + tiles_off), reinterpret_cast<const int*>(base + tx_off),
            hit->n, hit->total_tiles, hit->tomasi, hit->resp, s));
    }
    return cuda_status(cudaGraphLaunch(hit->exec, s));
}

hvx_status encode_u8_map_raw(CUtensorMap* map, const void* ptr, uint64_t pitch, uint32_t w,
                             uint32_t h, uint32_t box_w, uint32_t box_h) {
    return encode_u8_map_at(map, ptr, pitch, w, h, box_w, box_h);
}

}  // namespace hvx
