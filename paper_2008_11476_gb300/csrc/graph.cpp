// Graph verification and planning (Section 3.1, Section 5.2).
//
//  1. lower every CV-function node to single-output point / local ops
//     (Section 4: Sobel3x3 is two parallel local operators);
//  2. check parameters, single writers, bipartite edges and cycles;
//  3. resolve virtual image sizes and formats in dependency order;
//  4. dead-computation elimination, Algorithm 1 (Section 5.2.2);
//  5. valid regions;
//  6. fusion planning: group ops into kernels, keeping intermediates on chip
//     (the data-transfer reduction of Section 5.2.1 carried down to the
//     memory hierarchy: virtual images inside a group never reach HBM);
//  7. allocate device memory for virtual images that cross groups.
#include <algorithm>
#include <climits>
#include <functional>
#include <set>
#include <unordered_map>
#include <unordered_set>

#include "hvx_internal.h"

namespace hvx {

int bytes_per_pixel(int fmt) {
    switch (fmt) {
        case HVX_DF_U8: return 1;
        case HVX_DF_S16: return 2;
        case HVX_DF_S32: return 4;
        case HVX_DF_F32: return 4;
        case HVX_DF_UYVY: return 2;
    }
    return 0;
}

Rect rect_intersect(const Rect& a, const Rect& b) {
    Rect r;
    r.x0 = std::max(a.x0, b.x0);
    r.y0 = std::max(a.y0, b.y0);
    r.x1 = std::max(r.x0, std::min(a.x1, b.x1));
    r.y1 = std::max(r.y0, std::min(a.y1, b.y1));
    return r;
}

const char* op_name(int kind) {
    switch (kind) {
        case OP_GAUSS: return "gaussian3x3";
        case OP_BOX: return "box3x3";
        case OP_SOBEL_X: return "sobel_x";
        case OP_SOBEL_Y: return "sobel_y";
        case OP_MAG: return "magnitude";
        case OP_PHASE: return "phase";
        case OP_THRESH: return "threshold";
        case OP_CHX: return "channel_extract";
        case OP_ADD: return "add";
        case OP_SUB: return "subtract";
        case OP_ABSDIFF: return "absdiff";
        case OP_MUL: return "mul";
        case OP_HARRIS: return "harris_response";
        case OP_LSUM: return "window_sum";
        case OP_CONV: return "convolve";
        case OP_DILATE: return "dilate3x3";
        case OP_ERODE: return "erode3x3";
        case OP_MEDIAN: return "median3x3";
        case OP_AND: return "and";
        case OP_OR: return "or";
        case OP_XOR: return "xor";
        case OP_NOT: return "not";
        case OP_TOMASI: return "tomasi_response";
        case OP_MULTIPLY: return "multiply";
        case OP_MEANSTD: return "mean_stddev";
        case OP_MINMAX: return "minmaxloc";
        case OP_HIST: return "histogram";
        case OP_EQHIST: return "equalize_hist";
        case OP_CONVDEPTH: return "convert_depth";
        case OP_USER_POINT: return "user_point";
        case OP_USER_LOCAL: return "user_local";
    }
    return "?";
}

bool op_is_local(int kind) {
    return kind == OP_GAUSS || kind == OP_BOX || kind == OP_SOBEL_X || kind == OP_SOBEL_Y ||
           kind == OP_LSUM || kind == OP_CONV || kind == OP_DILATE || kind == OP_ERODE ||
           kind == OP_MEDIAN || kind == OP_USER_LOCAL;
}

const char* group_kernel_name(int gk) {
    switch (gk) {
        case GK_GENERIC: return "staged_tile";
        case GK_GAUSS: return "gaussian3x3_tma";
        case GK_EDGE: return "fused_edge_tma";
        case GK_BINOM5: return "binomial5x5_tma";
        case GK_HARRIS: return "fused_harris_tma";
        case GK_POINT: return "plain_point";
        case GK_CHX_UV: return "plain_channel_uv";
        case GK_EQHIST: return "equalize_hist";
    }
    return "?";
}

namespace {

struct VerifyError {
    hvx_status st;
};

[[noreturn]] void fail(hvx_status st) { throw VerifyError{st}; }

bool is_int_fmt(int f) { return f == HVX_DF_U8 || f == HVX_DF_S16 || f == HVX_DF_S32; }

// ---- 1. lowering ---------------------------------------------------------------
void lower(Graph* g, Plan& P) {
    for (auto& up : g->nodes) {
        Node* n = up.get();
        n->live_mask = 0;
        n->group = -1;
        auto add = [&](int kind, int out_index, int r) {
            Op op;
            op.kind = kind;
            op.node = n;
            op.out_index = out_index;
            op.n_in = (int)n->in.size();
            for (int i = 0; i < op.n_in; ++i) op.in[i] = n->in[i];
            op.out = n->out[out_index];
            op.rx = op.ry = r;
            P.ops.push_back(op);
        };
        for (Image* im : n->in)
            if (!im) fail(HVX_ERROR_INVALID_PARAMETERS);
        switch (n->kind) {
            case N_GAUSS: add(OP_GAUSS, 0, 1); break;
            case N_BOX: add(OP_BOX, 0, 1); break;
            case N_DILATE: add(OP_DILATE, 0, 1); break;
            case N_ERODE: add(OP_ERODE, 0, 1); break;
            case N_MEDIAN: add(OP_MEDIAN, 0, 1); break;
            case N_AND: add(OP_AND, 0, 0); break;
            case N_OR: add(OP_OR, 0, 0); break;
            case N_XOR: add(OP_XOR, 0, 0); break;
            case N_NOT: add(OP_NOT, 0, 0); break;
            case N_MULTIPLY: add(OP_MULTIPLY, 0, 0); break;
            case N_MEANSTD: add(OP_MEANSTD, 0, 0); break;
            case N_MINMAX: add(OP_MINMAX, 0, 0); break;
            case N_HIST: add(OP_HIST, 0, 0); break;
            case N_EQHIST: add(OP_EQHIST, 0, 0); break;
            case N_COPY:
            case N_CONVDEPTH: add(OP_CONVDEPTH, 0, 0); break;
            case N_USER_POINT: add(OP_USER_POINT, 0, 0); break;
            case N_USER_LOCAL: {
                add(OP_USER_LOCAL, 0, 0);
                P.ops.back().rx = n->p.kw / 2;
                P.ops.back().ry = n->p.kh / 2;
                break;
            }
            case N_SOBEL:
                if (!n->out[0] && !n->out[1]) fail(HVX_ERROR_INVALID_PARAMETERS);
                if (n->out[0]) add(OP_SOBEL_X, 0, 1);
                if (n->out[1]) add(OP_SOBEL_Y, 1, 1);
                break;
            case N_MAG: add(OP_MAG, 0, 0); break;
            case N_PHASE: add(OP_PHASE, 0, 0); break;
            case N_THRESH: add(OP_THRESH, 0, 0); break;
            case N_CHX: add(OP_CHX, 0, 0); break;
            case N_ADD: add(OP_ADD, 0, 0); break;
            case N_SUB: add(OP_SUB, 0, 0); break;
            case N_ABSDIFF: add(OP_ABSDIFF, 0, 0); break;
            case N_CONV: {
                add(OP_CONV, 0, 0);
                P.ops.back().rx = n->p.kw / 2;
                P.ops.back().ry = n->p.kh / 2;
                break;
            }
            case N_POINT:
                add(n->p.custom_op == HVX_POINT_MUL      ? OP_MUL
                    : n->p.custom_op == HVX_POINT_TOMASI_RESPONSE ? OP_TOMASI
                                                             : OP_HARRIS,
                    0, 0);
                break;
            case N_LOCAL: {
                add(OP_LSUM, 0, 0);
                P.ops.back().rx = n->p.kw / 2;
                P.ops.back().ry = n->p.kh / 2;
                break;
            }
            default: fail(HVX_ERROR_INVALID_PARAMETERS);
        }
    }
    for (Op& op : P.ops)
        if (!op.out) fail(HVX_ERROR_INVALID_PARAMETERS);
}

// ---- 3. format / size resolution ---------------------------------------------------
void infer(Op& op) {
    Image* const* in = op.in;
    auto need = [&](int i, std::initializer_list<int> fmts) {
        for (int f : fmts)
            if (in[i]->fmt == f) return;
        fail(HVX_ERROR_INVALID_FORMAT);
    };
    int of = 0;
    uint32_t ow = in[0]->w, oh = in[0]->h;
    switch (op.kind) {
        case OP_GAUSS:
        case OP_BOX:
        case OP_DILATE:
        case OP_ERODE:
        case OP_MEDIAN:
        case OP_NOT: need(0, {HVX_DF_U8}); of = HVX_DF_U8; break;
        case OP_AND:
        case OP_OR:
        case OP_XOR: need(0, {HVX_DF_U8}); need(1, {HVX_DF_U8}); of = HVX_DF_U8; break;
        case OP_SOBEL_X:
        case OP_SOBEL_Y: need(0, {HVX_DF_U8}); of = HVX_DF_S16; break;
        case OP_CONV: {
            need(0, {HVX_DF_U8});
            const int declared = op.out->is_virtual ? op.out->user_fmt : op.out->fmt;
            of = declared == HVX_DF_U8 ? HVX_DF_U8 : HVX_DF_S16;
            break;
        }
        case OP_LSUM: need(0, {HVX_DF_S32}); of = HVX_DF_S32; break;
        case OP_MAG: need(0, {HVX_DF_S16}); need(1, {HVX_DF_S16}); of = HVX_DF_S16; break;
        case OP_PHASE: need(0, {HVX_DF_S16}); need(1, {HVX_DF_S16}); of = HVX_DF_U8; break;
        case OP_THRESH: {
            need(0, {HVX_DF_U8, HVX_DF_S16, HVX_DF_S32, HVX_DF_F32});
            of = HVX_DF_U8;
            const NodeParams& p = op.node->p;
            if (is_int_fmt(in[0]->fmt)) {
                if (p.thr_value != (double)(int64_t)p.thr_value) fail(HVX_ERROR_INVALID_PARAMETERS);
                if (p.thr_type == HVX_THRESHOLD_RANGE &&
                    p.thr_upper != (double)(int64_t)p.thr_upper)
                    fail(HVX_ERROR_INVALID_PARAMETERS);
            }
            break;
        }
        case OP_CHX:
            need(0, {HVX_DF_UYVY});
            of = HVX_DF_U8;
            if (in[0]->w & 1) fail(HVX_ERROR_INVALID_PARAMETERS);
            if (op.node->p.channel != HVX_CHANNEL_Y) ow = in[0]->w / 2;
            break;
        case OP_ADD:
        case OP_SUB:
        case OP_ABSDIFF:
        case OP_MULTIPLY: {
            need(0, {HVX_DF_U8, HVX_DF_S16});
            need(1, {HVX_DF_U8, HVX_DF_S16});
            bool any16 = in[0]->fmt == HVX_DF_S16 || in[1]->fmt == HVX_DF_S16;
            int declared = op.out->is_virtual ? op.out->user_fmt : op.out->fmt;
            if (declared == HVX_DF_U8 || declared == HVX_DF_S16)
                of = declared;
            else
                of = any16 ? HVX_DF_S16 : HVX_DF_U8;
            if (of == HVX_DF_U8 && any16) fail(HVX_ERROR_INVALID_FORMAT);
            break;
        }
        case OP_MUL: need(0, {HVX_DF_S16}); need(1, {HVX_DF_S16}); of = HVX_DF_S32; break;
        case OP_HARRIS:
        case OP_TOMASI:
            need(0, {HVX_DF_S32});
            need(1, {HVX_DF_S32});
            need(2, {HVX_DF_S32});
            of = HVX_DF_F32;
            break;
        case OP_MEANSTD:
        case OP_MINMAX: need(0, {HVX_DF_U8, HVX_DF_S16}); of = HVX_DF_RESULT; break;
        case OP_HIST: need(0, {HVX_DF_U8}); of = HVX_DF_RESULT; break;
        case OP_EQHIST: need(0, {HVX_DF_U8}); of = HVX_DF_U8; break;
        case OP_USER_POINT:
        case OP_USER_LOCAL: {
            // integer inputs; the output image declares U8, S16 or S32
            for (int i = 0; i < op.n_in; ++i) need(i, {HVX_DF_U8, HVX_DF_S16, HVX_DF_S32});
            of = op.out->is_virtual ? op.out->user_fmt : op.out->fmt;
            if (of != HVX_DF_U8 && of != HVX_DF_S16 && of != HVX_DF_S32)
                fail(HVX_ERROR_INVALID_FORMAT);
            break;
        }
        case OP_CONVDEPTH: {
            // Copy keeps the format; ConvertDepth goes U8 <-> S16
            need(0, {HVX_DF_U8, HVX_DF_S16});
            if (op.node->kind == N_COPY)
                of = in[0]->fmt;
            else
                of = in[0]->fmt == HVX_DF_U8 ? HVX_DF_S16 : HVX_DF_U8;
            break;
        }
        default: fail(HVX_ERROR_INVALID_PARAMETERS);
    }
    if (op.kind != OP_CHX)
        for (int i = 1; i < op.n_in; ++i)
            if (in[i]->w != ow || in[i]->h != oh) fail(HVX_ERROR_INVALID_PARAMETERS);
    if (ow == 0 || oh == 0) fail(HVX_ERROR_INVALID_PARAMETERS);
    Image* o = op.out;
    if (o->is_virtual || o->is_result) {
        if (o->user_fixed_size && (o->w != ow || o->h != oh)) fail(HVX_ERROR_INVALID_PARAMETERS);
        if (o->user_fmt != HVX_DF_VIRT && o->user_fmt != of) fail(HVX_ERROR_INVALID_FORMAT);
        o->w = ow;
        o->h = oh;
        o->fmt = of;
    } else {
        if (o->w != ow || o->h != oh) fail(HVX_ERROR_INVALID_PARAMETERS);
        if (o->fmt != of) fail(HVX_ERROR_INVALID_FORMAT);
    }
}

// ---- 4. Algorithm 1 ---------------------------------------------------------------
// Vertices: images (D) and ops (N).  Edges image -> op for every input, op ->
// image for the output.
void eliminate_dead(Plan& P) {
    std::unordered_map<Image*, int> deg_in, deg_out;
    std::unordered_map<Image*, int> writer;
    std::set<Image*> images;
    for (size_t i = 0; i < P.ops.size(); ++i) {
        Op& op = P.ops[i];
        for (int k = 0; k < op.n_in; ++k) {
            deg_out[op.in[k]]++;
            images.insert(op.in[k]);
        }
        deg_in[op.out]++;
        writer[op.out] = (int)i;
        images.insert(op.out);
    }
    // candidate non-virtual roots (D_in) and leaves (D_out)
    std::set<Image*> D_in, D_out;
    for (Image* v : images) {
        if (v->is_virtual) continue;
        if (deg_in[v] == 0) {
            D_in.insert(v);
        } else if (deg_out[v] == 0) {
            D_out.insert(v);
        } else {
            D_in.insert(v);
            D_out.insert(v);
        }
    }
    // depth-first visits of the transposed graph from every leaf; a root other
    // than the start vertex ends its branch
    std::vector<char> op_alive(P.ops.size(), 0);
    for (Image* start : D_out) {
        std::unordered_set<Image*> seen_img{start};
        std::vector<Image*> stack{start};
        while (!stack.empty()) {
            Image* v = stack.back();
            stack.pop_back();
            if (v != start && D_in.count(v)) continue;
            auto w = writer.find(v);
            if (w == writer.end()) continue;
            Op& op = P.ops[w->second];
            op_alive[w->second] = 1;
            for (int k = 0; k < op.n_in; ++k)
                if (seen_img.insert(op.in[k]).second) stack.push_back(op.in[k]);
        }
    }
    for (size_t i = 0; i < P.ops.size(); ++i) {
        P.ops[i].alive = op_alive[i] != 0;
        if (P.ops[i].alive) P.ops[i].node->live_mask |= 1u << P.ops[i].out_index;
    }
}

// ---- 6. fusion planning ------------------------------------------------------------
struct Planner {
    Plan& P;
    bool fusion;
    std::unordered_map<Image*, int> writer;  // image -> op index (alive ops)

    explicit Planner(Plan& p, bool f) : P(p), fusion(f) {}

    // halo of every image inside group `gi` if op `extra` were added
    bool halos(const std::vector<int>& ops, std::unordered_map<Image*, int>& h_img) const {
        std::set<Image*> produced;
        for (int i : ops) produced.insert(P.ops[i].out);
        std::unordered_map<int, int> h_out;  // op -> halo of its output
        for (auto it = ops.rbegin(); it != ops.rend(); ++it) {
            const Op& op = P.ops[*it];
            if (op.out->is_result) continue;  // no pixels
            int h = 0;
            for (int j : ops) {
                const Op& c = P.ops[j];
                for (int k = 0; k < c.n_in; ++k)
                    if (c.in[k] == op.out) h = std::max(h, h_out[j] + std::max(c.rx, c.ry));
            }
            h_out[*it] = h;
            h_img[op.out] = std::max(h_img[op.out], h);
        }
        for (int j : ops) {
            const Op& c = P.ops[j];
            for (int k = 0; k < c.n_in; ++k)
                if (!produced.count(c.in[k]))
                    h_img[c.in[k]] = std::max(h_img[c.in[k]], h_out[j] + std::max(c.rx, c.ry));
        }
        for (auto& kv : h_img)
            if (kv.second > GEN_MAX_HALO) return false;
        return true;
    }

    bool fits_generic(const std::vector<int>& ops) const {
        std::unordered_map<Image*, int> h;
        if (!halos(ops, h)) return false;
        if ((int)ops.size() > GEN_MAX_STAGE || (int)h.size() > GEN_MAX_BUF) return false;
        std::set<Image*> produced;
        for (int i : ops) produced.insert(P.ops[i].out);
        int n_in = 0;
        for (auto& kv : h)
            if (!produced.count(kv.first)) ++n_in;
        // images the group would write: non-virtual ones, and those read by
        // alive ops outside the group
        std::set<int> members(ops.begin(), ops.end());
        int n_out = 0;
        int n_global = 0;
        for (int i : ops) n_global += op_is_global(P.ops[i].kind) ? 1 : 0;
        if (n_global > HVX_JIT_MAX_RES) return false;
        for (Image* im : produced) {
            if (im->is_result) continue;
            bool out = !im->is_virtual;
            for (int j : P.order)
                if (!members.count(j))
                    for (int k = 0; k < P.ops[j].n_in; ++k) out |= P.ops[j].in[k] == im;
            n_out += out;
        }
        if (n_in > GEN_MAX_EXT || n_out > GEN_MAX_EXT) return false;
        long words = 0;
        for (auto& kv : h) words += (long)(GEN_TW + 2 * kv.second) * (GEN_TH + 2 * kv.second);
        int coeffs = 0;
        for (int i : ops)
            if (P.ops[i].kind == OP_CONV) coeffs += (int)P.ops[i].node->p.coeffs.size();
        return words * 4 <= 200 * 1024 && coeffs <= GEN_MAX_COEFF;
    }

    // local consumers of one image must agree on how they read it outside the image
    bool border_compatible(const std::vector<int>& ops, const Op& o) const {
        if (!op_is_local(o.kind)) return true;
        for (int j : ops) {
            const Op& c = P.ops[j];
            if (!op_is_local(c.kind)) continue;
            for (int k = 0; k < c.n_in; ++k)
                for (int m = 0; m < o.n_in; ++m)
                    if (c.in[k] == o.in[m] &&
                        (c.node->border != o.node->border ||
                         (c.node->border == HVX_BORDER_CONSTANT && c.node->cval != o.node->cval)))
                        return false;
        }
        return true;
    }

    void run() {
        std::vector<int> op_group(P.ops.size(), -1);
        std::unordered_map<Node*, int> node_group;
        for (int i : P.order) {
            Op& op = P.ops[i];
            int target = -1;
            if (!fusion) {
                auto it = node_group.find(op.node);
                if (it != node_group.end()) target = it->second;
            } else {
                // ops that run alone: U/V extraction changes the size, and
                // EqualizeHist needs its whole histogram before any output
                bool size_change = (op.kind == OP_CHX && op.node->p.channel != HVX_CHANNEL_Y) ||
                                   op.kind == OP_EQHIST;
                // a MIRROR / REPEAT local op reads its inputs from memory, like
                // external inputs, whoever produces them
                const bool wraps = op_is_local(op.kind) && border_wraps(op.node->border);
                std::set<int> prod_groups;
                for (int k = 0; k < op.n_in && !wraps; ++k) {
                    auto w = writer.find(op.in[k]);
                    if (w != writer.end()) prod_groups.insert(op_group[w->second]);
                }
                // a global operator on an external image runs on its own
                // rather than joining a group that merely reads that image
                if (prod_groups.empty() && !op_is_global(op.kind)) {
                    // only external inputs: join the group of a sibling op of the
                    // same node (the two Sobel derivatives), else the latest group
                    // that already reads one of these inputs, so the input is read
                    // from memory once
                    auto it = node_group.find(op.node);
                    if (it != node_group.end()) {
                        prod_groups.insert(it->second);
                    } else {
                        for (int gi = (int)P.groups.size() - 1; gi >= 0 && prod_groups.empty();
                             --gi)
                            for (int j : P.groups[gi].ops)
                                for (int k = 0; k < P.ops[j].n_in; ++k)
                                    for (int m = 0; m < op.n_in; ++m)
                                        if (P.ops[j].in[k] == op.in[m]) prod_groups.insert(gi);
                    }
                }
                if (!size_change && prod_groups.size() == 1) {
                    int gi = *prod_groups.begin();
                    Group& G = P.groups[gi];
                    bool same_size = G.W == op.out->w && G.H == op.out->h;
                    // MIRROR / REPEAT read pixels anywhere in the input: never
                    // from a tile of the producer fused into the same kernel
                    if (op_is_local(op.kind) && border_wraps(op.node->border))
                        for (int j : G.ops)
                            for (int k = 0; k < op.n_in; ++k)
                                if (P.ops[j].out == op.in[k]) same_size = false;
                    std::vector<int> trial = G.ops;
                    trial.push_back(i);
                    if (!G.closed && same_size && border_compatible(G.ops, op) &&
                        fits_generic(trial))
                        target = gi;
                }
            }
            if (target < 0) {
                P.groups.emplace_back();
                target = (int)P.groups.size() - 1;
                P.groups[target].W = op.out->w;
                P.groups[target].H = op.out->h;
                P.groups[target].closed =
                    (op.kind == OP_CHX && op.node->p.channel != HVX_CHANNEL_Y) ||
                    op.kind == OP_EQHIST;
                node_group[op.node] = target;
            }
            P.groups[target].ops.push_back(i);
            if (!node_group.count(op.node)) node_group[op.node] = target;
            op_group[i] = target;
            op.group = target;
            if (op.node->group < 0) op.node->group = target;
        }
        // inputs / outputs of every group
        for (size_t gi = 0; gi < P.groups.size(); ++gi) {
            Group& G = P.groups[gi];
            std::set<Image*> produced;
            for (int i : G.ops) produced.insert(P.ops[i].out);
            std::set<Image*> seen_in;
            for (int i : G.ops) {
                const Op& op = P.ops[i];
                for (int k = 0; k < op.n_in; ++k)
                    if (!produced.count(op.in[k]) && seen_in.insert(op.in[k]).second)
                        G.inputs.push_back(op.in[k]);
            }
            for (int i : G.ops) {
                Image* o = P.ops[i].out;
                if (o->is_result) continue;
                bool needed = !o->is_virtual;
                for (int j : P.order)
                    if (op_group[j] != (int)gi)
                        for (int k = 0; k < P.ops[j].n_in; ++k)
                            if (P.ops[j].in[k] == o) needed = true;
                if (needed) G.outputs.push_back(o);
            }
        }
    }
};

void compute_valid(Plan& P) {
    std::set<Image*> produced;
    for (int i : P.order) produced.insert(P.ops[i].out);
    for (int i : P.order)
        for (int k = 0; k < P.ops[i].n_in; ++k) {
            Image* im = P.ops[i].in[k];
            if (!produced.count(im)) im->valid = Rect{0, 0, (int)im->w, (int)im->h};
        }
    for (int i : P.order) {
        Op& op = P.ops[i];
        Rect r;
        if (op.kind == OP_CHX) {
            r = Rect{0, 0, (int)op.out->w, (int)op.out->h};
        } else {
            r = op.in[0]->valid;
            for (int k = 1; k < op.n_in; ++k) r = rect_intersect(r, op.in[k]->valid);
            if (op_is_local(op.kind) && op.node->border == HVX_BORDER_UNDEFINED) {
                r.x0 += op.rx;
                r.y0 += op.ry;
                r.x1 -= op.rx;
                r.y1 -= op.ry;
                if (r.x1 < r.x0) r.x1 = r.x0;
                if (r.y1 < r.y0) r.y1 = r.y0;
            }
        }
        op.out->valid = r;
    }
}

}  // namespace

void release_plan(Graph* g) {
    for (Image* im : g->plan.materialized) {
        if (im->dev && im->owns_mem) g->ctx->pool.free(im->dev);
        im->dev = nullptr;
        im->pitch = 0;
        im->owns_mem = false;
        im->materialized = false;
    }
    g->plan = Plan();
    g->verified = false;
}

hvx_status verify_graph(Graph* g) {
    NvtxRange nvtx("hvx verify");
    release_plan(g);
    Plan& P = g->plan;
    try {
        // reset virtual images to what the user declared
        for (Image* v : g->virtuals) {
            if (!v->user_fixed_size) v->w = v->h = 0;
            v->fmt = v->user_fmt;
        }
        lower(g, P);
        // presence, ownership
        for (Op& op : P.ops) {
            for (int k = 0; k < op.n_in; ++k) {
                Image* im = op.in[k];
                if (im->magic != kMagicImage || im->ctx != g->ctx) fail(HVX_ERROR_INVALID_REFERENCE);
                if (im->is_virtual && im->owner_graph != g) fail(HVX_ERROR_INVALID_REFERENCE);
            }
            if (op.out->magic != kMagicImage || op.out->ctx != g->ctx)
                fail(HVX_ERROR_INVALID_REFERENCE);
            if (op.out->is_virtual && op.out->owner_graph != g) fail(HVX_ERROR_INVALID_REFERENCE);
        }
        // single writer per image
        std::unordered_map<Image*, int> writer;
        for (size_t i = 0; i < P.ops.size(); ++i) {
            if (writer.count(P.ops[i].out)) fail(HVX_ERROR_INVALID_GRAPH);
            writer[P.ops[i].out] = (int)i;
        }
        // bipartite edges: every edge joins an image and an op (Section 5.2).
        // The object model only links ops to images, so this holds by
        // construction; an op that reads its own output is the one way to
        // break it and is rejected as a cycle below.
        // cycles: Kahn's algorithm over op -> op dependencies
        std::vector<int> indeg(P.ops.size(), 0);
        std::vector<std::vector<int>> succ(P.ops.size());
        for (size_t j = 0; j < P.ops.size(); ++j)
            for (int k = 0; k < P.ops[j].n_in; ++k) {
                Image* im = P.ops[j].in[k];
                auto w = writer.find(im);
                if (w != writer.end()) {
                    succ[w->second].push_back((int)j);
                    indeg[j]++;
                } else if (im->is_virtual) {
                    fail(HVX_ERROR_INVALID_GRAPH);  // virtual image read but never written
                }
            }
        std::vector<int> topo, ready;
        for (size_t i = 0; i < P.ops.size(); ++i)
            if (indeg[i] == 0) ready.push_back((int)i);
        while (!ready.empty()) {
            int i = ready.front();
            ready.erase(ready.begin());
            topo.push_back(i);
            for (int j : succ[i])
                if (--indeg[j] == 0) ready.push_back(j);
        }
        if (topo.size() != P.ops.size()) fail(HVX_ERROR_INVALID_GRAPH);
        // parameter ranges
        for (Op& op : P.ops) {
            const NodeParams& p = op.node->p;
            if (op_is_local(op.kind)) {
                int b = op.node->border;
                if (b < HVX_BORDER_UNDEFINED || b > HVX_BORDER_REPEAT)
                    fail(HVX_ERROR_INVALID_PARAMETERS);
            }
            if (op.kind == OP_HARRIS && (p.kd < 1 || p.kd > 1000 || p.kn < 0 || p.kn > 1000))
                fail(HVX_ERROR_INVALID_PARAMETERS);
        }
        for (int i : topo) infer(P.ops[i]);
        eliminate_dead(P);
        for (int i : topo)
            if (P.ops[i].alive) P.order.push_back(i);
        compute_valid(P);
        Planner pl(P, g->fusion);
        for (int i : P.order) pl.writer[P.ops[i].out] = i;
        pl.run();
    } catch (const VerifyError& e) {
        g->plan = Plan();
        return e.st;
    }
    // memory for virtual images that cross group boundaries
    for (Group& G : P.groups)
        for (Image* o : G.outputs)
            if (o->is_virtual && !o->dev) {
                uint64_t pitch = ((uint64_t)o->w * bytes_per_pixel(o->fmt) + 127) / 128 * 128;
                if (g->ctx->plan_only) {
                    o->pitch = pitch;
                    o->bytes = pitch * o->h;
                    P.intermediate_bytes += o->bytes;
                    continue;
                }
                void* p = nullptr;
                hvx_status st = g->ctx->pool.alloc(pitch * o->h, &p);
                if (st != HVX_SUCCESS) {
                    release_plan(g);
                    return st;
                }
                o->dev = p;
                o->pitch = pitch;
                o->owns_mem = true;
                o->materialized = true;
                o->bytes = pitch * o->h;
                P.materialized.push_back(o);
                P.intermediate_bytes += o->bytes;
            }
    hvx_status st = prepare_launches(g);
    if (st != HVX_SUCCESS) {
        release_plan(g);
        return st;
    }
    P.kernel_kinds.clear();
    P.external_bytes = 0;
    for (Group& G : P.groups) {
        if (!P.kernel_kinds.empty()) P.kernel_kinds += ",";
        P.kernel_kinds += group_kernel_name(G.kernel);
        P.external_bytes += G.ext_bytes;
    }
    g->verified = true;
    return HVX_SUCCESS;
}

}  // namespace hvx
