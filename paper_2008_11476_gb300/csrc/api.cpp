// C ABI of the image-graph library: handle checks, object ownership and the
// node constructors (Section 3.1, Listing 1; Section 5.1, Listing 4).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <new>

#include "hvx_internal.h"

using namespace hvx;

namespace hvx {

hvx_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return HVX_SUCCESS;
    if (e == cudaErrorMemoryAllocation) return HVX_ERROR_NO_MEMORY;
    return HVX_ERROR_DEVICE;
}

// ---------------------------------------------------------------------------
// Host-side fault injection: a countdown per kind; the call that brings it
// from 1 to 0 fails.  0 = disarmed.
namespace {
std::atomic<int64_t> g_fault_count[3];
}

bool fault_fires(int kind) {
    std::atomic<int64_t>& c = g_fault_count[kind];
    int64_t v = c.load();
    while (v > 0)
        if (c.compare_exchange_weak(v, v - 1)) return v == 1;
    return false;
}

// ---------------------------------------------------------------------------
DevicePool::~DevicePool() {
    for (auto& kv : live_) cudaFree(kv.first);
    for (auto& kv : cache_) cudaFree(kv.second);
}

hvx_status DevicePool::alloc(uint64_t bytes, void** out) {
    std::lock_guard<std::mutex> lk(mu_);
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    // reuse a cached block of the same size
    auto it = cache_.find(bytes);
    if (it != cache_.end()) {
        void* p = it->second;
        cache_.erase(it);
        live_[p] = bytes;
        in_use_ += bytes;
        *out = p;
        return HVX_SUCCESS;
    }
    if (budget_ && in_use_ + bytes > budget_) return HVX_ERROR_OVER_BUDGET;
    // return cached blocks to the driver until the new block fits the budget
    while (budget_ && held_ + bytes > budget_ && !cache_.empty()) {
        auto c = cache_.begin();
        cudaFree(c->second);
        held_ -= c->first;
        cache_.erase(c);
    }
    void* p = nullptr;
    if (fault_fires(HVX_FAULT_DEVICE_ALLOC)) return HVX_ERROR_NO_MEMORY;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // retry once after emptying the cache
        for (auto& kv : cache_) {
            cudaFree(kv.second);
            held_ -= kv.first;
        }
        cache_.clear();
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return HVX_ERROR_NO_MEMORY;
        }
    }
    live_[p] = bytes;
    in_use_ += bytes;
    held_ += bytes;
    *out = p;
    return HVX_SUCCESS;
}

void DevicePool::free(void* p) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = live_.find(p);
    if (it == live_.end()) return;
    in_use_ -= it->second;
    cache_.emplace(it->second, p);
    live_.erase(it);
}

void DevicePool::trim() {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& kv : cache_) {
        cudaFree(kv.second);
        held_ -= kv.first;
    }
    cache_.clear();
}

}  // namespace hvx

namespace {

bool ok_ctx(hvx_context c) { return c && reinterpret_cast<Context*>(c)->magic == kMagicContext; }
bool ok_graph(hvx_graph g) { return g && reinterpret_cast<Graph*>(g)->magic == kMagicGraph; }
bool ok_image(hvx_image i) { return i && reinterpret_cast<Image*>(i)->magic == kMagicImage; }
bool ok_node(hvx_node n) { return n && reinterpret_cast<Node*>(n)->magic == kMagicNode; }

Context* C(hvx_context c) { return reinterpret_cast<Context*>(c); }
Graph* G(hvx_graph g) { return reinterpret_cast<Graph*>(g); }
Image* I(hvx_image i) { return reinterpret_cast<Image*>(i); }
Node* N(hvx_node n) { return reinterpret_cast<Node*>(n); }

bool valid_fmt(int f) { return f >= HVX_DF_U8 && f <= HVX_DF_UYVY; }

void destroy_image(Image* im) {
    if (im->dev && im->owns_mem) im->ctx->pool.free(im->dev);
    im->magic = 0;
    delete im;
}

void maybe_destroy(Image* im) {
    if (im->user_refs <= 0 && im->node_refs <= 0 && !im->is_virtual) {
        auto& v = im->ctx->images;
        v.erase(std::remove(v.begin(), v.end(), im), v.end());
        destroy_image(im);
    }
}

void destroy_graph(Graph* g) {
    if (g->scheduled && g->done) cudaEventSynchronize(g->done);
    release_plan(g);
    for (auto& n : g->nodes) {
        if (n->d_aux) cudaFree(n->d_aux);
        n->d_aux = nullptr;
        for (Image* im : n->in)
            if (im && !im->is_virtual) im->node_refs--;
        for (Image* im : n->out)
            if (im && !im->is_virtual) im->node_refs--;
        n->magic = 0;
    }
    g->nodes.clear();
    for (Image* v : g->virtuals) destroy_image(v);
    g->virtuals.clear();
    if (g->done) cudaEventDestroy(g->done);
    g->magic = 0;
    Context* ctx = g->ctx;
    auto& gv = ctx->graphs;
    gv.erase(std::remove(gv.begin(), gv.end(), g), gv.end());
    delete g;
    // images that were only kept alive by this graph's nodes
    std::vector<Image*> imgs = ctx->images;
    for (Image* im : imgs) maybe_destroy(im);
}

// A node is added only if every image argument is a live image of the
// graph's context (virtual images must belong to the graph itself).
bool image_usable(Graph* g, Image* im) {
    if (!ok_image(reinterpret_cast<hvx_image>(im))) return false;
    if (im->ctx != g->ctx) return false;
    if (im->is_virtual && im->owner_graph != g) return false;
    return true;
}

hvx_node add_node(hvx_graph hg, int kind, std::initializer_list<hvx_image> ins,
                  std::initializer_list<hvx_image> outs, int required_outs, const NodeParams& p) {
    if (!ok_graph(hg)) return nullptr;
    Graph* g = G(hg);
    std::unique_ptr<Node> n(new (std::nothrow) Node());
    if (!n) {
        g->last = HVX_ERROR_NO_MEMORY;
        return nullptr;
    }
    for (hvx_image h : ins) {
        if (!h || !image_usable(g, I(h))) {
            g->last = HVX_ERROR_INVALID_REFERENCE;
            return nullptr;
        }
        n->in.push_back(I(h));
    }
    int k = 0;
    for (hvx_image h : outs) {
        if (!h) {
            if (k < required_outs) {
                g->last = HVX_ERROR_INVALID_REFERENCE;
                return nullptr;
            }
            n->out.push_back(nullptr);
        } else {
            if (!image_usable(g, I(h))) {
                g->last = HVX_ERROR_INVALID_REFERENCE;
                return nullptr;
            }
            n->out.push_back(I(h));
        }
        ++k;
    }
    n->graph = g;
    n->kind = kind;
    n->p = p;
    for (Image* im : n->in)
        if (!im->is_virtual) im->node_refs++;
    for (Image* im : n->out)
        if (im && !im->is_virtual) im->node_refs++;
    Node* raw = n.get();
    g->nodes.push_back(std::move(n));
    release_plan(g);
    g->last = HVX_SUCCESS;
    return reinterpret_cast<hvx_node>(raw);
}

hvx_status set_last(Graph* g, hvx_status st) {
    g->last = st;
    return st;
}

}  // namespace

extern "C" {

const char* hvxStatusString(hvx_status s) {
    switch (s) {
        case HVX_SUCCESS: return "HVX_SUCCESS";
        case HVX_ERROR_INVALID_REFERENCE: return "HVX_ERROR_INVALID_REFERENCE";
        case HVX_ERROR_INVALID_PARAMETERS: return "HVX_ERROR_INVALID_PARAMETERS";
        case HVX_ERROR_INVALID_FORMAT: return "HVX_ERROR_INVALID_FORMAT";
        case HVX_ERROR_INVALID_GRAPH: return "HVX_ERROR_INVALID_GRAPH";
        case HVX_ERROR_NOT_VERIFIED: return "HVX_ERROR_NOT_VERIFIED";
        case HVX_ERROR_NO_MEMORY: return "HVX_ERROR_NO_MEMORY";
        case HVX_ERROR_OVER_BUDGET: return "HVX_ERROR_OVER_BUDGET";
        case HVX_ERROR_TIMEOUT: return "HVX_ERROR_TIMEOUT";
        case HVX_ERROR_DEVICE: return "HVX_ERROR_DEVICE";
        case HVX_ERROR_NOT_SUPPORTED: return "HVX_ERROR_NOT_SUPPORTED";
    }
    return "HVX_UNKNOWN_STATUS";
}

hvx_status hvxCreateContext(hvx_context* out) { return hvxCreateContextEx(0, out); }

hvx_status hvxCreateContextEx(int32_t flags, hvx_context* out) {
    if (!out || (flags & ~HVX_CONTEXT_PLAN_ONLY)) return HVX_ERROR_INVALID_PARAMETERS;
    Context* c = new (std::nothrow) Context();
    if (!c) return HVX_ERROR_NO_MEMORY;
    if (flags & HVX_CONTEXT_PLAN_ONLY) {
        c->plan_only = true;
        *out = reinterpret_cast<hvx_context>(c);
        return HVX_SUCCESS;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return HVX_ERROR_DEVICE;
    }
    hvx_status st = ensure_context_device_state(c);
    if (st != HVX_SUCCESS) {
        delete c;
        return st;
    }
    *out = reinterpret_cast<hvx_context>(c);
    return HVX_SUCCESS;
}

hvx_status hvxReleaseContext(hvx_context* pc) {
    if (!pc || !ok_ctx(*pc)) return HVX_ERROR_INVALID_REFERENCE;
    Context* c = C(*pc);
    if (!c->plan_only) cudaDeviceSynchronize();
    std::vector<Server*> servers = c->servers;
    for (Server* s : servers) server_destroy(s);
    std::vector<Graph*> graphs = c->graphs;
    for (Graph* g : graphs) destroy_graph(g);
    std::vector<Image*> images = c->images;
    for (Image* im : images) destroy_image(im);
    c->images.clear();
    destroy_batch_cache(c);
    if (c->d_error) cudaFree(c->d_error);
    for (cudaEvent_t e : c->io_events) cudaEventDestroy(e);
    if (c->io_in) cudaStreamDestroy(c->io_in);
    if (c->io_out) cudaStreamDestroy(c->io_out);
    c->magic = 0;
    delete c;
    *pc = nullptr;
    return HVX_SUCCESS;
}

hvx_status hvxSetContextMemoryBudget(hvx_context ctx, uint64_t bytes) {
    if (!ok_ctx(ctx)) return HVX_ERROR_INVALID_REFERENCE;
    C(ctx)->pool.set_budget(bytes);
    return HVX_SUCCESS;
}

hvx_status hvxGetContextMemoryUsage(hvx_context ctx, uint64_t* bytes) {
    if (!ok_ctx(ctx)) return HVX_ERROR_INVALID_REFERENCE;
    if (!bytes) return HVX_ERROR_INVALID_PARAMETERS;
    *bytes = C(ctx)->pool.in_use();
    return HVX_SUCCESS;
}

// ---- images -----------------------------------------------------------------

hvx_status hvxCreateImage(hvx_context ctx, uint32_t w, uint32_t h, int32_t fmt, hvx_image* out) {
    if (!ok_ctx(ctx)) return HVX_ERROR_INVALID_REFERENCE;
    if (!out || w == 0 || h == 0 || w > 32768u || h > 32768u)
        return HVX_ERROR_INVALID_PARAMETERS;
    if (!valid_fmt(fmt)) return HVX_ERROR_INVALID_FORMAT;
    if (fmt == HVX_DF_UYVY && (w & 1)) return HVX_ERROR_INVALID_PARAMETERS;
    Context* c = C(ctx);
    Image* im = new (std::nothrow) Image();
    if (!im) return HVX_ERROR_NO_MEMORY;
    im->ctx = c;
    im->w = w;
    im->h = h;
    im->fmt = fmt;
    im->pitch = ((uint64_t)w * bytes_per_pixel(fmt) + 127) / 128 * 128;
    im->bytes = im->pitch * h;
    if (!c->plan_only) {
        hvx_status st = c->pool.alloc(im->bytes, &im->dev);
        if (st != HVX_SUCCESS) {
            delete im;
            return st;
        }
        im->owns_mem = true;
    }
    im->valid = Rect{0, 0, (int)w, (int)h};
    c->images.push_back(im);
    *out = reinterpret_cast<hvx_image>(im);
    return HVX_SUCCESS;
}

hvx_status hvxCreateImageFromHandle(hvx_context ctx, uint32_t w, uint32_t h, int32_t fmt,
                                    void* dev_ptr, uint64_t pitch, hvx_image* out) {
    if (!ok_ctx(ctx)) return HVX_ERROR_INVALID_REFERENCE;
    if (!out || !dev_ptr || w == 0 || h == 0 || w > 32768u || h > 32768u)
        return HVX_ERROR_INVALID_PARAMETERS;
    if (!valid_fmt(fmt)) return HVX_ERROR_INVALID_FORMAT;
    if (fmt == HVX_DF_UYVY && (w & 1)) return HVX_ERROR_INVALID_PARAMETERS;
    if (((uintptr_t)dev_ptr & 15) || (pitch & 15) || pitch < (uint64_t)w * bytes_per_pixel(fmt))
        return HVX_ERROR_INVALID_PARAMETERS;
    Image* im = new (std::nothrow) Image();
    if (!im) return HVX_ERROR_NO_MEMORY;
    im->ctx = C(ctx);
    im->w = w;
    im->h = h;
    im->fmt = fmt;
    im->dev = dev_ptr;
    im->pitch = pitch;
    im->bytes = pitch * h;
    im->owns_mem = false;
    im->valid = Rect{0, 0, (int)w, (int)h};
    C(ctx)->images.push_back(im);
    *out = reinterpret_cast<hvx_image>(im);
    return HVX_SUCCESS;
}

hvx_status hvxSwapImageHandle(hvx_image img, void* dev_ptr, uint64_t pitch) {
    if (!ok_image(img)) return HVX_ERROR_INVALID_REFERENCE;
    Image* im = I(img);
    if (im->is_virtual || im->owns_mem) return HVX_ERROR_INVALID_REFERENCE;
    if (!dev_ptr || ((uintptr_t)dev_ptr & 15) || (pitch & 15) ||
        pitch < (uint64_t)im->w * bytes_per_pixel(im->fmt))
        return HVX_ERROR_INVALID_PARAMETERS;
    im->dev = dev_ptr;
    im->pitch = pitch;
    im->bytes = pitch * im->h;
    // launch parameters embed addresses and pitches: rebuild them for every
    // verified graph that uses the image
    for (Graph* g : im->ctx->graphs) {
        if (!g->verified) continue;
        bool uses = false;
        for (auto& n : g->nodes) {
            for (Image* x : n->in) uses |= x == im;
            for (Image* x : n->out) uses |= x == im;
        }
        if (uses) {
            if (g->scheduled) cudaEventSynchronize(g->done);
            hvx_status st = prepare_launches(g);
            if (st != HVX_SUCCESS) {
                release_plan(g);
                return st;
            }
        }
    }
    return HVX_SUCCESS;
}

hvx_status hvxCreateVirtualImage(hvx_graph hg, uint32_t w, uint32_t h, int32_t fmt,
                                 hvx_image* out) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    if (!out || (w == 0) != (h == 0)) return HVX_ERROR_INVALID_PARAMETERS;
    if (fmt != HVX_DF_VIRT && !valid_fmt(fmt)) return HVX_ERROR_INVALID_FORMAT;
    Graph* g = G(hg);
    Image* im = new (std::nothrow) Image();
    if (!im) return HVX_ERROR_NO_MEMORY;
    im->ctx = g->ctx;
    im->owner_graph = g;
    im->is_virtual = true;
    im->w = w;
    im->h = h;
    im->user_fixed_size = w != 0;
    im->fmt = fmt;
    im->user_fmt = fmt;
    g->virtuals.push_back(im);
    *out = reinterpret_cast<hvx_image>(im);
    return HVX_SUCCESS;
}

hvx_status hvxReleaseImage(hvx_image* pimg) {
    if (!pimg || !ok_image(*pimg)) return HVX_ERROR_INVALID_REFERENCE;
    Image* im = I(*pimg);
    *pimg = nullptr;
    if (im->is_virtual) return HVX_SUCCESS;  // owned by its graph
    im->user_refs--;
    maybe_destroy(im);
    return HVX_SUCCESS;
}

hvx_status hvxCopyImage(hvx_image img, void* host, uint64_t host_pitch, int32_t usage) {
    if (!ok_image(img)) return HVX_ERROR_INVALID_REFERENCE;
    Image* im = I(img);
    if (im->is_virtual) return HVX_ERROR_INVALID_REFERENCE;
    if (im->ctx->plan_only) return HVX_ERROR_NOT_SUPPORTED;
    uint64_t row = (uint64_t)im->w * bytes_per_pixel(im->fmt);
    if (!host || host_pitch < row) return HVX_ERROR_INVALID_PARAMETERS;
    cudaError_t e;
    if (usage == HVX_READ)
        e = cudaMemcpy2D(host, host_pitch, im->dev, im->pitch, row, im->h, cudaMemcpyDeviceToHost);
    else if (usage == HVX_WRITE)
        e = cudaMemcpy2D(im->dev, im->pitch, host, host_pitch, row, im->h, cudaMemcpyHostToDevice);
    else
        return HVX_ERROR_INVALID_PARAMETERS;
    return cuda_status(e);
}

}  // extern "C"

namespace hvx {

// Host-side copies of one batch call.  Consecutive copies whose images follow
// one another in device memory and whose host buffers follow one another too
// (same row size and pitches, e.g. frames of one tensor) are merged into one
// 2-D copy of all their rows.
hvx_status host_copies(std::vector<const hvx_host_copy*> copies, bool to_device, cudaStream_t s) {
    // in device-address order, so that images adjacent in memory meet
    std::stable_sort(copies.begin(), copies.end(),
                     [](const hvx_host_copy* a, const hvx_host_copy* b) {
                         return I(a->image)->dev < I(b->image)->dev;
                     });
    struct Run {
        char* dev;
        char* host;
        uint64_t dpitch, hpitch, row, rows;
    };
    std::vector<Run> runs;
    for (const hvx_host_copy* c : copies) {
        const Image* im = I(c->image);
        Run r{static_cast<char*>(im->dev), static_cast<char*>(c->host), im->pitch, c->pitch,
              (uint64_t)im->w * bytes_per_pixel(im->fmt), im->h};
        if (!runs.empty()) {
            Run& b = runs.back();
            if (b.dpitch == r.dpitch && b.hpitch == r.hpitch && b.row == r.row &&
                b.dev + b.rows * b.dpitch == r.dev && b.host + b.rows * b.hpitch == r.host) {
                b.rows += r.rows;
                continue;
            }
        }
        runs.push_back(r);
    }
    for (const Run& r : runs) {
        cudaError_t e = to_device ? cudaMemcpy2DAsync(r.dev, r.dpitch, r.host, r.hpitch, r.row,
                                                      r.rows, cudaMemcpyHostToDevice, s)
                                  : cudaMemcpy2DAsync(r.host, r.hpitch, r.dev, r.dpitch, r.row,
                                                      r.rows, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return HVX_SUCCESS;
}

hvx_status check_host_copies(const Context* ctx, const hvx_host_copy* copies, int32_t n) {
    if (n < 0 || (n > 0 && !copies)) return HVX_ERROR_INVALID_PARAMETERS;
    for (int32_t i = 0; i < n; ++i) {
        const hvx_host_copy& c = copies[i];
        if (!ok_image(c.image) || !c.host) return HVX_ERROR_INVALID_PARAMETERS;
        const Image* im = I(c.image);
        if (im->is_virtual || im->is_result || im->ctx != ctx || !im->dev)
            return HVX_ERROR_INVALID_REFERENCE;
        if (c.pitch < (uint64_t)im->w * bytes_per_pixel(im->fmt)) return HVX_ERROR_INVALID_PARAMETERS;
    }
    return HVX_SUCCESS;
}

// Whether graph g reads (inputs) or writes (outputs) image im from memory.
static bool graph_touches(const Graph* g, const Image* im, bool inputs) {
    for (const Group& G : g->plan.groups)
        for (const Image* x : inputs ? G.inputs : G.outputs)
            if (x == im) return true;
    return false;
}

}  // namespace hvx

extern "C" {

hvx_status hvxScheduleGraphBatchHost(const hvx_graph* gs, int32_t n, const hvx_host_copy* copies,
                                     int32_t n_copies, void* stream) {
    if (!gs || n <= 0 || n_copies < 0 || (n_copies > 0 && !copies))
        return HVX_ERROR_INVALID_PARAMETERS;
    std::vector<Graph*> v;
    for (int i = 0; i < n; ++i) {
        if (!ok_graph(gs[i])) return HVX_ERROR_INVALID_REFERENCE;
        if (!G(gs[i])->verified) return HVX_ERROR_NOT_VERIFIED;
        if (G(gs[i])->ctx != G(gs[0])->ctx) return HVX_ERROR_INVALID_REFERENCE;
        v.push_back(G(gs[i]));
    }
    Context* ctx = v[0]->ctx;
    if (ctx->plan_only) return HVX_ERROR_NOT_SUPPORTED;
    hvx_status vs = check_host_copies(ctx, copies, n_copies);
    if (vs != HVX_SUCCESS) return vs;
    std::lock_guard<std::mutex> lock(ctx->io_mu);
    // A pipeline over parts of the batch: part j's uploads (copy stream in),
    // its launches (the caller's stream), its downloads (copy stream out), so
    // that part j + 1's uploads and part j - 1's downloads overlap part j's
    // kernels.  Uploads are paced: part j's begin once part j - 2's downloads
    // have begun, so that they spread over the downloads instead of taking
    // the shared host link while the downloads (the larger direction for
    // graphs with more output than input bytes) wait.  The caller's stream
    // waits for the last download at the end.
    const int parts = std::min(n, 8);
    if (!ctx->io_in && (cudaStreamCreateWithFlags(&ctx->io_in, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&ctx->io_out, cudaStreamNonBlocking) != cudaSuccess))
        return HVX_ERROR_DEVICE;
    while ((int)ctx->io_events.size() < 3 * parts + 2) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HVX_ERROR_DEVICE;
        ctx->io_events.push_back(e);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t start = ctx->io_events[0];
    cudaError_t e = cudaEventRecord(start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_in, start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->io_out, start, 0);
    if (e != cudaSuccess) return cuda_status(e);
    // each copy goes with the first part whose graphs read / write its image
    std::vector<std::vector<const hvx_host_copy*>> up(parts), down(parts);
    for (int32_t i = 0; i < n_copies; ++i) {
        const hvx_host_copy& c = copies[i];
        const Image* im = I(c.image);
        int part = c.to_device ? 0 : parts - 1;
        for (int j = 0; j < parts; ++j) {
            const int a = (int)((int64_t)n * j / parts), b = (int)((int64_t)n * (j + 1) / parts);
            bool hit = false;
            for (int k = a; k < b && !hit; ++k) hit = graph_touches(v[k], im, c.to_device != 0);
            if (hit) {
                part = j;
                break;
            }
        }
        (c.to_device ? up : down)[part].push_back(&c);
    }
    for (int j = 0; j < parts; ++j) {
        const int a = (int)((int64_t)n * j / parts), b = (int)((int64_t)n * (j + 1) / parts);
        cudaEvent_t uploaded = ctx->io_events[1 + 3 * j], computed = ctx->io_events[2 + 3 * j];
        cudaEvent_t downloading = ctx->io_events[3 + 3 * j];
        if (j >= 2 && (e = cudaStreamWaitEvent(ctx->io_in, ctx->io_events[3 + 3 * (j - 2)], 0)) !=
                          cudaSuccess)
            return cuda_status(e);
        hvx_status st = host_copies(up[j], true, ctx->io_in);
        if (st != HVX_SUCCESS) return st;
        if ((e = cudaEventRecord(uploaded, ctx->io_in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, uploaded, 0)) != cudaSuccess)
            return cuda_status(e);
        st = process_batch(ctx, v.data() + a, b - a, s);
        if (st != HVX_SUCCESS) return st;
        if ((e = cudaEventRecord(computed, s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->io_out, computed, 0)) != cudaSuccess ||
            (e = cudaEventRecord(downloading, ctx->io_out)) != cudaSuccess)
            return cuda_status(e);
        st = host_copies(down[j], false, ctx->io_out);
        if (st != HVX_SUCCESS) return st;
    }
    cudaEvent_t done = ctx->io_events[3 * parts + 1];
    if ((e = cudaEventRecord(done, ctx->io_out)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, done, 0)) != cudaSuccess)
        return cuda_status(e);
    return HVX_SUCCESS;
}

hvx_status hvxGetImageDevicePtr(hvx_image img, void** dev, uint64_t* pitch) {
    if (!ok_image(img)) return HVX_ERROR_INVALID_REFERENCE;
    Image* im = I(img);
    if (im->is_virtual) return HVX_ERROR_INVALID_REFERENCE;
    if (!dev || !pitch) return HVX_ERROR_INVALID_PARAMETERS;
    *dev = im->dev;
    *pitch = im->pitch;
    return HVX_SUCCESS;
}

hvx_status hvxQueryImage(hvx_image img, uint32_t* w, uint32_t* h, int32_t* fmt) {
    if (!ok_image(img)) return HVX_ERROR_INVALID_REFERENCE;
    Image* im = I(img);
    if (w) *w = im->w;
    if (h) *h = im->h;
    if (fmt) *fmt = im->fmt;
    return HVX_SUCCESS;
}

hvx_status hvxGetValidRegion(hvx_image img, hvx_rect* r) {
    if (!ok_image(img)) return HVX_ERROR_INVALID_REFERENCE;
    if (!r) return HVX_ERROR_INVALID_PARAMETERS;
    Image* im = I(img);
    r->start_x = im->valid.x0;
    r->start_y = im->valid.y0;
    r->end_x = im->valid.x1;
    r->end_y = im->valid.y1;
    return HVX_SUCCESS;
}

// ---- graphs -----------------------------------------------------------------------

hvx_status hvxCreateGraph(hvx_context ctx, hvx_graph* out) {
    if (!ok_ctx(ctx)) return HVX_ERROR_INVALID_REFERENCE;
    if (!out) return HVX_ERROR_INVALID_PARAMETERS;
    Graph* g = new (std::nothrow) Graph();
    if (!g) return HVX_ERROR_NO_MEMORY;
    g->ctx = C(ctx);
    if (!g->ctx->plan_only &&
        cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return HVX_ERROR_DEVICE;
    }
    C(ctx)->graphs.push_back(g);
    *out = reinterpret_cast<hvx_graph>(g);
    return HVX_SUCCESS;
}

hvx_status hvxReleaseGraph(hvx_graph* pg) {
    if (!pg || !ok_graph(*pg)) return HVX_ERROR_INVALID_REFERENCE;
    destroy_graph(G(*pg));
    *pg = nullptr;
    return HVX_SUCCESS;
}

hvx_status hvxVerifyGraph(hvx_graph hg) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    Graph* g = G(hg);
    if (g->busy.load()) return set_last(g, HVX_ERROR_INVALID_GRAPH);
    if (g->scheduled) {
        cudaEventSynchronize(g->done);
        g->scheduled = false;
    }
    return set_last(g, verify_graph(g));
}

hvx_status hvxScheduleGraph(hvx_graph hg, void* stream) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    Graph* g = G(hg);
    if (!g->verified) return set_last(g, HVX_ERROR_NOT_VERIFIED);
    if (g->ctx->plan_only) return set_last(g, HVX_ERROR_NOT_SUPPORTED);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    hvx_status st = launch_plan(g, s);
    if (st != HVX_SUCCESS) return set_last(g, st);
    if (cudaEventRecord(g->done, s) != cudaSuccess) {
        cudaGetLastError();
        return set_last(g, HVX_ERROR_DEVICE);
    }
    g->scheduled = true;
    g->last_stream = s;
    return HVX_SUCCESS;
}

hvx_status hvxWaitGraph(hvx_graph hg) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    Graph* g = G(hg);
    if (!g->scheduled) return HVX_SUCCESS;
    cudaError_t e = cudaEventSynchronize(g->done);
    g->scheduled = false;
    if (e != cudaSuccess) return set_last(g, cuda_status(e));
    return set_last(g, check_device_error(g->ctx));
}

hvx_status hvxProcessGraph(hvx_graph hg) {
    hvx_status st = hvxScheduleGraph(hg, nullptr);
    if (st != HVX_SUCCESS) return st;
    return hvxWaitGraph(hg);
}

hvx_status hvxSetGraphFusion(hvx_graph hg, int32_t enable) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    Graph* g = G(hg);
    g->fusion = enable != 0;
    release_plan(g);
    return HVX_SUCCESS;
}

hvx_status hvxSetGraphCodegen(hvx_graph hg, int32_t mode) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    if (mode < HVX_CODEGEN_OFF || mode > HVX_CODEGEN_ONLY) return HVX_ERROR_INVALID_PARAMETERS;
    Graph* g = G(hg);
    g->codegen = mode;
    release_plan(g);
    return HVX_SUCCESS;
}

int64_t hvxGetGraphKernelSource(hvx_graph hg, int32_t group, char* buf, uint64_t size) {
    if (!ok_graph(hg)) return -1;
    Graph* g = G(hg);
    if (!g->verified || group < 0 || group >= (int32_t)g->plan.groups.size()) return -1;
    const Group& gr = g->plan.groups[group];
    if (!gr.jit_on) return -1;
    const std::string& s = jit_source(gr.jit);
    if (buf && size > 0) {
        const uint64_t n = std::min<uint64_t>(size - 1, s.size());
        std::memcpy(buf, s.data(), n);
        buf[n] = '\0';
    }
    return (int64_t)s.size();
}

hvx_status hvxGetGraphStatus(hvx_graph hg) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    return G(hg)->last;
}

hvx_status hvxQueryGraph(hvx_graph hg, int32_t attr, void* out, uint64_t size) {
    if (!ok_graph(hg)) return HVX_ERROR_INVALID_REFERENCE;
    Graph* g = G(hg);
    if (!out) return HVX_ERROR_INVALID_PARAMETERS;
    auto put32 = [&](int32_t v) {
        if (size < 4) return HVX_ERROR_INVALID_PARAMETERS;
        std::memcpy(out, &v, 4);
        return HVX_SUCCESS;
    };
    auto put64 = [&](uint64_t v) {
        if (size < 8) return HVX_ERROR_INVALID_PARAMETERS;
        std::memcpy(out, &v, 8);
        return HVX_SUCCESS;
    };
    switch (attr) {
        case HVX_GRAPH_NUM_NODES: return put32((int32_t)g->nodes.size());
        case HVX_GRAPH_FUSION: return put32(g->fusion ? 1 : 0);
        default: break;
    }
    if (!g->verified) return HVX_ERROR_NOT_VERIFIED;
    switch (attr) {
        case HVX_GRAPH_NUM_OPS: return put32((int32_t)g->plan.ops.size());
        case HVX_GRAPH_NUM_ALIVE_OPS: return put32((int32_t)g->plan.order.size());
        case HVX_GRAPH_NUM_LAUNCHES: return put32((int32_t)g->plan.groups.size());
        case HVX_GRAPH_INTERMEDIATE_BYTES: return put64(g->plan.intermediate_bytes);
        case HVX_GRAPH_EXTERNAL_BYTES: return put64(g->plan.external_bytes);
        case HVX_GRAPH_GENERATED_KERNELS: {
            int32_t n = 0;
            for (const Group& gr : g->plan.groups) n += gr.jit_on ? 1 : 0;
            return put32(n);
        }
        case HVX_GRAPH_KERNEL_KINDS: {
            const std::string& s = g->plan.kernel_kinds;
            if (size < s.size() + 1) return HVX_ERROR_INVALID_PARAMETERS;
            std::memcpy(out, s.c_str(), s.size() + 1);
            return HVX_SUCCESS;
        }
    }
    return HVX_ERROR_INVALID_PARAMETERS;
}

hvx_status hvxProcessGraphBatch(const hvx_graph* gs, int32_t n, void* stream) {
    if (!gs || n <= 0) return HVX_ERROR_INVALID_PARAMETERS;
    std::vector<Graph*> v;
    for (int i = 0; i < n; ++i) {
        if (!ok_graph(gs[i])) return HVX_ERROR_INVALID_REFERENCE;
        if (!G(gs[i])->verified) return HVX_ERROR_NOT_VERIFIED;
        if (G(gs[i])->ctx != G(gs[0])->ctx) return HVX_ERROR_INVALID_REFERENCE;
        v.push_back(G(gs[i]));
    }
    if (v[0]->ctx->plan_only) return HVX_ERROR_NOT_SUPPORTED;
    return process_batch(v[0]->ctx, v.data(), n, reinterpret_cast<cudaStream_t>(stream));
}

hvx_status hvxQueryBatch(const hvx_graph* gs, int32_t n, int32_t* rows_out, int32_t* grid_out) {
    if (!gs || n <= 0 || !rows_out || !grid_out) return HVX_ERROR_INVALID_PARAMETERS;
    std::vector<Graph*> v;
    for (int i = 0; i < n; ++i) {
        if (!ok_graph(gs[i])) return HVX_ERROR_INVALID_REFERENCE;
        if (G(gs[i])->ctx != G(gs[0])->ctx) return HVX_ERROR_INVALID_REFERENCE;
        v.push_back(G(gs[i]));
    }
    std::vector<int> rows(n);
    int grid = 0;
    hvx_status st = query_batch(v[0]->ctx, v.data(), n, rows.data(), &grid);
    if (st != HVX_SUCCESS) return st;
    for (int i = 0; i < n; ++i) rows_out[i] = rows[i];
    *grid_out = grid;
    return HVX_SUCCESS;
}

hvx_status hvxWaitBatch(hvx_context ctx, void* stream) {
    if (!ok_ctx(ctx)) return HVX_ERROR_INVALID_REFERENCE;
    if (C(ctx)->plan_only) return HVX_ERROR_NOT_SUPPORTED;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_status(e);
    return check_device_error(C(ctx));
}

// ---- nodes ----------------------------------------------------------------------------

hvx_node hvxGaussian3x3Node(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_GAUSS, {in}, {out}, 1, NodeParams());
}

hvx_node hvxBox3x3Node(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_BOX, {in}, {out}, 1, NodeParams());
}

hvx_node hvxDilate3x3Node(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_DILATE, {in}, {out}, 1, NodeParams());
}

hvx_node hvxErode3x3Node(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_ERODE, {in}, {out}, 1, NodeParams());
}

hvx_node hvxMedian3x3Node(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_MEDIAN, {in}, {out}, 1, NodeParams());
}

hvx_node hvxAndNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out) {
    return add_node(g, N_AND, {a, b}, {out}, 1, NodeParams());
}

hvx_node hvxOrNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out) {
    return add_node(g, N_OR, {a, b}, {out}, 1, NodeParams());
}

hvx_node hvxXorNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out) {
    return add_node(g, N_XOR, {a, b}, {out}, 1, NodeParams());
}

hvx_node hvxNotNode(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_NOT, {in}, {out}, 1, NodeParams());
}

hvx_node hvxSobel3x3Node(hvx_graph g, hvx_image in, hvx_image gx, hvx_image gy) {
    if (ok_graph(g) && !gx && !gy) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    return add_node(g, N_SOBEL, {in}, {gx, gy}, 0, NodeParams());
}

hvx_node hvxMagnitudeNode(hvx_graph g, hvx_image gx, hvx_image gy, hvx_image out) {
    return add_node(g, N_MAG, {gx, gy}, {out}, 1, NodeParams());
}

hvx_node hvxPhaseNode(hvx_graph g, hvx_image gx, hvx_image gy, hvx_image out) {
    return add_node(g, N_PHASE, {gx, gy}, {out}, 1, NodeParams());
}

hvx_node hvxThresholdNode(hvx_graph g, hvx_image in, int32_t type, double value, double upper,
                          int32_t tv, int32_t fv, hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    if ((type != HVX_THRESHOLD_BINARY && type != HVX_THRESHOLD_RANGE) || tv < 0 || tv > 255 ||
        fv < 0 || fv > 255 || !std::isfinite(value) ||
        (type == HVX_THRESHOLD_RANGE && (!std::isfinite(upper) || upper < value))) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.thr_type = type;
    p.thr_value = value;
    p.thr_upper = upper;
    p.true_value = tv;
    p.false_value = fv;
    return add_node(g, N_THRESH, {in}, {out}, 1, p);
}

hvx_node hvxChannelExtractNode(hvx_graph g, hvx_image in, int32_t channel, hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    if (channel < HVX_CHANNEL_Y || channel > HVX_CHANNEL_V) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.channel = channel;
    return add_node(g, N_CHX, {in}, {out}, 1, p);
}

static hvx_node arith_node(hvx_graph g, int kind, hvx_image a, hvx_image b, int32_t policy,
                           hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    if (policy != HVX_POLICY_WRAP && policy != HVX_POLICY_SATURATE) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.policy = policy;
    return add_node(g, kind, {a, b}, {out}, 1, p);
}

hvx_node hvxAddNode(hvx_graph g, hvx_image a, hvx_image b, int32_t policy, hvx_image out) {
    return arith_node(g, N_ADD, a, b, policy, out);
}

hvx_node hvxSubtractNode(hvx_graph g, hvx_image a, hvx_image b, int32_t policy, hvx_image out) {
    return arith_node(g, N_SUB, a, b, policy, out);
}

hvx_node hvxMultiplyNode(hvx_graph g, hvx_image a, hvx_image b, float scale, int32_t policy,
                         int32_t rounding, hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    if (!(scale >= 0.0f && scale <= 65536.0f) ||
        (policy != HVX_POLICY_WRAP && policy != HVX_POLICY_SATURATE) ||
        (rounding != HVX_ROUND_TO_ZERO && rounding != HVX_ROUND_TO_NEAREST_EVEN)) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.policy = policy;
    p.scale = scale;
    p.mul_rounding = rounding;
    return add_node(g, N_MULTIPLY, {a, b}, {out}, 1, p);
}

hvx_node hvxUserPointNode(hvx_graph g, const char* expr, const hvx_image* in, int32_t n_in,
                          hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    std::string code, why;
    if (!expr || !in || n_in < 1 || n_in > 3 ||
        !parse_user_expr(expr, false, n_in, 0, 0, &code, &why)) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        if (getenv("HVX_CODEGEN_VERBOSE") && !why.empty())
            fprintf(stderr, "hvx: user expression rejected: %s\n", why.c_str());
        return nullptr;
    }
    NodeParams p;
    p.user_code = code;
    if (n_in == 1) return add_node(g, N_USER_POINT, {in[0]}, {out}, 1, p);
    if (n_in == 2) return add_node(g, N_USER_POINT, {in[0], in[1]}, {out}, 1, p);
    return add_node(g, N_USER_POINT, {in[0], in[1], in[2]}, {out}, 1, p);
}

hvx_node hvxUserLocalNode(hvx_graph g, const char* expr, int32_t kw, int32_t kh, hvx_image in,
                          hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    std::string code, why;
    if (!expr || kw < 1 || kh < 1 || kw > 9 || kh > 9 || !(kw & 1) || !(kh & 1) ||
        !parse_user_expr(expr, true, 1, kw / 2, kh / 2, &code, &why)) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        if (getenv("HVX_CODEGEN_VERBOSE") && !why.empty())
            fprintf(stderr, "hvx: user expression rejected: %s\n", why.c_str());
        return nullptr;
    }
    NodeParams p;
    p.user_code = code;
    p.kw = kw;
    p.kh = kh;
    return add_node(g, N_USER_LOCAL, {in}, {out}, 1, p);
}

hvx_node hvxCopyNode(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_COPY, {in}, {out}, 1, NodeParams());
}

hvx_node hvxConvertDepthNode(hvx_graph g, hvx_image in, hvx_image out, int32_t policy,
                             int32_t shift) {
    if (!ok_graph(g)) return nullptr;
    if ((policy != HVX_POLICY_WRAP && policy != HVX_POLICY_SATURATE) || shift < 0 || shift > 7) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.policy = policy;
    p.shift = shift;
    return add_node(g, N_CONVDEPTH, {in}, {out}, 1, p);
}

hvx_node hvxAbsDiffNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out) {
    return arith_node(g, N_ABSDIFF, a, b, HVX_POLICY_SATURATE, out);
}

hvx_node hvxConvolveNode(hvx_graph g, hvx_image in, const int32_t* coeffs, int32_t kw,
                         int32_t kh, int32_t shift, hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    if (!coeffs || kw < 1 || kh < 1 || kw > 7 || kh > 7 || !(kw & 1) || !(kh & 1) || shift < 0 ||
        shift > 30) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.kw = kw;
    p.kh = kh;
    p.shift = shift;
    p.coeffs.assign(coeffs, coeffs + kw * kh);
    return add_node(g, N_CONV, {in}, {out}, 1, p);
}

hvx_node hvxPointNode(hvx_graph g, int32_t op, const hvx_image* ins, int32_t n_in,
                      hvx_image out, const double* params, int32_t n_params) {
    if (!ok_graph(g)) return nullptr;
    NodeParams p;
    p.custom_op = op;
    if (op == HVX_POINT_MUL) {
        if (n_in != 2 || !ins) {
            G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
            return nullptr;
        }
        return add_node(g, N_POINT, {ins[0], ins[1]}, {out}, 1, p);
    }
    if (op == HVX_POINT_HARRIS_RESPONSE) {
        if (n_in != 3 || !ins || n_params != 2 || !params || params[0] != std::floor(params[0]) ||
            params[1] != std::floor(params[1]) || params[0] < 0 || params[0] > 1000 ||
            params[1] < 1 || params[1] > 1000) {
            G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
            return nullptr;
        }
        p.kn = (int64_t)params[0];
        p.kd = (int64_t)params[1];
        return add_node(g, N_POINT, {ins[0], ins[1], ins[2]}, {out}, 1, p);
    }
    if (op == HVX_POINT_TOMASI_RESPONSE) {
        if (n_in != 3 || !ins) {
            G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
            return nullptr;
        }
        return add_node(g, N_POINT, {ins[0], ins[1], ins[2]}, {out}, 1, p);
    }
    G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
    return nullptr;
}

hvx_node hvxLocalNode(hvx_graph g, int32_t op, int32_t kw, int32_t kh, hvx_image in,
                      hvx_image out) {
    if (!ok_graph(g)) return nullptr;
    if (op != HVX_LOCAL_SUM || kw < 1 || kh < 1 || kw > 9 || kh > 9 || !(kw & 1) || !(kh & 1)) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.custom_op = op;
    p.kw = kw;
    p.kh = kh;
    return add_node(g, N_LOCAL, {in}, {out}, 1, p);
}

hvx_status hvxSetNodeBorder(hvx_node hn, int32_t mode, int32_t constant) {
    if (!ok_node(hn)) return HVX_ERROR_INVALID_REFERENCE;
    if (mode < HVX_BORDER_UNDEFINED || mode > HVX_BORDER_REPEAT) return HVX_ERROR_INVALID_PARAMETERS;
    Node* n = N(hn);
    n->border = mode;
    n->cval = constant;
    release_plan(n->graph);
    return HVX_SUCCESS;
}

hvx_status hvxSetNodeRounding(hvx_node hn, int32_t rounding) {
    if (!ok_node(hn)) return HVX_ERROR_INVALID_REFERENCE;
    if (rounding != HVX_ROUND_TO_ZERO && rounding != HVX_ROUND_TO_NEAREST)
        return HVX_ERROR_INVALID_PARAMETERS;
    Node* n = N(hn);
    n->rounding = rounding;
    release_plan(n->graph);
    return HVX_SUCCESS;
}

hvx_status hvxQueryNode(hvx_node hn, int32_t attr, void* out, uint64_t size) {
    if (!ok_node(hn)) return HVX_ERROR_INVALID_REFERENCE;
    Node* n = N(hn);
    if (!out || size < 4) return HVX_ERROR_INVALID_PARAMETERS;
    if (!n->graph->verified) return HVX_ERROR_NOT_VERIFIED;
    if (attr == HVX_NODE_LIVE_OUTPUTS) {
        uint32_t m = n->live_mask;
        std::memcpy(out, &m, 4);
        return HVX_SUCCESS;
    }
    if (attr == HVX_NODE_GROUP) {
        int32_t gi = n->live_mask ? n->group : -1;
        std::memcpy(out, &gi, 4);
        return HVX_SUCCESS;
    }
    return HVX_ERROR_INVALID_PARAMETERS;
}

// ---- global operators (Table 2 "reduce" / "histogram") ---------------------------

static hvx_node global_node(hvx_graph hg, int kind, hvx_image in, const NodeParams& p) {
    if (!ok_graph(hg)) return nullptr;
    Graph* g = G(hg);
    // the node's result: a non-virtual data vertex owned by the graph
    Image* r = new (std::nothrow) Image();
    if (!r) {
        g->last = HVX_ERROR_NO_MEMORY;
        return nullptr;
    }
    r->ctx = g->ctx;
    r->owner_graph = g;
    r->is_result = true;
    r->fmt = r->user_fmt = HVX_DF_RESULT;
    g->virtuals.push_back(r);
    return add_node(hg, kind, {in}, {reinterpret_cast<hvx_image>(r)}, 1, p);
}

hvx_node hvxMeanStdDevNode(hvx_graph g, hvx_image in) {
    return global_node(g, N_MEANSTD, in, NodeParams());
}

hvx_node hvxMinMaxLocNode(hvx_graph g, hvx_image in) {
    return global_node(g, N_MINMAX, in, NodeParams());
}

hvx_node hvxHistogramNode(hvx_graph g, hvx_image in, int32_t num_bins, int32_t offset,
                          int32_t range) {
    if (!ok_graph(g)) return nullptr;
    if (num_bins < 1 || num_bins > 256 || offset < 0 || range < 1 || offset + range > 256) {
        G(g)->last = HVX_ERROR_INVALID_PARAMETERS;
        return nullptr;
    }
    NodeParams p;
    p.hist_bins = num_bins;
    p.hist_offset = offset;
    p.hist_range = range;
    return global_node(g, N_HIST, in, p);
}

hvx_node hvxEqualizeHistNode(hvx_graph g, hvx_image in, hvx_image out) {
    return add_node(g, N_EQHIST, {in}, {out}, 1, NodeParams());
}

hvx_status hvxGetNodeResult(hvx_node hn, void* out, uint64_t size) {
    if (!ok_node(hn)) return HVX_ERROR_INVALID_REFERENCE;
    Node* n = N(hn);
    if (!out) return HVX_ERROR_INVALID_PARAMETERS;
    if (n->kind != N_MEANSTD && n->kind != N_MINMAX && n->kind != N_HIST)
        return HVX_ERROR_INVALID_PARAMETERS;
    if (!n->graph->verified) return HVX_ERROR_NOT_VERIFIED;
    if (n->graph->ctx->plan_only) return HVX_ERROR_NOT_SUPPORTED;
    Image* r = n->out[0];
    if (!r || !r->dev) return HVX_ERROR_NOT_VERIFIED;
    if (n->kind == N_HIST) {
        const uint64_t bytes = 4ull * (uint64_t)n->p.hist_bins;
        if (size < bytes) return HVX_ERROR_INVALID_PARAMETERS;
        return cuda_status(cudaMemcpy(out, r->dev, bytes, cudaMemcpyDeviceToHost));
    }
    uint64_t w[4] = {0, 0, 0, 0};
    const uint64_t bytes = n->kind == N_MEANSTD ? 24 : 32;
    cudaError_t e = cudaMemcpy(w, r->dev, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (n->kind == N_MEANSTD) {
        if (size < sizeof(hvx_mean_stddev)) return HVX_ERROR_INVALID_PARAMETERS;
        hvx_mean_stddev m;
        std::memset(&m, 0, sizeof(m));
        m.sum = (int64_t)w[0];
        m.sum_squares = w[1];
        m.count = w[2];
        if (m.count) {
            // mean = S1 / N, stddev = sqrt(N S2 - S1^2) / N, N S2 - S1^2 exact
            const __int128 var_n2 = (__int128)m.count * (__int128)m.sum_squares -
                                    (__int128)m.sum * (__int128)m.sum;
            m.mean = (float)((double)m.sum / (double)m.count);
            m.stddev = (float)(std::sqrt((double)var_n2) / (double)m.count);
        }
        std::memcpy(out, &m, sizeof(m));
        return HVX_SUCCESS;
    }
    if (size < sizeof(hvx_minmaxloc)) return HVX_ERROR_INVALID_PARAMETERS;
    hvx_minmaxloc m;
    std::memset(&m, 0, sizeof(m));
    m.min_x = m.min_y = m.max_x = m.max_y = -1;
    const uint64_t W = n->in[0]->w;
    const uint64_t cmask = (1ull << 40) - 1;
    if (w[0] != ~0ull) {
        m.min = (int32_t)(w[0] >> 32) - 32768;
        m.min_x = (int32_t)((w[0] & 0xFFFFFFFFull) % W);
        m.min_y = (int32_t)((w[0] & 0xFFFFFFFFull) / W);
        m.min_count = w[2] & cmask;
    }
    if (w[1] != ~0ull) {
        m.max = 32767 - (int32_t)(w[1] >> 32);
        m.max_x = (int32_t)((w[1] & 0xFFFFFFFFull) % W);
        m.max_y = (int32_t)((w[1] & 0xFFFFFFFFull) / W);
        m.max_count = w[3] & cmask;
    }
    std::memcpy(out, &m, sizeof(m));
    return HVX_SUCCESS;
}

}  // extern "C"

extern "C" hvx_status hvxTestInjectFault(int32_t kind, int64_t n) {
    if (kind == HVX_FAULT_NONE) {
        for (auto& c : g_fault_count) c.store(0);
        return HVX_SUCCESS;
    }
    if ((kind != HVX_FAULT_DEVICE_ALLOC && kind != HVX_FAULT_LAUNCH) || n < 1)
        return HVX_ERROR_INVALID_PARAMETERS;
    g_fault_count[kind].store(n);
    return HVX_SUCCESS;
}
