// Serving loop: verified graphs are submitted as requests; a dispatcher
// thread admits them in FIFO order while a slot and the device-memory budget
// allow, launches each on the next of several streams so that admitted work
// overlaps on the device, and retires requests as their completion events
// fire.  Requests that arrive while others are running are admitted as soon
// as slots and budget free up (continuous batching); latency is measured from
// submission to completion.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "hvx_internal.h"

namespace hvx {

namespace {
double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct Request {
    uint64_t ticket = 0;
    Graph* g = nullptr;
    uint64_t bytes = 0;
    double mpix = 0;
    double t_submit = 0;
    double t_admit = 0;
    double latency_ms = 0;
    hvx_status result = HVX_SUCCESS;
    bool done = false;
    cudaEvent_t ev = nullptr;
    std::vector<hvx_host_copy> copies;  // host data: copied in before, out after
};

struct Server {
    uint32_t magic = kMagicServer;
    Context* ctx = nullptr;
    uint64_t budget = 0;
    int max_inflight = 1;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> event_pool;
    int next_stream = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> inflight;
    std::unordered_map<uint64_t, Request*> by_ticket;
    uint64_t next_ticket = 1;
    uint64_t reserved = 0;
    bool stop = false;
    std::thread dispatcher;

    // statistics
    uint64_t submitted = 0, completed = 0, failed = 0, max_in_flight = 0, peak_reserved = 0;
    std::vector<double> latencies;
    std::vector<double> waits;  // submission -> admission of completed requests
    double mpix_completed = 0;

    void run();
};

void Server::run() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // retire finished requests
        for (size_t i = 0; i < inflight.size();) {
            Request* r = inflight[i];
            cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            r->latency_ms = now_ms() - r->t_submit;
            r->result = q == cudaSuccess ? HVX_SUCCESS : cuda_status(q);
            if (q != cudaSuccess) cudaGetLastError();
            r->done = true;
            reserved -= r->bytes;
            r->g->busy.store(0);
            event_pool.push_back(r->ev);
            r->ev = nullptr;
            if (r->result == HVX_SUCCESS) {
                ++completed;
                latencies.push_back(r->latency_ms);
                waits.push_back(r->t_admit - r->t_submit);
                mpix_completed += r->mpix;
            } else {
                ++failed;
            }
            inflight[i] = inflight.back();
            inflight.pop_back();
            cv_done.notify_all();
        }
        // admit in FIFO order while a slot and the budget allow.  A request
        // whose graph still has one in flight is passed over (it keeps its
        // place; requests on other graphs behind it go ahead); one that does
        // not fit the budget stops admission, so a large request is not
        // overtaken indefinitely by smaller ones.
        for (size_t qi = 0; qi < queue.size();) {
            Request* r = queue[qi];
            if ((int)inflight.size() >= max_inflight) break;
            if (r->g->busy.load()) {
                ++qi;
                continue;
            }
            if (budget && reserved + r->bytes > budget) break;
            queue.erase(queue.begin() + (std::ptrdiff_t)qi);
            r->g->busy.store(1);
            r->t_admit = now_ms();
            reserved += r->bytes;
            peak_reserved = std::max(peak_reserved, reserved);
            cudaStream_t s = streams[next_stream];
            next_stream = (next_stream + 1) % (int)streams.size();
            if (event_pool.empty()) {
                cudaEvent_t e;
                cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
                event_pool.push_back(e);
            }
            r->ev = event_pool.back();
            event_pool.pop_back();
            NvtxRange nvtx("hvx serve dispatch");
            std::vector<const hvx_host_copy*> up, down;
            for (const hvx_host_copy& c : r->copies) (c.to_device ? up : down).push_back(&c);
            hvx_status st = host_copies(up, true, s);
            if (st == HVX_SUCCESS) st = launch_plan(r->g, s);
            if (st == HVX_SUCCESS) st = host_copies(down, false, s);
            if (st == HVX_SUCCESS && cudaEventRecord(r->ev, s) != cudaSuccess) st = HVX_ERROR_DEVICE;
            if (st != HVX_SUCCESS) {
                cudaGetLastError();
                r->result = st;
                r->done = true;
                r->latency_ms = now_ms() - r->t_submit;
                reserved -= r->bytes;
                r->g->busy.store(0);
                event_pool.push_back(r->ev);
                r->ev = nullptr;
                ++failed;
                cv_done.notify_all();
                continue;
            }
            inflight.push_back(r);
            max_in_flight = std::max<uint64_t>(max_in_flight, inflight.size());
        }
        if (stop && queue.empty() && inflight.empty()) break;
        if (inflight.empty() && queue.empty()) {
            cv_work.wait(lk);
        } else {
            // poll completions; new submissions wake the loop at once
            cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

void server_destroy(Server* s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    for (auto& kv : s->by_ticket) {
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
        delete kv.second;
    }
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    auto& v = s->ctx->servers;
    v.erase(std::remove(v.begin(), v.end(), s), v.end());
    s->magic = 0;
    delete s;
}

}  // namespace hvx

using namespace hvx;

namespace {
bool ok_server(hvx_server s) { return s && reinterpret_cast<Server*>(s)->magic == kMagicServer; }
Server* S(hvx_server s) { return reinterpret_cast<Server*>(s); }
}  // namespace

extern "C" {

hvx_status hvxCreateServer(hvx_context ctx, uint64_t budget, int32_t max_inflight,
                           int32_t n_streams, hvx_server* out) {
    Context* c = reinterpret_cast<Context*>(ctx);
    if (!c || c->magic != kMagicContext) return HVX_ERROR_INVALID_REFERENCE;
    if (!out || max_inflight < 1 || n_streams < 1 || n_streams > 64)
        return HVX_ERROR_INVALID_PARAMETERS;
    Server* s = new (std::nothrow) Server();
    if (!s) return HVX_ERROR_NO_MEMORY;
    s->ctx = c;
    s->budget = budget;
    s->max_inflight = max_inflight;
    for (int i = 0; i < n_streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return HVX_ERROR_DEVICE;
        }
        s->streams.push_back(st);
    }
    c->servers.push_back(s);
    s->dispatcher = std::thread([s] { s->run(); });
    *out = reinterpret_cast<hvx_server>(s);
    return HVX_SUCCESS;
}

hvx_status hvxServerSubmit(hvx_server hs, hvx_graph hg, uint64_t* ticket) {
    return hvxServerSubmitHost(hs, hg, nullptr, 0, ticket);
}

namespace {

// Validate one request and build it (not yet queued).
hvx_status make_request(Server* s, hvx_graph hg, const hvx_host_copy* copies, int32_t n_copies,
                        Request** out) {
    Graph* g = reinterpret_cast<Graph*>(hg);
    if (!g || g->magic != kMagicGraph) return HVX_ERROR_INVALID_REFERENCE;
    if (g->ctx != s->ctx) return HVX_ERROR_INVALID_REFERENCE;
    if (!g->verified) return HVX_ERROR_NOT_VERIFIED;
    // device bytes the request holds while in flight: its images and the
    // plan's materialised intermediates
    uint64_t bytes = g->plan.intermediate_bytes;
    double mpix = 0;
    std::vector<const Image*> seen;
    for (const Group& G : g->plan.groups) {
        for (const Image* im : G.inputs)
            if (!im->is_virtual && std::find(seen.begin(), seen.end(), im) == seen.end()) {
                seen.push_back(im);
                bytes += im->bytes;
                mpix = std::max(mpix, (double)im->w * im->h / 1e6);
            }
        for (const Image* im : G.outputs)
            if (!im->is_virtual && std::find(seen.begin(), seen.end(), im) == seen.end()) {
                seen.push_back(im);
                bytes += im->bytes;
            }
    }
    if (s->budget && bytes > s->budget) return HVX_ERROR_OVER_BUDGET;
    hvx_status cs = check_host_copies(s->ctx, copies, n_copies);
    if (cs != HVX_SUCCESS) return cs;
    Request* r = new (std::nothrow) Request();
    if (!r) return HVX_ERROR_NO_MEMORY;
    if (n_copies > 0) r->copies.assign(copies, copies + n_copies);
    r->g = g;
    r->bytes = bytes;
    r->mpix = mpix;
    *out = r;
    return HVX_SUCCESS;
}

// Queue built requests under one lock (they arrive together).
hvx_status enqueue(Server* s, Request* const* rs, int n, uint64_t* tickets) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return HVX_ERROR_INVALID_REFERENCE;
        const double t = now_ms();
        for (int i = 0; i < n; ++i) {
            Request* r = rs[i];
            r->ticket = s->next_ticket++;
            r->t_submit = t;
            s->queue.push_back(r);
            s->by_ticket[r->ticket] = r;
            ++s->submitted;
            tickets[i] = r->ticket;
        }
    }
    s->cv_work.notify_all();
    return HVX_SUCCESS;
}

}  // namespace

hvx_status hvxServerSubmitHost(hvx_server hs, hvx_graph hg, const hvx_host_copy* copies,
                               int32_t n_copies, uint64_t* ticket) {
    if (!ok_server(hs)) return HVX_ERROR_INVALID_REFERENCE;
    if (!ticket) return HVX_ERROR_INVALID_PARAMETERS;
    Server* s = S(hs);
    Request* r = nullptr;
    hvx_status st = make_request(s, hg, copies, n_copies, &r);
    if (st != HVX_SUCCESS) return st;
    uint64_t t = 0;
    st = enqueue(s, &r, 1, &t);
    if (st != HVX_SUCCESS) {
        delete r;
        return st;
    }
    *ticket = t;
    return HVX_SUCCESS;
}

hvx_status hvxServerSubmitMany(hvx_server hs, const hvx_graph* graphs, int32_t n,
                               uint64_t* tickets) {
    if (!ok_server(hs)) return HVX_ERROR_INVALID_REFERENCE;
    if (!graphs || !tickets || n < 0) return HVX_ERROR_INVALID_PARAMETERS;
    if (n == 0) return HVX_SUCCESS;
    Server* s = S(hs);
    std::vector<Request*> rs;
    rs.reserve((size_t)n);
    hvx_status st = HVX_SUCCESS;
    for (int i = 0; i < n && st == HVX_SUCCESS; ++i) {
        Request* r = nullptr;
        st = make_request(s, graphs[i], nullptr, 0, &r);
        if (st == HVX_SUCCESS) rs.push_back(r);
    }
    std::vector<uint64_t> t((size_t)n);
    if (st == HVX_SUCCESS) st = enqueue(s, rs.data(), n, t.data());
    if (st != HVX_SUCCESS) {
        for (Request* r : rs) delete r;
        return st;
    }
    std::copy(t.begin(), t.end(), tickets);
    return HVX_SUCCESS;
}

hvx_status hvxServerWait(hvx_server hs, uint64_t ticket, int32_t timeout_ms, hvx_status* result,
                         double* latency_ms) {
    if (!ok_server(hs)) return HVX_ERROR_INVALID_REFERENCE;
    Server* s = S(hs);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) return HVX_ERROR_INVALID_PARAMETERS;
    Request* r = it->second;
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, [&] { return r->done; });
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                    [&] { return r->done; })) {
        return HVX_ERROR_TIMEOUT;
    }
    if (result) *result = r->result;
    if (latency_ms) *latency_ms = r->latency_ms;
    s->by_ticket.erase(it);
    delete r;
    return HVX_SUCCESS;
}

hvx_status hvxServerStats(hvx_server hs, hvx_server_stats* out) {
    if (!ok_server(hs)) return HVX_ERROR_INVALID_REFERENCE;
    if (!out) return HVX_ERROR_INVALID_PARAMETERS;
    Server* s = S(hs);
    std::lock_guard<std::mutex> lk(s->mu);
    hvx_server_stats st;
    std::memset(&st, 0, sizeof(st));
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.failed = s->failed;
    st.queued = s->queue.size();
    st.in_flight = s->inflight.size();
    st.max_in_flight = s->max_in_flight;
    st.bytes_reserved = s->reserved;
    st.peak_bytes_reserved = s->peak_reserved;
    st.mpix_completed = s->mpix_completed;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t k = (size_t)std::ceil(p * v.size()) - 1;
            return v[std::min(k, v.size() - 1)];
        };
        st.p50_ms = pct(0.50);
        st.p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st.mean_ms = sum / v.size();
        st.max_ms = v.back();
    }
    if (!s->waits.empty()) {
        std::vector<double> v = s->waits;
        std::sort(v.begin(), v.end());
        const size_t k = (size_t)std::ceil(0.99 * v.size()) - 1;
        st.wait_p99_ms = v[std::min(k, v.size() - 1)];
        st.wait_max_ms = v.back();
    }
    *out = st;
    return HVX_SUCCESS;
}

hvx_status hvxServerResetStats(hvx_server hs) {
    if (!ok_server(hs)) return HVX_ERROR_INVALID_REFERENCE;
    Server* s = S(hs);
    std::lock_guard<std::mutex> lk(s->mu);
    s->latencies.clear();
    s->waits.clear();
    s->mpix_completed = 0;
    s->max_in_flight = s->inflight.size();
    s->peak_reserved = s->reserved;
    return HVX_SUCCESS;
}

hvx_status hvxReleaseServer(hvx_server* hs) {
    if (!hs || !ok_server(*hs)) return HVX_ERROR_INVALID_REFERENCE;
    server_destroy(S(*hs));
    *hs = nullptr;
    return HVX_SUCCESS;
}

}  // extern "C"
