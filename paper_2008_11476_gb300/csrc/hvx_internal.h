// Internal C++ structures of the image-graph library: object model, the
// implementation graph of point/local ops, the verified plan and the kernel
// launch interfaces.  Host-only; included by the .cpp and .cu files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hvx.h"
#include <nvtx3/nvToolsExt.h>

#include "jit_params.h"
#include "kernel_params.h"

namespace hvx {

constexpr uint32_t kMagicContext = 0x43545831u;
constexpr uint32_t kMagicGraph = 0x47525031u;
constexpr uint32_t kMagicImage = 0x494D4731u;
constexpr uint32_t kMagicNode = 0x4E4F4431u;
constexpr uint32_t kMagicServer = 0x53525631u;

int bytes_per_pixel(int fmt);  // U8 1, S16 2, S32 4, F32 4, UYVY 2

struct Rect {
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    bool empty() const { return x1 <= x0 || y1 <= y0; }
};
Rect rect_intersect(const Rect& a, const Rect& b);

// ---------------------------------------------------------------------------
// Budgeted device memory pool.  Blocks are cached by size after release and
// handed out again; the budget counts bytes held by live blocks plus cached
// ones, and cached blocks are returned to the driver before an allocation is
// refused.
// Host-side fault injection (hvxTestInjectFault): true when the armed fault of
// this kind fires on this call.
bool fault_fires(int kind);

class DevicePool {
  public:
    explicit DevicePool(uint64_t budget = 0) : budget_(budget) {}
    ~DevicePool();
    hvx_status alloc(uint64_t bytes, void** out);
    void free(void* p);
    void set_budget(uint64_t b) { budget_ = b; }
    uint64_t in_use() const { return in_use_; }
    uint64_t held() const { return held_; }
    void trim();

  private:
    std::mutex mu_;
    uint64_t budget_;
    uint64_t in_use_ = 0;  // bytes of blocks handed out
    uint64_t held_ = 0;    // in_use_ + cached
    std::map<void*, uint64_t> live_;
    std::multimap<uint64_t, void*> cache_;
};

struct Context;
struct Graph;
struct Server;

struct Image {
    uint32_t magic = kMagicImage;
    Context* ctx = nullptr;
    Graph* owner_graph = nullptr;  // set for virtual images
    uint32_t w = 0, h = 0;
    int fmt = HVX_DF_VIRT;
    bool is_virtual = false;
    bool user_fixed_size = false;  // virtual image declared with a size
    int user_fmt = HVX_DF_VIRT;    // virtual image declared with a format
    void* dev = nullptr;
    uint64_t pitch = 0;
    bool owns_mem = false;
    uint64_t bytes = 0;
    Rect valid;
    int user_refs = 1;
    int node_refs = 0;
    // Set by verification: a virtual image whose values live only on chip.
    bool materialized = false;
    // The result of a global operator (MeanStdDev, MinMaxLoc, Histogram): a
    // non-virtual data vertex of the graph owned by it, with no pixels; dev
    // holds the device result block.
    bool is_result = false;
};

// Internal format of result images.
constexpr int HVX_DF_RESULT = 100;

const char* op_name(int kind);
bool op_is_local(int kind);

enum NodeKind : int {
    N_GAUSS = 1,
    N_BOX,
    N_SOBEL,
    N_MAG,
    N_PHASE,
    N_THRESH,
    N_CHX,
    N_ADD,
    N_SUB,
    N_ABSDIFF,
    N_CONV,
    N_POINT,
    N_LOCAL,
    N_DILATE,
    N_ERODE,
    N_MEDIAN,
    N_AND,
    N_OR,
    N_XOR,
    N_NOT,
    N_MULTIPLY,
    N_MEANSTD,
    N_MINMAX,
    N_HIST,
    N_EQHIST,
    N_COPY,
    N_CONVDEPTH,
    N_USER_POINT,
    N_USER_LOCAL,
};

struct NodeParams {
    int thr_type = HVX_THRESHOLD_BINARY;
    double thr_value = 0, thr_upper = 0;
    int true_value = 255, false_value = 0;
    int channel = 0;
    int policy = HVX_POLICY_SATURATE;
    int custom_op = 0;
    int64_t kn = 0, kd = 1;
    int kw = 3, kh = 3;
    int shift = 0;
    std::vector<int32_t> coeffs;
    float scale = 1.0f;        // Multiply
    int mul_rounding = HVX_ROUND_TO_ZERO;
    int hist_bins = 256, hist_offset = 0, hist_range = 256;  // Histogram
    std::string user_code;     // user-defined operator, rewritten (user_expr.cpp)
};

struct Node {
    uint32_t magic = kMagicNode;
    Graph* graph = nullptr;
    int kind = 0;
    std::vector<Image*> in;
    std::vector<Image*> out;  // entries may be null (optional outputs)
    NodeParams p;
    int border = HVX_BORDER_REPLICATE;
    int cval = 0;
    int rounding = HVX_ROUND_TO_ZERO;
    void* d_aux = nullptr;  // EqualizeHist: its 256-bin device histogram
    // set by verification
    uint32_t live_mask = 0;
    int group = -1;
};

// One point/local abstraction op of the implementation graph (Section 4):
// exactly one output image.
struct Op {
    int kind = 0;
    Node* node = nullptr;
    int out_index = 0;  // which output of the node
    Image* in[3] = {nullptr, nullptr, nullptr};
    int n_in = 0;
    Image* out = nullptr;
    int rx = 0, ry = 0;  // window radius (local ops)
    bool alive = false;
    int group = -1;
};

// NVTX range for profilers (nsys / ncu timelines): verification, code
// generation, launches, batches and server dispatch are marked; without a
// profiler attached the calls cost a few nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// MIRROR / REPEAT read arbitrary pixels of a local operator's input: such an
// input is read from memory, never from a fused producer's tile.
inline bool border_wraps(int border) {
    return border == HVX_BORDER_MIRROR || border == HVX_BORDER_REPEAT;
}

// A kernel generated for a staged-tile group (codegen.cpp) and its launch.
struct JitKernel;
struct JitLaunch {
    JitKernel* k = nullptr;  // cached for the life of the process
    HvxJitParams p;
    unsigned gx = 0, gy = 0;
};

// A fused group: ops run by one kernel launch.
enum GroupKernel : int {
    GK_GENERIC = 0,  // staged tile interpreter (any point/local ops)
    GK_GAUSS,        // Gaussian3x3, TMA tile loads
    GK_EDGE,         // Gaussian -> Sobel -> Magnitude/Threshold + Phase
    GK_BINOM5,       // 5x5 binomial Convolve, TMA tile loads
    GK_HARRIS,       // Sobel -> products -> window sums -> response -> threshold
    GK_POINT,        // plain point op
    GK_CHX_UV,       // ChannelExtract U/V (half width)
    GK_EQHIST,       // EqualizeHist: histogram, then the mapping
};

// A device block set before a group's launch (global operators' results).
struct ResultReset {
    void* p;
    int byte;
    uint64_t n;
};
const char* group_kernel_name(int gk);

struct Group {
    CUtensorMap tmap;              // TMA descriptor (64-byte aligned type) of the input (TMA kernels)
    std::vector<int> ops;        // indices into Plan::ops, topological order
    std::vector<Image*> inputs;  // images read from memory
    std::vector<Image*> outputs; // images written to memory
    int kernel = GK_GENERIC;
    int halo = 0;                // external input halo
    uint32_t W = 0, H = 0;
    // prepared launch state
    GenericDesc gdesc;           // for GK_GENERIC
    EdgeParams edge;             // for GK_EDGE / GK_GAUSS
    HarrisParams harris;         // for GK_HARRIS
    PlainParams plain;           // for GK_POINT / GK_CHX_UV
    JitLaunch jit;               // GK_GENERIC with a generated kernel
    bool jit_on = false;
    EqHistParams eqh;            // GK_EQHIST
    std::vector<ResultReset> resets;
    std::vector<std::string> user_code;  // user-defined operators' code (GenStage.i0)
    uint64_t ext_bytes = 0;      // bytes of non-virtual images read + written
    uint64_t mem_bytes = 0;      // bytes of every image read + written
    bool closed = false;         // planning: no further op may join
};

struct Plan {
    std::vector<Op> ops;
    std::vector<int> order;  // topological order of alive ops
    std::vector<Group> groups;
    std::vector<Image*> materialized;  // virtual images given device memory
    uint64_t intermediate_bytes = 0;
    uint64_t external_bytes = 0;
    std::string kernel_kinds;
};

struct Graph {
    uint32_t magic = kMagicGraph;
    uint64_t plan_id = 0;        // changes whenever a new plan is verified
    Context* ctx = nullptr;
    std::vector<std::unique_ptr<Node>> nodes;
    std::vector<Image*> virtuals;
    bool verified = false;
    bool fusion = true;
    int codegen = HVX_CODEGEN_AUTO;
    hvx_status last = HVX_SUCCESS;
    Plan plan;
    cudaEvent_t done = nullptr;
    bool scheduled = false;
    cudaStream_t last_stream = nullptr;
    std::atomic<int> busy{0};  // in flight on a server
};

struct BatchCache;  // persistent-kernel batch plans (runtime.cu)

struct Context {
    uint32_t magic = kMagicContext;
    int device = 0;
    bool plan_only = false;      // no device: verify and query only
    DevicePool pool;
    std::vector<Image*> images;  // non-virtual images
    std::vector<Graph*> graphs;
    std::vector<Server*> servers;
    int* d_error = nullptr;      // device error word (bounded waits that ran out)
    int num_sms = 0;
    BatchCache* batch = nullptr;
    // hvxScheduleGraphBatchHost: copy streams and events of its pipeline
    cudaStream_t io_in = nullptr, io_out = nullptr;
    std::vector<cudaEvent_t> io_events;
    // calls from several host threads: the batch cache and the host-data
    // pipeline are each used by one call at a time
    std::mutex batch_mu, io_mu;
};

// Driver-API work (tensor-map encoding, loading and launching generated
// kernels) runs in the calling thread's current context: runtime calls bind the
// device's primary context to a thread lazily, driver calls do not.  Entry
// points that do such work first make the context's device current in the
// calling thread, which may be a fresh one.
inline void bind_device(const Context* ctx) {
    if (!ctx->plan_only) cudaSetDevice(ctx->device);
}

// ---------------------------------------------------------------------------
// verification (graph.cpp)
hvx_status verify_graph(Graph* g);
void release_plan(Graph* g);

// execution (runtime.cu)
hvx_status prepare_launches(Graph* g);  // fill per-group kernel params
hvx_status launch_plan(Graph* g, cudaStream_t s);
hvx_status check_device_error(Context* ctx);
hvx_status ensure_context_device_state(Context* ctx);
void destroy_batch_cache(Context* ctx);
hvx_status process_batch(Context* ctx, Graph* const* gs, int n, cudaStream_t s);
// 2-D U8 tensor map of (w x h) bytes at ptr (16-byte aligned, pitch a multiple
// of 16) with a (box_w x box_h) box; cells outside the image read as 0.
hvx_status encode_u8_map_raw(CUtensorMap* map, const void* ptr, uint64_t pitch, uint32_t w,
                             uint32_t h, uint32_t box_w, uint32_t box_h);
// The tuned launch of a cached batch of exactly these graphs: rows per thread
// of each image's tiles (0 where the kernel has its own tile) and the
// persistent grid (0 for a direct launch).  HVX_ERROR_INVALID_PARAMETERS when
// no such batch has run.
hvx_status query_batch(Context* ctx, Graph* const* gs, int n, int* rows, int* grid);

// user-defined operators (user_expr.cpp): check an expression and rewrite it
// for the code generator
bool parse_user_expr(const std::string& src, bool local, int n_in, int rx, int ry,
                     std::string* code, std::string* why);

// code generation for staged-tile groups (codegen.cpp): generate, compile
// (cached by source) and, with load_module, load the group's kernel
bool jit_available();
bool jit_prepare(const GenericDesc& d, const std::vector<std::string>& user_code, bool load_module,
                 int device, JitLaunch* out, std::string* why);
cudaError_t jit_launch(const JitLaunch& j, cudaStream_t s);
// n images' groups that run the same generated kernel, in one launch: params
// and tile_start (n + 1 prefix sums of tiles per image) in device memory
cudaError_t jit_launch_batch(const JitKernel* k, const HvxJitParams* params, const int* tile_start,
                             int n, int total_tiles, cudaStream_t s);
void jit_tile(const JitKernel* k, int* tw, int* th);
const std::string& jit_source(const JitLaunch& j);

// host data of a call (api.cpp): checks, and the 2-D copies in one direction
// on a stream (adjacent images merged)
hvx_status check_host_copies(const Context* ctx, const hvx_host_copy* copies, int32_t n);
hvx_status host_copies(std::vector<const hvx_host_copy*> copies, bool to_device, cudaStream_t s);

// server (server.cpp)
void server_destroy(Server* s);

hvx_status cuda_status(cudaError_t e);

}  // namespace hvx
