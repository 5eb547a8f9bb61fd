// hvxEdgeBatchNoAlloc: the batched edge-graph launch for callers that cannot
// allocate device memory.
//
// hvxProcessGraphBatch keeps the per-image tensor maps, launch parameters and
// tile table of a batch in device memory it allocates (and caches) itself,
// and the context allocates a device error word.  This entry point runs the
// same persistent kernel (edge_batch_kernel) on caller-owned frames but keeps
// all of that scratch in one file-scope __device__ array of fixed size, so
// that no call allocates or frees device memory.
//
// The array lives on every device that loads the library until the process
// exits.  Its device address is looked up once per device (cudaGetSymbolAddress,
// with that device current) on the first call made on that device.  Every
// call rewrites the array's contents (the error word included, which is
// cleared), so two calls whose work overlaps on a GPU race on it.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/hvx.h"
#include "launchers.h"

namespace hvx {
namespace {

constexpr int kMaxFrames = HVX_NOALLOC_MAX_FRAMES;

// Scratch layout (bytes): [0, 256) device error word; then the tile prefix
// table (kMaxFrames + 1 ints); then the tile columns per frame (kMaxFrames
// ints); then kMaxFrames EdgeParams; then kMaxFrames tensor maps (64-byte
// aligned).
constexpr size_t kErrOff = 0;
constexpr size_t kTilesOff = 256;
constexpr size_t kTilesXOff = (kTilesOff + (kMaxFrames + 1) * sizeof(int) + 255) / 256 * 256;
constexpr size_t kParamsOff = (kTilesXOff + kMaxFrames * sizeof(int) + 255) / 256 * 256;
constexpr size_t kMapsOff =
    (kParamsOff + kMaxFrames * sizeof(EdgeParams) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kMapsOff + kMaxFrames * sizeof(CUtensorMap);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host staging copy of the scratch contents (written, then copied to the
// device in one cudaMemcpyAsync; pageable, so the copy has consumed it when
// the call returns).
static unsigned char g_host_stage[kScratchBytes];
static std::mutex g_mu;  // one call at a time per process for the host side

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

bool frame_ok(const hvx_edge_frame& f) {
    if (!f.in || f.width == 0 || f.height == 0 || f.width > 32768u || f.height > 32768u)
        return false;
    if (((uintptr_t)f.in & 15) || (f.in_pitch & 15) || f.in_pitch < f.width) return false;
    if (!f.mask && !f.phase) return false;
    if (f.mask && (((uintptr_t)f.mask & 15) || (f.mask_pitch & 15) || f.mask_pitch < f.width))
        return false;
    if (f.phase &&
        (((uintptr_t)f.phase & 15) || (f.phase_pitch & 15) || f.phase_pitch < f.width))
        return false;
    return true;
}

}  // namespace
}  // namespace hvx

using namespace hvx;

extern "C" hvx_status hvxEdgeBatchNoAlloc(const hvx_edge_frame* frames, int32_t n,
                                          int32_t border, int32_t threshold, void* stream) {
    if (!frames || n <= 0) return HVX_ERROR_INVALID_PARAMETERS;
    if (n > kMaxFrames) return HVX_ERROR_OVER_BUDGET;  // beyond the static scratch
    if (border != HVX_BORDER_UNDEFINED && border != HVX_BORDER_REPLICATE &&
        border != HVX_BORDER_CONSTANT)
        return HVX_ERROR_INVALID_PARAMETERS;
    const bool has_mask = frames[0].mask != nullptr, has_phase = frames[0].phase != nullptr;
    for (int i = 0; i < n; ++i)
        if (!frame_ok(frames[i]) || (frames[i].mask != nullptr) != has_mask ||
            (frames[i].phase != nullptr) != has_phase)
            return HVX_ERROR_INVALID_PARAMETERS;
    PFN_cuTensorMapEncodeTiled_v12000 encode = encoder();
    if (!encode) return HVX_ERROR_DEVICE;

    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return HVX_ERROR_DEVICE;
    }
    // set-up, once per device, with that device current
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return HVX_ERROR_DEVICE;
        }
        g_scratch_addr[dev] = p;
    }
    unsigned char* dscr = static_cast<unsigned char*>(g_scratch_addr[dev]);

    // host image of the scratch: error word 0, tile table, params, maps
    std::memset(g_host_stage, 0, kParamsOff);
    int* tiles = reinterpret_cast<int*>(g_host_stage + kTilesOff);
    int* tiles_x = reinterpret_cast<int*>(g_host_stage + kTilesXOff);
    EdgeParams* params = reinterpret_cast<EdgeParams*>(g_host_stage + kParamsOff);
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(g_host_stage + kMapsOff);
    int* d_err = reinterpret_cast<int*>(dscr + kErrOff);
    tiles[0] = 0;
    for (int i = 0; i < n; ++i) {
        const hvx_edge_frame& f = frames[i];
        EdgeParams& e = params[i];
        std::memset(&e, 0, sizeof(e));
        e.W = f.width;
        e.H = f.height;
        e.in = static_cast<const uint8_t*>(f.in);
        e.in_pitch = f.in_pitch;
        e.phase = static_cast<uint8_t*>(f.phase);
        e.phase_pitch = f.phase_pitch;
        e.mask = static_cast<uint8_t*>(f.mask);
        e.mask_pitch = f.mask_pitch;
        e.border_g = e.border_s = border;
        e.cval_g = e.cval_s = 0;
        e.rounding = HVX_ROUND_TO_ZERO;
        e.tv = 255;
        e.fv = 0;
        e.thr_type = HVX_THRESHOLD_BINARY;
        e.thr_general = 0;
        e.s_thr = threshold < 0 ? -1
                                : (threshold >= 32767 ? 0x7FFFFFFF : threshold * threshold + threshold);
        // valid regions: full, or shrunk by 1 (Gaussian) and 2 (Sobel) under UNDEFINED
        int g = border == HVX_BORDER_UNDEFINED ? 1 : 0, s = 2 * g;
        int32_t gv[4] = {g, g, (int32_t)f.width - g, (int32_t)f.height - g};
        int32_t sv[4] = {s, s, (int32_t)f.width - s, (int32_t)f.height - s};
        for (int k = 0; k < 2; ++k) {
            if (gv[2 + k] < gv[k]) gv[2 + k] = gv[k];
            if (sv[2 + k] < sv[k]) sv[2 + k] = sv[k];
        }
        std::memcpy(e.gvalid, gv, sizeof(gv));
        std::memcpy(e.valid, sv, sizeof(sv));
        e.err = d_err;
        cuuint64_t dims[2] = {f.width, f.height};
        cuuint64_t strides[1] = {f.in_pitch};
        cuuint32_t box[2] = {EDGE_LOAD_W, EDGE_LOAD_H};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(f.in), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return HVX_ERROR_INVALID_PARAMETERS;
        tiles_x[i] = (int)((f.width + EDGE_TW - 1) / EDGE_TW);
        tiles[i + 1] = tiles[i] + tiles_x[i] * (int)((f.height + EDGE_TH - 1) / EDGE_TH);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // one copy: error word cleared, tables and maps (only the used part)
    size_t used = kMapsOff + (size_t)n * sizeof(CUtensorMap);
    if (cudaMemcpyAsync(dscr, g_host_stage, used, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_DEVICE;
    }
    EdgeBatchDesc d;
    d.maps = reinterpret_cast<const CUtensorMap*>(dscr + kMapsOff);
    d.params = reinterpret_cast<const EdgeParams*>(dscr + kParamsOff);
    d.tile_start = reinterpret_cast<const int*>(dscr + kTilesOff);
    d.tiles_x = reinterpret_cast<const int*>(dscr + kTilesXOff);
    d.n_img = n;
    d.total_tiles = tiles[n];
    d.err = d_err;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = edge_batch_blocks_per_sm(edge_mode(params[0]));
    int grid = std::min(d.total_tiles, std::max(1, sms) * std::max(1, per_sm));
    if (launch_edge_batch(d, edge_mode(params[0]), grid, s) != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_DEVICE;
    }
    // wait, then report a bounded wait that ran out on the device
    int err = 0;
    if (cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return HVX_ERROR_DEVICE;
    }
    return err ? HVX_ERROR_TIMEOUT : HVX_SUCCESS;
}
