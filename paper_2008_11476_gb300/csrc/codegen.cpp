// Code generation for fused groups (Section 5: the paper's framework turns
// every fused OpenVX graph partition into source code specialised to it and
// compiles that; here the source is CUDA C++ for sm_103a, compiled at verify
// time with NVRTC and loaded with the driver API).
//
// The generated kernel computes one output tile per CTA, like the staged-tile
// interpreter (kernels_generic.cu), with the same results cell for cell:
//   * every operator, constant, format, border fill and coefficient is
//     compiled in (constant propagation); zero convolution taps disappear and
//     sums are accumulated in 32 bits where the input range allows;
//   * only images that a local operator reads are staged in shared memory;
//     point operators, and local operators read only by point operators, are
//     evaluated inline where their value is used, each once per cell;
//   * images staged at the same depth of local operators with the same halo
//     are produced by one pass over the cells (e.g. the three Harris / Tomasi
//     products, from one inline Sobel);
//   * tiles whose cells all lie inside every image's valid region (all but a
//     ring of tiles along the image border) run without a single bounds,
//     validity or fill test; the others run the checked instance of the same
//     template.
// Kernels are cached by source text, so graphs of the same shape share one.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "hvx_internal.h"
#include "jit_params.h"
#include "kernel_params.h"

namespace hvx {

static_assert(HVX_JIT_MAX_BUF == GEN_MAX_BUF, "generated kernels index the group's buffers");
static_assert(HVX_JIT_MAX_EXT == GEN_MAX_EXT, "generated kernels index the group's images");

namespace {

// Headers compiled into the library (written by _build.py from csrc/): the
// exact point arithmetic and the launch parameter block.
#include "jit_headers.inc"

// ---------------------------------------------------------------------------
// NVRTC, opened at run time (the toolkit's libnvrtc), and the driver calls
// that load and launch a compiled module.

typedef int (*FnCreate)(void**, const char*, const char*, int, const char* const*,
                        const char* const*);
typedef int (*FnCompile)(void*, int, const char* const*);
typedef int (*FnSize)(void*, size_t*);
typedef int (*FnGet)(void*, char*);
typedef int (*FnDestroy)(void**);
typedef CUresult (*FnModuleLoadData)(CUmodule*, const void*);
typedef CUresult (*FnModuleGetFunction)(CUfunction*, CUmodule, const char*);
typedef CUresult (*FnFuncSetAttribute)(CUfunction, CUfunction_attribute, int);
typedef CUresult (*FnLaunchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned,
                                   unsigned, unsigned, CUstream, void**, void**);
typedef CUresult (*FnLaunchKernelEx)(const CUlaunchConfig*, CUfunction, void**, void**);

struct Nvrtc {
    bool ok = false;
    std::string why;
    FnCreate create = nullptr;
    FnCompile compile = nullptr;
    FnSize cubin_size = nullptr, log_size = nullptr;
    FnGet cubin = nullptr, log = nullptr;
    FnDestroy destroy = nullptr;
};

Nvrtc& nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<std::string> dirs;
        if (const char* h = getenv("CUDA_HOME")) dirs.push_back(std::string(h) + "/lib64/");
        dirs.push_back("/usr/local/cuda/lib64/");
        dirs.push_back("");
        void* lib = nullptr;
        for (const std::string& d : dirs) {
            // the builtins library first, so that NVRTC finds it whatever the
            // loader's search path
            dlopen((d + "libnvrtc-builtins.so.13.0").c_str(), RTLD_NOW | RTLD_GLOBAL);
            lib = dlopen((d + "libnvrtc.so.13").c_str(), RTLD_NOW | RTLD_GLOBAL);
            if (lib) break;
        }
        if (!lib) {
            n.why = "libnvrtc.so.13 not found";
            return;
        }
        n.create = (FnCreate)dlsym(lib, "nvrtcCreateProgram");
        n.compile = (FnCompile)dlsym(lib, "nvrtcCompileProgram");
        n.cubin_size = (FnSize)dlsym(lib, "nvrtcGetCUBINSize");
        n.cubin = (FnGet)dlsym(lib, "nvrtcGetCUBIN");
        n.log_size = (FnSize)dlsym(lib, "nvrtcGetProgramLogSize");
        n.log = (FnGet)dlsym(lib, "nvrtcGetProgramLog");
        n.destroy = (FnDestroy)dlsym(lib, "nvrtcDestroyProgram");
        n.ok = n.create && n.compile && n.cubin_size && n.cubin && n.log_size && n.log &&
               n.destroy;
        if (!n.ok) n.why = "libnvrtc lacks an entry point";
    });
    return n;
}

struct Driver {
    bool ok = false;
    FnModuleLoadData load = nullptr;
    FnModuleGetFunction get = nullptr;
    FnFuncSetAttribute attr = nullptr;
    FnLaunchKernel launch = nullptr;
    FnLaunchKernelEx launch_ex = nullptr;  // optional: programmatic dependent launches
};

Driver& driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        auto entry = [](const char* name) -> void* {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion(name, &fn, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            return fn;
        };
        d.load = (FnModuleLoadData)entry("cuModuleLoadData");
        d.get = (FnModuleGetFunction)entry("cuModuleGetFunction");
        d.attr = (FnFuncSetAttribute)entry("cuFuncSetAttribute");
        d.launch = (FnLaunchKernel)entry("cuLaunchKernel");
        d.launch_ex = (FnLaunchKernelEx)entry("cuLaunchKernelEx");
        d.ok = d.load && d.get && d.attr && d.launch;
    });
    return d;
}

}  // namespace

// One compiled (and, with a device, loaded) generated kernel.
struct JitKernel {
    std::string source;
    std::string log;
    std::vector<char> cubin;
    bool compiled = false;
    int device = -1;           // loaded on this device (-1: not loaded)
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    CUfunction fn_batch = nullptr;  // several images per launch
    int smem_bytes = 0;
    int tw = 0, th = 0;
};

namespace {

// ---------------------------------------------------------------------------
// Source emission

constexpr int kThreads = 256;  // 8 warps: warps take rows, lanes columns

struct Emitter {
    const GenericDesc& d;
    const std::vector<std::string>& user;  // user-defined operators' code
    int tw = 0, th = 0;
    std::vector<int> producer;  // buffer -> stage index, or -1 (external input)
    std::vector<int> ext_in;    // buffer -> external input index, or -1
    std::vector<bool> staged;   // buffer lives in shared memory
    std::vector<int> level;     // depth of local operators
    // Separable window sums and convolutions (a rank-one integer kernel
    // r s^T of at least 15 taps): row sums with s are staged in shared
    // memory, the column sum with r is taken where the value is used.
    std::vector<std::vector<int>> sep_s, sep_r;  // per stage; empty: not separable
    // global operators (MeanStdDev, MinMaxLoc, Histogram): reductions of their
    // input over the output pass's cells; res[j] of the launch parameters
    std::vector<int> globals;

    // Shared-memory slots: staged images (slot = buffer) and row-sum buffers
    // (slot = n_buf + stage); live from the pass that writes them to the
    // last pass that reads them, so slots of disjoint lifetimes share words.
    struct Slot {
        int w = 0, h = 0;
        int def = -1, last = -1;
        int off = -1;
    };
    std::vector<Slot> slot;

    enum PassKind { LOAD, ROW, CELLS, OUT };
    struct Pass {
        PassKind kind = CELLS;
        int h = 0;                  // halo of the cells (CELLS / OUT)
        std::vector<int> targets;   // buffers (LOAD / CELLS) or stages (ROW)
        std::vector<bool> need_op;  // CELLS / OUT: stages evaluated at each cell
        std::vector<bool> need_ld;  // external images read directly
        std::vector<bool> read_cell;  // staged buffers read at the cell itself
    };
    std::vector<Pass> passes;
    int smem_words = 0;
    std::ostringstream o;

    Emitter(const GenericDesc& desc, const std::vector<std::string>& u) : d(desc), user(u) {
        const char* env = std::getenv("HVX_CODEGEN_TMA");
        tma = !(env && env[0] == '0');
    }
    bool tma = true;                 // stage U8 inputs of interior tiles by TMA
    std::vector<int> load_bar;       // per pass: word offset of its mbarrier, or -1

    static bool is_local(int op) {
        return op == OP_GAUSS || op == OP_BOX || op == OP_SOBEL_X || op == OP_SOBEL_Y ||
               op == OP_CONV || op == OP_LSUM || op == OP_DILATE || op == OP_ERODE ||
               op == OP_MEDIAN || op == OP_USER_LOCAL;
    }

    // A user operator's code with its placeholders replaced by reads, the
    // 64-bit result saturated to the output format.
    std::string user_expr(const GenStage& st, bool local) const {
        std::string s = user[st.i0];
        auto swap = [&](const std::string& from, const std::string& to) {
            for (size_t at = s.find(from); at != std::string::npos; at = s.find(from, at + to.size()))
                s.replace(at, from.size(), to);
        };
        if (local) {
            for (size_t at = s.find("HVX_TAP("); at != std::string::npos; at = s.find("HVX_TAP(")) {
                const size_t end = s.find(')', at);
                int dx = 0, dy = 0;
                std::sscanf(s.c_str() + at, "HVX_TAP(%d,%d)", &dx, &dy);
                s.replace(at, end + 1 - at, "((long long)" + tap(st.in[0], dx, dy) + ")");
            }
        } else {
            const char* names[3] = {"HVX_A", "HVX_B", "HVX_C"};
            for (int i = 0; i < 3; ++i)
                if (st.in[i] >= 0) swap(names[i], "((long long)" + val(st.in[i]) + ")");
        }
        const char* sat = st.i1 == HVX_DF_U8 ? "sat64_u8" : st.i1 == HVX_DF_S16 ? "sat64_s16"
                                                                             : "sat64_s32";
        return std::string(sat) + "(" + s + ")";
    }

    int bw(int b) const { return tw + 2 * d.buf[b].halo; }
    int bh(int b) const { return th + 2 * d.buf[b].halo; }

    // Staged U8 images are held as bytes (a U8 image's values are 0..255),
    // in rows that start on the 4-byte boundary at or left of the region
    // (image x = x0 - A, A = halo rounded up to a multiple of 4), so that
    // interior tiles load external ones with one 32-bit load per 4 pixels.
    // Other staged images hold int32 cells.
    bool byte_slot(int b) const {
        return b < d.n_buf && staged[b] && d.buf[b].fmt == HVX_DF_U8;
    }
    // A staged U8 external input of an interior tile arrives as one TMA box:
    // its slot rows start at image x = x0 - A with A the halo rounded up to 16
    // (the box's x must be a multiple of 16 bytes), and the slot's row pitch
    // is the box width.  Used for halos of 2 or more: on the Section 6
    // applications it measured 2-4 % faster there (Gauss 5x5, FChain,
    // EdgFig2) and 3-6 % slower on halo-1 groups (Sobel, SobelX, Unsharp),
    // whose per-thread loads are fewer.
    bool tma_slot(int b) const {
        return tma && byte_slot(b) && ext_in[b] >= 0 && d.in[ext_in[b]].fmt == HVX_DF_U8 &&
               d.buf[b].halo >= 2;
    }
    int align_x(int b) const {
        const int h = d.buf[b].halo;
        return tma_slot(b) ? (h + 15) & ~15 : (h + 3) & ~3;
    }
    int slot_w(int b) const { return byte_slot(b) ? tw + 2 * align_x(b) : bw(b); }
    int slot_x(int b) const { return byte_slot(b) ? align_x(b) - d.buf[b].halo : 0; }
    int slot_words(int s) const {
        const int n = slot[s].w * slot[s].h;
        return byte_slot(s) ? ((n / 4 + 3) & ~3) : ((n + 3) & ~3);  // 16-byte aligned
    }
    int row_slot(int k) const { return d.n_buf + k; }
    bool separable(int k) const { return !sep_s[k].empty(); }

    // c (kh x kw, row-major) = r s^T with integer r, s; s primitive.
    static bool factor(const int32_t* c, int kw, int kh, std::vector<int>& s, std::vector<int>& r) {
        int i0 = -1;
        for (int i = 0; i < kh && i0 < 0; ++i)
            for (int j = 0; j < kw; ++j)
                if (c[i * kw + j] != 0) {
                    i0 = i;
                    break;
                }
        if (i0 < 0) return false;
        int g = 0;
        for (int j = 0; j < kw; ++j) {
            int a = std::abs(c[i0 * kw + j]);
            while (a) {
                const int t = g % a;
                g = a;
                a = t;
            }
        }
        s.assign(kw, 0);
        r.assign(kh, 0);
        int j0 = -1;
        for (int j = 0; j < kw; ++j) {
            s[j] = c[i0 * kw + j] / g;
            if (s[j] != 0 && j0 < 0) j0 = j;
        }
        for (int i = 0; i < kh; ++i) {
            if (c[i * kw + j0] % s[j0] != 0) return false;
            r[i] = c[i * kw + j0] / s[j0];
            for (int j = 0; j < kw; ++j)
                if ((long long)c[i * kw + j] != (long long)r[i] * s[j]) return false;
        }
        return true;
    }

    void analyse() {
        const int nb = d.n_buf;
        producer.assign(nb, -1);
        ext_in.assign(nb, -1);
        staged.assign(nb, false);
        level.assign(nb, 0);
        sep_s.assign(d.n_stage, {});
        sep_r.assign(d.n_stage, {});
        for (int e = 0; e < d.n_in; ++e) ext_in[d.in[e].buf] = e;
        globals.clear();
        for (int k = 0; k < d.n_stage; ++k) {
            const GenStage& st = d.st[k];
            if (op_is_global(st.op)) {
                globals.push_back(k);
                continue;
            }
            producer[st.out] = k;
            if (is_local(st.op)) staged[st.in[0]] = true;
            const int kw = 2 * st.rx + 1, kh = 2 * st.ry + 1;
            if (kw < 3 || kh < 3 || kw * kh < 15) continue;
            if (st.op == OP_LSUM) {
                sep_s[k].assign(kw, 1);
                sep_r[k].assign(kh, 1);
            } else if (st.op == OP_CONV) {
                std::vector<int> fs, fr;
                long long bound = 0;
                for (int i = 0; i < kw * kh; ++i)
                    bound += std::llabs((long long)d.coeff[st.coeff_off + i]);
                bound *= max_abs(d.buf[st.in[0]].fmt);
                // row sums are stored as int32: only when the whole sum fits
                if (bound < (1ll << 31) && factor(d.coeff + st.coeff_off, kw, kh, fs, fr)) {
                    sep_s[k] = fs;
                    sep_r[k] = fr;
                }
            }
        }
        for (int k = 0; k < d.n_stage; ++k) {  // stages are in topological order
            const GenStage& st = d.st[k];
            if (st.out < 0) continue;
            int l = 0;
            for (int i = 0; i < 3; ++i)
                if (st.in[i] >= 0) l = std::max(l, level[st.in[i]]);
            level[st.out] = l + (is_local(st.op) ? 1 : 0);
        }
    }

    // Marks what a pass must evaluate to produce buffer b at a cell: ops
    // evaluated inline and external images read directly.  False if a local
    // operator's input is not staged yet.
    bool visit(int b, const std::vector<bool>& avail, Pass& p) {
        if (avail[b]) {
            p.read_cell[b] = true;
            return true;
        }
        if (ext_in[b] >= 0) {
            if (staged[b]) return false;
            p.need_ld[b] = true;
            return true;
        }
        const int k = producer[b];
        if (k < 0) return false;
        if (p.need_op[k]) return true;
        p.need_op[k] = true;
        const GenStage& st = d.st[k];
        if (is_local(st.op)) return avail[st.in[0]];
        for (int i = 0; i < 3; ++i)
            if (st.in[i] >= 0 && !visit(st.in[i], avail, p)) return false;
        return true;
    }

    bool add_cells_pass(const std::vector<int>& targets, int h, std::vector<bool>& avail,
                        std::vector<bool>& rows_done) {
        Pass p;
        p.kind = targets.empty() ? OUT : CELLS;
        p.h = h;
        p.targets = targets;
        p.need_op.assign(d.n_stage, false);
        p.need_ld.assign(d.n_buf, false);
        p.read_cell.assign(d.n_buf, false);
        std::vector<int> want = targets;
        if (targets.empty()) {
            for (int e = 0; e < d.n_out; ++e) want.push_back(d.out[e].buf);
            for (int k : globals) want.push_back(d.st[k].in[0]);
        }
        for (int b : want)
            if (!visit(b, avail, p)) return false;
        Pass rp;
        rp.kind = ROW;
        for (int k = 0; k < d.n_stage; ++k)
            if (p.need_op[k] && separable(k) && !rows_done[k]) {
                rp.targets.push_back(k);
                rows_done[k] = true;
            }
        if (!rp.targets.empty()) passes.push_back(rp);
        passes.push_back(p);
        for (int b : targets) avail[b] = true;
        return true;
    }

    // Pass list: staged external inputs, then staged op outputs by depth of
    // local operators and halo (larger first; equal ones share a pass), each
    // preceded by the row sums it needs, then the external outputs.
    bool plan() {
        passes.clear();
        std::vector<bool> avail(d.n_buf, false), rows_done(d.n_stage, false);
        Pass ld;
        ld.kind = LOAD;
        for (int b = 0; b < d.n_buf; ++b)
            if (staged[b] && ext_in[b] >= 0) {
                ld.targets.push_back(b);
                avail[b] = true;
            }
        if (!ld.targets.empty()) passes.push_back(ld);
        std::vector<int> order;
        for (int b = 0; b < d.n_buf; ++b)
            if (staged[b] && ext_in[b] < 0) order.push_back(b);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            if (level[a] != level[b]) return level[a] < level[b];
            return d.buf[a].halo > d.buf[b].halo;
        });
        for (size_t i = 0; i < order.size();) {
            std::vector<int> tg{order[i]};
            size_t j = i + 1;
            while (j < order.size() && level[order[j]] == level[order[i]] &&
                   d.buf[order[j]].halo == d.buf[order[i]].halo)
                tg.push_back(order[j++]);
            if (!add_cells_pass(tg, d.buf[order[i]].halo, avail, rows_done)) return false;
            i = j;
        }
        return add_cells_pass({}, 0, avail, rows_done);
    }

    // Slot sizes for the current tile, lifetimes, and first-fit offsets among
    // slots whose lifetimes overlap; returns the words needed.
    int allocate() {
        slot.assign(d.n_buf + d.n_stage, Slot{});
        for (int b = 0; b < d.n_buf; ++b)
            if (staged[b]) {
                slot[b].w = slot_w(b);
                slot[b].h = bh(b);
            }
        for (int k = 0; k < d.n_stage; ++k)
            if (separable(k)) {
                const int hl = d.buf[d.st[k].out].halo;
                slot[row_slot(k)].w = tw + 2 * hl;
                slot[row_slot(k)].h = th + 2 * hl + 2 * d.st[k].ry;
            }
        auto use = [&](int s, int i) { slot[s].last = std::max(slot[s].last, i); };
        for (int i = 0; i < (int)passes.size(); ++i) {
            const Pass& p = passes[i];
            if (p.kind == LOAD) {
                for (int b : p.targets) slot[b].def = i;
            } else if (p.kind == ROW) {
                for (int k : p.targets) {
                    slot[row_slot(k)].def = i;
                    use(d.st[k].in[0], i);
                }
            } else {
                for (int b : p.targets) slot[b].def = i;
                for (int b = 0; b < d.n_buf; ++b)
                    if (p.read_cell[b]) use(b, i);
                for (int k = 0; k < d.n_stage; ++k)
                    if (p.need_op[k] && is_local(d.st[k].op))
                        use(separable(k) ? row_slot(k) : d.st[k].in[0], i);
            }
        }
        std::vector<int> ids;
        for (int s = 0; s < (int)slot.size(); ++s)
            if (slot[s].w > 0) {
                if (slot[s].last < slot[s].def) slot[s].last = slot[s].def;
                ids.push_back(s);
            }
        std::stable_sort(ids.begin(), ids.end(),
                         [&](int a, int b) { return slot[a].def < slot[b].def; });
        int words = 0;
        std::vector<int> placed;
        for (int s : ids) {
            const int n = slot_words(s);
            std::vector<std::pair<int, int>> busy;
            for (int t : placed)
                if (slot[t].def <= slot[s].last && slot[s].def <= slot[t].last)
                    busy.push_back({slot[t].off, slot[t].off + slot_words(t)});
            std::sort(busy.begin(), busy.end());
            int off = 0;
            for (const auto& iv : busy) {
                if (off + n <= iv.first) break;
                off = std::max(off, iv.second);
            }
            slot[s].off = off;
            placed.push_back(s);
            words = std::max(words, off + n);
        }
        return words;
    }

    // Tile shape: the largest whose shared memory fits twice per SM.
    bool choose_tile() {
        static const int shapes[][2] = {{128, 32}, {128, 16}, {64, 16}, {32, 16}};
        for (const auto& sh : shapes) {
            tw = sh[0];
            th = sh[1];
            smem_words = allocate();
            if (smem_words * 4 <= 110 * 1024) return true;
        }
        return false;
    }

    static std::string lit64(long long v) {
        if (v == (-9223372036854775807ll - 1)) return "(-9223372036854775807LL - 1)";
        return "(" + std::to_string(v) + "LL)";
    }

    static std::string flit(float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return "__int_as_float(" + std::to_string((int32_t)u) + ")";
    }

    // Largest |value| an image of this format holds.
    static long long max_abs(int fmt) {
        switch (fmt) {
            case HVX_DF_U8: return 255;
            case HVX_DF_S16: return 32768;
            case HVX_DF_UYVY: return 65535;
            default: return 2147483648ll;
        }
    }

    // Cell passes are emitted row-blocked: a thread computes `row_block`
    // vertically adjacent cells of one column per iteration, and every
    // shared-memory value they read is loaded once into a named variable
    // (a window of k rows serves k cells).  While a row of the block is being
    // emitted, `row` is its index; reads register their (slot, row, column)
    // in `loads`.  The output pass of an unhaloed tile is also column-blocked
    // (`col`: the cell's column in a block of 4 adjacent ones).
    int row = -1, col = 0;
    const std::vector<bool>* need_now = nullptr;  // stages evaluated inline in the current pass
    mutable std::map<std::tuple<int, int, int>, std::string> loads;
    std::vector<bool> cell_read;  // staged buffers read at the cell itself this pass

    static std::string enc(int v) { return v < 0 ? "m" + std::to_string(-v) : std::to_string(v); }

    std::string load_var(int s, int r, int dx) const {
        const auto key = std::make_tuple(s, r, dx);
        auto it = loads.find(key);
        if (it != loads.end()) return it->second;
        const std::string name = "t" + std::to_string(s) + "_" + enc(r) + "_" + enc(dx);
        loads[key] = name;
        return name;
    }

    // Expression of the value of buffer b at the current cell.
    std::string val(int b) const {
        if (row < 0) return "v" + std::to_string(b);
        if (cell_read[b]) return load_var(b, row, col);
        return "v" + std::to_string(b) + "_" + std::to_string(row) +
               (col ? "_" + std::to_string(col) : "");
    }

    // Read of staged buffer b at offset (dx, dy) from the current cell.
    std::string tap(int b, int dx, int dy) const {
        if (row >= 0) return load_var(b, row + dy, dx + col);
        const int off = dy * slot_w(b) + dx;
        std::string s = "B" + std::to_string(b) + "[q" + std::to_string(b);
        if (off > 0) s += " + " + std::to_string(off);
        if (off < 0) s += " - " + std::to_string(-off);
        return s + "]";
    }

    std::string point_expr(const GenStage& st) const {
        const std::string a = st.in[0] >= 0 ? val(st.in[0]) : "0";
        const std::string b = st.in[1] >= 0 ? val(st.in[1]) : "0";
        const std::string c = st.in[2] >= 0 ? val(st.in[2]) : "0";
        switch (st.op) {
            case OP_MAG: return "magnitude_s16(" + a + ", " + b + ")";
            case OP_PHASE: return "(int)phase_u8(" + a + ", " + b + ")";
            case OP_THRESH: {
                std::string t;
                const int pm = producer[st.in[0]];
                if (!st.i3 && st.i0 == HVX_THRESHOLD_BINARY && pm >= 0 && d.st[pm].op == OP_MAG &&
                    need_now && (*need_now)[pm]) {
                    // Magnitude -> binary threshold: round(sqrt(s)) > T is s > T^2 + T
                    // for 0 <= T < 32767 (s = gx^2 + gy^2 an integer, the rounding
                    // half up, ties impossible); always for T < 0 and never for
                    // T >= 32767 (the magnitude saturates at 32767)
                    const long long T = st.k0;
                    if (T < 0) {
                        t = "true";
                    } else if (T >= 32767) {
                        t = "false";
                    } else {
                        const std::string gx = val(d.st[pm].in[0]), gy = val(d.st[pm].in[1]);
                        t = "((unsigned)(" + gx + " * " + gx + ") + (unsigned)(" + gy + " * " + gy +
                            ") > " + std::to_string(T * T + T) + "u)";
                    }
                } else if (st.i3) {
                    const std::string f = "__int_as_float(" + a + ")";
                    t = st.i0 == HVX_THRESHOLD_BINARY
                            ? "(" + f + " > " + flit(st.f0) + ")"
                            : "!(" + f + " > " + flit(st.f1) + " || " + f + " < " + flit(st.f0) +
                                  ")";
                } else {
                    const std::string v = "(long long)" + a;
                    t = st.i0 == HVX_THRESHOLD_BINARY
                            ? "(" + v + " > " + lit64(st.k0) + ")"
                            : "!(" + v + " > " + lit64(st.k1) + " || " + v + " < " +
                                  lit64(st.k0) + ")";
                }
                return "(" + t + " ? " + std::to_string(st.i1) + " : " + std::to_string(st.i2) +
                       ")";
            }
            case OP_CHX: return "((" + a + " >> 8) & 0xFF)";
            case OP_ADD:
            case OP_SUB:
            case OP_ABSDIFF: {
                std::string r = st.op == OP_ADD   ? "(" + a + " + " + b + ")"
                                : st.op == OP_SUB ? "(" + a + " - " + b + ")"
                                                  : "abs(" + a + " - " + b + ")";
                if (st.i1 == HVX_DF_U8) return st.i0 ? "sat_u8(" + r + ")" : "(" + r + " & 0xFF)";
                return st.i0 ? "sat_s16(" + r + ")"
                             : "(int)(short)(unsigned short)(" + r + " & 0xFFFF)";
            }
            case OP_MUL: return "(int)((unsigned)" + a + " * (unsigned)" + b + ")";
            case OP_AND: return "(" + a + " & " + b + ")";
            case OP_OR: return "(" + a + " | " + b + ")";
            case OP_XOR: return "(" + a + " ^ " + b + ")";
            case OP_NOT: return "(~" + a + " & 0xFF)";
            case OP_HARRIS:
                return "__float_as_int(ratio_to_float(harris_q(" + a + ", " + b + ", " + c + ", " +
                       lit64(st.k0) + ", " + lit64(st.k1) + "), " + lit64(st.k1) + "))";
            case OP_TOMASI:
                return "__float_as_int(tomasi_response_f32(" + a + ", " + b + ", " + c + "))";
            case OP_USER_POINT: return user_expr(st, false);
            case OP_CONVDEPTH:
                if (st.i1 == st.i3) return a;
                if (st.i1 == HVX_DF_S16)
                    return "(int)((unsigned)" + a + " << " + std::to_string(st.i0) + ")";
                return st.i2 ? "sat_u8(" + a + " >> " + std::to_string(st.i0) + ")"
                             : "((" + a + " >> " + std::to_string(st.i0) + ") & 0xFF)";
            case OP_MULTIPLY: {
                const std::string v = "multiply_scaled(" + a + ", " + b + ", " + lit64(st.k0) +
                                      ", " + std::to_string(st.i3) + ", " +
                                      (st.i2 ? "true" : "false") + ")";
                if (st.i1 == HVX_DF_U8)
                    return st.i0 ? "sat64_u8(" + v + ")" : "(int)(" + v + " & 0xFF)";
                return st.i0 ? "sat64_s16(" + v + ")" : "wrap64_s16(" + v + ")";
            }
        }
        return "0";
    }

    // Statements assigning the local operator of stage k at the current cell
    // to variable `dst` (its input is staged).
    void emit_local(const GenStage& st, const std::string& dst, const std::string& ind) {
        const int b = st.in[0];
        auto T = [&](int dx, int dy) { return tap(b, dx, dy); };
        switch (st.op) {
            case OP_GAUSS:
            case OP_BOX: {
                const bool g = st.op == OP_GAUSS, near = st.rounding == HVX_ROUND_TO_NEAREST;
                o << ind << "{\n" << ind << "  const int t = ";
                if (g)
                    o << "(" << T(-1, -1) << " + 2 * " << T(0, -1) << " + " << T(1, -1) << ") + 2 * ("
                      << T(-1, 0) << " + 2 * " << T(0, 0) << " + " << T(1, 0) << ") + (" << T(-1, 1)
                      << " + 2 * " << T(0, 1) << " + " << T(1, 1) << ");\n";
                else {
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx)
                            o << T(dx, dy) << ((dx == 1 && dy == 1) ? ";\n" : " + ");
                }
                if (g)
                    o << ind << "  " << dst << " = " << (near ? "(t + 8) >> 4" : "t >> 4") << ";\n";
                else
                    o << ind << "  " << dst << " = " << (near ? "(t + 4) / 9" : "t / 9") << ";\n";
                o << ind << "}\n";
                return;
            }
            case OP_SOBEL_X:
                o << ind << dst << " = (" << T(1, -1) << " - " << T(-1, -1) << ") + 2 * (" << T(1, 0)
                  << " - " << T(-1, 0) << ") + (" << T(1, 1) << " - " << T(-1, 1) << ");\n";
                return;
            case OP_SOBEL_Y:
                o << ind << dst << " = (" << T(-1, 1) << " - " << T(-1, -1) << ") + 2 * (" << T(0, 1)
                  << " - " << T(0, -1) << ") + (" << T(1, 1) << " - " << T(1, -1) << ");\n";
                return;
            case OP_DILATE:
            case OP_ERODE: {
                const char* f = st.op == OP_DILATE ? "max" : "min";
                o << ind << "{\n" << ind << "  int m = " << T(-1, -1) << ";\n";
                for (int k = 1; k < 9; ++k)
                    o << ind << "  m = " << f << "(m, " << T(k % 3 - 1, k / 3 - 1) << ");\n";
                o << ind << "  " << dst << " = m;\n" << ind << "}\n";
                return;
            }
            case OP_MEDIAN: {
                // median of nine by the exchange network of Paeth (Graphics Gems)
                o << ind << "{\n";
                for (int k = 0; k < 9; ++k)
                    o << ind << "  int m" << k << " = " << T(k % 3 - 1, k / 3 - 1) << ";\n";
                static const int net[19][2] = {{1, 2}, {4, 5}, {7, 8}, {0, 1}, {3, 4}, {6, 7},
                                               {1, 2}, {4, 5}, {7, 8}, {0, 3}, {5, 8}, {4, 7},
                                               {3, 6}, {1, 4}, {2, 5}, {4, 7}, {4, 2}, {6, 4},
                                               {4, 2}};
                for (const auto& e : net)
                    o << ind << "  { const int lo = min(m" << e[0] << ", m" << e[1]
                      << "), hi = max(m" << e[0] << ", m" << e[1] << "); m" << e[0] << " = lo; m"
                      << e[1] << " = hi; }\n";
                o << ind << "  " << dst << " = m4;\n" << ind << "}\n";
                return;
            }
            case OP_CONV: {
                const int kw = 2 * st.rx + 1, kh = 2 * st.ry + 1;
                long long bound = 0;
                for (int i = 0; i < kw * kh; ++i)
                    bound += std::llabs((long long)d.coeff[st.coeff_off + i]);
                bound *= max_abs(d.buf[b].fmt);
                const bool narrow = bound < (1ll << 31);
                const char* acc = narrow ? "int" : "long long";
                o << ind << "{\n" << ind << "  " << acc << " t = 0;\n";
                for (int dy = 0; dy < kh; ++dy)
                    for (int dx = 0; dx < kw; ++dx) {
                        const int c = d.coeff[st.coeff_off + dy * kw + dx];
                        if (c == 0) continue;
                        o << ind << "  t += ";
                        if (c != 1) o << "(" << acc << ")" << c << " * ";
                        o << "(" << acc << ")" << T(dx - st.rx, dy - st.ry) << ";\n";
                    }
                o << ind << "  t >>= " << st.shift << ";\n";
                if (st.i0 == HVX_DF_U8)
                    o << ind << "  " << dst << " = (int)(t > 255 ? 255 : (t < 0 ? 0 : t));\n";
                else
                    o << ind << "  " << dst
                      << " = (int)(t > 32767 ? 32767 : (t < -32768 ? -32768 : t));\n";
                o << ind << "}\n";
                return;
            }
            case OP_USER_LOCAL:
                o << ind << dst << " = " << user_expr(st, true) << ";\n";
                return;
            case OP_LSUM: {
                // int32 wrap-around sum: the low 32 bits of the exact sum
                o << ind << "{\n" << ind << "  unsigned t = 0;\n";
                for (int dy = -st.ry; dy <= st.ry; ++dy)
                    for (int dx = -st.rx; dx <= st.rx; ++dx)
                        o << ind << "  t += (unsigned)" << T(dx, dy) << ";\n";
                o << ind << "  " << dst << " = (int)t;\n" << ind << "}\n";
                return;
            }
        }
    }

    // The cell loop of a pass: warps take rows, lanes consecutive columns
    // (conflict-free shared-memory rows); cell (c, r) is image pixel
    // (x0 + c - xo, y0 + r - yo).
    void open_cells(int rows, int cols, int xo, int yo, bool unroll_rows, bool xy = true) {
        o << (unroll_rows ? "  #pragma unroll\n" : "  #pragma unroll 1\n")
          << "  for (int r = warp; r < " << rows << "; r += " << kThreads / 32 << ") {\n"
          << "    #pragma unroll\n"
          << "    for (int c = lane; c < " << cols << "; c += 32) {\n";
        if (xy) o << "      const int x = x0 + c - " << xo << ", y = y0 + r - " << yo << ";\n";
    }
    void close_cells() { o << "    }\n  }\n"; }

    // Fill value of a cell of staged buffer b outside the image:
    // `clamped_read` reads the buffer (or the external image) at the nearest
    // image pixel.
    std::string fill_expr(int b, const std::string& clamped_read) const {
        const GenBuf& g = d.buf[b];
        if (g.fill == FILL_CONSTANT) return std::to_string(g.cval);
        if (g.fill == FILL_REPLICATE) return clamped_read;
        return "0";
    }

    // Coordinates an external input's out-of-image cell reads.
    std::string fill_coords(int b) const {
        switch (d.buf[b].fill) {
            case FILL_MIRROR: return "hvx_mirror(x, p.W), hvx_mirror(y, p.H))";
            case FILL_REPEAT: return "hvx_repeat(x, p.W), hvx_repeat(y, p.H))";
            default: return "min(max(x, 0), p.W - 1), min(max(y, 0), p.H - 1))";
        }
    }

    std::string slot_name(int s) const {
        return s < d.n_buf ? "B" + std::to_string(s) : "R" + std::to_string(s - d.n_buf);
    }

    // Interior tiles: the staged U8 external inputs of a load pass as TMA
    // boxes on one mbarrier (thread 0 initialises and issues; every thread
    // waits, boundedly).  GMAP: the tensor maps are in global memory (the
    // batched entry point) and are acquired before use.
    void emit_tma_load(const std::vector<int>& T, int bar_words) {
        int bytes = 0;
        for (int b : T) bytes += slot_w(b) * bh(b);
        o << "  if (!CHECK) {  // TMA boxes of the staged U8 inputs\n"
          << "    unsigned long long* const bar = (unsigned long long*)(smem + " << bar_words
          << ");\n"
          << "    if (threadIdx.x == 0) hvx_mbar_init(bar);\n"
          << "    __syncthreads();\n"
          << "    if (threadIdx.x == 0) {\n"
          << "      hvx_expect_tx(bar, " << bytes << "u);\n";
        for (int b : T) {
            const int e = ext_in[b];
            o << "      if (GMAP) hvx_tmap_acquire(&p.tmap[" << e << "]);\n"
              << "      hvx_tma_2d(B" << b << ", &p.tmap[" << e << "], bar, x0 - " << align_x(b)
              << ", y0 - " << d.buf[b].halo << ");\n";
        }
        o << "    }\n    hvx_mbar_wait(bar, p.err);\n  }\n";
    }

    // Box of the TMA-staged input e: (e, width, height); none without TMA.
    std::vector<std::array<int, 3>> tma_boxes() const {
        std::vector<std::array<int, 3>> v;
        for (int b = 0; b < d.n_buf; ++b)
            if (tma_slot(b)) v.push_back({ext_in[b], slot_w(b), bh(b)});
        return v;
    }

    // All loads of a staged external input are independent: both loops are
    // unrolled so that they are all in flight at once.
    void emit_load(int b) {
        const int e = ext_in[b], h = d.buf[b].halo;
        const std::string ld = "hvx_ld<" + std::to_string(d.in[e].fmt) + ">(p.in[" +
                               std::to_string(e) + "], p.in_pitch[" + std::to_string(e) + "], ";
        o << "  // external input " << e << " -> B" << b << " (halo " << h << ")\n";
        if (tma_slot(b)) {  // interior tiles: the TMA box (emit_tma_load)
            o << "  if (CHECK) {\n";
            open_cells(bh(b), bw(b), h, h, true);
            o << "      int v;\n"
              << "      if (x >= 0 && x < p.W && y >= 0 && y < p.H) v = " << ld << "x, y);\n"
              << "      else v = "
              << (d.buf[b].fill == FILL_MIRROR || d.buf[b].fill == FILL_REPEAT
                      ? ld + fill_coords(b)
                      : fill_expr(b, ld + fill_coords(b)))
              << ";\n"
              << "      B" << b << "[r * " << slot_w(b) << " + c + " << slot_x(b)
              << "] = (unsigned char)v;\n";
            close_cells();
            o << "  }\n";
            return;
        }
        if (byte_slot(b)) {
            // interior tiles: the region's rows are inside the image, and the
            // words [x0 - A, x0 + tw + A) stay inside each row's pitch
            const int A = align_x(b), words = slot_w(b) / 4, rows = bh(b);
            o << "  if (!CHECK) {\n"
              << "    const unsigned char* const g0 = (const unsigned char*)p.in[" << e
              << "] + (unsigned long long)(y0 - " << h << ") * p.in_pitch[" << e << "] + (x0 - " << A
              << ");\n"
              << "    #pragma unroll 8\n"
              << "    for (int i = threadIdx.x; i < " << rows * words << "; i += " << kThreads
              << ") {\n"
              << "      const int r = i / " << words << ", k = i - r * " << words << ";\n"
              << "      ((unsigned*)B" << b << ")[i] = __ldg((const unsigned*)(g0 + "
                 "(unsigned long long)r * p.in_pitch["
              << e << "]) + k);\n"
              << "    }\n  } else {\n";
            open_cells(bh(b), bw(b), h, h, true);
            o << "      int v;\n"
              << "      if (x >= 0 && x < p.W && y >= 0 && y < p.H) v = " << ld << "x, y);\n"
              << "      else v = "
              << (d.buf[b].fill == FILL_MIRROR || d.buf[b].fill == FILL_REPEAT
                      ? ld + fill_coords(b)
                      : fill_expr(b, ld + fill_coords(b)))
              << ";\n"
              << "      B" << b << "[r * " << slot_w(b) << " + c + " << slot_x(b)
              << "] = (unsigned char)v;\n";
            close_cells();
            o << "  }\n";
            return;
        }
        open_cells(bh(b), bw(b), h, h, true);
        o << "      int v;\n"
          << "      if (!CHECK || (x >= 0 && x < p.W && y >= 0 && y < p.H)) v = " << ld
          << "x, y);\n"
          << "      else v = "
          << (d.buf[b].fill == FILL_MIRROR || d.buf[b].fill == FILL_REPEAT
                  ? ld + fill_coords(b)
                  : fill_expr(b, ld + fill_coords(b)))
          << ";\n"
          << "      B" << b << "[r * " << bw(b) << " + c] = v;\n";
        close_cells();
    }

    // Row sums of separable stage k over its output region grown by its row
    // radius; its staged input covers that region (input halo >= output
    // halo + radius) and holds border fills where it leaves the image.
    void emit_row(int k) {
        const GenStage& st = d.st[k];
        const int b = st.in[0], hb = d.buf[b].halo, hl = d.buf[st.out].halo;
        const Slot& R = slot[row_slot(k)];
        o << "  // row sums of op " << k << " -> R" << k << " (" << R.w << " x " << R.h << ")\n";
        // columns [0, W4) four at a time, the rest one cell per thread
        const int W4 = R.w & ~127;
        if (W4 > 0) emit_row4(k, W4);
        if (W4 == R.w) return;
        if (W4 > 0) {
            const int rest = R.w - W4;
            o << "  for (int i = threadIdx.x; i < " << R.h * rest << "; i += " << kThreads
              << ") {\n    {\n      const int r = i / " << rest << ", c = " << W4 << " + i % "
              << rest << ";\n";
        } else {
            open_cells(R.h, R.w, 0, 0, false, false);
        }
        o << "      const int q = (r + " << hb - hl - st.ry << ") * " << slot_w(b) << " + c + "
          << hb - hl + slot_x(b) << ";\n";
        const bool lsum = st.op == OP_LSUM;
        o << "      " << (lsum ? "unsigned" : "int") << " t = 0;\n";
        for (int j = 0; j < (int)sep_s[k].size(); ++j) {
            const int c = sep_s[k][j];
            if (c == 0) continue;
            const int off = j - st.rx;
            const std::string rd = "B" + std::to_string(b) + "[q" +
                                   (off > 0 ? " + " + std::to_string(off)
                                            : off < 0 ? " - " + std::to_string(-off) : "") +
                                   "]";
            if (lsum)
                o << "      t += (unsigned)" << rd << ";\n";
            else
                o << "      t += " << (c == 1 ? "" : std::to_string(c) + " * ") << rd << ";\n";
        }
        o << "      R" << k << "[r * " << R.w << " + c] = (int)t;\n";
        close_cells();
    }

    // Row sums of 4 adjacent cells per thread over columns [0, W) (W a
    // multiple of 128): the 4 + 2 rx input values of the block are read once
    // -- from a byte slot as the aligned 32-bit words that hold them, the
    // bytes taken by shifts -- and the 4 sums go out in one 16-byte store (two
    // 8-byte stores when the row length is not a multiple of 4).  Values and
    // their order of summation are the scalar form's.
    void emit_row4(int k, int W) {
        const GenStage& st = d.st[k];
        const int b = st.in[0], hb = d.buf[b].halo, hl = d.buf[st.out].halo;
        const Slot& R = slot[row_slot(k)];
        const int rx = st.rx, n = 4 + 2 * rx;
        const int dr = hb - hl - st.ry;          // slot row of block row r
        const int lo = hb - hl + slot_x(b) - rx;  // slot column of value 0 minus c
        const bool lsum = st.op == OP_LSUM;
        o << "  #pragma unroll 1\n"
          << "  for (int r = warp; r < " << R.h << "; r += " << kThreads / 32 << ") {\n"
          << "    #pragma unroll\n"
          << "    for (int c = 4 * lane; c < " << W << "; c += 128) {\n";
        std::vector<std::string> u(n);
        if (byte_slot(b)) {
            const int m = lo & 3, nw = (m + n + 3) / 4;
            o << "      const unsigned* const wp = (const unsigned*)B" << b << " + (r + " << dr
              << ") * " << slot_w(b) / 4 << " + (c >> 2) + " << (lo - m) / 4 << ";\n";
            for (int w = 0; w < nw; ++w) o << "      const unsigned w" << w << " = wp[" << w << "];\n";
            for (int i = 0; i < n; ++i) {
                const int pw = (m + i) / 4, pb = (m + i) % 4;
                u[i] = "u" + std::to_string(i);
                o << "      const int " << u[i] << " = (int)((w" << pw << " >> " << 8 * pb
                  << ") & 0xFFu);\n";
            }
        } else {
            o << "      const int q = (r + " << dr << ") * " << slot_w(b) << " + c + " << lo << ";\n";
            for (int i = 0; i < n; ++i) {
                u[i] = "u" + std::to_string(i);
                o << "      const int " << u[i] << " = B" << b << "[q + " << i << "];\n";
            }
        }
        for (int j = 0; j < 4; ++j) {
            o << "      " << (lsum ? "unsigned" : "int") << " t" << j << " = 0;\n";
            for (int jj = 0; jj < (int)sep_s[k].size(); ++jj) {
                const int c = sep_s[k][jj];
                if (c == 0) continue;
                const std::string& rd = u[j + jj];
                if (lsum)
                    o << "      t" << j << " += (unsigned)" << rd << ";\n";
                else
                    o << "      t" << j << " += " << (c == 1 ? "" : std::to_string(c) + " * ") << rd
                      << ";\n";
            }
        }
        if (R.w % 4 == 0)
            o << "      *(int4*)&R" << k << "[r * " << R.w << " + c] = make_int4((int)t0, (int)t1, "
              << "(int)t2, (int)t3);\n";
        else if (R.w % 2 == 0)
            o << "      *(int2*)&R" << k << "[r * " << R.w << " + c] = make_int2((int)t0, (int)t1);\n"
              << "      *(int2*)&R" << k << "[r * " << R.w << " + c + 2] = make_int2((int)t2, "
              << "(int)t3);\n";
        else
            for (int j = 0; j < 4; ++j)
                o << "      R" << k << "[r * " << R.w << " + c + " << j << "] = (int)t" << j << ";\n";
        o << "    }\n  }\n";
    }

    // Column sum of separable stage k at the current cell of a pass of halo h.
    void emit_sep(int k, const std::string& dst, const std::string& ind) {
        const GenStage& st = d.st[k];
        const Slot& R = slot[row_slot(k)];
        const bool lsum = st.op == OP_LSUM;
        o << ind << "{\n" << ind << "  " << (lsum ? "unsigned" : "int") << " t = 0;\n";
        for (int i = 0; i < (int)sep_r[k].size(); ++i) {
            const int c = sep_r[k][i];
            if (c == 0) continue;
            const int off = (i - st.ry) * R.w;
            const std::string rd =
                row >= 0 ? load_var(row_slot(k), row + i - st.ry, col)
                         : "R" + std::to_string(k) + "[qR" + std::to_string(k) +
                               (off > 0 ? " + " + std::to_string(off)
                                        : off < 0 ? " - " + std::to_string(-off) : "") +
                               "]";
            if (lsum)
                o << ind << "  t += (unsigned)" << rd << ";\n";
            else
                o << ind << "  t += " << (c == 1 ? "" : std::to_string(c) + " * ") << rd << ";\n";
        }
        if (lsum) {
            o << ind << "  " << dst << " = (int)t;\n";
        } else {
            o << ind << "  t >>= " << st.shift << ";\n";
            if (st.i0 == HVX_DF_U8)
                o << ind << "  " << dst << " = t > 255 ? 255 : (t < 0 ? 0 : t);\n";
            else
                o << ind << "  " << dst << " = t > 32767 ? 32767 : (t < -32768 ? -32768 : t);\n";
        }
        o << ind << "}\n";
    }

    // Interior tiles of a column-blocked output pass: the 4 values of row i of
    // the block go out in one 4-, 8- or 16-byte store per output (columns
    // xc .. xc + 3 of an image whose rows start 16-byte aligned).
    void emit_vector_stores(int i, int h) {
        for (int e = 0; e < d.n_out; ++e) {
            const int f = d.out[e].fmt;
            const std::string v = "so" + std::to_string(e) + "_" + std::to_string(i) + "_";
            o << "      if (!CHECK && va" << e << ") {\n"
              << "        unsigned char* const rp = (unsigned char*)p.out[" << e
              << "] + (unsigned long long)(y0 + rb + " << i - h << ") * p.out_pitch[" << e
              << "];\n";
            if (f == HVX_DF_U8)
                o << "        *(unsigned*)(rp + xc) = ((unsigned)" << v << "0 & 0xFFu) | (((unsigned)"
                  << v << "1 & 0xFFu) << 8) | (((unsigned)" << v << "2 & 0xFFu) << 16) | ((unsigned)"
                  << v << "3 << 24);\n";
            else if (f == HVX_DF_S16)
                o << "        *(uint2*)(rp + 2 * xc) = make_uint2(((unsigned)" << v
                  << "0 & 0xFFFFu) | ((unsigned)" << v << "1 << 16), ((unsigned)" << v
                  << "2 & 0xFFFFu) | ((unsigned)" << v << "3 << 16));\n";
            else
                o << "        *(int4*)(rp + 4 * xc) = make_int4(" << v << "0, " << v << "1, " << v
                  << "2, " << v << "3);\n";
            o << "      }\n";
        }
    }

    // One pass over the cells of halo p.h producing the pass's staged
    // buffers or, for the last pass, the external outputs (and the global
    // operators' partial results).  Row-blocked: see `row`.
    void emit_cells(const Pass& p) {
        const int h = p.h, BH = th + 2 * h, BW = tw + 2 * h;
        int RB = BH % 4 == 0 ? 4 : BH % 2 == 0 ? 2 : 1;  // rows per block, no tail
        // a pass evaluating the corner responses keeps its 64-bit arithmetic
        // for one cell per iteration (registers)
        for (int k = 0; k < d.n_stage; ++k)
            if (p.need_op[k] && (d.st[k].op == OP_TOMASI || d.st[k].op == OP_HARRIS)) RB = 1;
        if (const char* e = getenv("HVX_CODEGEN_ROWS")) {
            const int v = atoi(e);
            if ((v == 1 || v == 2 || v == 4) && BH % v == 0) RB = v;
        }
        const bool outputs = p.kind == OUT;
        // HVX_CODEGEN_COLS=4: the output pass of an unhaloed tile in blocks
        // of 4 adjacent columns (vector loads of the values they read, one
        // vector store per row of a block on interior tiles) and at most 2
        // rows.  Off by default: on the Section 6 applications it measured 3
        // to 14 % slower than 4 rows x 1 column (more live registers under
        // the 32-register bound of 8 resident CTAs per SM).
        const char* env_cols = getenv("HVX_CODEGEN_COLS");
        const bool cols_on = env_cols && atoi(env_cols) == 4;
        const int CB = outputs && h == 0 && BW % 128 == 0 && RB > 1 && cols_on ? 4 : 1;
        if (CB > 1 && RB > 2) RB = 2;
        o << "  // pass: ";
        if (outputs)
            o << "external outputs";
        else
            for (int b : p.targets) o << "B" << b << " ";
        o << "(halo " << h << ", " << RB << " rows";
        if (CB > 1) o << " x " << CB << " columns";
        o << " per thread iteration)\n";
        std::vector<bool> vec_ok(d.n_out, false);
        if (CB > 1)
            for (int e = 0; e < d.n_out; ++e) {
                // vector stores need the row starts 16-byte aligned
                o << "  const bool va" << e << " = ((reinterpret_cast<unsigned long long>(p.out["
                  << e << "]) | p.out_pitch[" << e << "]) & 15) == 0;\n";
                vec_ok[e] = true;
            }
        if (outputs)
            for (int k : globals) {
                if (d.st[k].op == OP_MEANSTD)
                    o << "  long long g" << k << "_s1 = 0;\n  unsigned long long g" << k
                      << "_s2 = 0;\n  unsigned g" << k << "_n = 0;\n";
                else if (d.st[k].op == OP_MINMAX)
                    o << "  HvxMinMaxAcc g" << k << "_mm;\n  hvx_mm_init(g" << k << "_mm);\n";
            }
        o << "  #pragma unroll 1\n"
          << "  for (int rb = warp * " << RB << "; rb < " << BH << "; rb += " << kThreads / 32 * RB
          << ") {\n"
          << "    #pragma unroll\n"
          << "    for (int c = lane * " << CB << "; c < " << BW << "; c += " << 32 * CB << ") {\n"
          << "      const int xc = x0 + c - " << h << ";\n";
        // the rows of the block, into a buffer: their reads decide the loads
        const std::string prefix = o.str();
        o.str("");
        o.clear();
        loads.clear();
        cell_read = p.read_cell;
        need_now = &p.need_op;
        for (int i = 0; i < RB; ++i) {
          if (CB > 1)
              for (int e = 0; e < d.n_out; ++e) {
                  o << "      int";
                  for (int j = 0; j < CB; ++j)
                      o << (j ? "," : "") << " so" << e << "_" << i << "_" << j << " = 0";
                  o << ";\n";
              }
          for (int j = 0; j < CB; ++j) {
            row = i;
            col = j;
            o << "      {\n        const int x = xc + " << j << ", y = y0 + rb + " << i - h << ";\n"
              << "        const bool in_img = !CHECK || (x >= 0 && x < p.W && y >= 0 && y < p.H);\n";
            for (int b = 0; b < d.n_buf; ++b)
                if (p.need_ld[b]) {
                    const int e = ext_in[b];
                    o << "        const int " << val(b) << " = in_img ? hvx_ld<" << d.in[e].fmt
                      << ">(p.in[" << e << "], p.in_pitch[" << e << "], x, y) : 0;\n";
                }
            for (int k = 0; k < d.n_stage; ++k) {
                if (!p.need_op[k]) continue;
                const GenStage& st = d.st[k];
                const std::string v = val(st.out);
                o << "        int " << v << ";\n";
                if (separable(k))
                    emit_sep(k, v, "        ");
                else if (is_local(st.op))
                    emit_local(st, v, "        ");
                else
                    o << "        " << v << " = " << point_expr(st) << ";\n";
                o << "        if (CHECK && !hvx_in(p.valid[" << st.out << "], x, y)) " << v
                  << " = 0;\n";
            }
            o << "        if (in_img) {\n";
            if (outputs) {
                for (int e = 0; e < d.n_out; ++e) {
                    const std::string st = "hvx_st<" + std::to_string(d.out[e].fmt) + ">(p.out[" +
                                           std::to_string(e) + "], p.out_pitch[" +
                                           std::to_string(e) + "], x, y, " + val(d.out[e].buf) +
                                           ");\n";
                    if (CB > 1)
                        o << "          so" << e << "_" << i << "_" << j << " = "
                          << val(d.out[e].buf) << ";\n          if (CHECK || !va" << e << ") " << st;
                    else
                        o << "          " << st;
                }
                for (int k : globals) {
                    const GenStage& st = d.st[k];
                    const std::string v = val(st.in[0]), g = "g" + std::to_string(k);
                    o << "          if (!CHECK || hvx_in(p.valid[" << st.in[0] << "], x, y)) {\n";
                    if (st.op == OP_MEANSTD)
                        o << "            " << g << "_s1 += " << v << ";\n            " << g
                          << "_s2 += (unsigned long long)((long long)" << v << " * " << v
                          << ");\n            ++" << g << "_n;\n";
                    else if (st.op == OP_MINMAX)
                        o << "            hvx_mm_add(" << g << "_mm, " << v
                          << ", (unsigned)y * (unsigned)p.W + (unsigned)x);\n";
                    else
                        o << "            if (" << v << " >= " << st.i1 << " && " << v << " < "
                          << st.i1 + st.i2 << ") atomicAdd(&" << g << "_bins[(" << v << " - "
                          << st.i1 << ") * " << st.i0 << " / " << st.i2 << "], 1u);\n";
                    o << "          }\n";
                }
            } else {
                for (int b : p.targets)
                    o << "          B" << b << "[(rb + " << i << ") * " << slot_w(b) << " + c + "
                      << slot_x(b) << "] = " << (byte_slot(b) ? "(unsigned char)" : "") << val(b)
                      << ";\n";
            }
            o << "        }\n      }\n";
          }
          if (CB > 1) emit_vector_stores(i, h);
        }
        row = -1;
        col = 0;
        need_now = nullptr;
        const std::string rows = o.str();
        o.str("");
        o.clear();
        o << prefix;
        // base index of every slot read, then each read once
        std::vector<bool> based(slot.size(), false);
        for (const auto& kv : loads) {
            const int s = std::get<0>(kv.first);
            if (based[s]) continue;
            based[s] = true;
            if (s < d.n_buf) {
                const int dh = d.buf[s].halo - h;
                o << "      const int qb" << s << " = (rb + " << dh << ") * " << slot_w(s)
                  << " + c + " << dh + slot_x(s) << ";\n";
            } else {
                const int k = s - d.n_buf, dh = d.buf[d.st[k].out].halo - h;
                o << "      const int qb" << s << " = (rb + " << dh + d.st[k].ry << ") * "
                  << slot[s].w << " + c + " << dh << ";\n";
            }
        }
        auto plus = [](int v) {
            return v > 0 ? " + " + std::to_string(v) : v < 0 ? " - " + std::to_string(-v) : "";
        };
        // reads of one slot row, grouped; in column blocks they are covered by
        // aligned chunks of 4 values (one 16-byte load from an int32 slot, one
        // 32-bit word from a byte slot) when the row stride keeps rows aligned
        std::map<std::pair<int, int>, std::vector<std::pair<int, std::string>>> groups;
        for (const auto& kv : loads)
            groups[{std::get<0>(kv.first), std::get<1>(kv.first)}].push_back(
                {std::get<2>(kv.first), kv.second});
        for (const auto& g : groups) {
            const int s = g.first.first, r = g.first.second, w = slot[s].w, base = r * w;
            if (CB == 1 || w % 4 != 0) {
                for (const auto& dn : g.second)
                    o << "      const int " << dn.second << " = " << slot_name(s) << "[qb" << s
                      << plus(base + dn.first) << "];\n";
                continue;
            }
            // qb's constant part (rb and c are multiples of 4 here, and so is w)
            int c0;
            if (s < d.n_buf) {
                const int dh = d.buf[s].halo - h;
                c0 = dh * w + dh + slot_x(s);
            } else {
                const int k = s - d.n_buf, dh = d.buf[d.st[k].out].halo - h;
                c0 = (dh + d.st[k].ry) * w + dh;
            }
            int lo = g.second.front().first;
            for (const auto& dn : g.second) lo = std::min(lo, dn.first);
            const int a = ((c0 + lo) & ~3) - c0;  // first chunk, from qb + base
            std::map<int, std::string> chunk;
            for (const auto& dn : g.second) {
                const int k = (dn.first - a) >> 2, comp = (dn.first - a) & 3;
                std::string& L = chunk[k];
                if (L.empty()) {
                    L = "L" + std::to_string(s) + "_" + enc(r) + "_" + std::to_string(k);
                    if (byte_slot(s))
                        o << "      const unsigned " << L << " = ((const unsigned*)" << slot_name(s)
                          << ")[(qb" << s << plus(base + a + 4 * k) << ") >> 2];\n";
                    else
                        o << "      const int4 " << L << " = *(const int4*)&" << slot_name(s)
                          << "[qb" << s << plus(base + a + 4 * k) << "];\n";
                }
                if (byte_slot(s))
                    o << "      const int " << dn.second << " = (int)((" << L << " >> " << 8 * comp
                      << ") & 0xFFu);\n";
                else
                    o << "      const int " << dn.second << " = " << L << "." << "xyzw"[comp]
                      << ";\n";
            }
        }
        o << rows << "    }\n  }\n";
        if (outputs) {
            for (size_t j = 0; j < globals.size(); ++j) {
                const int k = globals[j];
                const std::string g = "g" + std::to_string(k), res = "p.res[" + std::to_string(j) + "]";
                if (d.st[k].op == OP_MEANSTD)
                    o << "  hvx_ms_commit(" << res << ", " << g << "_s1, " << g << "_s2, " << g
                      << "_n);\n";
                else if (d.st[k].op == OP_MINMAX)
                    o << "  hvx_mm_commit_warp(" << res << ", " << g << "_mm);\n";
                else
                    o << "  __syncthreads();\n  for (int i = threadIdx.x; i < " << d.st[k].i0
                      << "; i += " << kThreads << ")\n    if (" << g << "_bins[i]) atomicAdd((unsigned*)"
                      << res << " + i, " << g << "_bins[i]);\n";
            }
            return;
        }
        // cells outside the image, the way the local consumers read them
        o << "  if (CHECK) {\n    __syncthreads();\n";
        for (int b : p.targets) {
            o << "    {\n";
            open_cells(bh(b), bw(b), h, h, false);
            o << "      if (x >= 0 && x < p.W && y >= 0 && y < p.H) continue;\n"
              << "      B" << b << "[r * " << slot_w(b) << " + c + " << slot_x(b) << "] = "
              << (byte_slot(b) ? "(unsigned char)" : "")
              << fill_expr(b, "B" + std::to_string(b) + "[(min(max(y, 0), p.H - 1) - y0 + " +
                                  std::to_string(h) + ") * " + std::to_string(slot_w(b)) +
                                  " + min(max(x, 0), p.W - 1) - x0 + " +
                                  std::to_string(h + slot_x(b)) + "]")
              << ";\n";
            close_cells();
            o << "    }\n";
        }
        o << "  }\n  __syncthreads();\n";
    }

    // Second launch bound: resident CTAs per SM the compiler must fit
    // registers for.  Measured on the Section 6 applications: groups of one
    // or two ops run fastest at 8 (Laplacian 584 -> 681, SobelX 657 -> 717
    // Gpix/s), larger groups at 6 (EdgFig2 247 -> 271, Unsharp 465 -> 497),
    // corner-response groups without a bound.  HVX_CODEGEN_MINBLOCKS (1..8,
    // 0 for none) in the environment overrides.
    std::string min_blocks() const {
        int v = d.n_stage <= 2 ? 8 : 6;
        for (int k = 0; k < d.n_stage; ++k)
            if (d.st[k].op == OP_TOMASI || d.st[k].op == OP_HARRIS) v = 0;
        if (const char* e = getenv("HVX_CODEGEN_MINBLOCKS")) v = atoi(e);
        return v >= 1 && v <= 8 ? ", " + std::to_string(v) : "";
    }

    bool emit() {
        analyse();
        // MIRROR / REPEAT fills are only possible for external inputs
        for (int b = 0; b < d.n_buf; ++b)
            if ((d.buf[b].fill == FILL_MIRROR || d.buf[b].fill == FILL_REPEAT) && ext_in[b] < 0)
                return false;
        if (!plan() || !choose_tile()) return false;
        // one mbarrier (2 words, kept 16-byte aligned) per load pass with TMA boxes
        load_bar.assign(passes.size(), -1);
        for (size_t i = 0; i < passes.size(); ++i) {
            if (passes[i].kind != LOAD) continue;
            for (int b : passes[i].targets)
                if (tma_slot(b)) load_bar[i] = 0;
            if (load_bar[i] == 0) {
                load_bar[i] = smem_words;
                smem_words += 4;
            }
        }
        o << "// generated kernel: " << d.n_stage << " ops, " << d.n_buf << " images, tile " << tw
          << " x " << th << ", " << passes.size() << " passes, " << smem_words * 4
          << " bytes of shared memory\n"
          << "#include \"point_math.cuh\"\n#include \"reduce_math.cuh\"\n"
          << "#include \"jit_params.h\"\n\n"
          << "__device__ __forceinline__ bool hvx_in(const int* r, int x, int y) {\n"
          << "  return x >= r[0] && x < r[2] && y >= r[1] && y < r[3];\n}\n"
          << "__device__ __forceinline__ long long hvx_min(long long x, long long y) { return x < y "
             "? x : y; }\n"
          << "__device__ __forceinline__ long long hvx_max(long long x, long long y) { return x > y "
             "? x : y; }\n"
          << "__device__ __forceinline__ long long hvx_abs(long long x) { return x < 0 ? -x : x; }\n"
          << "__device__ __forceinline__ int hvx_mirror(int v, int n) {\n"
          << "  const int p = 2 * n;\n  int m = v % p;\n  if (m < 0) m += p;\n"
          << "  return m < n ? m : p - 1 - m;\n}\n"
          << "__device__ __forceinline__ int hvx_repeat(int v, int n) {\n"
          << "  const int m = v % n;\n  return m < 0 ? m + n : m;\n}\n"
          << "template <int F>\n"
          << "__device__ __forceinline__ int hvx_ld(const void* base, unsigned long long pitch, "
             "int x, int y) {\n"
          << "  const unsigned char* row = (const unsigned char*)base + (unsigned long long)y * "
             "pitch;\n"
          << "  if (F == " << HVX_DF_U8 << ") return __ldg(row + x);\n"
          << "  if (F == " << HVX_DF_S16 << ") return __ldg((const short*)row + x);\n"
          << "  if (F == " << HVX_DF_UYVY << ") return __ldg((const unsigned short*)row + x);\n"
          << "  return __ldg((const int*)row + x);\n}\n"
          << "template <int F>\n"
          << "__device__ __forceinline__ void hvx_st(void* base, unsigned long long pitch, int x, "
             "int y, int v) {\n"
          << "  unsigned char* row = (unsigned char*)base + (unsigned long long)y * pitch;\n"
          << "  if (F == " << HVX_DF_U8 << ") row[x] = (unsigned char)v;\n"
          << "  else if (F == " << HVX_DF_S16 << ") ((short*)row)[x] = (short)v;\n"
          << "  else ((int*)row)[x] = v;\n}\n\n"
          << "__device__ __forceinline__ unsigned hvx_smem(const void* q) {\n"
          << "  return (unsigned)__cvta_generic_to_shared(q);\n}\n"
          << "__device__ __forceinline__ void hvx_mbar_init(unsigned long long* bar) {\n"
          << "  asm volatile(\"mbarrier.init.shared::cta.b64 [%0], 1;\" :: \"r\"(hvx_smem(bar)) "
             ": \"memory\");\n"
          << "  asm volatile(\"fence.mbarrier_init.release.cluster;\" ::: \"memory\");\n}\n"
          << "__device__ __forceinline__ void hvx_expect_tx(unsigned long long* bar, unsigned n) {\n"
          << "  asm volatile(\"mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\" :: "
             "\"r\"(hvx_smem(bar)), \"r\"(n) : \"memory\");\n}\n"
          << "__device__ __forceinline__ void hvx_tmap_acquire(const void* m) {\n"
          << "  asm volatile(\"fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\" :: "
             "\"l\"(m) : \"memory\");\n}\n"
          << "// 2-D tiled TMA load; x * 1 byte is a multiple of 16 (the emitter's slots)\n"
          << "__device__ __forceinline__ void hvx_tma_2d(void* dst, const void* map, "
             "unsigned long long* bar, int x, int y) {\n"
          << "  asm volatile(\"cp.async.bulk.tensor.2d.shared::cluster.global.tile."
             "mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\" :: \"r\"(hvx_smem(dst)), "
             "\"l\"((unsigned long long)map), \"r\"(hvx_smem(bar)), \"r\"(x), \"r\"(y) : "
             "\"memory\");\n}\n"
          << "__device__ __forceinline__ bool hvx_mbar_try(unsigned long long* bar) {\n"
          << "  unsigned ok;\n"
          << "  asm volatile(\"{\\n\\t.reg .pred q;\\n\\tmbarrier.try_wait.parity.shared::cta.b64 "
             "q, [%1], 0;\\n\\tselp.u32 %0, 1, 0, q;\\n\\t}\" : \"=r\"(ok) : "
             "\"r\"(hvx_smem(bar)) : \"memory\");\n"
          << "  return ok != 0;\n}\n"
          << "// phase 0 of bar, for at most ~2^31 cycles: on time-out record the error\n"
          << "// and wait once more with the same bound (a late copy must not land\n"
          << "// after the tile moved on)\n"
          << "__device__ __forceinline__ void hvx_mbar_wait(unsigned long long* bar, int* err) {\n"
          << "  const long long c0 = clock64();\n"
          << "  while (!hvx_mbar_try(bar)) {\n"
          << "    if (clock64() - c0 > (1ll << 31)) {\n"
          << "      if (err) atomicCAS(err, 0, 1);\n"
          << "      const long long c1 = clock64();\n"
          << "      while (!hvx_mbar_try(bar) && clock64() - c1 < (1ll << 31)) {}\n"
          << "      return;\n    }\n  }\n}\n\n"
          << "template <bool CHECK, bool GMAP>\n"
          << "__device__ __forceinline__ void hvx_tile(const HvxJitParams& p, int* smem, int x0, "
             "int y0) {\n"
          << "  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;\n";
        // the body is written first: every launch parameter it reads per cell
        // is then read once into a register (the batched entry point's
        // parameters live in global memory)
        const std::string head = o.str();
        o.str("");
        o.clear();
        bool hist = false;
        for (int k : globals)
            if (d.st[k].op == OP_HIST) {
                o << "  __shared__ unsigned g" << k << "_bins[" << d.st[k].i0 << "];\n"
                  << "  for (int i = threadIdx.x; i < " << d.st[k].i0 << "; i += " << kThreads
                  << ") g" << k << "_bins[i] = 0;\n";
                hist = true;
            }
        if (hist) o << "  __syncthreads();\n";
        for (int s = 0; s < (int)slot.size(); ++s)
            if (slot[s].w > 0)
                o << (byte_slot(s) ? "  unsigned char* const " : "  int* const ") << slot_name(s)
                  << (byte_slot(s) ? " = (unsigned char*)(smem + " : " = (smem + ") << slot[s].off
                  << ");  // "
                  << slot[s].w << " x " << slot[s].h << ", passes " << slot[s].def << ".."
                  << slot[s].last << "\n";
        for (size_t pi = 0; pi < passes.size(); ++pi) {
            const Pass& p = passes[pi];
            switch (p.kind) {
                case LOAD: {
                    std::vector<int> T;
                    for (int b : p.targets)
                        if (tma_slot(b)) T.push_back(b);
                    if (!T.empty()) emit_tma_load(T, load_bar[pi]);
                    for (int b : p.targets) emit_load(b);
                    o << "  __syncthreads();\n";
                    break;
                }
                case ROW:
                    for (int k : p.targets) emit_row(k);
                    o << "  __syncthreads();\n";
                    break;
                case CELLS:
                case OUT: emit_cells(p); break;
            }
        }
        std::string body = o.str();
        std::string regs = "  const int pW = p.W, pH = p.H;\n";
        auto swap_all = [&](const std::string& from, const std::string& to) {
            for (size_t at = body.find(from); at != std::string::npos;
                 at = body.find(from, at + to.size()))
                body.replace(at, from.size(), to);
        };
        for (int e = 0; e < d.n_in; ++e) {
            const std::string E = std::to_string(e);
            regs += "  const void* const in" + E + " = p.in[" + E +
                    "];\n  const unsigned long long ip" + E + " = p.in_pitch[" + E + "];\n";
            swap_all("p.in[" + E + "], p.in_pitch[" + E + "]", "in" + E + ", ip" + E);
        }
        for (int e = 0; e < d.n_out; ++e) {
            const std::string E = std::to_string(e);
            regs += "  void* const out" + E + " = p.out[" + E +
                    "];\n  const unsigned long long op" + E + " = p.out_pitch[" + E + "];\n";
            swap_all("p.out[" + E + "], p.out_pitch[" + E + "]", "out" + E + ", op" + E);
        }
        swap_all("p.W", "pW");
        swap_all("p.H", "pH");
        o.str("");
        o.clear();
        o << head << regs << body;
        o << "}\n\n"
          << "extern \"C\" __global__ void __launch_bounds__(" << kThreads << min_blocks()
          << ") hvx_generated(const __grid_constant__ HvxJitParams p) {\n"
          << "  // a programmatic dependent launch: no global-memory access before the\n"
          << "  // previous grid on the stream has completed\n"
          << "  asm volatile(\"griddepcontrol.launch_dependents;\");\n"
          << "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
          << "  extern __shared__ __align__(16) int smem[];\n"
          << "  const int tx = blockIdx.x, ty = blockIdx.y;\n"
          << "  if (tx >= p.ix0 && tx <= p.ix1 && ty >= p.iy0 && ty <= p.iy1)\n"
          << "    hvx_tile<false, false>(p, smem, tx * " << tw << ", ty * " << th << ");\n"
          << "  else\n"
          << "    hvx_tile<true, false>(p, smem, tx * " << tw << ", ty * " << th << ");\n"
          << "}\n\n"
          << "// n images in one launch: block t is tile t - tile_start[i] of the last\n"
          << "// image i with tile_start[i] <= t\n"
          << "extern \"C\" __global__ void __launch_bounds__(" << kThreads << min_blocks()
          << ") hvx_generated_batch(const HvxJitParams* __restrict__ ps, const int* __restrict__ "
             "tile_start, int n) {\n"
          << "  extern __shared__ __align__(16) int smem[];\n"
          << "  const int t = blockIdx.x;\n"
          << "  int lo = 0, hi = n - 1;\n"
          << "  while (lo < hi) {\n"
          << "    const int mid = (lo + hi + 1) >> 1;\n"
          << "    if (__ldg(tile_start + mid) <= t) lo = mid; else hi = mid - 1;\n"
          << "  }\n"
          << "  const HvxJitParams& p = ps[lo];\n"
          << "  const int local = t - __ldg(tile_start + lo), gx = (p.W + " << tw - 1 << ") / "
          << tw << ";\n"
          << "  const int ty = local / gx, tx = local - ty * gx;\n"
          << "  if (tx >= p.ix0 && tx <= p.ix1 && ty >= p.iy0 && ty <= p.iy1)\n"
          << "    hvx_tile<false, true>(p, smem, tx * " << tw << ", ty * " << th << ");\n"
          << "  else\n"
          << "    hvx_tile<true, true>(p, smem, tx * " << tw << ", ty * " << th << ");\n"
          << "}\n";
        return true;
    }
};

// ---------------------------------------------------------------------------
// Compilation and the kernel cache

std::mutex g_mu;

std::unordered_map<std::string, std::unique_ptr<JitKernel>>& cache() {
    static auto* c = new std::unordered_map<std::string, std::unique_ptr<JitKernel>>();
    return *c;
}

bool compile(JitKernel& k) {
    NvtxRange nvtx("hvx codegen compile");
    Nvrtc& n = nvrtc();
    if (!n.ok) {
        k.log = n.why;
        return false;
    }
    const char* names[] = {"point_math.cuh", "phase_table.h", "jit_params.h", "reduce_math.cuh"};
    const char* texts[] = {kJitPointMath, kJitPhaseTable, kJitParams, kJitReduceMath};
    void* prog = nullptr;
    if (n.create(&prog, k.source.c_str(), "hvx_generated.cu", 4, texts, names) != 0) {
        k.log = "nvrtcCreateProgram failed";
        return false;
    }
    // no fast-math flags: the exact arithmetic relies on IEEE division and sqrt
    const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--device-int128",
                          "-default-device"};
    const int r = n.compile(prog, 4, opts);
    size_t ls = 0;
    if (n.log_size(prog, &ls) == 0 && ls > 1) {
        k.log.assign(ls, '\0');
        n.log(prog, &k.log[0]);
        k.log.resize(ls - 1);
    }
    if (r == 0) {
        size_t cs = 0;
        if (n.cubin_size(prog, &cs) == 0 && cs > 0) {
            k.cubin.assign(cs, 0);
            k.compiled = n.cubin(prog, k.cubin.data()) == 0;
        }
    }
    n.destroy(&prog);
    return k.compiled;
}

bool load(JitKernel& k, int device, std::string* why) {
    Driver& dr = driver();
    if (!dr.ok) {
        *why = "driver entry points unavailable";
        return false;
    }
    if (dr.load(&k.mod, k.cubin.data()) != CUDA_SUCCESS ||
        dr.get(&k.fn, k.mod, "hvx_generated") != CUDA_SUCCESS ||
        dr.get(&k.fn_batch, k.mod, "hvx_generated_batch") != CUDA_SUCCESS) {
        *why = "cuModuleLoadData / cuModuleGetFunction failed";
        return false;
    }
    if (k.smem_bytes > 48 * 1024 &&
        (dr.attr(k.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, k.smem_bytes) !=
             CUDA_SUCCESS ||
         dr.attr(k.fn_batch, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, k.smem_bytes) !=
             CUDA_SUCCESS)) {
        *why = "cuFuncSetAttribute failed";
        return false;
    }
    k.device = device;
    return true;
}

int ceil_div(int a, int b) { return a >= 0 ? (a + b - 1) / b : -((-a) / b); }
int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

}  // namespace

bool jit_available() { return nvrtc().ok; }

bool jit_prepare(const GenericDesc& d, const std::vector<std::string>& user_code, bool load_module,
                 int device, JitLaunch* out, std::string* why) {
    Emitter em(d, user_code);
    if (!em.emit()) {
        *why = "group shape not handled by the code generator";
        return false;
    }
    const std::string src = em.o.str();
    JitKernel* k = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        std::unique_ptr<JitKernel>& slot =
            cache()[(load_module ? std::to_string(device) : std::string("-")) + "\n" + src];
        if (!slot) {
            slot.reset(new JitKernel);
            slot->source = src;
            slot->tw = em.tw;
            slot->th = em.th;
            slot->smem_bytes = em.smem_words * 4;
            compile(*slot);
        }
        if (!slot->compiled) {
            *why = "NVRTC: " + slot->log;
            return false;
        }
        if (load_module && slot->device != device && !load(*slot, device, why)) return false;
        k = slot.get();
    }
    JitLaunch& j = *out;
    j.k = k;
    std::memset(&j.p, 0, sizeof(j.p));
    HvxJitParams& p = j.p;
    p.W = d.W;
    p.H = d.H;
    for (int b = 0; b < d.n_buf; ++b)
        for (int i = 0; i < 4; ++i) p.valid[b][i] = d.buf[b].valid[i];
    for (int e = 0; e < d.n_in; ++e) {
        p.in[e] = d.in[e].ptr;
        p.in_pitch[e] = d.in[e].pitch;
    }
    for (int e = 0; e < d.n_out; ++e) {
        p.out[e] = d.out[e].ptr;
        p.out_pitch[e] = d.out[e].pitch;
    }
    int nres = 0;
    for (int k = 0; k < d.n_stage; ++k)
        if (op_is_global(d.st[k].op)) {
            if (nres >= HVX_JIT_MAX_RES) return false;
            p.res[nres++] = d.st[k].res;
        }
    // interior tiles: every image's cells of the tile grown by its halo lie in
    // its valid region (external inputs: in the image; they are read as stored)
    const int tw = k->tw, th = k->th;
    j.gx = (unsigned)((d.W + tw - 1) / tw);
    j.gy = (unsigned)((d.H + th - 1) / th);
    int ix0 = 0, iy0 = 0, ix1 = (int)j.gx - 1, iy1 = (int)j.gy - 1;
    std::vector<bool> is_in(d.n_buf, false);
    for (int e = 0; e < d.n_in; ++e) is_in[d.in[e].buf] = true;
    for (int b = 0; b < d.n_buf; ++b) {
        const int h = d.buf[b].halo;
        int r[4] = {0, 0, (int)d.W, (int)d.H};
        if (!is_in[b])
            for (int i = 0; i < 4; ++i) r[i] = d.buf[b].valid[i];
        ix0 = std::max(ix0, ceil_div(r[0] + h, tw));
        iy0 = std::max(iy0, ceil_div(r[1] + h, th));
        ix1 = std::min(ix1, floor_div(r[2] - h - tw, tw));
        iy1 = std::min(iy1, floor_div(r[3] - h - th, th));
    }
    p.ix0 = ix0;
    p.ix1 = ix1;
    p.iy0 = iy0;
    p.iy1 = iy1;
    // tensor maps of the TMA-staged inputs (box = the input's slot)
    static_assert(sizeof(HvxTensorMap) == sizeof(CUtensorMap), "tensor map blob");
    if (load_module)
        for (const auto& bx : em.tma_boxes()) {
            const GenExt& in = d.in[bx[0]];
            if (encode_u8_map_raw(reinterpret_cast<CUtensorMap*>(&p.tmap[bx[0]]), in.ptr, in.pitch,
                                  (uint32_t)d.W, (uint32_t)d.H, (uint32_t)bx[1],
                                  (uint32_t)bx[2]) != HVX_SUCCESS) {
                *why = "tensor map of a staged input";
                return false;
            }
        }
    return true;
}

cudaError_t jit_launch(const JitLaunch& j, cudaStream_t s) {
    void* args[] = {const_cast<HvxJitParams*>(&j.p)};
    const Driver& dr = driver();
    CUresult r;
    if (dr.launch_ex) {
        // programmatic stream serialisation: the launch may begin while the
        // previous kernel on the stream finishes (the kernel waits for it)
        CUlaunchAttribute attr = {};
        attr.id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
        attr.value.programmaticStreamSerializationAllowed = 1;
        CUlaunchConfig cfg = {};
        cfg.gridDimX = j.gx;
        cfg.gridDimY = j.gy;
        cfg.gridDimZ = 1;
        cfg.blockDimX = kThreads;
        cfg.blockDimY = 1;
        cfg.blockDimZ = 1;
        cfg.sharedMemBytes = (unsigned)j.k->smem_bytes;
        cfg.hStream = (CUstream)s;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        r = dr.launch_ex(&cfg, j.k->fn, args, nullptr);
    } else {
        r = dr.launch(j.k->fn, j.gx, j.gy, 1, kThreads, 1, 1, (unsigned)j.k->smem_bytes,
                      (CUstream)s, args, nullptr);
    }
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t jit_launch_batch(const JitKernel* k, const HvxJitParams* params, const int* tile_start,
                             int n, int total_tiles, cudaStream_t s) {
    void* args[] = {&params, &tile_start, &n};
    const CUresult r = driver().launch(k->fn_batch, (unsigned)total_tiles, 1, 1, kThreads, 1, 1,
                                       (unsigned)k->smem_bytes, (CUstream)s, args, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

void jit_tile(const JitKernel* k, int* tw, int* th) {
    *tw = k->tw;
    *th = k->th;
}

const std::string& jit_source(const JitLaunch& j) { return j.k->source; }

}  // namespace hvx
