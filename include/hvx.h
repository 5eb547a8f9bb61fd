/*
 * hvx.h -- C ABI of the GB300 image-graph library (OpenVX-style graphs of
 * point and local operators with graph-level kernel fusion).
 *
 * The calls follow the paper's statement of the problem (HipaccVX, Section
 * 3.1 and Listing 1): create a context, images and virtual images, add CV
 * function nodes to a graph, verify the graph, process it; release the
 * context to free everything it owns.  Custom point / local nodes stand in
 * for the paper's user-defined kernels (Section 5.1, Listing 4).
 *
 * Names carry an `hvx` prefix so that they cannot collide with a real OpenVX
 * implementation linked into the same process.
 *
 * General conventions
 *  - Every call returns an hvx_status (0 = HVX_SUCCESS, negative = error) or,
 *    for node constructors, an hvx_node that is NULL on failure; the reason is
 *    then available from hvxGetGraphStatus().  No C++ exception crosses this
 *    boundary.
 *  - Out-parameters are written only on success.
 *  - Images are 2-D, row-major, with a row pitch in bytes that is a multiple of
 *    16.  Pixel formats: U8 (uint8), S16 (int16), S32 (int32), F32 (binary32),
 *    UYVY (2 bytes per pixel, macro-pixels U0 Y0 V0 Y1; width must be even).
 *  - Device pointers are CUDA device addresses on the current device; a
 *    `stream` argument is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).
 *  - A context, and every graph and image it owns, is used by one host thread
 *    at a time, with two exceptions: hvxServerSubmit / hvxServerWait /
 *    hvxServerStats are thread-safe, and several threads may issue
 *    hvxProcessGraphBatch / hvxScheduleGraphBatchHost on one context (on
 *    disjoint graphs; the calls take turns on the context's batch cache and
 *    copy pipeline).  Calls that verify, launch or batch make the context's
 *    device current in the calling thread (cudaSetDevice), which may be a
 *    thread that has made no CUDA call yet.
 *  - Any change to a verified graph (new node, border or rounding change)
 *    marks it unverified; hvxProcessGraph then returns HVX_ERROR_NOT_VERIFIED
 *    until hvxVerifyGraph succeeds again.
 */
#ifndef HVX_H
#define HVX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hvx_status;

#define HVX_SUCCESS 0
#define HVX_ERROR_INVALID_REFERENCE (-1)  /* NULL or released handle, wrong context */
#define HVX_ERROR_INVALID_PARAMETERS (-2) /* bad size, value or missing argument */
#define HVX_ERROR_INVALID_FORMAT (-3)     /* pixel format not accepted by a node */
#define HVX_ERROR_INVALID_GRAPH (-4)      /* cycle, two writers, unwritten virtual */
#define HVX_ERROR_NOT_VERIFIED (-5)       /* graph changed since hvxVerifyGraph */
#define HVX_ERROR_NO_MEMORY (-6)          /* device or host allocation failed */
#define HVX_ERROR_OVER_BUDGET (-7)        /* request larger than a memory budget */
#define HVX_ERROR_TIMEOUT (-8)            /* a bounded wait ran out */
#define HVX_ERROR_DEVICE (-9)             /* a CUDA call failed */
#define HVX_ERROR_NOT_SUPPORTED (-10)     /* valid request this build cannot run */

/* Pixel formats.  HVX_DF_VIRT is accepted only by hvxCreateVirtualImage and
 * means "resolved by hvxVerifyGraph" (Section 3.1: verification resolves the
 * types of virtual data objects). */
#define HVX_DF_VIRT 0
#define HVX_DF_U8 1
#define HVX_DF_S16 2
#define HVX_DF_S32 3
#define HVX_DF_F32 4
#define HVX_DF_UYVY 5

/* Border modes of local operators.  REPLICATE clamps coordinates to the image
 * (Hipacc's CLAMP boundary condition, Section 3.2); CONSTANT reads a constant
 * outside the image; UNDEFINED computes only pixels whose whole window lies in
 * the input's valid region, so the valid region shrinks by the window radius
 * and pixels outside it are written as 0.  MIRROR and REPEAT are Hipacc's
 * other boundary conditions (Section 3.2 names them; the paper does not define
 * them): MIRROR reflects coordinates about the image edge with the edge pixel
 * repeated (... c b a | a b c ...), as often as needed; REPEAT continues the
 * image periodically.  Both read arbitrary pixels of their input, so a local
 * node under them reads its input from memory: the planner does not fuse it
 * with the node that produces that input. */
#define HVX_BORDER_UNDEFINED 0
#define HVX_BORDER_REPLICATE 1
#define HVX_BORDER_CONSTANT 2
#define HVX_BORDER_MIRROR 3
#define HVX_BORDER_REPEAT 4

/* Rounding of the divisions in Gaussian3x3 (by 16) and Box3x3 (by 9). */
#define HVX_ROUND_TO_ZERO 0
#define HVX_ROUND_TO_NEAREST 1 /* round half up */
#define HVX_ROUND_TO_NEAREST_EVEN 2 /* Multiply: ties to even */

#define HVX_THRESHOLD_BINARY 0 /* out = in > value ? true : false            */
#define HVX_THRESHOLD_RANGE 1  /* out = (in > upper || in < lower) ? f : t   */

#define HVX_POLICY_WRAP 0
#define HVX_POLICY_SATURATE 1

#define HVX_CHANNEL_Y 0
#define HVX_CHANNEL_U 1
#define HVX_CHANNEL_V 2

/* hvxCopyImage usage */
#define HVX_READ 1  /* device image -> host buffer */
#define HVX_WRITE 2 /* host buffer -> device image */

/* Custom point operators (hvxPointNode). */
#define HVX_POINT_MUL 1             /* S16 a, S16 b -> S32 a*b (exact)        */
#define HVX_POINT_HARRIS_RESPONSE 2 /* S32 Sxx, Syy, Sxy -> F32 R; params kn, kd */
#define HVX_POINT_TOMASI_RESPONSE 3 /* S32 Sxx, Syy, Sxy -> F32 smaller eigenvalue */

/* Custom local operators (hvxLocalNode). */
#define HVX_LOCAL_SUM 1 /* S32 -> S32: unweighted kw x kh window sum (exact) */

/* hvxQueryGraph attributes */
#define HVX_GRAPH_NUM_NODES 1       /* int32: nodes added                       */
#define HVX_GRAPH_NUM_OPS 2         /* int32: point/local ops after lowering    */
#define HVX_GRAPH_NUM_ALIVE_OPS 3   /* int32: ops kept by dead-code elimination */
#define HVX_GRAPH_NUM_LAUNCHES 4    /* int32: kernel launches per process       */
#define HVX_GRAPH_INTERMEDIATE_BYTES 5 /* uint64: device bytes of materialised
                                          virtual images                      */
#define HVX_GRAPH_EXTERNAL_BYTES 6  /* uint64: bytes of non-virtual images read
                                       plus written per process (algorithmic)  */
#define HVX_GRAPH_FUSION 7          /* int32: 1 if fusion is enabled            */
#define HVX_GRAPH_KERNEL_KINDS 8    /* char[size]: comma-separated kernel names
                                       of the verified plan, in launch order   */
#define HVX_GRAPH_GENERATED_KERNELS 9 /* int32: launches that run a kernel generated
                                         for the graph (hvxSetGraphCodegen)     */

/* Code generation modes (hvxSetGraphCodegen). */
#define HVX_CODEGEN_OFF 0     /* staged-tile groups run the library's interpreter kernel */
#define HVX_CODEGEN_AUTO 1    /* default: generate and compile a kernel per staged-tile
                                 group when a device is present; if NVRTC is missing or
                                 a group's shape is not handled, that group runs the
                                 interpreter kernel (same results)                      */
#define HVX_CODEGEN_REQUIRE 2 /* generate every staged-tile group's kernel, also in a
                                 plan-only context (compile only); verification fails
                                 with HVX_ERROR_NOT_SUPPORTED where that is impossible   */
#define HVX_CODEGEN_ONLY 3    /* as REQUIRE, and the fused groups that hand-written
                                 kernels cover (edge, Gaussian3x3, Harris / Shi-Tomasi
                                 corners) become staged-tile groups with generated
                                 kernels too (to compare the two; same results)         */

/* hvxQueryNode attributes */
#define HVX_NODE_LIVE_OUTPUTS 1 /* uint32 bitmask: output i computed if bit i set */
#define HVX_NODE_GROUP 2        /* int32: fused group index of the node's first
                                   live op, -1 if the whole node is dead      */

typedef struct hvx_context_s* hvx_context;
typedef struct hvx_graph_s* hvx_graph;
typedef struct hvx_image_s* hvx_image;
typedef struct hvx_node_s* hvx_node;
typedef struct hvx_server_s* hvx_server;

/* Half-open rectangle: pixels x in [start_x, end_x), y in [start_y, end_y). */
typedef struct {
    int32_t start_x, start_y, end_x, end_y;
} hvx_rect;

/* ------------------------------------------------------------------------ */
/* Status                                                                     */

/* Static string naming a status code; never NULL. */
const char* hvxStatusString(hvx_status status);

/* ------------------------------------------------------------------------ */
/* Context (Section 3.1: every object lives in a context, which frees its     */
/* memory on release).                                                        */

/* Create a context on the current CUDA device.  *out receives the handle. */
hvx_status hvxCreateContext(hvx_context* out);

/* Context flags for hvxCreateContextEx. */
#define HVX_CONTEXT_PLAN_ONLY 1 /* no device: images get no memory, graphs can be
                                   built, verified and queried (DCE, fusion plan,
                                   valid regions) but not processed or copied
                                   (HVX_ERROR_NOT_SUPPORTED) */

/* hvxCreateContext with flags (0 = hvxCreateContext). */
hvx_status hvxCreateContextEx(int32_t flags, hvx_context* out);

/* Release the context and every graph, node, image and server it owns, and
 * free their device memory.  Sets *ctx to NULL.  Pending work is waited for
 * first. */
hvx_status hvxReleaseContext(hvx_context* ctx);

/* Self-test of the device-side failure path: launches a kernel that waits on
 * a barrier nothing ever completes.  Every wait in this library's kernels is
 * bounded; this one must give up after a few milliseconds, record the
 * failure in the context's error word and exit.  Returns HVX_ERROR_TIMEOUT
 * when that happened (the expected result); the context remains usable. */
hvx_status hvxSelfTestBoundedWait(hvx_context ctx);

/* Self-test of the fused edge kernel's point arithmetic (Table 2 Phase and
 * Magnitude -> binary Threshold; the kernel's own device functions and Phase
 * table, not a copy): for every integer gradient pair (gx, gy) in
 * [-gmax, gmax]^2, element i = (gy + gmax) * (2 gmax + 1) + (gx + gmax) of
 * phase_out receives the Phase byte round(atan2(gy, gx) * 128 / pi) mod 256
 * and mask_out 255 when gx^2 + gy^2 > s_thr, else 0.  Both are HOST buffers
 * of (2 gmax + 1)^2 bytes, written on success.  0 <= gmax <= 4096 (Sobel3x3
 * on U8 input reaches 1020), else HVX_ERROR_INVALID_PARAMETERS; allocates
 * 2 (2 gmax + 1)^2 bytes of device memory for the call (HVX_ERROR_NO_MEMORY)
 * and synchronises the device. */
hvx_status hvxSelfTestEdgePoint(hvx_context ctx, int32_t gmax, int32_t s_thr, uint8_t* phase_out,
                                uint8_t* mask_out);

/* Host-side fault injection for failure-path tests (process-wide, off by
 * default; no device fault is ever made).  kind HVX_FAULT_DEVICE_ALLOC makes
 * the n-th device allocation the library attempts from now on (images,
 * materialised intermediates, result blocks; n >= 1) fail as if cudaMalloc
 * had, so that call returns HVX_ERROR_NO_MEMORY; HVX_FAULT_LAUNCH makes the
 * n-th graph launch from now on (hvxProcessGraph, hvxScheduleGraph, a server
 * dispatch) fail with HVX_ERROR_DEVICE before anything is enqueued.  Each armed fault fires once.  HVX_FAULT_NONE (n ignored) disarms
 * both.  Returns HVX_ERROR_INVALID_PARAMETERS for another kind or n < 1. */
#define HVX_FAULT_NONE 0
#define HVX_FAULT_DEVICE_ALLOC 1
#define HVX_FAULT_LAUNCH 2
hvx_status hvxTestInjectFault(int32_t kind, int64_t n);

/* Cap the device bytes the context may allocate for images and plans
 * (0 = unlimited).  Allocations beyond it fail with HVX_ERROR_OVER_BUDGET. */
hvx_status hvxSetContextMemoryBudget(hvx_context ctx, uint64_t bytes);

/* Device bytes currently allocated by the context. */
hvx_status hvxGetContextMemoryUsage(hvx_context ctx, uint64_t* bytes);

/* ------------------------------------------------------------------------ */
/* Images (Section 3.1: non-virtual images are host accessible; virtual      */
/* images are intermediates that cannot be read or written by the user).    */

/* Allocate a w x h image of format fmt (not VIRT) in device memory owned by
 * the context; the row pitch is rounded up to a multiple of 128 bytes.
 * 1 <= width, height <= 32768. */
hvx_status hvxCreateImage(hvx_context ctx, uint32_t width, uint32_t height, int32_t fmt,
                          hvx_image* out);

/* Wrap caller-owned device memory (for example a torch tensor's storage) as a
 * non-virtual image.  dev_ptr must be 16-byte aligned and pitch_bytes a
 * multiple of 16 and at least width * bytes-per-pixel.  The caller keeps
 * ownership and must keep the memory alive while any graph uses the image. */
hvx_status hvxCreateImageFromHandle(hvx_context ctx, uint32_t width, uint32_t height,
                                    int32_t fmt, void* dev_ptr, uint64_t pitch_bytes,
                                    hvx_image* out);

/* Point an image created by hvxCreateImageFromHandle at other caller-owned
 * memory of the same size and format (for example the next frame).  The
 * graphs using it stay verified. */
hvx_status hvxSwapImageHandle(hvx_image img, void* dev_ptr, uint64_t pitch_bytes);

/* Declare a virtual image owned by graph g.  width/height 0 and fmt
 * HVX_DF_VIRT leave the size / format to be inferred at verification. */
hvx_status hvxCreateVirtualImage(hvx_graph g, uint32_t width, uint32_t height, int32_t fmt,
                                 hvx_image* out);

/* Drop the caller's reference.  The image is destroyed once no node uses it
 * and its context or graph is released.  Sets *img to NULL. */
hvx_status hvxReleaseImage(hvx_image* img);

/* Synchronous copy between a non-virtual image and a host buffer with row
 * pitch host_pitch bytes.  usage HVX_READ copies device -> host, HVX_WRITE
 * host -> device.  Virtual images are rejected with
 * HVX_ERROR_INVALID_REFERENCE. */
hvx_status hvxCopyImage(hvx_image img, void* host_ptr, uint64_t host_pitch, int32_t usage);

/* Device address and row pitch (bytes) of a non-virtual image. */
hvx_status hvxGetImageDevicePtr(hvx_image img, void** dev_ptr, uint64_t* pitch_bytes);

/* Width, height and format (VIRT until a virtual image is resolved). */
hvx_status hvxQueryImage(hvx_image img, uint32_t* width, uint32_t* height, int32_t* fmt);

/* Valid region after the last successful verification: the whole image for
 * inputs; shrunk by the window radius at each local node under
 * HVX_BORDER_UNDEFINED. */
hvx_status hvxGetValidRegion(hvx_image img, hvx_rect* rect);

/* ------------------------------------------------------------------------ */
/* Graphs (Section 3.1: non-eager execution -- verify once, then process a   */
/* verified graph repeatedly).                                               */

hvx_status hvxCreateGraph(hvx_context ctx, hvx_graph* out);

/* Release a graph, its nodes and its virtual images.  Sets *g to NULL. */
hvx_status hvxReleaseGraph(hvx_graph* g);

/* Verification (Section 3.1 and Section 5.2): check node parameters
 * (presence, formats, sizes), reject cycles and non-bipartite edges, resolve
 * virtual image sizes and formats, drop dead computations (Algorithm 1),
 * compute valid regions, group ops for fusion, allocate the device memory of
 * every virtual image that crosses a fused-group boundary, and build the
 * launch plan.  Returns HVX_ERROR_INVALID_GRAPH / _FORMAT / _PARAMETERS with
 * the graph left unverified. */
hvx_status hvxVerifyGraph(hvx_graph g);

/* Run a verified graph and wait for it (Listing 1's process call). */
hvx_status hvxProcessGraph(hvx_graph g);

/* Enqueue a verified graph on `stream` and return without waiting.
 * hvxWaitGraph waits for the last scheduled run and reports a device-side
 * error (HVX_ERROR_TIMEOUT if a kernel's bounded wait ran out). */
hvx_status hvxScheduleGraph(hvx_graph g, void* stream);
hvx_status hvxWaitGraph(hvx_graph g);

/* Enable (1, default) or disable (0) kernel fusion.  Disabled, every CV
 * function node runs as its own kernel and every virtual image lives in
 * device memory: the plain one-launch-per-node form.  Marks the graph
 * unverified. */
hvx_status hvxSetGraphFusion(hvx_graph g, int32_t enable);

/* Code generation for the graph's staged-tile groups (Section 5: the fused
 * partitions of the graph become source code specialised to them).  At
 * verification each such group's kernel is emitted as CUDA C++ with every
 * operator, constant, border fill and coefficient compiled in, compiled with
 * NVRTC for sm_103a and loaded; kernels are cached by source text for the life
 * of the process, so graphs of the same shape compile once.  Generated
 * kernels give the same results as the interpreter, cell for cell.  mode is
 * HVX_CODEGEN_*; marks the graph unverified.  HVX_CODEGEN_ROWS=1, 2 or 4 in
 * the environment overrides how many vertically adjacent cells a thread
 * computes per iteration of a generated pass (a tuning knob; results are
 * the same); HVX_CODEGEN_COLS=4 turns on 4-column blocks (vector loads
 * and stores) in the output pass of 128-wide tiles (slower on the
 * applications measured; kept for experiments);
 * HVX_CODEGEN_VERBOSE=1 prints why a group got no generated kernel. */
hvx_status hvxSetGraphCodegen(hvx_graph g, int32_t mode);

/* Source text of the kernel generated for launch `group` of a verified graph
 * (0-based, in launch order).  Writes at most size bytes including the
 * terminating NUL to buf (buf may be NULL with size 0) and returns the full
 * length; -1 if that launch runs no generated kernel or the graph is invalid
 * or unverified. */
int64_t hvxGetGraphKernelSource(hvx_graph g, int32_t group, char* buf, uint64_t size);

/* Last error recorded on the graph (for NULL returns of node constructors). */
hvx_status hvxGetGraphStatus(hvx_graph g);

/* Read a graph attribute (HVX_GRAPH_*) into out (size bytes). */
hvx_status hvxQueryGraph(hvx_graph g, int32_t attribute, void* out, uint64_t size);

/* Process n verified graphs in as few launches as possible on `stream`,
 * without waiting.  Graphs whose plans are one fused edge group (Gaussian3x3
 * -> Sobel3x3 -> Magnitude/Threshold and/or Phase) are run by one persistent
 * kernel over the tiles of all images, replayed from a captured CUDA graph
 * when the same set of graphs is submitted again; other graphs are run one
 * after another.  Image sizes may differ.  Wait with hvxWaitBatch. */
hvx_status hvxProcessGraphBatch(const hvx_graph* graphs, int32_t n, void* stream);
hvx_status hvxWaitBatch(hvx_context ctx, void* stream);

/* The launch that hvxProcessGraphBatch tuned for exactly this sequence of
 * graphs (its first call times candidate tile heights per image-size class
 * and persistent grids, and caches the fastest): for each
 * graph, rows_out[i] = R, the rows per thread of the persistent edge kernel's
 * tiles for that image (its tiles are 128 x 8R pixels; 0 where the batch runs
 * another kernel, which keeps its own tile), and *grid_out = the persistent
 * grid of its first launch (CTAs; 0 for a direct launch; a batch whose
 * size classes got different tile heights runs one launch per class, all
 * replayed from one captured CUDA graph).  rows_out holds n entries.
 * HVX_ERROR_INVALID_PARAMETERS when no batch of these graphs has run since
 * they were last verified. */
hvx_status hvxQueryBatch(const hvx_graph* graphs, int32_t n, int32_t* rows_out, int32_t* grid_out);

/* ------------------------------------------------------------------------ */
/* Nodes.  Standard CV functions (Table 2).  Each returns NULL on failure.    */

/* Gaussian3x3 (local): U8 -> U8, weights [1 2 1; 2 4 2; 1 2 1] / 16. */
hvx_node hvxGaussian3x3Node(hvx_graph g, hvx_image in, hvx_image out);

/* Box3x3 (local): U8 -> U8, 3x3 sum / 9. */
hvx_node hvxBox3x3Node(hvx_graph g, hvx_image in, hvx_image out);

/* Dilate3x3 / Erode3x3 / Median3x3 (local, Table 2): U8 -> U8, the maximum /
 * minimum / median of the nine samples of the 3x3 window (border mode as set
 * on the node). */
hvx_node hvxDilate3x3Node(hvx_graph g, hvx_image in, hvx_image out);
hvx_node hvxErode3x3Node(hvx_graph g, hvx_image in, hvx_image out);
hvx_node hvxMedian3x3Node(hvx_graph g, hvx_image in, hvx_image out);

/* Sobel3x3 (local): U8 -> S16 gx (kernel [-1 0 1; -2 0 2; -1 0 1]) and S16 gy
 * (its transpose).  Either output may be NULL; an output no one reads is
 * removed by dead-computation elimination (Section 5.2.2). */
hvx_node hvxSobel3x3Node(hvx_graph g, hvx_image in, hvx_image gx, hvx_image gy);

/* Magnitude (point): S16 gx, gy -> S16 floor(sqrt(gx^2 + gy^2) + 1/2),
 * saturated to 32767. */
hvx_node hvxMagnitudeNode(hvx_graph g, hvx_image gx, hvx_image gy, hvx_image out);

/* Phase (point): S16 gx, gy -> U8 floor(atan2(gy, gx) * 256 / (2 pi) + 1/2)
 * mod 256, with the angle taken in [0, 2 pi) and atan2(0, 0) = 0. */
hvx_node hvxPhaseNode(hvx_graph g, hvx_image gx, hvx_image gy, hvx_image out);

/* Threshold (point): U8 / S16 / S32 / F32 -> U8.  type HVX_THRESHOLD_BINARY
 * uses value (strict >); HVX_THRESHOLD_RANGE uses lower = value and upper.
 * For integer inputs value and upper must be integers; for F32 they are
 * rounded to binary32 first. */
hvx_node hvxThresholdNode(hvx_graph g, hvx_image in, int32_t type, double value, double upper,
                          int32_t true_value, int32_t false_value, hvx_image out);

/* ChannelExtract (point): UYVY -> U8.  HVX_CHANNEL_Y gives a W x H image,
 * HVX_CHANNEL_U / _V give (W/2) x H. */
hvx_node hvxChannelExtractNode(hvx_graph g, hvx_image in, int32_t channel, hvx_image out);

/* Add / Subtract (point): U8 or S16 inputs -> U8 or S16 output (the output
 * image's format, or S16 if virtual and either input is S16, else U8); the
 * exact result is wrapped or saturated per policy.  AbsDiff: |a - b|,
 * saturated. */
hvx_node hvxAddNode(hvx_graph g, hvx_image a, hvx_image b, int32_t policy, hvx_image out);
hvx_node hvxSubtractNode(hvx_graph g, hvx_image a, hvx_image b, int32_t policy, hvx_image out);
hvx_node hvxAbsDiffNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out);

/* User-defined operators (Section 5.1: user kernels written against the
 * point / local abstractions run on the accelerator like the library's own
 * nodes).  The operator is an integer expression in a small C-like language:
 * integer literals; a, b, c (a point operator's inputs at the pixel) or
 * in(dx, dy) (a local operator's input at literal offsets within its kw x kh
 * window, read under the node's border mode); unary - + ~; binary * + -
 * << >> < > <= >= == != & ^ |; min(x, y), max(x, y), abs(x); parentheses.
 * C precedence, 64-bit two's-complement arithmetic, comparisons 0 or 1; the
 * result is saturated to the output image's format (U8, S16 or S32, which
 * the output must declare).  Inputs are U8, S16 or S32.  Such nodes fuse
 * with their neighbours like library nodes and run only in generated kernels
 * (NVRTC): verification fails with HVX_ERROR_NOT_SUPPORTED when code
 * generation is off or unavailable.  NULL (HVX_ERROR_INVALID_PARAMETERS) for
 * an expression outside the language, an offset outside the window, n_in
 * outside 1..3 or kw, kh not odd in 1..9; HVX_CODEGEN_VERBOSE=1 prints why. */
hvx_node hvxUserPointNode(hvx_graph g, const char* expr, const hvx_image* in, int32_t n_in,
                          hvx_image out);
hvx_node hvxUserLocalNode(hvx_graph g, const char* expr, int32_t kw, int32_t kh, hvx_image in,
                          hvx_image out);

/* Copy (point, Table 2): U8 -> U8 or S16 -> S16, unchanged. */
hvx_node hvxCopyNode(hvx_graph g, hvx_image in, hvx_image out);

/* ConvertDepth (point, Table 2): U8 -> S16 is v << shift; S16 -> U8 is
 * v >> shift (arithmetic: floor division by 2^shift), then wrapped to 8 bits
 * or saturated to 0..255 per policy.  0 <= shift <= 7; NULL
 * (HVX_ERROR_INVALID_PARAMETERS) otherwise. */
hvx_node hvxConvertDepthNode(hvx_graph g, hvx_image in, hvx_image out, int32_t policy,
                             int32_t shift);

/* Multiply (point, Table 2): U8 or S16 inputs -> U8 or S16 output (formats as
 * for Add).  out = a * b * scale, taken exactly for the binary32 scale given
 * (0 <= scale <= 65536), rounded once per rounding (HVX_ROUND_TO_ZERO or
 * HVX_ROUND_TO_NEAREST_EVEN), then wrapped or saturated per policy.  NULL
 * (graph status HVX_ERROR_INVALID_PARAMETERS) for a scale, policy or rounding
 * outside these values. */
hvx_node hvxMultiplyNode(hvx_graph g, hvx_image a, hvx_image b, float scale, int32_t policy,
                         int32_t rounding, hvx_image out);

/* Global operators (Table 2 "reduce" and "histogram"; Section 4: the output
 * depends on the whole image).  Each node owns a result that
 * hvxGetNodeResult copies out after the graph ran; the traversal covers the
 * input's valid region.  Fused after the group that produces their input,
 * they reduce that group's values as they are computed (no image is written
 * for them); otherwise they read their input from memory. */

/* MeanStdDev (U8 or S16): exact sums; mean = sum / count and stddev =
 * sqrt(count * sum_squares - sum^2) / count (population), each rounded to
 * binary32 from the double result of that expression. */
typedef struct hvx_mean_stddev_s {
    float mean, stddev;
    int64_t sum;
    uint64_t sum_squares, count;
} hvx_mean_stddev;
hvx_node hvxMeanStdDevNode(hvx_graph g, hvx_image in);

/* MinMaxLoc (U8 or S16): the minimum and maximum, how many pixels take each,
 * and the first pixel of each in raster order; an empty valid region gives
 * counts 0 and locations -1. */
typedef struct hvx_minmaxloc_s {
    int32_t min, max;
    uint64_t min_count, max_count;
    int32_t min_x, min_y, max_x, max_y;
} hvx_minmaxloc;
hvx_node hvxMinMaxLocNode(hvx_graph g, hvx_image in);

/* Histogram (U8): num_bins (1..256) bins over [offset, offset + range)
 * (offset + range <= 256); value v counts in bin (v - offset) * num_bins /
 * range (integer division); values outside are not counted.  The result is
 * uint32_t[num_bins].  NULL (HVX_ERROR_INVALID_PARAMETERS) for other values. */
hvx_node hvxHistogramNode(hvx_graph g, hvx_image in, int32_t num_bins, int32_t offset,
                          int32_t range);

/* EqualizeHist (U8 -> U8; histogram + point): with c the cumulative 256-bin
 * histogram of the input's valid region, cmin its value at the smallest
 * pixel value present and N the pixel count, v becomes
 * round((c[v] - cmin) * 255 / (N - cmin)), halves up; a constant image is
 * copied.  Runs as its own two launches (the histogram must be complete
 * before any pixel is mapped). */
hvx_node hvxEqualizeHistNode(hvx_graph g, hvx_image in, hvx_image out);

/* One image's host data for hvxScheduleGraphBatchHost: to_device 1 copies
 * host -> image before the launch, 0 copies image -> host after it.  host
 * rows are pitch bytes apart (pitch >= width * bytes per pixel); pinned
 * (page-locked) host memory lets the copies overlap other streams' work. */
typedef struct hvx_host_copy_s {
    hvx_image image;  /* non-virtual image of the graphs' context */
    void* host;
    uint64_t pitch;
    int32_t to_device;
} hvx_host_copy;

/* hvxProcessGraphBatch on host data, asynchronously on `stream`: every
 * to_device copy, then the batch (as few launches as hvxProcessGraphBatch
 * makes), then every device-to-host copy, each a cudaMemcpy2DAsync in the
 * stream's order.  Returns once enqueued; the host buffers must stay valid
 * until the stream reaches them (hvxWaitBatch).  Calls on several streams
 * overlap one batch's copies with another's kernels (transfers over the
 * CPU-GPU link are the bound of host-resident processing). */
hvx_status hvxScheduleGraphBatchHost(const hvx_graph* graphs, int32_t n,
                                     const hvx_host_copy* copies, int32_t n_copies,
                                     void* stream);

/* hvxServerSubmit on host data: the request's to_device copies run on its
 * stream right before its launches and the device-to-host copies right after
 * them, so that completion (hvxServerWait) means the results are in host
 * memory.  The host buffers must stay valid until then. */
hvx_status hvxServerSubmitHost(hvx_server server, hvx_graph g, const hvx_host_copy* copies,
                               int32_t n_copies, uint64_t* ticket);

/* Copy a global operator's result (hvx_mean_stddev, hvx_minmaxloc, or
 * uint32_t[num_bins]) to host memory out (size bytes).  Call after the
 * graph's processing has completed (hvxProcessGraph, or hvxWaitGraph /
 * hvxWaitBatch after scheduling).  HVX_ERROR_NOT_SUPPORTED in a plan-only
 * context; HVX_ERROR_INVALID_PARAMETERS for other nodes or a short buffer. */
hvx_status hvxGetNodeResult(hvx_node node, void* out, uint64_t size);

/* And / Or / Xor (point, Table 2): U8, U8 -> U8 bitwise; Not: U8 -> U8. */
hvx_node hvxAndNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out);
hvx_node hvxOrNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out);
hvx_node hvxXorNode(hvx_graph g, hvx_image a, hvx_image b, hvx_image out);
hvx_node hvxNotNode(hvx_graph g, hvx_image in, hvx_image out);

/* Convolve (local): U8 -> S16 (or U8, see hvxPointNode's notes), integer kw x kh coefficients (row-major,
 * applied without flipping, odd sizes up to 7x7), the sum floor-divided by
 * 2^shift and saturated to S16. */
hvx_node hvxConvolveNode(hvx_graph g, hvx_image in, const int32_t* coeffs, int32_t kw,
                         int32_t kh, int32_t shift, hvx_image out);

/* Custom point node (Section 5.1: user-defined kernels expressed with the
 * point abstraction).  op HVX_POINT_MUL takes 2 S16 inputs; op
 * HVX_POINT_HARRIS_RESPONSE takes S32 Sxx, Syy, Sxy and params = {kn, kd}
 * (integers, k = kn / kd, 0 <= kn <= 1000, 1 <= kd <= 1000) and returns the
 * binary32 value nearest to Sxx*Syy - Sxy^2 - k (Sxx + Syy)^2.  op
 * HVX_POINT_TOMASI_RESPONSE (the Tomasi application of Section 6) takes S32
 * Sxx, Syy, Sxy, no params, and returns the smaller eigenvalue of
 * [Sxx Sxy; Sxy Syy] in binary32, 2 det / (tr + sqrt(tr^2 - 4 det)) from the
 * exact 64-bit det and discriminant (a few binary32 rounding steps: within
 * 1e-6 relative of the exact value).
 *
 * Convolve's output may also be a U8 image (the sum saturated to 0 .. 255);
 * a virtual output is S16 unless created with format U8. */
hvx_node hvxPointNode(hvx_graph g, int32_t op, const hvx_image* ins, int32_t n_in,
                      hvx_image out, const double* params, int32_t n_params);

/* Custom local node (Section 5.1, local abstraction).  op HVX_LOCAL_SUM:
 * S32 -> S32 unweighted sum over an odd kw x kh window (kw, kh <= 9). */
hvx_node hvxLocalNode(hvx_graph g, int32_t op, int32_t kw, int32_t kh, hvx_image in,
                      hvx_image out);

/* Border mode of a local node (default HVX_BORDER_REPLICATE).  constant is
 * used by HVX_BORDER_CONSTANT, in the input's format. */
hvx_status hvxSetNodeBorder(hvx_node node, int32_t mode, int32_t constant);

/* Rounding of Gaussian3x3 / Box3x3 (default HVX_ROUND_TO_ZERO). */
hvx_status hvxSetNodeRounding(hvx_node node, int32_t rounding);

/* Read a node attribute (HVX_NODE_*) of a verified graph. */
hvx_status hvxQueryNode(hvx_node node, int32_t attribute, void* out, uint64_t size);

/* ------------------------------------------------------------------------ */
/* Serving: a request loop that admits verified graphs as they arrive.        */

typedef struct {
    uint64_t submitted;
    uint64_t completed;
    uint64_t failed;
    uint64_t queued;          /* waiting for admission now                   */
    uint64_t in_flight;       /* admitted, not yet complete                  */
    uint64_t max_in_flight;   /* largest number in flight at once            */
    uint64_t bytes_reserved;  /* budget bytes held by admitted requests      */
    uint64_t peak_bytes_reserved;
    double p50_ms;            /* latency (submit -> completion) percentiles  */
    double p99_ms;
    double mean_ms;
    double max_ms;
    double mpix_completed;    /* output megapixels of completed requests     */
    double wait_p99_ms;       /* submit -> admission (queueing) percentile   */
    double wait_max_ms;
} hvx_server_stats;

/* Create a server on ctx.  mem_budget_bytes bounds the device bytes held by
 * admitted requests (each request holds its graph's image and intermediate
 * bytes while in flight); max_in_flight bounds concurrent requests (slots);
 * n_streams device streams carry them so that their work overlaps. */
hvx_status hvxCreateServer(hvx_context ctx, uint64_t mem_budget_bytes, int32_t max_in_flight,
                           int32_t n_streams, hvx_server* out);

/* Submit verified graph g.  The request waits in FIFO order until a slot and
 * budget are free, then runs on the next stream.  A graph may have only one
 * request in flight at a time; a later request on it waits for the earlier
 * one, and requests on other graphs queued behind it are admitted meanwhile
 * (a request that does not fit the budget holds back all behind it).
 * *ticket identifies the request.  Fails with HVX_ERROR_OVER_BUDGET if g
 * alone exceeds the budget. */
hvx_status hvxServerSubmit(hvx_server s, hvx_graph g, uint64_t* ticket);

/* Submit n verified graphs that arrive together: all n requests enter the
 * queue at once, in array order, under one lock, so the dispatcher sees them
 * together and admits as many as slots and budget allow in one pass (their
 * work then overlaps on the server's streams).  tickets[i] identifies the
 * request on graphs[i].  All-or-nothing: on any error (an invalid or
 * unverified graph, one larger than the budget) nothing is queued and
 * tickets is untouched.  n = 0 does nothing. */
hvx_status hvxServerSubmitMany(hvx_server s, const hvx_graph* graphs, int32_t n,
                               uint64_t* tickets);

/* Wait up to timeout_ms (negative = forever) for a request.  On success
 * *result holds the request's own status and *latency_ms its latency; each
 * ticket can be waited for once.  HVX_ERROR_TIMEOUT if it has not finished. */
hvx_status hvxServerWait(hvx_server s, uint64_t ticket, int32_t timeout_ms, hvx_status* result,
                         double* latency_ms);

hvx_status hvxServerStats(hvx_server s, hvx_server_stats* stats);

/* Clear the latency record (counters keep running). */
hvx_status hvxServerResetStats(hvx_server s);

/* Drain outstanding requests and destroy the server.  Sets *s to NULL. */
hvx_status hvxReleaseServer(hvx_server* s);

/* ------------------------------------------------------------------------ */
/* Batched edge graph that allocates nothing.                                 */
/*                                                                            */
/* The paper has no counterpart to this call.  It exists for callers that     */
/* must not allocate device memory: a process whose device memory is fully   */
/* owned by another allocator (a framework's caching pool), a real-time loop  */
/* that cannot afford cudaMalloc's implicit device synchronisation, or code   */
/* running with a fixed memory footprint.  hvxProcessGraphBatch allocates     */
/* (and caches) device memory for per-frame launch tables, and every context  */
/* allocates a device error word; this call keeps all of that in one fixed    */
/* array inside the library instead.                                         */

/* Largest number of frames one hvxEdgeBatchNoAlloc call accepts.  The fixed
 * scratch array sized for it (about 80 KB) is part of the library's device
 * image: every GPU that loads the library holds it until the process exits. */
#define HVX_NOALLOC_MAX_FRAMES 256

/* One caller-owned frame: a U8 input and the U8 phase and / or mask outputs,
 * all device pointers 16-byte aligned, pitches in bytes, multiples of 16 and
 * at least width.  phase or mask may be NULL (not produced), the same way in
 * every frame of one call.  1 <= width, height <= 32768. */
typedef struct {
    const void* in;
    uint64_t in_pitch;
    void* phase;
    uint64_t phase_pitch;
    void* mask;
    uint64_t mask_pitch;
    uint32_t width, height;
} hvx_edge_frame;

/* Run the edge graph Gaussian3x3 -> Sobel3x3 -> Magnitude -> binary Threshold
 * (mask = 255 where round(magnitude) > threshold, else 0) and Phase on n
 * frames with one persistent kernel launch on `stream` -- the result equals
 * hvxProcessGraphBatch on edge graphs with the same border (applied to both
 * local nodes, constant 0) and truncating Gaussian rounding.
 *
 * Allocates nothing: no cudaMalloc / cudaFree or other allocating routine.
 * The launch tables and the device error word live in a fixed array of the
 * library; its address is looked up (cudaGetSymbolAddress) on the first call
 * made on each device, with that device current, so make that first call
 * before any stream capture.  Every call shares the array and rewrites it
 * (clearing the error word), so calls whose GPU work overlapped would race on
 * it; this implementation keeps them apart by holding one process-wide lock
 * from its first write of the array until its work on `stream` has finished
 * (it copies the tables in, launches, reads the error word back and waits
 * for `stream`), so calls from several host threads run one after another.
 * Work the caller puts on `stream` before the call runs before it.  Returns
 * HVX_ERROR_TIMEOUT if a kernel's bounded wait ran out.
 * Returns HVX_ERROR_OVER_BUDGET if n > HVX_NOALLOC_MAX_FRAMES and
 * HVX_ERROR_INVALID_PARAMETERS for a NULL, misaligned or inconsistent frame. */
hvx_status hvxEdgeBatchNoAlloc(const hvx_edge_frame* frames, int32_t n, int32_t border,
                               int32_t threshold, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HVX_H */
