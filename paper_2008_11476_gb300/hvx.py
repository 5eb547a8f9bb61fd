"""Python binding of the C ABI in include/hvx.h (ctypes, same names).

Argument marshalling only: every call goes straight to libhvx.so, and every
step of the image-graph path runs in the library's CUDA kernels.  A call that
returns an error status raises ``HvxError``; out-parameters are returned.
Handles are opaque ``ctypes.c_void_p`` values.

The library is built in-tree on first use (``_build.build()``); if it cannot be
built or loaded, importing any entry point raises — there is no fallback.
"""
from __future__ import annotations

import ctypes
import threading

from . import _build

# status codes
HVX_SUCCESS = 0
HVX_ERROR_INVALID_REFERENCE = -1
HVX_ERROR_INVALID_PARAMETERS = -2
HVX_ERROR_INVALID_FORMAT = -3
HVX_ERROR_INVALID_GRAPH = -4
HVX_ERROR_NOT_VERIFIED = -5
HVX_ERROR_NO_MEMORY = -6
HVX_ERROR_OVER_BUDGET = -7
HVX_ERROR_TIMEOUT = -8
HVX_ERROR_DEVICE = -9
HVX_ERROR_NOT_SUPPORTED = -10

HVX_DF_VIRT, HVX_DF_U8, HVX_DF_S16, HVX_DF_S32, HVX_DF_F32, HVX_DF_UYVY = 0, 1, 2, 3, 4, 5
HVX_BORDER_UNDEFINED, HVX_BORDER_REPLICATE, HVX_BORDER_CONSTANT = 0, 1, 2
HVX_BORDER_MIRROR, HVX_BORDER_REPEAT = 3, 4
HVX_ROUND_TO_ZERO, HVX_ROUND_TO_NEAREST = 0, 1
HVX_ROUND_TO_NEAREST_EVEN = 2
HVX_THRESHOLD_BINARY, HVX_THRESHOLD_RANGE = 0, 1
HVX_POLICY_WRAP, HVX_POLICY_SATURATE = 0, 1
HVX_CHANNEL_Y, HVX_CHANNEL_U, HVX_CHANNEL_V = 0, 1, 2
HVX_READ, HVX_WRITE = 1, 2
HVX_POINT_MUL, HVX_POINT_HARRIS_RESPONSE, HVX_POINT_TOMASI_RESPONSE = 1, 2, 3
HVX_LOCAL_SUM = 1
HVX_GRAPH_NUM_NODES = 1
HVX_GRAPH_NUM_OPS = 2
HVX_GRAPH_NUM_ALIVE_OPS = 3
HVX_GRAPH_NUM_LAUNCHES = 4
HVX_GRAPH_INTERMEDIATE_BYTES = 5
HVX_GRAPH_EXTERNAL_BYTES = 6
HVX_GRAPH_FUSION = 7
HVX_GRAPH_KERNEL_KINDS = 8
HVX_GRAPH_GENERATED_KERNELS = 9
HVX_CODEGEN_OFF, HVX_CODEGEN_AUTO, HVX_CODEGEN_REQUIRE, HVX_CODEGEN_ONLY = 0, 1, 2, 3
HVX_NODE_LIVE_OUTPUTS = 1
HVX_NODE_GROUP = 2

BYTES_PER_PIXEL = {HVX_DF_U8: 1, HVX_DF_S16: 2, HVX_DF_S32: 4, HVX_DF_F32: 4, HVX_DF_UYVY: 2}


class HvxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {hvxStatusString(status)} ({status})")


class hvx_rect(ctypes.Structure):
    _fields_ = [("start_x", ctypes.c_int32), ("start_y", ctypes.c_int32),
                ("end_x", ctypes.c_int32), ("end_y", ctypes.c_int32)]


class hvx_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "queued",
                                               "in_flight", "max_in_flight", "bytes_reserved",
                                               "peak_bytes_reserved")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "max_ms",
                                              "mpix_completed", "wait_p99_ms", "wait_max_ms")]


HVX_NOALLOC_MAX_FRAMES = 256


class hvx_edge_frame(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("in_pitch", ctypes.c_uint64),
                ("phase", ctypes.c_void_p), ("phase_pitch", ctypes.c_uint64),
                ("mask", ctypes.c_void_p), ("mask_pitch", ctypes.c_uint64),
                ("width", ctypes.c_uint32), ("height", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int32
U32 = ctypes.c_uint32
U64 = ctypes.c_uint64
PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes)
_SIGS = {
    "hvxStatusString": (ctypes.c_char_p, [I32]),
    "hvxCreateContext": (I32, [PP]),
    "hvxCreateContextEx": (I32, [I32, PP]),
    "hvxReleaseContext": (I32, [PP]),
    "hvxSetContextMemoryBudget": (I32, [P, U64]),
    "hvxSelfTestBoundedWait": (I32, [P]),
    "hvxSelfTestEdgePoint": (I32, [P, I32, I32, P, P]),
    "hvxTestInjectFault": (I32, [I32, ctypes.c_int64]),
    "hvxGetContextMemoryUsage": (I32, [P, ctypes.POINTER(U64)]),
    "hvxCreateImage": (I32, [P, U32, U32, I32, PP]),
    "hvxCreateImageFromHandle": (I32, [P, U32, U32, I32, P, U64, PP]),
    "hvxSwapImageHandle": (I32, [P, P, U64]),
    "hvxCreateVirtualImage": (I32, [P, U32, U32, I32, PP]),
    "hvxReleaseImage": (I32, [PP]),
    "hvxCopyImage": (I32, [P, P, U64, I32]),
    "hvxGetImageDevicePtr": (I32, [P, PP, ctypes.POINTER(U64)]),
    "hvxQueryImage": (I32, [P, ctypes.POINTER(U32), ctypes.POINTER(U32), ctypes.POINTER(I32)]),
    "hvxGetValidRegion": (I32, [P, ctypes.POINTER(hvx_rect)]),
    "hvxCreateGraph": (I32, [P, PP]),
    "hvxReleaseGraph": (I32, [PP]),
    "hvxVerifyGraph": (I32, [P]),
    "hvxProcessGraph": (I32, [P]),
    "hvxScheduleGraph": (I32, [P, P]),
    "hvxWaitGraph": (I32, [P]),
    "hvxSetGraphFusion": (I32, [P, I32]),
    "hvxSetGraphCodegen": (I32, [P, I32]),
    "hvxGetGraphKernelSource": (ctypes.c_int64, [P, I32, ctypes.c_char_p, U64]),
    "hvxGetGraphStatus": (I32, [P]),
    "hvxQueryGraph": (I32, [P, I32, P, U64]),
    "hvxProcessGraphBatch": (I32, [PP, I32, P]),
    "hvxWaitBatch": (I32, [P, P]),
    "hvxGaussian3x3Node": (P, [P, P, P]),
    "hvxBox3x3Node": (P, [P, P, P]),
    "hvxDilate3x3Node": (P, [P, P, P]),
    "hvxErode3x3Node": (P, [P, P, P]),
    "hvxMedian3x3Node": (P, [P, P, P]),
    "hvxAndNode": (P, [P, P, P, P]),
    "hvxOrNode": (P, [P, P, P, P]),
    "hvxXorNode": (P, [P, P, P, P]),
    "hvxNotNode": (P, [P, P, P]),
    "hvxSobel3x3Node": (P, [P, P, P, P]),
    "hvxMagnitudeNode": (P, [P, P, P, P]),
    "hvxPhaseNode": (P, [P, P, P, P]),
    "hvxThresholdNode": (P, [P, P, I32, ctypes.c_double, ctypes.c_double, I32, I32, P]),
    "hvxChannelExtractNode": (P, [P, P, I32, P]),
    "hvxAddNode": (P, [P, P, P, I32, P]),
    "hvxSubtractNode": (P, [P, P, P, I32, P]),
    "hvxAbsDiffNode": (P, [P, P, P, P]),
    "hvxMultiplyNode": (P, [P, P, P, ctypes.c_float, I32, I32, P]),
    "hvxCopyNode": (P, [P, P, P]),
    "hvxUserPointNode": (P, [P, ctypes.c_char_p, PP, I32, P]),
    "hvxUserLocalNode": (P, [P, ctypes.c_char_p, I32, I32, P, P]),
    "hvxConvertDepthNode": (P, [P, P, P, I32, I32]),
    "hvxMeanStdDevNode": (P, [P, P]),
    "hvxMinMaxLocNode": (P, [P, P]),
    "hvxHistogramNode": (P, [P, P, I32, I32, I32]),
    "hvxEqualizeHistNode": (P, [P, P, P]),
    "hvxGetNodeResult": (I32, [P, P, U64]),
    "hvxScheduleGraphBatchHost": (I32, [PP, I32, P, I32, P]),
    "hvxServerSubmitHost": (I32, [P, P, P, I32, ctypes.POINTER(ctypes.c_uint64)]),
    "hvxConvolveNode": (P, [P, P, ctypes.POINTER(I32), I32, I32, I32, P]),
    "hvxPointNode": (P, [P, I32, PP, I32, P, ctypes.POINTER(ctypes.c_double), I32]),
    "hvxLocalNode": (P, [P, I32, I32, I32, P, P]),
    "hvxSetNodeBorder": (I32, [P, I32, I32]),
    "hvxSetNodeRounding": (I32, [P, I32]),
    "hvxQueryNode": (I32, [P, I32, P, U64]),
    "hvxCreateServer": (I32, [P, U64, I32, I32, PP]),
    "hvxServerSubmit": (I32, [P, P, ctypes.POINTER(U64)]),
    "hvxServerSubmitMany": (I32, [P, P, I32, ctypes.POINTER(U64)]),
    "hvxQueryBatch": (I32, [P, I32, P, ctypes.POINTER(I32)]),
    "hvxServerWait": (I32, [P, U64, I32, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_double)]),
    "hvxServerStats": (I32, [P, ctypes.POINTER(hvx_server_stats)]),
    "hvxServerResetStats": (I32, [P]),
    "hvxReleaseServer": (I32, [PP]),
    "hvxEdgeBatchNoAlloc": (I32, [ctypes.c_void_p, I32, I32, I32, P]),
}


def lib():
    """Load libhvx.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def library_path() -> str:
    return _build.LIB


def _ck(st: int, where: str):
    if st != HVX_SUCCESS:
        raise HvxError(st, where)


def _node(h, g, where):
    if not h:
        raise HvxError(lib().hvxGetGraphStatus(g), where)
    return h


# --- status / context -----------------------------------------------------------

def hvxStatusString(status: int) -> str:
    return lib().hvxStatusString(status).decode()


def hvxCreateContext():
    out = ctypes.c_void_p()
    _ck(lib().hvxCreateContext(ctypes.byref(out)), "hvxCreateContext")
    return out


HVX_CONTEXT_PLAN_ONLY = 1


def hvxCreateContextEx(flags: int):
    out = ctypes.c_void_p()
    _ck(lib().hvxCreateContextEx(flags, ctypes.byref(out)), "hvxCreateContextEx")
    return out


def hvxReleaseContext(ctx):
    h = ctypes.c_void_p(ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx)
    _ck(lib().hvxReleaseContext(ctypes.byref(h)), "hvxReleaseContext")


def hvxSelfTestBoundedWait(ctx) -> int:
    """Status of the bounded-wait self-test (HVX_ERROR_TIMEOUT is the expected one)."""
    return lib().hvxSelfTestBoundedWait(ctx)


def hvxSelfTestEdgePoint(ctx, gmax: int, s_thr: int):
    """The fused edge kernel's Phase and mask bytes over every (gx, gy) in
    [-gmax, gmax]^2, as two (2 gmax + 1) x (2 gmax + 1) arrays indexed [gy, gx]."""
    import numpy as np
    n = 2 * gmax + 1
    ph = np.empty((n, n), np.uint8)
    mk = np.empty((n, n), np.uint8)
    _ck(lib().hvxSelfTestEdgePoint(ctx, gmax, s_thr, ph.ctypes.data, mk.ctypes.data),
        "hvxSelfTestEdgePoint")
    return ph, mk


HVX_FAULT_NONE, HVX_FAULT_DEVICE_ALLOC, HVX_FAULT_LAUNCH = 0, 1, 2


def hvxTestInjectFault(kind: int, n: int = 1):
    """Arm a host-side fault: the n-th device allocation (HVX_FAULT_DEVICE_ALLOC)
    or graph launch (HVX_FAULT_LAUNCH) from now on fails once; HVX_FAULT_NONE
    disarms both."""
    _ck(lib().hvxTestInjectFault(kind, n), "hvxTestInjectFault")


def hvxSetContextMemoryBudget(ctx, nbytes: int):
    _ck(lib().hvxSetContextMemoryBudget(ctx, nbytes), "hvxSetContextMemoryBudget")


def hvxGetContextMemoryUsage(ctx) -> int:
    v = U64()
    _ck(lib().hvxGetContextMemoryUsage(ctx, ctypes.byref(v)), "hvxGetContextMemoryUsage")
    return v.value


# --- images ------------------------------------------------------------------------

def hvxCreateImage(ctx, w, h, fmt):
    out = ctypes.c_void_p()
    _ck(lib().hvxCreateImage(ctx, w, h, fmt, ctypes.byref(out)), "hvxCreateImage")
    return out


def hvxCreateImageFromHandle(ctx, w, h, fmt, dev_ptr: int, pitch: int):
    out = ctypes.c_void_p()
    _ck(lib().hvxCreateImageFromHandle(ctx, w, h, fmt, dev_ptr, pitch, ctypes.byref(out)),
        "hvxCreateImageFromHandle")
    return out


def hvxSwapImageHandle(img, dev_ptr: int, pitch: int):
    _ck(lib().hvxSwapImageHandle(img, dev_ptr, pitch), "hvxSwapImageHandle")


def hvxCreateVirtualImage(graph, w=0, h=0, fmt=HVX_DF_VIRT):
    out = ctypes.c_void_p()
    _ck(lib().hvxCreateVirtualImage(graph, w, h, fmt, ctypes.byref(out)), "hvxCreateVirtualImage")
    return out


def hvxReleaseImage(img):
    h = ctypes.c_void_p(img.value if isinstance(img, ctypes.c_void_p) else img)
    _ck(lib().hvxReleaseImage(ctypes.byref(h)), "hvxReleaseImage")


def hvxCopyImage(img, host_ptr: int, host_pitch: int, usage: int):
    _ck(lib().hvxCopyImage(img, host_ptr, host_pitch, usage), "hvxCopyImage")


def hvxGetImageDevicePtr(img):
    p = ctypes.c_void_p()
    pitch = U64()
    _ck(lib().hvxGetImageDevicePtr(img, ctypes.byref(p), ctypes.byref(pitch)),
        "hvxGetImageDevicePtr")
    return p.value, pitch.value


def hvxQueryImage(img):
    w, h, f = U32(), U32(), I32()
    _ck(lib().hvxQueryImage(img, ctypes.byref(w), ctypes.byref(h), ctypes.byref(f)),
        "hvxQueryImage")
    return w.value, h.value, f.value


def hvxGetValidRegion(img):
    r = hvx_rect()
    _ck(lib().hvxGetValidRegion(img, ctypes.byref(r)), "hvxGetValidRegion")
    return (r.start_x, r.start_y, r.end_x, r.end_y)


# --- graphs ------------------------------------------------------------------------

def hvxCreateGraph(ctx):
    out = ctypes.c_void_p()
    _ck(lib().hvxCreateGraph(ctx, ctypes.byref(out)), "hvxCreateGraph")
    return out


def hvxReleaseGraph(g):
    h = ctypes.c_void_p(g.value if isinstance(g, ctypes.c_void_p) else g)
    _ck(lib().hvxReleaseGraph(ctypes.byref(h)), "hvxReleaseGraph")


def hvxVerifyGraph(g):
    _ck(lib().hvxVerifyGraph(g), "hvxVerifyGraph")


def hvxProcessGraph(g):
    _ck(lib().hvxProcessGraph(g), "hvxProcessGraph")


def hvxScheduleGraph(g, stream: int = 0):
    _ck(lib().hvxScheduleGraph(g, stream), "hvxScheduleGraph")


def hvxWaitGraph(g):
    _ck(lib().hvxWaitGraph(g), "hvxWaitGraph")


def hvxSetGraphFusion(g, enable: bool):
    _ck(lib().hvxSetGraphFusion(g, 1 if enable else 0), "hvxSetGraphFusion")


def hvxSetGraphCodegen(g, mode: int):
    _ck(lib().hvxSetGraphCodegen(g, mode), "hvxSetGraphCodegen")


def hvxGetGraphKernelSource(g, group: int):
    """Source of the kernel generated for launch `group`, or None."""
    n = lib().hvxGetGraphKernelSource(g, group, None, 0)
    if n < 0:
        return None
    buf = ctypes.create_string_buffer(n + 1)
    lib().hvxGetGraphKernelSource(g, group, buf, n + 1)
    return buf.value.decode()


def hvxGetGraphStatus(g) -> int:
    return lib().hvxGetGraphStatus(g)


def hvxQueryGraph(g, attribute: int):
    if attribute == HVX_GRAPH_KERNEL_KINDS:
        buf = ctypes.create_string_buffer(1024)
        _ck(lib().hvxQueryGraph(g, attribute, buf, 1024), "hvxQueryGraph")
        return buf.value.decode()
    if attribute in (HVX_GRAPH_INTERMEDIATE_BYTES, HVX_GRAPH_EXTERNAL_BYTES):
        v = U64()
        _ck(lib().hvxQueryGraph(g, attribute, ctypes.byref(v), 8), "hvxQueryGraph")
        return v.value
    v = I32()
    _ck(lib().hvxQueryGraph(g, attribute, ctypes.byref(v), 4), "hvxQueryGraph")
    return v.value


def hvxProcessGraphBatch(graphs, stream: int = 0):
    arr = (ctypes.c_void_p * len(graphs))(*[g.value if isinstance(g, ctypes.c_void_p) else g
                                            for g in graphs])
    _ck(lib().hvxProcessGraphBatch(arr, len(graphs), stream), "hvxProcessGraphBatch")


def hvxQueryBatch(graphs):
    """(rows per thread of each image's tiles, persistent grid) of the cached
    batch launch of exactly these graphs."""
    n = len(graphs)
    arr = (ctypes.c_void_p * n)(*[g.value if isinstance(g, ctypes.c_void_p) else g for g in graphs])
    rows = (I32 * n)()
    grid = I32()
    _ck(lib().hvxQueryBatch(arr, n, rows, ctypes.byref(grid)), "hvxQueryBatch")
    return [rows[i] for i in range(n)], grid.value


def hvxWaitBatch(ctx, stream: int = 0):
    _ck(lib().hvxWaitBatch(ctx, stream), "hvxWaitBatch")


# --- nodes -------------------------------------------------------------------------

def hvxGaussian3x3Node(g, i, o):
    return _node(lib().hvxGaussian3x3Node(g, i, o), g, "hvxGaussian3x3Node")


def hvxBox3x3Node(g, i, o):
    return _node(lib().hvxBox3x3Node(g, i, o), g, "hvxBox3x3Node")


def hvxDilate3x3Node(g, i, o):
    return _node(lib().hvxDilate3x3Node(g, i, o), g, "hvxDilate3x3Node")


def hvxErode3x3Node(g, i, o):
    return _node(lib().hvxErode3x3Node(g, i, o), g, "hvxErode3x3Node")


def hvxMedian3x3Node(g, i, o):
    return _node(lib().hvxMedian3x3Node(g, i, o), g, "hvxMedian3x3Node")


def hvxAndNode(g, a, b, o):
    return _node(lib().hvxAndNode(g, a, b, o), g, "hvxAndNode")


def hvxOrNode(g, a, b, o):
    return _node(lib().hvxOrNode(g, a, b, o), g, "hvxOrNode")


def hvxXorNode(g, a, b, o):
    return _node(lib().hvxXorNode(g, a, b, o), g, "hvxXorNode")


def hvxNotNode(g, i, o):
    return _node(lib().hvxNotNode(g, i, o), g, "hvxNotNode")


def hvxSobel3x3Node(g, i, gx, gy):
    return _node(lib().hvxSobel3x3Node(g, i, gx, gy), g, "hvxSobel3x3Node")


def hvxMagnitudeNode(g, gx, gy, o):
    return _node(lib().hvxMagnitudeNode(g, gx, gy, o), g, "hvxMagnitudeNode")


def hvxPhaseNode(g, gx, gy, o):
    return _node(lib().hvxPhaseNode(g, gx, gy, o), g, "hvxPhaseNode")


def hvxThresholdNode(g, i, type_, value, upper, true_value, false_value, o):
    return _node(lib().hvxThresholdNode(g, i, type_, float(value), float(upper), true_value,
                                        false_value, o), g, "hvxThresholdNode")


def hvxChannelExtractNode(g, i, channel, o):
    return _node(lib().hvxChannelExtractNode(g, i, channel, o), g, "hvxChannelExtractNode")


def hvxAddNode(g, a, b, policy, o):
    return _node(lib().hvxAddNode(g, a, b, policy, o), g, "hvxAddNode")


def hvxSubtractNode(g, a, b, policy, o):
    return _node(lib().hvxSubtractNode(g, a, b, policy, o), g, "hvxSubtractNode")


def hvxUserPointNode(g, expr: str, inputs, o):
    arr = (ctypes.c_void_p * len(inputs))(*[x.value if isinstance(x, ctypes.c_void_p) else x
                                            for x in inputs])
    return _node(lib().hvxUserPointNode(g, expr.encode(), arr, len(inputs), o), g,
                 "hvxUserPointNode")


def hvxUserLocalNode(g, expr: str, kw, kh, i, o):
    return _node(lib().hvxUserLocalNode(g, expr.encode(), kw, kh, i, o), g, "hvxUserLocalNode")


def hvxCopyNode(g, i, o):
    return _node(lib().hvxCopyNode(g, i, o), g, "hvxCopyNode")


def hvxConvertDepthNode(g, i, o, policy, shift):
    return _node(lib().hvxConvertDepthNode(g, i, o, policy, shift), g, "hvxConvertDepthNode")


def hvxMultiplyNode(g, a, b, scale, policy, rounding, o):
    return _node(lib().hvxMultiplyNode(g, a, b, float(scale), policy, rounding, o), g,
                 "hvxMultiplyNode")


def hvxAbsDiffNode(g, a, b, o):
    return _node(lib().hvxAbsDiffNode(g, a, b, o), g, "hvxAbsDiffNode")


def hvxConvolveNode(g, i, coeffs, kw, kh, shift, o):
    arr = (I32 * (kw * kh))(*[int(c) for c in coeffs])
    return _node(lib().hvxConvolveNode(g, i, arr, kw, kh, shift, o), g, "hvxConvolveNode")


def hvxPointNode(g, op, ins, out, params=()):
    arr = (ctypes.c_void_p * len(ins))(*[x.value if isinstance(x, ctypes.c_void_p) else x
                                         for x in ins])
    prm = (ctypes.c_double * max(1, len(params)))(*params)
    return _node(lib().hvxPointNode(g, op, arr, len(ins), out, prm, len(params)), g,
                 "hvxPointNode")


def hvxLocalNode(g, op, kw, kh, i, o):
    return _node(lib().hvxLocalNode(g, op, kw, kh, i, o), g, "hvxLocalNode")


def hvxSetNodeBorder(node, mode, constant=0):
    _ck(lib().hvxSetNodeBorder(node, mode, constant), "hvxSetNodeBorder")


def hvxSetNodeRounding(node, rounding):
    _ck(lib().hvxSetNodeRounding(node, rounding), "hvxSetNodeRounding")


def hvxQueryNode(node, attribute):
    v = I32()
    _ck(lib().hvxQueryNode(node, attribute, ctypes.byref(v), 4), "hvxQueryNode")
    return v.value if attribute != HVX_NODE_LIVE_OUTPUTS else v.value & 0xFFFFFFFF


# --- serving -----------------------------------------------------------------------

def hvxCreateServer(ctx, mem_budget: int, max_in_flight: int, n_streams: int):
    out = ctypes.c_void_p()
    _ck(lib().hvxCreateServer(ctx, mem_budget, max_in_flight, n_streams, ctypes.byref(out)),
        "hvxCreateServer")
    return out


def hvxServerSubmit(srv, g) -> int:
    t = U64()
    _ck(lib().hvxServerSubmit(srv, g, ctypes.byref(t)), "hvxServerSubmit")
    return t.value


def hvxServerSubmitMany(srv, graphs) -> list[int]:
    """Submit requests that arrive together (one queue insertion)."""
    n = len(graphs)
    arr = (ctypes.c_void_p * max(1, n))(*[g.value if isinstance(g, ctypes.c_void_p) else g
                                          for g in graphs])
    t = (U64 * max(1, n))()
    _ck(lib().hvxServerSubmitMany(srv, arr, n, t), "hvxServerSubmitMany")
    return [t[i] for i in range(n)]


def hvxServerWait(srv, ticket: int, timeout_ms: int = -1):
    """Returns (request status, latency ms)."""
    st = I32()
    lat = ctypes.c_double()
    _ck(lib().hvxServerWait(srv, ticket, timeout_ms, ctypes.byref(st), ctypes.byref(lat)),
        "hvxServerWait")
    return st.value, lat.value


def hvxServerStats(srv) -> dict:
    s = hvx_server_stats()
    _ck(lib().hvxServerStats(srv, ctypes.byref(s)), "hvxServerStats")
    return {n: getattr(s, n) for n, _ in hvx_server_stats._fields_}


def hvxServerResetStats(srv):
    _ck(lib().hvxServerResetStats(srv), "hvxServerResetStats")


def hvxReleaseServer(srv):
    h = ctypes.c_void_p(srv.value if isinstance(srv, ctypes.c_void_p) else srv)
    _ck(lib().hvxReleaseServer(ctypes.byref(h)), "hvxReleaseServer")


# --- batched edge graph without allocation --------------------------------------------

def hvxEdgeBatchNoAlloc(frames, border: int, threshold: int, stream: int = 0):
    """frames: sequence of hvx_edge_frame (device pointers and pitches)."""
    arr = (hvx_edge_frame * len(frames))(*frames)
    _ck(lib().hvxEdgeBatchNoAlloc(ctypes.cast(arr, ctypes.c_void_p), len(frames), border,
                                  threshold, stream), "hvxEdgeBatchNoAlloc")


# --- global operators ---------------------------------------------------------

class HvxMeanStdDev(ctypes.Structure):
    """hvx_mean_stddev of include/hvx.h."""
    _fields_ = [("mean", ctypes.c_float), ("stddev", ctypes.c_float), ("sum", ctypes.c_int64),
                ("sum_squares", ctypes.c_uint64), ("count", ctypes.c_uint64)]


class HvxMinMaxLoc(ctypes.Structure):
    """hvx_minmaxloc of include/hvx.h."""
    _fields_ = [("min", ctypes.c_int32), ("max", ctypes.c_int32),
                ("min_count", ctypes.c_uint64), ("max_count", ctypes.c_uint64),
                ("min_x", ctypes.c_int32), ("min_y", ctypes.c_int32),
                ("max_x", ctypes.c_int32), ("max_y", ctypes.c_int32)]


def hvxMeanStdDevNode(g, i):
    return _node(lib().hvxMeanStdDevNode(g, i), g, "hvxMeanStdDevNode")


def hvxMinMaxLocNode(g, i):
    return _node(lib().hvxMinMaxLocNode(g, i), g, "hvxMinMaxLocNode")


def hvxHistogramNode(g, i, num_bins, offset, range_):
    return _node(lib().hvxHistogramNode(g, i, num_bins, offset, range_), g, "hvxHistogramNode")


def hvxEqualizeHistNode(g, i, o):
    return _node(lib().hvxEqualizeHistNode(g, i, o), g, "hvxEqualizeHistNode")


def hvxGetNodeResult(node, out):
    """Copy a global operator's result into `out`: an HvxMeanStdDev, an
    HvxMinMaxLoc, or a uint32 numpy array of the histogram's bins."""
    if isinstance(out, ctypes.Structure):
        _ck(lib().hvxGetNodeResult(node, ctypes.byref(out), ctypes.sizeof(out)),
            "hvxGetNodeResult")
    else:
        _ck(lib().hvxGetNodeResult(node, out.ctypes.data, out.nbytes), "hvxGetNodeResult")
    return out


class HvxHostCopy(ctypes.Structure):
    """hvx_host_copy of include/hvx.h."""
    _fields_ = [("image", ctypes.c_void_p), ("host", ctypes.c_void_p), ("pitch", ctypes.c_uint64),
                ("to_device", ctypes.c_int32)]


def host_copies(items):
    """Array of HvxHostCopy from (image, host_pointer, pitch, to_device)
    tuples, for hvxScheduleGraphBatchHost."""
    arr = (HvxHostCopy * len(items))()
    for a, (img, ptr, pitch, to_dev) in zip(arr, items):
        a.image = img.value if isinstance(img, ctypes.c_void_p) else img
        a.host = ptr
        a.pitch = pitch
        a.to_device = 1 if to_dev else 0
    return arr


def hvxScheduleGraphBatchHost(graphs, copies, stream: int = 0):
    arr = (ctypes.c_void_p * len(graphs))(*[g.value if isinstance(g, ctypes.c_void_p) else g
                                            for g in graphs])
    cp = ctypes.cast(copies, ctypes.c_void_p) if len(copies) else None
    _ck(lib().hvxScheduleGraphBatchHost(arr, len(graphs), cp, len(copies), stream),
        "hvxScheduleGraphBatchHost")


def hvxServerSubmitHost(server, g, copies):
    """Submit a request whose host data (an array from host_copies) is copied
    in before and out after its launches; returns the ticket."""
    t = ctypes.c_uint64()
    cp = ctypes.cast(copies, ctypes.c_void_p) if len(copies) else None
    _ck(lib().hvxServerSubmitHost(server, g, cp, len(copies), ctypes.byref(t)),
        "hvxServerSubmitHost")
    return t.value
