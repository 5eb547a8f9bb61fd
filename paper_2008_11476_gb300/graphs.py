"""Builders for the standard image graphs, through the C ABI only.

* ``gaussian_graph``: one Gaussian3x3 node.
* ``edge_graph``: Gaussian3x3 -> Sobel3x3 -> Magnitude -> binary Threshold
  (mask) and Phase -- the edge detector of Listing 1 with both derivatives,
  as the Section 6 "Sobel"/"EdgFig" benchmarks use them.
* ``harris_graph``: Sobel3x3 -> gx^2, gy^2, gx*gy -> 5x5 window sums ->
  Harris response -> binary Threshold (HarrisCorners of Table 2 expressed as
  point + local + custom nodes).

Plus ``upload`` / ``download`` helpers that move numpy arrays in and out of
library images with hvxCopyImage.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import hvx as H

_NP = {H.HVX_DF_U8: np.uint8, H.HVX_DF_S16: np.int16, H.HVX_DF_S32: np.int32,
       H.HVX_DF_F32: np.float32, H.HVX_DF_UYVY: np.uint8}


def upload(ctx, arr: np.ndarray, fmt: int):
    """New library image holding `arr` ((H, W) array; UYVY: (H, 2W) bytes)."""
    a = np.ascontiguousarray(arr)
    h = a.shape[0]
    w = a.shape[1] // 2 if fmt == H.HVX_DF_UYVY else a.shape[1]
    img = H.hvxCreateImage(ctx, w, h, fmt)
    H.hvxCopyImage(img, a.ctypes.data, a.strides[0], H.HVX_WRITE)
    return img


def empty(ctx, w: int, h: int, fmt: int):
    return H.hvxCreateImage(ctx, w, h, fmt)


def download(img) -> np.ndarray:
    w, h, fmt = H.hvxQueryImage(img)
    cols = 2 * w if fmt == H.HVX_DF_UYVY else w
    out = np.empty((h, cols), _NP[fmt])
    H.hvxCopyImage(img, out.ctypes.data, out.strides[0], H.HVX_READ)
    return out


def gaussian_graph(ctx, inp, out, border=H.HVX_BORDER_REPLICATE, cval=0,
                   rounding=H.HVX_ROUND_TO_ZERO, fusion=True, verify=True):
    g = H.hvxCreateGraph(ctx)
    n = H.hvxGaussian3x3Node(g, inp, out)
    H.hvxSetNodeBorder(n, border, cval)
    H.hvxSetNodeRounding(n, rounding)
    H.hvxSetGraphFusion(g, fusion)
    if verify:
        H.hvxVerifyGraph(g)
    return g


def edge_graph(ctx, inp, phase=None, mask=None, border=H.HVX_BORDER_REPLICATE, cval=0,
               thr=100, mag_out=None, fusion=True, rounding=H.HVX_ROUND_TO_ZERO, verify=True,
               sobel_border=None, sobel_cval=None):
    g = H.hvxCreateGraph(ctx)
    G = H.hvxCreateVirtualImage(g)
    gx = H.hvxCreateVirtualImage(g)
    gy = H.hvxCreateVirtualImage(g)
    n1 = H.hvxGaussian3x3Node(g, inp, G)
    H.hvxSetNodeBorder(n1, border, cval)
    H.hvxSetNodeRounding(n1, rounding)
    n2 = H.hvxSobel3x3Node(g, G, gx, gy)
    H.hvxSetNodeBorder(n2, border if sobel_border is None else sobel_border,
                       cval if sobel_cval is None else sobel_cval)
    if mask is not None or mag_out is not None:
        m = mag_out if mag_out is not None else H.hvxCreateVirtualImage(g)
        H.hvxMagnitudeNode(g, gx, gy, m)
        if mask is not None:
            H.hvxThresholdNode(g, m, H.HVX_THRESHOLD_BINARY, thr, 0, 255, 0, mask)
    if phase is not None:
        H.hvxPhaseNode(g, gx, gy, phase)
    H.hvxSetGraphFusion(g, fusion)
    if verify:
        H.hvxVerifyGraph(g)
    return g


def harris_graph(ctx, inp, mask=None, resp_out=None, border=H.HVX_BORDER_UNDEFINED, cval=0,
                 kn=1, kd=25, thr=1e6, fusion=True, verify=True, tomasi=False):
    """Corner graph: Sobel3x3 -> products -> 5x5 window sums -> Harris
    response (kn / kd), or the Shi-Tomasi response when tomasi is set ->
    binary threshold."""
    g = H.hvxCreateGraph(ctx)
    gx = H.hvxCreateVirtualImage(g)
    gy = H.hvxCreateVirtualImage(g)
    n = H.hvxSobel3x3Node(g, inp, gx, gy)
    H.hvxSetNodeBorder(n, border, cval)
    prods = []
    for a, b in ((gx, gx), (gy, gy), (gx, gy)):
        p = H.hvxCreateVirtualImage(g)
        H.hvxPointNode(g, H.HVX_POINT_MUL, [a, b], p)
        prods.append(p)
    sums = []
    for p in prods:
        s = H.hvxCreateVirtualImage(g)
        ln = H.hvxLocalNode(g, H.HVX_LOCAL_SUM, 5, 5, p, s)
        H.hvxSetNodeBorder(ln, border, cval)
        sums.append(s)
    r = resp_out if resp_out is not None else H.hvxCreateVirtualImage(g)
    if tomasi:
        H.hvxPointNode(g, H.HVX_POINT_TOMASI_RESPONSE, sums, r)
    else:
        H.hvxPointNode(g, H.HVX_POINT_HARRIS_RESPONSE, sums, r, (kn, kd))
    if mask is not None:
        H.hvxThresholdNode(g, r, H.HVX_THRESHOLD_BINARY, thr, 0, 255, 0, mask)
    H.hvxSetGraphFusion(g, fusion)
    if verify:
        H.hvxVerifyGraph(g)
    return g


def kernel_kinds(g) -> list[str]:
    return H.hvxQueryGraph(g, H.HVX_GRAPH_KERNEL_KINDS).split(",")
