"""The applications of the paper's evaluation (Section 6) as graphs of this
library's nodes, for the suite benchmark (bench.py --workload apps) and tests.

    Gauss      5x5 binomial convolution (custom Convolve, U8 -> U8)
    Laplacian  3x3 Laplacian through the custom convolution API (U8 -> S16)
    FChain     three chained convolutions (3x3 binomial, 5x5 binomial, 3x3 sharpen)
    SobelX     Sobel3x3, horizontal derivative only
    EdgFig2    the edge detector of Listing 1 / Fig. 2 (Gaussian, Sobel,
               Magnitude of the vertical derivative -> Threshold; the
               horizontal derivative is the redundant kernel DCE removes)
    Sobel      Sobel3x3 -> Magnitude -> Threshold (three nodes)
    Unsharp    one Gaussian3x3 and three point nodes: in + 2 (in - blur), S16
    Harris     Sobel, three products, three 5x5 window sums, response, threshold
    Tomasi     as Harris with the Shi-Tomasi response (smaller eigenvalue)

Every builder takes (ctx, src U8 image, fusion) and returns (graph, outputs),
outputs being (name, image, format) of the graph's non-virtual results; all
nodes use BORDER_REPLICATE except Harris and Tomasi (BORDER_UNDEFINED).
"""
from __future__ import annotations

import numpy as np

from . import hvx as H

B5 = np.outer([1, 4, 6, 4, 1], [1, 4, 6, 4, 1]).astype(np.int32)          # sum 256
B3 = np.outer([1, 2, 1], [1, 2, 1]).astype(np.int32)                        # sum 16
LAPLACE = np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], np.int32)
SHARPEN = np.array([[0, -1, 0], [-1, 8, -1], [0, -1, 0]], np.int32)        # sum 4
TOMASI_THRESHOLD = 40000.0


def _img(ctx, w, h, fmt):
    return H.hvxCreateImage(ctx, w, h, fmt)


def _done(g, fusion):
    H.hvxSetGraphFusion(g, fusion)
    H.hvxVerifyGraph(g)
    return g


def _rep(n):
    H.hvxSetNodeBorder(n, H.HVX_BORDER_REPLICATE, 0)
    return n


def gauss(ctx, src, w, h, fusion=True):
    out = _img(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    _rep(H.hvxConvolveNode(g, src, B5.ravel(), 5, 5, 8, out))
    return _done(g, fusion), [("out", out, H.HVX_DF_U8)]


def laplacian(ctx, src, w, h, fusion=True):
    out = _img(ctx, w, h, H.HVX_DF_S16)
    g = H.hvxCreateGraph(ctx)
    _rep(H.hvxConvolveNode(g, src, LAPLACE.ravel(), 3, 3, 0, out))
    return _done(g, fusion), [("out", out, H.HVX_DF_S16)]


def fchain(ctx, src, w, h, fusion=True):
    out = _img(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    a = H.hvxCreateVirtualImage(g, 0, 0, H.HVX_DF_U8)
    b = H.hvxCreateVirtualImage(g, 0, 0, H.HVX_DF_U8)
    _rep(H.hvxConvolveNode(g, src, B3.ravel(), 3, 3, 4, a))
    _rep(H.hvxConvolveNode(g, a, B5.ravel(), 5, 5, 8, b))
    _rep(H.hvxConvolveNode(g, b, SHARPEN.ravel(), 3, 3, 2, out))
    return _done(g, fusion), [("out", out, H.HVX_DF_U8)]


def sobel_x(ctx, src, w, h, fusion=True):
    gx = _img(ctx, w, h, H.HVX_DF_S16)
    g = H.hvxCreateGraph(ctx)
    _rep(H.hvxSobel3x3Node(g, src, gx, None))
    return _done(g, fusion), [("gx", gx, H.HVX_DF_S16)]


def edg_fig2(ctx, src, w, h, fusion=True):
    # the graph of Listing 1 / Fig. 2 on a U8 input: only the vertical
    # derivative reaches the output, so the horizontal one is dead
    # (Algorithm 1 removes it) and Magnitude takes gy twice, as printed
    out = _img(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    blur, gx, gy, m = (H.hvxCreateVirtualImage(g) for _ in range(4))
    _rep(H.hvxGaussian3x3Node(g, src, blur))
    _rep(H.hvxSobel3x3Node(g, blur, gx, gy))
    H.hvxMagnitudeNode(g, gy, gy, m)
    H.hvxThresholdNode(g, m, H.HVX_THRESHOLD_BINARY, 100, 0, 255, 0, out)
    return _done(g, fusion), [("out", out, H.HVX_DF_U8)]


def sobel(ctx, src, w, h, fusion=True):
    out = _img(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    gx, gy, m = (H.hvxCreateVirtualImage(g) for _ in range(3))
    _rep(H.hvxSobel3x3Node(g, src, gx, gy))
    H.hvxMagnitudeNode(g, gx, gy, m)
    H.hvxThresholdNode(g, m, H.HVX_THRESHOLD_BINARY, 100, 0, 255, 0, out)
    return _done(g, fusion), [("out", out, H.HVX_DF_U8)]


def unsharp(ctx, src, w, h, fusion=True):
    out = _img(ctx, w, h, H.HVX_DF_S16)
    g = H.hvxCreateGraph(ctx)
    blur = H.hvxCreateVirtualImage(g)
    d = H.hvxCreateVirtualImage(g, 0, 0, H.HVX_DF_S16)
    d2 = H.hvxCreateVirtualImage(g, 0, 0, H.HVX_DF_S16)
    _rep(H.hvxGaussian3x3Node(g, src, blur))
    H.hvxSubtractNode(g, src, blur, H.HVX_POLICY_SATURATE, d)
    H.hvxAddNode(g, d, d, H.HVX_POLICY_SATURATE, d2)
    H.hvxAddNode(g, src, d2, H.HVX_POLICY_SATURATE, out)
    return _done(g, fusion), [("out", out, H.HVX_DF_S16)]


def harris(ctx, src, w, h, fusion=True):
    from . import graphs as PG
    mk = _img(ctx, w, h, H.HVX_DF_U8)
    return PG.harris_graph(ctx, src, mk, fusion=fusion), [("mask", mk, H.HVX_DF_U8)]


def tomasi(ctx, src, w, h, fusion=True):
    mk = _img(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    gx = H.hvxCreateVirtualImage(g)
    gy = H.hvxCreateVirtualImage(g)
    H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, src, gx, gy), H.HVX_BORDER_UNDEFINED, 0)
    sums = []
    for a, b in ((gx, gx), (gy, gy), (gx, gy)):
        p = H.hvxCreateVirtualImage(g)
        H.hvxPointNode(g, H.HVX_POINT_MUL, [a, b], p)
        s = H.hvxCreateVirtualImage(g)
        H.hvxSetNodeBorder(H.hvxLocalNode(g, H.HVX_LOCAL_SUM, 5, 5, p, s),
                           H.HVX_BORDER_UNDEFINED, 0)
        sums.append(s)
    r = H.hvxCreateVirtualImage(g)
    H.hvxPointNode(g, H.HVX_POINT_TOMASI_RESPONSE, sums, r)
    H.hvxThresholdNode(g, r, H.HVX_THRESHOLD_BINARY, TOMASI_THRESHOLD, 0, 255, 0, mk)
    return _done(g, fusion), [("mask", mk, H.HVX_DF_U8)]


APPS = [("Gauss", gauss), ("Laplacian", laplacian), ("FChain", fchain), ("SobelX", sobel_x),
        ("EdgFig2", edg_fig2), ("Sobel", sobel), ("Unsharp", unsharp), ("Harris", harris),
        ("Tomasi", tomasi)]
