"""GPU parity of the paper's Section 6 applications (paper_2008_11476_gb300/
apps.py) against the CPU oracle run node by node on the same graph (written
here again in the oracle's vocabulary), fused and unfused, with the
staged-tile groups run by the interpreter kernel and by kernels generated for
the graph, on a frame-sized and a ragged image.  Integer outputs must match exactly; the Tomasi mask may differ
only where the oracle's binary32 response lies within 1e-5 relative of the
threshold (the GPU evaluates the eigenvalue in binary32)."""
import numpy as np
import pytest

import oracle as O
from oracle import graph as OG
from paper_2008_11476_gb300 import apps as A
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu

B5 = [[1, 4, 6, 4, 1], [4, 16, 24, 16, 4], [6, 24, 36, 24, 6], [4, 16, 24, 16, 4],
      [1, 4, 6, 4, 1]]
B3 = [[1, 2, 1], [2, 4, 2], [1, 2, 1]]
LAP = [[0, 1, 0], [1, -4, 1], [0, 1, 0]]
SHARP = [[0, -1, 0], [-1, 8, -1], [0, -1, 0]]
REP = dict(border="replicate")
UND = dict(border="undefined")


def oracle_graph(name, w, h):
    """The application as an oracle graph; returns (graph, output names)."""
    g = OG.GraphDesc()
    g.image("in", w, h, "U8")
    n = g.node
    if name == "Gauss":
        g.image("out", w, h, "U8")
        n("convolve", ["in"], ["out"], coeffs=B5, shift=8, **REP)
        return g, ["out"]
    if name == "Laplacian":
        g.image("out", w, h, "S16")
        n("convolve", ["in"], ["out"], coeffs=LAP, shift=0, **REP)
        return g, ["out"]
    if name == "FChain":
        g.virtual("a", fmt="U8")
        g.virtual("b", fmt="U8")
        g.image("out", w, h, "U8")
        n("convolve", ["in"], ["a"], coeffs=B3, shift=4, **REP)
        n("convolve", ["a"], ["b"], coeffs=B5, shift=8, **REP)
        n("convolve", ["b"], ["out"], coeffs=SHARP, shift=2, **REP)
        return g, ["out"]
    if name == "SobelX":
        g.image("gx", w, h, "S16")
        n("sobel3x3", ["in"], ["gx", None], **REP)
        return g, ["gx"]
    if name == "EdgFig2":
        for v in ("G", "gx", "gy", "m"):
            g.virtual(v)
        g.image("out", w, h, "U8")
        n("gaussian3x3", ["in"], ["G"], **REP)
        n("sobel3x3", ["G"], ["gx", "gy"], **REP)
        n("magnitude", ["gy", "gy"], ["m"])
        n("threshold", ["m"], ["out"], value=100)
        return g, ["out"]
    if name == "Sobel":
        for v in ("gx", "gy", "m"):
            g.virtual(v)
        g.image("out", w, h, "U8")
        n("sobel3x3", ["in"], ["gx", "gy"], **REP)
        n("magnitude", ["gx", "gy"], ["m"])
        n("threshold", ["m"], ["out"], value=100)
        return g, ["out"]
    if name == "Unsharp":
        g.virtual("blur")
        g.virtual("d", fmt="S16")
        g.virtual("d2", fmt="S16")
        g.image("out", w, h, "S16")
        n("gaussian3x3", ["in"], ["blur"], **REP)
        n("subtract", ["in", "blur"], ["d"])
        n("add", ["d", "d"], ["d2"])
        n("add", ["in", "d2"], ["out"])
        return g, ["out"]
    # Harris / Tomasi
    for v in ("gx", "gy", "pxx", "pyy", "pxy", "sxx", "syy", "sxy", "r"):
        g.virtual(v)
    g.image("mask", w, h, "U8")
    n("sobel3x3", ["in"], ["gx", "gy"], **UND)
    for p, a, b in (("pxx", "gx", "gx"), ("pyy", "gy", "gy"), ("pxy", "gx", "gy")):
        n("mul", [a, b], [p])
        n("window_sum", [p], ["s" + p[1:]], kw=5, kh=5, **UND)
    if name == "Harris":
        n("harris_response", ["sxx", "syy", "sxy"], ["r"], kn=1, kd=25)
        n("threshold", ["r"], ["mask"], value=1e6)
    else:
        n("tomasi_response", ["sxx", "syy", "sxy"], ["r"])
        n("threshold", ["r"], ["mask"], value=A.TOMASI_THRESHOLD)
    return g, ["mask"]


def tomasi_response_oracle(img):
    gx, gy = O.sobel3x3(img, O.BORDER_UNDEFINED)
    s = [O.window_sum(O.mul_s32(a, b), 5, 5, O.BORDER_UNDEFINED)
         for a, b in ((gx, gx), (gy, gy), (gx, gy))]
    return O.tomasi_response(*s)


@pytest.fixture(scope="module")
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxReleaseContext(c)


@pytest.mark.parametrize("codegen", [H.HVX_CODEGEN_OFF, H.HVX_CODEGEN_REQUIRE,
                                     H.HVX_CODEGEN_ONLY])
@pytest.mark.parametrize("name", [a for a, _ in A.APPS])
@pytest.mark.parametrize("w,h", [(640, 480), (385, 361)])
def test_app_matches_oracle(ctx, name, w, h, codegen):
    img = synth.rects_noise(w, h, seed=13)
    og, outs = oracle_graph(name, w, h)
    ref = OG.run(og, {"in": img})
    build = dict(A.APPS)[name]
    for fusion in (True, False):
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        g, res = build(ctx, src, w, h, fusion)
        H.hvxSetGraphCodegen(g, codegen)
        H.hvxVerifyGraph(g)
        kinds = PG.kernel_kinds(g)
        if fusion:
            assert len(kinds) == 1, kinds
        gen = H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS)
        assert gen == (kinds.count("staged_tile") if codegen else 0)
        H.hvxProcessGraph(g)
        for (oname, im, fmt), rname in zip(res, outs):
            got = PG.download(im)
            want = ref[rname].data
            if name == "Tomasi":
                lam = tomasi_response_oracle(img).data
                near = np.abs(lam - A.TOMASI_THRESHOLD) <= 1e-5 * A.TOMASI_THRESHOLD
                assert near.sum() < 20
                np.testing.assert_array_equal(got[~near], want[~near])
                assert want.any() and not want.all()
            else:
                np.testing.assert_array_equal(got, want)
            assert H.hvxGetValidRegion(im) == ref[rname].rect
        H.hvxReleaseGraph(g)


def _listing1_graph(ctx, src, w, h, border, cval):
    # Listing 1 / Fig. 2: Gaussian3x3 -> Sobel3x3 -> Magnitude(gy, gy) ->
    # Threshold(100); gx has no consumer (Algorithm 1 removes it)
    out = PG.empty(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    blur, gx, gy, m = (H.hvxCreateVirtualImage(g) for _ in range(4))
    H.hvxSetNodeBorder(H.hvxGaussian3x3Node(g, src, blur), border, cval)
    H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, blur, gx, gy), border, cval)
    H.hvxMagnitudeNode(g, gy, gy, m)
    H.hvxThresholdNode(g, m, H.HVX_THRESHOLD_BINARY, 100, 0, 255, 0, out)
    H.hvxVerifyGraph(g)
    return g, out


def _listing1_oracle(img, border, cval):
    h, w = img.shape
    g = OG.GraphDesc()
    g.image("in", w, h, "U8")
    for v in ("G", "gx", "gy", "m"):
        g.virtual(v)
    g.image("out", w, h, "U8")
    b = dict(border=border, cval=cval)
    g.node("gaussian3x3", ["in"], ["G"], **b)
    g.node("sobel3x3", ["G"], ["gx", "gy"], **b)
    g.node("magnitude", ["gy", "gy"], ["m"])
    g.node("threshold", ["m"], ["out"], value=100)
    return OG.run(g, {"in": img})["out"]


@pytest.mark.parametrize("border", ["replicate", "constant", "undefined"])
def test_listing1_graph_on_the_fused_edge_kernel(ctx, border):
    # with gx dead, Magnitude(gy, gy) -> binary Threshold runs on the fused
    # edge kernel (its mask mode with 2 gy^2 > T^2 + T), one image per launch
    # and batched, every border, exact against the oracle
    hb = {"replicate": H.HVX_BORDER_REPLICATE, "constant": H.HVX_BORDER_CONSTANT,
          "undefined": H.HVX_BORDER_UNDEFINED}[border]
    sizes = [(1, 1), (97, 45), (300, 200), (129, 121), (1920, 1080)]
    items = []
    for i, (w, h) in enumerate(sizes):
        img = synth.rects_noise(w, h, seed=90 + i)
        g, out = _listing1_graph(ctx, PG.upload(ctx, img, H.HVX_DF_U8), w, h, hb, 7)
        assert PG.kernel_kinds(g) == ["fused_edge_tma"]
        items.append((img, g, out, _listing1_oracle(img, border, 7)))
    for img, g, out, ref in items:
        H.hvxProcessGraph(g)
        x0, y0, x1, y1 = ref.rect
        got = PG.download(out)
        np.testing.assert_array_equal(got[y0:y1, x0:x1], ref.data[y0:y1, x0:x1])
        assert H.hvxGetValidRegion(out) == ref.rect
    for _, _, out, _ in items:  # clear the outputs, then the batched form
        w, h, _ = H.hvxQueryImage(out)
        z = np.zeros((h, w), np.uint8)
        H.hvxCopyImage(out, z.ctypes.data, w, H.HVX_WRITE)
    H.hvxProcessGraphBatch([it[1] for it in items])
    H.hvxWaitBatch(ctx)
    for img, g, out, ref in items:
        x0, y0, x1, y1 = ref.rect
        np.testing.assert_array_equal(PG.download(out)[y0:y1, x0:x1], ref.data[y0:y1, x0:x1])


def _sobel_graph(ctx, src, w, h, border, cval, thr):
    out = PG.empty(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    gx, gy, m = (H.hvxCreateVirtualImage(g) for _ in range(3))
    H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, src, gx, gy), border, cval)
    H.hvxMagnitudeNode(g, gx, gy, m)
    H.hvxThresholdNode(g, m, H.HVX_THRESHOLD_BINARY, thr, 0, 255, 0, out)
    H.hvxVerifyGraph(g)
    return g, out


def _sobel_oracle(img, border, cval, thr):
    h, w = img.shape
    g = OG.GraphDesc()
    g.image("in", w, h, "U8")
    for v in ("gx", "gy", "m"):
        g.virtual(v)
    g.image("out", w, h, "U8")
    g.node("sobel3x3", ["in"], ["gx", "gy"], border=border, cval=cval)
    g.node("magnitude", ["gx", "gy"], ["m"])
    g.node("threshold", ["m"], ["out"], value=thr)
    return OG.run(g, {"in": img})["out"]


@pytest.mark.parametrize("border", ["replicate", "constant", "undefined"])
def test_sobel_graph_on_the_fused_edge_kernel(ctx, border):
    # Sobel3x3 -> Magnitude -> binary Threshold with no Gaussian node runs on
    # the fused edge kernel with the input rows in place of Gaussian rows: every
    # border, ragged sizes, thresholds at both ends, single and batched launches
    hb = {"replicate": H.HVX_BORDER_REPLICATE, "constant": H.HVX_BORDER_CONSTANT,
          "undefined": H.HVX_BORDER_UNDEFINED}[border]
    sizes = [(1, 1), (97, 45), (300, 200), (129, 121), (1920, 1080)]
    for thr in (100, 0, 1441):
        items = []
        for i, (w, h) in enumerate(sizes):
            img = synth.rects_noise(w, h, seed=110 + i)
            g, out = _sobel_graph(ctx, PG.upload(ctx, img, H.HVX_DF_U8), w, h, hb, 250, thr)
            assert PG.kernel_kinds(g) == ["fused_edge_tma"]
            items.append((g, out, _sobel_oracle(img, border, 250, thr)))
        for g, out, ref in items:
            H.hvxProcessGraph(g)
            x0, y0, x1, y1 = ref.rect
            np.testing.assert_array_equal(PG.download(out)[y0:y1, x0:x1],
                                          ref.data[y0:y1, x0:x1])
            assert H.hvxGetValidRegion(out) == ref.rect
        for _, out, _ in items:
            w, h, _ = H.hvxQueryImage(out)
            z = np.zeros((h, w), np.uint8)
            H.hvxCopyImage(out, z.ctypes.data, w, H.HVX_WRITE)
        H.hvxProcessGraphBatch([it[0] for it in items])
        H.hvxWaitBatch(ctx)
        for _, out, ref in items:
            x0, y0, x1, y1 = ref.rect
            np.testing.assert_array_equal(PG.download(out)[y0:y1, x0:x1],
                                          ref.data[y0:y1, x0:x1])


B5_COEFFS = np.outer([1, 4, 6, 4, 1], [1, 4, 6, 4, 1]).astype(np.int32)


@pytest.mark.parametrize("border", [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_CONSTANT,
                                    H.HVX_BORDER_UNDEFINED])
def test_binomial5x5_kernel(ctx, border):
    # the 5x5 binomial Convolve (shift 8, U8 -> U8) on its hand-written
    # kernel: every border, ragged tiles, images smaller than a tile, extreme
    # bytes (sums up to 255 * 256), single and batched launches, exact
    ob = {H.HVX_BORDER_REPLICATE: O.BORDER_REPLICATE, H.HVX_BORDER_CONSTANT: O.BORDER_CONSTANT,
          H.HVX_BORDER_UNDEFINED: O.BORDER_UNDEFINED}[border]
    sizes = [(1, 1), (3, 2), (97, 45), (300, 200), (129, 121), (1920, 1080)]
    items = []
    for i, (w, h) in enumerate(sizes):
        img = synth.rects_noise(w, h, seed=130 + i)
        if i == 3:
            img[::2] = 255  # saturated rows: the largest sums
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        out = PG.empty(ctx, w, h, H.HVX_DF_U8)
        g = H.hvxCreateGraph(ctx)
        H.hvxSetNodeBorder(H.hvxConvolveNode(g, src, B5_COEFFS.ravel(), 5, 5, 8, out), border, 251)
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g) == ["binomial5x5_tma"]
        items.append((g, out, O.convolve(img, B5_COEFFS, 8, ob, 251, out_dtype=np.uint8)))
    for g, out, ref in items:
        H.hvxProcessGraph(g)
        x0, y0, x1, y1 = ref.rect
        np.testing.assert_array_equal(PG.download(out)[y0:y1, x0:x1], ref.data[y0:y1, x0:x1])
        assert H.hvxGetValidRegion(out) == ref.rect
    for _, out, _ in items:
        w, h, _ = H.hvxQueryImage(out)
        z = np.zeros((h, w), np.uint8)
        H.hvxCopyImage(out, z.ctypes.data, w, H.HVX_WRITE)
    H.hvxProcessGraphBatch([it[0] for it in items])
    H.hvxWaitBatch(ctx)
    for _, out, ref in items:
        x0, y0, x1, y1 = ref.rect
        np.testing.assert_array_equal(PG.download(out)[y0:y1, x0:x1], ref.data[y0:y1, x0:x1])
    # other coefficients stay on the generated kernels
    g = H.hvxCreateGraph(ctx)
    c2 = B5_COEFFS.copy()
    c2[2, 2] += 1
    H.hvxConvolveNode(g, PG.upload(ctx, synth.rects_noise(40, 30, seed=1), H.HVX_DF_U8),
                      c2.ravel(), 5, 5, 8, PG.empty(ctx, 40, 30, H.HVX_DF_U8))
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) != ["binomial5x5_tma"]


@pytest.mark.parametrize("border", ["replicate", "constant", "undefined"])
def test_sobel_x_on_the_fused_edge_kernel(ctx, border):
    # Sobel3x3 with only gx exported (S16) runs on the fused edge kernel's
    # input-row mode, gx converted to S16 lanes in registers: every border,
    # ragged sizes, extreme gradients, single and batched launches, exact
    hb = {"replicate": H.HVX_BORDER_REPLICATE, "constant": H.HVX_BORDER_CONSTANT,
          "undefined": H.HVX_BORDER_UNDEFINED}[border]
    ob = {"replicate": O.BORDER_REPLICATE, "constant": O.BORDER_CONSTANT,
          "undefined": O.BORDER_UNDEFINED}[border]
    sizes = [(1, 1), (3, 2), (97, 45), (300, 200), (129, 121), (1920, 1080)]
    items = []
    for i, (w, h) in enumerate(sizes):
        img = synth.rects_noise(w, h, seed=150 + i)
        if i == 3:
            img[:, ::2] = 0      # vertical stripes: gx at the extremes +-1020
            img[:, 1::2] = 255
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        gx = PG.empty(ctx, w, h, H.HVX_DF_S16)
        g = H.hvxCreateGraph(ctx)
        H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, src, gx, None), hb, 77)
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g) == ["fused_edge_tma"]
        items.append((g, gx, O.sobel3x3(img, ob, 77)[0]))
    for g, gx, ref in items:
        H.hvxProcessGraph(g)
        x0, y0, x1, y1 = ref.rect
        np.testing.assert_array_equal(PG.download(gx)[y0:y1, x0:x1], ref.data[y0:y1, x0:x1])
        assert H.hvxGetValidRegion(gx) == ref.rect
    for _, gx, _ in items:
        w, h, _ = H.hvxQueryImage(gx)
        z = np.zeros((h, w), np.int16)
        H.hvxCopyImage(gx, z.ctypes.data, 2 * w, H.HVX_WRITE)
    H.hvxProcessGraphBatch([it[0] for it in items])
    H.hvxWaitBatch(ctx)
    for _, gx, ref in items:
        x0, y0, x1, y1 = ref.rect
        np.testing.assert_array_equal(PG.download(gx)[y0:y1, x0:x1], ref.data[y0:y1, x0:x1])
