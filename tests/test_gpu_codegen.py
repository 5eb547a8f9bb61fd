"""Kernels generated per graph (hvxSetGraphCodegen) against the CPU oracle and
against the staged-tile interpreter kernel: seeded random graphs of point and
local nodes (every border mode including MIRROR and REPEAT, U8 and S16
images, outputs that later nodes also read), fused and unfused, on sizes with no interior tile, with ragged
tiles and with many interior tiles.  Bit-exact."""
import numpy as np
import pytest

from oracle import graph as OG
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu

FMT = {"U8": H.HVX_DF_U8, "S16": H.HVX_DF_S16}
BORDER = {"replicate": H.HVX_BORDER_REPLICATE, "constant": H.HVX_BORDER_CONSTANT,
          "undefined": H.HVX_BORDER_UNDEFINED, "mirror": H.HVX_BORDER_MIRROR,
          "repeat": H.HVX_BORDER_REPEAT}


def random_graph(seed):
    """A random node list: (kind, inputs, outputs, params, output formats)."""
    rng = np.random.default_rng(seed)
    fmt = {"in": "U8"}
    sobel_out = set()
    nodes = []
    n = int(rng.integers(2, 8))
    for i in range(n):
        u8 = [k for k, f in fmt.items() if f == "U8"]
        s16 = [k for k, f in fmt.items() if f == "S16"]
        kinds = ["gaussian3x3", "box3x3", "dilate3x3", "erode3x3", "median3x3", "convolve",
                 "sobel3x3", "not", "threshold", "and", "add", "depth"]
        if s16:
            kinds += ["magnitude", "threshold16", "add16"]
        if len(sobel_out) >= 2:
            kinds += ["phase"]
        k = kinds[int(rng.integers(len(kinds)))]
        pick = lambda pool: pool[int(rng.integers(len(pool)))]  # noqa: E731
        o = f"t{i}"
        p = {}
        if k in ("gaussian3x3", "box3x3", "dilate3x3", "erode3x3", "median3x3", "convolve",
                 "sobel3x3"):
            p["border"] = ["replicate", "constant", "undefined", "mirror",
                           "repeat"][int(rng.integers(5))]
            p["cval"] = int(rng.integers(0, 256))
        if k in ("gaussian3x3", "box3x3"):
            p["rounding"] = ["zero", "nearest"][int(rng.integers(2))]
            nodes.append((k, [pick(u8)], [o], p, ["U8"]))
            fmt[o] = "U8"
        elif k in ("dilate3x3", "erode3x3", "median3x3"):
            nodes.append((k, [pick(u8)], [o], p, ["U8"]))
            fmt[o] = "U8"
        elif k == "convolve":
            ks = [3, 5][int(rng.integers(2))]
            p["coeffs"] = rng.integers(-6, 9, size=(ks, ks)).tolist()
            p["shift"] = int(rng.integers(0, 5))
            f = ["U8", "S16"][int(rng.integers(2))]
            nodes.append((k, [pick(u8)], [o], p, [f]))
            fmt[o] = f
        elif k == "sobel3x3":
            outs = [o + "x", o + "y"]
            if rng.random() < 0.3:
                outs[int(rng.integers(2))] = None
            nodes.append((k, [pick(u8)], outs, p, ["S16", "S16"]))
            for v in outs:
                if v:
                    fmt[v] = "S16"
                    sobel_out.add(v)
        elif k == "not":
            nodes.append((k, [pick(u8)], [o], p, ["U8"]))
            fmt[o] = "U8"
        elif k in ("threshold", "threshold16"):
            src = pick(u8) if k == "threshold" else pick(s16)
            lo = int(rng.integers(0, 200)) if k == "threshold" else int(rng.integers(-300, 300))
            if rng.random() < 0.5:
                p.update(type="binary", value=lo)
            else:
                p.update(type="range", lower=lo, upper=lo + int(rng.integers(0, 120)))
            p.update(true_value=int(rng.integers(0, 256)), false_value=int(rng.integers(0, 256)))
            nodes.append(("threshold", [src], [o], p, ["U8"]))
            fmt[o] = "U8"
        elif k == "and":
            kk = ["and", "or", "xor"][int(rng.integers(3))]
            nodes.append((kk, [pick(u8), pick(u8)], [o], p, ["U8"]))
            fmt[o] = "U8"
        elif k in ("add", "add16"):
            kk = ["add", "subtract", "absdiff", "multiply"][int(rng.integers(4))]
            a = pick(u8) if k == "add" else pick(s16)
            b = pick(u8) if rng.random() < 0.5 or not s16 else pick(s16)
            f = "S16" if "S16" in (fmt[a], fmt[b]) or rng.random() < 0.5 else "U8"
            if kk != "absdiff":
                p["policy"] = ["saturate", "wrap"][int(rng.integers(2))]
            if kk == "multiply":
                p["scale"] = [1.0, 1 / 255, 0.5, 3.0, 2.0 ** -7][int(rng.integers(5))]
                p["rounding"] = ["zero", "nearest_even"][int(rng.integers(2))]
            nodes.append((kk, [a, b], [o], p, [f]))
            fmt[o] = f
        elif k == "magnitude":
            nodes.append((k, [pick(s16), pick(s16)], [o], p, ["S16"]))
            fmt[o] = "S16"
        elif k == "depth":
            src = pick(u8 + s16)
            if rng.random() < 0.3:
                nodes.append(("copy", [src], [o], p, [fmt[src]]))
                fmt[o] = fmt[src]
            else:
                p.update(shift=int(rng.integers(0, 8)),
                         policy=["saturate", "wrap"][int(rng.integers(2))])
                f = "S16" if fmt[src] == "U8" else "U8"
                nodes.append(("convert_depth", [src], [o], p, [f]))
                fmt[o] = f
        elif k == "phase":
            so = sorted(sobel_out)
            nodes.append((k, [pick(so), pick(so)], [o], p, ["U8"]))
            fmt[o] = "U8"
    read = {i for _, ins, _, _, _ in nodes for i in ins}
    made = [v for _, _, outs, _, _ in nodes for v in outs if v]
    external = {v for v in made if v not in read or rng.random() < 0.3}
    return nodes, fmt, external


def build_oracle(nodes, fmt, external, w, h):
    g = OG.GraphDesc()
    g.image("in", w, h, "U8")
    for v, f in fmt.items():
        if v == "in":
            continue
        if v in external:
            g.image(v, w, h, f)
        else:
            g.virtual(v, fmt=f)
    for k, ins, outs, p, _ in nodes:
        g.node(k, ins, outs, **p)
    return g


def build_hvx(ctx, src, nodes, fmt, external, w, h):
    g = H.hvxCreateGraph(ctx)
    im = {"in": src}
    for v, f in fmt.items():
        if v == "in":
            continue
        im[v] = (PG.empty(ctx, w, h, FMT[f]) if v in external
                 else H.hvxCreateVirtualImage(g, 0, 0, FMT[f]))
    pol = {"saturate": H.HVX_POLICY_SATURATE, "wrap": H.HVX_POLICY_WRAP}
    for k, ins, outs, p, _ in nodes:
        a = [im[i] for i in ins]
        o = im[outs[0]] if outs[0] else None
        if k == "gaussian3x3":
            n = H.hvxGaussian3x3Node(g, a[0], o)
        elif k == "box3x3":
            n = H.hvxBox3x3Node(g, a[0], o)
        elif k == "dilate3x3":
            n = H.hvxDilate3x3Node(g, a[0], o)
        elif k == "erode3x3":
            n = H.hvxErode3x3Node(g, a[0], o)
        elif k == "median3x3":
            n = H.hvxMedian3x3Node(g, a[0], o)
        elif k == "convolve":
            c = np.asarray(p["coeffs"])
            n = H.hvxConvolveNode(g, a[0], c.ravel(), c.shape[1], c.shape[0], p["shift"], o)
        elif k == "sobel3x3":
            n = H.hvxSobel3x3Node(g, a[0], o, im[outs[1]] if outs[1] else None)
        elif k == "not":
            n = H.hvxNotNode(g, a[0], o)
        elif k in ("and", "or", "xor"):
            n = {"and": H.hvxAndNode, "or": H.hvxOrNode, "xor": H.hvxXorNode}[k](g, a[0], a[1], o)
        elif k == "threshold":
            if p["type"] == "binary":
                n = H.hvxThresholdNode(g, a[0], H.HVX_THRESHOLD_BINARY, p["value"], 0,
                                       p["true_value"], p["false_value"], o)
            else:
                n = H.hvxThresholdNode(g, a[0], H.HVX_THRESHOLD_RANGE, p["lower"], p["upper"],
                                       p["true_value"], p["false_value"], o)
        elif k == "add":
            n = H.hvxAddNode(g, a[0], a[1], pol[p["policy"]], o)
        elif k == "subtract":
            n = H.hvxSubtractNode(g, a[0], a[1], pol[p["policy"]], o)
        elif k == "absdiff":
            n = H.hvxAbsDiffNode(g, a[0], a[1], o)
        elif k == "multiply":
            n = H.hvxMultiplyNode(g, a[0], a[1], p["scale"], pol[p["policy"]],
                                  H.HVX_ROUND_TO_NEAREST_EVEN if p["rounding"] == "nearest_even"
                                  else H.HVX_ROUND_TO_ZERO, o)
        elif k == "magnitude":
            n = H.hvxMagnitudeNode(g, a[0], a[1], o)
        elif k == "copy":
            n = H.hvxCopyNode(g, a[0], o)
        elif k == "convert_depth":
            n = H.hvxConvertDepthNode(g, a[0], o, pol[p["policy"]], p["shift"])
        elif k == "phase":
            n = H.hvxPhaseNode(g, a[0], a[1], o)
        if "border" in p:
            H.hvxSetNodeBorder(n, BORDER[p["border"]], p["cval"])
        if p.get("rounding") == "nearest" and k != "multiply":
            H.hvxSetNodeRounding(n, H.HVX_ROUND_TO_NEAREST)
    return g, im


@pytest.fixture(scope="module")
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxReleaseContext(c)


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("w,h", [(7, 5), (300, 250)])
def test_random_graph_generated_matches_oracle(ctx, seed, w, h):
    nodes, fmt, external = random_graph(seed)
    img = synth.rects_noise(w, h, seed=seed + 100)
    ref = OG.run(build_oracle(nodes, fmt, external, w, h), {"in": img})
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    for fusion in (True, False):
        for codegen in (H.HVX_CODEGEN_REQUIRE, H.HVX_CODEGEN_OFF):
            g, im = build_hvx(ctx, src, nodes, fmt, external, w, h)
            H.hvxSetGraphFusion(g, fusion)
            H.hvxSetGraphCodegen(g, codegen)
            H.hvxVerifyGraph(g)
            kinds = PG.kernel_kinds(g)
            gen = H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS)
            assert gen == (kinds.count("staged_tile") if codegen else 0), kinds
            H.hvxProcessGraph(g)
            for v in external:
                if v not in ref:  # written by a node that dead-code elimination removed
                    continue
                np.testing.assert_array_equal(PG.download(im[v]), ref[v].data,
                                              err_msg=f"{v} fusion={fusion} codegen={codegen}")
                assert H.hvxGetValidRegion(im[v]) == ref[v].rect
            H.hvxReleaseGraph(g)


@pytest.mark.parametrize("w,h", [(1920, 1080), (1000, 999)])
def test_generated_interior_tiles_large(ctx, w, h):
    # frame-sized images: most tiles take the unchecked path
    for seed in (3, 11, 29):
        nodes, fmt, external = random_graph(seed)
        img = synth.rects_noise(w, h, seed=seed)
        ref = OG.run(build_oracle(nodes, fmt, external, w, h), {"in": img})
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        g, im = build_hvx(ctx, src, nodes, fmt, external, w, h)
        H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_REQUIRE)
        H.hvxVerifyGraph(g)
        H.hvxProcessGraph(g)
        for v in external:
            if v in ref:
                np.testing.assert_array_equal(PG.download(im[v]), ref[v].data)
        H.hvxReleaseGraph(g)


def test_generated_source_query(ctx):
    src = PG.upload(ctx, synth.rects_noise(64, 48, seed=1), H.HVX_DF_U8)
    out = PG.empty(ctx, 64, 48, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    H.hvxMedian3x3Node(g, src, out)
    H.hvxVerifyGraph(g)
    s = H.hvxGetGraphKernelSource(g, 0)
    assert s is not None and "hvx_generated" in s
    H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_OFF)
    H.hvxVerifyGraph(g)
    assert H.hvxGetGraphKernelSource(g, 0) is None
    H.hvxReleaseGraph(g)


@pytest.mark.parametrize("name", ["FChain", "Tomasi", "Harris", "Unsharp", "EdgFig2"])
def test_batched_generated_kernel(ctx, name):
    # graphs of the same shape on images of different sizes share one
    # generated kernel: hvxProcessGraphBatch runs them in one launch (the
    # corner groups get theirs under HVX_CODEGEN_ONLY)
    from paper_2008_11476_gb300 import apps as A
    build = dict(A.APPS)[name]
    sizes = [(300, 250), (1, 1), (640, 480), (97, 45), (129, 33)]
    graphs, outs, refs = [], [], []
    for i, (w, h) in enumerate(sizes):
        img = synth.rects_noise(w, h, seed=70 + i)
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        g, res = build(ctx, src, w, h, True)
        H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_ONLY)
        H.hvxVerifyGraph(g)
        assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == 1
        graphs.append(g)
        outs.append(res)
        g2, res2 = build(ctx, PG.upload(ctx, img, H.HVX_DF_U8), w, h, True)
        H.hvxSetGraphCodegen(g2, H.HVX_CODEGEN_OFF)
        H.hvxVerifyGraph(g2)
        H.hvxProcessGraph(g2)
        refs.append([PG.download(im) for _, im, _ in res2])
    for _ in range(2):  # the second call reuses the cached batch
        H.hvxProcessGraphBatch(graphs)
        H.hvxWaitBatch(ctx)
        for res, ref in zip(outs, refs):
            for (_, im, _), want in zip(res, ref):
                np.testing.assert_array_equal(PG.download(im), want)


def test_batch_of_different_generated_kernels(ctx):
    # different shapes: the batch call falls back to one launch per graph
    from paper_2008_11476_gb300 import apps as A
    graphs, outs, refs = [], [], []
    for i, (name, build) in enumerate(A.APPS):
        img = synth.rects_noise(200, 120, seed=90 + i)
        g, res = build(ctx, PG.upload(ctx, img, H.HVX_DF_U8), 200, 120, True)
        g2, res2 = build(ctx, PG.upload(ctx, img, H.HVX_DF_U8), 200, 120, True)
        H.hvxProcessGraph(g2)
        graphs.append(g)
        outs.append(res)
        refs.append([PG.download(im) for _, im, _ in res2])
    H.hvxProcessGraphBatch(graphs)
    H.hvxWaitBatch(ctx)
    for res, ref in zip(outs, refs):
        for (_, im, _), want in zip(res, ref):
            np.testing.assert_array_equal(PG.download(im), want)


WRAPS = [H.HVX_BORDER_MIRROR, H.HVX_BORDER_REPEAT]


@pytest.mark.parametrize("codegen", [H.HVX_CODEGEN_OFF, H.HVX_CODEGEN_REQUIRE])
@pytest.mark.parametrize("border", WRAPS)
@pytest.mark.parametrize("w,h", [(1, 1), (2, 3), (5, 4), (131, 37), (300, 250)])
def test_mirror_repeat_every_local_node(ctx, border, w, h, codegen):
    import oracle as O
    ob = O.BORDER_MIRROR if border == H.HVX_BORDER_MIRROR else O.BORDER_REPEAT
    img = synth.rects_noise(w, h, seed=w * 3 + h)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    c5 = np.arange(-12, 13).reshape(5, 5)
    cases = [
        (lambda g, o: H.hvxGaussian3x3Node(g, src, o), H.HVX_DF_U8, O.gaussian3x3(img, ob)),
        (lambda g, o: H.hvxBox3x3Node(g, src, o), H.HVX_DF_U8, O.box3x3(img, ob)),
        (lambda g, o: H.hvxDilate3x3Node(g, src, o), H.HVX_DF_U8,
         O.morph3x3(img, O.MORPH_DILATE, ob)),
        (lambda g, o: H.hvxMedian3x3Node(g, src, o), H.HVX_DF_U8,
         O.morph3x3(img, O.MORPH_MEDIAN, ob)),
        (lambda g, o: H.hvxConvolveNode(g, src, c5.ravel(), 5, 5, 2, o), H.HVX_DF_S16,
         O.convolve(img, c5, 2, ob)),
        (lambda g, o: H.hvxSobel3x3Node(g, src, o, None), H.HVX_DF_S16, O.sobel3x3(img, ob)[0]),
    ]
    for make, fmt, ref in cases:
        out = PG.empty(ctx, w, h, fmt)
        g = H.hvxCreateGraph(ctx)
        H.hvxSetNodeBorder(make(g, out), border, 0)
        H.hvxSetGraphCodegen(g, codegen)
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g) == ["staged_tile"]
        H.hvxProcessGraph(g)
        np.testing.assert_array_equal(PG.download(out), ref.data)
        assert H.hvxGetValidRegion(out) == (0, 0, w, h)
        H.hvxReleaseGraph(g)


@pytest.mark.parametrize("border", WRAPS)
def test_mirror_repeat_consumer_reads_materialised_producer(ctx, border):
    # Gaussian (REPLICATE) -> Sobel (MIRROR / REPEAT) -> Magnitude: the Sobel
    # does not fuse with the Gaussian; the Gaussian image goes through memory
    import oracle as O
    ob = O.BORDER_MIRROR if border == H.HVX_BORDER_MIRROR else O.BORDER_REPEAT
    w, h = 203, 77
    img = synth.rects_noise(w, h, seed=5)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    out = PG.empty(ctx, w, h, H.HVX_DF_S16)
    g = H.hvxCreateGraph(ctx)
    G, gx, gy = (H.hvxCreateVirtualImage(g) for _ in range(3))
    H.hvxGaussian3x3Node(g, src, G)
    H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, G, gx, gy), border, 0)
    H.hvxMagnitudeNode(g, gx, gy, out)
    H.hvxVerifyGraph(g)
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_LAUNCHES) == 2
    H.hvxProcessGraph(g)
    gxr, gyr = O.sobel3x3(O.gaussian3x3(img, O.BORDER_REPLICATE), ob)
    np.testing.assert_array_equal(PG.download(out), O.magnitude(gxr, gyr).data)
    H.hvxReleaseGraph(g)


@pytest.mark.parametrize("fmts", [("U8", "U8", "U8"), ("U8", "S16", "S16"), ("S16", "S16", "S16"),
                                  ("U8", "U8", "S16")])
@pytest.mark.parametrize("scale", [1.0, 1 / 255, 0.5, 3.0, 2.0 ** -20, 65536.0])
def test_multiply_node(ctx, fmts, scale):
    import oracle as O
    npf = {"U8": np.uint8, "S16": np.int16}
    w, h = 97, 31
    rng = np.random.default_rng(int(scale * 1000) % 97)
    arrs = []
    for f in fmts[:2]:
        arrs.append((rng.integers(0, 256, (h, w)) if f == "U8"
                     else rng.integers(-32768, 32768, (h, w))).astype(npf[f]))
    srcs = [PG.upload(ctx, a, FMT[f]) for a, f in zip(arrs, fmts[:2])]
    for pol, sat in ((H.HVX_POLICY_SATURATE, True), (H.HVX_POLICY_WRAP, False)):
        for rnd, ne in ((H.HVX_ROUND_TO_ZERO, False), (H.HVX_ROUND_TO_NEAREST_EVEN, True)):
            ref = O.multiply(arrs[0], arrs[1], scale, npf[fmts[2]], sat, ne)
            for fused in (False, True):
                out = PG.empty(ctx, w, h, FMT[fmts[2]])
                g = H.hvxCreateGraph(ctx)
                if fused:  # inside a generated kernel, behind a Dilate of the first input
                    d = H.hvxCreateVirtualImage(g)
                    if fmts[0] != "U8":
                        continue
                    H.hvxSetNodeBorder(H.hvxDilate3x3Node(g, srcs[0], d), H.HVX_BORDER_REPLICATE, 0)
                    H.hvxMultiplyNode(g, d, srcs[1], scale, pol, rnd, out)
                    want = O.multiply(O.morph3x3(arrs[0], O.MORPH_DILATE), arrs[1], scale,
                                      npf[fmts[2]], sat, ne).data
                else:
                    H.hvxMultiplyNode(g, srcs[0], srcs[1], scale, pol, rnd, out)
                    want = ref.data
                H.hvxVerifyGraph(g)
                H.hvxProcessGraph(g)
                np.testing.assert_array_equal(PG.download(out), want)
                H.hvxReleaseGraph(g)


@pytest.mark.parametrize("codegen", [H.HVX_CODEGEN_OFF, H.HVX_CODEGEN_REQUIRE])
@pytest.mark.parametrize("w,h", [(1, 1), (97, 31), (640, 480)])
def test_convert_depth_and_copy(ctx, w, h, codegen):
    import oracle as O
    rng = np.random.default_rng(w)
    u8 = rng.integers(0, 256, (h, w)).astype(np.uint8)
    s16 = rng.integers(-32768, 32768, (h, w)).astype(np.int16)
    for arr, fin, fout, npout in ((u8, H.HVX_DF_U8, H.HVX_DF_S16, np.int16),
                                  (s16, H.HVX_DF_S16, H.HVX_DF_U8, np.uint8)):
        src = PG.upload(ctx, arr, fin)
        for shift in (0, 3, 7):
            for pol, sat in ((H.HVX_POLICY_SATURATE, True), (H.HVX_POLICY_WRAP, False)):
                for fused in (False, True):
                    out = PG.empty(ctx, w, h, fout)
                    g = H.hvxCreateGraph(ctx)
                    if fused:  # behind a Copy and before nothing: one staged-tile group
                        c = H.hvxCreateVirtualImage(g)
                        H.hvxCopyNode(g, src, c)
                        H.hvxConvertDepthNode(g, c, out, pol, shift)
                    else:
                        H.hvxConvertDepthNode(g, src, out, pol, shift)
                    H.hvxSetGraphCodegen(g, codegen)
                    H.hvxVerifyGraph(g)
                    H.hvxProcessGraph(g)
                    np.testing.assert_array_equal(PG.download(out),
                                                  O.convert_depth(arr, npout, shift, sat).data)
                    H.hvxReleaseGraph(g)


@pytest.mark.parametrize("border", [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_CONSTANT,
                                    H.HVX_BORDER_UNDEFINED, H.HVX_BORDER_MIRROR,
                                    H.HVX_BORDER_REPEAT])
@pytest.mark.parametrize("w,h", [(1, 1), (45, 17), (640, 480)])
def test_user_defined_operators(ctx, border, w, h):
    # a user local operator (5x3 window) feeding a library Gaussian's output
    # and a user point operator on two images, fused into one generated kernel
    import oracle as O
    from oracle import user_ops as U
    ob = {H.HVX_BORDER_REPLICATE: O.BORDER_REPLICATE, H.HVX_BORDER_CONSTANT: O.BORDER_CONSTANT,
          H.HVX_BORDER_UNDEFINED: O.BORDER_UNDEFINED, H.HVX_BORDER_MIRROR: O.BORDER_MIRROR,
          H.HVX_BORDER_REPEAT: O.BORDER_REPEAT}[border]
    loc = "in(-2, 0) - 2 * in(0, 0) + in(2, 0) + max(in(0, -1), in(1, 1)) - abs(in(-1, 1) - 99)"
    pnt = "((a * 3 - b) >> 1) + (a < b) * 1000 - (a & 255 ^ b)"
    img = synth.rects_noise(w, h, seed=w + 7)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    out = PG.empty(ctx, w, h, H.HVX_DF_S16)
    g = H.hvxCreateGraph(ctx)
    G = H.hvxCreateVirtualImage(g)
    t = H.hvxCreateVirtualImage(g, 0, 0, H.HVX_DF_S16)
    H.hvxGaussian3x3Node(g, src, G)
    H.hvxSetNodeBorder(H.hvxUserLocalNode(g, loc, 5, 3, G, t), border, 17)
    H.hvxUserPointNode(g, pnt, [t, src], out)
    H.hvxVerifyGraph(g)
    if border not in (H.HVX_BORDER_MIRROR, H.HVX_BORDER_REPEAT):
        assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_LAUNCHES) == 1
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) >= 1
    H.hvxProcessGraph(g)
    Gr = O.gaussian3x3(img, O.BORDER_REPLICATE)
    tr = U.user_local(loc, Gr, 5, 3, ob, 17, np.int16)
    ref = U.user_point(pnt, [tr, O.Img(img)], np.int16)
    np.testing.assert_array_equal(PG.download(out), ref.data)
    assert H.hvxGetValidRegion(out) == ref.rect
    H.hvxReleaseGraph(g)


@pytest.mark.parametrize("name", ["Laplacian", "Sobel", "Unsharp", "Gauss"])
@pytest.mark.parametrize("w,h", [(1920, 1080), (385, 361)])
def test_column_blocks_match_the_interpreter(ctx, name, w, h, monkeypatch):
    # HVX_CODEGEN_COLS=4 (output pass in 2 x 4 cell blocks, vector loads,
    # vector stores on interior tiles) gives the interpreter's results
    from paper_2008_11476_gb300 import apps as A
    monkeypatch.setenv("HVX_CODEGEN_COLS", "4")
    build = dict(A.APPS)[name]
    img = synth.rects_noise(w, h, seed=w + h)
    g, res = build(ctx, PG.upload(ctx, img, H.HVX_DF_U8), w, h, True)
    # ONLY: a generated kernel also where a hand-written one exists (Sobel)
    H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_ONLY)
    H.hvxVerifyGraph(g)
    assert "columns per thread iteration" in H.hvxGetGraphKernelSource(g, 0)
    H.hvxProcessGraph(g)
    g2, res2 = build(ctx, PG.upload(ctx, img, H.HVX_DF_U8), w, h, True)
    H.hvxSetGraphCodegen(g2, H.HVX_CODEGEN_OFF)
    H.hvxVerifyGraph(g2)
    H.hvxProcessGraph(g2)
    for (_, a, _), (_, b, _) in zip(res, res2):
        np.testing.assert_array_equal(PG.download(a), PG.download(b))


@pytest.mark.parametrize("thr", [-5, 0, 1, 100, 1441, 32766, 32767, 40000])
def test_magnitude_threshold_compare(ctx, thr):
    # the generated kernel decides Magnitude -> Threshold as the integer
    # compare gx^2 + gy^2 > T^2 + T; the interpreter computes the rounded,
    # saturated magnitude first; both must give the oracle's mask.  S16
    # gradients from a 5x5 convolution reach magnitudes past 32767
    import oracle as O
    w, h = 333, 201
    img = synth.rects_noise(w, h, seed=thr & 0xFFFF)
    big = np.full((5, 5), 60, np.int32)
    big[:, :2] = -60
    outs = []
    for mode in (H.HVX_CODEGEN_REQUIRE, H.HVX_CODEGEN_OFF):
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
        g = H.hvxCreateGraph(ctx)
        gx, gy, m = (H.hvxCreateVirtualImage(g) for _ in range(3))
        a = H.hvxCreateVirtualImage(g, 0, 0, H.HVX_DF_S16)
        H.hvxSetNodeBorder(H.hvxConvolveNode(g, src, big.ravel(), 5, 5, 0, a),
                           H.HVX_BORDER_REPLICATE, 0)
        H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, src, gx, gy), H.HVX_BORDER_REPLICATE, 0)
        H.hvxMagnitudeNode(g, a, gy, m)
        H.hvxThresholdNode(g, m, H.HVX_THRESHOLD_BINARY, thr, 0, 255, 0, mk)
        H.hvxSetGraphCodegen(g, mode)
        H.hvxVerifyGraph(g)
        H.hvxProcessGraph(g)
        outs.append(PG.download(mk))
        H.hvxReleaseGraph(g)
    ga = O.convolve(img, big, 0, O.BORDER_REPLICATE)
    _, gyo = O.sobel3x3(img, O.BORDER_REPLICATE)
    want = O.threshold(O.magnitude(ga, gyo), thr).data
    np.testing.assert_array_equal(outs[0], want)
    np.testing.assert_array_equal(outs[1], want)
