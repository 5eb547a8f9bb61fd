"""GPU parity of the global operators (Table 2 "reduce" and "histogram":
MeanStdDev, MinMaxLoc, Histogram; EqualizeHist = histogram + point) against
the CPU oracle: alone on external images and fused as epilogues of the group
that computes their input, with the staged-tile interpreter and with
generated kernels, re-run (results reset per launch) and batched."""
import numpy as np
import pytest

import oracle as O
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu

CODEGEN = [H.HVX_CODEGEN_OFF, H.HVX_CODEGEN_REQUIRE]


@pytest.fixture(scope="module")
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxReleaseContext(c)


def check_meanstd(node, ref_img):
    m = H.hvxGetNodeResult(node, H.HvxMeanStdDev())
    mean, std, (s1, s2, n) = O.mean_stddev(ref_img)
    assert (m.sum, m.sum_squares, m.count) == (s1, s2, n)
    assert (m.mean, m.stddev) == (mean, std)


def check_minmax(node, ref_img):
    m = H.hvxGetNodeResult(node, H.HvxMinMaxLoc())
    r = O.minmaxloc(ref_img)
    if r["min_count"] == 0:
        assert m.min_count == 0 and m.max_count == 0 and m.min_x == -1
        return
    assert (m.min, m.max, m.min_count, m.max_count) == (r["min"], r["max"], r["min_count"],
                                                        r["max_count"])
    assert ((m.min_x, m.min_y), (m.max_x, m.max_y)) == (r["min_loc"], r["max_loc"])


def check_hist(node, ref_img, nb, off, rng_):
    got = H.hvxGetNodeResult(node, np.zeros(nb, np.uint32))
    np.testing.assert_array_equal(got, O.histogram(ref_img, nb, off, rng_))


@pytest.mark.parametrize("codegen", CODEGEN)
@pytest.mark.parametrize("fmt", [H.HVX_DF_U8, H.HVX_DF_S16])
@pytest.mark.parametrize("w,h", [(1, 1), (7, 5), (300, 250), (1920, 1080)])
def test_reductions_of_external_image(ctx, w, h, fmt, codegen):
    rng = np.random.default_rng(w + h)
    arr = (rng.integers(0, 256, (h, w)).astype(np.uint8) if fmt == H.HVX_DF_U8
           else rng.integers(-32768, 32768, (h, w)).astype(np.int16))
    src = PG.upload(ctx, arr, fmt)
    g = H.hvxCreateGraph(ctx)
    ms = H.hvxMeanStdDevNode(g, src)
    mm = H.hvxMinMaxLocNode(g, src)
    hs = H.hvxHistogramNode(g, src, 10, 50, 100) if fmt == H.HVX_DF_U8 else None
    H.hvxSetGraphCodegen(g, codegen)
    H.hvxVerifyGraph(g)
    for _ in range(2):  # results are reset before every launch
        H.hvxProcessGraph(g)
        check_meanstd(ms, arr)
        check_minmax(mm, arr)
        if hs:
            check_hist(hs, arr, 10, 50, 100)
    H.hvxReleaseGraph(g)


@pytest.mark.parametrize("codegen", CODEGEN)
@pytest.mark.parametrize("border", [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_UNDEFINED])
@pytest.mark.parametrize("w,h", [(97, 45), (640, 480)])
def test_reductions_fused_as_epilogues(ctx, w, h, border, codegen):
    # Gaussian -> Sobel -> Magnitude, with MeanStdDev and MinMaxLoc of the
    # magnitude and a histogram of the Gaussian image: one launch, no image
    # written (under UNDEFINED the valid regions shrink)
    img = synth.rects_noise(w, h, seed=21)
    ob = O.BORDER_REPLICATE if border == H.HVX_BORDER_REPLICATE else O.BORDER_UNDEFINED
    G_ref = O.gaussian3x3(img, ob)
    gx, gy = O.sobel3x3(G_ref, ob)
    mag = O.magnitude(gx, gy)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    G, x, y, m = (H.hvxCreateVirtualImage(g) for _ in range(4))
    H.hvxSetNodeBorder(H.hvxGaussian3x3Node(g, src, G), border, 0)
    H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, G, x, y), border, 0)
    H.hvxMagnitudeNode(g, x, y, m)
    ms = H.hvxMeanStdDevNode(g, m)
    mm = H.hvxMinMaxLocNode(g, m)
    hs = H.hvxHistogramNode(g, G, 16, 0, 256)
    H.hvxSetGraphCodegen(g, codegen)
    H.hvxVerifyGraph(g)
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_LAUNCHES) == 1
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_INTERMEDIATE_BYTES) == 0
    for _ in range(2):
        H.hvxProcessGraph(g)
        check_meanstd(ms, mag)
        check_minmax(mm, mag)
        check_hist(hs, G_ref, 16, 0, 256)
    H.hvxReleaseGraph(g)


def test_reductions_batched(ctx):
    # graphs sharing a generated kernel: one launch, every graph's own results
    graphs, refs = [], []
    for i, (w, h) in enumerate([(300, 250), (64, 33), (640, 480)]):
        img = synth.uniform_u8(w, h, seed=40 + i)
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        g = H.hvxCreateGraph(ctx)
        d = H.hvxCreateVirtualImage(g)
        H.hvxDilate3x3Node(g, src, d)
        nodes = (H.hvxMeanStdDevNode(g, d), H.hvxMinMaxLocNode(g, d),
                 H.hvxHistogramNode(g, d, 256, 0, 256))
        H.hvxVerifyGraph(g)
        assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == 1
        graphs.append(g)
        refs.append((nodes, O.morph3x3(img, O.MORPH_DILATE)))
    for _ in range(2):
        H.hvxProcessGraphBatch(graphs)
        H.hvxWaitBatch(ctx)
        for (ms, mm, hs), d in refs:
            check_meanstd(ms, d)
            check_minmax(mm, d)
            check_hist(hs, d, 256, 0, 256)


@pytest.mark.parametrize("w,h", [(1, 1), (5, 3), (300, 250), (1920, 1080)])
def test_equalize_hist(ctx, w, h):
    img = synth.rects_noise(w, h, seed=9)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    out = PG.empty(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    H.hvxEqualizeHistNode(g, src, out)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) == ["equalize_hist"]
    for _ in range(2):
        H.hvxProcessGraph(g)
        np.testing.assert_array_equal(PG.download(out), O.equalize_hist(img).data)
    H.hvxReleaseGraph(g)


def test_equalize_hist_of_computed_image_and_constant(ctx):
    w, h = 333, 111
    img = synth.rects_noise(w, h, seed=12)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    out = PG.empty(ctx, w, h, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    G = H.hvxCreateVirtualImage(g)
    H.hvxSetNodeBorder(H.hvxGaussian3x3Node(g, src, G), H.HVX_BORDER_UNDEFINED, 0)
    H.hvxEqualizeHistNode(g, G, out)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g)[-1] == "equalize_hist"
    H.hvxProcessGraph(g)
    ref = O.equalize_hist(O.gaussian3x3(img, O.BORDER_UNDEFINED))
    np.testing.assert_array_equal(PG.download(out), ref.data)
    assert H.hvxGetValidRegion(out) == ref.rect
    c = np.full((20, 30), 99, np.uint8)
    src = PG.upload(ctx, c, H.HVX_DF_U8)
    out = PG.empty(ctx, 30, 20, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    H.hvxEqualizeHistNode(g, src, out)
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    np.testing.assert_array_equal(PG.download(out), c)
