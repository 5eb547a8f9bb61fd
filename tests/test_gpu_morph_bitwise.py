"""GPU parity of the Table 2 nodes added beyond the edge and Harris graphs:
Dilate3x3, Erode3x3, Median3x3 (local) and And, Or, Xor, Not (point), alone
(one launch per node) and fused into one staged-tile group, against the CPU
oracle, bit-exact, under every border mode and on sizes with ragged tiles,
with the interpreter kernel and with kernels generated for the graph."""
import numpy as np
import pytest

import oracle as O
from oracle import graph as OG
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu

BORDERS = [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_CONSTANT, H.HVX_BORDER_UNDEFINED]
B_ORC = {H.HVX_BORDER_REPLICATE: O.BORDER_REPLICATE, H.HVX_BORDER_CONSTANT: O.BORDER_CONSTANT,
         H.HVX_BORDER_UNDEFINED: O.BORDER_UNDEFINED}
B_NAME = {H.HVX_BORDER_REPLICATE: "replicate", H.HVX_BORDER_CONSTANT: "constant",
          H.HVX_BORDER_UNDEFINED: "undefined"}
MORPH = [(H.hvxDilate3x3Node, O.MORPH_DILATE), (H.hvxErode3x3Node, O.MORPH_ERODE),
         (H.hvxMedian3x3Node, O.MORPH_MEDIAN)]


@pytest.fixture
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxReleaseContext(c)


CODEGEN = [H.HVX_CODEGEN_OFF, H.HVX_CODEGEN_REQUIRE]


@pytest.mark.parametrize("codegen", CODEGEN)
@pytest.mark.parametrize("w,h", [(1, 1), (3, 2), (65, 17), (131, 37), (300, 250)])
@pytest.mark.parametrize("border", BORDERS)
def test_morph_nodes_alone(ctx, w, h, border, codegen):
    # the three nodes read the same input: fused they form one staged-tile
    # group with three outputs, unfused three launches
    img = synth.rects_noise(w, h, seed=8 + w)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    for fusion, kinds in ((True, ["staged_tile"]), (False, ["staged_tile"] * 3)):
        outs = []
        g = H.hvxCreateGraph(ctx)
        for make, op in MORPH:
            o = PG.empty(ctx, w, h, H.HVX_DF_U8)
            n = make(g, src, o)
            H.hvxSetNodeBorder(n, border, 31)
            outs.append((o, op))
        H.hvxSetGraphFusion(g, fusion)
        H.hvxSetGraphCodegen(g, codegen)
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g) == kinds
        H.hvxProcessGraph(g)
        for o, op in outs:
            ref = O.morph3x3(img, op, B_ORC[border], 31)
            np.testing.assert_array_equal(PG.download(o), ref.data)
            assert H.hvxGetValidRegion(o) == ref.rect
        H.hvxReleaseGraph(g)


@pytest.mark.parametrize("w,h", [(1, 1), (64, 16), (129, 33)])
def test_bitwise_nodes(ctx, w, h):
    a = synth.uniform_u8(w, h, seed=31)
    b = synth.uniform_u8(w, h, seed=32)
    A = PG.upload(ctx, a, H.HVX_DF_U8)
    B = PG.upload(ctx, b, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    outs = []
    for make, op, two in ((H.hvxAndNode, O.BIT_AND, True), (H.hvxOrNode, O.BIT_OR, True),
                          (H.hvxXorNode, O.BIT_XOR, True), (H.hvxNotNode, O.BIT_NOT, False)):
        o = PG.empty(ctx, w, h, H.HVX_DF_U8)
        if two:
            make(g, A, B, o)
        else:
            make(g, A, o)
        outs.append((o, op, two))
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    for o, op, two in outs:
        np.testing.assert_array_equal(PG.download(o), O.bitwise(a, b if two else None, op).data)
    H.hvxReleaseGraph(g)


def _closing_tophat_oracle(img, border, cval):
    """Morphological closing, its difference from the input, a threshold,
    and the input's median ANDed with the mask: one oracle graph."""
    h, w = img.shape
    og = OG.GraphDesc()
    og.image("in", w, h, "U8")
    for v in ("d", "c", "diff", "mask", "med"):
        og.virtual(v)
    og.image("out", w, h, "U8")
    bn = B_NAME[border]
    og.node("dilate3x3", ["in"], ["d"], border=bn, cval=cval)
    og.node("erode3x3", ["d"], ["c"], border=bn, cval=cval)
    og.node("absdiff", ["c", "in"], ["diff"])
    og.node("threshold", ["diff"], ["mask"], value=20, true_value=255, false_value=0)
    og.node("median3x3", ["in"], ["med"], border=bn, cval=cval)
    og.node("and", ["med", "mask"], ["out"])
    return OG.run(og, {"in": img})["out"]


@pytest.mark.parametrize("codegen", CODEGEN)
@pytest.mark.parametrize("w,h", [(97, 45), (300, 250)])
@pytest.mark.parametrize("border", BORDERS)
def test_morph_graph_fused_matches_oracle(ctx, w, h, border, codegen):
    img = synth.rects_noise(w, h, seed=44)
    ref = _closing_tophat_oracle(img, border, 9)
    for fusion in (True, False):
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        out = PG.empty(ctx, w, h, H.HVX_DF_U8)
        g = H.hvxCreateGraph(ctx)
        d, c, diff, mask, med = (H.hvxCreateVirtualImage(g) for _ in range(5))
        for n in (H.hvxDilate3x3Node(g, src, d), H.hvxErode3x3Node(g, d, c),
                  H.hvxMedian3x3Node(g, src, med)):
            H.hvxSetNodeBorder(n, border, 9)
        H.hvxAbsDiffNode(g, c, src, diff)
        H.hvxThresholdNode(g, diff, H.HVX_THRESHOLD_BINARY, 20, 0, 255, 0, mask)
        H.hvxAndNode(g, med, mask, out)
        H.hvxSetGraphFusion(g, fusion)
        H.hvxSetGraphCodegen(g, codegen)
        H.hvxVerifyGraph(g)
        kinds = PG.kernel_kinds(g)
        if fusion:
            assert kinds == ["staged_tile"]
        else:
            assert len(kinds) == 6
        H.hvxProcessGraph(g)
        np.testing.assert_array_equal(PG.download(out), ref.data)
        assert H.hvxGetValidRegion(out) == ref.rect
        H.hvxReleaseGraph(g)
