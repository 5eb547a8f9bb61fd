"""Guard bands around output images: every kernel kind writes its outputs
into images placed inside larger device blocks filled with a canary byte,
and after processing every byte outside the images (guard rows above and
below, the 16 bytes before each row, the pitch padding after it) must still
hold the canary.  Catches out-of-bounds stores (vector stores at ragged
right edges, tile tails, batch tile tables) that output comparisons alone
would miss."""
import numpy as np
import pytest

from paper_2008_11476_gb300 import apps as A
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu

CANARY = 0xA5
GUARD_ROWS = 3
BPP = {H.HVX_DF_U8: 1, H.HVX_DF_S16: 2, H.HVX_DF_S32: 4, H.HVX_DF_F32: 4}


class Guarded:
    """An image inside a canary-filled device block."""

    def __init__(self, ctx, w, h, fmt):
        self.w, self.h, self.fmt = w, h, fmt
        row = w * BPP[fmt]
        self.bw = ((row + 16 + 48) + 127) // 128 * 128  # bytes of a block row
        self.bh = h + 2 * GUARD_ROWS
        self.block = H.hvxCreateImage(ctx, self.bw, self.bh, H.HVX_DF_U8)
        ptr, pitch = H.hvxGetImageDevicePtr(self.block)
        fill = np.full((self.bh, self.bw), CANARY, np.uint8)
        H.hvxCopyImage(self.block, fill.ctypes.data, self.bw, H.HVX_WRITE)
        self.img = H.hvxCreateImageFromHandle(ctx, w, h, fmt,
                                              ptr + GUARD_ROWS * pitch + 16, pitch)

    def check(self):
        got = np.empty((self.bh, self.bw), np.uint8)
        H.hvxCopyImage(self.block, got.ctypes.data, self.bw, H.HVX_READ)
        inside = np.zeros_like(got, dtype=bool)
        inside[GUARD_ROWS:GUARD_ROWS + self.h, 16:16 + self.w * BPP[self.fmt]] = True
        bad = np.argwhere((got != CANARY) & ~inside)
        assert bad.size == 0, f"{len(bad)} guard bytes overwritten, first at {bad[:4].tolist()}"


@pytest.fixture(scope="module")
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxReleaseContext(c)


SIZES = [(333, 77), (130, 17), (1920, 1080), (1, 1)]


@pytest.mark.parametrize("w,h", SIZES)
def test_guard_bands_edge_gauss_harris(ctx, w, h):
    img = synth.rects_noise(w, h, seed=3)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    outs = [Guarded(ctx, w, h, H.HVX_DF_U8) for _ in range(2)]
    g = PG.edge_graph(ctx, src, outs[0].img, outs[1].img)
    H.hvxProcessGraph(g)
    H.hvxProcessGraphBatch([g])
    H.hvxWaitBatch(ctx)
    gg = Guarded(ctx, w, h, H.HVX_DF_U8)
    g2 = H.hvxCreateGraph(ctx)
    H.hvxGaussian3x3Node(g2, src, gg.img)
    H.hvxVerifyGraph(g2)
    H.hvxProcessGraph(g2)
    H.hvxProcessGraphBatch([g2])
    H.hvxWaitBatch(ctx)
    hm = [Guarded(ctx, w, h, H.HVX_DF_U8) for _ in range(2)]
    g3 = PG.harris_graph(ctx, src, hm[0].img)                               # UNDEFINED: fast kernel
    g4 = PG.harris_graph(ctx, src, hm[1].img, border=H.HVX_BORDER_REPLICATE)  # general kernel
    H.hvxProcessGraph(g3)
    H.hvxProcessGraph(g4)
    for o in outs + [gg] + hm:
        o.check()


@pytest.mark.parametrize("codegen", [H.HVX_CODEGEN_OFF, H.HVX_CODEGEN_REQUIRE])
@pytest.mark.parametrize("w,h", SIZES)
def test_guard_bands_staged_tile_and_point(ctx, w, h, codegen):
    img = synth.rects_noise(w, h, seed=4)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    guards = []
    for name, fmt in (("FChain", H.HVX_DF_U8), ("Unsharp", H.HVX_DF_S16),
                      ("SobelMirror", H.HVX_DF_S16), ("SobelX", H.HVX_DF_S16)):
        o = Guarded(ctx, w, h, fmt)
        guards.append(o)
        g2 = H.hvxCreateGraph(ctx)
        if name == "FChain":
            a = H.hvxCreateVirtualImage(g2, 0, 0, H.HVX_DF_U8)
            H.hvxConvolveNode(g2, src, A.B3.ravel(), 3, 3, 4, a)
            H.hvxConvolveNode(g2, a, A.B5.ravel(), 5, 5, 8, o.img)
        elif name == "Unsharp":
            b = H.hvxCreateVirtualImage(g2)
            H.hvxGaussian3x3Node(g2, src, b)
            H.hvxSubtractNode(g2, src, b, H.HVX_POLICY_SATURATE, o.img)
        elif name == "SobelMirror":
            x = H.hvxCreateVirtualImage(g2)
            H.hvxSetNodeBorder(H.hvxSobel3x3Node(g2, src, x, None), H.HVX_BORDER_MIRROR, 0)
            H.hvxMultiplyNode(g2, x, x, 0.5, H.HVX_POLICY_SATURATE, H.HVX_ROUND_TO_ZERO, o.img)
        else:
            H.hvxSobel3x3Node(g2, src, o.img, None)
        H.hvxSetGraphCodegen(g2, codegen)
        H.hvxVerifyGraph(g2)
        H.hvxProcessGraph(g2)
    # a plain point node and EqualizeHist
    p = Guarded(ctx, w, h, H.HVX_DF_S16)
    g5 = H.hvxCreateGraph(ctx)
    H.hvxAddNode(g5, src, src, H.HVX_POLICY_WRAP, p.img)
    H.hvxVerifyGraph(g5)
    H.hvxProcessGraph(g5)
    e = Guarded(ctx, w, h, H.HVX_DF_U8)
    g6 = H.hvxCreateGraph(ctx)
    H.hvxEqualizeHistNode(g6, src, e.img)
    H.hvxVerifyGraph(g6)
    H.hvxProcessGraph(g6)
    for o in guards + [p, e]:
        o.check()
