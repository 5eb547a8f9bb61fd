"""GPU parity: every kernel of the image-graph path against the CPU oracle, on
the same seeded inputs, through the C ABI.  Integer outputs must match bit for
bit; the F32 Harris response within 1e-5 relative (it is in fact rounded once
from the exact value, so it is compared bit for bit as well)."""
import numpy as np
import pytest

import oracle as O
import oracle.graph as OG
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu

B_ORC = {H.HVX_BORDER_UNDEFINED: O.BORDER_UNDEFINED, H.HVX_BORDER_REPLICATE: O.BORDER_REPLICATE,
         H.HVX_BORDER_CONSTANT: O.BORDER_CONSTANT}
BORDERS = [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_CONSTANT, H.HVX_BORDER_UNDEFINED]
# sizes spanning several tiles and ragged tails, plus degenerate ones
SIZES = [(1, 1), (2, 1), (1, 3), (3, 3), (17, 5), (64, 16), (131, 37), (257, 70), (640, 480)]


@pytest.fixture(scope="module")
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxReleaseContext(c)


def circ_diff(a, b):
    d = np.abs(a.astype(np.int64) - b.astype(np.int64)) % 256
    return np.minimum(d, 256 - d)


# --- Gaussian3x3 (the plain one-node graph) --------------------------------------

# the single-image Gaussian kernel's tiles are 128 x 8R, R = 2 (fewer 128 x 40
# tiles than SMs) or 5: add sizes with several ragged tile rows of each
@pytest.mark.parametrize("w,h", SIZES + [(300, 250), (385, 361), (1921, 1083), (2500, 803)])
@pytest.mark.parametrize("border", BORDERS)
def test_gaussian(ctx, w, h, border):
    img = synth.uniform_u8(w, h, seed=1 + w + h)
    for rounding in (H.HVX_ROUND_TO_ZERO, H.HVX_ROUND_TO_NEAREST):
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        out = PG.empty(ctx, w, h, H.HVX_DF_U8)
        g = PG.gaussian_graph(ctx, inp, out, border=border, cval=77, rounding=rounding)
        assert PG.kernel_kinds(g) == ["gaussian3x3_tma"]
        H.hvxProcessGraph(g)
        ref = O.gaussian3x3(img, B_ORC[border], 77, rounding)
        np.testing.assert_array_equal(PG.download(out), ref.data)
        assert H.hvxGetValidRegion(out) == ref.rect
        H.hvxReleaseGraph(g)


def test_gaussian_config_640x480_replicate(ctx):
    img = synth.uniform_u8(640, 480, seed=1)
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    out = PG.empty(ctx, 640, 480, H.HVX_DF_U8)
    g = PG.gaussian_graph(ctx, inp, out)
    for _ in range(3):  # re-executable (Section 3.1)
        H.hvxProcessGraph(g)
    np.testing.assert_array_equal(PG.download(out), O.gaussian3x3(img).data)


# --- edge graph --------------------------------------------------------------------

def run_edge(ctx, img, border, cval=0, fusion=True, want_mag=False, rounding=0, thr=100):
    h, w = img.shape
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    ph = PG.empty(ctx, w, h, H.HVX_DF_U8)
    mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
    mg = PG.empty(ctx, w, h, H.HVX_DF_S16) if want_mag else None
    g = PG.edge_graph(ctx, inp, ph, mk, border=border, cval=cval, mag_out=mg, fusion=fusion,
                      rounding=rounding, thr=thr)
    kinds = PG.kernel_kinds(g)
    H.hvxProcessGraph(g)
    res = (PG.download(ph), PG.download(mk), PG.download(mg) if want_mag else None)
    H.hvxReleaseGraph(g)
    return res, kinds


@pytest.mark.parametrize("w,h", SIZES + [(385, 361), (1920, 1080)])
@pytest.mark.parametrize("border", BORDERS)
def test_edge_graph_fused_and_plain(ctx, w, h, border):
    img = synth.rects_noise(w, h, seed=2)
    ref_ph, ref_mk, ref_mg = O.edge_graph(img, B_ORC[border], 31, O.ROUND_ZERO, 100, want_mag=True)
    (ph, mk, mg), kinds = run_edge(ctx, img, border, 31, True, True)
    assert kinds == ["fused_edge_tma"]
    np.testing.assert_array_equal(mk, ref_mk)
    np.testing.assert_array_equal(mg, ref_mg)
    assert circ_diff(ph, ref_ph).max() <= 1
    np.testing.assert_array_equal(ph, ref_ph)  # exact in practice (boundary re-decision)
    (ph2, mk2, mg2), kinds2 = run_edge(ctx, img, border, 31, False, True)
    assert len(kinds2) == 5
    np.testing.assert_array_equal(ph2, ph)
    np.testing.assert_array_equal(mk2, mk)
    np.testing.assert_array_equal(mg2, mg)


# the fused kernel's specialisations (mask + phase, mask only, phase only) on
# sizes with several ragged 128 x 120 tiles in both directions
@pytest.mark.parametrize("w,h", [(131, 37), (385, 361), (1000, 250)])
@pytest.mark.parametrize("border", BORDERS)
def test_edge_output_modes(ctx, w, h, border):
    img = synth.rects_noise(w, h, seed=5 + w)
    ref_ph, ref_mk = O.edge_graph(img, B_ORC[border], 9, O.ROUND_ZERO, 100)
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    for want_ph, want_mk in ((True, True), (False, True), (True, False)):
        ph = PG.empty(ctx, w, h, H.HVX_DF_U8) if want_ph else None
        mk = PG.empty(ctx, w, h, H.HVX_DF_U8) if want_mk else None
        g = PG.edge_graph(ctx, inp, ph, mk, border=border, cval=9)
        assert PG.kernel_kinds(g) == ["fused_edge_tma"]
        H.hvxProcessGraph(g)
        if want_ph:
            np.testing.assert_array_equal(PG.download(ph), ref_ph)
        if want_mk:
            np.testing.assert_array_equal(PG.download(mk), ref_mk)
        H.hvxReleaseGraph(g)


@pytest.mark.parametrize("thr", [-5, 0, 1, 100, 1443, 40000])
def test_edge_threshold_strength_reduction(ctx, thr):
    img = synth.rects_noise(200, 90, seed=8)
    ref_ph, ref_mk = O.edge_graph(img, O.BORDER_REPLICATE, 0, O.ROUND_ZERO, thr)
    (ph, mk, _), kinds = run_edge(ctx, img, H.HVX_BORDER_REPLICATE, thr=thr)
    assert kinds == ["fused_edge_tma"]
    np.testing.assert_array_equal(mk, ref_mk)


def test_edge_rounding_nearest(ctx):
    img = synth.rects_noise(300, 77, seed=9)
    ref_ph, ref_mk = O.edge_graph(img, O.BORDER_REPLICATE, 0, O.ROUND_NEAREST, 100)
    (ph, mk, _), _ = run_edge(ctx, img, H.HVX_BORDER_REPLICATE, rounding=1)
    np.testing.assert_array_equal(ph, ref_ph)
    np.testing.assert_array_equal(mk, ref_mk)


def test_edge_mixed_borders_via_oracle_graph(ctx):
    """Gaussian UNDEFINED then Sobel REPLICATE: the Sobel reads the Gaussian's
    zeroed invalid border, as the node-by-node definition says."""
    w, h = 150, 40
    img = synth.uniform_u8(w, h, 12)
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    ph = PG.empty(ctx, w, h, H.HVX_DF_U8)
    mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
    g = PG.edge_graph(ctx, inp, ph, mk, border=H.HVX_BORDER_UNDEFINED,
                      sobel_border=H.HVX_BORDER_REPLICATE)
    assert PG.kernel_kinds(g) == ["fused_edge_tma"]
    H.hvxProcessGraph(g)
    og = OG.GraphDesc()
    og.image("in", w, h, "U8")
    og.image("ph", w, h, "U8")
    og.image("mk", w, h, "U8")
    for v in ("G", "gx", "gy", "m"):
        og.virtual(v)
    og.node("gaussian3x3", ["in"], ["G"], border="undefined")
    og.node("sobel3x3", ["G"], ["gx", "gy"], border="replicate")
    og.node("magnitude", ["gx", "gy"], ["m"])
    og.node("threshold", ["m"], ["mk"], value=100)
    og.node("phase", ["gx", "gy"], ["ph"])
    ref = OG.run(og, {"in": img})
    np.testing.assert_array_equal(PG.download(mk), ref["mk"].data)
    np.testing.assert_array_equal(PG.download(ph), ref["ph"].data)


# --- point operators, exhaustively -------------------------------------------------

def test_magnitude_phase_exhaustive(ctx):
    v = np.arange(-1020, 1021, dtype=np.int16)
    gx, gy = [np.ascontiguousarray(a) for a in np.meshgrid(v, v)]
    n = gx.shape[0]
    a = PG.upload(ctx, gx, H.HVX_DF_S16)
    b = PG.upload(ctx, gy, H.HVX_DF_S16)
    m = PG.empty(ctx, n, n, H.HVX_DF_S16)
    p = PG.empty(ctx, n, n, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    H.hvxMagnitudeNode(g, a, b, m)
    H.hvxPhaseNode(g, a, b, p)
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    np.testing.assert_array_equal(PG.download(m), O.magnitude(gx, gy).data)
    ref = O.phase(gx, gy).data
    got = PG.download(p)
    assert circ_diff(got, ref).max() <= 1
    assert int((got != ref).sum()) == 0


@pytest.mark.parametrize("thr", [0, 1, 100, 1000, 1442, 1443])
def test_edge_kernel_point_ops_exhaustive(ctx, thr):
    """The fused edge kernel's own Phase (octant guess, exact binary32 test,
    paired byte select) and Magnitude -> Threshold (packed fma, sign bytes)
    over every gradient pair (gx, gy) in [-1020, 1020]^2, bit-exact with the
    oracle's Phase and Threshold(Magnitude) definitions."""
    ph, mk = H.hvxSelfTestEdgePoint(ctx, 1020, thr * thr + thr)
    v = np.arange(-1020, 1021, dtype=np.int16)
    gx, gy = [np.ascontiguousarray(a) for a in np.meshgrid(v, v)]  # [gy, gx]
    np.testing.assert_array_equal(mk, O.threshold(O.magnitude(gx, gy), thr).data)
    if thr == 100:
        np.testing.assert_array_equal(ph, O.phase(gx, gy).data)


def test_threshold_all_s16_and_range(ctx):
    v = np.arange(-32768, 32768, dtype=np.int32).astype(np.int16).reshape(256, 256)
    a = PG.upload(ctx, v, H.HVX_DF_S16)
    o1 = PG.empty(ctx, 256, 256, H.HVX_DF_U8)
    o2 = PG.empty(ctx, 256, 256, H.HVX_DF_U8)
    g = H.hvxCreateGraph(ctx)
    H.hvxThresholdNode(g, a, H.HVX_THRESHOLD_BINARY, 100, 0, 255, 0, o1)
    H.hvxThresholdNode(g, a, H.HVX_THRESHOLD_RANGE, -7, 300, 9, 1, o2)
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    np.testing.assert_array_equal(PG.download(o1), O.threshold(v, 100).data)
    np.testing.assert_array_equal(PG.download(o2), O.threshold_range(v, -7, 300, 9, 1).data)


@pytest.mark.parametrize("op", ["add", "subtract", "absdiff"])
@pytest.mark.parametrize("policy", [H.HVX_POLICY_WRAP, H.HVX_POLICY_SATURATE])
@pytest.mark.parametrize("fmts", [("U8", "U8", "U8"), ("U8", "U8", "S16"), ("S16", "U8", "S16")])
def test_arith(ctx, op, policy, fmts):
    w, h = 133, 21
    npf = {"U8": np.uint8, "S16": np.int16}
    a = synth.randint(3, 0, w * h, -40000 if fmts[0] == "S16" else 0,
                      40000 if fmts[0] == "S16" else 255)
    a = np.clip(a, -32768, 32767).astype(npf[fmts[0]]).reshape(h, w)
    b = synth.uniform_u8(w, h, 4)
    A = PG.upload(ctx, a, getattr(H, "HVX_DF_" + fmts[0]))
    B = PG.upload(ctx, b, H.HVX_DF_U8)
    C = PG.empty(ctx, w, h, getattr(H, "HVX_DF_" + fmts[2]))
    g = H.hvxCreateGraph(ctx)
    if op == "add":
        H.hvxAddNode(g, A, B, policy, C)
    elif op == "subtract":
        H.hvxSubtractNode(g, A, B, policy, C)
    else:
        H.hvxAbsDiffNode(g, A, B, C)
        policy = H.HVX_POLICY_SATURATE
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    code = {"add": O.ARITH_ADD, "subtract": O.ARITH_SUB, "absdiff": O.ARITH_ABSDIFF}[op]
    ref = O.arith(a, b, npf[fmts[2]], code, policy == H.HVX_POLICY_SATURATE)
    np.testing.assert_array_equal(PG.download(C), ref.data)


def test_channel_extract_all_channels(ctx):
    w, h = 98, 13
    yuv = synth.uyvy(w, h, 5)
    src = PG.upload(ctx, yuv, H.HVX_DF_UYVY)
    outs = [PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w // 2, h, H.HVX_DF_U8),
            PG.empty(ctx, w // 2, h, H.HVX_DF_U8)]
    g = H.hvxCreateGraph(ctx)
    for ch, o in enumerate(outs):
        H.hvxChannelExtractNode(g, src, ch, o)
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    for ch, o in enumerate(outs):
        np.testing.assert_array_equal(PG.download(o), O.channel_extract_uyvy(yuv, ch).data)


# --- local operators through the staged-tile executor -------------------------------

@pytest.mark.parametrize("border", BORDERS)
@pytest.mark.parametrize("w,h", [(1, 1), (5, 3), (70, 17), (129, 33)])
def test_box_convolve_sobel_plain(ctx, border, w, h):
    img = synth.uniform_u8(w, h, 6)
    lap = np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], np.int32)
    g5 = synth.randint(9, 0, 25, -9, 9).astype(np.int32).reshape(5, 5)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    box = PG.empty(ctx, w, h, H.HVX_DF_U8)
    c3 = PG.empty(ctx, w, h, H.HVX_DF_S16)
    c5 = PG.empty(ctx, w, h, H.HVX_DF_S16)
    gx = PG.empty(ctx, w, h, H.HVX_DF_S16)
    gy = PG.empty(ctx, w, h, H.HVX_DF_S16)
    g = H.hvxCreateGraph(ctx)
    for n in (H.hvxBox3x3Node(g, src, box), H.hvxConvolveNode(g, src, lap.ravel(), 3, 3, 0, c3),
              H.hvxConvolveNode(g, src, g5.ravel(), 5, 5, 2, c5), H.hvxSobel3x3Node(g, src, gx, gy)):
        H.hvxSetNodeBorder(n, border, 200)
    H.hvxSetGraphFusion(g, False)
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    b = B_ORC[border]
    np.testing.assert_array_equal(PG.download(box), O.box3x3(img, b, 200).data)
    np.testing.assert_array_equal(PG.download(c3), O.convolve(img, lap, 0, b, 200).data)
    np.testing.assert_array_equal(PG.download(c5), O.convolve(img, g5, 2, b, 200).data)
    rx, ry = O.sobel3x3(img, b, 200)
    np.testing.assert_array_equal(PG.download(gx), rx.data)
    np.testing.assert_array_equal(PG.download(gy), ry.data)


# --- Harris graph ------------------------------------------------------------------

def run_harris(ctx, img, border, fusion=True, thr=1e6, cval=0):
    h, w = img.shape
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
    rs = PG.empty(ctx, w, h, H.HVX_DF_F32)
    g = PG.harris_graph(ctx, inp, mk, rs, border=border, fusion=fusion, thr=thr, cval=cval)
    kinds = PG.kernel_kinds(g)
    H.hvxProcessGraph(g)
    out = PG.download(mk), PG.download(rs)
    H.hvxReleaseGraph(g)
    return out, kinds


def harris_oracle(img, border, thr=1e6, cval=0):
    og = OG.GraphDesc()
    h, w = img.shape
    og.image("in", w, h, "U8")
    og.image("mk", w, h, "U8")
    og.image("r", w, h, "F32")
    for v in ("gx", "gy", "xx", "yy", "xy", "sxx", "syy", "sxy"):
        og.virtual(v)
    bn = {O.BORDER_UNDEFINED: "undefined", O.BORDER_REPLICATE: "replicate",
          O.BORDER_CONSTANT: "constant"}[border]
    og.node("sobel3x3", ["in"], ["gx", "gy"], border=bn, cval=cval)
    og.node("mul", ["gx", "gx"], ["xx"])
    og.node("mul", ["gy", "gy"], ["yy"])
    og.node("mul", ["gx", "gy"], ["xy"])
    for a, b in (("xx", "sxx"), ("yy", "syy"), ("xy", "sxy")):
        og.node("window_sum", [a], [b], kw=5, kh=5, border=bn, cval=cval)
    og.node("harris_response", ["sxx", "syy", "sxy"], ["r"], kn=1, kd=25)
    og.node("threshold", ["r"], ["mk"], value=thr)
    res = OG.run(og, {"in": img})
    return res["mk"].data, res["r"].data


def check_resp(got, ref):
    tol = 1e-5 * np.maximum(np.abs(ref.astype(np.float64)), 1.0)
    assert (np.abs(got.astype(np.float64) - ref.astype(np.float64)) <= tol).all()
    np.testing.assert_array_equal(got, ref)  # single rounding of the exact value


TOMASI_THR = 4.0e4


def tomasi_oracle(img, border, cval=0):
    og = OG.GraphDesc()
    h, w = img.shape
    og.image("in", w, h, "U8")
    og.image("r", w, h, "F32")
    for v in ("gx", "gy", "xx", "yy", "xy", "sxx", "syy", "sxy"):
        og.virtual(v)
    bn = {O.BORDER_UNDEFINED: "undefined", O.BORDER_REPLICATE: "replicate",
          O.BORDER_CONSTANT: "constant"}[border]
    og.node("sobel3x3", ["in"], ["gx", "gy"], border=bn, cval=cval)
    og.node("mul", ["gx", "gx"], ["xx"])
    og.node("mul", ["gy", "gy"], ["yy"])
    og.node("mul", ["gx", "gy"], ["xy"])
    for a, b in (("xx", "sxx"), ("yy", "syy"), ("xy", "sxy")):
        og.node("window_sum", [a], [b], kw=5, kh=5, border=bn, cval=cval)
    og.node("tomasi_response", ["sxx", "syy", "sxy"], ["r"])
    return OG.run(og, {"in": img})["r"].data


def run_tomasi(ctx, img, border, fusion=True, codegen=H.HVX_CODEGEN_AUTO, cval=0):
    h, w = img.shape
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
    rs = PG.empty(ctx, w, h, H.HVX_DF_F32)
    g = PG.harris_graph(ctx, inp, mk, rs, border=border, fusion=fusion, thr=TOMASI_THR,
                        cval=cval, tomasi=True, verify=False)
    H.hvxSetGraphCodegen(g, codegen)
    H.hvxVerifyGraph(g)
    kinds = PG.kernel_kinds(g)
    H.hvxProcessGraph(g)
    out = PG.download(mk), PG.download(rs)
    H.hvxReleaseGraph(g)
    return out, kinds


@pytest.mark.parametrize("w,h", [(1, 1), (7, 7), (97, 45), (300, 200), (385, 361)])
@pytest.mark.parametrize("border", BORDERS)
def test_tomasi_on_the_corner_kernel(ctx, w, h, border):
    # the Shi-Tomasi group runs on the hand-written corner kernels; its
    # binary32 response is the point operator's, bit for bit, so the fused,
    # generated and unfused forms agree exactly, and the oracle's singly
    # rounded eigenvalue within a few units in the last place
    img = synth.rects_noise(w, h, seed=5)
    ref = tomasi_oracle(img, B_ORC[border], cval=5).astype(np.float64)
    (mk, r), kinds = run_tomasi(ctx, img, border, cval=5)
    assert kinds == ["fused_harris_tma"]
    assert (np.abs(r - ref) <= 2e-6 * np.abs(ref)).all()
    near = np.abs(ref - TOMASI_THR) <= 1e-5 * TOMASI_THR
    np.testing.assert_array_equal((mk == 255)[~near], (ref > TOMASI_THR)[~near])
    # the mask is the kernel's own binary32 response compared with the
    # threshold, everywhere (near the threshold too)
    np.testing.assert_array_equal(mk == 255, r > np.float32(TOMASI_THR))
    # without the exported response the UNDEFINED kernel decides from a cheaper
    # estimate where that is safe: the same mask
    h_, w_ = img.shape
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    mk1 = PG.empty(ctx, w_, h_, H.HVX_DF_U8)
    g1 = PG.harris_graph(ctx, inp, mk1, None, border=border, thr=TOMASI_THR, cval=5, tomasi=True)
    assert PG.kernel_kinds(g1) == ["fused_harris_tma"]
    H.hvxProcessGraph(g1)
    np.testing.assert_array_equal(PG.download(mk1), mk)
    H.hvxReleaseGraph(g1)
    (mk2, r2), kinds2 = run_tomasi(ctx, img, border, codegen=H.HVX_CODEGEN_ONLY, cval=5)
    assert kinds2 == ["staged_tile"]
    (mk3, r3), kinds3 = run_tomasi(ctx, img, border, fusion=False, cval=5)
    assert len(kinds3) == 9
    for m, x in ((mk2, r2), (mk3, r3)):
        np.testing.assert_array_equal(m, mk)
        np.testing.assert_array_equal(x.view(np.uint32), r.view(np.uint32))


@pytest.mark.parametrize("w,h", [(1, 1), (7, 7), (64, 32), (97, 45), (300, 200), (385, 361)])
@pytest.mark.parametrize("border", BORDERS)
def test_harris_fused_and_plain(ctx, w, h, border):
    img = synth.rects_noise(w, h, seed=3)
    ref_mk, ref_r = harris_oracle(img, B_ORC[border], cval=5)
    (mk, r), kinds = run_harris(ctx, img, border, cval=5)
    assert kinds == ["fused_harris_tma"]
    np.testing.assert_array_equal(mk, ref_mk)
    check_resp(r, ref_r)
    (mk2, r2), kinds2 = run_harris(ctx, img, border, fusion=False, cval=5)
    assert len(kinds2) == 9
    np.testing.assert_array_equal(mk2, ref_mk)
    check_resp(r2, ref_r)


def test_harris_full_size_4096x2160(ctx):
    img = synth.rects_noise(4096, 2160, seed=3)
    ref_mk, ref_r = O.harris_graph(img, O.BORDER_UNDEFINED, 1, 25, 1e6)
    (mk, r), kinds = run_harris(ctx, img, H.HVX_BORDER_UNDEFINED)
    assert kinds == ["fused_harris_tma"]
    np.testing.assert_array_equal(mk, ref_mk)
    check_resp(r, ref_r)


def test_tomasi_full_size_4096x2160(ctx):
    # the Shi-Tomasi group at full size on the corner kernel, with the
    # response exported and (second run) without it, where the threshold is
    # decided from the estimate: both masks equal, and equal to the oracle's
    # eigenvalue test away from the threshold
    img = synth.rects_noise(4096, 2160, seed=9)
    ref = tomasi_oracle(img, O.BORDER_UNDEFINED).astype(np.float64)
    (mk, r), kinds = run_tomasi(ctx, img, H.HVX_BORDER_UNDEFINED)
    assert kinds == ["fused_harris_tma"]
    assert (np.abs(r - ref) <= 2e-6 * np.abs(ref)).all()
    near = np.abs(ref - TOMASI_THR) <= 1e-5 * TOMASI_THR
    np.testing.assert_array_equal((mk == 255)[~near], (ref > TOMASI_THR)[~near])
    np.testing.assert_array_equal(mk == 255, r > np.float32(TOMASI_THR))
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    mk1 = PG.empty(ctx, 4096, 2160, H.HVX_DF_U8)
    g = PG.harris_graph(ctx, inp, mk1, None, thr=TOMASI_THR, tomasi=True)
    H.hvxProcessGraph(g)
    np.testing.assert_array_equal(PG.download(mk1), mk)
    H.hvxReleaseGraph(g)


@pytest.mark.parametrize("w,h", [(1000, 700), (129, 241)])
def test_harris_mask_only_undefined(ctx, w, h):
    # the BORDER_UNDEFINED kernel without the response export (the benchmark's
    # form), on ragged 128 x 120 tiles, and with a non-default k = 3/50
    img = synth.rects_noise(w, h, seed=11)
    for kn, kd, thr in ((1, 25, 1e6), (3, 50, 2.5e7)):
        ref_mk, _ = O.harris_graph(img, O.BORDER_UNDEFINED, kn, kd, thr)
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
        g = PG.harris_graph(ctx, inp, mk, None, kn=kn, kd=kd, thr=thr)
        assert PG.kernel_kinds(g) == ["fused_harris_tma"]
        H.hvxProcessGraph(g)
        np.testing.assert_array_equal(PG.download(mk), ref_mk)
        assert ref_mk.any() and not ref_mk.all()
        H.hvxReleaseGraph(g)


def test_harris_clean_corners(ctx):
    img = np.zeros((60, 80), np.uint8)
    img[15:45, 20:60] = 200
    ref_mk, ref_r = O.harris_graph(img, O.BORDER_UNDEFINED, 1, 25, 1e6)
    (mk, r), _ = run_harris(ctx, img, H.HVX_BORDER_UNDEFINED)
    np.testing.assert_array_equal(mk, ref_mk)
    assert mk.any()
    check_resp(r, ref_r)


# --- arbitrary fused groups (staged-tile executor) ----------------------------------

def test_listing1_graph_from_uyvy(ctx):
    w, h = 200, 61
    yuv = synth.uyvy(w, h, 7)
    src = PG.upload(ctx, yuv, H.HVX_DF_UYVY)
    out = PG.empty(ctx, w, h, H.HVX_DF_U8)
    for fusion in (True, False):
        g = H.hvxCreateGraph(ctx)
        v = [H.hvxCreateVirtualImage(g) for _ in range(5)]
        H.hvxChannelExtractNode(g, src, H.HVX_CHANNEL_Y, v[0])
        H.hvxGaussian3x3Node(g, v[0], v[1])
        sob = H.hvxSobel3x3Node(g, v[1], v[2], v[3])
        H.hvxMagnitudeNode(g, v[3], v[3], v[4])
        H.hvxThresholdNode(g, v[4], H.HVX_THRESHOLD_BINARY, 100, 0, 255, 0, out)
        H.hvxSetGraphFusion(g, fusion)
        H.hvxVerifyGraph(g)
        assert H.hvxQueryNode(sob, H.HVX_NODE_LIVE_OUTPUTS) == 0b10
        H.hvxProcessGraph(g)
        Y = O.channel_extract_uyvy(yuv, 0)
        _, gy = O.sobel3x3(O.gaussian3x3(Y))
        ref = O.threshold(O.magnitude(gy, gy), 100).data
        np.testing.assert_array_equal(PG.download(out), ref)
        H.hvxReleaseGraph(g)


def _random_graph(seed, w, h):
    """A random DAG of Table 2 nodes, as (ABI graph builder, oracle GraphDesc)."""
    u = synth.uniform01(seed, 50, 200)
    k = [0]

    def nxt():
        k[0] += 1
        return u[k[0]]

    og = OG.GraphDesc()
    og.image("in", w, h, "U8")
    u8, s16, outs = ["in"], [], []
    steps = []
    borders = ["replicate", "constant", "undefined"]
    for i in range(3 + int(nxt() * 6)):
        c = int(nxt() * 6)
        name = f"d{i}"
        b = borders[int(nxt() * 3)]
        if c == 0:
            steps.append(("gaussian3x3", [u8[int(nxt() * len(u8))]], [name], b))
            u8.append(name)
        elif c == 1:
            steps.append(("box3x3", [u8[int(nxt() * len(u8))]], [name], b))
            u8.append(name)
        elif c == 2 or not s16:
            gy = f"e{i}"
            steps.append(("sobel3x3", [u8[int(nxt() * len(u8))]], [name, gy], b))
            s16 += [name, gy]
        elif c == 3:
            steps.append(("magnitude", [s16[int(nxt() * len(s16))], s16[int(nxt() * len(s16))]],
                          [name], b))
            s16.append(name)
        elif c == 4:
            steps.append(("phase", [s16[int(nxt() * len(s16))], s16[int(nxt() * len(s16))]],
                          [name], b))
            u8.append(name)
        else:
            steps.append(("threshold", [s16[int(nxt() * len(s16))]], [name], b))
            u8.append(name)
    produced = [o for s in steps for o in s[2]]
    # the last two produced images and one random other are outputs
    for o in set(produced[-2:] + [produced[int(nxt() * len(produced))]]):
        outs.append(o)
    fmt = {}
    for kind, ins, os_, b in steps:
        for o in os_:
            fmt[o] = "S16" if kind in ("sobel3x3", "magnitude") else "U8"
    for o in produced:
        if o in outs:
            og.image(o, w, h, fmt[o])
        else:
            og.virtual(o)
    for kind, ins, os_, b in steps:
        og.node(kind, ins, os_, border=b, cval=17, **({"value": 60} if kind == "threshold" else {}))
    return steps, outs, fmt, og


@pytest.mark.parametrize("seed", range(12))
def test_random_fused_graphs(ctx, seed):
    w, h = 150, 45
    img = synth.uniform_u8(w, h, 100 + seed)
    steps, outs, fmt, og = _random_graph(seed, w, h)
    ref = OG.run(og, {"in": img})
    for fusion in (True, False):
        g = H.hvxCreateGraph(ctx)
        imgs = {"in": PG.upload(ctx, img, H.HVX_DF_U8)}
        for o in fmt:
            imgs[o] = (PG.empty(ctx, w, h, getattr(H, "HVX_DF_" + fmt[o])) if o in outs
                       else H.hvxCreateVirtualImage(g))
        bm = {"replicate": H.HVX_BORDER_REPLICATE, "constant": H.HVX_BORDER_CONSTANT,
              "undefined": H.HVX_BORDER_UNDEFINED}
        for kind, ins, os_, b in steps:
            I = [imgs[x] for x in ins]
            Ot = [imgs[x] for x in os_]
            if kind == "gaussian3x3":
                n = H.hvxGaussian3x3Node(g, I[0], Ot[0])
            elif kind == "box3x3":
                n = H.hvxBox3x3Node(g, I[0], Ot[0])
            elif kind == "sobel3x3":
                n = H.hvxSobel3x3Node(g, I[0], Ot[0], Ot[1])
            elif kind == "magnitude":
                n = H.hvxMagnitudeNode(g, I[0], I[1], Ot[0])
            elif kind == "phase":
                n = H.hvxPhaseNode(g, I[0], I[1], Ot[0])
            else:
                n = H.hvxThresholdNode(g, I[0], H.HVX_THRESHOLD_BINARY, 60, 0, 255, 0, Ot[0])
            H.hvxSetNodeBorder(n, bm[b], 17)
        H.hvxSetGraphFusion(g, fusion)
        H.hvxVerifyGraph(g)
        H.hvxProcessGraph(g)
        for o in outs:
            if o in ref:
                np.testing.assert_array_equal(PG.download(imgs[o]), ref[o].data,
                                              err_msg=f"{o} fusion={fusion}")
        H.hvxReleaseGraph(g)
