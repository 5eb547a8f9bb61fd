"""CPU tests of the C ABI: the library builds and exports every declared entry
point, and the host-side graph logic (verification, Algorithm 1, valid
regions, fusion planning) behaves as the oracle's graph layer says, using a
plan-only context (no device)."""
import os
import re

import pytest

import oracle.graph as OG
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hvx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hvx[A-Z]\w*)\s*\(", src)))


def test_library_exports_every_declared_function():
    L = H.lib()
    names = declared_functions()
    assert len(names) >= 40
    for n in names:
        assert hasattr(L, n), n
        assert n in H._SIGS, f"binding lacks {n}"


@pytest.fixture
def pctx():
    c = H.hvxCreateContextEx(H.HVX_CONTEXT_PLAN_ONLY)
    yield c
    H.hvxReleaseContext(c)


def test_edge_graph_plans_one_fused_kernel(pctx):
    inp = H.hvxCreateImage(pctx, 1920, 1080, H.HVX_DF_U8)
    ph = H.hvxCreateImage(pctx, 1920, 1080, H.HVX_DF_U8)
    mk = H.hvxCreateImage(pctx, 1920, 1080, H.HVX_DF_U8)
    g = PG.edge_graph(pctx, inp, ph, mk)
    assert PG.kernel_kinds(g) == ["fused_edge_tma"]
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_LAUNCHES) == 1
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_INTERMEDIATE_BYTES) == 0
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_EXTERNAL_BYTES) == 3 * 1920 * 1080
    with pytest.raises(H.HvxError) as e:
        H.hvxProcessGraph(g)
    assert e.value.status == H.HVX_ERROR_NOT_SUPPORTED
    # the same graph unfused: one launch per node, every virtual image in memory
    g2 = PG.edge_graph(pctx, inp, ph, mk, fusion=False)
    kinds = PG.kernel_kinds(g2)
    assert kinds == ["gaussian3x3_tma", "staged_tile", "plain_point", "plain_point",
                     "plain_point"]
    # G (1 B) + gx, gy (2 B each) + magnitude (2 B), pitches padded to 128 B
    assert H.hvxQueryGraph(g2, H.HVX_GRAPH_INTERMEDIATE_BYTES) == 1080 * (1920 + 3 * 3840)


def test_harris_graph_plans_one_fused_kernel(pctx):
    inp = H.hvxCreateImage(pctx, 4096, 2160, H.HVX_DF_U8)
    mk = H.hvxCreateImage(pctx, 4096, 2160, H.HVX_DF_U8)
    g = PG.harris_graph(pctx, inp, mk)
    assert PG.kernel_kinds(g) == ["fused_harris_tma"]
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_ALIVE_OPS) == 10
    assert H.hvxGetValidRegion(mk) == (3, 3, 4093, 2157)
    g2 = PG.harris_graph(pctx, inp, mk, fusion=False)
    assert len(PG.kernel_kinds(g2)) == 9


def _build_both(pctx, spec_nodes, images):
    """The same graph through the C ABI and through the oracle's graph layer."""
    g = H.hvxCreateGraph(pctx)
    og = OG.GraphDesc()
    handles = {}
    for name, (virtual, w, h, fmt) in images.items():
        if virtual:
            handles[name] = H.hvxCreateVirtualImage(g)
            og.virtual(name)
        else:
            handles[name] = H.hvxCreateImage(pctx, w, h, getattr(H, "HVX_DF_" + fmt))
            og.image(name, w, h, fmt)
    nodes = []
    for kind, ins, outs in spec_nodes:
        hi = [handles[i] for i in ins]
        ho = [handles[o] if o else None for o in outs]
        if kind == "gaussian3x3":
            n = H.hvxGaussian3x3Node(g, hi[0], ho[0])
        elif kind == "box3x3":
            n = H.hvxBox3x3Node(g, hi[0], ho[0])
        elif kind == "sobel3x3":
            n = H.hvxSobel3x3Node(g, hi[0], ho[0], ho[1])
        elif kind == "magnitude":
            n = H.hvxMagnitudeNode(g, hi[0], hi[1], ho[0])
        elif kind == "phase":
            n = H.hvxPhaseNode(g, hi[0], hi[1], ho[0])
        elif kind == "threshold":
            n = H.hvxThresholdNode(g, hi[0], H.HVX_THRESHOLD_BINARY, 100, 0, 255, 0, ho[0])
        elif kind == "channel_extract":
            n = H.hvxChannelExtractNode(g, hi[0], 0, ho[0])
        else:
            raise ValueError(kind)
        nodes.append(n)
        og.node(kind, ins, outs, **({"value": 100} if kind == "threshold" else {}))
    return g, og, nodes, handles


def test_listing1_dead_sobel_output(pctx):
    import json
    spec = json.load(open(os.path.join(ROOT, "tests", "golden", "listing1_edge_graph.json")))
    images = {im["name"]: (im["virtual"], im.get("w", 0), im.get("h", 0), im.get("fmt", ""))
              for im in spec["images"]}
    nodes = [(n["kind"], n["ins"], n["outs"]) for n in spec["nodes"]]
    g, og, hn, _ = _build_both(pctx, nodes, images)
    H.hvxVerifyGraph(g)
    # Sobel's gx output (bit 0) is dead, gy (bit 1) alive
    assert H.hvxQueryNode(hn[2], H.HVX_NODE_LIVE_OUTPUTS) == 0b10
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_OPS) == 6
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_ALIVE_OPS) == 5
    alive, _ = OG.eliminate_dead(og, OG.verify(og))
    assert len(alive) == 5
    # all five live ops fuse into one staged-tile kernel
    assert PG.kernel_kinds(g) == ["staged_tile"]


def _alive_names_c(hn, spec_nodes):
    names = set()
    for i, (kind, ins, outs) in enumerate(spec_nodes):
        m = H.hvxQueryNode(hn[i], H.HVX_NODE_LIVE_OUTPUTS)
        if kind == "sobel3x3":
            if m & 1:
                names.add(f"n{i}.gx")
            if m & 2:
                names.add(f"n{i}.gy")
        elif m & 1:
            names.add(f"n{i}")
    return names


def test_dead_code_elimination_matches_oracle_on_random_graphs(pctx):
    from paper_2008_11476_gb300 import synth
    for seed in range(40):
        u = synth.uniform01(seed, 40, 400)
        k = 0
        images = {"in0": (False, 16, 8, "U8")}
        pool_u8 = ["in0"]
        pool_s16 = []
        nodes = []
        for i in range(2 + int(u[k] * 7)):
            k += 1
            choice = int(u[k] * 5)
            k += 1
            virt = u[k] < 0.65
            k += 1
            if choice <= 1 or not pool_s16:
                src = pool_u8[int(u[k] * len(pool_u8))]
                k += 1
                if choice == 0 or pool_s16 == [] and u[k] < 0.5:
                    name = f"u{i}"
                    images[name] = (virt, 16, 8, "U8")
                    nodes.append(("gaussian3x3", [src], [name]))
                    pool_u8.append(name)
                else:
                    gx, gy = f"gx{i}", f"gy{i}"
                    images[gx] = (virt, 16, 8, "S16")
                    images[gy] = (u[k] < 0.7, 16, 8, "S16")
                    nodes.append(("sobel3x3", [src], [gx, gy]))
                    pool_s16 += [gx, gy]
                k += 1
            else:
                a = pool_s16[int(u[k] * len(pool_s16))]
                k += 1
                b = pool_s16[int(u[k] * len(pool_s16))]
                k += 1
                name = f"m{i}"
                if choice == 2:
                    images[name] = (virt, 16, 8, "S16")
                    nodes.append(("magnitude", [a, b], [name]))
                    pool_s16.append(name)
                else:
                    images[name] = (virt, 16, 8, "U8")
                    nodes.append(("phase", [a, b], [name]))
                    pool_u8.append(name)
        g, og, hn, _ = _build_both(pctx, nodes, images)
        H.hvxVerifyGraph(g)
        alive, _ = OG.eliminate_dead(og, OG.verify(og))
        assert _alive_names_c(hn, nodes) == {op.name for op in alive}, seed
        H.hvxReleaseGraph(g)


def test_verify_rejects_bad_graphs(pctx):
    a = H.hvxCreateImage(pctx, 8, 8, H.HVX_DF_U8)
    b = H.hvxCreateImage(pctx, 8, 8, H.HVX_DF_U8)
    s16 = H.hvxCreateImage(pctx, 8, 8, H.HVX_DF_S16)
    # cycle through two virtual images
    g = H.hvxCreateGraph(pctx)
    v1 = H.hvxCreateVirtualImage(g)
    v2 = H.hvxCreateVirtualImage(g)
    H.hvxGaussian3x3Node(g, v1, v2)
    H.hvxGaussian3x3Node(g, v2, v1)
    H.hvxBox3x3Node(g, v2, b)
    with pytest.raises(H.HvxError) as e:
        H.hvxVerifyGraph(g)
    assert e.value.status == H.HVX_ERROR_INVALID_GRAPH
    # S16 into a U8-only input
    g = H.hvxCreateGraph(pctx)
    H.hvxGaussian3x3Node(g, s16, b)
    with pytest.raises(H.HvxError) as e:
        H.hvxVerifyGraph(g)
    assert e.value.status == H.HVX_ERROR_INVALID_FORMAT
    # virtual image read but never written
    g = H.hvxCreateGraph(pctx)
    v = H.hvxCreateVirtualImage(g)
    H.hvxGaussian3x3Node(g, v, b)
    with pytest.raises(H.HvxError) as e:
        H.hvxVerifyGraph(g)
    assert e.value.status == H.HVX_ERROR_INVALID_GRAPH
    # two writers of one image
    g = H.hvxCreateGraph(pctx)
    H.hvxGaussian3x3Node(g, a, b)
    H.hvxBox3x3Node(g, a, b)
    with pytest.raises(H.HvxError) as e:
        H.hvxVerifyGraph(g)
    assert e.value.status == H.HVX_ERROR_INVALID_GRAPH
    # size mismatch between inputs of a point node
    small = H.hvxCreateImage(pctx, 4, 4, H.HVX_DF_S16)
    g = H.hvxCreateGraph(pctx)
    H.hvxMagnitudeNode(g, s16, small, H.hvxCreateImage(pctx, 8, 8, H.HVX_DF_S16))
    with pytest.raises(H.HvxError) as e:
        H.hvxVerifyGraph(g)
    assert e.value.status == H.HVX_ERROR_INVALID_PARAMETERS
    # a virtual image of another graph
    g1 = H.hvxCreateGraph(pctx)
    foreign = H.hvxCreateVirtualImage(g1)
    g2 = H.hvxCreateGraph(pctx)
    with pytest.raises(H.HvxError) as e:
        H.hvxGaussian3x3Node(g2, a, foreign)
    assert e.value.status == H.HVX_ERROR_INVALID_REFERENCE
    # invalid node parameters are refused at creation
    with pytest.raises(H.HvxError):
        H.hvxLocalNode(g2, H.HVX_LOCAL_SUM, 4, 5, a, b)
    with pytest.raises(H.HvxError):
        H.hvxPointNode(g2, H.HVX_POINT_HARRIS_RESPONSE, [a, a, a], b, (1, 0))


def test_edit_after_verify_requires_reverify(pctx):
    a = H.hvxCreateImage(pctx, 8, 8, H.HVX_DF_U8)
    b = H.hvxCreateImage(pctx, 8, 8, H.HVX_DF_U8)
    g = H.hvxCreateGraph(pctx)
    n = H.hvxGaussian3x3Node(g, a, b)
    H.hvxVerifyGraph(g)
    H.hvxSetNodeBorder(n, H.HVX_BORDER_UNDEFINED, 0)
    with pytest.raises(H.HvxError) as e:
        H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_LAUNCHES)
    assert e.value.status == H.HVX_ERROR_NOT_VERIFIED
    H.hvxVerifyGraph(g)
    assert H.hvxGetValidRegion(b) == (1, 1, 7, 7)


def test_virtual_size_inference_and_declared_mismatch(pctx):
    a = H.hvxCreateImage(pctx, 20, 10, H.HVX_DF_U8)
    b = H.hvxCreateImage(pctx, 20, 10, H.HVX_DF_U8)
    g = H.hvxCreateGraph(pctx)
    v = H.hvxCreateVirtualImage(g)
    H.hvxGaussian3x3Node(g, a, v)
    H.hvxBox3x3Node(g, v, b)
    H.hvxVerifyGraph(g)
    assert H.hvxQueryImage(v) == (20, 10, H.HVX_DF_U8)
    g = H.hvxCreateGraph(pctx)
    v = H.hvxCreateVirtualImage(g, 0, 0, H.HVX_DF_S16)
    H.hvxGaussian3x3Node(g, a, v)
    H.hvxBox3x3Node(g, v, b)
    with pytest.raises(H.HvxError) as e:
        H.hvxVerifyGraph(g)
    assert e.value.status == H.HVX_ERROR_INVALID_FORMAT


def test_fusion_grouping_of_mixed_chain(pctx):
    """Channel extract (U plane: half width) closes its group; local -> local ->
    point chains share one staged-tile kernel."""
    yuv = H.hvxCreateImage(pctx, 64, 16, H.HVX_DF_UYVY)
    out_u = H.hvxCreateImage(pctx, 32, 16, H.HVX_DF_U8)
    out_y = H.hvxCreateImage(pctx, 64, 16, H.HVX_DF_U8)
    g = H.hvxCreateGraph(pctx)
    u = H.hvxCreateVirtualImage(g)
    H.hvxChannelExtractNode(g, yuv, H.HVX_CHANNEL_U, u)
    H.hvxBox3x3Node(g, u, out_u)
    y = H.hvxCreateVirtualImage(g)
    y2 = H.hvxCreateVirtualImage(g)
    H.hvxChannelExtractNode(g, yuv, H.HVX_CHANNEL_Y, y)
    H.hvxGaussian3x3Node(g, y, y2)
    H.hvxBox3x3Node(g, y2, out_y)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) == ["plain_channel_uv", "staged_tile", "staged_tile"]
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_INTERMEDIATE_BYTES) == 16 * 128


def test_morphology_graph_plans_one_staged_group(pctx):
    # closing -> |closing - in| -> threshold, AND the input's median: six
    # Table 2 nodes, one staged-tile launch fused, six unfused
    w, h = 640, 480
    for fusion, n_launch in ((True, 1), (False, 6)):
        src = H.hvxCreateImage(pctx, w, h, H.HVX_DF_U8)
        out = H.hvxCreateImage(pctx, w, h, H.HVX_DF_U8)
        g = H.hvxCreateGraph(pctx)
        d, c, diff, mask, med = (H.hvxCreateVirtualImage(g) for _ in range(5))
        for n in (H.hvxDilate3x3Node(g, src, d), H.hvxErode3x3Node(g, d, c),
                  H.hvxMedian3x3Node(g, src, med)):
            H.hvxSetNodeBorder(n, H.HVX_BORDER_UNDEFINED, 0)
        H.hvxAbsDiffNode(g, c, src, diff)
        H.hvxThresholdNode(g, diff, H.HVX_THRESHOLD_BINARY, 20, 0, 255, 0, mask)
        H.hvxAndNode(g, med, mask, out)
        H.hvxSetGraphFusion(g, fusion)
        H.hvxVerifyGraph(g)
        assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_LAUNCHES) == n_launch
        assert H.hvxGetValidRegion(out) == (2, 2, w - 2, h - 2)
        if fusion:
            assert PG.kernel_kinds(g) == ["staged_tile"]
            assert H.hvxQueryGraph(g, H.HVX_GRAPH_INTERMEDIATE_BYTES) == 0


def test_bitwise_and_morph_reject_wrong_formats(pctx):
    a16 = H.hvxCreateImage(pctx, 32, 8, H.HVX_DF_S16)
    u8 = H.hvxCreateImage(pctx, 32, 8, H.HVX_DF_U8)
    out = H.hvxCreateImage(pctx, 32, 8, H.HVX_DF_U8)
    for build in (lambda g: H.hvxAndNode(g, a16, u8, out), lambda g: H.hvxDilate3x3Node(g, a16, out),
                  lambda g: H.hvxNotNode(g, a16, out)):
        g = H.hvxCreateGraph(pctx)
        build(g)
        with pytest.raises(H.HvxError) as e:
            H.hvxVerifyGraph(g)
        assert e.value.status == H.HVX_ERROR_INVALID_FORMAT


def test_section6_applications_plan(pctx):
    # every application of the paper's evaluation fuses into one launch; the
    # unfused forms launch once per node (Sobel3x3 as one launch)
    from paper_2008_11476_gb300 import apps as A
    unfused = {"Gauss": 1, "Laplacian": 1, "FChain": 3, "SobelX": 1, "EdgFig2": 4, "Sobel": 3,
               "Unsharp": 4, "Harris": 9, "Tomasi": 9}
    # EdgFig2 (Listing 1, gx dead) maps onto the fused edge kernel's
    # Magnitude(gy, gy) mask mode, Sobel and SobelX (no Gaussian) onto its
    # input-row modes,
    # and Gauss (the 5x5 binomial Convolve) onto the binomial kernel
    special = {"Harris": "fused_harris_tma", "Tomasi": "fused_harris_tma",
               "EdgFig2": "fused_edge_tma", "Sobel": "fused_edge_tma",
               "SobelX": "fused_edge_tma", "Gauss": "binomial5x5_tma"}
    for name, build in A.APPS:
        src = H.hvxCreateImage(pctx, 1920, 1080, H.HVX_DF_U8)
        g, _ = build(pctx, src, 1920, 1080, True)
        assert PG.kernel_kinds(g) == [special.get(name, "staged_tile")], name
        # with HVX_CODEGEN_ONLY every application is one generated staged-tile kernel
        H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_ONLY)
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g) == ["staged_tile"], name
        assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == 1, name
        g2, _ = build(pctx, src, 1920, 1080, False)
        assert H.hvxQueryGraph(g2, H.HVX_GRAPH_NUM_LAUNCHES) == unfused[name], name
        if name == "EdgFig2":
            # the horizontal Sobel derivative is the redundant kernel of Fig. 2
            assert (H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_ALIVE_OPS)
                    == H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_OPS) - 1)


def test_mirror_repeat_plan(pctx):
    # MIRROR / REPEAT local nodes take the staged-tile path and never read a
    # fused producer's tile; their outputs keep the full valid region
    src = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)
    for border in (H.HVX_BORDER_MIRROR, H.HVX_BORDER_REPEAT):
        out = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)
        g = H.hvxCreateGraph(pctx)
        H.hvxSetNodeBorder(H.hvxGaussian3x3Node(g, src, out), border, 0)
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g) == ["staged_tile"]
        assert H.hvxGetValidRegion(out) == (0, 0, 640, 480)
        ph = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)
        mk = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)
        g = PG.edge_graph(pctx, src, ph, mk, border=border)
        kinds = PG.kernel_kinds(g)
        assert "fused_edge_tma" not in kinds and len(kinds) == 2  # Sobel reads G from memory
        g = PG.edge_graph(pctx, src, ph, mk, sobel_border=border)
        assert "fused_edge_tma" not in PG.kernel_kinds(g)
        assert H.hvxQueryGraph(g, H.HVX_GRAPH_INTERMEDIATE_BYTES) == 640 * 480
    g = H.hvxCreateGraph(pctx)
    with pytest.raises(H.HvxError):
        H.hvxSetNodeBorder(H.hvxGaussian3x3Node(g, src, H.hvxCreateVirtualImage(g)), 5, 0)


def test_multiply_node_parameters(pctx):
    a = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_U8)
    b = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_S16)
    g = H.hvxCreateGraph(pctx)
    for scale, rnd in ((-1.0, H.HVX_ROUND_TO_ZERO), (1e6, H.HVX_ROUND_TO_ZERO),
                       (float("nan"), H.HVX_ROUND_TO_ZERO), (1.0, H.HVX_ROUND_TO_NEAREST)):
        with pytest.raises(H.HvxError):
            H.hvxMultiplyNode(g, a, b, scale, H.HVX_POLICY_SATURATE, rnd,
                              H.hvxCreateVirtualImage(g))
    out8 = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_U8)
    g = H.hvxCreateGraph(pctx)
    H.hvxMultiplyNode(g, a, b, 0.5, H.HVX_POLICY_SATURATE, H.HVX_ROUND_TO_NEAREST_EVEN, out8)
    with pytest.raises(H.HvxError):  # an S16 input cannot give a U8 product
        H.hvxVerifyGraph(g)
    out16 = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_S16)
    g = H.hvxCreateGraph(pctx)
    H.hvxMultiplyNode(g, a, b, 0.5, H.HVX_POLICY_WRAP, H.HVX_ROUND_TO_ZERO, out16)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) == ["plain_point"]


def test_global_operator_plans(pctx):
    src = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)
    # alone on an external image: its own staged-tile launch
    g = H.hvxCreateGraph(pctx)
    H.hvxMeanStdDevNode(g, src)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) == ["staged_tile"]
    # fused as epilogues: one launch, no image written for them
    g = H.hvxCreateGraph(pctx)
    G, x, y, m = (H.hvxCreateVirtualImage(g) for _ in range(4))
    H.hvxGaussian3x3Node(g, src, G)
    H.hvxSobel3x3Node(g, G, x, y)
    H.hvxMagnitudeNode(g, x, y, m)
    mm = H.hvxMinMaxLocNode(g, m)
    H.hvxHistogramNode(g, G, 8, 0, 256)
    H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_REQUIRE)
    H.hvxVerifyGraph(g)
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_NUM_LAUNCHES) == 1
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_INTERMEDIATE_BYTES) == 0
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == 1
    with pytest.raises(H.HvxError):  # no device: no results
        H.hvxGetNodeResult(mm, H.HvxMinMaxLoc())
    # EqualizeHist runs on its own after its input is in memory
    out = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)
    g = H.hvxCreateGraph(pctx)
    G = H.hvxCreateVirtualImage(g)
    H.hvxGaussian3x3Node(g, src, G)
    H.hvxEqualizeHistNode(g, G, out)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) == ["gaussian3x3_tma", "equalize_hist"]
    # parameter ranges
    g = H.hvxCreateGraph(pctx)
    for args in ((0, 0, 256), (257, 0, 256), (16, 200, 100), (16, -1, 10), (16, 0, 0)):
        with pytest.raises(H.HvxError):
            H.hvxHistogramNode(g, src, *args)
    s16 = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_S16)
    g = H.hvxCreateGraph(pctx)
    H.hvxHistogramNode(g, s16, 16, 0, 256)
    with pytest.raises(H.HvxError):  # histograms take U8 only
        H.hvxVerifyGraph(g)


def test_convert_depth_and_copy_plans(pctx):
    a = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_U8)
    s = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_S16)
    g = H.hvxCreateGraph(pctx)
    for bad in ((H.HVX_POLICY_WRAP, 8), (H.HVX_POLICY_WRAP, -1), (5, 1)):
        with pytest.raises(H.HvxError):
            H.hvxConvertDepthNode(g, a, H.hvxCreateVirtualImage(g), *bad)
    g = H.hvxCreateGraph(pctx)
    H.hvxConvertDepthNode(g, a, s, H.HVX_POLICY_SATURATE, 2)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) == ["plain_point"]
    g = H.hvxCreateGraph(pctx)
    H.hvxCopyNode(g, a, s)  # Copy keeps the format: U8 -> S16 is rejected
    with pytest.raises(H.HvxError):
        H.hvxVerifyGraph(g)
    g = H.hvxCreateGraph(pctx)
    H.hvxConvertDepthNode(g, a, H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_U8),
                          H.HVX_POLICY_SATURATE, 0)
    with pytest.raises(H.HvxError):  # ConvertDepth changes the depth
        H.hvxVerifyGraph(g)


def test_user_defined_operator_checks(pctx):
    a = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_U8)
    o = H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_S16)
    g = H.hvxCreateGraph(pctx)
    for bad in ("a / 2", "a && 1", "!a", "b", "foo(a)", "a +", "asm(1)", "a; b", "in(0, 0)"):
        with pytest.raises(H.HvxError):
            H.hvxUserPointNode(g, bad, [a], o)
    for bad, kw, kh in (("in(2, 0)", 3, 3), ("in(x, 0)", 3, 3), ("a", 3, 3), ("in(0,0)", 4, 3),
                        ("in(0,0)", 11, 1)):
        with pytest.raises(H.HvxError):
            H.hvxUserLocalNode(g, bad, kw, kh, a, o)
    # only generated kernels run them
    g = H.hvxCreateGraph(pctx)
    H.hvxUserPointNode(g, "a * 2 - 1", [a], o)
    H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_OFF)
    with pytest.raises(H.HvxError):
        H.hvxVerifyGraph(g)
    H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_REQUIRE)
    H.hvxVerifyGraph(g)  # compiles with NVRTC, no device needed
    assert "sat64_s16" in H.hvxGetGraphKernelSource(g, 0)
    # a user operator's output must declare its format
    g = H.hvxCreateGraph(pctx)
    H.hvxUserPointNode(g, "a", [a], H.hvxCreateVirtualImage(g))
    H.hvxCopyNode(g, a, H.hvxCreateImage(pctx, 64, 48, H.HVX_DF_U8))
    with pytest.raises(H.HvxError):
        H.hvxVerifyGraph(g)


def test_fault_injection_arguments():
    """hvxTestInjectFault accepts the two fault kinds with n >= 1 and
    HVX_FAULT_NONE; anything else is refused (no GPU needed)."""
    from paper_2008_11476_gb300 import hvx as H
    L = H.lib()
    assert L.hvxTestInjectFault(H.HVX_FAULT_DEVICE_ALLOC, 0) == H.HVX_ERROR_INVALID_PARAMETERS
    assert L.hvxTestInjectFault(7, 1) == H.HVX_ERROR_INVALID_PARAMETERS
    assert L.hvxTestInjectFault(H.HVX_FAULT_LAUNCH, 5) == H.HVX_SUCCESS
    assert L.hvxTestInjectFault(H.HVX_FAULT_NONE, 0) == H.HVX_SUCCESS


def test_hand_written_kernel_matches(pctx):
    # which single groups the planner maps onto the hand-written edge-family
    # kernels, and which near misses it leaves to generated / interpreted code
    import numpy as np
    src = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)

    def kinds(build):
        g = H.hvxCreateGraph(pctx)
        build(g)
        H.hvxVerifyGraph(g)
        return PG.kernel_kinds(g)

    def u8():
        return H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)

    def s16():
        return H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_S16)

    def sobel_mag_thr(g, a_sel, b_sel, thr_type=H.HVX_THRESHOLD_BINARY, gauss=True):
        base = src
        if gauss:
            base = H.hvxCreateVirtualImage(g)
            H.hvxGaussian3x3Node(g, src, base)
        gx, gy, m = (H.hvxCreateVirtualImage(g) for _ in range(3))
        H.hvxSobel3x3Node(g, base, gx, gy)
        H.hvxMagnitudeNode(g, {"x": gx, "y": gy}[a_sel], {"x": gx, "y": gy}[b_sel], m)
        H.hvxThresholdNode(g, m, thr_type, 100, 120, 255, 0, u8())

    # Listing 1 (gx dead, Magnitude(gy, gy)) and the plain edge graph
    assert kinds(lambda g: sobel_mag_thr(g, "y", "y")) == ["fused_edge_tma"]
    assert kinds(lambda g: sobel_mag_thr(g, "x", "y")) == ["fused_edge_tma"]
    # Magnitude(gx, gx) with gy dead, or a range threshold on Magnitude(gy, gy): not mapped
    assert kinds(lambda g: sobel_mag_thr(g, "x", "x")) != ["fused_edge_tma"]
    assert kinds(lambda g: sobel_mag_thr(g, "y", "y", H.HVX_THRESHOLD_RANGE)) != ["fused_edge_tma"]
    # no Gaussian: Sobel -> Magnitude -> binary Threshold, and gx alone as S16
    assert kinds(lambda g: sobel_mag_thr(g, "x", "y", gauss=False)) == ["fused_edge_tma"]
    assert kinds(lambda g: H.hvxSobel3x3Node(g, src, s16(), None)) == ["fused_edge_tma"]
    # gy alone, both derivatives exported, or a MIRROR border: not mapped
    assert kinds(lambda g: H.hvxSobel3x3Node(g, src, None, s16())) != ["fused_edge_tma"]
    assert kinds(lambda g: H.hvxSobel3x3Node(g, src, s16(), s16())) != ["fused_edge_tma"]

    def mirrored(g):
        H.hvxSetNodeBorder(H.hvxSobel3x3Node(g, src, s16(), None), H.HVX_BORDER_MIRROR, 0)
    assert kinds(mirrored) != ["fused_edge_tma"]
    # the 5x5 binomial Convolve (shift 8, U8 -> U8) and near misses
    b5 = np.outer([1, 4, 6, 4, 1], [1, 4, 6, 4, 1]).astype(np.int32)
    assert kinds(lambda g: H.hvxConvolveNode(g, src, b5.ravel(), 5, 5, 8, u8())) == \
        ["binomial5x5_tma"]
    assert kinds(lambda g: H.hvxConvolveNode(g, src, b5.ravel(), 5, 5, 7, u8())) != \
        ["binomial5x5_tma"]
    assert kinds(lambda g: H.hvxConvolveNode(g, src, b5.ravel(), 5, 5, 8, s16())) != \
        ["binomial5x5_tma"]
    odd = b5.copy()
    odd[0, 0] = 2
    assert kinds(lambda g: H.hvxConvolveNode(g, src, odd.ravel(), 5, 5, 8, u8())) != \
        ["binomial5x5_tma"]
    # HVX_CODEGEN_ONLY generates code for every one of them instead
    g = H.hvxCreateGraph(pctx)
    H.hvxConvolveNode(g, src, b5.ravel(), 5, 5, 8, u8())
    H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_ONLY)
    H.hvxVerifyGraph(g)
    assert PG.kernel_kinds(g) == ["staged_tile"]
