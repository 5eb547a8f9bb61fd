"""Code generation without a GPU: in a plan-only context with
HVX_CODEGEN_REQUIRE, verification emits each staged-tile group's kernel and
compiles it with NVRTC for sm_103a (nothing is loaded or run).  Checks that the
applications of the paper's evaluation all compile, that the generator folds
the constants it is given, and the mode switches."""
import re

import numpy as np
import pytest

from paper_2008_11476_gb300 import apps as A
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H


@pytest.fixture
def pctx():
    c = H.hvxCreateContextEx(H.HVX_CONTEXT_PLAN_ONLY)
    yield c
    H.hvxReleaseContext(c)


def _gen(ctx, build, w=1920, h=1080, fusion=True, mode=H.HVX_CODEGEN_REQUIRE):
    src = H.hvxCreateImage(ctx, w, h, H.HVX_DF_U8)
    g, _ = build(ctx, src, w, h, fusion)
    H.hvxSetGraphCodegen(g, mode)
    H.hvxVerifyGraph(g)
    return g


@pytest.mark.parametrize("mode", [H.HVX_CODEGEN_REQUIRE, H.HVX_CODEGEN_ONLY])
@pytest.mark.parametrize("name", [a for a, _ in A.APPS])
def test_applications_compile(pctx, name, mode):
    g = _gen(pctx, dict(A.APPS)[name], mode=mode)
    kinds = PG.kernel_kinds(g)
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == kinds.count("staged_tile")
    if mode == H.HVX_CODEGEN_ONLY:
        assert kinds == ["staged_tile"]
    for i, k in enumerate(kinds):
        s = H.hvxGetGraphKernelSource(g, i)
        assert (s is not None) == (k == "staged_tile")
        if s:
            assert "hvx_generated" in s and "hvx_tile<false, false>" in s


def test_u8_inputs_staged_by_tma(pctx, monkeypatch):
    # interior tiles take a staged U8 input as one TMA box on an mbarrier; its
    # slot's rows start 16 bytes left of the tile (halo 2 of the 5x5 Gauss);
    # HVX_CODEGEN_TMA=0 keeps per-thread loads (the group has a hand-written
    # kernel, so the generated one is asked for)
    only = H.HVX_CODEGEN_ONLY
    s = H.hvxGetGraphKernelSource(_gen(pctx, A.gauss, mode=only), 0)
    assert s.count("hvx_tma_2d(B") == 1 and "hvx_mbar_wait(bar, p.err)" in s
    assert "x0 - 16, y0 - 2" in s
    monkeypatch.setenv("HVX_CODEGEN_TMA", "0")
    s0 = H.hvxGetGraphKernelSource(_gen(pctx, A.gauss, mode=only), 0)
    assert "hvx_tma_2d(B" not in s0 and "__ldg((const unsigned*)" in s0


def test_constants_are_folded(pctx):
    # Laplacian: the four zero taps of the 3x3 kernel are dropped and the sum
    # of U8 inputs with coefficients up to 4 is accumulated in 32 bits
    s = H.hvxGetGraphKernelSource(_gen(pctx, A.laplacian), 0)
    m = re.search(r"(\d+) rows(?: x (\d+) columns)? per thread iteration", s)
    rows, cols = int(m.group(1)), int(m.group(2) or 1)
    # one block of rows x cols cells per iteration
    assert s.count("t += ") == 5 * rows * cols
    assert "long long t" not in s
    if rows == 4:
        # a cross of 5 taps over 4 rows reads 14 distinct values, not 20
        assert s.count("= B0[qb0") == 14
    # the Sobel application's Magnitude -> Threshold(100) is the integer
    # compare gx^2 + gy^2 > 100^2 + 100, with the bound a literal (the group
    # has a hand-written kernel, so the generated one is asked for)
    s = H.hvxGetGraphKernelSource(_gen(pctx, A.sobel, mode=H.HVX_CODEGEN_ONLY), 0)
    assert "> 10100u)" in s


def test_column_blocks(pctx, monkeypatch):
    # HVX_CODEGEN_COLS=4: the output pass in blocks of 2 rows x 4 columns
    monkeypatch.setenv("HVX_CODEGEN_COLS", "4")
    s = H.hvxGetGraphKernelSource(_gen(pctx, A.laplacian, 1000, 600), 0)
    m = re.search(r"(\d+) rows(?: x (\d+) columns)? per thread iteration", s)
    rows, cols = int(m.group(1)), int(m.group(2) or 1)
    assert (rows, cols) == (2, 4)
    assert s.count("t += ") == 5 * rows * cols
    # a cross of 5 taps over 2 rows x 4 columns reads 20 distinct values,
    # not 40, from at most 3 aligned words of each of the 4 input rows
    assert len(set(re.findall(r"const int (t0_\w+) = ", s))) == 20
    assert s.count("const unsigned L0_") <= 12
    assert "if (!CHECK && va0)" in s


def test_products_share_one_pass(pctx):
    # Tomasi: the three products are staged by one pass that evaluates the
    # Sobel derivatives once; the sums, response and threshold are evaluated
    # inline in the output pass
    s = H.hvxGetGraphKernelSource(_gen(pctx, A.tomasi, mode=H.HVX_CODEGEN_ONLY), 0)
    assert s.count("// pass:") == 2
    assert "tomasi_response_f32" in s


def test_codegen_only_replaces_hand_written_kernels(pctx):
    # the edge graph, Gaussian3x3 alone and the Harris group have hand-written
    # kernels; HVX_CODEGEN_ONLY generates theirs instead
    src = H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8)
    ph, mk, go = (H.hvxCreateImage(pctx, 640, 480, H.HVX_DF_U8) for _ in range(3))
    ge = PG.edge_graph(pctx, src, ph, mk, verify=False)
    gg = H.hvxCreateGraph(pctx)
    H.hvxGaussian3x3Node(gg, src, go)
    gh, _ = A.harris(pctx, src, 640, 480, True)
    for g in (ge, gg, gh):
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g)[0] != "staged_tile"
        H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_ONLY)
        H.hvxVerifyGraph(g)
        assert PG.kernel_kinds(g) == ["staged_tile"]
        assert "hvx_generated" in H.hvxGetGraphKernelSource(g, 0)
    with pytest.raises(H.HvxError):
        H.hvxSetGraphCodegen(gg, 4)


def test_same_shape_same_source(pctx):
    a = H.hvxGetGraphKernelSource(_gen(pctx, A.fchain, 640, 480), 0)
    b = H.hvxGetGraphKernelSource(_gen(pctx, A.fchain, 1920, 1080), 0)
    assert a == b  # the image size is a launch parameter, not compiled in


def test_modes(pctx):
    g = _gen(pctx, A.unsharp, mode=H.HVX_CODEGEN_OFF)
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == 0
    assert H.hvxGetGraphKernelSource(g, 0) is None
    # a plan-only context does not compile unless required
    g = _gen(pctx, A.unsharp, mode=H.HVX_CODEGEN_AUTO)
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == 0
    with pytest.raises(H.HvxError):
        H.hvxSetGraphCodegen(g, 7)


def test_unfused_nodes_compile(pctx):
    # one generated kernel per staged-tile node when fusion is off
    g = _gen(pctx, A.tomasi, fusion=False, mode=H.HVX_CODEGEN_ONLY)
    kinds = PG.kernel_kinds(g)
    assert H.hvxQueryGraph(g, H.HVX_GRAPH_GENERATED_KERNELS) == kinds.count("staged_tile") > 0


def test_every_border_mode_compiles(pctx):
    for border in (H.HVX_BORDER_UNDEFINED, H.HVX_BORDER_REPLICATE, H.HVX_BORDER_CONSTANT):
        src = H.hvxCreateImage(pctx, 333, 77, H.HVX_DF_U8)
        out = H.hvxCreateImage(pctx, 333, 77, H.HVX_DF_S16)
        g = H.hvxCreateGraph(pctx)
        a = H.hvxCreateVirtualImage(g)
        H.hvxSetNodeBorder(H.hvxMedian3x3Node(g, src, a), border, 7)
        n = H.hvxConvolveNode(g, a, np.arange(-12, 13), 5, 5, 1, out)
        H.hvxSetNodeBorder(n, border, 9)
        H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_REQUIRE)
        H.hvxVerifyGraph(g)
        s = H.hvxGetGraphKernelSource(g, 0)
        fill = re.search(r"= (\(unsigned char\))?9;", s) is not None  # the fill constant
        assert fill == (border == H.HVX_BORDER_CONSTANT)
