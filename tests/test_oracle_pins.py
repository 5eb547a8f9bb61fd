"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, invariants, library routines that a special case reduces to, and
brute force.  CPU only."""
import json
import os
from fractions import Fraction

import mpmath
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle as O
from oracle import graph as G
from paper_2008_11476_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BORDERS = [O.BORDER_REPLICATE, O.BORDER_CONSTANT, O.BORDER_UNDEFINED]


def interior(a, r):
    return a[r:-r, r:-r] if r else a


# --- Gaussian3x3 -------------------------------------------------------------------

@pytest.mark.parametrize("c", [0, 1, 77, 255])
@pytest.mark.parametrize("border", BORDERS)
def test_gaussian_constant_is_fixed_point(orc, c, border):
    img = np.full((9, 13), c, np.uint8)
    out = O.gaussian3x3(img, border, cval=c)
    if border == O.BORDER_UNDEFINED:
        assert out.rect == (1, 1, 12, 8)
        assert (interior(out.data, 1) == c).all()
        assert (out.data[0] == 0).all() and (out.data[:, -1] == 0).all()
    else:
        assert out.rect == (0, 0, 13, 9)
        assert (out.data == c).all()


def test_gaussian_linear_ramp_interior(orc):
    y, x = np.mgrid[0:20, 0:30]
    img = (3 * x + 5 * y + 7).astype(np.uint8)  # max 3*29+5*19+7 = 189
    out = O.gaussian3x3(img, O.BORDER_REPLICATE)
    assert (interior(out.data, 1) == interior(img, 1)).all()


@pytest.mark.parametrize("rounding,expect", [(O.ROUND_ZERO, (63, 31, 15)),
                                              (O.ROUND_NEAREST, (64, 32, 16))])
def test_gaussian_impulse(orc, rounding, expect):
    img = np.zeros((7, 7), np.uint8)
    img[3, 3] = 255
    out = O.gaussian3x3(img, O.BORDER_REPLICATE, rounding=rounding).data
    centre, edge, corner = expect
    assert out[3, 3] == centre
    assert out[2, 3] == out[4, 3] == out[3, 2] == out[3, 4] == edge
    assert out[2, 2] == out[2, 4] == out[4, 2] == out[4, 4] == corner
    assert out.sum() == centre + 4 * edge + 4 * corner


def test_gaussian_one_pixel(orc):
    img = np.array([[200]], np.uint8)
    assert O.gaussian3x3(img, O.BORDER_REPLICATE).data[0, 0] == 200
    # constant 10 around a single 200: (4*200 + 12*10) / 16 = 57.5 -> 57
    assert O.gaussian3x3(img, O.BORDER_CONSTANT, cval=10).data[0, 0] == 57
    assert O.gaussian3x3(img, O.BORDER_UNDEFINED).rect == (1, 1, 1, 1)


@pytest.mark.parametrize("shape", [(1, 5), (5, 1), (2, 2), (17, 23), (32, 45)])
def test_gaussian_matches_scipy_correlate(orc, shape):
    img = synth.uniform_u8(shape[1], shape[0], seed=11)
    w = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], np.int64)
    ref_rep = ndi.correlate(img.astype(np.int64), w, mode="nearest") // 16
    ref_con = ndi.correlate(img.astype(np.int64), w, mode="constant", cval=33) // 16
    assert (O.gaussian3x3(img, O.BORDER_REPLICATE).data == ref_rep).all()
    assert (O.gaussian3x3(img, O.BORDER_CONSTANT, cval=33).data == ref_con).all()


def test_box3x3_matches_scipy(orc):
    img = synth.uniform_u8(31, 17, seed=3)
    ref = ndi.correlate(img.astype(np.int64), np.ones((3, 3), np.int64), mode="nearest")
    assert (O.box3x3(img, O.BORDER_REPLICATE).data == ref // 9).all()
    assert (O.box3x3(img, O.BORDER_REPLICATE, rounding=O.ROUND_NEAREST).data
            == (ref + 4) // 9).all()


# --- Sobel3x3 ------------------------------------------------------------------------

def test_sobel_constant_is_zero(orc):
    for border in BORDERS:
        gx, gy = O.sobel3x3(np.full((6, 8), 99, np.uint8), border, cval=99)
        assert (gx.data == 0).all() and (gy.data == 0).all()


@pytest.mark.parametrize("a,b", [(1, 0), (0, 1), (2, 3), (4, 1)])
def test_sobel_linear_ramp(orc, a, b):
    y, x = np.mgrid[0:16, 0:20]
    img = (a * x + b * y).astype(np.uint8)
    gx, gy = O.sobel3x3(img, O.BORDER_REPLICATE)
    assert (interior(gx.data, 1) == 8 * a).all()
    assert (interior(gy.data, 1) == 8 * b).all()
    # replicated edge columns / rows see half the difference
    assert (gx.data[1:-1, 0] == 4 * a).all() and (gx.data[1:-1, -1] == 4 * a).all()
    assert (gy.data[0, 1:-1] == 4 * b).all() and (gy.data[-1, 1:-1] == 4 * b).all()


def test_sobel_matches_scipy_correlate(orc):
    img = synth.uniform_u8(37, 29, seed=5)
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
    gx, gy = O.sobel3x3(img, O.BORDER_REPLICATE)
    assert (gx.data == ndi.correlate(img.astype(np.int64), kx, mode="nearest")).all()
    assert (gy.data == ndi.correlate(img.astype(np.int64), kx.T, mode="nearest")).all()
    gx, gy = O.sobel3x3(img, O.BORDER_UNDEFINED)
    ref = ndi.correlate(img.astype(np.int64), kx.T, mode="constant")
    assert gx.rect == (1, 1, 36, 28)
    assert (interior(gy.data, 1) == interior(ref, 1)).all()
    assert (gy.data[0] == 0).all()


# --- Magnitude / Phase -------------------------------------------------------------

def _all_pairs(lim=1020):
    v = np.arange(-lim, lim + 1, dtype=np.int16)
    gx, gy = np.meshgrid(v, v)
    return np.ascontiguousarray(gx), np.ascontiguousarray(gy)


def test_magnitude_exhaustive_against_integer_sqrt(orc):
    gx, gy = _all_pairs()
    m = O.magnitude(gx, gy).data.astype(np.int64)
    s4 = 4 * (gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2)
    # floor(sqrt(s) + 1/2) == (isqrt(4 s) + 1) // 2, isqrt by integer correction
    r = np.floor(np.sqrt(s4.astype(np.float64))).astype(np.int64)
    r -= (r * r > s4)
    r += ((r + 1) * (r + 1) <= s4)
    assert (m == (r + 1) // 2).all()


def test_phase_cardinal_and_diagonal_directions(orc):
    cases = {(5, 0): 0, (0, 5): 64, (-5, 0): 128, (0, -5): 192, (7, 7): 32, (-7, 7): 96,
             (-7, -7): 160, (7, -7): 224, (0, 0): 0}
    gx = np.array([[k[0] for k in cases]], np.int16)
    gy = np.array([[k[1] for k in cases]], np.int16)
    assert list(O.phase(gx, gy).data[0]) == list(cases.values())


def test_phase_symmetries(orc):
    gx, gy = _all_pairs(300)
    q = O.phase(gx, gy).data.astype(np.int64)
    q_neg = O.phase(np.ascontiguousarray(-gx), np.ascontiguousarray(-gy)).data
    q_swap = O.phase(gy, gx).data.astype(np.int64)
    nz = (gx != 0) | (gy != 0)
    assert (((q + 128) % 256)[nz] == q_neg[nz]).all()       # rotation by pi
    assert (((64 - q) % 256)[nz] == q_swap[nz]).all()        # reflection in y = x


def test_phase_against_mpmath_sample(orc):
    mpmath.mp.dps = 40
    rng = synth.randint(21, 0, 4000, -1020, 1020).reshape(2000, 2)
    gx = np.ascontiguousarray(rng[:, 0].astype(np.int16)).reshape(1, -1)
    gy = np.ascontiguousarray(rng[:, 1].astype(np.int16)).reshape(1, -1)
    q = O.phase(gx, gy).data[0]
    for i in range(gx.shape[1]):
        a, b = int(gx[0, i]), int(gy[0, i])
        if a == 0 and b == 0:
            assert q[i] == 0
            continue
        phi = mpmath.atan2(b, a)
        if phi < 0:
            phi += 2 * mpmath.pi
        exp = int(mpmath.floor(phi * 128 / mpmath.pi + mpmath.mpf(1) / 2)) % 256
        assert q[i] == exp, (a, b)


# --- Threshold ---------------------------------------------------------------------

def test_threshold_step_at_value(orc):
    v = np.arange(-32768, 32768, dtype=np.int32).astype(np.int16).reshape(256, 256)
    out = O.threshold(v, 100).data.reshape(-1)
    idx = np.arange(-32768, 32768)
    assert out[idx == 100][0] == 0 and out[idx == 101][0] == 255
    assert (np.diff(out.astype(np.int64)) >= 0).all()        # one step only
    assert int((out == 255).sum()) == 32767 - 100
    r = O.threshold_range(v, -5, 7, true_val=9, false_val=1).data.reshape(-1)
    assert int((r == 9).sum()) == 13 and set(np.unique(r)) == {1, 9}


def test_threshold_f32_uses_binary32_value(orc):
    # 1e6 + 0.04 rounds to 1e6 + 0.0625 in binary32 (spacing 1/16 at 2^19..2^20)
    x = np.array([[1e6, np.float32(1e6 + 0.04), np.nextafter(np.float32(1e6), 0)]],
                 np.float32)
    assert list(O.threshold(x, 1e6).data[0]) == [0, 255, 0]


# --- ChannelExtract / arithmetic -----------------------------------------------------

def test_channel_extract_inverts_interleave(orc):
    w, h = 10, 3
    Y = synth.uniform_u8(w, h, 1)
    U = synth.uniform_u8(w // 2, h, 2)
    V = synth.uniform_u8(w // 2, h, 3)
    uyvy = np.empty((h, 2 * w), np.uint8)
    uyvy[:, 0::4], uyvy[:, 1::4], uyvy[:, 2::4], uyvy[:, 3::4] = U, Y[:, 0::2], V, Y[:, 1::2]
    assert (O.channel_extract_uyvy(uyvy, 0).data == Y).all()
    assert (O.channel_extract_uyvy(uyvy, 1).data == U).all()
    assert (O.channel_extract_uyvy(uyvy, 2).data == V).all()


def test_arith_special_values(orc):
    a = np.array([[200, 0, 255, 17]], np.uint8)
    b = np.array([[100, 0, 255, 3]], np.uint8)
    assert list(O.arith(a, b, np.uint8, O.ARITH_ADD, True).data[0]) == [255, 0, 255, 20]
    assert list(O.arith(a, b, np.uint8, O.ARITH_ADD, False).data[0]) == [44, 0, 254, 20]
    assert list(O.arith(a, b, np.int16, O.ARITH_ADD, True).data[0]) == [300, 0, 510, 20]
    assert list(O.arith(b, a, np.uint8, O.ARITH_SUB, True).data[0]) == [0, 0, 0, 0]
    assert list(O.arith(b, a, np.int16, O.ARITH_SUB, True).data[0]) == [-100, 0, 0, -14]
    assert list(O.arith(b, a, np.uint8, O.ARITH_ABSDIFF, True).data[0]) == [100, 0, 0, 14]
    s = np.array([[32000, -32000]], np.int16)
    assert list(O.arith(s, s, np.int16, O.ARITH_ADD, True).data[0]) == [32767, -32768]
    assert list(O.arith(s, s, np.int16, O.ARITH_ADD, False).data[0]) == [-1536, 1536]


def test_arith_commutes_and_has_identity(orc):
    a = synth.uniform_u8(40, 7, 8)
    b = synth.uniform_u8(40, 7, 9)
    z = np.zeros_like(a)
    for sat in (True, False):
        assert (O.arith(a, b, np.uint8, 0, sat).data == O.arith(b, a, np.uint8, 0, sat).data).all()
        assert (O.arith(a, z, np.uint8, 0, sat).data == a).all()


def test_convolve_laplacian_matches_scipy(orc):
    img = synth.uniform_u8(25, 19, 4)
    lap = np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], np.int32)
    ref = ndi.correlate(img.astype(np.int64), lap, mode="nearest")
    assert (O.convolve(img, lap, 0, O.BORDER_REPLICATE).data == ref).all()
    # floor division by 2 for negative sums
    assert (O.convolve(img, lap, 1, O.BORDER_REPLICATE).data == np.floor_divide(ref, 2)).all()


# --- Harris pieces -----------------------------------------------------------------

def test_window_sum_matches_scipy(orc):
    a = synth.randint(3, 0, 21 * 15, -50000, 50000).astype(np.int32).reshape(15, 21)
    ref = ndi.correlate(a.astype(np.int64), np.ones((5, 5), np.int64), mode="constant")
    out = O.window_sum(a, 5, 5, O.BORDER_UNDEFINED)
    assert out.rect == (2, 2, 19, 13)
    assert (interior(out.data, 2) == interior(ref, 2)).all()
    assert (out.data[:2] == 0).all() and (out.data[:, -2:] == 0).all()
    rep = ndi.correlate(a.astype(np.int64), np.ones((3, 5), np.int64), mode="nearest")
    assert (O.window_sum(a, 5, 3, O.BORDER_REPLICATE).data == rep).all()


def _mp_round24(fr: Fraction) -> float:
    """p/q rounded once to a 24-bit significand, ties to even (mpmath)."""
    return float(mpmath.mpf(mpmath.libmp.from_rational(fr.numerator, fr.denominator, 24, "n")))


def test_round_ratio_is_correctly_rounded(orc):
    nums = [1, 2, 3, 7, 24, 25, 26, 16777217, 16777219, 25000001, 10**15 + 7,
            -(10**14) - 3, 2**53 + 1, -5, 0]
    nums += [int(v) for v in synth.randint(17, 0, 300, -(2**40), 2**40)]
    for den in (1, 3, 7, 25, 1000):
        for n in nums:
            assert O.round_ratio(n, den) == _mp_round24(Fraction(n, den)), (n, den)
    # ties go to the even significand
    assert O.round_ratio(16777217, 1) == 16777216.0
    assert O.round_ratio(16777219, 1) == 16777220.0


def test_harris_response_closed_forms(orc):
    s = np.array([[0, 5, 1000, 26010000]], np.int32)
    z = np.zeros_like(s)
    # Sxx = Syy = s, Sxy = 0, k = 1/25: R = s^2 - 4 s^2 / 25 = 21 s^2 / 25
    r = O.harris_response(s, s, z, 1, 25).data[0]
    for i, v in enumerate(s[0]):
        assert r[i] == _mp_round24(Fraction(21 * int(v) ** 2, 25))
    # a pure edge (Syy = Sxy = 0): R = -k Sxx^2 <= 0
    r = O.harris_response(s, z, z, 1, 25).data[0]
    assert (r <= 0).all() and r[2] == -40000.0
    # Sxy^2 = Sxx Syy (rank one): det = 0
    a = np.array([[4, 9]], np.int32)
    b = np.array([[9, 4]], np.int32)
    c = np.array([[6, -6]], np.int32)
    r = O.harris_response(a, b, c, 1, 25).data[0]
    assert list(r) == [_mp_round24(Fraction(-169, 25))] * 2


def test_harris_graph_flat_edge_corner(orc):
    img = np.full((40, 48), 90, np.uint8)
    mask, resp = O.harris_graph(img, thr=1e6)
    assert (resp == 0).all() and (mask == 0).all()
    # vertical step edge: no positive response anywhere
    img[:, 24:] = 200
    mask, resp = O.harris_graph(img, thr=0.0)
    assert (resp <= 0).all() and (mask == 0).all()
    # bright square on dark: positive responses at its four corners only
    img = np.zeros((40, 48), np.uint8)
    img[10:30, 12:36] = 200
    mask, resp = O.harris_graph(img, thr=1e6)
    ys, xs = np.nonzero(mask)
    assert len(ys) > 0
    for y, x in zip(ys, xs):
        assert min(abs(y - 10), abs(y - 29)) <= 3 and min(abs(x - 12), abs(x - 35)) <= 3
    # undefined border: 3 pixels on each side stay zero
    assert (resp[:3] == 0).all() and (resp[:, -3:] == 0).all()


def test_edge_graph_ramp_and_constant(orc):
    img = np.full((24, 32), 140, np.uint8)
    ph, mk = O.edge_graph(img)
    assert (ph == 0).all() and (mk == 0).all()
    y, x = np.mgrid[0:24, 0:32]
    ramp = (3 * x + 4 * y).astype(np.uint8)
    ph, mk, mag = O.edge_graph(ramp, want_mag=True)
    # Gaussian keeps the ramp inside 1 px; Sobel there sees gx = 24, gy = 32
    assert (mag[2:-2, 2:-2] == 40).all()
    assert (mk[2:-2, 2:-2] == 0).all()
    # atan2(32, 24) = 0.9273 rad -> 0.9273 * 128 / pi = 37.78 -> 38
    assert (ph[2:-2, 2:-2] == 38).all()


# --- graph verification and Algorithm 1 ---------------------------------------------

def _load_listing1():
    spec = json.load(open(os.path.join(GOLDEN, "listing1_edge_graph.json")))
    g = G.GraphDesc()
    for im in spec["images"]:
        if im["virtual"]:
            g.virtual(im["name"])
        else:
            g.image(im["name"], im["w"], im["h"], im["fmt"])
    for n in spec["nodes"]:
        g.node(n["kind"], n["ins"], n["outs"], **n["params"])
    return spec, g


def test_listing1_dead_sobel_output(orc):
    spec, g = _load_listing1()
    ops = G.verify(g)
    alive, alive_data = G.eliminate_dead(g, ops)
    assert sorted(op.name for op in alive) == sorted(spec["expected_alive_ops"])
    dead = sorted({op.name for op in ops} - {op.name for op in alive})
    assert dead == spec["expected_dead_ops"]
    for d in spec["expected_dead_data"]:
        assert d not in alive_data


def test_listing1_runs(orc):
    spec, g = _load_listing1()
    img0 = synth.uyvy(64, 48, 3)
    out = G.run(g, {"img0": img0})["img1"].data
    Y = O.channel_extract_uyvy(img0, 0)
    _, gy = O.sobel3x3(O.gaussian3x3(Y, O.BORDER_REPLICATE))
    ref = O.threshold(O.magnitude(gy, gy), 100).data
    assert (out == ref).all()


def _brute_alive(g, ops):
    """An op is alive iff a directed path leads from it to a non-virtual image."""
    readers = {}
    for op in ops:
        for i in op.ins:
            readers.setdefault(i, []).append(op)
    alive = set()
    for op in ops:
        stack, seen, hit = [op], set(), False
        while stack and not hit:
            o = stack.pop()
            if o.name in seen:
                continue
            seen.add(o.name)
            if not g.data[o.out].virtual:
                hit = True
            stack.extend(readers.get(o.out, ()))
        if hit:
            alive.add(op.name)
    return alive


def test_algorithm1_matches_brute_force_on_random_dags(orc):
    kinds_1in = ["gaussian3x3", "box3x3"]
    for seed in range(60):
        u = synth.uniform01(seed, 30, 200)
        k = 0
        g = G.GraphDesc()
        g.image("in0", 8, 8, "U8")
        pool = ["in0"]
        n_nodes = 2 + int(u[k] * 8); k += 1
        for i in range(n_nodes):
            src = pool[int(u[k] * len(pool))]; k += 1
            virt = u[k] < 0.6; k += 1
            name = f"d{i}"
            if virt:
                g.virtual(name)
            else:
                g.image(name, 8, 8, "U8")
            g.node(kinds_1in[int(u[k] * 2)], [src], [name]); k += 1
            pool.append(name)
        ops = G.verify(g)
        alive, _ = G.eliminate_dead(g, ops)
        assert {op.name for op in alive} == _brute_alive(g, ops), seed


def test_verify_rejects_cycle_and_bad_graphs(orc):
    g = G.GraphDesc()
    g.virtual("a", 8, 8, "U8")
    g.virtual("b", 8, 8, "U8")
    g.node("gaussian3x3", ["a"], ["b"])
    g.node("gaussian3x3", ["b"], ["a"])
    with pytest.raises(G.GraphError):
        G.verify(g)
    g = G.GraphDesc()
    g.image("in", 8, 8, "S16")
    g.image("out", 8, 8, "U8")
    g.node("gaussian3x3", ["in"], ["out"])            # S16 into a U8-only input
    with pytest.raises(G.GraphError):
        G.verify(g)
    g = G.GraphDesc()
    g.image("in", 8, 8, "U8")
    g.virtual("v")
    g.image("out", 8, 8, "U8")
    g.node("gaussian3x3", ["v"], ["out"])              # virtual never written
    with pytest.raises(G.GraphError):
        G.verify(g)
    g = G.GraphDesc()
    g.image("in", 8, 8, "U8")
    g.image("out", 8, 8, "U8")
    g.node("gaussian3x3", ["in"], ["out"])
    g.node("box3x3", ["in"], ["out"])                  # two writers
    with pytest.raises(G.GraphError):
        G.verify(g)
    assert not G.is_bipartite([(("D", "a"), ("D", "b"))])


def test_nonvirtual_intermediate_keeps_upstream_alive(orc):
    g = G.GraphDesc()
    g.image("in", 8, 8, "U8")
    g.image("mid", 8, 8, "U8")        # non-virtual, read downstream
    g.virtual("dead")
    g.node("gaussian3x3", ["in"], ["mid"])
    g.node("box3x3", ["mid"], ["dead"])
    g.image("iso", 8, 8, "U8")        # isolated image
    ops = G.verify(g)
    alive, data = G.eliminate_dead(g, ops)
    assert [op.name for op in alive] == ["n0"]
    assert "iso" not in data and "dead" not in data


# --- Dilate3x3 / Erode3x3 / Median3x3, And / Or / Xor / Not (Table 2) ----------------

MORPH_REF = {O.MORPH_DILATE: ndi.grey_dilation, O.MORPH_ERODE: ndi.grey_erosion,
             O.MORPH_MEDIAN: ndi.median_filter}


@pytest.mark.parametrize("op", [O.MORPH_DILATE, O.MORPH_ERODE, O.MORPH_MEDIAN])
@pytest.mark.parametrize("shape", [(1, 1), (2, 5), (17, 23)])
def test_morph_matches_scipy(orc, op, shape):
    img = synth.uniform_u8(shape[1], shape[0], seed=11 + op)
    f = MORPH_REF[op]
    r = O.morph3x3(img, op, O.BORDER_REPLICATE)
    assert (r.data == f(img, size=3, mode="nearest")).all()
    r = O.morph3x3(img, op, O.BORDER_CONSTANT, cval=77)
    assert (r.data == f(img, size=3, mode="constant", cval=77)).all()
    r = O.morph3x3(img, op, O.BORDER_UNDEFINED)
    h, w = shape
    assert r.rect == (1, 1, max(1, w - 1), max(1, h - 1))
    inner = f(img, size=3, mode="nearest")[1:h - 1, 1:w - 1]
    assert (r.data[1:h - 1, 1:w - 1] == inner).all()
    mask = np.ones_like(img, bool)
    mask[1:h - 1, 1:w - 1] = False
    assert (r.data[mask] == 0).all()


def test_morph_impulses(orc):
    z = np.zeros((7, 9), np.uint8)
    z[3, 4] = 255
    d = O.morph3x3(z, O.MORPH_DILATE, O.BORDER_REPLICATE).data
    assert (d[2:5, 3:6] == 255).all() and d.sum() == 9 * 255
    assert (O.morph3x3(z, O.MORPH_MEDIAN, O.BORDER_REPLICATE).data == 0).all()
    hole = np.full((7, 9), 200, np.uint8)
    hole[3, 4] = 0
    e = O.morph3x3(hole, O.MORPH_ERODE, O.BORDER_REPLICATE).data
    assert (e[2:5, 3:6] == 0).all() and (e == 0).sum() == 9
    # median of the window values 0..8 (a permutation) is 4
    perm = np.array([[5, 1, 7], [0, 8, 3], [6, 2, 4]], np.uint8)
    assert O.morph3x3(perm, O.MORPH_MEDIAN, O.BORDER_UNDEFINED).data[1, 1] == 4


def test_bitwise_matches_numpy(orc):
    a = synth.uniform_u8(19, 13, seed=21)
    b = synth.uniform_u8(19, 13, seed=22)
    assert (O.bitwise(a, b, O.BIT_AND).data == (a & b)).all()
    assert (O.bitwise(a, b, O.BIT_OR).data == (a | b)).all()
    assert (O.bitwise(a, b, O.BIT_XOR).data == (a ^ b)).all()
    assert (O.bitwise(a, None, O.BIT_NOT).data == (~a)).all()
    # valid regions intersect
    ra = O.Img(a, (1, 2, 18, 12))
    rb = O.Img(b, (3, 0, 19, 10))
    r = O.bitwise(ra, rb, O.BIT_AND)
    assert r.rect == (3, 2, 18, 10)
    assert (r.data[:2] == 0).all() and (r.data[:, :3] == 0).all()


def test_graph_runner_morphology_closing(orc):
    # closing (dilate then erode) as an oracle graph equals the two calls
    img = synth.uniform_u8(24, 16, seed=5)
    g = G.GraphDesc()
    g.image("in", 24, 16, "U8")
    g.virtual("d")
    g.image("out", 24, 16, "U8")
    g.node("dilate3x3", ["in"], ["d"], border="replicate")
    g.node("erode3x3", ["d"], ["out"], border="replicate")
    res = G.run(g, {"in": img})["out"]
    ref = O.morph3x3(O.morph3x3(img, O.MORPH_DILATE), O.MORPH_ERODE)
    assert (res.data == ref.data).all()


# --- Convolve with U8 output, Shi-Tomasi response (the Section 6 applications) ------

def test_convolve_u8_output_is_saturated_s16(orc):
    img = synth.uniform_u8(23, 19, seed=17)
    sharpen = np.array([[0, -1, 0], [-1, 8, -1], [0, -1, 0]], np.int32)
    for border in BORDERS:
        s16 = O.convolve(img, sharpen, 2, border, 40)
        u8 = O.convolve(img, sharpen, 2, border, 40, np.uint8)
        assert u8.rect == s16.rect
        assert (u8.data == np.clip(s16.data, 0, 255)).all()
    assert (O.convolve(img, sharpen, 2, out_dtype=np.uint8).data == 255).any()


def test_tomasi_closed_forms_and_eigvalsh(orc):
    a = np.array([[100, 7, 5000, 0, 26010000]], np.int32)
    b = np.array([[30, 7, 5000, 9, 26010000]], np.int32)
    c = np.array([[0, 3, 5000, 0, -26010000]], np.int32)
    r = O.tomasi_response(a, b, c).data[0]
    # diagonal: min(a, b); a = b: a - |c|; rank one (c^2 = a b): 0
    assert r[0] == 30 and r[1] == 4 and r[2] == 0 and r[3] == 0 and r[4] == 0
    rng = np.random.default_rng(5)
    A = rng.integers(0, 2 ** 24, 500)
    B = rng.integers(0, 2 ** 24, 500)
    C = (rng.uniform(-1, 1, 500) * np.sqrt(A * B.astype(np.float64))).astype(np.int64)
    got = O.tomasi_response(A.astype(np.int32)[None], B.astype(np.int32)[None],
                            C.astype(np.int32)[None]).data[0].astype(np.float64)
    ref = np.array([np.linalg.eigvalsh(np.array([[x, z], [z, y]], np.float64))[0]
                    for x, y, z in zip(A, B, C)])
    scale = np.maximum(np.abs(A) + np.abs(B), 1)
    assert np.all(np.abs(got - ref) <= 1e-6 * scale)


# --- MIRROR / REPEAT boundary conditions (Hipacc's MIRROR, REPEAT) ----------
# scipy.ndimage's "reflect" extends ... c b a | a b c ... and "wrap" is
# periodic: the two readings of the oracle.  Small images exercise repeated
# reflection (windows wider than the image).

def _bm(mode):
    import oracle as O
    return O.BORDER_MIRROR if mode == "reflect" else O.BORDER_REPEAT


@pytest.mark.parametrize("mode", ["reflect", "wrap"])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (3, 2), (9, 13), (40, 31)])
def test_mirror_repeat_gaussian_box_sobel_match_scipy(orc, mode, shape):
    img = synth.uniform_u8(shape[1], shape[0], seed=shape[0] * 7 + shape[1])
    b = _bm(mode)
    a = img.astype(np.int64)
    w = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], np.int64)
    assert (orc.gaussian3x3(img, b).data == ndi.correlate(a, w, mode=mode) // 16).all()
    assert (orc.box3x3(img, b).data == ndi.correlate(a, np.ones((3, 3), np.int64), mode=mode) // 9).all()
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], np.int64)
    gx, gy = orc.sobel3x3(img, b)
    assert (gx.data == ndi.correlate(a, kx, mode=mode)).all()
    assert (gy.data == ndi.correlate(a, kx.T, mode=mode)).all()
    for r in (orc.gaussian3x3(img, b), gx):
        assert r.rect == (0, 0, shape[1], shape[0])  # no shrinking


@pytest.mark.parametrize("mode", ["reflect", "wrap"])
@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (4, 3), (23, 17)])
def test_mirror_repeat_convolve_window_sum_morph_match_scipy(orc, mode, shape):
    img = synth.uniform_u8(shape[1], shape[0], seed=91 + shape[0])
    b = _bm(mode)
    a = img.astype(np.int64)
    c = np.arange(-12, 13, dtype=np.int64).reshape(5, 5)
    want = np.clip(ndi.correlate(a, c, mode=mode) >> 2, -32768, 32767)
    assert (orc.convolve(img, c, 2, b).data == want).all()
    s32 = synth.uniform_u8(shape[1], shape[0], seed=5).astype(np.int32) * 1000 - 100000
    ws = orc.window_sum(orc.Img(s32), 5, 3, b)
    assert (ws.data == ndi.correlate(s32.astype(np.int64), np.ones((3, 5), np.int64),
                                     mode=mode)).all()
    for op, f in ((orc.MORPH_DILATE, ndi.grey_dilation), (orc.MORPH_ERODE, ndi.grey_erosion),
                  (orc.MORPH_MEDIAN, ndi.median_filter)):
        assert (orc.morph3x3(img, op, b).data == f(img, size=3, mode=mode)).all()


def test_mirror_repeat_brute_force_coordinates(orc):
    # the reading written out on a 1-D ramp: index i of a 3-pixel row
    img = np.array([[10, 20, 30]], np.uint8)
    c = np.zeros((1, 5), np.int64)
    c[0, 0] = 1  # reads x - 2
    got_m = orc.convolve(img, c, 0, orc.BORDER_MIRROR).data[0].tolist()
    got_r = orc.convolve(img, c, 0, orc.BORDER_REPEAT).data[0].tolist()
    # x - 2 for x = 0, 1, 2 is -2, -1, 0: mirror -> 1, 0, 0; repeat -> 1, 2, 0
    assert got_m == [20, 10, 10]
    assert got_r == [20, 30, 10]


# --- Multiply (Table 2 point operator) --------------------------------------

def _mul_exact(a, b, scale, out_dtype, saturate, nearest_even):
    """a * b * scale as an exact fraction, rounded once, then wrapped or
    saturated: element by element in Python integers."""
    s = Fraction(float(np.float32(scale)))
    lo, hi, bits = (0, 255, 8) if out_dtype == np.uint8 else (-32768, 32767, 16)
    out = np.empty(a.shape, out_dtype)
    for i in np.ndindex(a.shape):
        v = Fraction(int(a[i])) * int(b[i]) * s
        r = round(v) if nearest_even else int(v)  # round(): ties to even; int(): toward zero
        if saturate:
            r = min(max(r, lo), hi)
        else:
            r &= (1 << bits) - 1
            if out_dtype == np.int16 and r >= 1 << 15:
                r -= 1 << 16
        out[i] = r
    return out


@pytest.mark.parametrize("scale", [1.0, 1 / 255, 0.5, 0.75, 3.0, 2.0 ** -10, 1 / 3, 0.0, 65536.0])
@pytest.mark.parametrize("fmts", [(np.uint8, np.uint8, np.uint8), (np.uint8, np.int16, np.int16),
                                  (np.int16, np.int16, np.int16)])
def test_multiply_exact_rounding(orc, scale, fmts):
    ta, tb, to = fmts
    rng = np.random.default_rng(7)
    a = (rng.integers(0, 256, (9, 11)) if ta == np.uint8
         else rng.integers(-32768, 32768, (9, 11))).astype(ta)
    b = (rng.integers(0, 256, (9, 11)) if tb == np.uint8
         else rng.integers(-32768, 32768, (9, 11))).astype(tb)
    for sat in (True, False):
        for ne in (False, True):
            got = orc.multiply(a, b, scale, to, sat, ne).data
            np.testing.assert_array_equal(got, _mul_exact(a, b, scale, to, sat, ne))


def test_multiply_ties_and_signs(orc):
    a = np.array([[3, 5, -3, -5, 7]], np.int16)
    one = np.ones_like(a)
    half_even = orc.multiply(a, one, 0.5, np.int16, True, True).data[0].tolist()
    half_zero = orc.multiply(a, one, 0.5, np.int16, True, False).data[0].tolist()
    assert half_even == [2, 2, -2, -2, 4]   # 1.5, 2.5, -1.5, -2.5, 3.5 to even
    assert half_zero == [1, 2, -1, -2, 3]
    big = np.array([[255]], np.uint8)
    assert orc.multiply(big, big, 1.0, np.uint8, True).data[0, 0] == 255
    assert orc.multiply(big, big, 1.0, np.uint8, False).data[0, 0] == (255 * 255) & 0xFF


# --- Global operators (Table 2 reduce / histogram) ---------------------------

@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_mean_stddev_against_numpy(orc, dtype):
    rng = np.random.default_rng(3)
    a = (rng.integers(0, 256, (37, 53)) if dtype == np.uint8
         else rng.integers(-32768, 32768, (37, 53))).astype(dtype)
    mean, std, (s1, s2, n) = orc.mean_stddev(a)
    wide = a.astype(np.int64)
    assert (s1, s2, n) == (int(wide.sum()), int((wide * wide).sum()), a.size)
    assert mean == np.float32(np.mean(wide, dtype=np.float64))
    assert abs(std - np.std(wide.astype(np.float64))) <= 2e-7 * max(1.0, std)
    # a valid rectangle restricts the traversal
    m2, s2_, (t1, _, t3) = orc.mean_stddev(orc.Img(a, (5, 7, 40, 30)))
    assert (t1, t3) == (int(wide[7:30, 5:40].sum()), 35 * 23)


def test_mean_stddev_closed_forms(orc):
    c = np.full((9, 9), 77, np.uint8)
    assert orc.mean_stddev(c)[:2] == (77.0, 0.0)
    two = np.array([[10, 30] * 8] * 4, np.uint8)   # half 10, half 30
    assert orc.mean_stddev(two)[:2] == (20.0, 10.0)
    assert orc.mean_stddev(orc.Img(c, (3, 3, 3, 3)))[:2] == (0.0, 0.0)  # empty


@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_minmaxloc_against_numpy(orc, dtype):
    rng = np.random.default_rng(11)
    a = (rng.integers(0, 256, (41, 29)) if dtype == np.uint8
         else rng.integers(-500, 500, (41, 29))).astype(dtype)
    r = orc.minmaxloc(a)
    assert r["min"] == a.min() and r["max"] == a.max()
    assert r["min_count"] == (a == a.min()).sum() and r["max_count"] == (a == a.max()).sum()
    iy, ix = np.unravel_index(np.argmin(a), a.shape)    # argmin: first occurrence
    assert r["min_loc"] == (ix, iy)
    iy, ix = np.unravel_index(np.argmax(a), a.shape)
    assert r["max_loc"] == (ix, iy)
    sub = orc.minmaxloc(orc.Img(a, (4, 6, 20, 33)))
    s = a[6:33, 4:20]
    iy, ix = np.unravel_index(np.argmax(s), s.shape)
    assert sub["max"] == s.max() and sub["max_loc"] == (ix + 4, iy + 6)


@pytest.mark.parametrize("nb,off,rng_", [(256, 0, 256), (16, 0, 256), (3, 0, 256), (10, 50, 100),
                                         (7, 200, 56), (1, 0, 1)])
def test_histogram_against_numpy(orc, nb, off, rng_):
    a = synth.uniform_u8(61, 47, seed=nb + off)
    got = orc.histogram(a, nb, off, rng_)
    want, _ = np.histogram(a, bins=nb, range=(off, off + rng_))
    # numpy's last bin is closed on the right: drop the value offset + range
    if off + rng_ <= 255:
        want[-1] -= int((a == off + rng_).sum())
    np.testing.assert_array_equal(got, want)
    assert got.sum() == ((a >= off) & (a < off + rng_)).sum()


def test_equalize_hist_closed_forms_and_brute_force(orc):
    c = np.full((6, 7), 123, np.uint8)
    assert (orc.equalize_hist(c).data == c).all()            # constant: unchanged
    two = np.array([[40, 90] * 5] * 3, np.uint8)
    e = orc.equalize_hist(two).data
    assert set(np.unique(e)) == {0, 255}                      # two levels spread to the extremes
    ramp = np.repeat(np.arange(256, dtype=np.uint8)[None, :], 3, axis=0)
    assert (orc.equalize_hist(ramp).data == ramp).all()       # flat histogram: identity
    a = synth.uniform_u8(13, 9, seed=2) // 16 * 16 + 3
    out = orc.equalize_hist(a).data
    n = a.size
    cmin = (a <= a.min()).sum()
    for v in np.unique(a):                                     # rank form of the definition
        cv = int((a <= v).sum())
        want = ((cv - cmin) * 255 * 2 + (n - cmin)) // (2 * (n - cmin))
        assert (out[a == v] == want).all()
    assert (np.diff(out.ravel()[np.argsort(a.ravel(), kind="stable")].astype(int)) >= 0).all()


# --- ConvertDepth / Copy (Table 2 point operators) ---------------------------

def test_convert_depth_exhaustive(orc):
    u8 = np.arange(256, dtype=np.uint8).reshape(16, 16)
    s16 = np.arange(-32768, 32768, dtype=np.int64).astype(np.int16).reshape(256, 256)
    for shift in range(8):
        up = orc.convert_depth(u8, np.int16, shift).data
        assert (up.astype(np.int64) == u8.astype(np.int64) * 2 ** shift).all()
        down_sat = orc.convert_depth(s16, np.uint8, shift, True).data.astype(np.int64)
        down_wrap = orc.convert_depth(s16, np.uint8, shift, False).data.astype(np.int64)
        q = np.floor_divide(s16.astype(np.int64), 2 ** shift)   # floor, also for negatives
        assert (down_sat == np.clip(q, 0, 255)).all()
        assert (down_wrap == np.mod(q, 256)).all()
    assert (orc.convert_depth(u8, np.uint8).data == u8).all()          # Copy
    assert (orc.convert_depth(s16, np.int16).data == s16).all()
    with pytest.raises(Exception):
        orc.convert_depth(u8, np.int16, 8)


# --- User-defined operators (Section 5.1) -----------------------------------

def test_user_expression_semantics_are_c():
    from oracle import user_ops as U
    one = np.ones((1, 1), np.int64)

    def ev(expr, a=0, b=0, dtype=np.int32):
        return int(U.user_point(expr, [one * a, one * b], dtype).data[0, 0])

    assert ev("1 + 2 * 3") == 7
    assert ev("a & 2 == 2", a=6) == 0            # C: 6 & (2 == 2); not (6 & 2) == 2
    assert ev("1 << 2 + 1") == 8
    assert ev("-a >> 1", a=3) == -2              # arithmetic shift: floor
    assert ev("~0") == -1
    assert ev("(a < b) * 10 + (a == b)", a=2, b=5) == 10
    assert ev("min(a, b) - max(a, b) + abs(0 - 7)", a=9, b=4) == 2
    assert ev("a * 100", a=3, dtype=np.uint8) == 255     # saturated to U8
    assert ev("a - 1000", a=3, dtype=np.uint8) == 0
    assert ev("a * a * a", a=40000, dtype=np.int32) == 2 ** 31 - 1


@pytest.mark.parametrize("border,mode", [(O.BORDER_REPLICATE, "nearest"),
                                         (O.BORDER_MIRROR, "reflect"), (O.BORDER_REPEAT, "wrap"),
                                         (O.BORDER_CONSTANT, "constant")])
def test_user_local_matches_scipy(border, mode):
    from oracle import user_ops as U
    img = synth.uniform_u8(23, 17, seed=5)
    a = img.astype(np.int64)
    r = U.user_local("2 * in(-1, 0) - in(1, 1) + in(0, -2)", img, 3, 5, border, 9, np.int16)
    k = np.zeros((5, 3), np.int64)
    k[2, 0] += 2
    k[3, 2] -= 1
    k[0, 1] += 1
    want = ndi.correlate(a, k, mode=mode, cval=9)
    assert (r.data == want).all() and r.rect == (0, 0, 23, 17)
    mx = U.user_local("max(max(in(-1, 0), in(1, 0)), in(0, 0))", img, 3, 1, border, 9, np.uint8)
    assert (mx.data == ndi.maximum_filter(img, size=(1, 3), mode=mode, cval=9)).all()


def test_user_local_undefined_shrinks():
    from oracle import user_ops as U
    img = synth.uniform_u8(11, 9, seed=6)
    r = U.user_local("in(-2, -1) + in(2, 1)", img, 5, 3, O.BORDER_UNDEFINED, 0, np.int16)
    assert r.rect == (2, 1, 9, 8)
    a = img.astype(np.int64)
    assert (r.data[1:8, 2:9] == a[0:7, 0:7] + a[2:9, 4:11]).all()
    assert (r.data[0] == 0).all() and (r.data[:, :2] == 0).all()
