"""CPU replays of the 16-bit-lane (SWAR) arithmetic of the hand-written
kernels' newer modes, operation by operation on uint32 words (numpy, with
32-bit wraparound), against direct definitions of what they compute:

* the 5x5 binomial row of the Convolve kernel (two pixels per 32-bit word:
  vertical then horizontal 1-4-6-4-1 sums, a shift by 8, byte packing),
  on random and saturated windows;
* the Sobel gx of the input-row mode converted to S16 lanes in registers
  ((lane >> 4) - 1024 per lane with the top-bit trick), over every gx pair;
* the Magnitude(gy, gy) -> Threshold rewrite 2 gy^2 > T^2 + T against
  round(sqrt(2 gy^2)) > T, over every gy and a range of T.

Each replay follows the kernel's steps; a planted mistake (a borrow between
lanes, a wrong weight) must fail."""
import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def u32(x):
    return np.asarray(x, np.uint64) & M32


def lo_pair(w):   # bytes 0, 1 of w as 16-bit lanes
    w = u32(w)
    return (w & 0xFF) | (((w >> 8) & 0xFF) << 16)


def hi_pair(w):   # bytes 2, 3 of w as 16-bit lanes
    w = u32(w)
    return ((w >> 16) & 0xFF) | (((w >> 24) & 0xFF) << 16)


def shift_pair(a, b):  # lane 1 of a, lane 0 of b
    return u32((u32(a) >> 16) | (u32(b) << 16))


def word(row, i):  # little-endian 32-bit word of 4 bytes starting at i
    r = row.astype(np.uint64)
    return r[..., i] | (r[..., i + 1] << 8) | (r[..., i + 2] << 16) | (r[..., i + 3] << 24)


def load_pairs(row, c):
    """Pairs (x - 2, x - 1) .. (x + 8, x + 9) of a row, the strip at column c."""
    wl, mx, my, wr = word(row, c - 4), word(row, c), word(row, c + 4), word(row, c + 8)
    return [hi_pair(wl), lo_pair(mx), hi_pair(mx), lo_pair(my), hi_pair(my), lo_pair(wr)]


def byte_perm_6420(a, b):  # bytes 0 and 2 of a, then of b
    a, b = u32(a), u32(b)
    return (a & 0xFF) | (((a >> 16) & 0xFF) << 8) | ((b & 0xFF) << 16) | (((b >> 16) & 0xFF) << 24)


def binom5_row(rows, c, w4=4, w6=6):
    """The kernel's output bytes x .. x + 7 from five input rows (y - 2 .. y + 2)."""
    P = [load_pairs(r, c) for r in rows]
    V = [u32((P[0][k] + P[4][k]) + w4 * (P[1][k] + P[3][k]) + w6 * P[2][k]) for k in range(6)]
    S = [shift_pair(V[k], V[k + 1]) for k in range(5)]
    o = [u32((V[j] + V[j + 2]) + 4 * (S[j] + S[j + 1]) + 6 * V[j + 1]) >> 8 for j in range(4)]
    lo, hi = byte_perm_6420(o[0], o[1]), byte_perm_6420(o[2], o[3])
    out = np.empty(rows[0].shape[:-1] + (8,), np.int64)
    for j in range(4):
        out[..., j] = (lo >> (8 * j)) & 0xFF
        out[..., 4 + j] = (hi >> (8 * j)) & 0xFF
    return out


def binom5_direct(rows, c):
    w = np.array([1, 4, 6, 4, 1], np.int64)
    x = np.stack([r.astype(np.int64) for r in rows], axis=-2)  # (..., 5, cols)
    out = np.empty(x.shape[:-2] + (8,), np.int64)
    for j in range(8):
        win = x[..., :, c + j - 2:c + j + 3]
        out[..., j] = np.einsum("...ij,i,j->...", win, w, w) // 256
    return out


def _windows(rng, n):
    rows = [rng.integers(0, 256, (n, 24), dtype=np.uint8) for _ in range(5)]
    rows[0][: n // 8] = 255  # saturated windows: the largest sums
    for r in rows[1:]:
        r[: n // 8] = 255
    return rows


def test_binomial_row_matches_the_convolution():
    rng = np.random.default_rng(5)
    rows = _windows(rng, 20000)
    np.testing.assert_array_equal(binom5_row(rows, 8), binom5_direct(rows, 8))


def test_binomial_row_planted_weight_fails():
    rng = np.random.default_rng(6)
    rows = _windows(rng, 2000)
    assert (binom5_row(rows, 8, w6=5) != binom5_direct(rows, 8)).any()


def gx_s16_pair(gxp, bias=0x80008000):
    t = (((u32(gxp) >> 4) & 0x0FFF0FFF) | bias)
    return u32(u32(t - 0x04000400) ^ bias)


def test_gx_to_s16_lanes_every_pair():
    g = np.arange(-1020, 1021, dtype=np.int64)
    g0, g1 = [a.ravel() for a in np.meshgrid(g, g)]
    gxp = u32((16 * g0 + 16384) | ((16 * g1 + 16384) << 16))
    w = gx_s16_pair(gxp)
    lo = (w & 0xFFFF).astype(np.int64)
    hi = ((w >> 16) & 0xFFFF).astype(np.int64)
    lo = np.where(lo >= 32768, lo - 65536, lo)
    hi = np.where(hi >= 32768, hi - 65536, hi)
    np.testing.assert_array_equal(lo, g0)
    np.testing.assert_array_equal(hi, g1)
    # without the top-bit trick a negative low lane borrows from the high one
    w_plain = u32(((u32(gxp) >> 4) & 0x0FFF0FFF) - 0x04000400)
    hi_plain = ((w_plain >> 16) & 0xFFFF).astype(np.int64)
    hi_plain = np.where(hi_plain >= 32768, hi_plain - 65536, hi_plain)
    assert (hi_plain != g1).any()


def test_sobel_gx_from_input_rows():
    # input rows times 16 in 16-bit lanes stand in for the Gaussian rows; vs =
    # a + 2b + c, gxp = vs[j + 1] + 0x40004000 - vs[j] never borrows between
    # lanes, and gx_s16_pair gives the Sobel's gx
    rng = np.random.default_rng(7)
    n = 20000
    rows = [rng.integers(0, 256, (n, 24), dtype=np.uint8) for _ in range(3)]
    for r in rows:              # steps up and down: gradients at the extremes
        r[: n // 10, :12], r[: n // 10, 12:] = 0, 255
        r[n // 10: n // 5, :12], r[n // 10: n // 5, 12:] = 255, 0
    G = []
    for r in rows:
        P = load_pairs(r, 8)
        G.append([u32(shift_pair(P[j], P[j + 1]) << 4) for j in range(5)])
    vs = [u32(G[0][j] + 2 * G[1][j] + G[2][j]) for j in range(5)]
    got = np.empty((n, 8), np.int64)
    for j in range(4):
        w = gx_s16_pair(u32(vs[j + 1] + 0x40004000 - vs[j]))
        for h in range(2):
            v = ((w >> (16 * h)) & 0xFFFF).astype(np.int64)
            got[:, 2 * j + h] = np.where(v >= 32768, v - 65536, v)
    x = np.stack([r.astype(np.int64) for r in rows], axis=1)  # (n, 3, 24)
    want = np.empty((n, 8), np.int64)
    for j in range(8):
        c = 8 + j
        col = lambda k: x[:, 0, k] + 2 * x[:, 1, k] + x[:, 2, k]
        want[:, j] = col(c + 1) - col(c - 1)
    np.testing.assert_array_equal(got, want)
    assert want.max() == 1020 and want.min() == -1020


def test_magnitude_of_gy_twice_threshold_rewrite():
    # round(sqrt(2 gy^2)) > T  <=>  2 gy^2 > T^2 + T for T >= 0 (the mask the
    # Magnitude(gy, gy) mode evaluates), every gy, T up to past the largest
    # magnitude (1442)
    gy = np.arange(-1020, 1021, dtype=np.int64)
    s = 2 * gy * gy
    mag = np.floor(np.sqrt(s.astype(np.float64)) + 0.5).astype(np.int64)
    for T in range(0, 1500):
        np.testing.assert_array_equal(s > T * T + T, mag > T)
