"""The corner kernels keep their vertical 5-sums of gx^2, gy^2 and gx gy as
binary32 and turn them into integers through bit patterns.  That is exact
only inside the ranges the products of a 3x3 Sobel of bytes allow; these
tests pin the ranges and the conversion on the CPU:

* |gx gy| <= 765^2 for every 3x3 byte patch (gx = 2 e1 + u + v and
  gy = 2 e2 + u - v with e1, e2, u, v differences of distinct bytes), by the
  closed form over all (u, v) and by brute force on random and extremal
  patches, while gx^2, gy^2 reach 1020^2;
* five-row sums of such products (at most 5 * 1020^2 and 5 * 765^2 in
  magnitude) are exact in binary32 under any order of additions and
  subtractions, and v + 2^23 (squares) / v + 1.5 * 2^23 (cross products) has
  the bit pattern 0x4B000000 + v / 0x4B400000 + v over the whole range."""
import numpy as np

F32 = np.float32


def sobel(p):
    """gx, gy of 3x3 patches p[..., 3, 3] (int64)."""
    w = np.array([1, 2, 1], np.int64)
    gx = ((p[..., :, 2] - p[..., :, 0]) * w).sum(-1)
    gy = ((p[..., 2, :] - p[..., 0, :]) * w).sum(-1)
    return gx, gy


def test_cross_product_bound_closed_form():
    # for fixed u, v the largest |gx gy| takes e1, e2 = +-255:
    # (510 + |u + v|) (510 + |u - v|) <= 765^2, equality at |u| = 255, v = 0 (or u = 0,
    # |v| = 255)
    u, v = np.meshgrid(np.arange(-255, 256), np.arange(-255, 256))
    m = (510 + np.abs(u + v)) * (510 + np.abs(u - v))
    assert m.max() == 765 ** 2


def test_cross_product_bound_brute_force():
    rng = np.random.default_rng(3)
    p = rng.integers(0, 256, (400000, 3, 3)).astype(np.int64)
    p[:1000] = rng.choice([0, 255], (1000, 3, 3))  # extremal patches
    gx, gy = sobel(p)
    assert np.abs(gx * gy).max() <= 765 ** 2
    assert np.abs(gx).max() <= 1020 and np.abs(gy).max() <= 1020
    # the bound is reached: the corner patch of the closed form
    c = np.array([[0, 0, 255], [0, 0, 255], [255, 255, 255]], np.int64)
    gxc, gyc = sobel(c)
    assert gxc * gyc == 765 ** 2
    edge = np.array([[0, 0, 255]] * 3, np.int64)
    assert sobel(edge)[0] == 1020


def _pattern_check(v, magic, bits):
    got = (F32(v.astype(np.float64)) + F32(magic)).view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(got - bits, v)


def test_bit_patterns_over_the_whole_ranges():
    sq = np.arange(0, 5 * 1020 ** 2 + 1, dtype=np.int64)
    _pattern_check(sq, 2.0 ** 23, 0x4B000000)
    xy = np.arange(-5 * 765 ** 2, 5 * 765 ** 2 + 1, dtype=np.int64)
    _pattern_check(xy, 1.5 * 2.0 ** 23, 0x4B400000)
    # one step past the ranges the patterns would break
    assert 5 * 1020 ** 2 < 2 ** 23 and 5 * 765 ** 2 < 2 ** 22
    bad = np.array([2 ** 23 + 1], np.int64)
    got = (F32(bad.astype(np.float64)) + F32(2.0 ** 23)).view(np.uint32).astype(np.int64)
    assert got[0] - 0x4B000000 != bad[0]


def test_five_row_sums_exact_in_binary32():
    # random sliding windows: add the entering row's products, subtract the
    # leaving one's, in binary32 (each step rounded), against int64
    rng = np.random.default_rng(9)
    n, steps = 20000, 40
    g = rng.integers(-1020, 1021, (steps + 5, n, 2)).astype(np.int64)
    g[:, : n // 10] = rng.choice([-1020, 1020], (steps + 5, n // 10, 2))
    prod = g[..., 0] * g[..., 0]
    acc32 = np.zeros(n, F32)
    acc = np.zeros(n, np.int64)
    for t in range(steps + 5):
        acc32 = F32(acc32 + F32(prod[t]))
        acc += prod[t]
        if t >= 5:
            acc32 = F32(acc32 - F32(prod[t - 5]))
            acc -= prod[t - 5]
        np.testing.assert_array_equal(acc32.astype(np.int64), acc)
