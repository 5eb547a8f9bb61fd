"""The BORDER_UNDEFINED corner kernel decides r > T for the binary32 Shi-Tomasi
response r = tomasi_response_f32(a, b, c) (2 det / (tr + sqrt(disc)), exact
integer det and disc, IEEE square root and division) two pixels per packed
binary32 operation: with A, B, C, E the sums a, b, c and a - b rounded to
binary32,
    h = D rcp(den) - T / 2,  D = A B - C^2,  den = S + disc rsqrt(disc),
    S = A + B,  disc = (2C)^2 + (E^2 + 2^-100),
lo = h - 2^-20 S and hi = h + 2^-20 S; lo > 0 decides r > T, hi < 0 decides
r < T, and the exact response decides the rest.  rsqrt and rcp are hardware
approximations with relative errors of at most 2^-22.9 and 2^-23 (PTX
rsqrt.approx / rcp.approx).

This file replays the procedure operation by operation (each multiply, add and
fused multiply-add rounded once to binary32 from its exact value), the
approximations modelled as the exact reciprocal (square root) times 1 + e for
each extreme e, and checks every decision it takes against r > T on window
sums of random, edge-like, corner-like, flat and degenerate 5x5 gradient
windows, with thresholds at r and right next to it."""
from fractions import Fraction

import numpy as np

F32 = np.float32
E_RSQ = 2.0 ** -22.9
E_RCP = 2.0 ** -23
K = 2.0 ** -20


def round32(x: Fraction) -> np.float32:
    """x rounded once to binary32 (nearest, ties to even)."""
    f = F32(float(x))
    lo, hi = f, f
    for _ in range(2):
        lo = np.nextafter(lo, F32(-np.inf))
        hi = np.nextafter(hi, F32(np.inf))
    best, bd = None, None
    v = lo
    while v <= hi:
        d = abs(Fraction(float(v)) - x)
        if bd is None or d < bd or (d == bd and (int(v.view(np.uint32)) & 1) == 0):
            best, bd = v, d
        v = np.nextafter(v, F32(np.inf))
    return best


def fma32(x, y, z) -> np.float32:
    return round32(Fraction(float(x)) * Fraction(float(y)) + Fraction(float(z)))


def mul32(x, y) -> np.float32:
    return fma32(x, y, 0.0)


def response(a, b, c):
    """The binary32 response as the kernels compute it (all values exact ints)."""
    det = a * b - c * c
    disc = (a - b) * (a - b) + 4 * c * c
    s = np.sqrt(F32(disc))
    tr = F32(a + b)
    den = F32(tr + s)
    if den == 0:
        return tr
    return F32(F32(2) * F32(det) / den)


def bracket(a, b, c, T, e_rsq, e_rcp, k=K):
    """(lo, hi) of the kernel's packed procedure for one pixel, with the
    hardware approximations off by the relative errors e_rsq and e_rcp."""
    A, B, C = round32(Fraction(a)), round32(Fraction(b)), round32(Fraction(c))
    E = round32(Fraction(a - b))
    D = fma32(mul32(C, C), -1.0, mul32(A, B))
    S = round32(Fraction(float(A)) + Fraction(float(B)))
    C2 = round32(2 * Fraction(float(C)))
    disc = fma32(C2, C2, fma32(E, E, 2.0 ** -100))
    rs = F32(1.0 / np.sqrt(float(disc)) * (1 + e_rsq))
    den = fma32(disc, rs, S)
    rc = F32(1.0 / float(den) * (1 + e_rcp))
    h = fma32(D, rc, F32(-0.5 * F32(T)))
    return fma32(S, -F32(k), h), fma32(S, F32(k), h)


def decide(a, b, c, T, e_rsq, e_rcp, k=K):
    lo, hi = bracket(a, b, c, T, e_rsq, e_rcp, k)
    assert lo <= hi
    if min(-lo, hi) >= 0:
        return None
    return bool(lo > 0)


def windows(rng, n):
    for k in range(n):
        kind = k % 4
        if kind == 0:    # texture
            gx = rng.integers(-1020, 1021, 25)
            gy = rng.integers(-1020, 1021, 25)
        elif kind == 1:  # straight edge: gy proportional to gx, det near 0
            gx = rng.integers(-1020, 1021, 25)
            gy = (gx * rng.integers(-3, 4)) // 3 + rng.integers(-1, 2, 25)
        elif kind == 2:  # corner: two orientations
            gx = np.where(rng.random(25) < 0.5, rng.integers(300, 1021, 25), 0)
            gy = np.where(gx == 0, rng.integers(300, 1021, 25), 0)
        else:            # flat with noise of a few levels
            gx = rng.integers(-8, 9, 25)
            gy = rng.integers(-8, 9, 25)
        gx, gy = np.clip(gx, -1020, 1020), np.clip(gy, -1020, 1020)
        yield (int(np.sum(gx * gx)), int(np.sum(gy * gy)), int(np.sum(gx * gy)))




ERRS = [(e1, e2) for e1 in (-E_RSQ, E_RSQ) for e2 in (-E_RCP, E_RCP)]


def test_decisions_next_to_the_threshold():
    # thresholds at r, its binary32 neighbours, a few relative steps away and
    # beyond the undecided band: whenever the bracket decides, it agrees with
    # r > T; thresholds beyond the band are decided
    rng = np.random.default_rng(11)
    undecided = far_undecided = 0
    for a, b, c in windows(rng, 600):
        assert a * b >= c * c and a < 2 ** 25 and b < 2 ** 25
        r = response(a, b, c)
        near = (r, np.nextafter(r, F32(np.inf)), np.nextafter(r, F32(-np.inf)),
                F32(float(r) * (1 + 2.0 ** -18)), F32(float(r) * (1 - 2.0 ** -18)))
        # the undecided band is |r - T| <= 2 K (a + b) (plus rounding)
        band = 2 * K * (a + b)
        far = (F32(float(r) * 1.001 + 2 * band + 1), F32(float(r) * 0.999 - 2 * band - 1))
        for T in near + far:
            for e1, e2 in ERRS:
                got = decide(a, b, c, T, e1, e2)
                if got is None:
                    undecided += 1
                    far_undecided += T in far
                    continue
                assert got == bool(r > T), (a, b, c, float(T), e1, e2)
    assert far_undecided == 0
    assert undecided > 0  # the thresholds at r itself are left to the exact test


def test_bracket_margin_holds_on_random_windows():
    # the replayed h stays within half of the margin K S of r / 2 - T / 2
    rng = np.random.default_rng(7)
    worst = 0.0
    for a, b, c in windows(rng, 1500):
        r = float(response(a, b, c))
        for e1, e2 in ERRS:
            lo, hi = bracket(a, b, c, 0.0, e1, e2)
            h = (float(lo) + float(hi)) / 2
            if a + b > 0:
                worst = max(worst, abs(h - r / 2) / (K * (a + b)))
    assert worst < 0.5, worst


def test_planted_smaller_margin_fails():
    # with the margin 2^8 times smaller the bracket must err somewhere near the
    # threshold: the checks above have teeth
    rng = np.random.default_rng(5)
    wrong = 0
    for a, b, c in windows(rng, 400):
        r = response(a, b, c)
        for T in (np.nextafter(r, F32(np.inf)), np.nextafter(r, F32(-np.inf))):
            for e1, e2 in ERRS:
                got = decide(a, b, c, T, e1, e2, k=K * 2.0 ** -8)
                if got is not None and got != bool(r > T):
                    wrong += 1
    assert wrong > 0


def test_degenerate_windows():
    # all-zero window: disc and den stay positive, D = 0, h = -T / 2 exactly;
    # collinear gradients: det = 0 and r = 0
    assert response(0, 0, 0) == 0
    for e1, e2 in ERRS:
        assert decide(0, 0, 0, 5.0, e1, e2) is False
        assert decide(0, 0, 0, -5.0, e1, e2) is True
        assert decide(0, 0, 0, 0.0, e1, e2) is None
    a, b, c = 25 * 9, 25 * 4, 25 * 6  # gx = 3, gy = 2 everywhere
    assert a * b == c * c and response(a, b, c) == 0
    for e1, e2 in ERRS:
        assert decide(a, b, c, 1.0, e1, e2) is False
        assert decide(a, b, c, -1.0, e1, e2) is True
