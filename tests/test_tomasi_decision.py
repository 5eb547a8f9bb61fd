"""The BORDER_UNDEFINED corner kernel decides r > T for the binary32 Shi-Tomasi
response r = tomasi_response_f32(a, b, c) (2 det / (tr + sqrt(disc)), IEEE
square root and division) from a cheaper estimate r' when r' is farther than
2^-19 r' from T.  r' replaces the square root by disc * rsqrt(disc) and the
division by a multiplication with rcp(den), two hardware approximations with
relative errors of at most 2^-22.9 and 2^-23 (PTX rsqrt.approx / rcp.approx).

This file replays both computations with numpy float32 (IEEE, round to
nearest), the approximations modelled as the exact reciprocal (square root)
times 1 + e for each extreme e, and checks that |r - r'| stays well inside
the decision margin 2^-19 r' on window sums of squares and cross products of
random, edge-like, corner-like and degenerate 5x5 gradient windows."""
import numpy as np

F32 = np.float32
E_RSQ = 2.0 ** -22.9
E_RCP = 2.0 ** -23


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


def estimates(a, b, c):
    """r' for each combination of extreme approximation errors."""
    det = a * b - c * c
    disc = F32((a - b) * (a - b) + 4 * c * c)
    out = []
    for e1 in (-E_RSQ, E_RSQ):
        for e2 in (-E_RCP, E_RCP):
            rs = F32(1.0 / np.sqrt(float(disc)) * (1 + e1)) if disc > 0 else F32(np.inf)
            with np.errstate(invalid="ignore"):
                den = F32(F32(a + b) + F32(disc * rs))
                rc = F32(1.0 / float(den) * (1 + e2)) if den > 0 else F32(np.inf)
                out.append(F32(F32(F32(2) * F32(det)) * rc))
    return out


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


def test_estimate_within_margin():
    rng = np.random.default_rng(7)
    worst = 0.0
    for a, b, c in windows(rng, 20000):
        assert a * b >= c * c and a < 2 ** 25 and b < 2 ** 25
        r = response(a, b, c)
        for rp in estimates(a, b, c):
            if np.isnan(rp):  # disc = 0: the kernel takes r itself
                continue
            assert rp >= 0
            gap = abs(float(r) - float(rp))
            if rp > 0:
                worst = max(worst, gap / float(rp))
            else:
                assert r == 0
    # the decision margin is 2^-19 r'; the replayed error (about 2^-21 at
    # worst) stays below half of it
    assert worst < 2.0 ** -20, worst


def test_decisions_next_to_the_threshold():
    # thresholds at r and its binary32 neighbours: whenever the estimate
    # decides (gap above 2^-19 r'), it agrees with r > T
    rng = np.random.default_rng(11)
    for a, b, c in windows(rng, 3000):
        r = response(a, b, c)
        for T in (r, np.nextafter(r, F32(np.inf)), np.nextafter(r, F32(-np.inf)),
                  F32(float(r) * (1 + 2.0 ** -18)), F32(float(r) * (1 - 2.0 ** -18))):
            for rp in estimates(a, b, c):
                if np.isnan(rp):
                    continue
                g = F32(rp * F32(2.0 ** -19))
                if F32(rp - T) > g:
                    assert r > T
                elif F32(T - rp) > g:
                    assert not r > T


def test_degenerate_windows():
    # all-zero window: disc = 0, the estimate is NaN and the kernel takes r = 0;
    # collinear gradients: det = 0 and both r and r' are exactly 0
    assert response(0, 0, 0) == 0
    assert all(np.isnan(x) for x in estimates(0, 0, 0))
    a, b, c = 25 * 9, 25 * 4, 25 * 6  # gx = 3, gy = 2 everywhere
    assert a * b == c * c
    assert response(a, b, c) == 0
    assert all(x == 0 for x in estimates(a, b, c))
