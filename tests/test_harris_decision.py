"""The BORDER_UNDEFINED Harris kernel decides q > q_thr (q = kd (a b - c^2) -
kn (a + b)^2, the exact integer form of R > T) in binary32 when the computed
value is farther from the threshold than an error bound, and exactly in 64-bit
integers otherwise, two pixels per packed (f32x2) operation.  This file
replays that binary32 procedure operation by
operation (numpy float32 arithmetic is IEEE round-to-nearest; each fused
multiply-add is rounded once from its exact value) and checks that every
decision it takes agrees with exact integer arithmetic, on random window sums
and on thresholds placed right next to q."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def round32(x: Fraction) -> np.float32:
    """x rounded once to binary32 (nearest, ties to even)."""
    f = F32(float(x))  # at most one binary32 ulp away
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


def decide32(a, b, c, kn, kd, q_thr, kb_scale=1.0):
    """The kernel's packed binary32 decision for one pixel (each lane of a
    packed operation rounds as a scalar one would): True / False, or None
    (left to the exact test).  kb_scale shrinks the bound (planted mistake)."""
    kb = F32(F32(kd + 2 * kn) * F32(2.0 ** -19) * F32(kb_scale))
    qt = round32(Fraction(q_thr))
    qb = F32(abs(qt) * F32(2.0 ** -21) * F32(kb_scale))
    n1, n2 = -(F32(kn) + kb), -(qt + qb)
    m1, m2 = -(F32(kn) - kb), -(qt - qb)
    A, B, C = round32(Fraction(a)), round32(Fraction(b)), round32(Fraction(c))
    P = A * B
    CC = C * C
    D = fma32(CC, F32(-1), P)
    S = A + B
    S2 = S * S
    lo = fma32(F32(kd), D, fma32(S2, n1, n2))
    hi = fma32(F32(kd), D, fma32(S2, m1, m2))
    assert lo <= hi
    if min(-lo, hi) >= 0:
        return None
    return bool(lo > 0)


def exact_q(a, b, c, kn, kd):
    return kd * (a * b - c * c) - kn * (a + b) ** 2


def test_decision_matches_exact_arithmetic():
    rng = np.random.default_rng(7)
    undecided = 0
    n = 0
    for trial in range(3000):
        scale = 2 ** int(rng.integers(4, 26))
        a = int(rng.integers(0, min(scale, 2 ** 25)))
        b = int(rng.integers(0, min(scale, 2 ** 25)))
        lim = int(np.sqrt(a * b))
        c = int(rng.integers(-lim, lim + 1)) if lim > 0 else 0
        kn, kd = [(1, 25), (3, 50), (1, 1), (7, 1000)][trial % 4]
        q = exact_q(a, b, c, kn, kd)
        # thresholds far away, close, and right next to q
        for q_thr in (q - 10 ** 12, q - 10 ** 6, q - 1, q, q + 1, q + 10 ** 6,
                      int(25e6 * kd / 25), -5):
            n += 1
            got = decide32(a, b, c, kn, kd, q_thr)
            if got is None:
                undecided += 1
                continue
            assert got == (q > q_thr), (a, b, c, kn, kd, q_thr)
    # the exact path is taken only next to the threshold
    assert undecided < 0.5 * n


def test_planted_tighter_bound_fails():
    # with the bound 2^10 times smaller the procedure must err somewhere: the
    # check above has teeth
    rng = np.random.default_rng(3)
    wrong = 0
    for _ in range(1500):
        a = int(rng.integers(2 ** 23, 2 ** 25))
        b = int(rng.integers(2 ** 23, 2 ** 25))
        lim = int(np.sqrt(a * b))
        c = int(rng.integers(-lim, lim + 1))
        q = exact_q(a, b, c, 1, 25)
        for q_thr in (q - 10 ** 6, q + 10 ** 6):
            got = decide32(a, b, c, 1, 25, q_thr, kb_scale=2.0 ** -10)
            if got is not None and got != (q > q_thr):
                wrong += 1
    assert wrong > 0
