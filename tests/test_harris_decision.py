"""The BORDER_UNDEFINED Harris kernel decides q > q_thr (q = kd (a b - c^2) -
kn (a + b)^2, the exact integer form of R > T) in binary32 when the computed
value is farther from the threshold than an error bound, and exactly in 64-bit
integers otherwise.  This file replays that binary32 procedure operation by
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


def decide32(a, b, c, kn, kd, q_thr):
    """The kernel's binary32 decision: True / False, or None (exact path)."""
    A, B, C = F32(a), F32(b), F32(c)
    knf, kdf = F32(kn), F32(kd)
    qtf = F32(float(q_thr))
    qtb = F32(abs(qtf) * F32(2.0 ** -21))
    P = A * B
    D = fma32(-C, C, P)
    S = A + B
    V = knf * (S * S)
    Q = fma32(kdf, D, -V)
    M = fma32(kdf, fma32(C, C, P), V)
    bound = fma32(F32(2.0 ** -19), M, qtb)
    d = Q - qtf
    if abs(d) > bound:
        return bool(d > 0)
    return None


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
    # with a bound 2^10 times smaller the procedure must err somewhere: the
    # check above has teeth
    rng = np.random.default_rng(3)
    wrong = 0
    for _ in range(4000):
        a = int(rng.integers(2 ** 23, 2 ** 25))
        b = int(rng.integers(2 ** 23, 2 ** 25))
        lim = int(np.sqrt(a * b))
        c = int(rng.integers(-lim, lim + 1))
        q = exact_q(a, b, c, 1, 25)
        for q_thr in (q - 10 ** 6, q + 10 ** 6):
            A, B, C = F32(a), F32(b), F32(c)
            P = A * B
            D = fma32(-C, C, P)
            S = A + B
            V = F32(1) * (S * S)
            Q = fma32(F32(25), D, -V)
            d = Q - F32(float(q_thr))
            if d != 0 and bool(d > 0) != (q > q_thr):
                wrong += 1
    assert wrong > 0
