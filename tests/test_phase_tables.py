"""The constants of the fused edge kernel's Phase evaluation (Table 2 Phase
point operator): the one-guess-plus-one-exact-test scheme of gen_phase_poly.py
is emulated bit-exactly over every integer gradient pair a Sobel3x3 of U8
input can produce, and the committed header holds what the generator makes."""
import importlib.util
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2008_11476_gb300", "csrc")


def _gen():
    pytest.importorskip("mpmath")
    spec = importlib.util.spec_from_file_location("gen_phase_poly",
                                                  os.path.join(CSRC, "gen_phase_poly.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_tan_test_exact_over_all_integer_pairs():
    g = _gen()
    bad, gap = g.verify_tan_test()
    assert bad == 0
    assert gap > 3e-5  # smallest |mn - mx tan(beta_n)| over all pairs


def test_phase_all_gradient_pairs():
    # the kernel's whole Phase path (guess, octant table, exact test) on every
    # (gx, gy) in [-1020, 1020]^2 against round(atan2(gy, gx) * 128 / pi) mod 256
    assert _gen().verify_phase_all() == 0


def test_planted_octant_table_error_is_caught():
    g = _gen()
    tan8, q_ge, q_lt = g.phase_table()
    bad = q_ge.copy()
    bad[5 * 34 + 7] = (bad[5 * 34 + 7] + 1) % 256  # one octant entry off by one bin
    assert g.verify_phase_all(table=(tan8, bad, q_lt)) > 0
    assert g.verify_phase_all(table=(tan8, q_lt, q_ge)) > 0  # outcomes swapped


def test_planted_table_error_is_caught():
    g = _gen()
    T, _ = g.tan_table()
    T2 = T.copy()
    T2[10] = np.float32(T2[10] * np.float32(1.0001))
    assert g.verify_tan_test(T=T2)[0] > 0
    A, B = g.fit_guess()
    assert g.verify_tan_test(A=np.float32(40.7), B=np.float32(-8.0))[0] > 0


def test_header_matches_generator():
    g = _gen()
    with open(os.path.join(CSRC, "phase_table.h")) as f:
        text = f.read()
    body = re.search(r"kPhaseTan\[34\] = \{(.*?)\};", text, re.S).group(1)
    vals = np.array([float(v.rstrip("f")) for v in re.findall(r"-?[0-9.e+-]+f", body)],
                    np.float32)
    T, _ = g.tan_table()
    assert vals.shape == (34,) and np.array_equal(vals, T)
    A, B = g.fit_guess()
    assert np.float32(float(re.search(r"kPhaseGuessA = (\S+)f;", text).group(1))) == A
    assert np.float32(float(re.search(r"kPhaseGuessB = (\S+)f;", text).group(1))) == B
