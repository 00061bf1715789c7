"""The degree-18 evaluation scheme of the exponential (five matrix products).

The coefficients in csrc/taylor18.h must make B2 + (B3 + A9) A9, with
A9 = B1 B5 + B4, equal to the Taylor polynomial sum_{k<=18} A^k/k!.  Checked in
exact rational arithmetic from the stored doubles, so the check is independent
of any floating-point evaluation order."""
import math
import os
import re
from fractions import Fraction

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2411_09982_gb300", "csrc", "taylor18.h")


def coefficients():
    text = open(HEADER).read()
    body = text[text.index("{", text.index("kTaylor18")) + 1:text.index("};")]
    vals = [float(v) for v in re.findall(r"(-?[0-9][0-9.eE+-]*)\s*,", body)]
    assert len(vals) == 24
    return [Fraction(v) for v in vals]


def series(c, pows):
    a = [Fraction(0)] * 19
    for v, k in zip(c, pows):
        a[k] += v
    return a


def mul(a, b):
    out = [Fraction(0)] * 37
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def test_scheme_reproduces_taylor_coefficients():
    x = coefficients()
    P5 = [0, 1, 2, 3, 6]
    B1 = series(x[0:4], [0, 1, 2, 3])
    B5, B4, B3, B2 = (series(x[q:q + 5], P5) for q in (4, 9, 14, 19))
    A9 = [p + q for p, q in zip(mul(B1, B5)[:19], B4)]
    assert all(v == 0 for v in mul(B1, B5)[19:])          # A9 has degree <= 9
    full = mul([p + q for p, q in zip(B3, A9)], A9)
    assert all(v == 0 for v in full[19:])                  # T has degree <= 18
    T = [p + q for p, q in zip(B2, full[:19])]
    for k in range(19):
        rel = abs(T[k] * math.factorial(k) - 1)
        assert rel < Fraction(1, 10**15), (k, float(rel))


def test_header_is_what_the_derivation_script_writes():
    pytest = __import__("pytest")
    pytest.importorskip("mpmath")
    import importlib.util
    path = os.path.join(os.path.dirname(__file__), "..", "paper_2411_09982_gb300", "taylor18_coefficients.py")
    spec = importlib.util.spec_from_file_location("taylor18_coefficients", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    rounded, worst = mod.derive()
    assert [Fraction(v) for v in rounded] == coefficients()
    assert worst < 1e-15
