"""The chunk build's Rodrigues coefficients (csrc/track.cu, so3_exp_d with
SERIES): a = sin(th)/th and b = (1 - cos th)/th^2 from their Taylor series
in th^2 up to th = 1 rad.  Checked on the host against the mathematics: the
coefficient tables are (-1)^n/(2n+1)! and (-1)^n/(2n+2)! rounded to double,
the first omitted terms are below 1e-17 at th = 1, and the Horner sums in
double agree with the closed form to a few ulp over (0, 1]."""
import math
import os
import re
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tables():
    src = open(os.path.join(ROOT, "paper_2509_24236_gb300", "csrc", "track.cu")).read()
    out = {}
    for name in ("ca", "cb"):
        m = re.search(r"const double " + name + r"\[9\] = \{([^}]*)\}", src)
        assert m, name
        out[name] = [float(v) for v in m.group(1).replace("\n", " ").split(",")]
    return out["ca"], out["cb"]


def test_coefficients_are_the_series_terms():
    ca, cb = _tables()
    for n in range(9):
        assert ca[n] == float(Fraction((-1) ** n, math.factorial(2 * n + 1))), n
        assert cb[n] == float(Fraction((-1) ** n, math.factorial(2 * n + 2))), n
    # the first omitted terms at th^2 = 1, against the smallest values of a and b there
    assert 1.0 / math.factorial(19) < 1e-17 * math.sin(1.0)
    assert 1.0 / math.factorial(20) < 1e-17 * (1.0 - math.cos(1.0))


def test_horner_sums_match_the_closed_form():
    ca, cb = _tables()
    th = np.concatenate([np.linspace(1e-3, 1.0, 2001), np.geomspace(1e-12, 1e-3, 200)])
    x = th * th
    a = np.full_like(x, ca[8])
    b = np.full_like(x, cb[8])
    for n in range(7, -1, -1):
        a = a * x + ca[n]
        b = b * x + cb[n]
    a_ref = np.sin(th) / th
    # 1 - cos(th) without cancellation: 2 sin^2(th/2)
    b_ref = 2.0 * np.sin(0.5 * th) ** 2 / x
    assert np.max(np.abs(a / a_ref - 1.0)) < 1e-15
    assert np.max(np.abs(b / b_ref - 1.0)) < 1e-15
