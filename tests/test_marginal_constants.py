"""The mixed-precision distance marginal evaluates ln I0(x) - x per quadrature node from the
polynomial approximations of Abramowitz & Stegun 9.8.1 (x < 3.75) and 9.8.2 (x >= 3.75).
Their coefficients are read here from the CUDA header itself and checked against scipy's
exponentially scaled Bessel function, so a mistyped constant fails on the CPU."""
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2410_05190_gb300", "csrc",
                      "marg.cuh")


def _function_body(src, name):
    start = src.index(f"float {name}(")
    depth, i = 0, src.index("{", start)
    for j in range(i, len(src)):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        if depth == 0:
            return src[i:j + 1]
    raise AssertionError("unbalanced braces")


def _coefficients():
    body = _function_body(open(HEADER).read(), "log_i0_minus_x_f")
    small, large = body.split("const float t = __fdividef")
    num = r"(-?\d+\.\d+)f"
    # Horner nests innermost first: fmaf(t, 0.0045813f, 0.0360768f) -> highest degree first
    cs = [float(v) for v in re.findall(num, small.split("const float p =", 1)[1].split(";", 1)[0])]
    cl = [float(v) for v in re.findall(num, large.split("const float p =", 1)[1].split(";", 1)[0])]
    return cs[::-1], cl[::-1]


def _horner(coef_low_first, t):
    p = np.zeros_like(t)
    for c in coef_low_first[::-1]:
        p = p * t + c
    return p


def test_abramowitz_stegun_i0_constants_in_the_header():
    special = pytest.importorskip("scipy.special")
    cs, cl = _coefficients()
    assert len(cs) == 7 and cs[0] == 1.0, cs          # 9.8.1: 1 + 3.5156229 t^2 + ... (t = x / 3.75)
    assert len(cl) == 9 and abs(cl[0] - 1 / np.sqrt(2 * np.pi)) < 1e-8, cl   # 9.8.2 -> (2 pi)^(-1/2)
    x = np.linspace(1e-6, 3.75, 20001)
    got = np.log(_horner(cs, (x / 3.75) ** 2)) - x
    assert np.abs(got - np.log(special.i0e(x))).max() < 1e-7
    x = np.concatenate([np.linspace(3.75, 100.0, 20001), np.geomspace(100.0, 1e7, 2001)])
    got = np.log(_horner(cl, 3.75 / x)) - 0.5 * np.log(x)
    assert np.abs(got - np.log(special.i0e(x))).max() < 6e-7
