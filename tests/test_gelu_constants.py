"""The BF16 epilogues' GELU (gelu.cuh): erf from Abramowitz & Stegun 7.1.28 with the 1/sqrt(2)
and the factor 1/2 of GELU folded into the coefficients (each times 2^(1/16), the constant term
2^(1/16), so that the 16th power carries the factor 2).  Pinned against the exact erf form on the
host, in FP64, from the constants as written in the header."""
import math
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2312_13513_gb300",
                   "csrc", "gelu.cuh")


def _body(signature):
    text = open(HDR).read().split(signature)[1]
    return text.split("__device__ __forceinline__")[0]


def _coefficients():
    body = _body("float gelu_f(float v)")
    c = [float(x) for x in re.findall(r"([0-9]\.[0-9]+e[-+][0-9]+)f", body)]
    assert len(c) == 7
    # Horner from the highest power: fmaf(x, c6, c5), then c4 .. c1, then the constant term
    return c[6], [c[5], c[4], c[3], c[2], c[1], c[0]]      # c0', (a1' .. a6')


def test_folded_coefficients_are_the_handbook_ones_over_sqrt2_powers():
    a = [0.0705230784, 0.0422820123, 0.0092705272, 0.0001520143, 0.0002765672, 0.0000430638]
    c = 2.0 ** (1.0 / 16.0)
    c0, b = _coefficients()
    assert c0 == np.float32(c)
    for i in range(6):
        assert b[i] == np.float32(a[i] * 2.0 ** (-(i + 1) / 2) * c), i


def test_gelu_within_5e7_of_the_erf_form():
    c0, b = _coefficients()
    worst = 0.0
    for v in np.linspace(-12.0, 12.0, 48001):
        x = abs(v)
        q = c0 + sum(b[i] * x ** (i + 1) for i in range(6))
        g = max(v, 0.0) - x * q ** -16
        worst = max(worst, abs(g - 0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0)))))
    assert worst <= 5e-7, worst


def test_packed_gelu_uses_the_same_coefficients():
    """gelu2 (two lanes of fma.rn.f32x2) carries each coefficient twice, the same as gelu_f's."""
    c = [float(x) for x in re.findall(r"([0-9]\.[0-9]+e[-+][0-9]+)f", _body("void gelu2(float& v0, float& v1)"))]
    assert len(c) == 14
    assert all(c[2 * i] == c[2 * i + 1] for i in range(7))
    single = [float(x) for x in re.findall(r"([0-9]\.[0-9]+e[-+][0-9]+)f", _body("float gelu_f(float v)"))]
    assert c[0::2] == single
