"""The windowed kernel's own approximations, read from its source as text and
evaluated in emulated FP64 (every FMA rounded once, exactly) against 40-digit
references: the Gaussian weight's exp(z), z <= 0, and the Hann weight's cos(x),
|x| <= pi/2.  A changed constant or step fails here without a GPU."""
import math
import os
import random
import re
import struct
from fractions import Fraction

import mpmath as mp
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2609_03866_b300", "csrc", "k_scan.cu")
mp.mp.dps = 40


def fma(a, b, c):
    if not all(math.isfinite(v) for v in (a, b, c)):
        return a * b + c
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _src():
    return open(SRC).read()


def _const(name):
    m = re.search(r"constexpr double " + name + r" = ([-0-9.xa-fp+]+);", _src())
    v = m.group(1)
    return float.fromhex(v) if "0x" in v else float(v)


def test_cos_half_range_within_2e16():
    body = _src()[_src().index("cos_half_range(double x)"):]
    body = body[:body.index("}")]
    coefs = [float.fromhex(h) for h in re.findall(r"(-?0x1\.[0-9a-f]+p[-+]\d+)", body)]
    assert len(coefs) == 8 and "return fma(a, w, 1.0);" in body

    def ev(x):
        w = x * x
        a = coefs[0]
        for c in coefs[1:]:
            a = fma(a, w, c)
        return fma(a, w, 1.0)

    rng = random.Random(5)
    xs = [0.0, math.pi / 2, -math.pi / 2] + [rng.uniform(-math.pi / 2, math.pi / 2) for _ in range(1500)]
    worst = max(float(abs(ev(x) - mp.cos(x))) for x in xs)
    assert worst < 2.2e-16, worst


def test_exp_neg_within_1p5_ulp_near_the_peak_and_1p3e16_absolute():
    inv_l, c = _const("kExpInvL"), _const("kExpC")
    assert "constexpr int kExpTable = 256;" in _src()
    assert abs(inv_l * c - 1.0) < 1e-15
    table = [float(mp.mpf(2) ** (mp.mpf(j) / 256)) for j in range(256)]
    magic = float.fromhex("0x1.8p52")

    def d2ll(v):
        return struct.unpack("<q", struct.pack("<d", v))[0]

    def ll2d(v):
        return struct.unpack("<d", struct.pack("<q", v))[0]

    src = _src()
    assert "constexpr long long kExpFloor = 0x4338000000000000ll - 1021ll * kExpTable;" in src
    assert "if (__double_as_longlong(nd) < kExpFloor) return 0.0;" in src
    floor = 0x4338000000000000 - 1021 * 256

    def exp_neg(z):
        nd = fma(z, inv_l, magic)
        if d2ll(nd) < floor:
            return 0.0
        n = d2ll(nd) & 0xFFFFFFFF
        n = n - (1 << 32) if n >= 1 << 31 else n
        N = nd - magic
        r = fma(-N, c, z)
        p = r * fma(r, fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5), 1.0)
        t = table[n & 255]
        v = fma(t, p, t)
        return ll2d(d2ll(v) + ((n >> 8) << 52))

    rng = random.Random(6)
    near = [0.0, -1e-300] + [-rng.uniform(0.0, 1.0) for _ in range(1500)]
    far = [-rng.uniform(1.0, 707.0) for _ in range(1500)]
    worst_ulp = max(float(abs(exp_neg(z) - mp.e ** z) / math.ulp(float(mp.e ** z))) for z in near)
    worst_abs = max(float(abs(exp_neg(z) - mp.e ** z)) for z in near + far)
    assert worst_ulp < 1.5, worst_ulp
    assert worst_abs < 1.3e-16, worst_abs
    assert exp_neg(-800.0) == 0.0
    # far from the window centre (a wide or untruncated window): d / h = 3500, 4000,
    # 6000 and beyond, where a guard on the low word alone would wrap
    for d in (3500.0, 4000.0, 6000.0, 1e5, 1e150):
        assert exp_neg(-d * d / 2.0) == 0.0, d
    assert exp_neg(-math.inf) == 0.0
    # the last arguments above the floor still give the exponential (relative error
    # below |z| 3.4e-17 from the reduction, plus the polynomial's and the table's)
    for z in (-707.0, -700.0):
        assert abs(exp_neg(z) / float(mp.e ** z) - 1.0) < 5e-14, z
