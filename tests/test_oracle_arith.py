"""Pins of the oracle's (e,f) arithmetic (Sect. 2, eqs. (unary), (binary), (plus), (minus),
(prec)) and of eq. (EXT) against exact rational arithmetic."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import rn, to_float

NU = 1.7976931348623157e308
MU = 2.2250738585072014e-308


def _val(e, f):
    return Fraction(float(f)) * Fraction(2) ** int(e)


def _rand(rng, elo, ehi, prec="d"):
    m = 1 + rng.random()
    x = math.ldexp(m, rng.randint(elo, ehi)) * (1 if rng.random() < 0.5 else -1)
    return float(np.float32(x)) if prec == "s" else x


@pytest.mark.parametrize("prec", ["d", "s"])
def test_ef_of_is_exact_and_normalized(prec):
    rng = random.Random(1)
    lo, hi = (-1074, 1023) if prec == "d" else (-149, 127)
    for _ in range(2000):
        x = _rand(rng, lo, hi, prec)
        if x == 0:
            continue
        e, f = oracle.efops(x, 1.0, prec)
        assert 1 <= abs(f[4]) < 2
        assert _val(e[4], f[4]) == Fraction(x)
        assert e[4] == math.floor(math.log2(abs(x))) or _val(e[4], 1) <= abs(Fraction(x)) < _val(e[4] + 1, 1)
    e, f = oracle.efops(0.0, 1.0, prec)
    assert e[4] == 0 and f[4] == 0


@pytest.mark.parametrize("prec", ["d", "s"])
def test_mul_div_match_exact_rounding(prec):
    """x (.) y and x (/) y equal the p-bit rounding of the exact product/quotient of the
    mantissas, scaled by the exact exponent sum/difference."""
    rng = random.Random(2)
    fmt = prec
    lo, hi = (-1074, 1023) if prec == "d" else (-149, 127)
    for _ in range(3000):
        x, y = _rand(rng, lo, hi, prec), _rand(rng, lo, hi, prec)
        e, f = oracle.efops(x, y, prec)
        ex, fx, ey, fy = e[4], Fraction(float(f[4])), e[5], Fraction(float(f[5]))
        pm = rn(fx * fy, fmt) * Fraction(2) ** int(ex + ey)
        pd = rn(fx / fy, fmt) * Fraction(2) ** int(ex - ey)
        assert _val(e[0], f[0]) == pm
        assert _val(e[1], f[1]) == pd
        assert 1 <= abs(f[0]) < 2 and 1 <= abs(f[1]) < 2


def test_fl_single_rounding_into_subnormals():
    """fl(e,f) = scalbn(f, e) is one rounding of the exact f 2^e, including gradual underflow
    and overflow (the definition after Cor. 2.3)."""
    rng = random.Random(3)
    for _ in range(3000):
        f = 1 + rng.getrandbits(52) / 2.0 ** 52
        e = rng.randint(-1080, 1025)
        got = oracle.effl(e, f, "d")
        exp = rn(Fraction(f) * Fraction(2) ** e, "d")
        assert got == (math.inf if exp == math.inf else to_float(exp)), (e, f)
    for _ in range(2000):
        f = float(np.float32(1 + rng.getrandbits(23) / 2.0 ** 23))
        e = rng.randint(-155, 130)
        got = oracle.effl(e, f, "s")
        exp = rn(Fraction(f) * Fraction(2) ** e, "s")
        assert got == (math.inf if exp == math.inf else to_float(exp)), (e, f)


def test_plus_overflow_avoiding():
    # eq. (plus): exact rounding of x + y, represented without overflow
    assert NU / 2 + NU / 2 == NU                        # fl(nu/2 + nu/2) = nu (Sect. 2)
    rng = random.Random(4)
    for _ in range(2000):
        x = abs(_rand(rng, 1000, 1023))
        y = abs(_rand(rng, 990, 1023))
        e, f = oracle.efops(x, y, "d")
        v = _val(e[2], f[2])
        exact = Fraction(x) + Fraction(y)
        if exact <= Fraction(NU):
            assert v == rn(exact, "d")
        assert 1 <= f[2] < 2
        assert abs(v - exact) <= exact * Fraction(1, 2 ** 52)


def test_minus_underflow_avoiding():
    """eq. (minus) and Lemma 2.4: the difference is normal after the upscaling by 2^c (c > 0)
    and represents x - y exactly when the exact difference fits in p bits."""
    rng = random.Random(5)
    for _ in range(2000):
        # x, y close and tiny so that x - y is subnormal
        y = rng.getrandbits(52) * 2.0 ** -1074 + 2.0 ** -1074
        x = y + rng.randint(1, 1 << 20) * 2.0 ** -1074
        e, f = oracle.efops(x, y, "d")
        v = _val(e[3], f[3])
        assert v == Fraction(x) - Fraction(y)
        assert 1 <= abs(f[3]) < 2
    for _ in range(1000):
        x, y = abs(_rand(rng, -1000, 1000)), abs(_rand(rng, -1000, 1000))
        if x == y:
            continue
        e, f = oracle.efops(x, y, "d")
        assert _val(e[3], f[3]) == rn(Fraction(x) - Fraction(y), "d")
    e, f = oracle.efops(3.0, 3.0, "d")
    assert e[3] == 0 and f[3] == 0


def test_prec_order():
    rng = random.Random(6)
    for _ in range(3000):
        ex, ey = rng.randint(-3000, 3000), rng.randint(-3000, 3000)
        if rng.random() < 0.3:
            ey = ex
        fx = 1 + rng.getrandbits(52) / 2.0 ** 52
        fy = 1 + rng.getrandbits(52) / 2.0 ** 52
        if rng.random() < 0.1:
            fy = fx
        assert oracle.prec(ex, fx, ey, fy) == (_val(ex, fx) < _val(ey, fy))
    assert oracle.prec(0, 0.0, -5000, 1.0)          # 0 precedes any positive value
    assert not oracle.prec(-5000, 1.0, 0, 0.0)


def _ext_exact(x1, y1, x2, y2, neg, d, sec, prec):
    """eq. (EXT) by exact rational arithmetic: FL = rounding to the wide format T, fl = to the
    working format."""
    wide, work = ("q", "d") if prec == "d" else ("d", "s")
    p1, p2 = Fraction(x1) * Fraction(y1), Fraction(x2) * Fraction(y2)
    num = rn(p1 - p2 if neg else p1 + p2, wide)
    q = rn(num / Fraction(d), wide)
    r = rn(q, work)
    return rn(r / Fraction(sec), work)


@pytest.mark.parametrize("prec", ["d", "s"])
def test_ext_matches_exact_double_rounding(prec):
    rng = random.Random(8 if prec == "d" else 9)
    top = 1021 if prec == "d" else 125
    for _ in range(3000):
        # elements of a pivoted G''': g11 >= g21 > 0, others signed, all at most nu/4
        g11 = abs(_rand(rng, top - 3, top, prec))
        g21 = abs(_rand(rng, top - 60, top, prec))
        if g21 > g11:
            g11, g21 = g21, g11
        g12 = _rand(rng, top - 60, top, prec)
        g22 = _rand(rng, top - 60, top, prec)
        tth = g21 / g11 if prec == "d" else float(np.float32(g21) / np.float32(g11))
        sec = oracle.hypot(tth, 1.0, prec)
        for neg in (0, 1):
            x1, y1, x2, y2 = (g22, g11, g12, g21) if neg else (g12, g11, g22, g21)
            got = oracle.ext(x1, y1, x2, y2, neg, g11, sec, prec)
            assert got == to_float(_ext_exact(x1, y1, x2, y2, neg, g11, sec, prec))
    # near-cancellation: g22 g11 - g12 g21 tiny relative to the products
    for _ in range(1000):
        g11 = abs(_rand(rng, top - 2, top, prec))
        g21 = abs(_rand(rng, top - 5, top, prec))
        if g21 > g11:
            g11, g21 = g21, g11
        g12 = abs(_rand(rng, top - 5, top, prec))
        g22 = to_float(rn(Fraction(g12) * Fraction(g21) / Fraction(g11), prec))
        if rng.random() < 0.5:
            g22 = float(np.nextafter(np.float32(g22), np.float32(math.inf))) if prec == "s" \
                else float(np.nextafter(g22, math.inf))
        tth = g21 / g11 if prec == "d" else float(np.float32(g21) / np.float32(g11))
        sec = oracle.hypot(tth, 1.0, prec)
        got = oracle.ext(g22, g11, g12, g21, 1, g11, sec, prec)
        assert got == to_float(_ext_exact(g22, g11, g12, g21, 1, g11, sec, prec))
