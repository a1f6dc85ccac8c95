"""Pins of the oracle's correctly rounded hypot (Sect. 2) against exact integer arithmetic:
hypot(a, b) must equal the rounding of sqrt(a^2 + b^2) computed from the exact rational
a^2 + b^2 (tests/exact.py), including exact ties, subnormals and huge exponent gaps."""
import math
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import cr_hypot, to_float

NU_D = 1.7976931348623157e308
MU_D = 2.2250738585072014e-308
NU_S = float(np.float32(3.4028234663852886e38))


def _f32(x):
    return struct.unpack("f", struct.pack("f", x))[0]


def _rand_double(rng, elo, ehi):
    m = rng.getrandbits(52)
    e = rng.randint(elo, ehi)
    return math.ldexp(1.0 + m / 2.0 ** 52, e) * (1 if rng.random() < 0.5 else -1)


def _rand_sub(rng):
    return rng.getrandbits(52) * 2.0 ** -1074 or 2.0 ** -1074


def _check(a, b, prec="d"):
    got = oracle.hypot(a, b, prec)
    exp = cr_hypot(a, b, "d" if prec == "d" else "s")
    exp = math.inf if exp == math.inf else to_float(exp)
    assert got == exp, (a, b, got, exp)


def test_small_triples_exact():
    for (a, b, c) in [(3, 4, 5), (5, 12, 13), (8, 15, 17), (20, 21, 29), (0, 7, 7), (7, 0, 7)]:
        for k in (-1070, -500, 0, 300, 1000):
            for prec in ("d", "s"):
                if prec == "s" and not -140 <= k <= 100:
                    continue
                a2, b2, c2 = math.ldexp(a, k), math.ldexp(b, k), math.ldexp(c, k)
                assert oracle.hypot(a2, b2, prec) == c2
                assert oracle.hypot(-a2, b2, prec) == c2


def test_lemma_nu():
    # Lemma 2.1: fl(nu + 1) = nu = hypot(nu, 1)
    assert NU_D + 1.0 == NU_D
    assert oracle.hypot(NU_D, 1.0) == NU_D
    assert oracle.hypot(1.0, NU_D) == NU_D
    assert oracle.hypot(NU_S, 1.0, "s") == np.float32(NU_S)


def test_zero_iff_both_zero():
    assert oracle.hypot(0.0, 0.0) == 0.0
    assert oracle.hypot(0.0, -0.0) == 0.0
    assert oracle.hypot(2.0 ** -1074, 0.0) == 2.0 ** -1074
    assert oracle.hypot(2.0 ** -1074, 2.0 ** -1074) == 2.0 ** -1074  # sqrt(2) * 2^-1074 rounds to 1 quantum
    assert oracle.hypot(float(np.float32(2.0 ** -149)), 0.0, "s") > 0


def test_random_double_vs_exact():
    rng = random.Random(20240713)
    for _ in range(3000):
        kind = rng.random()
        if kind < 0.4:
            a, b = _rand_double(rng, -30, 30), _rand_double(rng, -30, 30)
        elif kind < 0.6:
            a, b = _rand_double(rng, -1022, 1023), _rand_double(rng, -1022, 1023)
        elif kind < 0.75:
            a = _rand_double(rng, -10, 10)
            b = math.ldexp(a, -rng.randint(20, 60)) * (1 + rng.random())
        elif kind < 0.9:
            a, b = _rand_sub(rng), _rand_sub(rng)
        else:
            a, b = _rand_double(rng, -1030, -1000), _rand_sub(rng)
        _check(a, b)


def test_near_midpoints_double():
    """Inputs whose exact hypot lies within a tiny distance of a midpoint between doubles."""
    rng = random.Random(7)
    for _ in range(400):
        # c = odd 54-bit integer (a midpoint), a random; b = sqrt(c^2 - a^2) rounded
        c = (1 << 53) | rng.getrandbits(53) | 1
        a = rng.getrandbits(52) | (1 << 51)
        b2 = c * c - a * a
        b = math.isqrt(b2)
        for bb in (b - 1, b, b + 1):
            if 0 < bb < (1 << 53):
                k = rng.randint(-900, 900)
                _check(math.ldexp(a, k), math.ldexp(bb, k))


def _euclid_ties(p, count, rng):
    """Pythagorean triples (a, b, c) with c odd and of p+1 bits (a midpoint between two
    p-bit values) while a (odd) and b (even) are representable in p bits: exact ties.
    Primitive triples have c = 1 (mod 4), so their ties round down to c - 1; odd multiples
    k (a, b, c) with k = 3 (mod 4) give c = 3 (mod 4), whose ties round up to c + 1."""
    out = []
    lo, hi = 1 << p, 1 << (p + 1)
    tries = 0
    while len(out) < count and tries < 400000:
        tries += 1
        k = rng.choice((1, 3, 5, 7, 11))
        m = rng.randint(int(math.isqrt(lo // (2 * k))), int(math.isqrt(hi // k)))
        n = rng.randint(1, m - 1)
        if (m - n) % 2 == 0 or math.gcd(m, n) != 1:
            continue
        a, b, c = k * (m * m - n * n), k * 2 * m * n, k * (m * m + n * n)
        if not (lo <= c < hi) or a >= lo or b >= hi:
            continue
        out.append((a, b, c))
    return out


@pytest.mark.parametrize("prec", ["d", "s"])
def test_exact_ties_round_to_even(prec):
    p = 53 if prec == "d" else 24
    rng = random.Random(11 + p)
    trip = _euclid_ties(p, 120, rng)
    ups = downs = 0
    for (a, b, c) in trip:
        # the exact hypotenuse c is odd with p+1 bits: a tie between c-1 and c+1 (ulp 2)
        exp = c - 1 if ((c - 1) // 2) % 2 == 0 else c + 1
        ups += exp > c
        downs += exp < c
        got = oracle.hypot(float(a), float(b), prec)
        assert got == float(exp), (a, b, c, got)
        assert got == to_float(cr_hypot(a, b, prec))
    assert ups >= 10 and downs >= 10


def test_single_vs_exact():
    rng = random.Random(3)
    for _ in range(4000):
        kind = rng.random()
        if kind < 0.5:
            a = _f32(math.ldexp(1 + rng.random(), rng.randint(-20, 20)))
            b = _f32(math.ldexp(1 + rng.random(), rng.randint(-20, 20)))
        elif kind < 0.8:
            a = _f32(math.ldexp(1 + rng.random(), rng.randint(-126, 127)))
            b = _f32(math.ldexp(1 + rng.random(), rng.randint(-126, 127)))
        else:
            a = _f32(rng.getrandbits(23) * 2.0 ** -149)
            b = _f32(math.ldexp(1 + rng.random(), rng.randint(-140, -120)))
        _check(a, b, "s")


def test_single_dense_window():
    """All pairs in a small window of consecutive floats against the exact rounding."""
    base = np.float32(1.5)
    xs = base + np.arange(64, dtype=np.float32) * np.float32(2.0 ** -23)
    ys = np.float32(0.75) + np.arange(64, dtype=np.float32) * np.float32(2.0 ** -24)
    for x in xs:
        for y in ys:
            _check(float(x), float(y), "s")


def test_symmetric_and_monotone():
    rng = random.Random(5)
    for _ in range(500):
        a, b = abs(_rand_double(rng, -40, 40)), abs(_rand_double(rng, -40, 40))
        h = oracle.hypot(a, b)
        assert h == oracle.hypot(b, a) == oracle.hypot(-a, -b)
        assert oracle.hypot(np.nextafter(a, math.inf), b) >= h
        assert oracle.hypot(a, np.nextafter(b, math.inf)) >= h
        assert h >= max(a, b)
