"""Exact reference arithmetic for the pins: rational rounding to a binary format,
exact correctly rounded square roots of rationals, and high-precision closed-form
singular values.  Pure Python integers, fractions and decimals: it shares nothing
with the oracle's C code or the CUDA path."""
import decimal
import math
from fractions import Fraction

# all Decimal arithmetic in the pins runs with 90 digits and a wide exponent range
decimal.getcontext().prec = 90
decimal.getcontext().Emax = 10 ** 6
decimal.getcontext().Emin = -10 ** 6

FMT = {
    # name: (p, smallest quantum exponent, emax)
    "d": (53, -1074, 1023),
    "s": (24, -149, 127),
    "q": (113, -16494, 16383),
}
EPS = {"d": 2.0 ** -53, "s": 2.0 ** -24}


def floor_log2(x: Fraction) -> int:
    """floor(lg x) for a positive rational."""
    n, d = x.numerator, x.denominator
    e = n.bit_length() - d.bit_length()
    # 2^e <= x < 2^(e+1) ?
    if e >= 0:
        if n < (d << e):
            e -= 1
    else:
        if (n << -e) < d:
            e -= 1
    return e


def _round_int(m: Fraction, up_half_even=True) -> int:
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return fl


def rn(x, fmt="d"):
    """Round a rational to nearest (ties to even) in the given binary format, with gradual
    underflow; returns a Fraction, or +-inf on overflow."""
    x = Fraction(x)
    p, qmin, emax = FMT[fmt]
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    x = abs(x)
    e = floor_log2(x)
    q = max(e - (p - 1), qmin)
    m = x / Fraction(2) ** q
    r = _round_int(m) * Fraction(2) ** q
    if r >= Fraction(2) ** (emax + 1):
        return s * math.inf
    return s * r


def to_float(r):
    if isinstance(r, float):
        return r
    return float(r)  # exact for values representable in double


def cr_sqrt(X: Fraction, fmt="d"):
    """Correctly rounded sqrt of a non-negative rational in the given format."""
    X = Fraction(X)
    if X == 0:
        return Fraction(0)
    p, qmin, emax = FMT[fmt]
    e = floor_log2(X) // 2                 # floor(lg sqrt(X))
    q = max(e - (p - 1), qmin)
    Y = X / Fraction(4) ** q               # sqrt(X) / 2^q = sqrt(Y)
    fy = Y.numerator // Y.denominator
    fl = math.isqrt(fy)                    # floor(sqrt(Y))
    lhs = 4 * Y
    mid2 = (2 * fl + 1) ** 2               # (fl + 1/2)^2 * 4
    if lhs > mid2 or (lhs == mid2 and fl % 2 == 1):
        fl += 1
    r = fl * Fraction(2) ** q
    if r >= Fraction(2) ** (emax + 1):
        return math.inf
    return r


def cr_hypot(a, b, fmt="d"):
    """hypot(a, b) correctly rounded, from the exact value a^2 + b^2."""
    a, b = Fraction(a), Fraction(b)
    return cr_sqrt(a * a + b * b, fmt)


def dec(x, prec=90):
    with decimal.localcontext() as c:
        c.prec = prec
        return decimal.Decimal(x) if not isinstance(x, Fraction) else decimal.Decimal(x.numerator) / decimal.Decimal(x.denominator)


def sigma_closed(g11, g21, g12, g22, prec=90):
    """Singular values of [[g11, g12], [g21, g22]] from the closed form
    sigma1 = (|(a+d, c-b)| + |(a-d, b+c)|)/2, sigma2 = |ad - bc| / sigma1, in prec digits."""
    D = decimal.Decimal
    with decimal.localcontext() as c:
        c.prec = prec
        c.Emax = 10 ** 6
        c.Emin = -10 ** 6
        a, b, cc, d = D(g11), D(g12), D(g21), D(g22)
        p = ((a + d) ** 2 + (cc - b) ** 2).sqrt()
        q = ((a - d) ** 2 + (b + cc) ** 2).sqrt()
        s1 = (p + q) / 2
        det = abs(a * d - b * cc)
        s2 = det / s1 if s1 != 0 else D(0)
        return s1, s2


def ef_value(e, f, prec=90):
    """f * 2^e as a Decimal."""
    D = decimal.Decimal
    with decimal.localcontext() as c:
        c.prec = prec
        c.Emax = 10 ** 6
        c.Emin = -10 ** 6
        return D(f) * (D(2) ** int(e))


def relerr(x, ref, prec=90):
    D = decimal.Decimal
    with decimal.localcontext() as c:
        c.prec = prec
        c.Emax = 10 ** 6
        c.Emin = -10 ** 6
        x, ref = D(x), D(ref)
        if ref == 0:
            return 0.0 if x == 0 else math.inf
        return float(abs(x - ref) / ref)
