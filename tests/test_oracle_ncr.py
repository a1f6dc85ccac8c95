"""Pins of the oracle's variant with a hypot that is not correctly rounded (Alg. 1's branch
for that case, Sect. 3.3.1): the hypot's error bound against the exact value, its exact
and special cases, closed forms of tan(2 phi) reached through the branch, the precedence of
Alg. 1's special cases, |tan phi| <= 1, the rotation-orthogonality bound that follows from
the hypot's error bound, operation counts read off the formulas, and empirical accuracy on
the paper's input classes (the paper gives no bound for this variant)."""
import decimal
import math
import sys

import numpy as np
import pytest

import oracle
from exact import EPS, cr_hypot, rn, to_float
from paper_2407_13116_gb300 import inputs as I

NU = sys.float_info.max
T2NCR = oracle.FLAGS["t2ncr"]


def _exact_hypot(a, b):
    D = decimal.Decimal
    with decimal.localcontext() as c:
        c.prec = 90
        c.Emax = 10 ** 6
        c.Emin = -10 ** 6
        return (D(a) * D(a) + D(b) * D(b)).sqrt()


def _rel(h, ref):
    D = decimal.Decimal
    with decimal.localcontext() as c:
        c.prec = 90
        c.Emax = 10 ** 6
        c.Emin = -10 ** 6
        return float(abs(D(h) - ref) / ref)


@pytest.mark.parametrize("prec", ["d", "s"])
def test_hypot_ncr_exact_and_special_cases(prec):
    T = np.float64 if prec == "d" else np.float32
    h = lambda x, y: float(oracle.hypot_ncr(float(T(x)), float(T(y)), prec))
    # every step exact: q = 3/4, 1 + q^2 = 25/16, sqrt = 5/4
    for k in (-60, -3, 0, 7, 60):
        assert h(3 * 2.0 ** k, 4 * 2.0 ** k) == 5 * 2.0 ** k
        assert h(-4 * 2.0 ** k, 3 * 2.0 ** k) == 5 * 2.0 ** k
    for x in (1.5, -2.0 ** -30, 1e30):
        assert h(x, 0.0) == abs(float(T(x))) and h(0.0, x) == abs(float(T(x)))
    assert h(0.0, -0.0) == 0.0
    assert math.isinf(h(math.inf, math.nan)) and math.isinf(h(1.0, -math.inf))
    assert math.isnan(h(math.nan, 1.0))
    # symmetric in its arguments and in their signs
    rng = np.random.default_rng(5)
    for _ in range(200):
        x, y = (float(T(v)) for v in rng.standard_normal(2) * 2.0 ** rng.integers(-20, 20, 2))
        assert h(x, y) == h(y, x) == h(-x, y) == h(x, -y)
    # the scaled formula does not overflow below the largest value: h(nu/2, nu/2) = nu/sqrt(2)
    big = float(np.finfo(T).max) / 2
    hb = h(big, big)
    assert math.isfinite(hb) and _rel(hb, _exact_hypot(big, big)) <= 3.5 * EPS[prec]
    # the smallest subnormal: sqrt(2) quanta round to one quantum
    tiny = float(np.finfo(T).smallest_subnormal)
    assert h(tiny, tiny) == tiny


@pytest.mark.parametrize("prec", ["d", "s"])
def test_hypot_ncr_error_bound_and_not_correctly_rounded(prec):
    """Relative error below 3.5 u (u = 2^-p, first-order bound of the four roundings of
    w sqrt(fma(q, q, 1))), and on some inputs the result is not the correctly rounded one:
    the variant really is the non-CR case of Alg. 1."""
    T = np.float64 if prec == "d" else np.float32
    rng = np.random.default_rng(17 if prec == "d" else 18)
    n = 3000
    e = rng.integers(-30, 30, (2, n))
    spread = rng.integers(0, 3, n)
    e[1] = e[0] - spread * rng.integers(0, 20, n)
    x = (rng.uniform(1, 2, n) * np.exp2(e[0])).astype(T)
    y = (rng.uniform(1, 2, n) * np.exp2(e[1])).astype(T)
    hn = oracle.hypot_ncr_n(x, y, prec)
    worst, not_cr = 0.0, 0
    for i in range(n):
        a, b, v = float(x[i]), float(y[i]), float(hn[i])
        worst = max(worst, _rel(v, _exact_hypot(a, b)))
        not_cr += v != to_float(cr_hypot(a, b, prec))
    assert worst <= 3.5 * EPS[prec], worst / EPS[prec]
    assert worst > 0.5 * EPS[prec] and not_cr > 0


def _tr(r11, r12, r22, ncr=True, prec="d"):
    return oracle.trace(np.array([r11, 0.0, r12, r22]), prec, ncr=ncr)


def test_tan2phi_closed_forms_through_the_branch():
    """tan(2 phi) = 2 r12 r22 / (r11^2 + r12^2 - r22^2) for R = [[r11, r12], [0, r22]]; with
    dyadic inputs whose x, y, x - y, x + y and fma are exact it is one rounding of that
    quotient, in both sub-branches (r11 > r12 and r11 <= r12) and after the transpose-swap."""
    for (r11, r12, r22), (num, den) in (((4.0, 2.0, 1.0), (4, 19)), ((2.0, 4.0, 1.0), (8, 19)),
                                         ((1.0, 2.0, 4.0), (4, 19)), ((8.0, 2.0, 4.0), (16, 52)),
                                         ((4.0, 8.0, 2.0), (32, 76))):
        tr, ints = _tr(r11, r12, r22)
        assert ints[3] & T2NCR
        assert tr[3] == to_float(rn(__import__("fractions").Fraction(num, den))), (r11, r12, r22, tr[3])
        assert 0 <= tr[4] <= 1
        # the correctly rounded mode takes the eq. (t2f') branch on the same input
        tr0, ints0 = _tr(r11, r12, r22, ncr=False)
        assert not (ints0[3] & T2NCR)


def test_alg1_special_cases_precede_the_branch():
    F = oracle.FLAGS
    for (r11, r12, r22), flag in (((3.0, 5.0, 3.0), F["t2f2"]), ((4.0, 1.0, 1.0), F["t2f3"]),
                                  ((1.0, 2.0 ** 60, 0.5), F["t2f2"])):
        tr, ints = _tr(r11, r12, r22)
        assert ints[3] & flag and not (ints[3] & T2NCR), (r11, r12, r22, ints[3])


def test_tanphi_in_unit_interval():
    """Every case of Alg. 1 gives 0 <= tan phi <= 1 (Sect. 3.3.1), the new branch included."""
    G = np.concatenate([I.general(3000, 7, "d", "narrow"), I.general(3000, 8, "d", "wide"),
                        I.safe_range(3000, 9, 0, triangular_=True)], axis=1)
    seen = 0
    for i in range(G.shape[1]):
        tr, ints = oracle.trace(G[:, i], "d", ncr=True)
        if ints[3] & T2NCR:
            seen += 1
            assert 0 <= tr[4] <= 1 and math.isfinite(tr[3]) and tr[3] >= 0
    assert seen > 3000


def test_operation_counts_by_hand():
    """Counts read off the formulas (the hypot: one division, fma, square root and product).
    * one nonzero column: tan = small/big, sec = hypot(tan, 1), cos, sin, sigma1 = hypot:
      5 div, 2 fma, 2 sqrt, 2 mul;
    * triangular with r11 > r12 (no swap after R = [[2, 1], [0, 3]] is swapped to
      ra = 3, rb = 1, rc = 2): the test r11/r12 < eps, x, y, fl(2x)y, x - y, x + y, fma, the
      quotient; tan phi = t2/(1 + hypot(t2, 1)); sec, cos, sin of phi; Alg. 2's fma and
      quotient, sec, cos, sin of psi; sec phi (/) sec psi, r11 (/) it and r22 (.) it:
      3 add, 5 mul, 5 fma, 15 div, 3 sqrt;
    * r11 <= r12: the same without fl(2x)y's product: 4 mul."""
    def count(g):
        return oracle.opcount(np.array(g, dtype=np.float64).reshape(3, 1), triangular=True, ncr=True)
    z = dict(add=0, mul=0, fma=0, div=0, hypot=0, ext=0, sqrt=0)
    assert oracle.opcount(np.array([2.0, 3.0, 0.0, 0.0]).reshape(4, 1), ncr=True) == dict(z, div=5, fma=2, sqrt=2, mul=2)
    assert count([2.0, 1.0, 3.0]) == dict(z, add=3, mul=5, fma=5, div=15, sqrt=3)
    assert count([2.0, 4.0, 1.0]) == dict(z, add=3, mul=4, fma=5, div=15, sqrt=3)


def _metrics(G, r):
    return oracle.dmetrics(np.asarray(G, np.float64),
                           {k: np.asarray(r[k], np.float64) if k != "Se" else r[k] for k in ("U", "V", "Se", "Sf")})


@pytest.mark.parametrize("prec", ["d", "s"])
def test_accuracy_on_the_paper_input_classes(prec):
    """Empirical: the paper proves no bound for this variant.  Orthogonality follows from the
    hypot's bound: c = 1/sec and s = t/sec with sec within 3.5 u of sqrt(1 + t^2) give
    |c^2 + s^2 - 1| <= 8 u to first order, 11.3 u in the Frobenius norm of U^T U - I.  The
    singular values stay within the single-digit multiples of eps the correctly rounded
    method shows (sigma1 <= 6 eps, sigma2 <= 9 eps on narrow-range general and safe-range
    triangular inputs; measured 4.3 and 5.1)."""
    E = EPS[prec]
    cases = [I.general(1 << 13, 21 if prec == "d" else 81, prec, "narrow"),
             I.safe_range(1 << 13, 31 if prec == "d" else 82, 0, prec, triangular_=True)]
    for G in cases:
        r = oracle.gesvd2(G, prec, nthreads=4, ncr=True)
        m = _metrics(G, r)
        assert m[0].max() <= 6 * E and m[1].max() <= 9 * E, (m[0].max() / E, m[1].max() / E)
        assert m[2].max() <= 11.4 * E and m[3].max() <= 11.4 * E, (m[2].max() / E, m[3].max() / E)
        assert m[4].max() <= 8 * E, m[4].max() / E
        assert np.all(r["S"][0] >= r["S"][1]) and np.all(r["S"][1] >= 0)


@pytest.mark.parametrize("prec", ["d", "s"])
def test_triangular_entry_equals_general_and_no_inf_nan(prec):
    T3 = I.triangular(4000, 41, prec, "wide")
    G = np.stack([T3[0], np.zeros_like(T3[0]), T3[1], T3[2]])
    a = oracle.trsvd2(T3[0], T3[1], T3[2], prec, ncr=True)
    b = oracle.gesvd2(G, prec, ncr=True)
    for k in ("U", "V", "S", "Se", "Sf", "info"):
        assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8))
    W = I.general(4000, 42, prec, "wide")
    r = oracle.gesvd2(W, prec, ncr=True)
    assert np.isfinite(r["U"]).all() and np.isfinite(r["V"]).all()
    r2 = oracle.gesvd2(W, prec, ncr=True, nthreads=4)
    assert np.array_equal(r["U"].view(np.uint8), r2["U"].view(np.uint8))
