"""Pins of the oracle's 2x2 SVD against what the paper and the mathematics fix:
closed-form singular values (binary128 and 90-digit decimal), the invariants
sigma1 sigma2 = |det G| and sigma1^2 + sigma2^2 = ||G||_F^2, the accuracy claims of
Sect. 4 over the safe ranges, the bounds of Thm. 3.5 / Table 1 (t:d), Cor. 2.2
(|tan phi| <= 1), the worked example of Sect. 4, the error-free simple types of
Sect. 3.1, the absence of Inf/NaN in U and V and bitwise reproducibility (end of
Sect. 3.3.2), and one constructed input per branch."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import EPS, ef_value, relerr, sigma_closed
from paper_2407_13116_gb300 import inputs as I

EPSD = EPS["d"]
EPSS = EPS["s"]
NU = 1.7976931348623157e308
MU = 2.2250738585072014e-308


def _G(*rows):
    """planes (g11, g21, g12, g22) of a list of 2x2 matrices [[a, b], [c, d]]."""
    return np.array([[m[0][0] for m in rows], [m[1][0] for m in rows],
                     [m[0][1] for m in rows], [m[1][1] for m in rows]], dtype=np.float64)


def _mat(r, k, i):
    X = r[k]
    return np.array([[X[0, i], X[2, i]], [X[1, i], X[3, i]]])


def test_brute_force_matches_decimal_closed_form():
    G = np.concatenate([I.general(150, 11, "d", "narrow"), I.general(150, 12, "d", "wide")], axis=1)
    for i in range(G.shape[1]):
        g = G[:, i]
        s1, s2 = sigma_closed(*g)
        b = oracle.brute_sigma(g)
        for (e, hi, lo), ref in zip(b, (s1, s2)):
            v = ef_value(e, hi) + ef_value(e, lo)
            assert relerr(v, ref) < 1e-30


def _check_accuracy(G, r, s1_tol, s2_tol, orth_tol, res_tol, eps=EPSD):
    m = oracle.dmetrics(np.asarray(G, np.float64),
                        {k: np.asarray(r[k], np.float64) if k != "Se" else r[k] for k in ("U", "V", "Se", "Sf")})
    assert m[0].max() <= s1_tol * eps, m[0].max() / eps
    if s2_tol is not None:
        assert m[1].max() <= s2_tol * eps, m[1].max() / eps
    assert m[2].max() <= orth_tol * eps and m[3].max() <= orth_tol * eps, (m[2].max() / eps, m[3].max() / eps)
    assert m[4].max() <= res_tol * eps, m[4].max() / eps
    return m


def test_narrow_accuracy_and_invariants():
    """Sect. 4: sigma1 to a few eps always; sigma2 to a single-digit multiple of eps when the
    exponent spread is below (e_nu - e_mu)/2; U, V orthogonal to 4 * 2^-52 (= 8 eps)."""
    G = I.general(1 << 14, 21, "d", "narrow")
    r = oracle.gesvd2(G, nthreads=4)
    _check_accuracy(G, r, 5, 9, 8, 8)
    assert np.all(r["S"][0] >= r["S"][1]) and np.all(r["S"][1] >= 0)


def test_invariants_decimal():
    """sigma1 sigma2 = |det G| and sigma1^2 + sigma2^2 = ||G||_F^2, evaluated in 90 digits."""
    import decimal
    D = decimal.Decimal
    G = np.concatenate([I.general(200, 22, "d", "narrow"), I.safe_range(200, 23, 1000)], axis=1)
    r = oracle.gesvd2(G)
    with decimal.localcontext() as c:
        c.prec = 90; c.Emax = 10 ** 6; c.Emin = -10 ** 6
        for i in range(G.shape[1]):
            a, cc, b, d = (D(float(x)) for x in G[:, i])
            s1 = ef_value(r["Se"][0, i], r["Sf"][0, i])
            s2 = ef_value(r["Se"][1, i], r["Sf"][1, i])
            det = abs(a * d - b * cc)
            fro = a * a + b * b + cc * cc + d * d
            assert relerr(s1 * s1 + s2 * s2, fro) <= 12 * EPSD
            if det != 0:
                assert relerr(s1 * s2, det) <= 12 * EPSD


def test_triangular_safe_range_both_sigma_accurate():
    """Abstract and Sect. 4, Fig. 2: on upper-triangular inputs with elements in the safe range
    [mu, nu/4] both singular values are relatively accurate."""
    G = I.safe_range(1 << 14, 31, 0, triangular_=True)
    r = oracle.gesvd2(G, nthreads=4)
    _check_accuracy(G, r, 5, 5, 8, 8)


@pytest.mark.parametrize("c", [953, 1000, 1027])
def test_general_safe_range_search(c):
    """Sect. 4, Fig. 4: with |g| in [2^c mu, nu/4] (exponent spread about half the normal range
    or less) sigma2 stays within a single-digit multiple of eps."""
    G = I.safe_range(1 << 13, 40 + c, c)
    r = oracle.gesvd2(G, nthreads=4)
    _check_accuracy(G, r, 5, 9, 8, 8)


def test_worked_example():
    """G = [[mu, nu/4], [0, mu]] (Sect. 4).  The paper derives sigma2 ~ 4 mu^2/nu; sigma1 is
    ~ nu/4 (the paper's printed nu^2/(16 mu) and kappa ~ nu^3/(64 mu^3) contradict
    sigma1 sigma2 = |det G| = mu^2 and its own measured max kappa ~ 9.45e1229 ~ nu^2/(16 mu^2))."""
    g = [MU, 0.0, NU / 4, MU]
    r = oracle.gesvd2(np.array(g).reshape(4, 1))
    s1, s2 = sigma_closed(*g)
    c1 = ef_value(r["Se"][0, 0], r["Sf"][0, 0])
    c2 = ef_value(r["Se"][1, 0], r["Sf"][1, 0])
    assert relerr(c1, s1) <= 4 * EPSD and relerr(c2, s2) <= 4 * EPSD
    assert relerr(c2, ef_value(0, 4.0) * ef_value(0, MU) ** 2 / ef_value(0, NU)) < 1e-12
    assert relerr(c1, ef_value(0, NU) / 4) < 1e-12
    assert r["S"][1, 0] == 0.0           # sigma2 underflows as a double ...
    assert r["Se"][1, 0] < -3000          # ... but not in the (e,f) form
    tr, ints = oracle.trace(np.array(g))
    assert ints[3] & oracle.FLAGS["tpinf"]  # tan(psi) overflows: eq. (tp')


def test_simple_types_error_free():
    """Sect. 3.1: classes 9 (diagonal, anti-diagonal, one element, zero) are error free; classes 3
    and 5 give sigma1 = hypot of the non-zero column/row and sigma2 = 0."""
    cases = [
        ([[0.0, 0.0], [0.0, 0.0]], (0.0, 0.0)),
        ([[-3.0, 0.0], [0.0, 0.0]], (3.0, 0.0)),
        ([[0.0, 0.0], [-5e-300, 0.0]], (5e-300, 0.0)),
        ([[0.0, 7e300], [0.0, 0.0]], (7e300, 0.0)),
        ([[0.0, 0.0], [0.0, -2.0]], (2.0, 0.0)),
        ([[2.0, 0.0], [0.0, -3.0]], (3.0, 2.0)),
        ([[-3.0, 0.0], [0.0, 3.0]], (3.0, 3.0)),
        ([[0.0, -1.5], [4.0, 0.0]], (4.0, 1.5)),
        ([[0.0, 1e-310], [-1e-310, 0.0]], (1e-310, 1e-310)),
        ([[3.0, 0.0], [-4.0, 0.0]], (5.0, 0.0)),
        ([[0.0, -3.0], [0.0, 4.0]], (5.0, 0.0)),
        ([[3.0, 4.0], [0.0, 0.0]], (5.0, 0.0)),
        ([[0.0, 0.0], [-4.0, 3.0]], (5.0, 0.0)),
        ([[1.5e308, 1.5e308], [0.0, 0.0]], None),
    ]
    G = _G(*[c[0] for c in cases])
    r = oracle.gesvd2(G)
    for i, (m, sv) in enumerate(cases):
        if sv is not None:
            assert (r["S"][0, i], r["S"][1, i]) == sv, (m, r["S"][:, i])
        U, V = _mat(r, "U", i), _mat(r, "V", i)
        S = np.diag(r["S"][:, i])
        if sv is not None and m[0][1] * m[1][0] == 0 or (m[0][0] == 0 and m[1][1] == 0):
            # signed permutations: exact reconstruction
            if (r["info"][i] >> 4) & 15 in (0, 1, 2, 4, 6, 8, 9):
                assert np.array_equal(U @ S @ V.T, np.array(m))
                assert set(np.abs(U).ravel()) <= {0.0, 1.0}
    # 1.5e308 row: sigma1 = sqrt(2) 1.5e308 > nu overflows as a double, not in (e,f) form
    i = len(cases) - 1
    assert math.isinf(r["S"][0, i])
    assert relerr(ef_value(r["Se"][0, i], r["Sf"][0, i]), sigma_closed(1.5e308, 0.0, 1.5e308, 0.0)[0]) <= EPSD


def _exact_R(g, s):
    """Exact R of Sect. 3.2.2 for the prescaled G' = 2^s G: r11 = larger column norm,
    |r12| = |c1 . c2| / r11, |r22| = |det G'| / r11 (90-digit decimal)."""
    import decimal
    D = decimal.Decimal
    with decimal.localcontext() as c:
        c.prec = 90; c.Emax = 10 ** 6; c.Emin = -10 ** 6
        sc = D(2) ** s
        a, cc, b, d = (D(float(x)) * sc for x in g)
        w1 = (a * a + cc * cc).sqrt(); w2 = (b * b + d * d).sqrt()
        r11 = max(w1, w2)
        return r11, abs(a * b + cc * d) / r11, abs(a * d - b * cc) / r11


def test_table_td_bounds_on_R():
    """Thm. 3.5 and Table 1 (t:d): without underflow, r11 is within eps, and r12, r22 within
    4.5 eps (delta_2) -- the element computed by eq. (EXT) within 3.5 eps (delta_3).  The
    near-singular inputs make r22 the result of a massive cancellation, which only eq. (EXT)
    keeps accurate."""
    rng = random.Random(77)
    tol2 = 4.500000001 * EPSD
    count_ext = 0
    for k in range(1200):
        if k % 2 == 0:
            g = I.safe_range(1, 1000 + k, 1000)[:, 0]
        else:
            # nearly rank-one: g22 ~ g12 g21 / g11 (cancellation in r22)
            a = math.ldexp(1 + rng.random(), rng.randint(-20, 20))
            c = math.ldexp(1 + rng.random(), rng.randint(-20, 20))
            b = math.ldexp(1 + rng.random(), rng.randint(-20, 20)) * rng.choice((-1, 1))
            d = float(Fraction(b) * Fraction(c) / Fraction(a)) * (1 + rng.choice((-1, 1)) * rng.random() * 1e-9)
            g = np.array([a, c, b, d])
        tr, ints = oracle.trace(g)
        t, tp, s, flags = ints
        if tp != 15 or flags & oracle.FLAGS["fallback"]:
            continue
        r11, r12, r22 = _exact_R(g, int(s))
        assert relerr(tr[0], r11) <= EPSD * (1 + 1e-9)
        # the trace holds R'' before the sign normalisation of Sect. 3.2.2
        e12, e22 = relerr(abs(tr[1]), r12), relerr(abs(tr[2]), r22)
        assert e12 <= tol2 and e22 <= tol2, (e12 / EPSD, e22 / EPSD)
        if flags & oracle.FLAGS["ext"]:
            count_ext += 1
            # the EXT element is the one with the essential subtraction
            assert min(e12, e22) <= 3.500000001 * EPSD
    assert count_ext > 500


def test_tanphi_in_unit_interval():
    """Cor. 2.2 / Alg. 1: 0 <= tan(phi) <= 1."""
    G = np.concatenate([I.general(400, 51, "d", "narrow"), I.general(400, 52, "d", "wide")], axis=1)
    for i in range(G.shape[1]):
        tr, ints = oracle.trace(G[:, i])
        if ints[1] in (7, 11, 13, 14, 15) and not ints[3] & oracle.FLAGS["fallback"]:
            assert 0 <= tr[4] <= 1


BRANCH_CASES = {
    # name: (matrix, flag that must be set)
    "t2f2_equal_diag": ([[3.0, 1.0], [0.0, 3.0]], "t2f2"),
    "t2f2_small_ratio": ([[1.0, 2.0 ** 60], [0.0, 0.5]], "t2f2"),
    "t2f3": ([[3.0, 1.25], [0.0, 1.25]], "t2f3"),
    "t2inf": ([[2.0 ** 1000, 2.0 ** -1074], [0.0, 2.0 ** 1000]], "t2inf"),
    "tpinf": ([[MU, NU / 4], [0.0, MU]], "tpinf"),
    "swap": ([[1.0, 1.0], [0.0, 2.0]], "swap"),
    "fallback9": ([[1.0, -1.0], [1.0, 1.0]], "fallback"),
    "fallback5": ([[1.0, 2.0], [3.0, 6.0]], "fallback"),
    "ext": ([[1.0, 3.0], [0.3, 0.7]], "ext"),
}


@pytest.mark.parametrize("name", sorted(BRANCH_CASES))
def test_branch_cases(name):
    m, flag = BRANCH_CASES[name]
    G = _G(m)
    r = oracle.gesvd2(G)
    assert (r["info"][0] >> 8) & oracle.FLAGS[flag], (name, r["info"][0])
    assert np.isfinite(r["U"]).all() and np.isfinite(r["V"]).all()
    s1, s2 = sigma_closed(*G[:, 0])
    c1 = ef_value(r["Se"][0, 0], r["Sf"][0, 0]); c2 = ef_value(r["Se"][1, 0], r["Sf"][1, 0])
    assert relerr(c1, s1) <= 5 * EPSD
    if name != "t2inf":
        assert relerr(c2, s2) <= 9 * EPSD or (s2 == 0 and c2 == 0)
    m_ = oracle.dmetrics(G, r)
    assert m_[2, 0] <= 8 * EPSD and m_[3, 0] <= 8 * EPSD


def test_no_inf_nan_in_vectors_and_reproducible():
    """End of Sect. 3.3.2: no Inf/NaN in U and V for any finite G, and bitwise reproducibility."""
    G = np.concatenate([I.general(1 << 13, 61, "d", "wide"), I.general(1 << 12, 62, "d", "narrow")], axis=1)
    G[1, : 1 << 11] = 0
    r1 = oracle.gesvd2(G, nthreads=1)
    r2 = oracle.gesvd2(G, nthreads=4)
    assert np.isfinite(r1["U"]).all() and np.isfinite(r1["V"]).all()
    for k in ("U", "V", "S", "Se", "Sf", "info"):
        assert np.array_equal(r1[k].view(np.uint8), r2[k].view(np.uint8))
    assert np.all(np.isfinite(r1["Sf"]))


def test_nonfinite_input_reported():
    G = _G([[1.0, math.nan], [0.0, 1.0]], [[math.inf, 1.0], [0.0, 1.0]], [[1.0, 2.0], [3.0, 4.0]])
    r = oracle.gesvd2(G)
    assert list(r["info"][:2]) == [-1, -1] and r["info"][2] >= 0
    assert np.isnan(r["S"][:, :2]).all() and np.isfinite(r["S"][:, 2]).all()


def test_trsvd2_equals_gesvd2_on_triangular():
    T = I.triangular(4096, 71, "d", "wide")
    G = np.stack([T[0], np.zeros_like(T[0]), T[1], T[2]])
    a, b = oracle.trsvd2(T[0], T[1], T[2]), oracle.gesvd2(G)
    for k in ("U", "V", "S", "Se", "Sf", "info"):
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8))


def test_single_precision_accuracy():
    """The float variant with T = double in eq. (EXT): same accuracy claims, eps = 2^-24."""
    G = I.general(1 << 13, 81, "s", "narrow")
    r = oracle.gesvd2(G, "s", nthreads=4)
    _check_accuracy(G.astype(np.float64), r, 5, 9, 8, 8, eps=EPSS)
    G = I.safe_range(1 << 12, 82, 0, "s", triangular_=True)
    r = oracle.gesvd2(G, "s")
    _check_accuracy(G.astype(np.float64), r, 5, 5, 8, 8, eps=EPSS)
    T = I.triangular(1024, 83, "s", "wide")
    a = oracle.trsvd2(T[0], T[1], T[2], "s")
    assert np.isfinite(a["U"]).all() and np.isfinite(a["V"]).all()


def test_operation_counts_by_hand():
    """The oracle's operation counters against counts read off the formulas, one input per
    class.  These counts feed the roofline (tests/golden/opcounts.json).
    * diagonal (t = 9): a signed permutation, no arithmetic;
    * one nonzero column or row (t = 3, 5; Sect. 3.1): tan = small/big, sigma1 = hypot,
      sec = hypot(tan, 1), cos = 1/sec, sin = tan/sec: 3 div, 2 hypot;
    * upper triangular, general Alg. 1 branch (t' = 13): h = hypot(r11, r12), the test
      r11/r12 < eps, h (+) r22 and h (-) r22, 2 (.) r12 (.) r22 and d (.) s, their quotient;
      tan phi = t2/(1 + hypot(t2, 1)), sec, cos and sin of phi; Alg. 2: t = fma(r22, tan phi,
      r12), tan psi = t/r11, sec, cos and sin of psi, sec phi (/) sec psi, r11 (/) it and
      r22 (.) it: 3 add, 3 mul, 1 fma, 10 div, 4 hypot;
    * no zeros (t' = 15, Sect. 3.2.2) with an inexact tan theta: two column hypots,
      tan theta and sec theta, the exactness fma, one element by fma and division, the
      other by (EXT) and division; the triangular SVD as above; the heuristic's
      tan phi +- tan theta, its fma denominator, the quotient and its sec, cos and sin:
      4 add, 3 mul, 4 fma, 16 div, 8 hypot, 1 (EXT)."""
    def count(g, tri=False):
        if tri:
            return oracle.opcount(np.array(g, dtype=np.float64).reshape(3, 1), triangular=True)
        return oracle.opcount(np.array(g, dtype=np.float64).reshape(4, 1))
    z = dict(add=0, mul=0, fma=0, div=0, hypot=0, ext=0, sqrt=0)
    assert count([2.0, 0.0, 0.0, 3.0]) == z
    assert count([2.0, 3.0, 0.0, 0.0]) == dict(z, div=3, hypot=2)
    assert count([2.0, 0.0, 3.0, 0.0]) == dict(z, div=3, hypot=2)
    tri = dict(add=3, mul=3, fma=1, div=10, hypot=4, ext=0, sqrt=0)
    assert count([2.0, 0.0, 1.0, 3.0]) == tri
    assert count([2.0, 1.0, 3.0], tri=True) == tri
    assert count([2.0, 1.0, 0.5, 3.0]) == dict(add=4, mul=3, fma=4, div=16, hypot=8, ext=1, sqrt=0)
