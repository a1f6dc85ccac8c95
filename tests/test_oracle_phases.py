"""Pins of the oracle's standalone phases: the prescaling of Sect. 3.1 (eqs. (eG), (s)) as
its own entry, and the xLASV2 argument shape computed by the method.  Independent checks:
exact power-of-two scaling by Python's ldexp, the type classes restated from their
definitions, LAPACK's defining identity of xLASV2 in exact rational arithmetic, and
LAPACK's own DLASV2 singular values where the bundled LAPACK exports it."""
import ctypes as C
import glob
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2407_13116_gb300 import inputs as I

E_NU = {"d": 1023, "s": 127}
EPS = {"d": 2.0 ** -53, "s": 2.0 ** -24}


def _class(g11, g21, g12, g22):
    """Class of a zero pattern (Sect. 3.1): 15 = no zeros; 13 = three nonzeros; 3 = one
    column nonzero in both rows; 5 = one row nonzero in both columns; 9 = at most one
    nonzero in every row and every column (zero, one element, diagonal, anti-diagonal)."""
    nz = [x != 0 for x in (g11, g21, g12, g22)]
    k = sum(nz)
    if k == 4:
        return 15
    if k == 3:
        return 13
    if k == 2:
        if nz[0] and nz[1] or nz[2] and nz[3]:
            return 3
        if nz[0] and nz[2] or nz[1] and nz[3]:
            return 5
    return 9


def _expo(x):
    return math.frexp(x)[1] - 1      # floor(lg |x|), also for subnormals


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("extra", [0, 1, 3])
def test_prescale_definition(prec, extra):
    T = np.float64 if prec == "d" else np.float32
    rng = np.random.default_rng(5 + extra)
    G = np.concatenate([I.general(3000, 41, prec, "wide"), I.general(3000, 42, prec, "narrow")], axis=1)
    # zero patterns of every class
    mask = rng.random(G.shape) < 0.25
    G = np.where(mask, T(0), G).astype(T)
    Gs, s, types = oracle.prescale2(G, prec, extra)
    for i in range(G.shape[1]):
        g = [float(x) for x in G[:, i]]
        cls = _class(g[0], g[1], g[2], g[3])
        t = sum(1 << k for k, x in enumerate(g) if x != 0)
        if cls == 9:
            want_s = 0
        else:
            eG = max(_expo(x) for x in g if x != 0)
            want_s = E_NU[prec] - eG - (2 if cls == 15 else 1) - extra
        assert s[i] == want_s, (g, s[i], want_s)
        want = [T(math.ldexp(x, want_s)) for x in g]          # one correct rounding each
        assert all(float(a) == float(b) and math.copysign(1, a) == math.copysign(1, b)
                   for a, b in zip(Gs[:, i], want)), (g, Gs[:, i], want)
        tp = sum(1 << k for k, x in enumerate(Gs[:, i]) if x != 0)
        assert types[i] == t | (tp << 4)
        if cls != 9:
            assert max(_expo(float(x)) for x in Gs[:, i] if x != 0) == E_NU[prec] - (2 if cls == 15 else 1) - extra


def test_prescale_nonfinite_copied():
    G = np.array([[1.0, np.inf], [2.0, 1.0], [np.nan, 0.5], [3.0, 2.0]])
    Gs, s, types = oracle.prescale2(G)
    assert list(types) == [-1, -1] and list(s) == [0, 0]
    assert np.array_equal(Gs, G, equal_nan=True)


def _lapack_dlasv2():
    import scipy
    for lib in glob.glob(os.path.join(os.path.dirname(os.path.dirname(scipy.__file__)), "scipy.libs", "*openblas*.so*")):
        h = C.CDLL(lib)
        for name in ("scipy_dlasv2_", "dlasv2_"):
            if hasattr(h, name):
                f = getattr(h, name)
                f.argtypes = [C.POINTER(C.c_double)] * 9
                return f
    return None


def _frac_identity_residual(f, g, h, ssmin, ssmax, snr, csr, snl, csl):
    F = [Fraction(x) for x in (f, g, h, ssmin, ssmax, snr, csr, snl, csl)]
    f, g, h, ssmin, ssmax, snr, csr, snl, csl = F
    L = [[csl, snl], [-snl, csl]]
    A = [[f, g], [0, h]]
    R = [[csr, -snr], [snr, csr]]
    LA = [[sum(L[i][k] * A[k][j] for k in range(2)) for j in range(2)] for i in range(2)]
    M = [[sum(LA[i][k] * R[k][j] for k in range(2)) for j in range(2)] for i in range(2)]
    D = [[ssmax, 0], [0, ssmin]]
    return max(abs(M[i][j] - D[i][j]) for i in range(2) for j in range(2))


@pytest.mark.parametrize("prec", ["d", "s"])
def test_lasv2_identity_and_signs(prec):
    T = np.float64 if prec == "d" else np.float32
    Fh = I.triangular(4000, 43, prec, "narrow")
    F, Gp, H = Fh[0], Fh[1], Fh[2]
    out = oracle.lasv2(F, Gp, H, prec)
    ssmin, ssmax, snr, csr, snl, csl = out
    eps = EPS[prec]
    for i in range(len(F)):
        vals = [float(x[i]) for x in out]
        f, g, h = float(F[i]), float(Gp[i]), float(H[i])
        assert vals[1] >= 0 and abs(vals[0]) <= vals[1]
        res = _frac_identity_residual(f, g, h, *vals)
        assert res <= 16 * eps * Fraction(vals[1]), (f, g, h, vals, float(res))
        for c, sn in ((csl[i], snl[i]), (csr[i], snr[i])):
            assert abs(Fraction(float(c)) ** 2 + Fraction(float(sn)) ** 2 - 1) <= 4 * eps
        if f != 0 and h != 0:
            assert (vals[0] > 0) == ((f > 0) == (h > 0))        # sign of det R = F H
            assert abs(Fraction(vals[0]) * Fraction(vals[1]) - Fraction(f) * Fraction(h)) <= 8 * eps * abs(Fraction(f) * Fraction(h))


def test_lasv2_against_lapack():
    """|SSMAX|, |SSMIN| against LAPACK's DLASV2 (a different algorithm): both are accurate to a
    few ulps on triangular inputs of moderate range (Sect. 4)."""
    f_l = _lapack_dlasv2()
    if f_l is None:
        pytest.skip("the bundled LAPACK does not export dlasv2")
    Fh = I.triangular(3000, 44, "d", "narrow")
    ssmin, ssmax, snr, csr, snl, csl = oracle.lasv2(Fh[0], Fh[1], Fh[2])
    for i in range(Fh.shape[1]):
        a = [C.c_double(float(Fh[k][i])) for k in range(3)] + [C.c_double() for _ in range(6)]
        f_l(*[C.byref(x) for x in a])
        lmin, lmax = abs(a[3].value), abs(a[4].value)
        assert abs(lmax - ssmax[i]) <= 4 * 2.0 ** -52 * lmax
        assert abs(lmin - abs(ssmin[i])) <= 8 * 2.0 ** -52 * max(lmin, 1e-300) + 4 * 2.0 ** -52 * lmax * (lmin == 0)
        # LAPACK's SSMAX * SSMIN = F H as well: the same sign of the determinant
        if lmin != 0:
            assert (a[3].value * a[4].value > 0) == (ssmin[i] * ssmax[i] > 0)


def test_lasv2_matches_triangular_entry():
    """The wrapper is the triangular SVD re-expressed: SSMAX = sigma1, |SSMIN| = sigma2, and
    (CSL, SNL), (CSR, SNR) are the first columns of U, V."""
    Fh = I.triangular(2000, 45, "d", "wide")
    ssmin, ssmax, snr, csr, snl, csl = oracle.lasv2(Fh[0], Fh[1], Fh[2])
    r = oracle.trsvd2(Fh[0], Fh[1], Fh[2])
    assert np.array_equal(ssmax, r["S"][0]) and np.array_equal(np.abs(ssmin), r["S"][1])
    assert np.array_equal(csl, r["U"][0]) and np.array_equal(snl, r["U"][1])
    assert np.array_equal(csr, r["V"][0]) and np.array_equal(snr, r["V"][1])


def test_lasv2_nonfinite():
    out = oracle.lasv2(np.array([1.0, np.inf]), np.array([2.0, 0.0]), np.array([3.0, 1.0]))
    assert all(np.isnan(o[1]) for o in out) and not any(np.isnan(o[0]) for o in out)
