"""Pins of the oracle's complex 2x2 SVD (Sect. 3.4), independent of its code: LAPACK's complex
SVD (numpy), |det G| and ||G||_F in exact rational arithmetic, unitarity and the residual,
the real method bit for bit on real input, i times the real method on purely imaginary
input, and invariance of the singular values under row and column phases."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

EPS = {"d": 2.0 ** -53, "s": 2.0 ** -24}


def _cm(P, i):
    return np.array([[P[0, i] + 1j * P[1, i], P[4, i] + 1j * P[5, i]],
                     [P[2, i] + 1j * P[3, i], P[6, i] + 1j * P[7, i]]], dtype=np.complex128)


def _planes(mats, T):
    G = np.empty((8, len(mats)), T)
    for i, A in enumerate(mats):
        for e, (r, c) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
            G[2 * e, i] = A[r, c].real
            G[2 * e + 1, i] = A[r, c].imag
    return G


def _random(n, rng, emin, emax, T, pattern=None):
    mats = []
    for _ in range(n):
        e = rng.integers(emin, emax + 1, size=(2, 2, 2))
        m = rng.uniform(1, 2, size=(2, 2, 2)) * rng.choice((-1, 1), size=(2, 2, 2)) * np.ldexp(1.0, e)
        A = (m[..., 0] + 1j * m[..., 1]).astype(np.complex128)
        pat = pattern if pattern is not None else rng.integers(1, 16)
        for k, (r, c) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
            if not (pat >> k) & 1:
                A[r, c] = 0
        if T == np.float32:
            A = A.astype(np.complex64).astype(np.complex128)
        mats.append(A)
    return mats


def _fr(x):
    return Fraction(float(x))


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("pattern", [None, 15, 7, 11, 13, 14, 3, 5, 9, 6, 1])
def test_against_lapack_and_invariants(prec, pattern):
    T = np.float64 if prec == "d" else np.float32
    eps = EPS[prec]
    rng = np.random.default_rng(11 + (pattern or 0))
    er = 20 if prec == "d" else 8
    mats = _random(600, rng, -er, er, T, pattern)
    U, V, S, info = oracle.cgesvd2(_planes(mats, T), prec)
    for i, A in enumerate(mats):
        u, v, s = _cm(U, i), _cm(V, i), S[:, i].astype(np.float64)
        assert s[0] >= s[1] >= 0
        # the complex assembly adds the roundings of the complex products (Sect. 3.4 item 2)
        assert np.abs(u.conj().T @ u - np.eye(2)).max() <= 16 * eps
        assert np.abs(v.conj().T @ v - np.eye(2)).max() <= 16 * eps
        nA = np.linalg.norm(A)
        assert np.linalg.norm(A - u @ np.diag(s) @ v.conj().T) <= 16 * eps * nA
        ref = np.linalg.svd(A, compute_uv=False)
        assert abs(s[0] - ref[0]) <= 8 * eps * ref[0]
        assert abs(s[1] - ref[1]) <= 8 * eps * ref[0]
        # ||G||_F^2 and |det G|^2 exactly
        comps = [(_fr(z.real), _fr(z.imag)) for z in (A[0, 0], A[1, 0], A[0, 1], A[1, 1])]
        fro2 = sum(a * a + b * b for a, b in comps)
        (a11, b11), (a21, b21), (a12, b12), (a22, b22) = comps
        dre = a11 * a22 - b11 * b22 - (a12 * a21 - b12 * b21)
        dim = a11 * b22 + b11 * a22 - (a12 * b21 + b12 * a21)
        det2 = dre * dre + dim * dim
        s0, s1 = _fr(s[0]), _fr(s[1])
        assert abs(s0 * s0 + s1 * s1 - fro2) <= 32 * Fraction(eps) * fro2
        if det2:
            assert abs(s0 * s0 * s1 * s1 - det2) <= 32 * Fraction(eps) * s0 * s0 * s0 * s0 + Fraction(0)


def test_real_input_is_the_real_method():
    rng = np.random.default_rng(3)
    from paper_2407_13116_gb300 import inputs as I
    Gr = I.general(3000, 21, "d", "narrow")
    G8 = np.zeros((8, Gr.shape[1]))
    G8[0::2] = Gr
    U, V, S, info = oracle.cgesvd2(G8)
    r = oracle.gesvd2(Gr)
    assert np.array_equal(U[0::2], r["U"]) and np.array_equal(V[0::2], r["V"]) and np.array_equal(S, r["S"])
    assert not U[1::2].any() and not V[1::2].any()


def test_imaginary_input_is_i_times_the_real_method():
    from paper_2407_13116_gb300 import inputs as I
    Gr = I.general(3000, 22, "d", "wide")
    G8 = np.zeros((8, Gr.shape[1]))
    G8[1::2] = Gr
    U, V, S, info = oracle.cgesvd2(G8)
    r = oracle.gesvd2(Gr)
    assert np.array_equal(U[1::2], r["U"]) and not U[0::2].any()
    assert np.array_equal(V[0::2], r["V"]) and not V[1::2].any()
    assert np.array_equal(S, r["S"])
    assert ((info >> 8) & 0x100).all()


def test_phase_invariance():
    rng = np.random.default_rng(5)
    mats = _random(500, rng, -10, 10, np.float64, 15)
    ph = np.exp(1j * rng.uniform(0, 2 * np.pi, (500, 4)))
    mats2 = [np.diag(p[:2]) @ A @ np.diag(p[2:]) for A, p in zip(mats, ph)]
    S1 = oracle.cgesvd2(_planes(mats, np.float64))[2]
    S2 = oracle.cgesvd2(_planes(mats2, np.float64))[2]
    assert np.all(np.abs(S1 - S2) <= 16 * EPS["d"] * S1[0])


def test_near_overflow_and_tiny():
    rng = np.random.default_rng(6)
    big = _random(300, rng, 1015, 1022, np.float64, 15)
    tiny = _random(300, rng, -1070, -1000, np.float64, 15)
    for mats in (big, tiny):
        U, V, S, info = oracle.cgesvd2(_planes(mats, np.float64))
        assert np.isfinite(S).all() and np.isfinite(U).all() and np.isfinite(V).all()
        for i, A in enumerate(mats):
            k = -int(np.floor(np.log2(np.abs(A).max())))
            As = np.ldexp(A.real, k) + 1j * np.ldexp(A.imag, k)
            ref = np.ldexp(np.linalg.svd(As, compute_uv=False), -k)
            assert abs(S[0, i] - ref[0]) <= 8 * EPS["d"] * ref[0]


def test_nonfinite():
    G = np.zeros((8, 2))
    G[:, 0] = 1.0
    G[3, 1] = np.inf
    U, V, S, info = oracle.cgesvd2(G)
    assert info[1] == -1 and np.isnan(S[:, 1]).all() and np.isnan(U[:, 1]).all()
    assert info[0] != -1 and np.isfinite(S[:, 0]).all()
