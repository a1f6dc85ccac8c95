"""Pins of the oracle's rectangular SVD (QR with column pivoting to a square matrix, then the
n x n Kogbetliantz method; Sect. 1): LAPACK's SVD (numpy), orthonormal U and V, the
residual, exact scaling by powers of two, the transpose relation, special matrices."""
import numpy as np
import pytest

import oracle

EPS = {"d": 2.0 ** -52, "s": 2.0 ** -23}


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("shape", [(10, 4), (4, 10), (7, 7), (1, 5), (5, 1), (1, 1), (60, 33), (33, 60), (96, 17)])
def test_against_lapack(prec, shape):
    T = np.float64 if prec == "d" else np.float32
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    m, n = shape
    k = min(m, n)
    for rep in range(3):
        A = (rng.standard_normal((m, n)) * 2.0 ** rng.integers(-20, 20)).astype(T)
        U, S, V, sw, info = oracle.gesvdr(A, prec)
        assert info == 0 and U.shape == (m, k) and V.shape == (n, k) and S.shape == (k,)
        tol = 8 * max(m, n) * EPS[prec]
        ref = np.linalg.svd(A.astype(np.float64), compute_uv=False)
        assert np.all(np.diff(S) <= 0) and np.all(S >= 0)
        assert np.abs(S - ref).max() <= tol * ref[0]
        assert np.abs(U.T.astype(np.float64) @ U - np.eye(k)).max() <= tol
        assert np.abs(V.T.astype(np.float64) @ V - np.eye(k)).max() <= tol
        Ad = A.astype(np.float64)
        assert np.linalg.norm(Ad - (U * S) @ V.T) <= tol * np.linalg.norm(Ad)


def test_power_of_two_scaling_is_exact():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((23, 9))
    U, S, V, _, _ = oracle.gesvdr(A)
    for k in (-300, -7, 5, 600):
        U2, S2, V2, _, _ = oracle.gesvdr(np.ldexp(A, k))
        assert np.array_equal(S2, np.ldexp(S, k)) and np.array_equal(U2, U) and np.array_equal(V2, V)


def test_transpose_exchanges_the_factors():
    rng = np.random.default_rng(5)
    for shape in ((17, 6), (6, 17), (1, 8)):
        A = rng.standard_normal(shape)
        U, S, V, _, _ = oracle.gesvdr(A)
        Ut, St, Vt, _, _ = oracle.gesvdr(A.T)
        assert np.array_equal(S, St) and np.array_equal(U, Vt) and np.array_equal(V, Ut)


def test_special_matrices():
    U, S, V, sw, info = oracle.gesvdr(np.zeros((6, 4)))
    assert info == 0 and not S.any() and np.allclose(U.T @ U, np.eye(4)) and np.allclose(V.T @ V, np.eye(4))
    rng = np.random.default_rng(6)
    B = rng.standard_normal((12, 2)) @ rng.standard_normal((2, 5))          # rank 2
    U, S, V, sw, info = oracle.gesvdr(B)
    ref = np.linalg.svd(B, compute_uv=False)
    assert info == 0 and np.abs(S - ref).max() <= 100 * EPS["d"] * ref[0]
    A = np.ones((5, 3)); A[2, 1] = np.nan
    U, S, V, sw, info = oracle.gesvdr(A)
    assert info == -1 and np.isnan(S).all() and np.isnan(U).all() and np.isnan(V).all()
