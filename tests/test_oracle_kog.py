"""Pins of the oracle's n x n Kogbetliantz driver (eq. (SVD) with the modulus strategy):
order 2 reduces to one 2x2 SVD of Sect. 3; the singular values match the construction
Q1 diag(sigma) Q2^T and LAPACK's SVD (numpy) to within the backward-error bound; U and V are
orthogonal; the residual is small; the off-norm test holds at exit; exact special cases."""
import numpy as np
import pytest

import oracle
from paper_2407_13116_gb300 import inputs as I

EPS = 2.0 ** -52


def test_order_two_is_the_2x2_method():
    # exponent spreads below 1000, so the n x n method's power-of-two prescaling stays exact
    G = np.concatenate([I.general(200, 91, "d", "narrow"), I.safe_range(200, 92, 1043)], axis=1)
    r = oracle.gesvd2(G)
    for i in range(G.shape[1]):
        A = np.array([[G[0, i], G[2, i]], [G[1, i], G[3, i]]])
        U, S, V, sw, info = oracle.kogbet(A)
        assert info == 0 and sw <= 1
        if sw == 1:
            assert np.array_equal(S, r["S"][:, i])
            assert np.array_equal(U.T.ravel(), r["U"][:, i]) and np.array_equal(V.T.ravel(), r["V"][:, i])
        else:   # off-diagonal below n eps ||A||_F from the start: signs and order only
            assert np.array_equal(S, np.sort(np.abs(np.diag(A)))[::-1]) or np.allclose(S, r["S"][:, i], rtol=4e-16)
            assert np.all(S >= 0)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 8, 17, 32, 33, 64])
def test_accuracy_against_construction_and_lapack(n):
    A, sig = I.kog_matrix(n, 3, n)
    U, S, V, sw, info = oracle.kogbet(A)
    assert info == 0 and sw < 40
    s1 = sig[0]
    assert np.all(np.diff(S) <= 0) and np.all(S >= 0)
    assert np.abs(S - sig).max() <= 8 * n * EPS * s1
    assert np.abs(S - np.linalg.svd(A, compute_uv=False)).max() <= 8 * n * EPS * s1
    assert np.abs(U.T @ U - np.eye(n)).max() <= 4 * n * EPS
    assert np.abs(V.T @ V - np.eye(n)).max() <= 4 * n * EPS
    assert np.linalg.norm(A - (U * S) @ V.T) <= 4 * n * EPS * np.linalg.norm(A)
    # the stopping test: off(U^T A V) small relative to ||A||_F
    B = U.T @ A @ V
    off = np.linalg.norm(B - np.diag(np.diag(B)))
    assert off <= 4 * n * EPS * np.linalg.norm(A)


def test_special_matrices_exact():
    # zero: no sweep
    U, S, V, sw, info = oracle.kogbet(np.zeros((6, 6)))
    assert sw == 0 and info == 0 and (S == 0).all() and np.array_equal(U, np.eye(6))
    # diagonal with mixed signs: the sweep fixes signs and the sort orders
    d = np.array([3.0, -5.0, 0.5, 2.0, -0.25])
    U, S, V, sw, info = oracle.kogbet(np.diag(d))
    assert np.array_equal(S, np.sort(np.abs(d))[::-1])
    assert np.array_equal(np.abs(U), np.abs(U).round()) and np.array_equal((U * S) @ V.T, np.diag(d))
    # a permutation matrix scaled by a power of two
    P = np.eye(7)[[3, 0, 6, 1, 5, 2, 4]] * 2.0 ** 40
    U, S, V, sw, info = oracle.kogbet(P)
    assert np.array_equal(S, np.full(7, 2.0 ** 40)) and np.array_equal((U * S) @ V.T, P)


def test_nonfinite_input():
    A = np.eye(4)
    A[2, 1] = np.inf
    U, S, V, sw, info = oracle.kogbet(A)
    assert info == -1 and sw == 0 and np.isnan(S).all()


def test_single_precision():
    A, sig = I.kog_matrix(24, 5, 0, smin=1e-4)
    U, S, V, sw, info = oracle.kogbet(A.astype(np.float32), "s")
    e = 2.0 ** -23
    assert info == 0
    assert np.abs(S - sig).max() <= 8 * 24 * e * sig[0]
    U, V = U.astype(np.float64), V.astype(np.float64)
    assert np.abs(U.T @ U - np.eye(24)).max() <= 4 * 24 * e


def test_sigma_gradient_closed_form():
    A, _ = I.kog_matrix(9, 6, 0, smin=0.1)      # singular values well above the FD step
    U, S, V, sw, info = oracle.kogbet(A)
    dS = np.linspace(-1, 1, 9)
    dA = oracle.kog_sigma_bwd(U, V, dS)
    assert np.allclose(dA, (U * dS) @ V.T, rtol=0, atol=16 * 9 * EPS)
    # finite differences of the oracle's singular values
    h = 1e-6
    for (r, c) in [(0, 0), (3, 7), (8, 2)]:
        Ap, Am = A.copy(), A.copy()
        Ap[r, c] += h
        Am[r, c] -= h
        fd = (dS @ oracle.kogbet(Ap)[1] - dS @ oracle.kogbet(Am)[1]) / (2 * h)
        assert abs(fd - dA[r, c]) <= 1e-8
