"""Pins of the oracle's analytic adjoint of the 2x2 SVD (oracle/k2ref_bwd.c) against central
finite differences of the oracle's forward (the method of Sect. 3), which is separate code.

Loss L(G) = <dS, S(G)> + <dU, U(G)> + <dV, V(G)>.  For well-separated singular values the
derivative of the method's smooth branch is compared with the analytic formula; near-equal
singular values use the singular-value part only (dU = dV = 0), whose gradient
U diag(dS) V^T stays well conditioned."""
import numpy as np
import pytest

import oracle
from paper_2407_13116_gb300 import inputs as I


def _loss(G, dS, dU, dV):
    r = oracle.gesvd2(G)
    return (dS * r["S"]).sum(axis=0) + (dU * r["U"]).sum(axis=0) + (dV * r["V"]).sum(axis=0)


def _fd(G, dS, dU, dV, h):
    """Richardson-extrapolated central differences, one element at a time, with the per-matrix
    step h (it must stay well below sigma2 and sigma1 - sigma2: where det G changes sign the
    convention sigma2 >= 0 flips the second singular pair, a true kink of U and V)."""
    out = np.zeros_like(G)
    for k in range(4):
        def d(hh):
            Gp, Gm = G.copy(), G.copy()
            Gp[k] += hh
            Gm[k] -= hh
            hp, hm = Gp[k] - G[k], G[k] - Gm[k]          # the steps actually taken
            return (_loss(Gp, dS, dU, dV) - _loss(Gm, dS, dU, dV)) / (hp + hm)
        out[k] = (4 * d(h / 2) - d(h)) / 3
    return out


def _step(G):
    r = oracle.gesvd2(G)
    return 1e-3 * np.minimum(r["S"][1], r["S"][0] - r["S"][1])


def _rel(a, b):
    return np.sqrt(((a - b) ** 2).sum(axis=0)) / np.maximum(np.sqrt((b * b).sum(axis=0)), 1e-300)


def test_adjoint_matches_finite_differences_separated():
    G, s1, s2 = I.rotated(512, 77, ecount=10, close_frac=0.0)
    keep = ((s2 / s1) < 0.9) & ((s2 / s1) > 1e-3)
    G = np.ascontiguousarray(G[:, keep])
    n = G.shape[1]
    rng = np.random.default_rng(1)
    dS, dU, dV = rng.standard_normal((2, n)), rng.standard_normal((4, n)), rng.standard_normal((4, n))
    r = oracle.gesvd2(G)
    an = oracle.gesvd2_bwd(r["U"], r["S"], r["V"], dS, dU, dV)
    fd = _fd(G, dS, dU, dV, _step(G))
    err = _rel(fd, an)
    assert np.median(err) < 1e-10 and err.max() < 1e-8, (np.median(err), err.max())


def test_adjoint_sigma_only_near_equal():
    """s2/s1 in (1 - 1e-6, 1]: the singular values kink where they cross, so the step must stay
    below s1 - s2 (here 1e-2 of it); central differences in double then resolve the gradient only
    to about eps * s1 / h, which the bound states per matrix.  The closed form U diag(dS) V^T
    is checked exactly."""
    G, s1, s2 = I.rotated(128, 78, ecount=10, close_frac=1.0)
    n = G.shape[1]
    rng = np.random.default_rng(2)
    dS = rng.standard_normal((2, n))
    z = np.zeros((4, n))
    r = oracle.gesvd2(G)
    an = oracle.gesvd2_bwd(r["U"], r["S"], r["V"], dS, None, None)
    gap = r["S"][0] - r["S"][1]
    h = 1e-2 * gap
    fd = _fd(G, dS, z, z, h)
    err = _rel(fd, an)
    floor = 200 * 2.0 ** -53 * r["S"][0] / h       # rounding floor of a double central difference
    assert np.all(err <= 1e-8 + floor), (err / (1e-8 + floor)).max()
    assert np.median(err) < 1e-6
    for i in range(n):
        U = np.array([[r["U"][0, i], r["U"][2, i]], [r["U"][1, i], r["U"][3, i]]])
        V = np.array([[r["V"][0, i], r["V"][2, i]], [r["V"][1, i], r["V"][3, i]]])
        ref = (U @ np.diag(dS[:, i]) @ V.T).T.ravel()     # column-major planes
        assert np.allclose(ref, an[:, i], rtol=1e-14, atol=1e-14 * np.abs(ref).max())


def test_gap_threshold_keeps_degenerate_finite():
    # identity and scaled orthogonal matrices: sigma1 = sigma2, the rotation part uses tau * sigma1
    G = np.array([[1.0, 2.0, 0.0], [0.0, 0.0, 3.0], [0.0, 0.0, -3.0], [1.0, 2.0, 0.0]])
    r = oracle.gesvd2(G)
    rng = np.random.default_rng(3)
    dG = oracle.gesvd2_bwd(r["U"], r["S"], r["V"], rng.standard_normal((2, 3)), rng.standard_normal((4, 3)),
                           rng.standard_normal((4, 3)), tau=1e-10)
    assert np.isfinite(dG).all()
    z = oracle.gesvd2_bwd(r["U"], r["S"], r["V"], None, None, None)
    assert (z == 0).all()


def test_adjoint_closed_form_diagonal():
    """G = diag(s1, s2): dL/dG21 = -s1/(s1^2-s2^2) and dL/dG12 = -s2/(s1^2-s2^2) for L = U12
    (the first-order rotation of the left singular vectors)."""
    s1, s2 = 3.0, 2.0
    G = np.array([[s1], [0.0], [0.0], [s2]])
    r = oracle.gesvd2(G)
    dU = np.zeros((4, 1)); dU[2, 0] = 1.0      # L = U12
    dG = oracle.gesvd2_bwd(r["U"], r["S"], r["V"], None, dU, None)
    assert np.isclose(dG[1, 0], -s1 / (s1 ** 2 - s2 ** 2), rtol=1e-15)
    assert np.isclose(dG[2, 0], -s2 / (s1 ** 2 - s2 ** 2), rtol=1e-15)
    assert dG[0, 0] == 0 and dG[3, 0] == 0
