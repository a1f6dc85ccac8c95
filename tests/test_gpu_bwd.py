"""GPU backward (adjoint) of the batched 2x2 SVD: k2svd_{d,s}gesvd2_bwd and the autograd
Function, against the oracle's analytic binary128 adjoint and against central finite
differences of the GPU forward."""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_13116_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EPS = 2.0 ** -53


def k2():
    from paper_2407_13116_gb300 import k2svd
    return k2svd


def _fwd(G):
    U, V, S, _, _, _ = k2().gesvd2(torch.from_numpy(np.ascontiguousarray(G)).to(DEV), want_info=False)
    return U, V, S


def _mag(U, S, V, dS, dU, dV, tau=1e-10):
    """|dS1| + |dS2| + |m12| + |m21| with the formula's magnitudes (for error bounds)."""
    a = np.abs(U[0] * dU[2]) + np.abs(U[1] * dU[3]) + np.abs(U[2] * dU[0]) + np.abs(U[3] * dU[1])
    b = np.abs(V[0] * dV[2]) + np.abs(V[1] * dV[3]) + np.abs(V[2] * dV[0]) + np.abs(V[3] * dV[1])
    s1, s2 = S
    g = np.maximum(s1 - s2, tau * s1)
    f = np.where(s1 > 0, 1.0 / np.where(s1 > 0, g * (s1 + s2), 1.0), 0.0)
    return np.abs(dS[0]) + np.abs(dS[1]) + f * (a * s2 + b * s1) + f * (a * s1 + b * s2)


@pytest.mark.parametrize("n", [1, 33, (1 << 16) + 5])
def test_adjoint_matches_oracle(n):
    G, _, _ = I.rotated(n, 500 + n)
    U, V, S = _fwd(G)
    rng = np.random.default_rng(n)
    dS, dU, dV = rng.standard_normal((2, n)), rng.standard_normal((4, n)), rng.standard_normal((4, n))
    t = lambda x: torch.from_numpy(x).to(DEV)
    dG = k2().gesvd2_bwd(U, S, V, t(dS), t(dU), t(dV)).cpu().numpy()
    Un, Sn, Vn = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    ref = oracle.gesvd2_bwd(Un, Sn, Vn, dS, dU, dV)
    err = np.sqrt(((dG - ref) ** 2).sum(axis=0))
    bound = 64 * EPS * _mag(Un, Sn, Vn, dS, dU, dV)
    assert np.all(err <= bound), (err / bound).max()


def test_optional_upstream_gradients():
    n = 4096
    G, _, _ = I.rotated(n, 601)
    U, V, S = _fwd(G)
    rng = np.random.default_rng(9)
    dS = rng.standard_normal((2, n))
    Un, Sn, Vn = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    got = k2().gesvd2_bwd(U, S, V, torch.from_numpy(dS).to(DEV), None, None).cpu().numpy()
    ref = oracle.gesvd2_bwd(Un, Sn, Vn, dS, None, None)
    assert np.allclose(got, ref, rtol=0, atol=16 * EPS * np.abs(dS).sum(axis=0).max())
    zero = k2().gesvd2_bwd(U, S, V).cpu().numpy()
    assert (zero == 0).all()


def _loss_gpu(G, dS, dU, dV):
    U, V, S = _fwd(G)
    return ((dS * S.cpu().numpy()).sum(axis=0) + (dU * U.cpu().numpy()).sum(axis=0)
            + (dV * V.cpu().numpy()).sum(axis=0))


def _fd_gpu(G, dS, dU, dV, h, richardson=True):
    """Central differences of the loss per matrix and element, divided by the step actually
    taken (G[k] +- h rounded to a double); Richardson extrapolation over h and h/2."""
    out = np.zeros_like(G)
    for k in range(4):
        def d(hh):
            Gp, Gm = G.copy(), G.copy()
            Gp[k] += hh
            Gm[k] -= hh
            return (_loss_gpu(Gp, dS, dU, dV) - _loss_gpu(Gm, dS, dU, dV)) / ((Gp[k] - G[k]) + (G[k] - Gm[k]))
        out[k] = (4 * d(h / 2) - d(h)) / 3 if richardson else d(h)
    return out


def _rel(fd, an):
    return np.sqrt(((fd - an) ** 2).sum(axis=0)) / np.sqrt((an ** 2).sum(axis=0))


def test_finite_differences_4096():
    """The differentiation workload: all 4096 matrices R(theta) diag(s1, s2) R(phi)^T
    (s2/s1 log-uniform in [1e-12, 1], 10% within 1e-6 of 1), checked against central
    differences of the GPU forward, each group with the loss and step its conditioning allows:
      * 1e-3 < s2/s1 <= 1 - 2e-6: the full loss (dS, dU, dV ~ N(0,1)), step 1e-3 min(s2, s1 - s2),
        to 1e-8 relative;
      * s2/s1 > 1 - 2e-6 (near-equal, where U and V are ill-conditioned): the singular-value
        loss, step 1e-2 (s1 - s2), to 1e-8 plus the rounding floor 200 eps s1 / h of a double
        central difference;
      * s2/s1 <= 1e-3: the singular-value loss, since any step above the rounding floor of U
        and V is far above sigma2 and can flip the sign of det G, and with it the sign of the
        second singular pair: sigma1 alone with step 1e-6 s1, and sigma2 alone with step
        1e-3 s2 (a few ulps of the entries; the exact differences divide), each to 1e-8 plus
        64 eps sigma_i / h -- the second holds only because the method computes a tiny sigma2
        to a few ulps relative (Sect. 4)."""
    n = 4096
    G, s1, s2 = I.rotated(n, 0x240713116 + 3)
    U, V, S = _fwd(G)
    Sn = S.cpu().numpy()
    ratio = Sn[1] / Sn[0]
    rng = np.random.default_rng(4)
    dS, dU, dV = rng.standard_normal((2, n)), rng.standard_normal((4, n)), rng.standard_normal((4, n))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    sep = (ratio > 1e-3) & (ratio <= 1 - 2e-6)
    near = ratio > 1 - 2e-6
    small = ratio <= 1e-3
    assert (sep | near | small).all() and sep.sum() > 500 and near.sum() > 200 and small.sum() > 2000
    # separated
    Gs = np.ascontiguousarray(G[:, sep])
    Us, Vs, Ss = _fwd(Gs)
    an = k2().gesvd2_bwd(Us, Ss, Vs, t(dS[:, sep]), t(dU[:, sep]), t(dV[:, sep])).cpu().numpy()
    S_s = Ss.cpu().numpy()
    h = 1e-3 * np.minimum(S_s[1], S_s[0] - S_s[1])
    rel = _rel(_fd_gpu(Gs, dS[:, sep], dU[:, sep], dV[:, sep], h), an)
    assert rel.max() < 1e-8, rel.max()
    # near-equal singular values
    Gn = np.ascontiguousarray(G[:, near])
    Un, Vn, Sn2 = _fwd(Gn)
    z = np.zeros((4, near.sum()))
    an = k2().gesvd2_bwd(Un, Sn2, Vn, t(dS[:, near])).cpu().numpy()
    S_n = Sn2.cpu().numpy()
    h = 1e-2 * (S_n[0] - S_n[1])
    rel = _rel(_fd_gpu(Gn, dS[:, near], z, z, h), an)
    floor = 200 * EPS * S_n[0] / h
    assert np.all(rel <= 1e-8 + floor)
    # widely separated: sigma1 alone with a step on its scale ...
    Gw = np.ascontiguousarray(G[:, small])
    Uw, Vw, Sw = _fwd(Gw)
    S_w = Sw.cpu().numpy()
    z = np.zeros((4, small.sum()))
    dSa = np.zeros((2, small.sum()))
    dSa[0] = dS[0, small]
    an = k2().gesvd2_bwd(Uw, Sw, Vw, t(dSa)).cpu().numpy()
    h = 1e-6 * S_w[0]
    rel = _rel(_fd_gpu(Gw, dSa, z, z, h), an)
    floor = 64 * EPS * S_w[0] / h
    assert np.all(rel <= 1e-8 + floor), (rel / (1e-8 + floor)).max()
    # ... and sigma2 alone with a step on its own scale
    dSb = np.zeros_like(dSa)
    dSb[1] = dS[1, small]
    an = k2().gesvd2_bwd(Uw, Sw, Vw, t(dSb)).cpu().numpy()
    h = 1e-3 * S_w[1]
    rel = _rel(_fd_gpu(Gw, dSb, z, z, h, richardson=False), an)
    floor = 64 * EPS * S_w[1] / h
    assert np.all(rel <= 1e-8 + floor), (rel / (1e-8 + floor)).max()


def test_autograd_function_gradcheck():
    from paper_2407_13116_gb300.autograd import svd2x2
    G, s1, s2 = I.rotated(256, 777, ecount=2, close_frac=0.0)
    G = G[:, (s2 / s1 > 0.1) & (s2 / s1 < 0.8)][:, :6]       # smooth away from kinks
    A = torch.from_numpy(np.stack([G[0], G[2], G[1], G[3]], -1).reshape(-1, 2, 2)).to(DEV).requires_grad_(True)
    U, S, V = svd2x2(A)
    rec = U @ torch.diag_embed(S) @ V.mT
    assert torch.allclose(rec, A, atol=1e-13 * A.abs().max().item())
    assert torch.autograd.gradcheck(lambda x: svd2x2(x)[1], (A,), eps=1e-7, atol=1e-6, rtol=1e-6)
    assert torch.autograd.gradcheck(lambda x: svd2x2(x)[0], (A,), eps=1e-7, atol=1e-6, rtol=1e-6)
    assert torch.autograd.gradcheck(lambda x: svd2x2(x)[2], (A,), eps=1e-7, atol=1e-6, rtol=1e-6)
    # the backward of the Function is the C-ABI adjoint
    gU, gS, gV = torch.randn_like(A), torch.randn_like(S), torch.randn_like(A)
    (dA,) = torch.autograd.grad((U * gU).sum() + (S * gS).sum() + (V * gV).sum(), A)
    k2svd = k2()
    Up, Vp, Sp = k2svd.to_planes(U.detach()), k2svd.to_planes(V.detach()), S.detach().t().contiguous()
    ref = k2svd.gesvd2_bwd(Up, Sp, Vp, gS.t().contiguous(), k2svd.to_planes(gU), k2svd.to_planes(gV))
    assert torch.equal(k2svd.to_planes(dA), ref)


def test_single_precision_backward():
    n = 20000
    G, _, _ = I.rotated(n, 801, ecount=10, close_frac=0.0)
    G32 = G.astype(np.float32)
    U, V, S, _, _, _ = k2().gesvd2(torch.from_numpy(G32).to(DEV), want_info=False)
    rng = np.random.default_rng(5)
    dS, dU, dV = (rng.standard_normal(s).astype(np.float32) for s in ((2, n), (4, n), (4, n)))
    t = lambda x: torch.from_numpy(x).to(DEV)
    dG = k2().gesvd2_bwd(U, S, V, t(dS), t(dU), t(dV)).cpu().numpy().astype(np.float64)
    Un, Sn, Vn = (x.cpu().numpy().astype(np.float64) for x in (U, S, V))
    ref = oracle.gesvd2_bwd(Un, Sn, Vn, dS.astype(np.float64), dU.astype(np.float64), dV.astype(np.float64))
    err = np.sqrt(((dG - ref) ** 2).sum(axis=0))
    bound = 64 * 2.0 ** -24 * _mag(Un, Sn, Vn, dS, dU, dV)
    assert np.all(err <= bound), (err / bound).max()


def test_backward_argument_errors():
    import ctypes as C
    L = k2().lib()
    x = torch.zeros((4, 8), dtype=torch.float64, device=DEV)
    p = C.c_void_p(x.data_ptr())
    assert L.k2svd_dgesvd2_bwd(-1, p, p, p, 8, None, None, None, p, 1e-10, None) == -1
    assert L.k2svd_dgesvd2_bwd(8, None, p, p, 8, None, None, None, p, 1e-10, None) == -2
    assert L.k2svd_dgesvd2_bwd(8, p, p, p, 7, None, None, None, p, 1e-10, None) == -5
    assert L.k2svd_dgesvd2_bwd(8, p, p, p, 8, None, None, None, None, 1e-10, None) == -9
    assert L.k2svd_dgesvd2_bwd(8, p, p, p, 8, None, None, None, p, -1.0, None) == -10
