"""torch.autograd.Function for the batched 2x2 SVD: forward by k2svd_?gesvd2, backward by
k2svd_?gesvd2_bwd (the adjoint with a gap threshold for near-equal singular values).

    U, S, V = svd2x2(A)          # A: (..., 2, 2) float64/float32 CUDA tensor
    A ~ U @ diag_embed(S) @ V.mT, S[..., 0] >= S[..., 1] >= 0

Only argument marshalling happens here: the (..., 2, 2) tensors are repacked into the SoA
planes of the C ABI and back.
"""
import torch

from . import k2svd


class SVD2x2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, gap_rtol):
        if A.shape[-2:] != (2, 2):
            raise k2svd.K2SVDError("svd2x2 expects (..., 2, 2) matrices, got %s" % (tuple(A.shape),))
        shape = A.shape[:-2]
        G = k2svd.to_planes(A)
        U, V, S, _, _, _ = k2svd.gesvd2(G, want_info=False)
        ctx.save_for_backward(U, S, V)
        ctx.shape = shape
        ctx.gap_rtol = gap_rtol
        ctx.set_materialize_grads(False)
        return (k2svd.from_planes(U, shape), S.t().reshape(*shape, 2), k2svd.from_planes(V, shape))

    @staticmethod
    def backward(ctx, gU, gS, gV):
        U, S, V = ctx.saved_tensors
        dU = None if gU is None else k2svd.to_planes(gU.to(U.dtype))
        dV = None if gV is None else k2svd.to_planes(gV.to(U.dtype))
        dS = None if gS is None else gS.to(U.dtype).reshape(-1, 2).t().contiguous()
        dG = k2svd.gesvd2_bwd(U, S, V, dS, dU, dV, ctx.gap_rtol)
        return k2svd.from_planes(dG, ctx.shape), None


def svd2x2(A, gap_rtol=1e-10):
    """SVD of a batch of real 2x2 matrices with autograd support: returns (U, S, V)."""
    return SVD2x2.apply(A, gap_rtol)


class KogbetSigma(torch.autograd.Function):
    """Batched n x n SVD by the persistent Kogbetliantz driver with the gradient of the
    singular values: dA_i = U_i diag(dS_i) V_i^T (k2svd_?kog_sigma_bwd).  Inputs and outputs
    are packed (flat, column-major per matrix)."""

    @staticmethod
    def forward(ctx, A, orders, max_sweeps, flags):
        U, S, V, sweeps, info = k2svd.kogbet(A, orders, max_sweeps=max_sweeps, flags=flags)
        ctx.save_for_backward(U, V)
        ctx.orders = list(orders)
        ctx.mark_non_differentiable(U, V, sweeps, info)
        ctx.set_materialize_grads(False)
        return U, S, V, sweeps, info

    @staticmethod
    def backward(ctx, gU, gS, gV, gsw, ginfo):
        if gU is not None or gV is not None:
            raise k2svd.K2SVDError("kogbet_sigma differentiates the singular values only")
        if gS is None:
            return None, None, None, None
        U, V = ctx.saved_tensors
        dA = k2svd.kog_sigma_bwd(U, V, gS.contiguous(), ctx.orders)
        return dA, None, None, None


def kogbet_sigma(A, orders, max_sweeps=40, flags=0):
    """(U, S, V, sweeps, info) of a packed batch, differentiable in S."""
    return KogbetSigma.apply(A, list(orders), max_sweeps, flags)
