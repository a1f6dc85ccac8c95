"""GPU parity of the complex 2x2 SVD (k2svd_zgesvd2 / k2svd_cgesvd2, Sect. 3.4) against the
oracle, bit for bit: every zero pattern, real and purely imaginary input, non-finite input,
ragged sizes, and sampled outputs at the benchmark's size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_13116_gb300 import inputs as I
from test_oracle_complex import _planes, _random

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def k2():
    from paper_2407_13116_gb300 import k2svd
    return k2svd


def _bits(x):
    x = np.ascontiguousarray(x)
    return x.view({8: np.uint64, 4: np.uint32}[x.dtype.itemsize])


def _same(G, prec):
    U, V, S, info = k2().cgesvd2(torch.from_numpy(np.ascontiguousarray(G)).to(DEV))
    rU, rV, rS, rinfo = oracle.cgesvd2(G, prec, nthreads=8)
    got = (U.cpu().numpy(), V.cpu().numpy(), S.cpu().numpy())
    for g, r, nm in zip(got, (rU, rV, rS), "UVS"):
        nan = np.isnan(g) & np.isnan(r)
        bad = (_bits(g) != _bits(r)) & ~nan
        assert not bad.any(), (nm, np.argwhere(bad)[:4].tolist())
    assert np.array_equal(info.cpu().numpy(), rinfo)


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("pattern", [None, 15, 7, 11, 13, 14, 3, 12, 5, 10, 9, 6, 1, 8])
def test_parity_patterns(prec, pattern):
    T = np.float64 if prec == "d" else np.float32
    rng = np.random.default_rng(31 + (pattern or 0))
    er = 300 if prec == "d" else 40
    mats = _random(4000, rng, -er, er, T, pattern) + _random(1001, rng, -8, 8, T, pattern)
    _same(_planes(mats, T), prec)


@pytest.mark.parametrize("prec", ["d", "s"])
def test_parity_real_imaginary_nonfinite_ragged(prec):
    T = np.float64 if prec == "d" else np.float32
    Gr = I.general(3001, 33, prec, "wide")
    n = Gr.shape[1]
    G = np.zeros((8, 3 * n + 3), T)
    G[0::2, :n] = Gr                       # real
    G[1::2, n:2 * n] = Gr                  # purely imaginary
    G[:, 2 * n:3 * n] = np.concatenate([Gr, I.general(n, 34, prec, "wide")])[[0, 4, 1, 5, 2, 6, 3, 7]]
    G[:, -3] = 1.0
    G[5, -3] = np.inf
    G[:, -2] = 0.0                          # zero matrix
    G[2, -1] = np.nan
    for m in (1, 33, G.shape[1]):
        _same(G[:, :m], prec)


@pytest.mark.parametrize("prec", ["d", "s"])
def test_full_size_sampled(prec):
    n = 1 << (26 if prec == "d" else 27)
    G = torch.empty((8, n), dtype=torch.float64 if prec == "d" else torch.float32, device=DEV)
    G[0::2] = I.general(n, 0x240713116 + 6, prec, "wide", xp="torch", device=DEV)
    G[1::2] = I.general(n, 0x240713116 + 7, prec, "wide", xp="torch", device=DEV)
    U, V, S, info = k2().cgesvd2(G)
    idx = np.unique(np.concatenate([np.arange(32), n - 1 - np.arange(32), np.random.default_rng(9).integers(0, n, 3000)]))
    it = torch.from_numpy(idx).to(DEV)
    Gh = np.empty((8, len(idx)), np.float64 if prec == "d" else np.float32)
    Gh[0::2] = I.general(len(idx), 0x240713116 + 6, prec, "wide", idx=idx)
    Gh[1::2] = I.general(len(idx), 0x240713116 + 7, prec, "wide", idx=idx)
    rU, rV, rS, rinfo = oracle.cgesvd2(Gh, prec, nthreads=8)
    assert np.array_equal(_bits(U[:, it].cpu().numpy()), _bits(rU))
    assert np.array_equal(_bits(V[:, it].cpu().numpy()), _bits(rV))
    assert np.array_equal(_bits(S[:, it].cpu().numpy()), _bits(rS))


def test_torch_helpers_roundtrip():
    A = torch.randn(5, 2, 2, dtype=torch.complex128, device=DEV)
    X = k2().complex_to_planes(A)
    assert torch.equal(k2().planes_to_complex(X), A)
    U, V, S, _ = k2().cgesvd2(X)
    Uc, Vc = k2().planes_to_complex(U), k2().planes_to_complex(V)
    R = Uc @ torch.diag_embed(S.T.to(torch.complex128)) @ Vc.conj().transpose(-1, -2)
    assert torch.allclose(R, A, atol=1e-14 * A.abs().max().item())


def test_large_batch_all_patterns_strided():
    """One batch of more than 65536 double matrices: every zero pattern, real, purely
    imaginary and non-finite input, on strided planes, checked against the oracle bit for
    bit, and nothing written past the batch."""
    T = np.float64
    rng = np.random.default_rng(77)
    parts = []
    for pattern in (None, 15, 7, 11, 13, 14, 3, 12, 5, 10, 9, 6, 1, 8):
        parts.append(_planes(_random(4000, rng, -300, 300, T, pattern) + _random(1001, rng, -8, 8, T, pattern), T))
    Gr = I.general(3001, 35, "d", "wide")
    n = Gr.shape[1]
    G = np.zeros((8, 2 * n + 3), T)
    G[0::2, :n] = Gr
    G[1::2, n:2 * n] = Gr
    G[:, -3] = 1.0
    G[5, -3] = np.inf
    G[2, -1] = np.nan
    parts.append(G)
    G = np.ascontiguousarray(np.concatenate(parts, axis=1))
    m = G.shape[1]
    assert m >= (1 << 16)
    ld = m + 5
    Gt = torch.zeros((8, ld), dtype=torch.float64, device=DEV)
    Gt[:, :m] = torch.from_numpy(G).to(DEV)
    U = torch.full((8, ld), 7.0, dtype=torch.float64, device=DEV)
    V = torch.full((8, ld), 7.0, dtype=torch.float64, device=DEV)
    S = torch.full((2, ld), 7.0, dtype=torch.float64, device=DEV)
    info = torch.full((ld,), 7, dtype=torch.int32, device=DEV)
    import ctypes as C
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = k2().lib().k2svd_zgesvd2(m, p(Gt), ld, p(U), ld, p(V), ld, p(S), ld, p(info),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    rU, rV, rS, rinfo = oracle.cgesvd2(G, "d", nthreads=8)
    for g, r, nm in ((U[:, :m], rU, "U"), (V[:, :m], rV, "V"), (S[:, :m], rS, "S")):
        g = g.cpu().numpy()
        nan = np.isnan(g) & np.isnan(r)
        bad = (_bits(g) != _bits(r)) & ~nan
        assert not bad.any(), (nm, np.argwhere(bad)[:4].tolist())
    assert np.array_equal(info[:m].cpu().numpy(), rinfo)
    assert (U[:, m:] == 7.0).all() and (V[:, m:] == 7.0).all() and (S[:, m:] == 7.0).all() and (info[m:] == 7).all()
