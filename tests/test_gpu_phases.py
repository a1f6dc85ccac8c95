"""GPU parity of the standalone phase 1 (k2svd_?prescale2) and of the xLASV2 argument shape
(k2svd_?lasv2) against the oracle, bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_13116_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def k2():
    from paper_2407_13116_gb300 import k2svd
    return k2svd


def _bits(x):
    x = np.ascontiguousarray(x)
    return x.view({8: np.uint64, 4: np.uint32}[x.dtype.itemsize])


def _with_zeros(G, seed, frac=0.2):
    rng = np.random.default_rng(seed)
    return np.where(rng.random(G.shape) < frac, G.dtype.type(0), G)


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("extra", [0, 1, 5])
@pytest.mark.parametrize("n", [1, 33, (1 << 18) + 7])
def test_prescale_parity(prec, extra, n):
    G = np.concatenate([I.general(n, 61, prec, "wide"), I.general(n, 62, prec, "narrow")], axis=1)
    G = _with_zeros(G, 63)
    Gs, s, types = k2().prescale2(torch.from_numpy(np.ascontiguousarray(G)).to(DEV), extra=extra)
    rG, rs, rt = oracle.prescale2(G, prec, extra, nthreads=8)
    assert np.array_equal(_bits(Gs.cpu().numpy()), _bits(rG))
    assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(types.cpu().numpy(), rt)


def test_prescale_in_place_and_nonfinite():
    G = np.concatenate([I.general(1000, 64, "d", "wide"), np.array([[np.inf], [1.0], [np.nan], [0.0]])], axis=1)
    t = torch.from_numpy(np.ascontiguousarray(G)).to(DEV)
    Gs, s, types = k2().prescale2(t, extra=1, Gs=t)
    rG, rs, rt = oracle.prescale2(G, "d", 1)
    out = t.cpu().numpy()
    fin = np.isfinite(rG)
    assert np.array_equal(_bits(out[fin]), _bits(rG[fin])) and np.array_equal(np.isnan(out), np.isnan(rG))
    assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(types.cpu().numpy(), rt)
    assert types[-1].item() == -1


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("kind", ["narrow", "wide"])
@pytest.mark.parametrize("n", [1, 129, (1 << 18) + 3])
def test_lasv2_parity(prec, kind, n):
    Th = I.triangular(n, 65, prec, kind)
    Th = _with_zeros(Th, 66, 0.1)
    T = [torch.from_numpy(np.ascontiguousarray(Th[k])).to(DEV) for k in range(3)]
    got = [x.cpu().numpy() for x in k2().lasv2(*T)]
    ref = oracle.lasv2(Th[0], Th[1], Th[2], prec, nthreads=8)
    for g, r in zip(got, ref):
        assert np.array_equal(_bits(g), _bits(r))
    # the same numbers as the triangular entry
    U, V, S, _, _, _ = k2().trsvd2(*T, want_info=False)
    S, U, V = S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()
    assert np.array_equal(_bits(got[1]), _bits(S[0])) and np.array_equal(_bits(np.abs(got[0])), _bits(S[1]))
    assert np.array_equal(_bits(got[5]), _bits(U[0])) and np.array_equal(_bits(got[3]), _bits(V[0]))


def test_lasv2_nonfinite_and_errors():
    F = torch.tensor([1.0, float("nan"), 2.0], dtype=torch.float64, device=DEV)
    G = torch.tensor([0.5, 1.0, float("inf")], dtype=torch.float64, device=DEV)
    H = torch.tensor([3.0, 1.0, 1.0], dtype=torch.float64, device=DEV)
    out = k2().lasv2(F, G, H)
    for o in out:
        assert not torch.isnan(o[0]) and bool(torch.isnan(o[1:]).all())
    L = k2().lib()
    p = F.data_ptr()
    assert L.k2svd_dlasv2(-1, p, p, p, p, p, p, p, p, p, None) == -1
    assert L.k2svd_dlasv2(3, p, None, p, p, p, p, p, p, p, None) == -3
    assert L.k2svd_dlasv2(3, p, p, p, p, p, p, p, p, None, None) == -10
    assert L.k2svd_dprescale2(3, p, 2, p, 3, p, None, 0, None) == -3
    assert L.k2svd_dprescale2(3, p, 3, p, 3, p, None, 65, None) == -8
    assert L.k2svd_dprescale2(0, None, 0, None, 0, None, None, 0, None) == 0


@pytest.mark.parametrize("prec", ["d", "s"])
def test_full_size_sampled(prec):
    """At the benchmark's size (2^27 double / 2^28 float matrices of the wide workload,
    generated on the device), sampled outputs of both entries against the oracle."""
    n = 1 << (27 if prec == "d" else 28)
    G = I.general(n, 0x240713116 + 2, prec, "wide", xp="torch", device=DEV)
    Gs, s, types = k2().prescale2(G, extra=1)
    idx = np.unique(np.concatenate([np.arange(64), n - 1 - np.arange(64), np.random.default_rng(7).integers(0, n, 4000)]))
    it = torch.from_numpy(idx).to(DEV)
    Gh = I.general(len(idx), 0x240713116 + 2, prec, "wide", idx=idx)
    rG, rs, rt = oracle.prescale2(Gh, prec, 1)
    assert np.array_equal(_bits(Gs[:, it].cpu().numpy()), _bits(rG))
    assert np.array_equal(s[it].cpu().numpy(), rs)
    del G, Gs
    T3 = I.triangular(n, 0x240713116 + 3, prec, "wide", xp="torch", device=DEV)
    out = k2().lasv2(T3[0], T3[1], T3[2])
    Th = I.triangular(len(idx), 0x240713116 + 3, prec, "wide", idx=idx)
    ref = oracle.lasv2(Th[0], Th[1], Th[2], prec)
    for g, r in zip(out, ref):
        assert np.array_equal(_bits(g[it].cpu().numpy()), _bits(r))
