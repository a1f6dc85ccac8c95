"""GPU parity of the variant with a hypot that is not correctly rounded
(k2svd_{d,s}gesvd2_ncr, k2svd_{d,s}trsvd2_ncr; Alg. 1's branch for that case) and of its
hypot (k2probe_hypot_ncr, k2probe_hypotf_ncr) against the oracle, bit for bit: every step
is an IEEE operation with one rounding."""
import ctypes as C
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2407_13116_gb300 import inputs as I
from test_gpu_primitives import _bits_double, _bits_float
from test_gpu_svd2 import _assert_same, _special_cases, _u

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def k2():
    from paper_2407_13116_gb300 import k2svd
    return k2svd


def _lib():
    L = k2().probe_lib()
    for f in ("k2probe_hypot_ncr", "k2probe_hypotf_ncr"):
        getattr(L, f).argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        getattr(L, f).restype = C.c_int
    return L


def _hyp(a, b):
    h = torch.empty_like(a)
    f = _lib().k2probe_hypot_ncr if a.dtype == torch.float64 else _lib().k2probe_hypotf_ncr
    assert f(a.numel(), a.data_ptr(), b.data_ptr(), h.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    return h


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("case", ["full", "narrow", "subnormal", "overflow"])
def test_hypot_ncr_matches_oracle(prec, case):
    gen = torch.Generator(device=DEV).manual_seed(31 + (hash(case) & 0xFF) + (prec == "s"))
    n = 1 << 21
    rng = {"d": {"full": (-1022, 1023), "narrow": (-30, 30), "subnormal": (-1022, -1000), "overflow": (1010, 1023)},
           "s": {"full": (-126, 127), "narrow": (-20, 20), "subnormal": (-126, -110), "overflow": (115, 127)}}[prec][case]
    sub = 0.6 if case == "subnormal" else (0.05 if case == "full" else 0.0)
    bits = _bits_double if prec == "d" else _bits_float
    a, b = bits(n, gen, rng[0], rng[1], sub), bits(n, gen, rng[0], rng[1], sub)
    T = np.float64 if prec == "d" else np.float32
    sp = np.array([0.0, -0.0, 1.0, 3.0, 4.0, np.finfo(T).max, np.finfo(T).tiny, np.finfo(T).smallest_subnormal,
                   np.inf, -np.inf], dtype=T)
    a = torch.cat([a, torch.from_numpy(np.repeat(sp, len(sp))).to(DEV)])
    b = torch.cat([b, torch.from_numpy(np.tile(sp, len(sp))).to(DEV)])
    got = _hyp(a, b).cpu().numpy()
    ref = oracle.hypot_ncr_n(a.cpu().numpy(), b.cpu().numpy(), prec, nthreads=os.cpu_count() or 1)
    bad = _u(got) != _u(ref)
    assert not bad.any(), (a.cpu().numpy()[bad][:4].tolist(), b.cpu().numpy()[bad][:4].tolist(),
                           got[bad][:4].tolist(), ref[bad][:4].tolist())
    nan = torch.tensor([np.nan, 1.0, np.nan], dtype=a.dtype, device=DEV)
    one = torch.tensor([1.0, np.nan, np.nan], dtype=a.dtype, device=DEV)
    assert bool(torch.isnan(_hyp(nan, one)).all())


def _gpu(G=None, T3=None):
    if G is not None:
        out = k2().gesvd2_ncr(torch.from_numpy(np.ascontiguousarray(G)).to(DEV), want_ef=True)
    else:
        F, Gu, H = (torch.from_numpy(np.ascontiguousarray(T3[k])).to(DEV) for k in range(3))
        out = k2().trsvd2_ncr(F, Gu, H, want_ef=True)
    torch.cuda.synchronize()
    return {nm: t.cpu().numpy() for nm, t in zip(("U", "V", "S", "Se", "Sf", "info"), out)}


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("kind", ["narrow", "wide"])
def test_parity_general(prec, kind):
    n = (1 << 17) + 77
    G = I.general(n, 5100 + len(kind), prec, kind)
    ref = oracle.gesvd2(G, prec, nthreads=8, ncr=True)
    _assert_same(_gpu(G=G), ref, "gesvd2_ncr %s %s" % (prec, kind))
    assert (np.bitwise_or.reduce(ref["info"][ref["info"] >= 0]) >> 8) & oracle.FLAGS["t2ncr"]


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("kind", ["narrow", "wide"])
def test_parity_triangular(prec, kind):
    n = (1 << 16) + 13
    T3 = I.triangular(n, 5200 + len(kind), prec, kind)
    _assert_same(_gpu(T3=T3), oracle.trsvd2(T3[0], T3[1], T3[2], prec, nthreads=8, ncr=True),
                 "trsvd2_ncr %s %s" % (prec, kind))


@pytest.mark.parametrize("prec", ["d", "s"])
def test_parity_special_values_safe_ranges_and_nonfinite(prec):
    T = np.float64 if prec == "d" else np.float32
    parts = [_special_cases(prec), I.safe_range(20000, 5300, 0, prec),
             I.safe_range(20000, 5301, 0, prec, triangular_=True),
             np.array([[1, np.nan, 2, 3], [np.inf, 1, 1, 1], [0, 0, -np.inf, 0]], dtype=T).T]
    G = np.ascontiguousarray(np.concatenate(parts, axis=1))
    _assert_same(_gpu(G=G), oracle.gesvd2(G, prec, nthreads=8, ncr=True), "special ncr %s" % prec)


@pytest.mark.parametrize("n", [1, 31, 33, 129])
def test_small_and_ragged_batches(n):
    G = I.general(n, 5400 + n, "d", "wide")
    _assert_same(_gpu(G=G), oracle.gesvd2(G, "d", ncr=True), "ncr n=%d" % n)


def test_argument_errors_and_empty_batch():
    L = k2().lib()
    x = torch.zeros(4, 8, dtype=torch.float64, device=DEV)
    assert L.k2svd_dgesvd2_ncr(-1, x.data_ptr(), 8, x.data_ptr(), 8, x.data_ptr(), 8, x.data_ptr(), 8,
                               None, None, None, None) == -1
    assert L.k2svd_dgesvd2_ncr(8, None, 8, x.data_ptr(), 8, x.data_ptr(), 8, x.data_ptr(), 8,
                               None, None, None, None) == -2
    assert L.k2svd_dtrsvd2_ncr(8, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, x.data_ptr(), 8,
                               x.data_ptr(), 8, None, None, None, None) == -6
    assert L.k2svd_sgesvd2_ncr(0, None, 0, None, 0, None, 0, None, 0, None, None, None, None) == 0


@pytest.mark.parametrize("prec", ["d", "s"])
def test_full_size_sampled_parity(prec):
    """The benchmark's variant leg: 2^27 (double) or 2^28 (float) wide-range general matrices
    generated on the device, checked on a sample against the oracle by index."""
    n = (1 << 27) if prec == "d" else (1 << 28)
    seed = 0x240713116 + 2
    G = I.general(n, seed, prec, "wide", xp="torch", device=DEV)
    out = k2().gesvd2_ncr(G, want_ef=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([rng.integers(0, n, 6000), np.arange(64), np.arange(n - 64, n)]))
    it = torch.from_numpy(idx).to(DEV)
    got = {nm: (t[..., it] if t.dim() == 2 else t[it]).cpu().numpy()
           for nm, t in zip(("U", "V", "S", "Se", "Sf", "info"), out)}
    host = I.general(0, seed, prec, "wide", idx=idx)
    _assert_same(got, oracle.gesvd2(host, prec, nthreads=8, ncr=True), "full-size ncr %s" % prec)
    del G, out
    torch.cuda.empty_cache()
