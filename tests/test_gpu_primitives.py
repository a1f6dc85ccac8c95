"""The two correctly rounded primitives of the 2x2 kernels, checked on the device:
the integer-pipe binary64 division against the FP64 divider (IEEE division, correctly
rounded by definition) on about 1.3e9 operand pairs, and hypot against the oracle's exact
midpoint hypot on a sample."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _lib():
    from paper_2407_13116_gb300 import k2svd
    L = k2svd.lib()
    for f in ("k2probe_div", "k2probe_hypot"):
        getattr(L, f).argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        getattr(L, f).restype = C.c_int
    return L


def _bits_double(n, gen, elo, ehi, subnormal_frac=0.0):
    """Random finite doubles with exponents uniform in [elo, ehi] and random signs/mantissas."""
    m = torch.randint(0, 1 << 52, (n,), generator=gen, device=DEV, dtype=torch.int64)
    e = torch.randint(elo + 1023, ehi + 1024, (n,), generator=gen, device=DEV, dtype=torch.int64)
    s = torch.randint(0, 2, (n,), generator=gen, device=DEV, dtype=torch.int64)
    if subnormal_frac:
        sub = torch.rand(n, generator=gen, device=DEV) < subnormal_frac
        e = torch.where(sub, torch.zeros_like(e), e)
        m = torch.where(sub, m | 1, m)
    bits = (s << 63) | (e << 52) | m
    return bits.view(torch.float64)


def _div(L, a, b):
    q = torch.empty_like(a)
    assert L.k2probe_div(a.numel(), a.data_ptr(), b.data_ptr(), q.data_ptr(),
                         torch.cuda.current_stream().cuda_stream) == 0
    return q


@pytest.mark.parametrize("case", ["full", "narrow", "subnormal_results", "subnormal_operands", "overflow", "near_equal", "ties"])
def test_division_matches_fp64_divider(case):
    L = _lib()
    gen = torch.Generator(device=DEV).manual_seed(hash(case) & 0xFFFF)
    n = 1 << 26
    for rep in range(3):
        if case == "full":
            a, b = _bits_double(n, gen, -1022, 1023, 0.02), _bits_double(n, gen, -1022, 1023, 0.02)
        elif case == "narrow":
            a, b = _bits_double(n, gen, -30, 30), _bits_double(n, gen, -30, 30)
        elif case == "subnormal_results":
            a, b = _bits_double(n, gen, -1022, -990), _bits_double(n, gen, 0, 70)
        elif case == "subnormal_operands":
            a, b = _bits_double(n, gen, -1022, 1023, 0.5), _bits_double(n, gen, -1022, 1023, 0.5)
        elif case == "overflow":
            a, b = _bits_double(n, gen, 990, 1023), _bits_double(n, gen, -70, 0)
        elif case == "near_equal":
            a = _bits_double(n, gen, 0, 0)
            d = torch.randint(-3, 4, (n,), generator=gen, device=DEV, dtype=torch.int64)
            b = (a.view(torch.int64) + d).view(torch.float64)
        else:   # exact ties at the subnormal quantum: odd multiples of 2^-1074 over powers of two
            k = torch.randint(1, 1 << 20, (n,), generator=gen, device=DEV, dtype=torch.int64) * 2 + 1
            a = k.view(torch.float64)
            p = torch.randint(1, 8, (n,), generator=gen, device=DEV, dtype=torch.int64)
            b = ((p + 1023) << 52).view(torch.float64)
        got = _div(L, a, b)
        ref = a / b
        bad = got.view(torch.int64) != ref.view(torch.int64)
        assert not bool(bad.any()), (case, a[bad][:4].tolist(), b[bad][:4].tolist(), got[bad][:4].tolist())


def test_division_special_operands():
    L = _lib()
    v = torch.tensor([0.0, -0.0, 1.0, -3.5, float("inf"), float("-inf"), 5e-324, 1.7976931348623157e308],
                     dtype=torch.float64, device=DEV)
    a = v.repeat_interleave(len(v))
    b = v.repeat(len(v))
    got, ref = _div(L, a, b), a / b
    same = (got.view(torch.int64) == ref.view(torch.int64)) | (torch.isnan(got) & torch.isnan(ref))
    assert bool(same.all())


def test_hypot_matches_oracle_sample():
    L = _lib()
    gen = torch.Generator(device=DEV).manual_seed(7)
    n = 1 << 16
    a = torch.cat([_bits_double(n, gen, -1022, 1023, 0.05), _bits_double(n, gen, -30, 30)])
    b = torch.cat([_bits_double(n, gen, -1022, 1023, 0.05), _bits_double(n, gen, -40, 30)])
    h = torch.empty_like(a)
    assert L.k2probe_hypot(a.numel(), a.data_ptr(), b.data_ptr(), h.data_ptr(),
                           torch.cuda.current_stream().cuda_stream) == 0
    an, bn, hn = a.cpu().numpy(), b.cpu().numpy(), h.cpu().numpy()
    for i in range(0, len(an), 7):
        assert hn[i] == oracle.hypot(float(an[i]), float(bn[i])), (an[i], bn[i])
