"""The two correctly rounded primitives of the 2x2 kernels, checked on the device:
the integer-pipe binary64 division against the FP64 divider (IEEE division, correctly
rounded by definition) on about 1.3e9 operand pairs, and hypot against the oracle's exact
midpoint hypot on 2.5e7 pairs, exact ties and special operands."""
import ctypes as C
import math
import os

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _lib():
    from paper_2407_13116_gb300 import k2svd
    L = k2svd.probe_lib()
    for f in ("k2probe_div", "k2probe_hypot", "k2probe_hypotf"):
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


def _hyp(L, a, b):
    h = torch.empty_like(a)
    assert L.k2probe_hypot(a.numel(), a.data_ptr(), b.data_ptr(), h.data_ptr(),
                           torch.cuda.current_stream().cuda_stream) == 0
    return h


def _check_hypot(a, b, h):
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    ref = oracle.hypot_n(an, bn, "d", nthreads=os.cpu_count() or 1)
    got = h.cpu().numpy()
    bad = got.view(np.int64) != ref.view(np.int64)
    assert not bad.any(), (an[bad][:4].tolist(), bn[bad][:4].tolist(), got[bad][:4].tolist(), ref[bad][:4].tolist())


@pytest.mark.parametrize("case", ["full", "narrow", "ratio_edge", "subnormal", "overflow", "near_one_to_two"])
def test_hypot_matches_oracle(case):
    """2^22 pairs per case, every result compared with the oracle's hypot (exact midpoint
    tests on big integers)."""
    L = _lib()
    gen = torch.Generator(device=DEV).manual_seed(7 + (hash(case) & 0xFF))
    n = 1 << 22
    if case == "full":
        a, b = _bits_double(n, gen, -1022, 1023, 0.05), _bits_double(n, gen, -1022, 1023, 0.05)
    elif case == "narrow":
        a, b = _bits_double(n, gen, -30, 30), _bits_double(n, gen, -40, 30)
    elif case == "ratio_edge":           # exponent differences around the (p+1)/2 = 27 cut
        a = _bits_double(n, gen, -100, 100)
        d = torch.randint(20, 31, (n,), generator=gen, device=DEV, dtype=torch.int64)
        b = (_bits_double(n, gen, 0, 0).view(torch.int64) + ((a.view(torch.int64) >> 52 & 0x7FF) - 1023 - d << 52)).view(torch.float64)
    elif case == "subnormal":
        a, b = _bits_double(n, gen, -1022, -1000, 0.6), _bits_double(n, gen, -1022, -1000, 0.6)
    elif case == "overflow":
        a, b = _bits_double(n, gen, 1018, 1023), _bits_double(n, gen, 1010, 1023)
    else:                                # a', b' both near 2: sums of squares near 2^113
        a = _bits_double(n, gen, 0, 0)
        a = (a.view(torch.int64) | (0xFFFFF << 32)).view(torch.float64)
        b = (a.view(torch.int64) - torch.randint(0, 1 << 30, (n,), generator=gen, device=DEV, dtype=torch.int64)).view(torch.float64)
    _check_hypot(a, b, _hyp(L, a, b))


def _bits_float(n, gen, elo, ehi, subnormal_frac=0.0):
    m = torch.randint(0, 1 << 23, (n,), generator=gen, device=DEV, dtype=torch.int32)
    e = torch.randint(elo + 127, ehi + 128, (n,), generator=gen, device=DEV, dtype=torch.int32)
    s = torch.randint(0, 2, (n,), generator=gen, device=DEV, dtype=torch.int32)
    if subnormal_frac:
        sub = torch.rand(n, generator=gen, device=DEV) < subnormal_frac
        e = torch.where(sub, torch.zeros_like(e), e)
        m = torch.where(sub, m | 1, m)
    return ((s << 31) | (e << 23) | m).view(torch.float32)


@pytest.mark.parametrize("case", ["full", "narrow", "ratio_edge", "subnormal", "overflow"])
def test_hypotf_matches_oracle(case):
    """The binary32 hypot on 2^22 pairs per case against the oracle's, bit for bit."""
    import random
    from test_oracle_hypot import _euclid_ties
    L = _lib()
    gen = torch.Generator(device=DEV).manual_seed(17 + (hash(case) & 0xFF))
    n = 1 << 22
    if case == "full":
        a, b = _bits_float(n, gen, -126, 127, 0.05), _bits_float(n, gen, -126, 127, 0.05)
    elif case == "narrow":
        a, b = _bits_float(n, gen, -20, 20), _bits_float(n, gen, -30, 20)
    elif case == "ratio_edge":
        a = _bits_float(n, gen, -40, 40)
        d = torch.randint(9, 16, (n,), generator=gen, device=DEV, dtype=torch.int32)
        b = (_bits_float(n, gen, 0, 0).view(torch.int32) + ((a.view(torch.int32) >> 23 & 0xFF) - 127 - d << 23)).view(torch.float32)
    elif case == "subnormal":
        a, b = _bits_float(n, gen, -126, -110, 0.6), _bits_float(n, gen, -126, -110, 0.6)
    else:
        a, b = _bits_float(n, gen, 120, 127), _bits_float(n, gen, 115, 127)
    xs, ys = [], []
    for (p, q, c) in _euclid_ties(24, 200, random.Random(8)):
        for sc in (0, -60, 70):
            xs.append(math.ldexp(p, sc)); ys.append(math.ldexp(q, sc))
    a = torch.cat([a, torch.tensor(xs, dtype=torch.float32, device=DEV)])
    b = torch.cat([b, torch.tensor(ys, dtype=torch.float32, device=DEV)])
    h = torch.empty_like(a)
    assert L.k2probe_hypotf(a.numel(), a.data_ptr(), b.data_ptr(), h.data_ptr(),
                            torch.cuda.current_stream().cuda_stream) == 0
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    ref = oracle.hypot_n(an, bn, "s", nthreads=os.cpu_count() or 1)
    got = h.cpu().numpy()
    bad = got.view(np.int32) != ref.view(np.int32)
    assert not bad.any(), (an[bad][:4].tolist(), bn[bad][:4].tolist(), got[bad][:4].tolist(), ref[bad][:4].tolist())


def test_hypot_exact_ties_and_specials():
    """Pythagorean triples whose hypotenuse is a midpoint between two doubles (ties to
    even), exact triples, and zero / infinite / NaN / extreme operands."""
    import random
    from test_oracle_hypot import _euclid_ties
    L = _lib()
    xs, ys = [], []
    for (p, q, c) in _euclid_ties(53, 200, random.Random(5)):
        for sc in (0, -540, 600, -1000, 960):
            xs += [math.ldexp(p, sc), math.ldexp(q, sc)]
            ys += [math.ldexp(q, sc), -math.ldexp(p, sc)]
    for k in range(-1070, 1020, 7):
        xs.append(math.ldexp(3.0, k)); ys.append(math.ldexp(4.0, k))
    sp = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1.0, 1.7976931348623157e308, float("inf"), float("-inf")]
    for u in sp:
        for v in sp:
            xs.append(u); ys.append(v)
    a = torch.tensor(xs, dtype=torch.float64, device=DEV)
    b = torch.tensor(ys, dtype=torch.float64, device=DEV)
    _check_hypot(a, b, _hyp(L, a, b))
    u = torch.tensor([float("nan"), 1.0, float("nan"), 0.0], dtype=torch.float64, device=DEV)
    v = torch.tensor([1.0, float("nan"), float("nan"), float("nan")], dtype=torch.float64, device=DEV)
    assert bool(torch.isnan(_hyp(L, u, v)).all())
