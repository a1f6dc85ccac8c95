"""Seeded synthetic inputs shaped like the random tests of Sect. 4 of arXiv 2407.13116.

This module holds input generation only (none of the SVD arithmetic).  It serves
both the CUDA path and the oracle.  Every random draw is a counter-based value,
the splitmix64 output for state ``seed + (counter + 1) * 0x9E3779B97F4A7C15``
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), so the same code gives bit-identical values with numpy on the
host and with torch integer ops on any device, and a sample of a large batch can
be regenerated by index.

Element recipes (the paper's own inputs were Fortran pseudorandom numbers and
rdrand bit patterns, which are not reproducible; these stand in for them):

* ``narrow``: each entry sign * m * 2^e, m uniform in [1,2) (52 random mantissa
  bits), e uniform in [-20, 20]; 25% of the matrices forced upper triangular
  (g21 = 0), 5% with one zero row or column (which one uniformly of four).
* ``wide``: e uniform over the normal range [-1021, 1021] (double) or
  [-125, 125] (single); each entry independently, with probability 2%, is
  replaced by a random subnormal (1%) or a near-overflow value |x| in
  [nu/4, nu] (1%).  Used for general matrices and for (F, G, H) triples.
* ``safe``: magnitudes with exponents uniform in [e_mu + c, e_nu - 2]
  (the safe range [2^c mu, nu/4] of Sect. 4, Fig. 4 uses c = varsigma).
"""
import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# draws per matrix: elements k = 0..3 use counters 16*i + 4*k + {0,1,2}; 16*i + 12.. are per-matrix draws
_PER = 16


class _Numpy:
    """uint64 arithmetic on numpy arrays (wrapping)."""

    def __init__(self):
        self.np = np

    def const(self, c):
        return np.uint64(c & MASK64)

    def arange(self, i0, i1, device=None):
        return np.arange(i0, i1, dtype=np.uint64)

    def shr(self, x, k):
        return x >> np.uint64(k)

    def shl(self, x, k):
        return x << np.uint64(k)

    def where(self, c, a, b):
        return np.where(c, a, b)

    def f64(self, bits):
        return bits.view(np.float64)

    def f32(self, bits):
        return (bits & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)

    def full_like(self, x, c):
        return np.full(x.shape, c & MASK64, dtype=np.uint64)


class _Torch:
    """The same arithmetic on torch int64 tensors (two's complement, logical shifts by masking)."""

    def __init__(self):
        import torch
        self.torch = torch

    def const(self, c):
        c &= MASK64
        return c - (1 << 64) if c >= (1 << 63) else c

    def arange(self, i0, i1, device=None):
        return self.torch.arange(i0, i1, dtype=self.torch.int64, device=device)

    def shr(self, x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)

    def shl(self, x, k):
        return x << k

    def where(self, c, a, b):
        return self.torch.where(c, a, b)

    def f64(self, bits):
        return bits.view(self.torch.float64)

    def f32(self, bits):
        b = bits & 0xFFFFFFFF
        b = b - ((b >> 31) & 1) * (1 << 32)
        return b.to(self.torch.int32).view(self.torch.float32)

    def full_like(self, x, c):
        return self.torch.full_like(x, self.const(c))


NUMPY = _Numpy()


def _backend(xp):
    if xp is None or xp == "numpy":
        return NUMPY
    return _Torch()


def splitmix(B, seed, ctr):
    """splitmix64 output number ctr+1 of the generator started at state ``seed``."""
    z = B.const(seed) + (ctr + B.const(1)) * B.const(GOLDEN)
    z = (z ^ B.shr(z, 30)) * B.const(_M1)
    z = (z ^ B.shr(z, 27)) * B.const(_M2)
    return z ^ B.shr(z, 31)


def _uniform_off(B, bits, lo, hi, off):
    """integer uniform in [lo, hi] plus off (lo + off >= 0), from the top 53 bits
    (modulo bias below 2^-40)."""
    return B.shr(bits, 11) % (hi - lo + 1) + (lo + off)


def _elem_bits(B, seed, idx, k, prec, kind):
    """Bit pattern (uint64 / int64) of element k of matrices idx, as a value of type prec."""
    c0 = idx * B.const(_PER) + B.const(4 * k)
    d_m = splitmix(B, seed, c0)            # sign and mantissa
    d_e = splitmix(B, seed, c0 + B.const(1))  # exponent
    if prec == "d":
        mbits, ebias, sbit = 52, 1023, 63
        if kind == "narrow":
            elo, ehi = -20, 20
        else:
            elo, ehi = -1021, 1021
        emax_field = 2046
    else:
        mbits, ebias, sbit = 23, 127, 31
        if kind == "narrow":
            elo, ehi = -20, 20
        else:
            elo, ehi = -125, 125
        emax_field = 254
    mant = d_m & B.const((1 << mbits) - 1)
    sign = B.shr(d_m, 63)
    efield = _uniform_off(B, d_e, elo, ehi, ebias)
    if kind == "wide":
        d_x = splitmix(B, seed, c0 + B.const(2))
        u = B.shr(d_x, 11) % 10000
        sub = u < 100                       # 1%: subnormal (exponent field 0, non-zero mantissa)
        big = (u >= 100) & (u < 200)        # 1%: |x| in [nu/4, nu]: exponent field emax-1 or emax
        efield = B.where(sub, efield * 0, efield)
        mant = B.where(sub, mant | 1, mant)
        efield = B.where(big, B.shr(d_x, 5) % 2 + (emax_field - 1), efield)
    return B.shl(sign, sbit) | B.shl(efield, mbits) | mant


def _as_real(B, bits, prec):
    return B.f64(bits) if prec == "d" else B.f32(bits)


def _indices(B, n, i0, idx, device):
    if idx is None:
        return B.arange(i0, i0 + n, device=device)
    if B is NUMPY:
        return np.asarray(idx, dtype=np.uint64)
    return B.torch.as_tensor(np.asarray(idx, dtype=np.int64), device=device)


def general(n, seed, prec="d", kind="wide", i0=0, xp=None, device=None, idx=None):
    """Planes G[4, n] (g11, g21, g12, g22) of matrices i0 .. i0+n-1 (or of the matrices with
    the given indices).  kind = "narrow" also applies the 25% triangular and 5% zero
    row/column patterns."""
    B = _backend(xp)
    idx = _indices(B, n, i0, idx, device)
    planes = [_as_real(B, _elem_bits(B, seed, idx, k, prec, kind), prec) for k in range(4)]
    if kind == "narrow":
        d = splitmix(B, seed, idx * B.const(_PER) + B.const(12))
        u = B.shr(d, 11) % 100
        which = B.shr(d, 5) % 4              # zero: 0 row 1, 1 row 2, 2 column 1, 3 column 2
        tri = u < 25
        zrc = (u >= 25) & (u < 30)
        zero = planes[0] - planes[0]      # +0 (the inputs are finite)
        g11, g21, g12, g22 = planes
        g21 = B.where(tri, zero, g21)
        g11 = B.where(zrc & ((which == 0) | (which == 2)), zero, g11)
        g12 = B.where(zrc & ((which == 0) | (which == 3)), zero, g12)
        g21 = B.where(zrc & ((which == 1) | (which == 2)), zero, g21)
        g22 = B.where(zrc & ((which == 1) | (which == 3)), zero, g22)
        planes = [g11, g21, g12, g22]
    if B is NUMPY:
        return np.stack(planes)
    return B.torch.stack(planes)


def triangular(n, seed, prec="d", kind="wide", i0=0, xp=None, device=None, idx=None):
    """(F, G, H) planes [3, n] of upper-triangular matrices [[F, G], [0, H]]."""
    B = _backend(xp)
    idx = _indices(B, n, i0, idx, device)
    planes = [_as_real(B, _elem_bits(B, seed, idx, k, prec, kind), prec) for k in (0, 2, 3)]
    if B is NUMPY:
        return np.stack(planes)
    return B.torch.stack(planes)


def safe_range(n, seed, c, prec="d", triangular_=False):
    """Planes with |g| exponents uniform in [e_mu + c, e_nu - 2] (the safe range [2^c mu, nu/4])."""
    B = NUMPY
    idx = B.arange(0, n)
    out = []
    emu, enu, mbits, ebias, sbit = (-1022, 1023, 52, 1023, 63) if prec == "d" else (-126, 127, 23, 127, 31)
    for k in range(4):
        c0 = idx * B.const(_PER) + B.const(4 * k)
        d_m = splitmix(B, seed, c0)
        d_e = splitmix(B, seed, c0 + B.const(1))
        efield = _uniform_off(B, d_e, emu + c, enu - 2, ebias)
        bits = B.shl(B.shr(d_m, 63), sbit) | B.shl(efield, mbits) | (d_m & B.const((1 << mbits) - 1))
        out.append(_as_real(B, bits, prec))
    G = np.stack(out)
    if triangular_:
        G[1] = 0
    return G


def uniform01(n, seed, stream, i0=0):
    """float64 uniform in [0,1) with 53 random bits, from counter stream ``stream``."""
    B = NUMPY
    idx = B.arange(i0, i0 + n)
    d = splitmix(B, seed, idx * B.const(_PER) + B.const(12 + stream))
    return B.shr(d, 11).astype(np.float64) * 2.0 ** -53


def normal(shape, seed, stream):
    """N(0,1) by the Box-Muller transform of two counter-based uniforms."""
    n = int(np.prod(shape))
    u1 = uniform01(n, seed, stream)
    u2 = uniform01(n, seed + 1, stream)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return (r * np.cos(2.0 * math.pi * u2)).reshape(shape)


def rotated(n, seed, ecount=30, close_frac=0.10):
    """Differentiation workload: G = R(theta) diag(s1, s2) R(phi)^T with theta, phi uniform in
    [0, 2 pi), s1 = 2^e (e uniform in [-ecount, ecount]), s2/s1 log-uniform in [1e-12, 1], and a
    fraction close_frac of the matrices with s2/s1 in (1 - 1e-6, 1].  Returns planes G[4, n] and
    the exact (s1, s2) used."""
    th = 2.0 * math.pi * uniform01(n, seed, 0)
    ph = 2.0 * math.pi * uniform01(n, seed, 1)
    e = np.floor(uniform01(n, seed, 2) * (2 * ecount + 1)) - ecount
    s1 = np.ldexp(1.0, e.astype(np.int64))
    u = uniform01(n, seed, 3)
    ratio = 10.0 ** (-12.0 * u)
    close = uniform01(n, seed + 7, 0) < close_frac
    ratio = np.where(close, 1.0 - 1e-6 * u, ratio)
    s2 = s1 * ratio
    ct, st, cp, sp = np.cos(th), np.sin(th), np.cos(ph), np.sin(ph)
    # G = R(th) diag(s1,s2) R(ph)^T, R(x) = [[cos x, -sin x], [sin x, cos x]]
    g11 = ct * s1 * cp + st * s2 * sp
    g21 = st * s1 * cp - ct * s2 * sp
    g12 = ct * s1 * sp - st * s2 * cp
    g22 = st * s1 * sp + ct * s2 * cp
    return np.stack([g11, g21, g12, g22]), s1, s2


def kog_orders(count, nlo, nhi, seed):
    """Matrix orders uniform in {nlo, ..., nhi}."""
    u = uniform01(count, seed, 4)
    return (nlo + np.floor(u * (nhi - nlo + 1))).astype(np.int32)


def kog_matrix(n, seed, index, smin=1e-12, dtype=np.float64):
    """A = Q1 diag(sigma) Q2^T, Q1 and Q2 products of n Householder reflectors built from N(0,1)
    vectors, sigma log-uniform in [smin, 1].  Column-major n x n array (Fortran order)."""
    rng_seed = (seed * 1000003 + index) & MASK64
    z = normal((2, n, n), rng_seed, 5)
    qs = []
    for t in range(2):
        Q = np.eye(n)
        for k in range(n):
            v = z[t, k]
            nv = v @ v
            if nv == 0:
                continue
            Q = Q - np.outer(Q @ v, (2.0 / nv) * v)
        qs.append(Q)
    lu = uniform01(n, rng_seed, 6)
    sigma = smin ** lu
    A = (qs[0] * sigma) @ qs[1].T
    return np.asfortranarray(A.astype(dtype)), np.sort(sigma)[::-1]


def kog_batch(orders, seed, smin=1e-12, dtype=np.float64):
    """Packed batch (flat, column-major per matrix) of Q1 diag(sigma) Q2^T for the given
    orders, grouped by order: Q1, Q2 are the orthogonal factors of the Householder QR
    (LAPACK) of N(0,1) matrices, i.e. products of n Householder reflectors built from
    N(0,1) data; sigma log-uniform in [smin, 1].  Returns (flat, list of sigma arrays)."""
    orders = np.asarray(orders, dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(orders ** 2)[:-1]]).astype(np.int64)
    flat = np.empty(int((orders ** 2).sum()), dtype=dtype)
    sigmas = [None] * len(orders)
    for n in np.unique(orders):
        idx = np.flatnonzero(orders == n)
        b, n = len(idx), int(n)
        z = normal((2, b, n, n), (seed * 7919 + n) & MASK64, 7)
        q1 = np.linalg.qr(z[0])[0]
        q2 = np.linalg.qr(z[1])[0]
        u = uniform01(b * n, (seed * 7919 + n) & MASK64, 8).reshape(b, n)
        sig = smin ** u
        A = np.matmul(q1 * sig[:, None, :], np.swapaxes(q2, 1, 2))
        At = np.ascontiguousarray(np.swapaxes(A, 1, 2)).reshape(b, n * n)   # column-major rows
        for q, i in enumerate(idx):
            flat[offs[i]:offs[i] + n * n] = At[q]
            sigmas[i] = np.sort(sig[q])[::-1]
    return flat.astype(dtype, copy=False), sigmas
