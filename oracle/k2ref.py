"""numpy front end of the oracle library (TEST INFRASTRUCTURE ONLY).

The C sources next to this file are compiled with gcc into ``_build/libk2ref.so``
on first use (or by ``build()``), with -ffp-contract=off so that the only fused
operations are the explicit ``fma`` calls of the paper's formulas.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libk2ref.so")
_SRC = [os.path.join(_HERE, f) for f in ("k2ref.c", "k2ref_body.inc", "k2ref_kog.c", "k2ref_bwd.c", "k2ref_rect.c")]
_lock = threading.Lock()
_lib = None

# Branch flags of info bits 8..15 (see k2ref.c)
FLAGS = {"ext": 0x01, "fallback": 0x02, "swap": 0x04, "t2f2": 0x08, "t2f3": 0x10,
         "t2inf": 0x20, "tpinf": 0x40, "psig": 0x80, "t2ncr": 0x400}


def _sources():
    return [s for s in _SRC if os.path.exists(s)]


def build(force=False):
    """Compile the oracle library (gcc, -O2, no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = _sources()
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    cfiles = [s for s in srcs if s.endswith(".c")]
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = base + ["-fopenmp"] + cfiles + ["-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # retry without OpenMP (the oracle then runs on one thread)
        cmd = base + cfiles + ["-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P, I64, I32, D, F = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_float
            for sfx in ("d", "s"):
                for nm in ("k2ref_gesvd2_", "k2ref_gesvd2_ncr_"):
                    fn = getattr(L, nm + sfx)
                    fn.argtypes = [I64, P, I64, P, I64, P, I64, P, I64, P, P, P, C.c_int]
                    fn.restype = C.c_int
                for nm in ("k2ref_trsvd2_", "k2ref_trsvd2_ncr_"):
                    fn = getattr(L, nm + sfx)
                    fn.argtypes = [I64, P, P, P, P, I64, P, I64, P, I64, P, P, P, C.c_int]
                    fn.restype = C.c_int
                T = D if sfx == "d" else F
                fn = getattr(L, "k2ref_hypot_ncr_" + sfx)
                fn.argtypes = [T, T]
                fn.restype = T
                getattr(L, "k2ref_hypot_ncr_n_" + sfx).argtypes = [I64, P, P, P, C.c_int]
                getattr(L, "k2ref_trace_m_" + sfx).argtypes = [P, P, P, C.c_int]
                fn = getattr(L, "k2ref_hypot_" + sfx)
                fn.argtypes = [T, T]
                getattr(L, "k2ref_hypot_n_" + sfx).argtypes = [I64, P, P, P, C.c_int]
                getattr(L, "k2ref_prescale2_" + sfx).argtypes = [I64, P, I64, P, I64, P, P, I32, C.c_int]
                getattr(L, "k2ref_lasv2_" + sfx).argtypes = [I64, P, P, P, P, P, P, P, P, P, C.c_int]
                getattr(L, "k2ref_cgesvd2_" + sfx).argtypes = [I64, P, I64, P, I64, P, I64, P, I64, P, C.c_int]
                fn.restype = T
                getattr(L, "k2ref_trace_" + sfx).argtypes = [P, P, P]
                getattr(L, "k2ref_efops_" + sfx).argtypes = [T, T, P, P]
                fn = getattr(L, "k2ref_prec_" + sfx)
                fn.argtypes = [I32, T, I32, T]
                fn.restype = C.c_int
                fn = getattr(L, "k2ref_effl_" + sfx)
                fn.argtypes = [I32, T]
                fn.restype = T
                fn = getattr(L, "k2ref_ext_" + sfx)
                fn.argtypes = [T, T, T, T, C.c_int, T, T]
                fn.restype = T
            L.k2ref_brute_sigma.argtypes = [P, P, P, P]
            L.k2ref_opcount.argtypes = [C.c_int, P, C.c_int]
            L.k2ref_dmetrics.argtypes = [I64, P, I64, P, I64, P, I64, P, P, I64, P]
            _lib = L
            _bind_extra(L)
    return _lib


def _bind_extra(L):
    """Bindings of the n x n driver and the backward reference, when compiled in."""
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    for sfx in ("d", "s"):
        for nm in ("k2ref_kogbet_", "k2ref_kogbet_dyn_"):
            fn = getattr(L, nm + sfx)
            fn.argtypes = [I32, P, P, P, P, C.c_int, D, P, P]
            fn.restype = C.c_int
        fn = getattr(L, "k2ref_dyn_pairs_" + sfx)
        fn.argtypes = [I32, P, P, P]
        fn.restype = C.c_int
        getattr(L, "k2ref_kog_sigma_bwd_" + sfx).argtypes = [I32, P, P, P, P]
    if hasattr(L, "k2ref_gesvd2_bwd_d"):
        L.k2ref_gesvd2_bwd_d.argtypes = [I64, P, P, P, I64, P, P, P, P, D]
        L.k2ref_gesvd2_bwd_d.restype = C.c_int


def _ptr(a):
    return None if a is None else a.ctypes.data


def _dt(prec):
    return np.float64 if prec == "d" else np.float32


def gesvd2(G, prec="d", nthreads=1, ncr=False):
    """SVD of a batch of 2x2 matrices given as SoA planes G[4, n] (g11, g21, g12, g22).

    Returns a dict with U[4,n], V[4,n] (column-major planes), S[2,n] (rounded singular
    values), Se[2,n] and Sf[2,n] (exact (e,f) form) and info[n].  ncr: the method with the
    hypot that is not correctly rounded (xLAPY2's formula) and Alg. 1's branch for it."""
    T = _dt(prec)
    G = np.ascontiguousarray(G, dtype=T)
    n = G.shape[1]
    U = np.empty((4, n), T); V = np.empty((4, n), T); S = np.empty((2, n), T)
    Se = np.empty((2, n), np.int32); Sf = np.empty((2, n), T); info = np.empty(n, np.int32)
    rc = getattr(lib(), ("k2ref_gesvd2_ncr_" if ncr else "k2ref_gesvd2_") + prec)(n, _ptr(G), n, _ptr(U), n, _ptr(V), n, _ptr(S), n,
                                                 _ptr(Se), _ptr(Sf), _ptr(info), int(nthreads))
    if rc != 0:
        raise ValueError("k2ref_gesvd2 returned %d" % rc)
    return {"U": U, "V": V, "S": S, "Se": Se, "Sf": Sf, "info": info}


def trsvd2(F, Gp, H, prec="d", nthreads=1, ncr=False):
    """SVD of upper-triangular R = [[F, Gp], [0, H]] given as three planes (ncr: as gesvd2)."""
    T = _dt(prec)
    F = np.ascontiguousarray(F, dtype=T); Gp = np.ascontiguousarray(Gp, dtype=T)
    H = np.ascontiguousarray(H, dtype=T)
    n = F.shape[0]
    U = np.empty((4, n), T); V = np.empty((4, n), T); S = np.empty((2, n), T)
    Se = np.empty((2, n), np.int32); Sf = np.empty((2, n), T); info = np.empty(n, np.int32)
    rc = getattr(lib(), ("k2ref_trsvd2_ncr_" if ncr else "k2ref_trsvd2_") + prec)(n, _ptr(F), _ptr(Gp), _ptr(H), _ptr(U), n, _ptr(V), n,
                                                 _ptr(S), n, _ptr(Se), _ptr(Sf), _ptr(info), int(nthreads))
    if rc != 0:
        raise ValueError("k2ref_trsvd2 returned %d" % rc)
    return {"U": U, "V": V, "S": S, "Se": Se, "Sf": Sf, "info": info}


def hypot(x, y, prec="d"):
    """Correctly rounded hypot (Sect. 2)."""
    return getattr(lib(), "k2ref_hypot_" + prec)(x, y)


def hypot_n(x, y, prec="d", nthreads=1):
    """Correctly rounded hypot (Sect. 2) of arrays x, y, elementwise."""
    T = _dt(prec)
    x = np.ascontiguousarray(x, dtype=T); y = np.ascontiguousarray(y, dtype=T)
    h = np.empty_like(x)
    getattr(lib(), "k2ref_hypot_n_" + prec)(x.size, _ptr(x), _ptr(y), _ptr(h), int(nthreads))
    return h


def hypot_ncr(x, y, prec="d"):
    """The hypot that is not correctly rounded (xLAPY2's scaled formula, every step rounded once)."""
    return getattr(lib(), "k2ref_hypot_ncr_" + prec)(x, y)


def hypot_ncr_n(x, y, prec="d", nthreads=1):
    """hypot_ncr of arrays x, y, elementwise."""
    T = _dt(prec)
    x = np.ascontiguousarray(x, dtype=T); y = np.ascontiguousarray(y, dtype=T)
    h = np.empty_like(x)
    getattr(lib(), "k2ref_hypot_ncr_n_" + prec)(x.size, _ptr(x), _ptr(y), _ptr(h), int(nthreads))
    return h


def prescale2(G, prec="d", extra=0, nthreads=1):
    """Phase 1 alone (Sect. 3.1): (Gs, s, types) for SoA planes G[4, n]: Gs = 2^s G with the
    scale type raised by `extra`, types = t | t' << 4 (-1 for non-finite input)."""
    T = _dt(prec)
    G = np.ascontiguousarray(G, dtype=T)
    n = G.shape[1]
    Gs = np.empty_like(G); s = np.empty(n, np.int32); types = np.empty(n, np.int32)
    rc = getattr(lib(), "k2ref_prescale2_" + prec)(n, _ptr(G), n, _ptr(Gs), n, _ptr(s), _ptr(types), int(extra),
                                                    int(nthreads))
    if rc != 0:
        raise ValueError("k2ref_prescale2 returned %d" % rc)
    return Gs, s, types


def lasv2(F, Gp, H, prec="d", nthreads=1):
    """The xLASV2 argument shape by the method: (ssmin, ssmax, snr, csr, snl, csl) with
    [csl snl; -snl csl] [[F, Gp], [0, H]] [csr -snr; snr csr] = diag(ssmax, ssmin)."""
    T = _dt(prec)
    F = np.ascontiguousarray(F, dtype=T); Gp = np.ascontiguousarray(Gp, dtype=T)
    H = np.ascontiguousarray(H, dtype=T)
    n = F.shape[0]
    out = [np.empty(n, T) for _ in range(6)]
    rc = getattr(lib(), "k2ref_lasv2_" + prec)(n, _ptr(F), _ptr(Gp), _ptr(H), *[_ptr(o) for o in out], int(nthreads))
    if rc != 0:
        raise ValueError("k2ref_lasv2 returned %d" % rc)
    return tuple(out)


def cgesvd2(G, prec="d", nthreads=1):
    """SVD of complex 2x2 matrices (Sect. 3.4) given as 8 planes G[8, n]: (re, im) of g11, g21,
    g12, g22.  Returns U, V (8, n) in the same layout, S (2, n) and info (n,)."""
    T = _dt(prec)
    G = np.ascontiguousarray(G, dtype=T)
    n = G.shape[1]
    U = np.empty((8, n), T); V = np.empty((8, n), T); S = np.empty((2, n), T); info = np.empty(n, np.int32)
    rc = getattr(lib(), "k2ref_cgesvd2_" + prec)(n, _ptr(G), n, _ptr(U), n, _ptr(V), n, _ptr(S), n, _ptr(info),
                                                  int(nthreads))
    if rc != 0:
        raise ValueError("k2ref_cgesvd2 returned %d" % rc)
    return U, V, S, info


def trace(g, prec="d", ncr=False):
    """Intermediate values of one SVD: (r11, r12, r22, tan2phi, tanphi, tanpsi, tantheta), (t, t', s, flags)."""
    T = _dt(prec)
    g = np.ascontiguousarray(g, dtype=T)
    tr = np.zeros(7, T); ints = np.zeros(4, np.int32)
    getattr(lib(), "k2ref_trace_m_" + prec)(_ptr(g), _ptr(tr), _ptr(ints), int(bool(ncr)))
    return tr, ints


def efops(x, y, prec="d"):
    """(e,f) of x*y, x/y, |x|(+)|y|, |x|(-)|y|, x, y by eqs. (binary), (plus), (minus)."""
    T = _dt(prec)
    e = np.zeros(6, np.int32); f = np.zeros(6, T)
    getattr(lib(), "k2ref_efops_" + prec)(x, y, _ptr(e), _ptr(f))
    return e, f


def prec(ex, fx, ey, fy, p="d"):
    return bool(getattr(lib(), "k2ref_prec_" + p)(ex, fx, ey, fy))


def effl(e, f, prec="d"):
    return getattr(lib(), "k2ref_effl_" + prec)(e, f)


def ext(x1, y1, x2, y2, neg, d, sec, prec="d"):
    """eq. (EXT): fl(fl(FL(FL(x1*y1 +- x2*y2)/d))/sec)."""
    return getattr(lib(), "k2ref_ext_" + prec)(x1, y1, x2, y2, int(neg), d, sec)


OPS = ("add", "mul", "fma", "div", "hypot", "ext", "sqrt")


def opcount(G, prec="d", triangular=False, complex_planes=False, ncr=False):
    """Mean algorithmic operation counts per matrix of the method on a batch (one thread):
    {add, mul, fma, div, hypot, ext, sqrt} (exact scalings, comparisons and sign changes
    excluded; sqrt counts the square roots of the hypot that is not correctly rounded).
    complex_planes: G is 8 planes of complex matrices (Sect. 3.4); ncr: see gesvd2."""
    L = lib()
    buf = np.zeros(7, np.int64)
    L.k2ref_opcount(1 if prec == "d" else 0, _ptr(buf), 1)
    if complex_planes:
        cgesvd2(G, prec, nthreads=1)
        n = G.shape[1]
    elif triangular:
        trsvd2(G[0], G[1], G[2], prec, nthreads=1, ncr=ncr)
        n = G.shape[1]
    else:
        gesvd2(G, prec, nthreads=1, ncr=ncr)
        n = G.shape[1]
    L.k2ref_opcount(1 if prec == "d" else 0, _ptr(buf), 1)
    return {k: float(v) / n for k, v in zip(OPS, buf)}


def gesvd2_bwd(U, S, V, dS=None, dU=None, dV=None, tau=1e-10):
    """Analytic adjoint of the batched 2x2 SVD in binary128 (double in and out):
    dG (4, n) from U, V (4, n), S (2, n) and the optional upstream gradients."""
    U = np.ascontiguousarray(U, np.float64); V = np.ascontiguousarray(V, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    n = U.shape[1]
    cv = lambda a: None if a is None else np.ascontiguousarray(a, np.float64)
    dS, dU, dV = cv(dS), cv(dU), cv(dV)
    dG = np.empty((4, n))
    rc = lib().k2ref_gesvd2_bwd_d(n, _ptr(U), _ptr(S), _ptr(V), n, _ptr(dS), _ptr(dU), _ptr(dV), _ptr(dG), float(tau))
    if rc != 0:
        raise ValueError("k2ref_gesvd2_bwd_d returned %d" % rc)
    return dG


def kogbet(A, prec="d", max_sweeps=40, tol_factor=1.0, dynamic=False):
    """n x n Kogbetliantz SVD of one square matrix (column-major / any numpy array):
    returns (U, S, V, sweeps, info) with A ~ U diag(S) V^T, S descending.  dynamic: the
    dynamic pivot ordering instead of the modulus strategy."""
    T = _dt(prec)
    A = np.asfortranarray(A, dtype=T)
    n = A.shape[0]
    U = np.empty((n, n), T, order="F"); V = np.empty((n, n), T, order="F"); S = np.empty(n, T)
    sw = C.c_int32(0); info = C.c_int32(0)
    fn = getattr(lib(), ("k2ref_kogbet_dyn_" if dynamic else "k2ref_kogbet_") + prec)
    rc = fn(n, _ptr(A), _ptr(U), _ptr(V), _ptr(S), int(max_sweeps), float(tol_factor), C.byref(sw), C.byref(info))
    if rc != 0:
        raise ValueError("k2ref_kogbet returned %d" % rc)
    return U, S, V, sw.value, info.value


def dyn_pairs(G, prec="d"):
    """The pivot pairs of one step of the dynamic ordering taken on the square matrix G, in
    the order taken: a list of (i, j)."""
    T = _dt(prec)
    G = np.asfortranarray(G, dtype=T)
    n = G.shape[0]
    pi = np.zeros(max(n, 1), np.int32); pj = np.zeros(max(n, 1), np.int32)
    np_ = getattr(lib(), "k2ref_dyn_pairs_" + prec)(n, _ptr(G), _ptr(pi), _ptr(pj))
    return [(int(pi[p]), int(pj[p])) for p in range(np_)]


def gesvdr(A, prec="d", max_sweeps=40, tol_factor=1.0):
    """SVD of one rectangular m x n matrix by QR with column pivoting to a square one and the
    n x n Kogbetliantz method (Sect. 1): returns (U (m x k), S (k), V (n x k), sweeps, info),
    k = min(m, n), A ~ U diag(S) V^T."""
    T = _dt(prec)
    A = np.asfortranarray(A, dtype=T)
    m, n = A.shape
    k = min(m, n)
    U = np.empty((m, k), T, order="F"); V = np.empty((n, k), T, order="F"); S = np.empty(k, T)
    sw = C.c_int32(0); info = C.c_int32(0)
    fn = getattr(lib(), "k2ref_gesvdr_" + prec)
    fn.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                   C.c_void_p, C.c_void_p]
    rc = fn(m, n, _ptr(A), _ptr(U), _ptr(V), _ptr(S), int(max_sweeps), float(tol_factor), C.byref(sw), C.byref(info))
    if rc != 0:
        raise ValueError("k2ref_gesvdr returned %d" % rc)
    return U, S, V, sw.value, info.value


def kog_sigma_bwd(U, V, dS, prec="d"):
    """dA = U diag(dS) V^T for one n x n matrix (column-major), in the order of the C ABI."""
    T = _dt(prec)
    U = np.asfortranarray(U, dtype=T); V = np.asfortranarray(V, dtype=T)
    dS = np.ascontiguousarray(dS, dtype=T)
    n = U.shape[0]
    dA = np.empty((n, n), T, order="F")
    getattr(lib(), "k2ref_kog_sigma_bwd_" + prec)(n, _ptr(U), _ptr(V), _ptr(dS), _ptr(dA))
    return dA


def brute_sigma(g):
    """Closed-form singular values of one double 2x2 matrix in binary128 (not the method):
    returns [(e, hi, lo), (e, hi, lo)] with sigma = (hi + lo) * 2^e."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    e = np.zeros(2, np.int32); hi = np.zeros(2); lo = np.zeros(2)
    lib().k2ref_brute_sigma(_ptr(g), _ptr(e), _ptr(hi), _ptr(lo))
    return [(int(e[k]), float(hi[k]), float(lo[k])) for k in range(2)]


def dmetrics(G, out):
    """re sigma1, re sigma2, re U, re V, re G (Sect. 4) in binary128 for double results."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    n = G.shape[1]
    U = np.ascontiguousarray(out["U"], np.float64); V = np.ascontiguousarray(out["V"], np.float64)
    Se = np.ascontiguousarray(out["Se"], np.int32); Sf = np.ascontiguousarray(out["Sf"], np.float64)
    m = np.empty((5, n))
    lib().k2ref_dmetrics(n, _ptr(G), n, _ptr(U), n, _ptr(V), n, _ptr(Se), _ptr(Sf), n, _ptr(m))
    return m
