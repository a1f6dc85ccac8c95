"""Python binding of libk2svd (include/k2svd.h): argument marshalling only.

Every function takes torch tensors that live on the current CUDA device, checks their
dtype, device and layout, and calls the C ABI on torch's current stream.  All arithmetic
runs in the library's kernels; there is no CPU path.  Loading fails with an error when
the library has not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_lib = None
_probe = None

INFO_FLAGS = {"ext": 1 << 8, "fallback": 1 << 9, "swap": 1 << 10, "t2f2": 1 << 11,
              "t2f3": 1 << 12, "t2inf": 1 << 13, "tpinf": 1 << 14, "psig": 1 << 15}


class K2SVDError(RuntimeError):
    pass


def lib():
    """The loaded libk2svd (ctypes.CDLL)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise K2SVDError("libk2svd is not built (%s missing); run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        P, I64 = C.c_void_p, C.c_int64
        for p in ("d", "s"):
            for sfx in ("", "_ncr"):
                f = getattr(L, "k2svd_%sgesvd2%s" % (p, sfx))
                f.argtypes = [I64, P, I64, P, I64, P, I64, P, I64, P, P, P, P]
                f.restype = C.c_int
                f = getattr(L, "k2svd_%strsvd2%s" % (p, sfx))
                f.argtypes = [I64, P, P, P, P, I64, P, I64, P, I64, P, P, P, P]
                f.restype = C.c_int
        _bind_extra(L)
        _lib = L
    return _lib


def probe_lib():
    """The loaded measurement library libk2probe (include/k2probe.h): pipe-rate probes and
    elementwise checks of the division and hypot primitives; not part of the method."""
    global _probe
    if _probe is None:
        path = _build.PROBE_LIB
        if not os.path.exists(path):
            raise K2SVDError("libk2probe is not built (%s missing); run __graft_entry__.build()" % path)
        _probe = C.CDLL(path)
    return _probe


def _bind_extra(L):
    P, I64, I32, D, F, SZ = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_float, C.c_size_t
    L.k2svd_dgesvd2_bwd.argtypes = [I64, P, P, P, I64, P, P, P, P, D, P]
    L.k2svd_dgesvd2_bwd.restype = C.c_int
    L.k2svd_sgesvd2_bwd.argtypes = [I64, P, P, P, I64, P, P, P, P, F, P]
    L.k2svd_sgesvd2_bwd.restype = C.c_int
    for p in ("d", "s"):
        f = getattr(L, "k2svd_%sgesvdr_ws" % p)
        f.argtypes = [I64, P, P, I32, C.POINTER(SZ)]
        f.restype = C.c_int
        f = getattr(L, "k2svd_%sgesvdr" % p)
        f.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, P, P, I32, D, I32, P, SZ, P]
        f.restype = C.c_int
    for p in ("z", "c"):
        f = getattr(L, "k2svd_%sgesvd2" % p)
        f.argtypes = [I64, P, I64, P, I64, P, I64, P, I64, P, P]
        f.restype = C.c_int
    for p, T in (("d", D), ("s", F)):
        f = getattr(L, "k2svd_%sprescale2" % p)
        f.argtypes = [I64, P, I64, P, I64, P, P, I32, P]
        f.restype = C.c_int
        f = getattr(L, "k2svd_%slasv2" % p)
        f.argtypes = [I64, P, P, P, P, P, P, P, P, P, P]
        f.restype = C.c_int
    for p in ("d", "s"):
        f = getattr(L, "k2svd_%skogbet_ws" % p)
        f.argtypes = [I64, P, I32, C.POINTER(SZ)]
        f.restype = C.c_int
        f = getattr(L, "k2svd_%skogbet" % p)
        f.argtypes = [I64, P, P, P, P, P, P, P, P, P, I32, D, I32, P, SZ, P]
        f.restype = C.c_int
        f = getattr(L, "k2svd_%skog_sigma_bwd" % p)
        f.argtypes = [I64, P, P, P, P, P, P, P, P, SZ, P]
        f.restype = C.c_int


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _prefix(dtype):
    if dtype == torch.float64:
        return "d"
    if dtype == torch.float32:
        return "s"
    raise K2SVDError("dtype must be float64 or float32, got %s" % dtype)


def _check(t, name, dtype, device):
    if t.dtype != dtype:
        raise K2SVDError("%s: dtype %s, expected %s" % (name, t.dtype, dtype))
    if t.device != device:
        raise K2SVDError("%s: device %s, expected %s" % (name, t.device, device))
    if not t.is_cuda:
        raise K2SVDError("%s must be a CUDA tensor" % name)


def _planes(t, k, name):
    """(k, n) tensor with unit stride inside a plane; returns its leading dimension."""
    if t.dim() != 2 or t.shape[0] != k:
        raise K2SVDError("%s must have shape (%d, n), got %s" % (name, k, tuple(t.shape)))
    if t.stride(1) != 1 and t.shape[1] > 1:
        raise K2SVDError("%s: planes must be contiguous" % name)
    return t.stride(0) if t.shape[0] > 1 else t.shape[1]


def gesvd2(G, U=None, V=None, S=None, Se=None, Sf=None, info=None, want_ef=False, want_info=True, ncr=False):
    """SVD of the 2x2 matrices in the SoA planes G (4, n): (g11, g21, g12, g22).

    Returns (U, V, S, Se, Sf, info) with U, V (4, n) column-major planes, S (2, n) rounded
    singular values, Se/Sf (2, n) the exact (e,f) form (None unless requested) and info (n,).
    ncr: k2svd_?gesvd2_ncr, the variant with a hypot that is not correctly rounded."""
    p = _prefix(G.dtype)
    dev = G.device
    _check(G, "G", G.dtype, dev)
    n = G.shape[1]
    ldg = _planes(G, 4, "G")
    U = torch.empty((4, n), dtype=G.dtype, device=dev) if U is None else U
    V = torch.empty((4, n), dtype=G.dtype, device=dev) if V is None else V
    S = torch.empty((2, n), dtype=G.dtype, device=dev) if S is None else S
    if want_ef:
        Se = torch.empty((2, n), dtype=torch.int32, device=dev) if Se is None else Se
        Sf = torch.empty((2, n), dtype=G.dtype, device=dev) if Sf is None else Sf
    if want_info and info is None:
        info = torch.empty((n,), dtype=torch.int32, device=dev)
    for t, nm, dt in ((U, "U", G.dtype), (V, "V", G.dtype), (S, "S", G.dtype)):
        _check(t, nm, dt, dev)
    ldu, ldv, lds = _planes(U, 4, "U"), _planes(V, 4, "V"), _planes(S, 2, "S")
    if Se is not None:
        _check(Se, "Se", torch.int32, dev)
        if _planes(Se, 2, "Se") != lds:
            raise K2SVDError("Se must have the leading dimension of S")
    if Sf is not None:
        _check(Sf, "Sf", G.dtype, dev)
        if _planes(Sf, 2, "Sf") != lds:
            raise K2SVDError("Sf must have the leading dimension of S")
    if info is not None:
        _check(info, "info", torch.int32, dev)
    name = "k2svd_%sgesvd2%s" % (p, "_ncr" if ncr else "")
    with torch.cuda.device(dev):
        rc = getattr(lib(), name)(n, _ptr(G), ldg, _ptr(U), ldu, _ptr(V), ldv, _ptr(S), lds,
                                  _ptr(Se), _ptr(Sf), _ptr(info), _stream())
    if rc != 0:
        raise K2SVDError("%s returned %d" % (name, rc))
    return U, V, S, Se, Sf, info


def gesvd2_ncr(G, **kw):
    """k2svd_?gesvd2_ncr: gesvd2 with the hypot that is not correctly rounded (Alg. 1's branch for it)."""
    return gesvd2(G, ncr=True, **kw)


def trsvd2(F, Gu, H, U=None, V=None, S=None, Se=None, Sf=None, info=None, want_ef=False, want_info=True,
           ncr=False):
    """SVD of the upper-triangular matrices [[F, Gu], [0, H]] given as three (n,) planes
    (ncr: k2svd_?trsvd2_ncr)."""
    p = _prefix(F.dtype)
    dev = F.device
    for t, nm in ((F, "F"), (Gu, "Gu"), (H, "H")):
        _check(t, nm, F.dtype, dev)
        if t.dim() != 1 or (t.numel() > 1 and t.stride(0) != 1):
            raise K2SVDError("%s must be a contiguous vector" % nm)
    n = F.shape[0]
    if Gu.shape[0] != n or H.shape[0] != n:
        raise K2SVDError("F, Gu, H must have the same length")
    U = torch.empty((4, n), dtype=F.dtype, device=dev) if U is None else U
    V = torch.empty((4, n), dtype=F.dtype, device=dev) if V is None else V
    S = torch.empty((2, n), dtype=F.dtype, device=dev) if S is None else S
    if want_ef:
        Se = torch.empty((2, n), dtype=torch.int32, device=dev) if Se is None else Se
        Sf = torch.empty((2, n), dtype=F.dtype, device=dev) if Sf is None else Sf
    if want_info and info is None:
        info = torch.empty((n,), dtype=torch.int32, device=dev)
    ldu, ldv, lds = _planes(U, 4, "U"), _planes(V, 4, "V"), _planes(S, 2, "S")
    name = "k2svd_%strsvd2%s" % (p, "_ncr" if ncr else "")
    with torch.cuda.device(dev):
        rc = getattr(lib(), name)(n, _ptr(F), _ptr(Gu), _ptr(H), _ptr(U), ldu, _ptr(V), ldv,
                                  _ptr(S), lds, _ptr(Se), _ptr(Sf), _ptr(info), _stream())
    if rc != 0:
        raise K2SVDError("%s returned %d" % (name, rc))
    return U, V, S, Se, Sf, info


def trsvd2_ncr(F, Gu, H, **kw):
    """k2svd_?trsvd2_ncr: trsvd2 with the hypot that is not correctly rounded."""
    return trsvd2(F, Gu, H, ncr=True, **kw)


def rect_layout(shapes):
    """Packed layout of a batch of m x n matrices: (m, n, aoffs, uoffs, voffs, soffs, sizes)
    with A_i, U_i (m x k), V_i (n x k), S_i (k), k = min(m, n), consecutive and column-major;
    sizes = (total A, total U, total V, total S)."""
    shp = np.asarray(shapes, dtype=np.int64).reshape(-1, 2)
    m, n = shp[:, 0], shp[:, 1]
    k = np.minimum(m, n)
    cum = lambda x: np.concatenate([[0], np.cumsum(x)[:-1]]).astype(np.int64)
    return (m.astype(np.int32), n.astype(np.int32), cum(m * n), cum(m * k), cum(n * k), cum(k),
            (int((m * n).sum()), int((m * k).sum()), int((n * k).sum()), int(k.sum())))


def gesvdr(A, shapes, max_sweeps=40, tol_factor=1.0, flags=0):
    """SVD of a packed batch of rectangular matrices (k2svd_?gesvdr): QR with column pivoting
    to square, then the n x n Kogbetliantz driver.  A: flat tensor in rect_layout order.
    Returns (U, S, V, sweeps, info), each flat in the same layout."""
    p = _prefix(A.dtype)
    dev = A.device
    _check(A, "A", A.dtype, dev)
    m, n, ao, uo, vo, so, (na, nu, nv, ns) = rect_layout(shapes)
    if A.numel() < na:
        raise K2SVDError("A holds %d elements, the shapes need %d" % (A.numel(), na))
    b = len(m)
    U = torch.empty(nu, dtype=A.dtype, device=dev)
    V = torch.empty(nv, dtype=A.dtype, device=dev)
    S = torch.empty(ns, dtype=A.dtype, device=dev)
    sw = torch.empty(b, dtype=torch.int32, device=dev)
    info = torch.empty(b, dtype=torch.int32, device=dev)
    L = lib()
    wsb = C.c_size_t(0)
    rc = getattr(L, "k2svd_%sgesvdr_ws" % p)(b, m.ctypes.data, n.ctypes.data, int(flags), C.byref(wsb))
    if rc != 0:
        raise K2SVDError("k2svd_%sgesvdr_ws returned %d" % (p, rc))
    ws = torch.empty(wsb.value + 256, dtype=torch.uint8, device=dev)
    wp = (ws.data_ptr() + 255) // 256 * 256
    with torch.cuda.device(dev):
        rc = getattr(L, "k2svd_%sgesvdr" % p)(b, m.ctypes.data, n.ctypes.data, ao.ctypes.data, uo.ctypes.data,
                                              vo.ctypes.data, so.ctypes.data, _ptr(A), _ptr(U), _ptr(V), _ptr(S),
                                              _ptr(sw), _ptr(info), int(max_sweeps), float(tol_factor), int(flags),
                                              C.c_void_p(wp), wsb.value, _stream())
    if rc != 0:
        raise K2SVDError("k2svd_%sgesvdr returned %d" % (p, rc))
    torch.cuda.current_stream(dev).synchronize()      # the workspace is released on return
    return U, S, V, sw, info


def cgesvd2(G, U=None, V=None, S=None, want_info=True):
    """SVD of complex 2x2 matrices (k2svd_zgesvd2 / k2svd_cgesvd2).  G is (8, n) real planes
    (re, im of g11, g21, g12, g22) of float64 or float32; returns (U, V, S, info) with U, V
    (8, n) in the same layout and S (2, n).  See complex_to_planes / planes_to_complex."""
    p = {"d": "z", "s": "c"}[_prefix(G.dtype)]
    dev = G.device
    _check(G, "G", G.dtype, dev)
    n = G.shape[1]
    ldg = _planes(G, 8, "G")
    U = torch.empty((8, n), dtype=G.dtype, device=dev) if U is None else U
    V = torch.empty((8, n), dtype=G.dtype, device=dev) if V is None else V
    S = torch.empty((2, n), dtype=G.dtype, device=dev) if S is None else S
    info = torch.empty((n,), dtype=torch.int32, device=dev) if want_info else None
    for t, nm, k in ((U, "U", 8), (V, "V", 8), (S, "S", 2)):
        _check(t, nm, G.dtype, dev)
    ldu, ldv, lds = _planes(U, 8, "U"), _planes(V, 8, "V"), _planes(S, 2, "S")
    with torch.cuda.device(dev):
        rc = getattr(lib(), "k2svd_%sgesvd2" % p)(n, _ptr(G), ldg, _ptr(U), ldu, _ptr(V), ldv, _ptr(S), lds,
                                                  _ptr(info), _stream())
    if rc != 0:
        raise K2SVDError("k2svd_%sgesvd2 returned %d" % (p, rc))
    return U, V, S, info


def complex_to_planes(A):
    """(..., 2, 2) complex tensor -> (8, n) real planes (re, im of a11, a21, a12, a22)."""
    A = A.reshape(-1, 2, 2)
    X = torch.stack([A[:, 0, 0], A[:, 1, 0], A[:, 0, 1], A[:, 1, 1]])
    return torch.stack([X.real, X.imag], dim=1).reshape(8, -1).contiguous()


def planes_to_complex(X, shape=None):
    """(8, n) real planes -> (n, 2, 2) complex tensor (or `shape` + (2, 2))."""
    Y = X.reshape(4, 2, -1)
    Z = torch.complex(Y[:, 0], Y[:, 1])
    A = torch.stack([torch.stack([Z[0], Z[2]], -1), torch.stack([Z[1], Z[3]], -1)], -2)
    return A if shape is None else A.reshape(tuple(shape) + (2, 2))


def prescale2(G, extra=0, Gs=None, want_types=True):
    """Phase 1 alone (k2svd_?prescale2): returns (Gs, s, types) with Gs = 2^s G (4, n) planes,
    s the int32 exponents and types = t | t' << 4 (-1 for non-finite input)."""
    p = _prefix(G.dtype)
    dev = G.device
    _check(G, "G", G.dtype, dev)
    n = G.shape[1]
    ldg = _planes(G, 4, "G")
    Gs = torch.empty((4, n), dtype=G.dtype, device=dev) if Gs is None else Gs
    _check(Gs, "Gs", G.dtype, dev)
    ldgs = _planes(Gs, 4, "Gs")
    s = torch.empty((n,), dtype=torch.int32, device=dev)
    types = torch.empty((n,), dtype=torch.int32, device=dev) if want_types else None
    with torch.cuda.device(dev):
        rc = getattr(lib(), "k2svd_%sprescale2" % p)(n, _ptr(G), ldg, _ptr(Gs), ldgs, _ptr(s), _ptr(types),
                                                     int(extra), _stream())
    if rc != 0:
        raise K2SVDError("k2svd_%sprescale2 returned %d" % (p, rc))
    return Gs, s, types


def lasv2(F, G, H):
    """The xLASV2 argument shape by the method (k2svd_?lasv2): (ssmin, ssmax, snr, csr, snl,
    csl), each (n,), with [csl snl; -snl csl] [[F, G], [0, H]] [csr -snr; snr csr] =
    diag(ssmax, ssmin)."""
    p = _prefix(F.dtype)
    dev = F.device
    for t, nm in ((F, "F"), (G, "G"), (H, "H")):
        _check(t, nm, F.dtype, dev)
        if t.dim() != 1 or (t.numel() > 1 and t.stride(0) != 1) or t.shape[0] != F.shape[0]:
            raise K2SVDError("%s must be a contiguous vector of the length of F" % nm)
    n = F.shape[0]
    out = [torch.empty((n,), dtype=F.dtype, device=dev) for _ in range(6)]
    with torch.cuda.device(dev):
        rc = getattr(lib(), "k2svd_%slasv2" % p)(n, _ptr(F), _ptr(G), _ptr(H), *[_ptr(o) for o in out], _stream())
    if rc != 0:
        raise K2SVDError("k2svd_%slasv2 returned %d" % (p, rc))
    return tuple(out)


def gesvd2_bwd(U, S, V, dS=None, dU=None, dV=None, gap_rtol=1e-10, dG=None):
    """Adjoint of gesvd2: dG (4, n) from U, V (4, n), S (2, n) and the optional upstream
    gradients dS (2, n), dU, dV (4, n).  All planes must share one leading dimension."""
    p = _prefix(U.dtype)
    dev = U.device
    n = U.shape[1]
    ld = _planes(U, 4, "U")
    for t, nm, k in ((S, "S", 2), (V, "V", 4), (dS, "dS", 2), (dU, "dU", 4), (dV, "dV", 4)):
        if t is None:
            continue
        _check(t, nm, U.dtype, dev)
        if t.shape[1] != n or _planes(t, k, nm) != ld:
            raise K2SVDError("%s must have shape (%d, %d) and the leading dimension of U" % (nm, k, n))
    if dG is None:
        dG = torch.empty((4, ld), dtype=U.dtype, device=dev)[:, :n]
    _check(dG, "dG", U.dtype, dev)
    if _planes(dG, 4, "dG") != ld:
        raise K2SVDError("dG must have the leading dimension of U")
    with torch.cuda.device(dev):
        rc = getattr(lib(), "k2svd_%sgesvd2_bwd" % p)(n, _ptr(U), _ptr(S), _ptr(V), ld, _ptr(dS), _ptr(dU), _ptr(dV),
                                                      _ptr(dG), float(gap_rtol), _stream())
    if rc != 0:
        raise K2SVDError("k2svd_%sgesvd2_bwd returned %d" % (p, rc))
    return dG


def svd2_host(jobs, depth=3, device=None, trace=None, in_depth=8, streams=None):
    """Batched 2x2 SVDs of matrices that live in pinned host memory, streamed through the
    device chunk by chunk.  `jobs` is a list of (inputs, outputs, triangular) with
    inputs (nc, 4, c) planes g11, g21, g12, g22 (or (nc, 3, c): F, Gu, H when triangular)
    and outputs (nc, 10, c): per chunk U (4 planes), V (4 planes), S (2 planes), both
    pinned and contiguous, so that each chunk moves in one copy each way.  Three streams
    run the stages -- host-to-device copies, the kernels (k2svd_?gesvd2 / k2svd_?trsvd2),
    device-to-host copies.  Input buffers (`in_depth` of them) are reused once the kernel
    that read them is done, output buffers (`depth`) once their copy to the host is done,
    so the uploads run up to `in_depth` chunks ahead of the kernels whatever the pace of
    the downloads, and copies in both directions overlap the kernels of other chunks.
    Returns when every output is in host memory.  Only data movement happens here; the
    arithmetic is the library's kernels.
    trace: if a list, CUDA events bracket every copy and kernel, and one dict per chunk is
    appended with the start (ms after the call's first event) and duration of each stage.
    streams: the (copy-in, kernel, copy-out) torch streams to use; three streams from
    torch's pool when None."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    jobs = list(jobs)
    if not jobs:
        return
    if depth < 1 or in_depth < 1:
        raise K2SVDError("svd2_host: depth and in_depth must be at least 1")
    dt, c = jobs[0][0].dtype, jobs[0][0].shape[2]
    for x, y, tri in jobs:
        if x.dtype != dt or y.dtype != dt or x.shape[2] != c or y.shape[2] != c or y.shape[1] != 10:
            raise K2SVDError("svd2_host: every job needs (nc, 4|3, c) inputs and (nc, 10, c) outputs of one dtype")
        if x.shape[1] != (3 if tri else 4) or x.shape[0] != y.shape[0]:
            raise K2SVDError("svd2_host: input planes or chunk counts do not match")
        if x.is_cuda or y.is_cuda or not (x.is_pinned() and y.is_pinned()):
            raise K2SVDError("svd2_host: inputs and outputs must be pinned host tensors")
        if not (x.is_contiguous() and y.is_contiguous()):
            raise K2SVDError("svd2_host: inputs and outputs must be contiguous")
    if streams is None:
        s_in, s_run, s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
    else:
        s_in, s_run, s_out = streams
    bin_ = [torch.empty((4, c), dtype=dt, device=dev) for _ in range(in_depth)]
    bout = [torch.empty((10, c), dtype=dt, device=dev) for _ in range(depth)]
    in_free = [None] * in_depth                 # the kernel that last read input buffer i is done
    out_free = [None] * depth                   # output buffer k is back in host memory
    main = torch.cuda.current_stream(dev)
    s_in.wait_stream(main)
    s_run.wait_stream(main)
    timed = trace is not None
    mark = lambda: torch.cuda.Event(enable_timing=True) if timed else None
    ev = []
    t0 = mark()
    if timed:
        t0.record(s_in)
    j = 0
    for x, y, tri in jobs:
        for q in range(x.shape[0]):
            ki, ko = j % in_depth, j % depth
            j += 1
            e = [mark() for _ in range(6)] if timed else None
            with torch.cuda.stream(s_in):
                if in_free[ki] is not None:
                    s_in.wait_event(in_free[ki])
                dst = bin_[ki][: x.shape[1]]
                if timed:
                    e[0].record(s_in)
                dst.copy_(x[q], non_blocking=True)
                loaded = torch.cuda.Event(enable_timing=timed)
                loaded.record(s_in)
            with torch.cuda.stream(s_run):
                s_run.wait_event(loaded)
                if out_free[ko] is not None:
                    s_run.wait_event(out_free[ko])
                if timed:
                    e[2].record(s_run)
                b = bout[ko]
                if tri:
                    trsvd2(dst[0], dst[1], dst[2], U=b[0:4], V=b[4:8], S=b[8:10], want_info=False)
                else:
                    gesvd2(dst, U=b[0:4], V=b[4:8], S=b[8:10], want_info=False)
                done = torch.cuda.Event(enable_timing=timed)
                done.record(s_run)
                in_free[ki] = done
            with torch.cuda.stream(s_out):
                s_out.wait_event(done)
                if timed:
                    e[4].record(s_out)
                y[q].copy_(b, non_blocking=True)
                out_free[ko] = torch.cuda.Event(enable_timing=timed)
                out_free[ko].record(s_out)
            if timed:
                e[1], e[3], e[5] = loaded, done, out_free[ko]
                ev.append(e)
    main.wait_stream(s_out)
    torch.cuda.synchronize(dev)
    for e in ev:
        trace.append({"start_ms": t0.elapsed_time(e[0]), "h2d_ms": e[0].elapsed_time(e[1]),
                      "kernel_ms": e[2].elapsed_time(e[3]), "d2h_ms": e[4].elapsed_time(e[5]),
                      "end_ms": t0.elapsed_time(e[5])})


def to_planes(A):
    """(..., 2, 2) matrices -> (4, n) SoA planes in column-major element order."""
    a = A.reshape(-1, 2, 2)
    return torch.stack([a[:, 0, 0], a[:, 1, 0], a[:, 0, 1], a[:, 1, 1]]).contiguous()


def from_planes(X, shape):
    """(4, n) planes -> (..., 2, 2)."""
    m = torch.stack([torch.stack([X[0], X[2]], -1), torch.stack([X[1], X[3]], -1)], -2)
    return m.reshape(*shape, 2, 2)


# ------------------------------------------------------------------------------------------
# batched n x n Kogbetliantz SVD
# ------------------------------------------------------------------------------------------
KOG_PLAIN, KOG_GRAPH, KOG_NOTUNE, KOG_DYNAMIC = 1, 2, 4, 8


def kog_layout(orders):
    """Host arrays (n, offs, soffs) of a packed batch: matrix i occupies n_i^2 consecutive
    elements (column-major), its singular values n_i consecutive elements."""
    import numpy as np
    n = np.ascontiguousarray(orders, dtype=np.int32)
    sq = n.astype(np.int64) ** 2
    offs = np.concatenate([[0], np.cumsum(sq)[:-1]]).astype(np.int64)
    soffs = np.concatenate([[0], np.cumsum(n.astype(np.int64))[:-1]]).astype(np.int64)
    return n, offs, soffs, int(sq.sum()), int(n.sum())


def pack(mats):
    """List of (n_i, n_i) tensors -> (flat column-major tensor, orders)."""
    flat = torch.cat([m.t().contiguous().reshape(-1) for m in mats]) if mats else torch.empty(0)
    return flat, [int(m.shape[0]) for m in mats]


def unpack(flat, orders, square=True):
    """Inverse of pack (square=True) or the split of a packed vector of singular values."""
    out, o = [], 0
    for n in orders:
        k = n * n if square else n
        x = flat[o:o + k]
        out.append(x.reshape(n, n).t() if square else x)
        o += k
    return out


def kogbet_workspace(orders, dtype, flags=0, device=None):
    """A workspace tensor (uint8) sized by k2svd_?kogbet_ws for this batch and flags."""
    n, _, _, _, _ = kog_layout(orders)
    size = C.c_size_t(0)
    rc = getattr(lib(), "k2svd_%skogbet_ws" % _prefix(dtype))(len(n), n.ctypes.data, int(flags), C.byref(size))
    if rc != 0:
        raise K2SVDError("k2svd_kogbet_ws returned %d" % rc)
    return torch.empty((max(int(size.value), 256),), dtype=torch.uint8, device=device)


def kogbet(A, orders, max_sweeps=40, tol_factor=1.0, flags=0, workspace=None, U=None, V=None, S=None,
           sweeps=None, info=None):
    """SVD of the packed batch A (flat, column-major per matrix, orders[i] each) by the
    persistent Kogbetliantz driver (flags: KOG_PLAIN for the per-step form, KOG_GRAPH to
    launch through a cached CUDA graph, KOG_DYNAMIC for the dynamic pivot ordering).
    Returns (U, S, V, sweeps, info) packed like A."""
    p = _prefix(A.dtype)
    dev = A.device
    n, offs, soffs, tot, stot = kog_layout(orders)
    if A.dim() != 1 or A.numel() < tot or (A.numel() > 1 and A.stride(0) != 1):
        raise K2SVDError("A must be a contiguous vector of at least %d elements" % tot)
    U = torch.empty(tot, dtype=A.dtype, device=dev) if U is None else U
    V = torch.empty(tot, dtype=A.dtype, device=dev) if V is None else V
    S = torch.empty(stot, dtype=A.dtype, device=dev) if S is None else S
    sweeps = torch.empty(len(n), dtype=torch.int32, device=dev) if sweeps is None else sweeps
    info = torch.empty(len(n), dtype=torch.int32, device=dev) if info is None else info
    for t, nm in ((U, "U"), (V, "V"), (S, "S")):
        _check(t, nm, A.dtype, dev)
    if workspace is None:
        workspace = kogbet_workspace(orders, A.dtype, flags, dev)
    with torch.cuda.device(dev):
        rc = getattr(lib(), "k2svd_%skogbet" % p)(len(n), n.ctypes.data, offs.ctypes.data, soffs.ctypes.data,
                                                  _ptr(A), _ptr(U), _ptr(V), _ptr(S), _ptr(sweeps), _ptr(info),
                                                  int(max_sweeps), float(tol_factor), int(flags), _ptr(workspace),
                                                  workspace.numel(), _stream())
    if rc != 0:
        raise K2SVDError("k2svd_%skogbet returned %d" % (p, rc))
    return U, S, V, sweeps, info


def kog_sigma_bwd(U, V, dS, orders, workspace=None, dA=None):
    """dA = U diag(dS) V^T for every matrix of a packed batch."""
    p = _prefix(U.dtype)
    dev = U.device
    n, offs, soffs, tot, stot = kog_layout(orders)
    dA = torch.empty(tot, dtype=U.dtype, device=dev) if dA is None else dA
    if workspace is None:
        workspace = torch.empty((max(256, 32 * len(n)),), dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        rc = getattr(lib(), "k2svd_%skog_sigma_bwd" % p)(len(n), n.ctypes.data, offs.ctypes.data, soffs.ctypes.data,
                                                         _ptr(U), _ptr(V), _ptr(dS), _ptr(dA), _ptr(workspace),
                                                         workspace.numel(), _stream())
    if rc != 0:
        raise K2SVDError("k2svd_%skog_sigma_bwd returned %d" % (p, rc))
    return dA
