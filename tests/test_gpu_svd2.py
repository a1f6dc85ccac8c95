"""GPU parity of k2svd_{d,s}gesvd2 and k2svd_{d,s}trsvd2 against the oracle.

Every operation of the method is an IEEE operation with one rounding, so the CUDA path
must reproduce the oracle bit for bit: U, V, the rounded and the (e,f) singular values
and the info word (type, type after prescaling, branch flags)."""
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


def _u(a):
    a = np.ascontiguousarray(a)
    return a.view({8: np.uint64, 4: np.uint32}[a.dtype.itemsize])


def _gpu_ge(G, prec):
    Gt = torch.from_numpy(np.ascontiguousarray(G)).to(DEV)
    U, V, S, Se, Sf, info = k2().gesvd2(Gt, want_ef=True)
    torch.cuda.synchronize()
    return {"U": U.cpu().numpy(), "V": V.cpu().numpy(), "S": S.cpu().numpy(), "Se": Se.cpu().numpy(),
            "Sf": Sf.cpu().numpy(), "info": info.cpu().numpy()}


def _gpu_tr(T3):
    F, Gu, H = (torch.from_numpy(np.ascontiguousarray(T3[k])).to(DEV) for k in range(3))
    U, V, S, Se, Sf, info = k2().trsvd2(F, Gu, H, want_ef=True)
    torch.cuda.synchronize()
    return {"U": U.cpu().numpy(), "V": V.cpu().numpy(), "S": S.cpu().numpy(), "Se": Se.cpu().numpy(),
            "Sf": Sf.cpu().numpy(), "info": info.cpu().numpy()}


def _assert_same(got, ref, tag=""):
    bad = np.zeros(got["info"].shape[0], bool)
    for k in ("U", "V", "S", "Sf"):
        g, r = got[k], ref[k]
        both_nan = np.isnan(g) & np.isnan(r)
        diff = (_u(g) != _u(r)) & ~both_nan
        bad |= diff.any(axis=0)
    bad |= (got["Se"] != ref["Se"]).any(axis=0)
    bad |= got["info"] != ref["info"]
    if bad.any():
        i = int(np.flatnonzero(bad)[0])
        msg = {k: (got[k][..., i], ref[k][..., i]) for k in ("U", "V", "S", "Se", "Sf", "info")}
        raise AssertionError("%s: %d of %d matrices differ; first %d: %s" % (tag, bad.sum(), bad.size, i, msg))


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("kind", ["narrow", "wide"])
def test_parity_general(prec, kind):
    n = (1 << 17) + 77                      # several persistent-grid strides and a ragged tail
    G = I.general(n, 1000 + len(kind), prec, kind)
    _assert_same(_gpu_ge(G, prec), oracle.gesvd2(G, prec, nthreads=8), "gesvd2 %s %s" % (prec, kind))


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("kind", ["narrow", "wide"])
def test_parity_triangular(prec, kind):
    n = (1 << 16) + 13
    T3 = I.triangular(n, 2000 + len(kind), prec, kind)
    _assert_same(_gpu_tr(T3), oracle.trsvd2(T3[0], T3[1], T3[2], prec, nthreads=8), "trsvd2 %s %s" % (prec, kind))


@pytest.mark.parametrize("prec", ["d", "s"])
def test_parity_safe_ranges_and_rotated(prec):
    parts = [I.safe_range(20000, 3000 + c, c, prec) for c in (0, 500 if prec == "d" else 60, 953 if prec == "d" else 120)]
    parts.append(I.safe_range(20000, 3100, 0, prec, triangular_=True))
    G = np.concatenate(parts, axis=1)
    if prec == "d":
        R, _, _ = I.rotated(20000, 3200)
        G = np.concatenate([G, R], axis=1)
    _assert_same(_gpu_ge(G, prec), oracle.gesvd2(G, prec, nthreads=8), "safe/rotated %s" % prec)


def _special_cases(prec):
    T = np.float64 if prec == "d" else np.float32
    fi = np.finfo(T)
    nu, mu, tiny = float(fi.max), float(fi.tiny), float(fi.smallest_subnormal)
    vals = [0.0, -0.0, 1.0, -1.0, 3.0, 4.0, nu, -nu, nu / 4, mu, -mu, tiny, -tiny, 5 * tiny,
            mu * 3, nu / 3, 2.0 ** 60, 2.0 ** -60, 1.5, -2.5]
    rng = np.random.default_rng(5)
    rows = []
    for _ in range(20000):
        rows.append([vals[j] for j in rng.integers(0, len(vals), 4)])
    # the branch cases of the oracle pins, scaled into range for single precision
    if prec == "d":
        rows += [[3.0, 0.0, 1.0, 3.0], [1.0, 0.0, 2.0 ** 60, 0.5], [3.0, 0.0, 1.25, 1.25],
                 [2.0 ** 1000, 0.0, 2.0 ** -1074, 2.0 ** 1000], [mu, 0.0, nu / 4, mu], [1.0, 0.0, 1.0, 2.0],
                 [1.0, 1.0, -1.0, 1.0], [1.0, 3.0, 2.0, 6.0], [1.0, 0.3, 3.0, 0.7]]
    else:
        rows += [[3.0, 0.0, 1.0, 3.0], [1.0, 0.0, 2.0 ** 30, 0.5], [3.0, 0.0, 1.25, 1.25],
                 [2.0 ** 100, 0.0, 2.0 ** -149, 2.0 ** 100], [mu, 0.0, nu / 4, mu], [1.0, 1.0, -1.0, 1.0],
                 [1.0, 3.0, 2.0, 6.0]]
    A = np.array(rows, dtype=T)            # (g11, g21, g12, g22)
    return np.ascontiguousarray(A.T)


@pytest.mark.parametrize("prec", ["d", "s"])
def test_parity_special_values_and_branches(prec):
    G = _special_cases(prec)
    got = _gpu_ge(G, prec)
    ref = oracle.gesvd2(G, prec)
    _assert_same(got, ref, "special %s" % prec)
    flags = np.bitwise_or.reduce(ref["info"][ref["info"] >= 0]) >> 8
    for name in ("ext", "fallback", "swap", "t2f2", "t2f3", "t2inf", "tpinf"):
        assert flags & oracle.FLAGS[name], name


@pytest.mark.parametrize("prec", ["d", "s"])
def test_nonfinite_inputs(prec):
    T = np.float64 if prec == "d" else np.float32
    G = np.array([[1, np.nan, 2, 3], [np.inf, 1, 1, 1], [1, 2, 3, 4], [0, 0, -np.inf, 0]], dtype=T).T.copy()
    got = _gpu_ge(G, prec)
    assert list(got["info"]) [0:2] == [-1, -1] and got["info"][2] >= 0 and got["info"][3] == -1
    assert np.isnan(got["U"][:, 0]).all() and np.isnan(got["S"][:, 3]).all()
    _assert_same(got, oracle.gesvd2(G, prec), "nonfinite")


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 127, 128, 129, 1000])
def test_small_and_ragged_batches(n):
    G = I.general(n, 4000 + n, "d", "narrow")
    _assert_same(_gpu_ge(G, "d"), oracle.gesvd2(G, "d"), "n=%d" % n)


@pytest.mark.parametrize("n", [5000, 70001])        # the fused kernel; the split FP64 path (>= 65536)
def test_strided_planes_and_optional_outputs(n):
    ld = n + 123
    G = I.general(n, 4100, "d", "narrow")
    Gt = torch.zeros((4, ld), dtype=torch.float64, device=DEV)
    Gt[:, :n] = torch.from_numpy(G).to(DEV)
    U = torch.full((4, ld + 7), 7.0, dtype=torch.float64, device=DEV)
    V = torch.full((4, ld), 7.0, dtype=torch.float64, device=DEV)
    S = torch.full((2, ld + 1), 7.0, dtype=torch.float64, device=DEV)
    k2svd = k2()
    L = k2svd.lib()
    import ctypes as C
    rc = L.k2svd_dgesvd2(n, C.c_void_p(Gt.data_ptr()), ld, C.c_void_p(U.data_ptr()), ld + 7,
                         C.c_void_p(V.data_ptr()), ld, C.c_void_p(S.data_ptr()), ld + 1, None, None, None,
                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    ref = oracle.gesvd2(G, "d")
    assert np.array_equal(_u(U[:, :n].cpu().numpy()), _u(ref["U"]))
    assert np.array_equal(_u(V[:, :n].cpu().numpy()), _u(ref["V"]))
    assert np.array_equal(_u(S[:, :n].cpu().numpy()), _u(ref["S"]))
    assert (U[:, n:] == 7.0).all() and (S[:, n:] == 7.0).all()     # nothing written past n
    # (e,f) outputs and info on strided planes too
    Se = torch.full((2, ld + 1), 7, dtype=torch.int32, device=DEV)
    Sf = torch.full((2, ld + 1), 7.0, dtype=torch.float64, device=DEV)
    info = torch.full((n + 5,), 7, dtype=torch.int32, device=DEV)
    rc = L.k2svd_dgesvd2(n, C.c_void_p(Gt.data_ptr()), ld, C.c_void_p(U.data_ptr()), ld + 7,
                         C.c_void_p(V.data_ptr()), ld, C.c_void_p(S.data_ptr()), ld + 1, C.c_void_p(Se.data_ptr()),
                         C.c_void_p(Sf.data_ptr()), C.c_void_p(info.data_ptr()),
                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert np.array_equal(Se[:, :n].cpu().numpy(), ref["Se"])
    assert np.array_equal(_u(Sf[:, :n].cpu().numpy()), _u(ref["Sf"]))
    assert np.array_equal(info[:n].cpu().numpy(), ref["info"])
    assert (info[n:] == 7).all() and (Se[:, n:] == 7).all()


def test_argument_errors():
    import ctypes as C
    L = k2().lib()
    x = torch.zeros((4, 10), dtype=torch.float64, device=DEV)
    p = C.c_void_p(x.data_ptr())
    assert L.k2svd_dgesvd2(-1, p, 10, p, 10, p, 10, p, 10, None, None, None, None) == -1
    assert L.k2svd_dgesvd2(0, None, 0, None, 0, None, 0, None, 0, None, None, None, None) == 0
    assert L.k2svd_dgesvd2(10, None, 10, p, 10, p, 10, p, 10, None, None, None, None) == -2
    assert L.k2svd_dgesvd2(10, p, 9, p, 10, p, 10, p, 10, None, None, None, None) == -3
    assert L.k2svd_dgesvd2(10, p, 10, p, 10, p, 10, p, 9, None, None, None, None) == -9
    assert L.k2svd_dtrsvd2(10, p, p, None, p, 10, p, 10, p, 10, None, None, None, None) == -4
    assert L.k2svd_strsvd2(10, p, p, p, p, 10, p, 10, p, 5, None, None, None, None) == -10


def test_deterministic_repeat():
    G = I.general(1 << 16, 4200, "d", "wide")
    a, b = _gpu_ge(G, "d"), _gpu_ge(G, "d")
    for k in a:
        assert np.array_equal(np.ascontiguousarray(a[k]).view(np.uint8), np.ascontiguousarray(b[k]).view(np.uint8))


@pytest.mark.parametrize("prec", ["d", "s"])
def test_full_size_sampled_parity(prec):
    """The benchmark's workload (wide-range, half general through gesvd2, half triangular through
    trsvd2: 2^27 + 2^27 double or 2^28 + 2^28 float matrices) generated on the device, in the
    benchmark's launch configuration, checked on a sample against the oracle on inputs
    regenerated on the host by index."""
    n = (1 << 27) if prec == "d" else (1 << 28)
    seed_g, seed_t = 0x240713116 + 2, 0x240713116 + 3
    k2svd = k2()
    G = I.general(n, seed_g, prec, "wide", xp="torch", device=DEV)
    outg = k2svd.gesvd2(G, want_ef=True)
    T3 = I.triangular(n, seed_t, prec, "wide", xp="torch", device=DEV)
    outt = k2svd.trsvd2(T3[0], T3[1], T3[2], want_ef=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.integers(0, n, 6000), np.arange(64), np.arange(n - 64, n)]))
    it = torch.from_numpy(idx).to(DEV)
    names = ("U", "V", "S", "Se", "Sf", "info")
    for out, gen, fn, tag in ((outg, lambda ix: I.general(0, seed_g, prec, "wide", idx=ix), "ge", "gesvd2"),
                              (outt, lambda ix: I.triangular(0, seed_t, prec, "wide", idx=ix), "tr", "trsvd2")):
        got = {}
        for nm, t in zip(names, out):
            got[nm] = (t[..., it] if t.dim() == 2 else t[it]).cpu().numpy()
        host = gen(idx)
        dev_in = (G if fn == "ge" else T3)[:, it].cpu().numpy()
        assert np.array_equal(_u(host), _u(dev_in))       # the generator agrees across devices
        ref = oracle.gesvd2(host, prec, nthreads=8) if fn == "ge" else \
            oracle.trsvd2(host[0], host[1], host[2], prec, nthreads=8)
        _assert_same(got, ref, "full-size %s %s" % (tag, prec))
    del G, T3, outg, outt
    torch.cuda.empty_cache()


def test_split_path_many_chunks_parity():
    """The FP64 general path on more than 2^24 matrices: many chunks of the two-launch split
    form with its state parked in the output planes, a ragged last chunk, non-finite inputs
    and all optional outputs; every matrix checked against the oracle bit for bit, and
    nothing written past the batch."""
    n = (1 << 24) + 4097
    G = I.general(n, 4300, "d", "narrow")
    rng = np.random.default_rng(11)
    bad = rng.integers(0, n, 64)
    G[rng.integers(0, 4, 64), bad] = np.where(np.arange(64) % 2 == 0, np.nan, -np.inf)
    ld = n + 3
    Gt = torch.zeros((4, ld), dtype=torch.float64, device=DEV)
    Gt[:, :n] = torch.from_numpy(G).to(DEV)
    U = torch.full((4, ld), 7.0, dtype=torch.float64, device=DEV)
    V = torch.full((4, ld), 7.0, dtype=torch.float64, device=DEV)
    S = torch.full((2, ld), 7.0, dtype=torch.float64, device=DEV)
    Se = torch.full((2, ld), 7, dtype=torch.int32, device=DEV)
    Sf = torch.full((2, ld), 7.0, dtype=torch.float64, device=DEV)
    info = torch.full((ld,), 7, dtype=torch.int32, device=DEV)
    import ctypes as C
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = k2().lib().k2svd_dgesvd2(n, p(Gt), ld, p(U), ld, p(V), ld, p(S), ld, p(Se), p(Sf), p(info),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    got = {"U": U[:, :n].cpu().numpy(), "V": V[:, :n].cpu().numpy(), "S": S[:, :n].cpu().numpy(),
           "Se": Se[:, :n].cpu().numpy(), "Sf": Sf[:, :n].cpu().numpy(), "info": info[:n].cpu().numpy()}
    ref = oracle.gesvd2(G, "d", nthreads=16)
    assert (ref["info"] == -1).sum() >= 32
    _assert_same(got, ref, "split chunks")
    for t in (U, V, S, Sf):
        assert (t[:, n:] == 7.0).all()
    assert (Se[:, n:] == 7).all() and (info[n:] == 7).all()
    del Gt, U, V, S, Se, Sf, info
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["d", "s"])
def test_svd2_host_pipeline(prec):
    """k2svd.svd2_host: matrices in pinned host memory streamed through the device in chunks
    (three streams, input and output buffers in rotation), general and triangular jobs in
    one call; every output equals the oracle's bit for bit, with the default buffer counts
    (inputs recycled after the kernels, outputs after the copies back), with one or two
    buffers, where every chunk waits for the buffers of the one before, and on streams the
    caller passes."""
    k2svd = k2()
    dt = torch.float64 if prec == "d" else torch.float32
    nc, c = 5, 70001                          # above the split path's threshold, not a power of two
    G = I.general(nc * c, 4400, prec, "wide")
    T3 = I.triangular(nc * c, 4401, prec, "wide")
    Gh = torch.from_numpy(np.ascontiguousarray(G.reshape(4, nc, c).transpose(1, 0, 2))).pin_memory()
    Th = torch.from_numpy(np.ascontiguousarray(T3.reshape(3, nc, c).transpose(1, 0, 2))).pin_memory()
    Og = torch.full((nc, 10, c), 7.0, dtype=dt).pin_memory()
    Ot = torch.full((nc, 10, c), 7.0, dtype=dt).pin_memory()
    refg = oracle.gesvd2(G, prec, nthreads=8)
    reft = oracle.trsvd2(T3[0], T3[1], T3[2], prec, nthreads=8)
    own = tuple(torch.cuda.Stream() for _ in range(3))
    for kw in ({}, {"depth": 1, "in_depth": 2}, {"depth": 2, "in_depth": 1}, {"streams": own}):
        Og.fill_(7.0)
        Ot.fill_(7.0)
        k2svd.svd2_host([(Gh, Og, False), (Th, Ot, True)], **kw)
        for O, ref in ((Og, refg), (Ot, reft)):
            got = O.numpy().transpose(1, 0, 2).reshape(10, nc * c)
            assert np.array_equal(_u(got[0:4]), _u(ref["U"])), kw
            assert np.array_equal(_u(got[4:8]), _u(ref["V"])), kw
            assert np.array_equal(_u(got[8:10]), _u(ref["S"])), kw
