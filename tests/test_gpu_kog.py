"""GPU parity of the batched n x n Kogbetliantz driver (k2svd_{d,s}kogbet) and its sigma
gradient against the oracle.  The off-norm is summed in a fixed order and every rotation
has one fixed fma form, so the persistent, graph and per-step forms must all reproduce the
oracle bit for bit (U, S, V, sweep counts, info)."""
import threading

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


def _batch(orders, seed, prec, smin=1e-12):
    T = np.float64 if prec == "d" else np.float32
    mats = [I.kog_matrix(int(n), seed, i, smin=smin)[0].astype(T) for i, n in enumerate(orders)]
    flat = np.concatenate([m.T.reshape(-1) for m in mats])      # column-major per matrix
    return flat, mats


def _gpu(flat, orders, flags=0, max_sweeps=40):
    A = torch.from_numpy(np.ascontiguousarray(flat)).to(DEV)
    U, S, V, sw, info = k2().kogbet(A, list(orders), max_sweeps=max_sweeps, flags=flags)
    torch.cuda.synchronize()
    return U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), sw.cpu().numpy(), info.cpu().numpy()


def _oracle(mats, prec, max_sweeps=40, dynamic=False):
    U, S, V, sw, info = [], [], [], [], []
    for m in mats:
        u, s, v, a, b = oracle.kogbet(m, prec, max_sweeps=max_sweeps, dynamic=dynamic)
        U.append(u.T.reshape(-1)); V.append(v.T.reshape(-1)); S.append(s); sw.append(a); info.append(b)
    return np.concatenate(U), np.concatenate(S), np.concatenate(V), np.array(sw), np.array(info)


def _bits(x):
    x = np.ascontiguousarray(x)
    return x.view({8: np.uint64, 4: np.uint32}[x.dtype.itemsize])


def _same(a, b, tag):
    for k, (x, y) in enumerate(zip(a, b)):
        x, y = np.asarray(x), np.asarray(y)
        if x.dtype.kind == "f":
            nan = np.isnan(x) & np.isnan(y)
            bad = (_bits(x) != _bits(y)) & ~nan
        else:
            bad = x != y
        assert not bad.any(), "%s: output %d differs at %d places (first %d)" % (tag, k, bad.sum(), np.flatnonzero(bad)[0])


ORDERS_D = [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 31, 32, 33, 48, 63, 64, 65, 100, 127, 128, 129, 150]
ORDERS_S = [1, 2, 3, 5, 8, 17, 32, 33, 64, 65, 127, 128, 129, 200, 224, 225, 240]


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("flags", [0, 2, 1, 4])
def test_parity_all_buckets_and_forms(prec, flags):
    orders = ORDERS_D if prec == "d" else ORDERS_S
    flat, mats = _batch(orders, 11 + flags, prec, smin=1e-12 if prec == "d" else 1e-5)
    got = _gpu(flat, orders, flags)
    ref = _oracle(mats, prec)
    _same(got, ref, "kogbet %s flags=%d" % (prec, flags))
    assert (got[4] == 0).all()


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("flags", [8, 8 | 2, 8 | 4])
def test_dynamic_ordering_parity(prec, flags):
    """The dynamic ordering (K2SVD_KOG_DYNAMIC) in every bucket, plain persistent, graph and
    untuned, bit for bit against the oracle's dynamic ordering."""
    orders = ORDERS_D if prec == "d" else ORDERS_S
    flat, mats = _batch(orders, 41 + flags, prec, smin=1e-12 if prec == "d" else 1e-5)
    got = _gpu(flat, orders, flags)
    ref = _oracle(mats, prec, dynamic=True)
    _same(got, ref, "kogbet dynamic %s flags=%d" % (prec, flags))
    assert (got[4] == 0).all()


def test_dynamic_ordering_max_sweeps_and_errors():
    orders = [40, 9, 128]
    flat, mats = _batch(orders, 51, "d")
    got = _gpu(flat, orders, 8, max_sweeps=2)
    ref = _oracle(mats, "d", max_sweeps=2, dynamic=True)
    _same(got, ref, "dynamic max_sweeps=2")
    assert (got[3] == 2).all() and (got[4] == 1).all()
    A = torch.from_numpy(flat).to(DEV)
    with pytest.raises(k2().K2SVDError, match="-13"):
        k2().kogbet(A, orders, flags=8 | 1)


@pytest.mark.parametrize("flags", [0, 2])
def test_concurrent_buckets_keep_the_callers_stream_order(flags):
    """The order buckets run concurrently on library streams forked from the caller's stream
    and joined back to it.  Work queued on the caller's stream before the call (a delay, then
    the copy that fills A and the zeroing of the outputs) must be done before any bucket
    starts, and work queued after it (copies of the outputs) must see every bucket's
    results; persistent and graph form, twice each (the second graph call replays)."""
    k = k2()
    orders = [12, 40, 70, 100, 128, 33, 90, 56]
    flat, mats = _batch(orders, 61, "d")
    ref = _oracle(mats, "d")
    src = torch.from_numpy(flat).to(DEV)
    side = torch.cuda.Stream(device=DEV)
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        A = torch.zeros_like(src)
        U, S, V, sw, info = k.kogbet(A, orders, flags=flags)          # tunes on zero matrices
        ws = k.kogbet_workspace(orders, torch.float64, flags, torch.device(DEV))
        for _ in range(2):
            A.zero_()
            torch.cuda._sleep(50_000_000)
            A.copy_(src)
            for t in (U, S, V, sw, info):
                t.zero_()
            k.kogbet(A, orders, flags=flags, workspace=ws, U=U, V=V, S=S, sweeps=sw, info=info)
            got = [t.clone() for t in (U, S, V, sw, info)]
            torch.cuda.synchronize()
            _same([t.cpu().numpy() for t in got], ref, "side stream flags=%d" % flags)


def test_two_host_threads_share_the_bucket_streams():
    """Two host threads call the driver at once, each on a stream of its own: one in the graph
    form with a new argument set every call (so every call captures a new graph, during
    which the library's bucket streams belong to that capture), the other in the direct
    persistent form on the same bucket streams.  Every result equals the oracle's."""
    k = k2()
    orders = [12, 40, 70, 100, 128, 33]
    flat, mats = _batch(orders, 81, "d")
    ref = _oracle(mats, "d")
    src = torch.from_numpy(flat).to(DEV)
    k.kogbet(src.clone(), orders)                      # tunes the block sizes first
    torch.cuda.synchronize()
    errors, results = [], {0: [], 1: []}

    def worker(tid, flags):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream(device=DEV)
            with torch.cuda.stream(s):
                for _ in range(4):
                    results[tid].append(k.kogbet(src.clone(), orders, flags=flags))
            s.synchronize()
        except Exception as e:                         # reported below, in the test's thread
            errors.append(repr(e))

    ts = [threading.Thread(target=worker, args=(0, 2)), threading.Thread(target=worker, args=(1, 0))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for tid in (0, 1):
        assert len(results[tid]) == 4
        for r in results[tid]:
            _same([t.cpu().numpy() for t in r], ref, "thread %d" % tid)


def test_graph_replay_and_reuse():
    orders = [40, 8, 70, 33, 128, 5]
    flat, mats = _batch(orders, 21, "d")
    a = _gpu(flat, orders, 2)
    b = _gpu(flat, orders, 2)            # cached graph
    _same(a, b, "graph replay")
    _same(a, _oracle(mats, "d"), "graph vs oracle")


def test_max_sweeps_and_info():
    orders = [16, 40, 3]
    flat, mats = _batch(orders, 31, "d")
    for ms in (0, 1, 2):
        got = _gpu(flat, orders, 0, max_sweeps=ms)
        ref = _oracle(mats, "d", max_sweeps=ms)
        _same(got, ref, "max_sweeps=%d" % ms)
    got = _gpu(flat, orders, 0, max_sweeps=1)
    assert got[4][0] == 1 and got[3][0] == 1


def test_nonfinite_matrix_isolated():
    orders = [6, 6, 6]
    flat, mats = _batch(orders, 41, "d")
    flat[36 + 7] = np.nan
    mats[1] = mats[1].copy()
    mats[1][1, 1] = np.nan
    got = _gpu(flat, orders, 0)
    assert list(got[4]) == [0, -1, 0]
    assert np.isnan(got[1][6:12]).all()
    _same(got, _oracle(mats, "d"), "nonfinite")


def test_zero_and_diagonal_matrices():
    orders = [4, 5]
    flat = np.concatenate([np.zeros(16), np.diag([3.0, -5.0, 0.5, 2.0, -0.25]).T.reshape(-1)])
    mats = [np.zeros((4, 4)), np.diag([3.0, -5.0, 0.5, 2.0, -0.25])]
    got = _gpu(flat, orders, 0)
    _same(got, _oracle(mats, "d"), "zero/diagonal")
    assert np.array_equal(got[1][4:], [5.0, 3.0, 2.0, 0.5, 0.25])


def test_workspace_and_argument_errors():
    import ctypes as C
    k2svd = k2()
    L = k2svd.lib()
    orders = [8, 9]
    n, offs, soffs, tot, stot = k2svd.kog_layout(orders)
    A = torch.zeros(tot, dtype=torch.float64, device=DEV)
    p = C.c_void_p(A.data_ptr())
    size = C.c_size_t(0)
    assert L.k2svd_dkogbet_ws(2, n.ctypes.data, 0, C.byref(size)) == 0 and size.value > 0
    ws = torch.empty(size.value + 512, dtype=torch.uint8, device=DEV)
    w = C.c_void_p(ws.data_ptr())
    args = lambda **kw: [kw.get("batch", 2), n.ctypes.data, offs.ctypes.data, soffs.ctypes.data, p, p, p, p, None, None,
                         kw.get("ms", 10), kw.get("tol", 1.0), kw.get("flags", 0), kw.get("ws", w),
                         kw.get("wsb", size.value), None]
    assert L.k2svd_dkogbet(*args(batch=-1)) == -1
    assert L.k2svd_dkogbet(*args(ms=-1)) == -11
    assert L.k2svd_dkogbet(*args(tol=0.0)) == -12
    assert L.k2svd_dkogbet(*args(flags=3)) == -13
    assert L.k2svd_dkogbet(*args(ws=C.c_void_p(ws.data_ptr() + 8))) == -14
    assert L.k2svd_dkogbet(*args(wsb=size.value - 1)) == -15
    bad = np.array([8, 0], dtype=np.int32)
    assert L.k2svd_dkogbet_ws(2, bad.ctypes.data, 0, C.byref(size)) == -2


@pytest.mark.parametrize("prec", ["d", "s"])
def test_sigma_gradient_parity(prec):
    orders = [8, 33, 64, 100] if prec == "d" else [8, 33, 64, 150]
    flat, mats = _batch(orders, 51, prec, smin=1e-3)
    got = _gpu(flat, orders)
    U, V = torch.from_numpy(got[0]).to(DEV), torch.from_numpy(got[2]).to(DEV)
    T = np.float64 if prec == "d" else np.float32
    dS = np.linspace(-1, 1, sum(orders)).astype(T)
    dA = k2().kog_sigma_bwd(U, V, torch.from_numpy(dS).to(DEV), orders).cpu().numpy()
    o = so = 0
    for n in orders:
        u = got[0][o:o + n * n].reshape(n, n).T
        v = got[2][o:o + n * n].reshape(n, n).T
        ref = oracle.kog_sigma_bwd(u, v, dS[so:so + n], prec)
        assert np.array_equal(_bits(dA[o:o + n * n]), _bits(ref.T.reshape(-1)))
        o += n * n
        so += n


def test_autograd_sigma():
    from paper_2407_13116_gb300.autograd import kogbet_sigma
    orders = [12, 20]
    flat, mats = _batch(orders, 61, "d", smin=0.1)
    A = torch.from_numpy(flat).to(DEV).requires_grad_(True)
    U, S, V, sw, info = kogbet_sigma(A, orders)
    w = torch.linspace(-1, 1, S.numel(), dtype=torch.float64, device=DEV)
    (g,) = torch.autograd.grad((S * w).sum(), A)
    ref = k2().kog_sigma_bwd(U, V, w, orders)
    assert torch.equal(g, ref)
    # central differences on two elements
    h = 1e-7
    for e in (3, 150 + 21):
        Ap, Am = A.detach().clone(), A.detach().clone()
        Ap[e] += h
        Am[e] -= h
        fp = (k2().kogbet(Ap, orders)[1] * w).sum().item()
        fm = (k2().kogbet(Am, orders)[1] * w).sum().item()
        assert abs((fp - fm) / (2 * h) - g[e].item()) <= 1e-7


def test_config4_sampled_and_forms_agree():
    """The batched Kogbetliantz workload: 8192 FP64 matrices of order uniform in {8..128}, run
    through the persistent graph form; 24 sampled matrices (the largest, the smallest, random)
    are compared with the oracle bit for bit, and a 512-matrix slice with the per-step form."""
    orders = I.kog_orders(8192, 8, 128, 0x240713116 + 4)
    flat, sig = I.kog_batch(orders, 0x240713116 + 4)
    got = _gpu(flat, orders, 2)
    assert (got[4] == 0).all()
    offs = np.concatenate([[0], np.cumsum(orders.astype(np.int64) ** 2)[:-1]])
    soffs = np.concatenate([[0], np.cumsum(orders.astype(np.int64))[:-1]])
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([[int(np.argmax(orders)), int(np.argmin(orders))], rng.integers(0, 8192, 22)]))
    for i in pick:
        n = int(orders[i])
        A = flat[offs[i]:offs[i] + n * n].reshape(n, n).T
        u, s, v, a, b = oracle.kogbet(A)
        assert np.array_equal(_bits(got[1][soffs[i]:soffs[i] + n]), _bits(s))
        assert np.array_equal(_bits(got[0][offs[i]:offs[i] + n * n]), _bits(u.T.reshape(-1)))
        assert np.array_equal(_bits(got[2][offs[i]:offs[i] + n * n]), _bits(v.T.reshape(-1)))
        assert got[3][i] == a
        # the construction's singular values, to the backward-error bound
        assert np.abs(s - sig[i]).max() <= 8 * n * 2.0 ** -52 * sig[i][0]
    sl = orders[:512]
    end = int(offs[512])
    plain = _gpu(flat[:end], sl, 1)
    _same(plain, tuple(x[:end] if k in (0, 2) else (x[:int(soffs[512])] if k == 1 else x[:512])
                       for k, x in enumerate(got)), "plain vs persistent")


def test_config5_gradients():
    """Batched Kogbetliantz with gradients: 2048 FP64 matrices of order uniform in {32..256}
    and 4096 FP32 matrices of order uniform in {8..128} (built as the batched workload),
    sigma backpropagated to A (dA = U diag(dsigma) V^T) through the autograd function with
    the tuned block sizes.  Sampled matrices match the oracle bit for bit (U, S, V and the
    gradient); central differences on 64 FP64 matrices, all perturbed at once (the matrices
    are independent), agree with the gradient."""
    from paper_2407_13116_gb300.autograd import kogbet_sigma
    seed = 0x240713116 + 5
    for prec, count, lo, hi in (("d", 2048, 32, 256), ("s", 4096, 8, 128)):
        T = np.float64 if prec == "d" else np.float32
        orders = I.kog_orders(count, lo, hi, seed + (prec == "s"))
        flat, sig = I.kog_batch(orders, seed + (prec == "s"), dtype=T)
        A = torch.from_numpy(flat).to(DEV).requires_grad_(True)
        U, S, V, sw, info = kogbet_sigma(A, list(orders))
        assert bool((info == 0).all())
        w = torch.from_numpy(np.cos(np.arange(S.numel()) * 0.37).astype(T)).to(DEV)
        (g,) = torch.autograd.grad((S * w).sum(), A, retain_graph=True)
        Un, Sn, Vn, gn, wn = (x.detach().cpu().numpy() for x in (U, S, V, g, w))
        offs = np.concatenate([[0], np.cumsum(orders.astype(np.int64) ** 2)[:-1]])
        soffs = np.concatenate([[0], np.cumsum(orders.astype(np.int64))[:-1]])
        pick = [int(np.argmax(orders)), int(np.argmin(orders))] + list(np.random.default_rng(5).integers(0, count, 3))
        for i in pick:
            n = int(orders[i])
            a = flat[offs[i]:offs[i] + n * n].reshape(n, n).T
            u, s, v, _, _ = oracle.kogbet(a, prec)
            assert np.array_equal(_bits(Sn[soffs[i]:soffs[i] + n]), _bits(s))
            assert np.array_equal(_bits(Un[offs[i]:offs[i] + n * n]), _bits(u.T.reshape(-1)))
            assert np.array_equal(_bits(Vn[offs[i]:offs[i] + n * n]), _bits(v.T.reshape(-1)))
            ref = oracle.kog_sigma_bwd(u, v, wn[soffs[i]:soffs[i] + n], prec)
            assert np.array_equal(_bits(gn[offs[i]:offs[i] + n * n]), _bits(ref.T.reshape(-1)))
        if prec != "d":
            continue
        # central differences: loss sum_k c_k sigma_k over the four largest singular values of
        # each of 64 matrices whose top five are separated by more than 1e-2 relative
        h = 1e-6
        cand = [i for i in range(count) if np.all(-np.diff(sig[i][:5]) > 1e-2 * sig[i][0])][:64]
        assert len(cand) == 64
        sel = [int(i) for i in cand]
        so = [list(range(int(soffs[i]), int(soffs[i]) + 4)) for i in sel]
        c = np.array([1.0, -0.7, 0.4, 0.25])
        dAp, dAm = flat.copy(), flat.copy()
        rng = np.random.default_rng(9)
        pos = []
        for i in sel:
            n = int(orders[i])
            e = int(offs[i]) + int(rng.integers(0, n * n))
            pos.append(e)
            dAp[e] += h
            dAm[e] -= h
        Sp = k2().kogbet(torch.from_numpy(dAp).to(DEV), list(orders))[1].cpu().numpy()
        Sm = k2().kogbet(torch.from_numpy(dAm).to(DEV), list(orders))[1].cpu().numpy()
        wt = torch.zeros_like(S)
        for idx in so:
            wt[idx] = torch.from_numpy(c).to(DEV)
        (g4,) = torch.autograd.grad((S * wt).sum(), A)
        g4 = g4.cpu().numpy()
        for i, e, idx in zip(sel, pos, so):
            fd = float(((Sp[idx] - Sm[idx]) * c).sum()) / (2 * h)
            assert abs(fd - g4[e]) <= 1e-6 * max(1.0, abs(g4[e])), (i, e, fd, g4[e])
