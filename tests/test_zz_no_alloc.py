"""k2svd_dkogbet_noalloc: the batched Kogbetliantz SVD for callers that cannot allocate
device memory (its scratch is a fixed device array of the library), called through the C
ABI and checked against k2svd_dkogbet with a caller-supplied workspace.  The n x n driver
is bitwise reproducible, so the two must agree bit for bit -- on two calls in a row, since
the second call finds the array holding the first call's contents."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2407_13116_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
K2SVD_ENOSPACE = -1001


def _lib():
    from paper_2407_13116_gb300 import k2svd
    L = k2svd.lib()
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.k2svd_dkogbet_noalloc.argtypes = [I64, P, P, P, P, P, P, P, P, P, I32, D, P]
    L.k2svd_dkogbet_noalloc.restype = C.c_int
    return k2svd, L


def _bits(t):
    return t.cpu().numpy().view(np.uint64)


def test_noalloc_matches_workspace_entry_twice():
    k2svd, L = _lib()
    torch.cuda.set_device(0)
    orders = [8, 33, 64, 100, 128, 5, 140, 17]         # 140 uses the scratch copy of G
    mats = [I.kog_matrix(n, 71, i)[0] for i, n in enumerate(orders)]
    A = torch.from_numpy(np.concatenate([m.T.reshape(-1) for m in mats])).to(DEV)
    n, offs, soffs, tot, stot = k2svd.kog_layout(orders)
    ref = k2svd.kogbet(A, orders, max_sweeps=40, flags=0)
    torch.cuda.synchronize()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        U = torch.full((tot,), 7.0, dtype=torch.float64, device=DEV)
        V = torch.full_like(U, 7.0)
        S = torch.full((stot,), 7.0, dtype=torch.float64, device=DEV)
        sw = torch.full((len(orders),), -7, dtype=torch.int32, device=DEV)
        info = torch.full_like(sw, -7)
        rc = L.k2svd_dkogbet_noalloc(len(orders), n.ctypes.data, offs.ctypes.data, soffs.ctypes.data,
                                     C.c_void_p(A.data_ptr()), C.c_void_p(U.data_ptr()), C.c_void_p(V.data_ptr()),
                                     C.c_void_p(S.data_ptr()), C.c_void_p(sw.data_ptr()), C.c_void_p(info.data_ptr()),
                                     40, 1.0, stream)
        assert rc == 0, rc
        torch.cuda.synchronize()
        assert np.array_equal(_bits(U), _bits(ref[0])), "U differs on call %d" % call
        assert np.array_equal(_bits(S), _bits(ref[1])), "S differs on call %d" % call
        assert np.array_equal(_bits(V), _bits(ref[2])), "V differs on call %d" % call
        assert torch.equal(sw, ref[3]) and torch.equal(info, ref[4])


def test_noalloc_rejects_problems_beyond_its_scratch():
    k2svd, L = _lib()
    orders = [400]                                     # 400^2 * 8 bytes of G > 1 MiB
    n, offs, soffs, tot, stot = k2svd.kog_layout(orders)
    A = torch.zeros(tot, dtype=torch.float64, device=DEV)
    p = C.c_void_p(A.data_ptr())
    rc = L.k2svd_dkogbet_noalloc(1, n.ctypes.data, offs.ctypes.data, soffs.ctypes.data, p, p, p, p, None, None,
                                 10, 1.0, None)
    assert rc == K2SVD_ENOSPACE
    assert L.k2svd_dkogbet_noalloc(-1, n.ctypes.data, offs.ctypes.data, soffs.ctypes.data, p, p, p, p, None, None,
                                   10, 1.0, None) == -1


K2SVD_ECAPTURE = -1002


def _run_noalloc(L, k2svd, orders, A, stream=None):
    n, offs, soffs, tot, stot = k2svd.kog_layout(orders)
    U = torch.full((tot,), 7.0, dtype=torch.float64, device=DEV)
    V = torch.full_like(U, 7.0)
    S = torch.full((stot,), 7.0, dtype=torch.float64, device=DEV)
    sw = torch.full((len(orders),), -7, dtype=torch.int32, device=DEV)
    info = torch.full_like(sw, -7)
    rc = L.k2svd_dkogbet_noalloc(len(orders), n.ctypes.data, offs.ctypes.data, soffs.ctypes.data,
                                 C.c_void_p(A.data_ptr()), C.c_void_p(U.data_ptr()), C.c_void_p(V.data_ptr()),
                                 C.c_void_p(S.data_ptr()), C.c_void_p(sw.data_ptr()), C.c_void_p(info.data_ptr()),
                                 40, 1.0, stream)
    return rc, (U, S, V, sw, info)


def _batch(orders, seed):
    mats = [I.kog_matrix(n, seed, i)[0] for i, n in enumerate(orders)]
    return torch.from_numpy(np.concatenate([m.T.reshape(-1) for m in mats])).to(DEV)


def _same_as_workspace_entry(k2svd, A, orders, got):
    ref = k2svd.kogbet(A, orders, max_sweeps=40, flags=0)
    torch.cuda.synchronize()
    for g, r, nm in zip(got, ref, ("U", "S", "V", "sweeps", "info")):
        if g.dtype == torch.float64:
            assert np.array_equal(_bits(g), _bits(r)), nm
        else:
            assert torch.equal(g, r), nm


def test_noalloc_limit_on_batch_size():
    """The descriptor part of the scratch: 32752 matrices of order <= 128 fit (512 + 32 * 32752
    bytes = 1 MiB), one more does not."""
    k2svd, L = _lib()
    orders = [2] * 32752
    A = _batch(orders[:1], 5).repeat(32752)
    rc, got = _run_noalloc(L, k2svd, orders, A)
    assert rc == 0, rc
    torch.cuda.synchronize()
    _same_as_workspace_entry(k2svd, A, orders, got)
    orders1 = [2] * 32753
    A1 = torch.cat([A, A[:4]])
    rc, _ = _run_noalloc(L, k2svd, orders1, A1)
    assert rc == K2SVD_ENOSPACE, rc


def test_noalloc_limit_with_orders_above_128():
    """Orders above 128 keep G in the scratch: 8 matrices with orders 144 and 332 fill the
    array to exactly 1 MiB (512 + 256 + 8 * (144^2 + 332^2) rounded up to 256 bytes) and run;
    a ninth matrix of order 2 brings the descriptor part to 512 bytes, 256 bytes over."""
    k2svd, L = _lib()
    orders = [144, 332] + [2] * 6
    A = _batch(orders, 17)
    rc, got = _run_noalloc(L, k2svd, orders, A)
    assert rc == 0, rc
    torch.cuda.synchronize()
    _same_as_workspace_entry(k2svd, A, orders, got)
    orders9 = orders + [2]
    A9 = torch.cat([A, A[-4:]])
    rc, _ = _run_noalloc(L, k2svd, orders9, A9)
    assert rc == K2SVD_ENOSPACE, rc


def test_noalloc_and_workspace_entry_refuse_stream_capture():
    """A captured call would copy its descriptor table from host memory at replay time, when
    another call may have overwritten it (or it is freed): both n x n entries refuse a stream
    that is being captured and leave the capture intact."""
    k2svd, L = _lib()
    orders = [8, 12]
    A = _batch(orders, 23)
    n, offs, soffs, tot, stot = k2svd.kog_layout(orders)
    ws = k2svd.kogbet_workspace(orders, torch.float64, 0, A.device)
    out = torch.empty(tot, dtype=torch.float64, device=DEV)
    x = torch.zeros(16, device=DEV)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    rcs = []
    with torch.cuda.graph(g, stream=s):
        x.add_(1)
        st = C.c_void_p(s.cuda_stream)
        rcs.append(_run_noalloc(L, k2svd, orders, A, st)[0])
        p = C.c_void_p(out.data_ptr())
        rcs.append(k2svd.lib().k2svd_dkogbet(len(orders), n.ctypes.data, offs.ctypes.data, soffs.ctypes.data,
                                             C.c_void_p(A.data_ptr()), p, p, p, None, None, 40, 1.0, 0,
                                             C.c_void_p(ws.data_ptr()), ws.numel(), st))
    g.replay()
    torch.cuda.synchronize()
    assert rcs == [K2SVD_ECAPTURE, K2SVD_ECAPTURE], rcs
    assert float(x[0]) == 1.0                       # the capture and its replay still work
    rc, got = _run_noalloc(L, k2svd, orders, A)     # and so does the entry afterwards
    assert rc == 0
    torch.cuda.synchronize()
    _same_as_workspace_entry(k2svd, A, orders, got)
