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
