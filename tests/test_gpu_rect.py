"""GPU parity of the rectangular SVD (k2svd_?gesvdr: QR with column pivoting to a square
matrix, then the n x n Kogbetliantz driver; Sect. 1) against the oracle, bit for bit: tall,
wide, square, single-row and single-column matrices of uneven shapes in one batch, zero and
non-finite matrices, both precisions."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def k2():
    from paper_2407_13116_gb300 import k2svd
    return k2svd


def _bits(x):
    x = np.ascontiguousarray(x)
    return x.view({8: np.uint64, 4: np.uint32}[x.dtype.itemsize])


SHAPES = [(10, 4), (4, 10), (7, 7), (1, 5), (5, 1), (1, 1), (60, 33), (33, 60), (96, 17), (130, 129),
          (200, 40), (3, 150), (64, 64), (2, 2), (300, 5)]


@pytest.mark.parametrize("prec", ["d", "s"])
def test_parity_uneven_shapes(prec):
    T = np.float64 if prec == "d" else np.float32
    rng = np.random.default_rng(71)
    mats = []
    for (m, n) in SHAPES:
        A = (rng.standard_normal((m, n)) * 2.0 ** rng.integers(-30, 30)).astype(T)
        mats.append(A)
    mats.append(np.zeros((6, 4), T))
    bad = np.ones((5, 3), T); bad[2, 1] = np.nan
    mats.append(bad)
    shapes = [a.shape for a in mats]
    flat = np.concatenate([a.reshape(-1, order="F") for a in mats])
    U, S, V, sw, info = k2().gesvdr(torch.from_numpy(flat).to(DEV), shapes)
    U, S, V, sw, info = (x.cpu().numpy() for x in (U, S, V, sw, info))
    m_, n_, ao, uo, vo, so, _ = k2().rect_layout(shapes)
    for i, A in enumerate(mats):
        m, n = A.shape
        k = min(m, n)
        rU, rS, rV, rsw, rinfo = oracle.gesvdr(A, prec)
        gU = U[uo[i]:uo[i] + m * k].reshape(k, m).T
        gV = V[vo[i]:vo[i] + n * k].reshape(k, n).T
        gS = S[so[i]:so[i] + k]
        assert info[i] == rinfo and sw[i] == rsw, (i, A.shape, info[i], rinfo, sw[i], rsw)
        if rinfo < 0:
            assert np.isnan(gS).all() and np.isnan(gU).all() and np.isnan(gV).all()
            continue
        assert np.array_equal(_bits(gS), _bits(rS)), (i, A.shape)
        assert np.array_equal(_bits(gU), _bits(rU)), (i, A.shape)
        assert np.array_equal(_bits(gV), _bits(rV)), (i, A.shape)


def test_errors():
    L = k2().lib()
    m = np.array([4], np.int32); n = np.array([3], np.int32); o = np.zeros(1, np.int64)
    import ctypes as C
    wsb = C.c_size_t(0)
    assert L.k2svd_dgesvdr_ws(1, m.ctypes.data, n.ctypes.data, 0, C.byref(wsb)) == 0 and wsb.value > 0
    bad = np.array([0], np.int32)
    assert L.k2svd_dgesvdr_ws(1, bad.ctypes.data, n.ctypes.data, 0, C.byref(wsb)) == -2
    t = torch.zeros(64, dtype=torch.float64, device=DEV)
    p = t.data_ptr()
    r = L.k2svd_dgesvdr(1, m.ctypes.data, n.ctypes.data, o.ctypes.data, o.ctypes.data, o.ctypes.data,
                        o.ctypes.data, p, p, p, p, None, None, 10, 1.0, 0, None, 0, None)
    assert r == -17
