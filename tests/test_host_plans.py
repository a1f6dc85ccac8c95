"""Host-side planning of the n x n driver, checked on the CPU through the workspace queries
k2svd_{d,s}kogbet_ws (they only plan: no device work): the dynamic ordering's extra
workspace (n(n-1)/2 pair weights per matrix, after the G scratch of the matrices kept in
global memory) and the argument checks."""
import ctypes as C

import numpy as np
import pytest

KOG_PLAIN, KOG_GRAPH, KOG_NOTUNE, KOG_DYNAMIC = 1, 2, 4, 8
SMEM_MAX = {"d": 128, "s": 224}


def _lib():
    from paper_2407_13116_gb300 import build
    L = C.CDLL(build.build())
    for p in ("d", "s"):
        f = getattr(L, "k2svd_%skogbet_ws" % p)
        f.argtypes = [C.c_int64, C.c_void_p, C.c_int32, C.POINTER(C.c_size_t)]
        f.restype = C.c_int
    return L


def _ws(L, p, orders, flags):
    n = np.ascontiguousarray(orders, np.int32)
    out = C.c_size_t(0)
    rc = getattr(L, "k2svd_%skogbet_ws" % p)(len(n), n.ctypes.data if len(n) else None, flags, C.byref(out))
    return rc, out.value


def _align(x):
    return (x + 255) & ~255


@pytest.mark.parametrize("p", ["d", "s"])
def test_dynamic_ordering_workspace(p):
    L = _lib()
    size = 8 if p == "d" else 4
    rng = np.random.default_rng(1)
    orders = [int(x) for x in rng.integers(1, 300, 60)] + [1, 2, SMEM_MAX[p], SMEM_MAX[p] + 1]
    rc0, ws0 = _ws(L, p, orders, 0)
    rc1, ws1 = _ws(L, p, orders, KOG_DYNAMIC)
    assert rc0 == 0 and rc1 == 0
    g0 = sum((n * n + 1) & ~1 for n in orders if n > SMEM_MAX[p])
    w = sum((n * (n - 1) // 2 + 1) & ~1 for n in orders)
    assert ws1 - ws0 == _align((g0 + w) * size) - _align(g0 * size)
    # graph and tuning flags do not change the plan
    assert _ws(L, p, orders, KOG_DYNAMIC | KOG_GRAPH | KOG_NOTUNE) == (0, ws1)
    # the per-step form keeps every G in the workspace
    rcp, wsp = _ws(L, p, orders, KOG_PLAIN)
    assert rcp == 0 and wsp > ws0


def test_workspace_query_argument_checks():
    L = _lib()
    out = C.c_size_t(0)
    n = np.array([4, 5], np.int32)
    f = L.k2svd_dkogbet_ws
    assert f(-1, n.ctypes.data, 0, C.byref(out)) == -1
    assert f(2, None, 0, C.byref(out)) == -2
    assert f(2, n.ctypes.data, 0, None) == -4
    assert f(1, np.array([0], np.int32).ctypes.data, 0, C.byref(out)) == -2
    assert f(1, np.array([4097], np.int32).ctypes.data, 0, C.byref(out)) == -2
    assert f(0, None, 0, C.byref(out)) == 0
