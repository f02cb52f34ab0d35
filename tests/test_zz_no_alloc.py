"""The allocation-free correlation integral (cil_features_static) against the
regular entry point (cil_features), called directly through the C ABI.

Callers such as a sampler that must not trigger a device-wide
synchronisation, or a host application that owns all device memory, cannot
hand the library a workspace; this entry point keeps its scratch in a
static device array instead.  It must give the same bins, counts, radii and
correlation vector (bit-exact, as every CIL result is) on consecutive calls,
because the shared array keeps the previous call's contents.  Collected last
on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as p
    L = p.lib()
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.cil_features_static.restype = i32
    L.cil_features_static.argtypes = [vp, i64, i64, vp, i64, i64, i64, vp, dbl, i32, vp, vp, vp, vp, vp, vp]
    return L


def outputs(n1, n2, M):
    dev = torch.device("cuda")
    return {"radii": torch.empty(M + 1, dtype=torch.float64, device=dev),
            "bins": torch.empty((n1, n2), dtype=torch.uint8, device=dev),
            "counts": torch.empty(M, dtype=torch.int64, device=dev),
            "C": torch.empty(M, dtype=torch.float64, device=dev),
            "nre": torch.empty(1, dtype=torch.int64, device=dev)}


def call(L, fn, X1, X2, b, M, work=None):
    n1, d = X1.shape
    n2 = X2.shape[0]
    o = outputs(n1, n2, M)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = [ptr(X1), d, n1, ptr(X2), d, n2, d, None, b, M, ptr(o["radii"]), ptr(o["bins"]),
            ptr(o["counts"]), ptr(o["C"]), ptr(o["nre"])]
    if fn == "cil_features":
        args += [ptr(work), work.numel()]
    args.append(stream)
    assert getattr(L, fn)(*args) == 0
    torch.cuda.synchronize()
    return o


def test_static_scratch_matches_workspace_path_twice(lib):
    M, b = 16, 1.1
    sets = [(W.clustered_patterns(64, 4096, 31), W.clustered_patterns(64, 4096, 32)),
            (W.clustered_patterns(100, 3001, 33), W.clustered_patterns(77, 3001, 34))]
    for X1n, X2n in sets:                      # two calls in a row, different shapes
        X1 = torch.from_numpy(X1n).cuda()
        X2 = torch.from_numpy(X2n).cuda()
        sz = C.c_size_t()
        assert lib.cil_workspace_size(X1.shape[0], X2.shape[0], X1.shape[1], C.byref(sz)) == 0
        work = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
        ref = call(lib, "cil_features", X1, X2, b, M, work)
        got = call(lib, "cil_features_static", X1, X2, b, M)
        for k in ("radii", "bins", "counts", "C"):
            assert torch.equal(got[k], ref[k]), k
        assert int(got["nre"]) >= 0


def test_static_limits_rejected(lib):
    X = torch.zeros((129, 16), dtype=torch.float32, device="cuda")
    o = outputs(129, 129, 4)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    rc = lib.cil_features_static(ptr(X), 16, 129, ptr(X), 16, 129, 16, None, 1.2, 4, ptr(o["radii"]),
                                 ptr(o["bins"]), ptr(o["counts"]), ptr(o["C"]), None, None)
    assert rc == 1
