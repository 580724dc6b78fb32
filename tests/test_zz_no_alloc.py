"""gp_query_static: the query entry point that allocates no memory.

It exists for callers that cannot allocate device memory at query time (a
framework that owns all device memory and hands out fixed buffers, or a loop
that cannot afford cudaFree's device-wide synchronisation or a failing
cudaMalloc).  Its scratch is one fixed-size array in device memory shared by
every call, so the test makes two calls in a row and checks each against the
regular gp_query at the same K, within the parity tolerance the other GPU
tests use.  This file is collected last so that a run stopping at the first
failure has already run every other test; it builds what it needs itself and
passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg

L1_BAR = 1e-6
MAX_BAR = 1e-8


def _lib():
    from paper_2412_10789_gb300 import build, gp
    build.build()
    lib = gp.load_library()
    f = lib.gp_query_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    return gp, lib


def test_rejects_graphs_beyond_the_static_limit():
    gp, lib = _lib()
    rc = lib.gp_query_static(1 << 21, 0, None, None, 0, 0, 0.2, 10, None, None)
    assert rc == gp.GP_EINVAL
    assert "exceeds the static scratch limit" in gp.gp_last_error()


@pytest.mark.gpu
def test_static_query_matches_gp_query_twice():
    import torch
    gp, lib = _lib()
    g = gg.rmat(16, 16, seed=3)
    rp = torch.from_numpy(g.row_ptr32()).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
    try:
        stream = torch.cuda.current_stream()
        srcs = [int(s) for s in gg.sources(g, 2, 41)]
        for (fn, param, K), s in zip([(gp.GP_FN_PPR, 0.2, 24), (gp.GP_FN_HKPR, 5.0, 16)], srcs):
            y_static = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.gp_query_static(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), fn, s, param, K,
                                     y_static.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == gp.GP_OK, gp.gp_last_error()
            y_ref = torch.empty(g.n, dtype=torch.float64, device="cuda")
            gp.gp_query(dg, fn, s, param, 1e-6, y_ref, k_rule=gp.GP_K_FIXED, k_fixed=K)
            torch.cuda.synchronize()
            a, b = y_static.cpu().numpy(), y_ref.cpu().numpy()
            assert np.isfinite(a).all()
            assert np.abs(a - b).sum() <= L1_BAR
            assert np.abs(a - b).max() <= MAX_BAR
    finally:
        dg.close()
