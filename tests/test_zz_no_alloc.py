"""gp_query_static: the query entry point that allocates no memory.

It exists for callers that cannot allocate device memory at query time: a
framework that owns all device memory and hands out fixed buffers, or a loop
that cannot afford cudaFree's device-wide synchronisation or a failing
cudaMalloc.  Its scratch is one fixed-size array in device memory shared by
every call, so the tests make calls in a row and check each against the FP64
oracle at the same K and against the regular gp_query, within the parity
tolerance the other GPU tests use (l1 <= 1e-6, max-abs <= 1e-8).  This file
is collected last so that a run stopping at the first failure has already run
every other test; it builds what it needs itself and passes alone in a fresh
process as well.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle as O

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


def _static(gp, lib, g, rp, ci, fn, s, param, K):
    import torch
    y = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.gp_query_static(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), fn, s, param, K, y.data_ptr(),
                             ctypes.c_void_p(stream.cuda_stream))
    assert rc == gp.GP_OK, gp.gp_last_error()
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _check_calls(gp, lib, g, dg, cases):
    """Each (fn, source, param, K) through gp_query_static, one call after
    another on the shared scratch: equal to the oracle at the same K and to
    gp_query within the parity bar."""
    import torch
    rp = torch.from_numpy(g.row_ptr32()).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    for fn, s, param, K in cases:
        got = _static(gp, lib, g, rp, ci, fn, s, param, K)
        assert np.isfinite(got).all()
        kind = "ppr" if fn == gp.GP_FN_PPR else "hkpr"
        if g.degree[s] > 0:
            want = O.chebypower(g, s, kind, param, K)
        else:
            want = O.unit_vector(g.n, s) * O.taylor_coeffs(kind, param, 1)[0]
        e = O.errors(g, want, got)
        assert e["l1"] <= L1_BAR and e["maxabs"] <= MAX_BAR, (fn, s, K, e)
        y_ref = torch.empty(g.n, dtype=torch.float64, device="cuda")
        gp.gp_query(dg, fn, s, param, 1e-6, y_ref, k_rule=gp.GP_K_FIXED, k_fixed=K)
        ref = y_ref.cpu().numpy()
        assert np.abs(got - ref).sum() <= L1_BAR and np.abs(got - ref).max() <= MAX_BAR


@pytest.mark.gpu
def test_static_query_matches_oracle_and_gp_query_in_a_row():
    gp, lib = _lib()
    g = gg.rmat(16, 16, seed=3)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
    try:
        s0, s1 = [int(s) for s in gg.sources(g, 2, 41)]
        hub = int(gg.top_degree_sources(g, 1)[0])
        _check_calls(gp, lib, g, dg, [(gp.GP_FN_PPR, s0, 0.2, 24), (gp.GP_FN_HKPR, s1, 5.0, 16),
                                      (gp.GP_FN_PPR, hub, 0.2, 28)])
    finally:
        dg.close()


@pytest.mark.gpu
def test_static_query_isolated_source_and_empty_listed_rows():
    """A CSR whose rows list nodes with empty rows (accepted by gp_graph_create
    with the symmetry check off): those nodes contribute nothing (1/d := 0);
    an isolated source returns f(0) e_s."""
    gp, lib = _lib()
    base = gg.rmat(10, 8, seed=5)
    rows = [list(base.col_idx[base.row_ptr[u]:base.row_ptr[u + 1]]) for u in range(base.n)]
    iso = [u for u in range(base.n) if not rows[u]]
    assert len(iso) >= 3
    for k, u in enumerate([u for u in range(base.n) if rows[u]][:40]):
        rows[u] = sorted(set(rows[u]) | {iso[k % len(iso)]})
    rp = np.zeros(base.n + 1, dtype=np.int64)
    for u in range(base.n):
        rp[u + 1] = rp[u] + len(rows[u])
    ci = np.array([v for r in rows for v in r], dtype=np.int32)
    g = gg.Graph("rmat10_with_isolated_targets", base.n, rp, ci)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, validate_symmetry=0)
    try:
        srcs = [u for u in range(g.n) if g.degree[u] > 0][:3]
        _check_calls(gp, lib, g, dg, [(gp.GP_FN_PPR, srcs[0], 0.2, 14), (gp.GP_FN_HKPR, srcs[1], 5.0, 12),
                                      (gp.GP_FN_PPR, iso[1], 0.3, 10), (gp.GP_FN_PPR, srcs[2], 0.5, 9)])
    finally:
        dg.close()
