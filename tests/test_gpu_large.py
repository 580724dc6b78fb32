"""Parity at the benchmark configurations' sizes and index widths.

* More than 2^31 CSR entries: the complete graph K_50000 (2,499,950,000
  entries, int64 row offsets; tiles of the rows past entry 2^31 carry a
  nonzero high half of their 64-bit start).  Ingest is bit-exact, single-source
  FP32 queries match the oracle element by element at fixed K, and the l1 stop
  rule and a BF16 batched block meet their tolerances against the exact
  vector.  K_n's P = (J - I)/(n - 1) has the eigenvalue 1 on the all-ones
  vector and mu = -1/(n - 1) on its complement, so
  y* = f(P) e_s = f(1) 1/n + f(mu) (e_s - 1/n) exactly.
* The mixed 256-column block of R-MAT scale 24 (16.8M nodes, ~521M entries):
  sampled columns of every function type against the converged oracle, in
  BF16 at l1 <= 1e-4 and in FP32 at l1 <= 1e-6.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

KINDS = {0: "ppr", 1: "hkpr"}


@pytest.fixture(scope="module")
def gp():
    import torch
    from paper_2412_10789_gb300 import build, gp as gpmod
    build.build()
    assert torch.cuda.is_available()
    return gpmod


def _f(kind, param, x):
    return param / (1.0 - (1.0 - param) * x) if kind == "ppr" else np.exp(-param * (1.0 - x))


def complete_exact(n, s, kind, param):
    mu = -1.0 / (n - 1)
    y = np.full(n, (1.0 - _f(kind, param, mu)) / n)
    y[s] = 1.0 / n + _f(kind, param, mu) * (1.0 - 1.0 / n)
    return y


@pytest.fixture(scope="module")
def k50000(gp):
    g = gg.complete(50000)
    assert g.nnz > 2**31 and g.nnz == 50000 * 49999
    dg = gp.gp_graph_create(g.n, g.row_ptr, g.col_idx, g.degree, block_width=16, storage=gp.GP_BF16)
    yield g, dg
    dg.close()


def test_complete_graph_ingest_is_bit_exact(gp, k50000):
    g, dg = k50000
    rp, ci, deg = gp.gp_graph_export(dg)
    assert np.array_equal(rp, g.row_ptr)
    assert np.array_equal(deg, g.degree)
    assert np.array_equal(ci, g.col_idx)


@pytest.mark.parametrize("kind,param,K,s", [("ppr", 0.2, 16, 49999), ("hkpr", 5.0, 12, 0), ("ppr", 0.5, 9, 46000)])
def test_complete_graph_single_source_fixed_K(gp, k50000, kind, param, K, s):
    import torch
    g, dg = k50000
    y = torch.empty(g.n, dtype=torch.float64, device="cuda")
    info = gp.gp_query(dg, 0 if kind == "ppr" else 1, s, param, 1e-6, y, k_rule=gp.GP_K_FIXED, k_fixed=K)
    assert info["K"] == K
    got = y.cpu().numpy()
    want = O.chebypower(g, s, kind, param, K)
    e = O.errors(g, want, got)
    assert e["l1"] <= 1e-6 and e["maxabs"] <= 1e-8, e


def test_complete_graph_stop_rule_and_bf16_block(gp, k50000):
    import torch
    g, dg = k50000
    y = torch.empty(g.n, dtype=torch.float64, device="cuda")
    for kind, param, s in (("ppr", 0.2, 49998), ("hkpr", 5.0, 3)):
        gp.gp_query(dg, 0 if kind == "ppr" else 1, s, param, 1e-6, y)
        l1 = np.abs(y.cpu().numpy() - complete_exact(g.n, s, kind, param)).sum()
        assert l1 <= 1e-6, (kind, l1)
    srcs = [0, 7, 25000, 46341, 49999, 12345]
    ys = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in srcs]
    reqs = [gp.make_request(i % 2, s, 0.2 if i % 2 == 0 else 5.0, 1e-4, ys[i]) for i, s in enumerate(srcs)]
    infos = gp.gp_batch(dg, reqs)
    for i, s in enumerate(srcs):
        kind, param = ("ppr", 0.2) if i % 2 == 0 else ("hkpr", 5.0)
        l1 = np.abs(ys[i].cpu().numpy() - complete_exact(g.n, s, kind, param)).sum()
        assert l1 <= 1e-4, (i, l1, infos[i])


MIX = [(0, 0.1), (0, 0.2), (0, 0.5), (1, 3.0), (1, 5.0), (1, 10.0)]


def test_rmat24_mixed_block_sampled_parity(gp):
    """The mixed block of the R-MAT 24 workload: 256 sources, columns cycling
    through SSPPR alpha in {0.1, 0.2, 0.5} and HKPR t in {3, 5, 10}, one
    256-column block; the first column of each function type is checked."""
    import torch
    g = gg.rmat(24, 16, 0.57, 0.19, 0.19, seed=3)
    srcs = [int(s) for s in gg.sources(g, 256, 3)]
    sample = list(range(6))
    ystar = {}
    for i in sample:
        fn, p = MIX[i]
        ystar[i], _, _ = O.chebypower_tol(g, srcs[i], KINDS[fn], p, 1e-9)
    for storage, tol in ((gp.GP_BF16, 1e-4), (gp.GP_F32, 1e-6)):
        dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, storage=storage, block_width=256)
        try:
            ys = [torch.empty(g.n, dtype=torch.float32, device="cuda") for _ in range(len(sample))]
            scratch = torch.empty(g.n, dtype=torch.float32, device="cuda")
            reqs = [gp.make_request(MIX[i % 6][0], s, MIX[i % 6][1], tol, ys[i] if i in sample else scratch)
                    for i, s in enumerate(srcs)]
            infos = gp.gp_batch(dg, reqs)
            for i in sample:
                l1 = np.abs(ys[i].cpu().numpy().astype(np.float64) - ystar[i]).sum()
                assert l1 <= tol, (storage, i, MIX[i], l1, infos[i])
        finally:
            dg.close()
