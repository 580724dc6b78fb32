"""GPU tests of ChebyPush (Algorithm 4, gp_chebypush) against the FP64 oracle's
Algorithm 4 (the algorithm's push rule |r(u)| > eps_k d_u) and against
Theorem 3's degree-normalised bound, through the C ABI."""
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


_G = {}


def graph(name):
    if name not in _G:
        _G[name] = {"er4096": lambda: gg.erdos_renyi(4096, 16384, 1), "rmat14": lambda: gg.rmat(14, 16, seed=2),
                    "chunglu20k": lambda: gg.chung_lu(20011, 30.0, 2.1, seed=4)}[name]()
    return _G[name]


def _oracle_K(kind, param, eps_a):
    c = O.cheb_coeffs(kind, param, 400)
    tail = np.array([np.abs(c[k:]).sum() for k in range(1, len(c) + 1)])  # tail[k-1] = sum_{l>=k} |c_l|
    K = 1
    while tail[K - 1] > eps_a / 2:
        K += 1
    return K, c


@pytest.mark.parametrize("gname", ["er4096", "rmat14", "chunglu20k"])
@pytest.mark.parametrize("fn,param", [(0, 0.2), (1, 5.0)])
@pytest.mark.parametrize("eps_a", [1e-3, 1e-6])
def test_chebypush_matches_oracle(gp, gname, fn, param, eps_a):
    import torch
    g = graph(gname)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
    try:
        for s in list(gg.sources(g, 2, 29)) + [int(gg.top_degree_sources(g, 1)[0])]:
            y = torch.empty(g.n, dtype=torch.float64, device="cuda")
            info = gp.gp_chebypush(dg, fn, int(s), param, eps_a, y)
            K, c = _oracle_K(KINDS[fn], param, eps_a)
            assert info["K"] == K
            want = O.chebypush(g, int(s), KINDS[fn], param, K, eps_a=eps_a, coeffs=c[:K + 1])
            got = y.cpu().numpy()
            assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.abs(want).max()), (s, np.max(np.abs(got - want)))
    finally:
        dg.close()


@pytest.mark.parametrize("fn,param", [(0, 0.2), (1, 5.0)])
def test_chebypush_degree_normalised_bound(gp, fn, param):
    import torch
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
    try:
        d = np.maximum(g.degree, 1)
        for eps_a in (1e-3, 1e-5):
            for s in gg.sources(g, 3, 31):
                y = torch.empty(g.n, dtype=torch.float64, device="cuda")
                gp.gp_chebypush(dg, fn, int(s), param, eps_a, y)
                ystar = O.chebypower(g, int(s), KINDS[fn], param, 150)
                assert np.max(np.abs(ystar - y.cpu().numpy()) / d) < eps_a
    finally:
        dg.close()


def test_chebypush_outputs_isolated_source_and_errors(gp):
    import torch
    g = gg.from_edges(40, [(i, i + 1) for i in range(30)] + [(35, 36)], "path_with_isolated")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
    try:
        # host FP64 and device FP32 outputs agree with the oracle
        yh = np.zeros(g.n)
        gp.gp_chebypush(dg, 0, 3, 0.2, 1e-6, yh)
        K, c = _oracle_K("ppr", 0.2, 1e-6)
        want = O.chebypush(g, 3, "ppr", 0.2, K, eps_a=1e-6, coeffs=c[:K + 1])
        assert np.max(np.abs(yh - want)) < 1e-12
        yf = torch.empty(g.n, dtype=torch.float32, device="cuda")
        gp.gp_chebypush(dg, 0, 3, 0.2, 1e-6, yf)
        assert np.max(np.abs(yf.cpu().numpy() - want)) < 1e-6
        # node 33 is isolated: y = f(0) e_s up to the truncation, as the oracle's Algorithm 4
        yi = np.zeros(g.n)
        gp.gp_chebypush(dg, 1, 33, 4.0, 1e-8, yi)
        K, c = _oracle_K("hkpr", 4.0, 1e-8)
        want = O.chebypush(g, 33, "hkpr", 4.0, K, eps_a=1e-8, coeffs=c[:K + 1])
        assert np.max(np.abs(yi - want)) < 1e-12
        assert abs(yi[33] - np.exp(-4.0)) < 1e-8
        # fixed K
        info = gp.gp_chebypush(dg, 0, 3, 0.2, 1e-6, yh, K=7)
        assert info["K"] == 7
        for bad in (dict(source=-1), dict(source=40), dict(param=1.5), dict(eps=0.0), dict(K=-1)):
            with pytest.raises(Exception):
                gp.gp_chebypush(dg, 0, bad.get("source", 3), bad.get("param", 0.2), bad.get("eps", 1e-6), yh,
                                K=bad.get("K", 0))
    finally:
        dg.close()


def _paper_K(alpha, eps_r, delta, n):
    W = 2 * (2 * eps_r / 3 + 2) * np.log(n) / (eps_r ** 2 * delta)
    return max(1, int(np.ceil(np.log(W / np.sqrt(alpha)) / np.sqrt(alpha))))


@pytest.mark.parametrize("gname", ["er4096", "rmat14"])
@pytest.mark.parametrize("eps_r,delta", [(1.0, 0.5), (0.5, 1e-3)])
def test_bidirectional_matches_oracle(gp, gname, eps_r, delta):
    """Same generator streams, same walks: the device equals the oracle's
    Algorithm 5 up to the rounding order of its FP64 sums."""
    import torch
    g = graph(gname)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
    try:
        alpha = 0.2
        K = _paper_K(alpha, eps_r, delta, g.n)
        for s, seed in zip(list(gg.sources(g, 2, 37)) + [int(gg.top_degree_sources(g, 1)[0])], (1, 2, 3)):
            y = torch.empty(g.n, dtype=torch.float64, device="cuda")
            info = gp.gp_ppr_bidirectional(dg, int(s), alpha, eps_r, delta, y, seed=seed)
            assert info["K"] == K
            want, walks = O.bidirectional(g, int(s), alpha, K, eps_r, delta, seed)
            assert int(info["max_r_l1"]) == walks
            got = y.cpu().numpy()
            assert np.max(np.abs(got - want)) <= 1e-12, (s, np.max(np.abs(got - want)))
        # another seed draws other walks
        y2 = torch.empty(g.n, dtype=torch.float64, device="cuda")
        gp.gp_ppr_bidirectional(dg, int(s), alpha, eps_r, delta, y2, seed=99)
        if eps_r == 1.0:
            assert not torch.equal(y, y2)
    finally:
        dg.close()


def test_bidirectional_isolated_source_and_errors(gp):
    g = gg.from_edges(40, [(i, i + 1) for i in range(30)] + [(35, 36)], "path_with_isolated")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
    try:
        y = np.zeros(g.n)
        K = _paper_K(0.2, 0.5, 0.01, g.n)
        gp.gp_ppr_bidirectional(dg, 33, 0.2, 0.5, 0.01, y, seed=4)
        want, _ = O.bidirectional(g, 33, 0.2, K, 0.5, 0.01, 4)
        assert np.max(np.abs(y - want)) < 1e-12
        assert abs(y[33] - 0.2) < 1e-6
        for bad in (dict(source=40), dict(alpha=1.0), dict(eps_r=0.0), dict(delta=2.0)):
            with pytest.raises(Exception):
                gp.gp_ppr_bidirectional(dg, bad.get("source", 3), bad.get("alpha", 0.2), bad.get("eps_r", 0.5),
                                        bad.get("delta", 0.01), y)
    finally:
        dg.close()


def test_int64_row_offsets(gp):
    """The same queries with row offsets stored as int64 (cfg.row_ptr_64): the
    ChebyPush, bidirectional, batched and propagation paths agree with the oracle."""
    import torch
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, row_ptr_64=1, block_width=16)
    try:
        s = int(gg.sources(g, 1, 41)[0])
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        gp.gp_chebypush(dg, 0, s, 0.2, 1e-5, y, K=20)
        assert np.max(np.abs(y.cpu().numpy() - O.chebypush(g, s, "ppr", 0.2, 20, eps_a=1e-5))) < 1e-12
        K = _paper_K(0.2, 1.0, 0.5, g.n)
        gp.gp_ppr_bidirectional(dg, s, 0.2, 1.0, 0.5, y, seed=5)
        assert np.max(np.abs(y.cpu().numpy() - O.bidirectional(g, s, 0.2, K, 1.0, 0.5, 5)[0])) < 1e-12
        ys = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in range(3)]
        reqs = [gp.make_request(1, int(v), 5.0, 1e-6, ys[i], k_rule=gp.GP_K_FIXED, k_fixed=15)
                for i, v in enumerate(gg.sources(g, 3, 43))]
        gp.gp_batch(dg, reqs)
        for i, v in enumerate(gg.sources(g, 3, 43)):
            want = O.chebypower(g, int(v), "hkpr", 5.0, 15)
            e = O.errors(g, want, ys[i].cpu().numpy())
            assert e["l1"] <= 1e-6 and e["maxabs"] <= 1e-7 + 15 * 2.0 ** -24 * np.abs(want).max(), e
    finally:
        dg.close()


def test_chebypush_unvalidated_asymmetric_csr(gp):
    """Rows that list nodes without neighbours (asymmetric CSR, symmetry check
    off): pushes reach those nodes, which hold residual but push nothing, on
    the device as in the oracle's Algorithm 4."""
    import torch
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
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        for s in [u for u in range(g.n) if rows[u]][:3]:
            info = gp.gp_chebypush(dg, 0, int(s), 0.2, 1e-6, y)
            K, c = _oracle_K("ppr", 0.2, 1e-6)
            assert info["K"] == K
            want = O.chebypush(g, int(s), "ppr", 0.2, K, eps_a=1e-6, coeffs=c[:K + 1])
            got = y.cpu().numpy()
            assert np.max(np.abs(got - want)) <= 1e-12, (s, np.max(np.abs(got - want)))
            assert np.any(want[iso] != 0.0)  # the isolated targets did take residual
    finally:
        dg.close()
