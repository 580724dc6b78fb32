"""GPU parity of single-source ChebyPower (gp_ppr / gp_hkpr / gp_query) and the
PwMethod baseline (gp_power) against the FP64 oracle, through the C ABI.

Bar (FP32 storage, compensated FP32 sums, float-pair y): element-wise against
the oracle run with the same K, l1 <= 1e-6 and max-abs <= 1e-8; with the l1
stop rule, l1 <= tol against the converged oracle vector.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

L1_BAR = 1e-6
MAX_BAR = 1e-8
KINDS = {"ppr": 0, "hkpr": 1}


@pytest.fixture(scope="module")
def gp():
    import torch
    from paper_2412_10789_gb300 import build, gp as gpmod
    build.build()
    assert torch.cuda.is_available()
    return gpmod


def _graphs():
    return {
        "er4096": gg.erdos_renyi(4096, 16384, 1),
        "rmat13": gg.rmat(13, 16, seed=2),
        "rmat16": gg.rmat(16, 16, seed=3),
        "chunglu20k": gg.chung_lu(20011, 30.0, 2.1, seed=4),
    }


_G = {}


def graph(name):
    if name not in _G:
        _G[name] = _graphs()[name]
    return _G[name]


def make(gp, g, **opt):
    rp = g.row_ptr if opt.pop("rp_int64_input", False) else g.row_ptr32()
    return gp.gp_graph_create(g.n, rp, g.col_idx, g.degree, **opt)


def run(gp, dg, g, kind, s, param, tol=1e-6, K=None, dtype="float64", device=True):
    import torch
    y = torch.empty(g.n, dtype=getattr(torch, dtype), device="cuda" if device else "cpu")
    if K is None:
        info = gp.gp_query(dg, KINDS[kind], s, param, tol, y)
    else:
        info = gp.gp_query(dg, KINDS[kind], s, param, tol, y, k_rule=gp.GP_K_FIXED, k_fixed=K)
    return y.cpu().numpy().astype(np.float64), info


SCHEDULES = {
    "default": {},
    "pieces": {"t_heavy": 24},                       # every row of degree >= 24 summed in pieces
    "int64_rows": {"row_ptr_64": 1},
}


@pytest.mark.parametrize("gname", ["er4096", "rmat13", "rmat16", "chunglu20k"])
@pytest.mark.parametrize("sched", sorted(SCHEDULES))
@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_fixed_K_parity(gp, gname, sched, kind, param):
    g = graph(gname)
    dg = make(gp, g, **SCHEDULES[sched])
    try:
        for s in list(gg.sources(g, 2, 17)) + [int(gg.top_degree_sources(g, 1)[0])]:
            K = 28 if kind == "ppr" else 16
            got, info = run(gp, dg, g, kind, int(s), param, K=K)
            want = O.chebypower(g, int(s), kind, param, K)
            e = O.errors(g, want, got)
            assert info["K"] == K
            assert e["l1"] <= L1_BAR and e["maxabs"] <= MAX_BAR, (s, e)
    finally:
        dg.close()


@pytest.mark.parametrize("gname", ["er4096", "rmat16", "chunglu20k"])
@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("ppr", 0.1), ("ppr", 0.5), ("hkpr", 3.0),
                                        ("hkpr", 5.0), ("hkpr", 10.0)])
@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_stop_rule_accuracy(gp, gname, kind, param, tol):
    g = graph(gname)
    dg = make(gp, g)
    try:
        for s in gg.sources(g, 2, 29):
            s = int(s)
            got, info = run(gp, dg, g, kind, s, param, tol=tol)
            ystar = O.chebypower(g, s, kind, param, 160)
            assert O.errors(g, ystar, got)["l1"] <= tol, info
            # the oracle takes the same stop decision in FP64 (the device measures the
            # norms in FP32; a near-tie may move K by one step)
            _, Ko, norms = O.chebypower_tol(g, s, kind, param, tol)
            assert abs(info["K"] - Ko) <= 1, (info, Ko)
            if info["K"] != Ko:
                c = O.cheb_coeffs(kind, param, 200)
                k = min(info["K"], Ko)
                margin = np.abs(c[k + 1:]).sum() * norms[: k + 1].max() / tol
                assert abs(margin - 1.0) < 1e-3, (info, Ko, margin)
    finally:
        dg.close()


def test_config1_against_dense_solve(gp):
    # ER n=4096, average degree 8, source 0, PPR alpha=0.2: K chosen (by the
    # oracle) so that the FP64 ChebyPower is within l1 1e-8 of the dense solve.
    g = graph("er4096")
    assert g.degree[0] > 0
    ydense = O.dense_ppr(g, 0, 0.2)
    K = next(k for k in range(1, 80) if O.errors(g, ydense, O.chebypower(g, 0, "ppr", 0.2, k))["l1"] <= 1e-8)
    dg = make(gp, g)
    try:
        got, info = run(gp, dg, g, "ppr", 0, 0.2, K=K)
        e_or = O.errors(g, O.chebypower(g, 0, "ppr", 0.2, K), got)
        e_dense = O.errors(g, ydense, got)
        assert e_or["l1"] <= L1_BAR and e_or["maxabs"] <= MAX_BAR, e_or
        assert e_dense["l1"] <= 1e-8 + L1_BAR, e_dense
    finally:
        dg.close()


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_power_baseline_parity(gp, kind, param):
    import torch
    g = graph("rmat13")
    dg = make(gp, g)
    try:
        for s in gg.sources(g, 2, 3):
            s = int(s)
            y = torch.empty(g.n, dtype=torch.float64, device="cuda")
            info = gp.gp_power(dg, KINDS[kind], s, param, 1e-6, y)
            z = O.taylor_coeffs(kind, param, 2000)
            N = next(n for n in range(1, 2000) if z[n:].sum() <= 1e-6)
            assert info["K"] == N - 1
            want = O.power(g, s, kind, param, N)
            e = O.errors(g, want, y.cpu().numpy())
            assert e["l1"] <= L1_BAR and e["maxabs"] <= MAX_BAR, e
            assert O.errors(g, O.chebypower(g, s, kind, param, 160), y.cpu().numpy())["l1"] <= 1e-6 + 1e-7
    finally:
        dg.close()


def test_output_forms_agree(gp):
    import torch
    g = graph("rmat13")
    dg = make(gp, g)
    try:
        s = int(gg.sources(g, 1, 5)[0])
        y64 = torch.empty(g.n, dtype=torch.float64, device="cuda")
        gp.gp_ppr(dg, s, 0.2, 1e-6, y64)
        a = y64.cpu().numpy()
        h64 = np.empty(g.n, dtype=np.float64)
        gp.gp_ppr(dg, s, 0.2, 1e-6, h64)
        pinned = torch.empty(g.n, dtype=torch.float32).pin_memory()
        gp.gp_ppr(dg, s, 0.2, 1e-6, pinned)
        d32 = torch.empty(g.n, dtype=torch.float32, device="cuda")
        gp.gp_ppr(dg, s, 0.2, 1e-6, d32, info=False)
        torch.cuda.synchronize()
        assert np.array_equal(a, h64)  # deterministic: same K, same sums
        assert np.array_equal(a.astype(np.float32), pinned.numpy())
        assert np.array_equal(a.astype(np.float32), d32.cpu().numpy())
        assert abs(a.sum() - 1.0) < 1e-6 and a.min() > -1e-6
    finally:
        dg.close()


def test_edge_cases(gp):
    cases = [
        ("star", gg.from_edges(4, [(0, 1), (0, 2), (0, 3)])),
        ("pair", gg.from_edges(2, [(0, 1)])),
        ("cycle64", gg.from_edges(64, [(i, (i + 1) % 64) for i in range(64)])),
        ("path_with_isolated", gg.from_edges(7, [(0, 1), (1, 2), (2, 3), (5, 6)])),
    ]
    for name, g in cases:
        dg = make(gp, g)
        try:
            for s in range(g.n):
                for kind, param in (("ppr", 0.2), ("hkpr", 5.0)):
                    got, info = run(gp, dg, g, kind, s, param, tol=1e-8)
                    ystar = O.chebypower(g, s, kind, param, 200) if g.degree[s] else \
                        O.unit_vector(g.n, s) * O.taylor_coeffs(kind, param, 1)[0]
                    e = O.errors(g, ystar, got)
                    assert e["l1"] <= 1e-8 + 1e-7 and e["maxabs"] <= MAX_BAR, (name, s, kind, e, info)
        finally:
            dg.close()


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_float_pair_path_parity(gp, kind, param):
    # The float-pair storage path (used on tiny graphs) forced on a larger one:
    # ~48-bit arithmetic, so the bar is far below the FP32 path's.
    g = graph("rmat13")
    dg = make(gp, g, precise_rows=1 << 20)
    try:
        for s in list(gg.sources(g, 2, 5)) + [int(gg.top_degree_sources(g, 1)[0])]:
            got, info = run(gp, dg, g, kind, int(s), param, K=25)
            e = O.errors(g, O.chebypower(g, int(s), kind, param, 25), got)
            assert e["l1"] <= 1e-10 and e["maxabs"] <= 1e-12, e
            got, info = run(gp, dg, g, kind, int(s), param, tol=1e-8)
            assert O.errors(g, O.chebypower(g, int(s), kind, param, 160), got)["l1"] <= 1e-8
    finally:
        dg.close()


def test_isolated_only_graph(gp):
    g = gg.from_edges(5, [])
    dg = make(gp, g)
    try:
        got, info = run(gp, dg, g, "ppr", 3, 0.3)
        assert np.array_equal(got, 0.3 * O.unit_vector(5, 3))
        got, info = run(gp, dg, g, "hkpr", 0, 2.0)
        assert abs(got[0] - np.exp(-2.0)) < 1e-15 and np.count_nonzero(got) == 1
    finally:
        dg.close()


@pytest.mark.parametrize("opt", [{}, {"row_ptr_64": 1}, {"rp_int64_input": True}])
def test_export_is_bit_exact(gp, opt):
    g = graph("rmat16")
    dg = make(gp, g, **dict(opt))
    try:
        rp, ci, dg_ = gp.gp_graph_export(dg)
        assert np.array_equal(rp, g.row_ptr)
        assert np.array_equal(ci, g.col_idx)
        assert np.array_equal(dg_, g.degree)
        assert dg.n_active == int((g.degree > 0).sum()) and dg.max_degree == int(g.degree.max())
    finally:
        dg.close()


def test_device_inputs(gp):
    import torch
    g = graph("rmat13")
    dg = gp.gp_graph_create(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(),
                            torch.from_numpy(g.degree).cuda())
    try:
        rp, ci, d = gp.gp_graph_export(dg)
        assert np.array_equal(ci, g.col_idx) and np.array_equal(rp, g.row_ptr)
    finally:
        dg.close()


def _bad(g, mutate):
    rp = g.row_ptr32().copy()
    ci = g.col_idx.copy()
    deg = g.degree.copy()
    mutate(rp, ci, deg)
    return rp, ci, deg


def test_validation_rejects_bad_csr(gp):
    g = gg.from_edges(6, [(0, 1), (0, 2), (1, 2), (3, 4), (4, 5)])

    def unsorted(rp, ci, deg):
        ci[0], ci[1] = ci[1], ci[0]

    def selfloop(rp, ci, deg):
        ci[rp[3]] = 3

    def out_of_range(rp, ci, deg):
        ci[-1] = 99

    def degree_mismatch(rp, ci, deg):
        deg[2] += 1

    def asymmetric(rp, ci, deg):
        ci[rp[5]] = 3  # row 5: (5,4) -> (5,3), with no (3,5)

    for name, mut in [("unsorted", unsorted), ("selfloop", selfloop), ("range", out_of_range),
                      ("degree", degree_mismatch), ("asymmetric", asymmetric)]:
        rp, ci, deg = _bad(g, mut)
        with pytest.raises(gp.GPError) as ei:
            gp.gp_graph_create(g.n, rp, ci, deg)
        assert ei.value.status == gp.GP_EINVAL, name
    # bad query arguments
    dg = make(gp, g)
    try:
        import torch
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        for args in [(0, 1.5, 1e-6), (0, 0.0, 1e-6), (9, 0.2, 1e-6), (0, 0.2, 0.0), (0, 0.2, 1.0)]:
            with pytest.raises(gp.GPError):
                gp.gp_ppr(dg, *args, y)
        with pytest.raises(gp.GPError):
            gp.gp_hkpr(dg, 0, -1.0, 1e-6, y)
        # the context survives: a valid query still works
        got, _ = run(gp, dg, g, "ppr", 0, 0.2, tol=1e-8)
        assert abs(got.sum() - 1.0) < 1e-6
    finally:
        dg.close()


def test_launch_counter_and_profile(gp):
    import torch
    g = graph("rmat13")
    dg = make(gp, g)
    try:
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        gp.gp_profile_enable(dg, True)
        before = gp.gp_launch_count()
        info = gp.gp_ppr(dg, int(gg.sources(g, 1, 1)[0]), 0.2, 1e-6, y)
        launched = gp.gp_launch_count() - before
        prof = gp.gp_profile_read(dg)
        assert prof["step_launches"] == info["K"] - 1
        assert launched >= info["K"]  # init + passes + finalize
        assert prof["step_ms"] > 0 and prof["step_bytes"] > 0
    finally:
        dg.close()


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_full_size_rmat22(gp, kind, param):
    """R-MAT scale 22 (4.19M nodes, ~128M nnz), the benchmark's workload and launch
    configuration: fixed-K parity element by element and stop-rule accuracy."""
    g = graph_rmat22()
    dg = make(gp, g)
    try:
        s = int(gg.sources(g, 1, 2)[0])
        _, Ko, _ = O.chebypower_tol(g, s, kind, param, 1e-6)
        got, info = run(gp, dg, g, kind, s, param, K=Ko)
        want = O.chebypower(g, s, kind, param, Ko)
        e = O.errors(g, want, got)
        assert e["l1"] <= L1_BAR and e["maxabs"] <= MAX_BAR, e
        got2, info2 = run(gp, dg, g, kind, s, param, tol=1e-6)
        ystar = O.chebypower(g, s, kind, param, Ko + 25)
        assert O.errors(g, ystar, got2)["l1"] <= 1e-6, info2
        assert abs(info2["K"] - Ko) <= 1
    finally:
        dg.close()


def graph_rmat22():
    if "rmat22" not in _G:
        _G["rmat22"] = gg.rmat(22, 16, seed=2)
    return _G["rmat22"]


def _with_isolated_targets(scale, extra_rows):
    """An R-MAT CSR whose first `extra_rows` non-empty rows also list a node
    with an empty row (asymmetric; accepted with the symmetry check off)."""
    base = gg.rmat(scale, 8, seed=5)
    rows = [list(base.col_idx[base.row_ptr[u]:base.row_ptr[u + 1]]) for u in range(base.n)]
    iso = [u for u in range(base.n) if not rows[u]]
    assert len(iso) >= 3
    for k, u in enumerate([u for u in range(base.n) if rows[u]][:extra_rows]):
        rows[u] = sorted(set(rows[u]) | {iso[k % len(iso)]})
    rp = np.zeros(base.n + 1, dtype=np.int64)
    for u in range(base.n):
        rp[u + 1] = rp[u] + len(rows[u])
    ci = np.array([v for r in rows for v in r], dtype=np.int32)
    return gg.Graph(f"rmat{scale}_with_isolated_targets", base.n, rp, ci)


@pytest.mark.parametrize("precise_rows", [0, -1])
def test_unvalidated_asymmetric_csr(gp, precise_rows):
    """Rows that list nodes with empty rows: those nodes contribute nothing
    (1/d := 0) and their result entries stay 0, as in the oracle's pull form of
    P; sources whose own row lists such a node included.  precise_rows 0 runs
    the float-pair path on this small graph, -1 the FP32 step kernel."""
    g = _with_isolated_targets(11, 60)
    dg = make(gp, g, validate_symmetry=0, precise_rows=precise_rows)
    try:
        srcs = [u for u in range(g.n) if g.degree[u] > 0][:4]
        for kind, param, K in (("ppr", 0.2, 20), ("hkpr", 5.0, 14)):
            for s in srcs:
                got, info = run(gp, dg, g, kind, s, param, K=K)
                want = O.chebypower(g, s, kind, param, K)
                e = O.errors(g, want, got)
                assert np.isfinite(got).all()
                assert e["l1"] <= L1_BAR and e["maxabs"] <= MAX_BAR, (kind, s, e)
    finally:
        dg.close()
