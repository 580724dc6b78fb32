"""GPU tests of the batched column engine (gp_batch) and the serving loop
(gp_submit / gp_poll) against the FP64 oracle, through the C ABI.

Batched columns accumulate the SpMM in FP32 and keep y in FP32 (the single
query uses compensated sums and a float-pair y), so the fixed-K parity bar
here is l1 <= 1e-6 and max-abs <= 1e-7 + K 2^-24 max|y|: y is rounded once per
step, by at most half an ulp of max|y|.  With 16-bit storage the bar is the
query's own l1 tolerance against the converged oracle vector.
"""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

KINDS = {0: "ppr", 1: "hkpr"}
MIX = [(0, 0.1), (0, 0.2), (0, 0.5), (1, 3.0), (1, 5.0), (1, 10.0)]


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
        _G[name] = {"rmat14": lambda: gg.rmat(14, 16, seed=2), "er4096": lambda: gg.erdos_renyi(4096, 16384, 1),
                    "chunglu20k": lambda: gg.chung_lu(20011, 30.0, 2.1, seed=4)}[name]()
    return _G[name]


def _outputs(g, count, device=True):
    import torch
    return [torch.empty(g.n, dtype=torch.float64, device="cuda" if device else "cpu") for _ in range(count)]


def _requests(gp, g, srcs, tol, ys, k_rule=None, K=None):
    reqs = []
    for i, s in enumerate(srcs):
        fn, p = MIX[i % len(MIX)]
        if k_rule is None:
            reqs.append(gp.make_request(fn, int(s), p, tol, ys[i]))
        else:
            reqs.append(gp.make_request(fn, int(s), p, tol, ys[i], k_rule=k_rule, k_fixed=K[i]))
    return reqs


def _fp32_maxabs_bar(want, K):
    """The batched form keeps y in FP32 and rounds it once per step: at most
    K * 2^-24 * max|y| over K steps, plus 1e-7 for the rest of the FP32 path."""
    return 1e-7 + K * 2.0 ** -24 * float(np.abs(want).max())


@pytest.mark.parametrize("B", [8, 64, 256])
def test_batch_fixed_K_parity_fp32(gp, B):
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=B)
    try:
        srcs = list(gg.sources(g, 20, 7)) + [int(gg.top_degree_sources(g, 1)[0])]
        ys = _outputs(g, len(srcs))
        Ks = [12 + (i % 9) for i in range(len(srcs))]
        infos = gp.gp_batch(dg, _requests(gp, g, srcs, 1e-6, ys, gp.GP_K_FIXED, Ks))
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            want = O.chebypower(g, int(s), KINDS[fn], p, Ks[i])
            e = O.errors(g, want, ys[i].cpu().numpy())
            assert infos[i]["K"] == Ks[i]
            assert e["l1"] <= 1e-6 and e["maxabs"] <= _fp32_maxabs_bar(want, Ks[i]), (i, e)
    finally:
        dg.close()


@pytest.mark.parametrize("gname", ["rmat14", "chunglu20k"])
@pytest.mark.parametrize("storage,tol", [("f32", 1e-6), ("f32", 1e-4), ("bf16", 1e-4), ("f16", 1e-4),
                                         ("bf16", 1e-5), ("bf16", 1e-6), ("f16", 1e-6)])
def test_batch_stop_rule_accuracy(gp, gname, storage, tol):
    g = graph(gname)
    st = {"f32": gp.GP_F32, "bf16": gp.GP_BF16, "f16": gp.GP_F16}[storage]
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=32, storage=st)
    try:
        srcs = gg.sources(g, 40, 11)  # two blocks of 32
        ys = _outputs(g, len(srcs))
        infos = gp.gp_batch(dg, _requests(gp, g, srcs, tol, ys))
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            ystar = O.chebypower(g, int(s), KINDS[fn], p, 150)
            l1 = O.errors(g, ystar, ys[i].cpu().numpy())["l1"]
            assert l1 <= tol, (i, storage, l1, infos[i])
    finally:
        dg.close()


@pytest.mark.parametrize("t_heavy", [2, 65, 257])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_batch_chunk_threshold(gp, t_heavy, storage):
    """Rows of degree >= t_heavy summed as chunk tiles (one chunk for rows of at
    most 508 entries) give the same sums: fixed-K parity with the oracle."""
    g = graph("rmat14")
    st = {"f32": gp.GP_F32, "bf16": gp.GP_BF16}[storage]
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=64, storage=st,
                            t_heavy=t_heavy)
    try:
        srcs = list(gg.sources(g, 12, 17)) + [int(gg.top_degree_sources(g, 1)[0])]
        ys = _outputs(g, len(srcs))
        Ks = [14 + (i % 5) for i in range(len(srcs))]
        infos = gp.gp_batch(dg, _requests(gp, g, srcs, 1e-6, ys, gp.GP_K_FIXED, Ks))
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            want = O.chebypower(g, int(s), KINDS[fn], p, Ks[i])
            e = O.errors(g, want, ys[i].cpu().numpy())
            assert infos[i]["K"] == Ks[i]
            bar = (1e-6, _fp32_maxabs_bar(want, Ks[i])) if storage == "f32" else (1e-4, 1e-5)
            assert e["l1"] <= bar[0] and e["maxabs"] <= bar[1], (i, e)
    finally:
        dg.close()


@pytest.mark.parametrize("gname", ["rmat14", "chunglu20k"])
@pytest.mark.parametrize("B", [128, 256])
def test_batch_fp32_wide_blocks_meet_1e6(gp, gname, B):
    """Wide FP32 blocks: one or two lane groups sum a whole 508-entry chunk, and
    the two-level lane sums keep every column within l1 <= 1e-6 (HKPR t = 10
    included, the mix's longest sums)."""
    g = graph(gname)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=B)
    try:
        srcs = list(gg.sources(g, 36, 13)) + [int(v) for v in gg.top_degree_sources(g, 4)]
        ys = _outputs(g, len(srcs))
        infos = gp.gp_batch(dg, _requests(gp, g, srcs, 1e-6, ys))
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            ystar = O.chebypower(g, int(s), KINDS[fn], p, 150)
            l1 = O.errors(g, ystar, ys[i].cpu().numpy())["l1"]
            assert l1 <= 1e-6, (i, l1, infos[i])
    finally:
        dg.close()


@pytest.mark.parametrize("fn,param", [(0, 0.1), (1, 10.0)])
def test_batch_bf16_homogeneous_slow_decay(gp, fn, param):
    """A BF16 block of only slowly decaying expansions (SSPPR alpha = 0.1, HKPR
    t = 10) switches to 16 bits at its own, early warm-up step; the weight of
    that switch counts the linear growth of uncompensated rounding errors, and
    every column stays within l1 <= 1e-4."""
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=16, storage=gp.GP_BF16)
    try:
        srcs = gg.sources(g, 16, 21)
        ys = _outputs(g, len(srcs))
        infos = gp.gp_batch(dg, [gp.make_request(fn, int(s), param, 1e-4, ys[i]) for i, s in enumerate(srcs)])
        for i, s in enumerate(srcs):
            ystar = O.chebypower(g, int(s), KINDS[fn], param, 150)
            l1 = O.errors(g, ystar, ys[i].cpu().numpy())["l1"]
            assert l1 <= 1e-4, (i, l1, infos[i])
            assert infos[i]["k16_from"] <= infos[i]["K"]  # the 16-bit phase did run
    finally:
        dg.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_batch_narrow_16bit_block(gp, storage):
    """Eight columns per block: lanes own 8 columns and the FP32 -> 16-bit
    transition passes split a lane's Q_{k-1} segment into 4-column pieces."""
    g = graph("rmat14")
    st = {"bf16": gp.GP_BF16, "f16": gp.GP_F16}[storage]
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=8, storage=st)
    try:
        srcs = gg.sources(g, 12, 23)  # a block of 8, then a block of 4 (compacted to 8 columns)
        ys = _outputs(g, len(srcs))
        infos = gp.gp_batch(dg, _requests(gp, g, srcs, 1e-4, ys))
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            l1 = O.errors(g, O.chebypower(g, int(s), KINDS[fn], p, 150), ys[i].cpu().numpy())["l1"]
            assert l1 <= 1e-4, (i, storage, l1, infos[i])
    finally:
        dg.close()


def test_batch_host_outputs_and_isolated_source(gp):
    g = gg.from_edges(40, [(i, i + 1) for i in range(30)] + [(35, 36)], "path_with_isolated")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=8)
    try:
        ys = [np.zeros(g.n, dtype=np.float64) for _ in range(3)]
        ys.append(np.zeros(g.n, dtype=np.float32))
        reqs = [gp.make_request(0, 3, 0.2, 1e-8, ys[0]), gp.make_request(1, 33, 4.0, 1e-8, ys[1]),
                gp.make_request(0, 36, 0.3, 1e-8, ys[2]), gp.make_request(1, 10, 2.0, 1e-8, ys[3])]
        gp.gp_batch(dg, reqs)
        assert np.array_equal(ys[1], np.exp(-4.0) * O.unit_vector(g.n, 33))  # node 33 is isolated
        for y, (k, s, p) in ((ys[0], ("ppr", 3, 0.2)), (ys[2], ("ppr", 36, 0.3)), (ys[3], ("hkpr", 10, 2.0))):
            assert O.errors(g, O.chebypower(g, s, k, p, 200), y)["l1"] <= 1e-6
    finally:
        dg.close()


def _serve_all(gp, dg, reqs, timeout=120.0):
    tickets = [gp.gp_submit(dg, r) for r in reqs]
    infos = [None] * len(tickets)
    t0 = time.time()
    while any(i is None for i in infos):
        for j, t in enumerate(tickets):
            if infos[j] is None:
                infos[j] = gp.gp_poll(dg, t)
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.002)
    return infos


STORAGES = {"f32": 0, "bf16": 2, "f16": 3}


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_serving_matches_oracle_and_alone(gp, storage):
    """Continuous batching: 48 mixed requests through a 16-slot service, each
    within its tolerance of the oracle and the same alone as in the mix.  With
    16-bit storage the columns start in the FP32 block and move to the 16-bit
    block after their own warm-up when enough steps remain (k16_from <= K
    reports it)."""
    g = graph("rmat14")
    srcs = gg.sources(g, 48, 19)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=16,
                            storage=STORAGES[storage])
    try:
        ys = _outputs(g, len(srcs))
        reqs = []
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            tol = [1e-4, 1e-5, 1e-6][i % 3]
            reqs.append(gp.make_request(fn, int(s), p, tol, ys[i]))
        infos = _serve_all(gp, dg, reqs)
        stats = gp.gp_serve_stats(dg)
        assert stats["completed"] == len(srcs)
        assert stats["mean_active"] > 1.0  # the queries shared passes
        moved = sum(1 for i, inf in enumerate(infos) if inf["k16_from"] <= inf["K"])
        if storage == "f32":
            assert moved == 0
        else:  # columns past their warm-up, moved while requests wait and enough of them are eligible
            assert moved >= len(srcs) // 8, [(inf["K"], inf["k16_from"]) for inf in infos]
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            tol = [1e-4, 1e-5, 1e-6][i % 3]
            ystar = O.chebypower(g, int(s), KINDS[fn], p, 150)
            assert O.errors(g, ystar, ys[i].cpu().numpy())["l1"] <= tol, (i, infos[i])
        # the same query alone in the service gives the same vector, within the
        # query's tolerance (the pass width follows the load, and with it the
        # grouping of the FP32 neighbour sums of the longest rows)
        for i in (0, 7, 29):
            fn, p = MIX[i % len(MIX)]
            tol = [1e-4, 1e-5, 1e-6][i % 3]
            y1 = _outputs(g, 1)[0]
            info1 = _serve_all(gp, dg, [gp.make_request(fn, int(srcs[i]), p, tol, y1)])[0]
            assert abs(info1["K"] - infos[i]["K"]) <= 1
            assert O.errors(g, ys[i].cpu().numpy(), y1.cpu().numpy())["l1"] <= tol
            ystar = O.chebypower(g, int(srcs[i]), KINDS[fn], p, 150)
            assert O.errors(g, ystar, y1.cpu().numpy())["l1"] <= tol
    finally:
        dg.close()


def test_serving_16bit_moves_only_under_load(gp):
    """The 16-bit block of a service is used only while the FP32 block is
    busy: requests served one at a time stay in FP32 (k16_from = K + 1, one
    pass per iteration), and a burst of l1 1e-4 requests four times larger
    than the block moves columns past their warm-up into the FP16 block.
    Every result lies within its tolerance of the oracle."""
    g = graph("rmat14")
    srcs = [int(s) for s in gg.sources(g, 72, 29)]
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=16, storage=STORAGES["f16"])
    try:
        spec = [(MIX[i % len(MIX)][0], srcs[i], MIX[i % len(MIX)][1]) for i in range(72)]
        ys = _outputs(g, 72)
        alone = [_serve_all(gp, dg, [gp.make_request(fn, s, p, 1e-4, ys[i])])[0]
                 for i, (fn, s, p) in enumerate(spec[:8])]
        assert all(inf["k16_from"] == inf["K"] + 1 for inf in alone), [(inf["K"], inf["k16_from"]) for inf in alone]
        burst = _serve_all(gp, dg, [gp.make_request(fn, s, p, 1e-4, ys[8 + i]) for i, (fn, s, p) in
                                    enumerate(spec[8:])])
        moved = sum(1 for inf in burst if inf["k16_from"] <= inf["K"])
        assert moved >= len(burst) // 8, [(inf["K"], inf["k16_from"]) for inf in burst]
        for i, (fn, s, p) in enumerate(spec):
            ystar = O.chebypower(g, s, KINDS[fn], p, 150)
            assert O.errors(g, ystar, ys[i].cpu().numpy())["l1"] <= 1e-4, (i, (alone + burst)[i])
    finally:
        dg.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_serving_512_slots(gp, storage):
    """A 512-slot block (two 256-column engines; with BF16 storage two more
    16-bit ones): 320 queries at once fill both halves, and every result meets
    its tolerance."""
    g = graph("rmat14")
    srcs = gg.sources(g, 320, 23)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=512,
                            storage=STORAGES[storage])
    try:
        ys = _outputs(g, len(srcs))
        reqs = []
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            reqs.append(gp.make_request(fn, int(s), p, [1e-4, 1e-6][i % 2], ys[i]))
        _serve_all(gp, dg, reqs)
        stats = gp.gp_serve_stats(dg)
        assert stats["completed"] == len(srcs)
        assert stats["mean_active"] > 128
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            ystar = O.chebypower(g, int(s), KINDS[fn], p, 150)
            assert O.errors(g, ystar, ys[i].cpu().numpy())["l1"] <= [1e-4, 1e-6][i % 2], i
    finally:
        dg.close()


def test_serving_errors(gp):
    g = graph("er4096")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=8)
    try:
        import torch
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        with pytest.raises(gp.GPError) as ei:
            gp.gp_submit(dg, gp.make_request(0, g.n + 5, 0.2, 1e-6, y))
        assert ei.value.status == gp.GP_EINVAL
        with pytest.raises(gp.GPError) as ei:
            gp.gp_poll(dg, 987654321)
        assert ei.value.status == gp.GP_ENOTFOUND
        t = gp.gp_submit(dg, gp.make_request(1, 0, 5.0, 1e-6, y))
        info = None
        t0 = time.time()
        while info is None and time.time() - t0 < 60:
            info = gp.gp_poll(dg, t)
        assert info is not None and info["K"] > 0
        with pytest.raises(gp.GPError):  # collected tickets are gone
            gp.gp_poll(dg, t)
    finally:
        dg.close()


def test_destroy_with_pending_tickets(gp):
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=8)
    ys = _outputs(g, 30)
    for i, s in enumerate(gg.sources(g, 30, 3)):
        gp.gp_submit(dg, gp.make_request(0, int(s), 0.1, 1e-6, ys[i]))
    dg.close()  # must not hang or fault with work queued and in flight


def test_batch_profile_counts_passes(gp):
    """gp_profile_* time every SpMM pass of gp_batch and count its algorithmic bytes."""
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=16)
    try:
        srcs = gg.sources(g, 6, 31)
        ys = _outputs(g, len(srcs))
        K = 9
        reqs = [gp.make_request(0, int(s), 0.2, 1e-6, ys[i], k_rule=gp.GP_K_FIXED, k_fixed=K)
                for i, s in enumerate(srcs)]
        gp.gp_profile_enable(dg, True)
        gp.gp_profile_read(dg)
        gp.gp_batch(dg, reqs)
        prof = gp.gp_profile_read(dg)
        gp.gp_profile_enable(dg, False)
        # passes k = 1 .. K-1 compute r_2 .. r_K; the control kernel retires the
        # columns before the pass after the last, which still runs (empty)
        assert K - 1 <= prof["step_launches"] <= K + 4
        assert prof["step_ms"] > 0.0
        na = int((g.degree > 0).sum())
        per_pass_min = 4.0 * g.nnz + na * 8 * (4 + 4 + 4 + 8)  # the narrowest pass: 8 FP32 columns
        assert prof["step_bytes"] >= prof["step_launches"] * per_pass_min
    finally:
        dg.close()


def test_autotune_picks_a_candidate_and_batches_with_it(gp):
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, storage=gp.GP_BF16, autotune=1)
    try:
        r = gp.gp_autotune(dg, widths=[16, 32, 64])
        assert r["width"] in (16, 32, 64) and r["us_per_column_pass"] > 0.0
        d = gp.gp_autotune(dg)  # default candidates: measured once, then cached per graph structure
        assert d["width"] in (8, 16, 32, 64, 128, 256)
        assert d["t_heavy"] in (65, 129, 257, 509)
        assert gp.gp_autotune(dg) == d
        # another handle on the same graph structure reuses the cached choice
        dg2 = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, storage=gp.GP_BF16, autotune=1)
        try:
            assert gp.gp_autotune(dg2) == d
        finally:
            dg2.close()
        # gp_batch with block_width 0 and autotune runs at the tuned width and stays accurate
        srcs = gg.sources(g, 10, 41)
        ys = _outputs(g, len(srcs))
        infos = gp.gp_batch(dg, _requests(gp, g, srcs, 1e-4, ys))
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            l1 = O.errors(g, O.chebypower(g, int(s), KINDS[fn], p, 150), ys[i].cpu().numpy())["l1"]
            assert l1 <= 1e-4, (i, l1, infos[i])
        with pytest.raises(Exception):
            gp.gp_autotune(dg, widths=[48])  # not a power of two
    finally:
        dg.close()


def test_batch_unvalidated_asymmetric_csr(gp):
    """A CSR whose rows list nodes of degree 0 (asymmetric, symmetry check off):
    those neighbours contribute 0 (1/d := 0), in the batched kernel as in the
    oracle, through the kernel variant that checks gathered rows."""
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
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=16, validate_symmetry=0)
    try:
        srcs = [u for u in range(g.n) if g.degree[u] > 0][:6]
        ys = _outputs(g, len(srcs))
        K = 14
        reqs = [gp.make_request(0, int(s), 0.2, 1e-6, ys[i], k_rule=gp.GP_K_FIXED, k_fixed=K)
                for i, s in enumerate(srcs)]
        gp.gp_batch(dg, reqs)
        for i, s in enumerate(srcs):
            want = O.chebypower(g, int(s), "ppr", 0.2, K)
            e = O.errors(g, want, ys[i].cpu().numpy())
            assert e["l1"] <= 1e-6 and e["maxabs"] <= _fp32_maxabs_bar(want, K), (i, e)
    finally:
        dg.close()


@pytest.mark.parametrize("B", [8, 64])
def test_clenshaw_matches_forward_sum(gp, B):
    """Clenshaw's backward form evaluates the same truncated sum as Algorithm 3:
    each column equals the oracle's forward ChebyPower at its K (FP32 batched
    bar), for mixed functions, mixed K (1 and 2 included) and PAPER-rule K."""
    g = graph("rmat14")
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=B)
    try:
        srcs = list(gg.sources(g, 14, 43)) + [int(gg.top_degree_sources(g, 1)[0])]
        ys = _outputs(g, len(srcs))
        Ks = [1, 2] + [5 + 3 * (i % 8) for i in range(len(srcs) - 3)] + [0]
        reqs = []
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            if Ks[i] == 0:
                reqs.append(gp.make_request(fn, int(s), p, 1e-4, ys[i], k_rule=gp.GP_K_PAPER))
            else:
                reqs.append(gp.make_request(fn, int(s), p, 1e-6, ys[i], k_rule=gp.GP_K_FIXED, k_fixed=Ks[i]))
        infos = gp.gp_batch_clenshaw(dg, reqs)
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            K = infos[i]["K"]
            if Ks[i]:
                assert K == Ks[i]
            want = O.chebypower(g, int(s), KINDS[fn], p, K)
            e = O.errors(g, want, ys[i].cpu().numpy())
            assert e["l1"] <= 1e-6 and e["maxabs"] <= _fp32_maxabs_bar(want, K), (i, K, e)
        with pytest.raises(Exception):
            gp.gp_batch_clenshaw(dg, [gp.make_request(0, int(srcs[0]), 0.2, 1e-4, ys[0])])  # tail rule: no K up front
    finally:
        dg.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_propagate_matches_definition(gp, storage):
    """Z = f(D^-a A D^-b) X (a + b = 1) against the definition written out
    with dense matrices: alpha (I - (1-alpha) M)^-1 X for SSPPR, expm(-t (I - M)) X
    for HKPR, M = D^-a A D^-b with zero rows and columns at isolated nodes."""
    import torch
    scipy_linalg = pytest.importorskip("scipy.linalg")
    g = gg.rmat(9, 8, seed=3)
    n = g.n
    assert (g.degree == 0).any()
    A = np.zeros((n, n))
    for u in range(n):
        A[u, g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]] = 1.0
    d = g.degree.astype(np.float64)
    rng = np.random.default_rng(7)
    F = 12
    X = rng.standard_normal((n, F)).astype(np.float32)
    st = {"f32": gp.GP_F32, "bf16": gp.GP_BF16}[storage]
    tol = 1e-6 if storage == "f32" else 1e-4
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, storage=st, block_width=8)
    try:
        for fn, param in ((0, 0.2), (1, 4.0)):
            for a in (0.0, 0.5, 1.0):
                ds = np.where(d > 0, d, 1.0)
                dma = np.where(d > 0, ds ** -a, 0.0)
                dmb = np.where(d > 0, ds ** -(1.0 - a), 0.0)
                M = dma[:, None] * A * dmb[None, :]
                if fn == 0:
                    want = param * np.linalg.solve(np.eye(n) - (1 - param) * M, X.astype(np.float64))
                else:
                    want = scipy_linalg.expm(-param * (np.eye(n) - M)) @ X.astype(np.float64)
                Xd = torch.from_numpy(X).cuda()
                Zd = torch.empty_like(Xd)
                infos = gp.gp_propagate(dg, fn, param, a, Xd, Zd, tol)
                Z = Zd.cpu().numpy().astype(np.float64)
                for f in range(F):
                    scale = np.abs(ds ** a * X[:, f]).sum()
                    err = np.abs(Z[:, f] - want[:, f]).sum()
                    assert err <= 2 * tol * scale, (fn, a, f, err, scale, infos[f])
                iso = d == 0
                f0 = param if fn == 0 else np.exp(-param)
                assert np.allclose(Z[iso], f0 * X[iso].astype(np.float64), rtol=1e-6, atol=0)
        # host arrays give the same result (column norms are summed by float
        # atomics, so equal to rounding, not bit for bit)
        Zh = np.zeros_like(X)
        gp.gp_propagate(dg, 0, 0.2, 0.5, X, Zh, tol)
        Xd = torch.from_numpy(X).cuda()
        Zd = torch.empty_like(Xd)
        gp.gp_propagate(dg, 0, 0.2, 0.5, Xd, Zd, tol)
        assert np.allclose(Zh, Zd.cpu().numpy(), rtol=1e-4, atol=1e-6)
    finally:
        dg.close()


def test_serving_host_outputs_reuse_staging(gp):
    """Host outputs go through a few device staging buffers, reused as
    requests complete: 40 requests with numpy outputs at once, every result
    within its tolerance of the oracle."""
    g = graph("rmat14")
    srcs = gg.sources(g, 40, 31)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=16)
    try:
        outs = [np.full(g.n, np.nan) for _ in srcs]
        reqs = []
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            reqs.append(gp.make_request(fn, int(s), p, 1e-5, outs[i]))
        _serve_all(gp, dg, reqs)
        for i, s in enumerate(srcs):
            fn, p = MIX[i % len(MIX)]
            ystar = O.chebypower(g, int(s), KINDS[fn], p, 150)
            assert O.errors(g, ystar, outs[i])["l1"] <= 1e-5, i
    finally:
        dg.close()


def test_serving_request_ring_wraps(gp):
    """More requests than the device-side request ring holds (1024), all at
    once: the service publishes them as the ring drains, and every result is
    right (checked on a sample against the oracle, all against the isolated
    query's own K range)."""
    import torch
    g = graph("er4096")
    n_req = 1300
    srcs = [int(s) for s in gg.sources(g, 100, 37)]
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=64)
    try:
        ys = torch.empty((n_req, g.n), dtype=torch.float32, device="cuda")
        reqs = [gp.make_request(0, srcs[i % len(srcs)], 0.5, 1e-4, ys[i]) for i in range(n_req)]
        infos = _serve_all(gp, dg, reqs, timeout=300.0)
        assert gp.gp_serve_stats(dg)["completed"] >= n_req
        Y = ys.cpu().numpy().astype(np.float64)
        for i in (0, 511, 1023, 1024, 1299):
            ystar = O.chebypower(g, srcs[i % len(srcs)], "ppr", 0.5, 150)
            assert O.errors(g, ystar, Y[i])["l1"] <= 1e-4, (i, infos[i])
        for i in range(len(srcs), n_req):  # the same query gives the same vector
            assert np.abs(Y[i] - Y[i % len(srcs)]).sum() <= 1e-4
    finally:
        dg.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_serving_staggered_arrivals(gp, storage):
    """Requests arriving in waves while earlier ones are mid-flight join the
    running block (continuous batching on the device): mixed functions and
    tolerances on a Chung-Lu graph, every result within its tolerance of the
    oracle, and in FP32 each ticket's K within one step of the oracle's own
    stop."""
    g = graph("chunglu20k")
    srcs = [int(s) for s in gg.sources(g, 60, 43)]
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=32,
                            storage=STORAGES[storage])
    try:
        ys = _outputs(g, len(srcs))
        spec = []
        tickets = []
        for wave in range(6):
            for i in range(wave * 10, wave * 10 + 10):
                fn, p = MIX[i % len(MIX)]
                tol = [1e-4, 1e-5, 1e-6][i % 3]
                spec.append((fn, p, tol))
                tickets.append(gp.gp_submit(dg, gp.make_request(fn, srcs[i], p, tol, ys[i])))
            time.sleep(0.003)
        infos = [gp.gp_wait(dg, t, 120000.0) for t in tickets]
        for i, (fn, p, tol) in enumerate(spec):
            ystar = O.chebypower(g, srcs[i], KINDS[fn], p, 150)
            assert O.errors(g, ystar, ys[i].cpu().numpy())["l1"] <= tol, (i, infos[i])
            if storage == "f32":  # 16-bit terms move the measured norms, and with them K
                _, Ko, _ = O.chebypower_tol(g, srcs[i], KINDS[fn], p, tol)
                assert abs(infos[i]["K"] - Ko) <= 1, (i, infos[i], Ko)
    finally:
        dg.close()
