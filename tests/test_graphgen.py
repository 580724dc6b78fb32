"""The seeded generators produce simple undirected graphs, deterministically."""
import numpy as np
import pytest

import graphgen as gg


def _check_simple_undirected(g):
    rp, ci = g.row_ptr, g.col_idx
    assert rp[0] == 0 and rp[-1] == len(ci)
    assert np.all(np.diff(rp) >= 0)
    assert ci.min(initial=0) >= 0 and ci.max(initial=0) < g.n
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(rows == ci), "self-loop"
    # sorted, unique within each row
    same_row = rows[1:] == rows[:-1]
    assert np.all(ci[1:][same_row] > ci[:-1][same_row])
    # symmetric: the edge multiset equals its transpose
    fwd = rows.astype(np.int64) * g.n + ci
    bwd = ci.astype(np.int64) * g.n + rows
    assert np.array_equal(np.sort(fwd), np.sort(bwd))
    assert np.array_equal(g.degree, np.diff(rp))


@pytest.mark.parametrize("make", [
    lambda: gg.erdos_renyi(4096, 16384, 1),
    lambda: gg.rmat(12, 16, seed=2),
    lambda: gg.chung_lu(5000, 30.0, 2.1, seed=4),
])
def test_simple_undirected_and_deterministic(make):
    a, b = make(), make()
    _check_simple_undirected(a)
    assert a.digest() == b.digest()


def test_seed_changes_graph():
    assert gg.rmat(10, seed=1).digest() != gg.rmat(10, seed=2).digest()


def test_er_config1_shape():
    g = gg.erdos_renyi(4096, 16384, 1)
    assert g.n == 4096
    # 16384 draws, a few lost to self-loops and duplicates, both directions stored
    assert 2 * 16000 < g.nnz <= 2 * 16384
    assert g.degree[0] > 0


def test_rmat_power_law_skew():
    g = gg.rmat(14, 16, seed=2)
    d = g.degree
    # (a, b, c, d) = (0.57, 0.19, 0.19, 0.05): node 0 is the hub, many nodes isolated
    assert d[0] == d.max()
    assert d.max() > 50 * d[d > 0].mean()
    assert 0.1 < (d == 0).mean() < 0.6


def test_sources_are_distinct_non_isolated():
    g = gg.rmat(12, 16, seed=2)
    s = gg.sources(g, 64, 2)
    assert len(s) == 64 and len(set(s.tolist())) == 64
    assert np.all(g.degree[s] > 0)
    assert np.array_equal(s, gg.sources(g, 64, 2))
    top = gg.top_degree_sources(g, 10)
    assert np.all(np.diff(g.degree[top]) <= 0)


def test_uniform_stream():
    u = gg.uniform(5, 0, 100000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(u, gg.uniform(5, 0, 100000))
    assert not np.array_equal(u, gg.uniform(5, 1, 100000))


def test_from_edges():
    g = gg.from_edges(4, [(0, 1), (1, 0), (2, 2), (1, 3)])
    _check_simple_undirected(g)
    assert g.nnz == 4


def test_complete_graph_csr():
    g = gg.complete(7)
    assert g.nnz == 42 and (g.degree == 6).all()
    for u in range(7):
        row = g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]
        assert list(row) == [v for v in range(7) if v != u]
