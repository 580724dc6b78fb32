"""Pins for the FP64 oracle: each test ties it to something other than itself.

The oracle is checked against closed forms the paper prints (Lemma 2 at
alpha = 0.2, the star-graph example of Section 4.2), library routines
(scipy's scaled Bessel function, Poisson pmf, dense solve / expm), spectral
closed forms of regular graphs, and identities that any correct
implementation satisfies (Property 1's column sums, reversibility, the
D^{-1/2}-weighted truncation bound).  Each is chosen so that a plausible
slip -- 1/pi vs 2/pi on c_0, A D^-1 vs D^-1 A, a dropped r_{k-1}, an
off-by-one in K -- fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_ppr_coefficients_alpha_02_exact():
    # Lemma 2 with alpha = 0.2: sqrt(2a - a^2) = 0.6, gamma = 0.2/0.6 = 1/3,
    # beta = (1 - 0.6)/0.8 = 1/2, so c_0 = 1/3 and c_k = (2/3) 2^-k.
    c = O.cheb_coeffs("ppr", 0.2, 40)
    want = np.array([1 / 3] + [(2 / 3) * 0.5 ** k for k in range(1, 41)])
    # 8192-node trapezoid sums round at the 1e-15 level; a formula slip is >= 1e-3.
    assert np.max(np.abs(c - want)) < 1e-14


@pytest.mark.parametrize("alpha", [0.01, 0.05, 0.1, 0.5, 0.9])
def test_ppr_coefficients_lemma2(alpha):
    # The quadrature of Lemma 1 against the closed form of Lemma 2 (an analytic
    # evaluation of the same integral, derived independently in the paper).
    K = 60
    c = O.cheb_coeffs("ppr", alpha, K, M=1 << 15)
    root = math.sqrt(2 * alpha - alpha * alpha)
    gamma = alpha / root
    beta = (1 - root) / (1 - alpha)
    want = np.array([gamma] + [2 * gamma * beta ** k for k in range(1, K + 1)])
    assert np.max(np.abs(c - want)) < 1e-13


@pytest.mark.parametrize("t", [0.5, 1.0, 3.0, 5.0, 10.0, 20.0, 40.0])
def test_hkpr_coefficients_bessel(t):
    # Lemma 3: c_0 = e^-t I_0(t), c_k = 2 e^-t I_k(t); scipy's ive(k, t) = e^-t I_k(t).
    special = pytest.importorskip("scipy.special")
    K = 50
    c = O.cheb_coeffs("hkpr", t, K)
    want = np.array([special.ive(0, t)] + [2 * special.ive(k, t) for k in range(1, K + 1)])
    assert np.max(np.abs(c - want)) < 1e-14


def test_hkpr_tabulated_bessel_values():
    # Tabulated modified Bessel values: e^-5 I_0(5) = 0.183541, 2 e^-5 I_1(5) = 0.327945
    # (six printed digits).
    c = O.cheb_coeffs("hkpr", 5.0, 2)
    assert abs(c[0] - 0.183541) < 5e-7
    assert abs(c[1] - 0.327945) < 5e-7


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("ppr", 0.05), ("hkpr", 5.0), ("hkpr", 20.0)])
def test_coefficients_reconstruct_f(kind, param):
    # sum_k c_k T_k(x) = f(x) on [-1, 1] (Lemma 1); at x = 1 this is sum c_k = 1 (Lemma 4's proof).
    K = 400
    c = O.cheb_coeffs(kind, param, K, M=1 << 14)
    theta = np.linspace(0, math.pi, 37)
    x = np.cos(theta)
    series = np.array([np.sum(c * np.cos(np.arange(K + 1) * th)) for th in theta])
    assert np.max(np.abs(series - O.gp_f(kind, param, x))) < 1e-12
    assert abs(c.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_taylor_coefficients(kind, param):
    stats = pytest.importorskip("scipy.stats")
    z = O.taylor_coeffs(kind, param, 400)
    if kind == "ppr":
        want = param * (1 - param) ** np.arange(400)
    else:
        want = stats.poisson.pmf(np.arange(400), param)
    assert np.max(np.abs(z - want)) < 1e-15
    assert abs(z.sum() - 1.0) < 1e-12


def _frac_vec(v):
    return np.array([float(Fraction(s)) for s in v])


def test_star_graph_worked_example():
    with open(os.path.join(GOLDEN, "star_chebyshev_basis.json")) as f:
        gold = json.load(f)
    g = gg.from_edges(gold["n"], gold["edges"])
    R = O.cheb_basis(g, gold["source"], 3)
    for k, v in gold["r"].items():
        assert np.max(np.abs(R[int(k)] - _frac_vec(v))) < 1e-15, k


def test_star_graph_truncated_sum():
    # Algorithm 3 with K = 1, 2, 3 on the star from v1: y_K = sum_{k<=K} c_k r_k with the
    # example's exact r_k and Lemma 2's coefficients at alpha = 0.2 (1/3, 1/3, 1/6, 1/12).
    with open(os.path.join(GOLDEN, "star_chebyshev_basis.json")) as f:
        gold = json.load(f)
    g = gg.from_edges(gold["n"], gold["edges"])
    c = [Fraction(1, 3), Fraction(1, 3), Fraction(1, 6), Fraction(1, 12)]
    r = [[Fraction(x) for x in gold["r"][str(k)]] for k in range(4)]
    for K in (1, 2, 3):
        want = np.array([float(sum(c[k] * r[k][u] for k in range(K + 1))) for u in range(4)])
        y = O.chebypower(g, gold["source"], "ppr", 0.2, K)
        assert np.max(np.abs(y - want)) < 1e-14, K  # quadrature-rounded c_k


def _cycle(n):
    return gg.from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def _cycle_closed_form(n, s, kind, param):
    # P of the cycle is symmetric circulant with eigenvalues cos(2 pi j / n) and
    # Fourier eigenvectors, so y(u) = (1/n) sum_j f(cos(2 pi j/n)) cos(2 pi j (u-s)/n).
    j = np.arange(n)
    lam = np.cos(2 * np.pi * j / n)
    fl = O.gp_f(kind, param, lam)
    u = np.arange(n)
    return np.array([np.sum(fl * np.cos(2 * np.pi * j * (uu - s) / n)) / n for uu in u])


@pytest.mark.parametrize("n", [64, 101])
@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("ppr", 0.5), ("hkpr", 5.0), ("hkpr", 3.0)])
def test_cycle_closed_form(n, kind, param):
    g = _cycle(n)
    s = 7
    want = _cycle_closed_form(n, s, kind, param)
    y_cheb = O.chebypower(g, s, kind, param, 120)
    y_pow = O.power(g, s, kind, param)
    y_dense = O.dense_gp(g, s, kind, param)
    for y in (y_cheb, y_pow, y_dense):
        assert np.max(np.abs(y - want)) < 1e-13


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_complete_graph_closed_form(kind, param):
    # K_n: P = (J - I)/(n-1) has eigenvalue 1 on the all-ones vector and -1/(n-1)
    # on its complement, so f(P) e_s = f(1) 1/n + f(-1/(n-1)) (e_s - 1/n).
    n = 33
    g = gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], "K33")
    s = 4
    es = O.unit_vector(n, s)
    want = O.gp_f(kind, param, 1.0) / n + O.gp_f(kind, param, -1.0 / (n - 1)) * (es - 1.0 / n)
    for y in (O.chebypower(g, s, kind, param, 60), O.power(g, s, kind, param),
              O.dense_gp(g, s, kind, param)):
        assert np.max(np.abs(y - want)) < 1e-14


def _small_graphs():
    return [gg.erdos_renyi(300, 1200, 5), gg.rmat(9, 16, seed=3), gg.chung_lu(400, 8.0, 2.1, seed=6)]


@pytest.mark.parametrize("gi", [0, 1, 2])
@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("ppr", 0.1), ("hkpr", 5.0), ("hkpr", 10.0)])
def test_dense_power_cheby_agree(gi, kind, param):
    g = _small_graphs()[gi]
    s = int(gg.sources(g, 1, 13)[0])
    y_dense = O.dense_gp(g, s, kind, param)
    y_pow = O.power(g, s, kind, param)
    y_cheb = O.chebypower(g, s, kind, param, 150)
    assert O.errors(g, y_dense, y_pow)["l1"] < 1e-12
    assert O.errors(g, y_dense, y_cheb)["l1"] < 1e-12
    # SSPPR / HKPR are probability vectors (column-stochastic P).
    assert abs(y_dense.sum() - 1.0) < 1e-12
    assert y_dense.min() > -1e-15


def test_property1_column_sums():
    # Property 1: sum_u T_k(P) e_s (u) = 1 for every k (P is column-stochastic).
    # With D^-1 A in place of A D^-1 the sums drift on a non-regular graph.
    g = gg.rmat(10, 16, seed=9)
    s = int(gg.sources(g, 1, 3)[0])
    R = O.cheb_basis(g, s, 40)
    assert np.max(np.abs(R.sum(axis=1) - 1.0)) < 1e-9


def test_reversibility():
    # (f(P))_{uv} = (d_u / d_v) (f(P))_{vu}: P = A D^-1 is similar to a symmetric matrix.
    g = gg.rmat(9, 16, seed=4)
    a, b = [int(x) for x in gg.sources(g, 2, 21)]
    for kind, param in (("ppr", 0.2), ("hkpr", 5.0)):
        ya = O.chebypower(g, a, kind, param, 150)
        yb = O.chebypower(g, b, kind, param, 150)
        assert abs(ya[b] / g.degree[b] - yb[a] / g.degree[a]) < 1e-14


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_truncation_bound(kind, param):
    # Theorem 1 in the norm where it is exact: D^{-1/2} T_k(P) D^{1/2} = T_k(A~) has
    # 2-norm <= 1, so ||D^{-1/2}(y - y_K)||_2 <= tail(K) ||D^{-1/2} e_s||_2 = tail(K)/sqrt(d_s).
    g = gg.rmat(10, 16, seed=5)
    s = int(gg.sources(g, 1, 8)[0])
    ystar = O.chebypower(g, s, kind, param, 200)
    c = O.cheb_coeffs(kind, param, 200)
    w = np.zeros(g.n)
    w[g.degree > 0] = 1.0 / np.sqrt(g.degree[g.degree > 0])
    for K in range(1, 40):
        yK = O.chebypower(g, s, kind, param, K)
        tail = np.abs(c[K + 1:]).sum()
        lhs = np.linalg.norm(w * (ystar - yK))
        assert lhs <= tail / math.sqrt(g.degree[s]) * (1 + 1e-9) + 1e-15


def test_isolated_source():
    # With 1/d := 0 an isolated source has r_k = T_k(0) e_s, so y -> f(0) e_s = zeta_0 e_s.
    g = gg.from_edges(6, [(0, 1), (1, 2), (2, 3)], "with_isolated")
    for kind, param in (("ppr", 0.2), ("hkpr", 5.0)):
        y = O.chebypower(g, 5, kind, param, 120)
        want = O.unit_vector(6, 5) * O.taylor_coeffs(kind, param, 1)[0]
        assert np.max(np.abs(y - want)) < 1e-14
        assert np.max(np.abs(O.dense_gp(g, 5, kind, param) - want)) < 1e-14


def test_degree_zero_column_is_zero():
    # Reading 1/d := 0 on a CSR that lists a node with an empty row (asymmetric,
    # accepted only with the symmetry check off).  Rows 0 -> {1, 2}, 1 -> {0},
    # 2 -> {}: d = (2, 1, 0) and P = A D^-1 = [[0, 1, 0], [1/2, 0, 0], [0, 0, 0]].
    g = gg.Graph("asym3", 3, np.array([0, 2, 3, 3], dtype=np.int64), np.array([1, 2, 0], dtype=np.int32))
    x = np.array([0.75, -1.5, 4.0])
    assert np.array_equal(O.P_apply(g, x), np.array([-1.5, 0.375, 0.0]))
    assert np.array_equal(O.P_apply(g, np.array([0.0, 0.0, 1.0])), np.zeros(3))


def test_stopping_rule_meets_l1():
    # The l1 stopping reading stops where tail(K) * max_l ||r_l||_1 <= tol, which bounds
    # ||y - y_K||_1 by the triangle inequality as long as later ||r_k||_1 stay below the max.
    g = gg.rmat(11, 16, seed=2)
    for s in gg.sources(g, 3, 5):
        for kind, param in (("ppr", 0.2), ("hkpr", 5.0)):
            ystar = O.chebypower(g, int(s), kind, param, 150)
            for tol in (1e-4, 1e-6, 1e-8):
                y, K, norms = O.chebypower_tol(g, int(s), kind, param, tol)
                assert O.errors(g, ystar, y)["l1"] <= tol
                yK = O.chebypower(g, int(s), kind, param, K)
                assert np.max(np.abs(yK - y)) < 1e-15


def test_stopping_rule_margin_covers_growing_norms():
    # On R-MAT 14 the norms ||r_k||_1 of this HKPR t = 3 query still grow after
    # the running-maximum rule would stop (K = 11, truncation 1.07e-6 > 1e-6):
    # the margin of 2 on the measured C keeps the truncation within tol.
    g = gg.rmat(14, 16, seed=2)
    s = int(gg.sources(g, 320, 23)[177])
    ystar = O.chebypower(g, s, "hkpr", 3.0, 150)
    y11 = O.chebypower(g, s, "hkpr", 3.0, 11)
    assert O.errors(g, ystar, y11)["l1"] > 1e-6  # where the rule without margin stops
    y, K, norms = O.chebypower_tol(g, s, "hkpr", 3.0, 1e-6)
    assert K == 12
    c = O.cheb_coeffs("hkpr", 3.0, 200)
    assert np.abs(c[12:]).sum() * norms.max() > 1e-6 / 2  # K = 11 fails the margin
    assert np.abs(c[13:]).sum() * norms.max() <= 1e-6 / 2
    assert O.errors(g, ystar, y)["l1"] <= 1e-6


def test_chebypower_norms_and_K1():
    g = gg.erdos_renyi(200, 800, 2)
    s = int(gg.sources(g, 1, 1)[0])
    c = O.cheb_coeffs("ppr", 0.2, 1)
    y, nr = O.chebypower(g, s, "ppr", 0.2, 1, return_norms=True)
    # K = 1: y = c_0 e_s + c_1 P e_s.
    want = c[0] * O.unit_vector(g.n, s) + c[1] * O.P_apply(g, O.unit_vector(g.n, s))
    assert np.max(np.abs(y - want)) < 1e-16
    assert abs(nr[0] - 1.0) < 1e-15 and abs(nr[1] - 1.0) < 1e-15


def test_error_metrics():
    g = gg.from_edges(3, [(0, 1), (1, 2)])
    e = O.errors(g, np.array([0.5, 0.25, 0.25]), np.array([0.4, 0.25, 0.35]))
    assert abs(e["l1"] - 0.2) < 1e-15
    assert abs(e["l2"] - math.sqrt(0.02)) < 1e-15
    assert abs(e["maxabs"] - 0.1) < 1e-15
    assert abs(e["degnorm"] - 0.1) < 1e-15  # d_0 = d_2 = 1


def test_thread_count_does_not_change_results():
    g = gg.rmat(12, 16, seed=1)
    s = int(gg.sources(g, 1, 4)[0])
    t0 = O.num_threads()
    try:
        O.set_threads(1)
        a = O.chebypower(g, s, "hkpr", 5.0, 20)
        O.set_threads(max(2, t0))
        b = O.chebypower(g, s, "hkpr", 5.0, 20)
    finally:
        O.set_threads(t0)
    assert np.array_equal(a, b)


def test_chebypush_worked_example():
    # Section 4 (ChebyPush), the illustrative example: the star v0 - {v1, v2, v3},
    # f = T_3 from s = v1, threshold 1/3.  The pushes it describes (v0 at k = 1,
    # v2 and v3 but not v1 at k = 2) are the decisions r^2 >= eps d (rule 1).
    # After k = 1: r_cur = [0, -1/3, 2/3, 2/3]; after k = 2: r^_3 = [5/3, 0, 0, 0].
    g = gg.from_edges(4, [(0, 1), (0, 2), (0, 3)], "star4")
    c = np.array([0.0, 0.0, 0.0, 1.0])
    eps = np.full(4, 1.0 / 3.0)
    _, r2 = O.chebypush(g, 1, "ppr", 0.2, 2, eps=eps, coeffs=c[:3], rule=1, return_r=True)
    assert np.allclose(r2, [0.0, -1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0], rtol=0, atol=1e-15)
    y3, r3 = O.chebypush(g, 1, "ppr", 0.2, 3, eps=eps, coeffs=c, rule=1, return_r=True)
    assert np.allclose(r3, [5.0 / 3.0, 0.0, 0.0, 0.0], rtol=0, atol=1e-15)
    assert np.array_equal(y3, np.zeros(4))  # c_0 = c_1 = c_2 = 0
    # the exact T_3(P) e_v1 is [1, 0, 0, 0]: the example's rounding of the recurrence
    assert np.allclose(O.cheb_basis(g, 1, 3)[3], [1.0, 0.0, 0.0, 0.0], atol=1e-15)


def test_chebypush_rule_of_the_algorithm_by_hand():
    # Algorithm 4's own test |r(u)| > eps_k d_u on the same star, eps = 0.4, f = T_3:
    # k = 1: r_cur = [1, 0, 0, 0]; the hub has |1| <= 0.4 * 3, so nothing is pushed
    #        and the swap gives r_cur = [0, -1, 0, 0], r_new = [1, 0, 0, 0];
    # k = 2: v1 has |-1| > 0.4 * 1: r_new(v0) += 2 * (-1) / 1 -> -1, r_cur(v1) -> 1;
    # after the swap r^_3 = [-1, 0, 0, 0].
    g = gg.from_edges(4, [(0, 1), (0, 2), (0, 3)], "star4")
    _, r3 = O.chebypush(g, 1, "ppr", 0.2, 3, eps=np.full(4, 0.4), coeffs=np.array([0.0, 0.0, 0.0, 1.0]),
                        rule=0, return_r=True)
    assert np.array_equal(r3, np.array([-1.0, 0.0, 0.0, 0.0]))


@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
def test_chebypush_without_pruning_is_chebypower(kind, param):
    # With every threshold 0, every node with r != 0 pushes: the subset recurrence
    # is the full recurrence, y = sum_{k<K} c_k r_k and r^_K = T_K(P) e_s.
    g = gg.erdos_renyi(300, 900, 5)
    s = int(np.nonzero(g.degree)[0][0])
    K = 18
    c = O.cheb_coeffs(kind, param, K)
    y, r = O.chebypush(g, s, kind, param, K, eps=np.zeros(K + 1), coeffs=c, rule=0, return_r=True)
    assert np.max(np.abs(y - O.chebypower(g, s, kind, param, K - 1, coeffs=c[:K]))) < 1e-13
    assert np.max(np.abs(r - O.cheb_basis(g, s, K)[K])) < 1e-12


@pytest.mark.parametrize("gi", [0, 1])
@pytest.mark.parametrize("kind,param", [("ppr", 0.2), ("hkpr", 5.0)])
@pytest.mark.parametrize("eps_a", [1e-3, 1e-5])
def test_chebypush_degree_normalised_bound(gi, kind, param, eps_a):
    # Theorem 3: max_u |y(u) - y^(u)| / d_u < eps_a once K makes the truncation
    # small (here tail(K-1) <= eps_a / 2: Algorithm 4 adds c_0 .. c_{K-1}).
    g = [gg.erdos_renyi(400, 1600, 3), gg.chung_lu(500, 8.0, 2.1, seed=9)][gi]
    s = int(np.argmax(g.degree))
    c = O.cheb_coeffs(kind, param, 200)
    tail = np.array([np.abs(c[k + 1:]).sum() for k in range(len(c))])
    K = 1 + int(np.nonzero(tail <= eps_a / 2)[0][0])
    yhat = O.chebypush(g, s, kind, param, K, eps_a=eps_a, coeffs=c[:K + 1])
    ystar = O.dense_gp(g, s, kind, param)
    d = np.maximum(g.degree, 1)
    assert np.max(np.abs(ystar - yhat) / d) < eps_a


def test_alpha_walk_endpoints_follow_ppr():
    # The node where an alpha-random walk from v stops is distributed as the SSPPR
    # vector pi_v (each step stops with probability alpha, else moves to a uniform
    # neighbour): the walk generator of Algorithm 5 against the dense solve.
    g = gg.from_edges(7, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 5), (5, 6), (6, 4)], "two_rings")
    v, alpha, N = 1, 0.3, 40000
    ends = np.bincount([O.alpha_walk(g, v, alpha, 11, j) for j in range(N)], minlength=g.n) / N
    want = O.dense_ppr(g, v, alpha)
    sd = np.sqrt(want * (1 - want) / N)
    assert np.all(np.abs(ends - want) <= 5 * sd + 1e-12)


def test_bidirectional_is_unbiased_and_meets_its_guarantee():
    # Algorithm 5: E[pi^] = pi_s (each walk from v adds r(v)/W_v at its end, so the
    # walks add r(v) pi_v in expectation, and pi_s = pi^_push + sum_v r(v) pi_v by
    # the residual invariant).  A rough push (eps_r = 1, delta = 0.5) leaves a large
    # residual; the mean over seeds converges to the dense solve.
    g = gg.erdos_renyi(120, 300, 7)
    s = int(np.argmax(g.degree))
    alpha = 0.2
    ystar = O.dense_ppr(g, s, alpha)
    runs = [O.bidirectional(g, s, alpha, 6, 1.0, 0.5, seed)[0] for seed in range(300)]
    mean = np.mean(runs, axis=0)
    sd = np.std(runs, axis=0) / np.sqrt(len(runs))
    assert np.std(runs, axis=0).max() > 1e-4  # the walks do change the estimate
    assert np.all(np.abs(mean - ystar) <= 5 * sd + 1e-12)
    # the (eps_r, delta) guarantee at eps_r = 0.5, delta = 0.01, one run
    y, walks = O.bidirectional(g, s, alpha, 20, 0.5, 0.01, 3)
    big = ystar > 0.01
    assert np.all(np.abs(y[big] - ystar[big]) < 0.5 * ystar[big])
    assert walks > 0
