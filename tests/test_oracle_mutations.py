"""Plant mistakes in a copy of the oracle (on the CPU) and check that the pins catch them.

Each mutant is oracle.c with one plausible slip; it is compiled into a scratch
directory and loaded through the same Python wrapper.  The pins used here are
the star-graph example of Section 4.2, Property 1's column sums, the cycle's
spectral closed form, Lemma 2 at alpha = 0.2 and the dense solve.
"""
import ctypes
import importlib.util
import math
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import graphgen as gg
import oracle as O

ORACLE_DIR = os.path.dirname(os.path.abspath(O.__file__))

MUTANTS = {
    # the l1 stop rule with the running maximum alone (no margin on C)
    "no_c_margin": ("tail[k] * OR_C_MARGIN * C > tol", "tail[k] * C > tol"),
    # alpha-walk: stops with probability 1 - alpha
    "walk_stop_flipped": ("if (u < alpha || d == 0) return v;", "if (u >= alpha || d == 0) return v;"),
    # Algorithm 5: the residual with the wrong sign of the (1 - alpha) P term
    "residual_sign": ("(y[u] - (1.0 - alpha) * pp[u]) / alpha", "(y[u] + (1.0 - alpha) * pp[u]) / alpha"),
    # ChebyPush: the pushed node keeps r instead of -r (Eq. subset-cheby-implement)
    "push_no_negation": ("      rcur[u] = -r;", "      rcur[u] = r;"),
    # ChebyPush: r(u)/d_u pushed instead of 2 r(u)/d_u
    "push_half": ("rnew[col_idx[e]] += 2.0 * r / d;", "rnew[col_idx[e]] += r / d;"),
    # ChebyPush: the threshold against eps_k without the degree
    "push_no_degree": ("fabs(r) > eps[k] * d", "fabs(r) > eps[k]"),
    # r_{k+1} = 2 P r_k + r_{k-1}
    "sign_of_rkm1": ("2.0 * pr[u] - r", "2.0 * pr[u] + r"),
    # D^-1 A instead of A D^-1 (divide by the row's degree)
    "row_degree": ("const double d = deg_of(row_ptr, v);", "const double d = deg_of(row_ptr, u);"),
    # c_0 with 2/pi like the other coefficients
    "c0_weight": ("c[k] = (k == 0 ? 1.0 : 2.0) / OR_PI * integral;", "c[k] = 2.0 / OR_PI * integral;"),
    # the last term c_K r_K dropped
    "drop_last_term": ("for (int64_t u = 0; u < n; ++u) y[u] += c[K] * rcur[u];\n  free(rprev); free(rcur); free(pr);\n  return 0;\n}\n\n/* Algorithm 4 (ChebyPush)",
                       "free(rprev); free(rcur); free(pr);\n  return 0;\n}\n\n/* Algorithm 4 (ChebyPush)"),
}


def _load_mutant(tmp_path, name):
    src = open(os.path.join(ORACLE_DIR, "oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, name
    d = tmp_path / name / "oracle"
    d.mkdir(parents=True)
    (d / "oracle.c").write_text(src.replace(old, new))  # every occurrence
    shutil.copy(os.path.join(ORACLE_DIR, "__init__.py"), d / "__init__.py")
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pins_hold(M):
    """True when every pin below holds for module M."""
    ok = True
    star = gg.from_edges(4, [(0, 1), (0, 2), (0, 3)])
    R = M.cheb_basis(star, 1, 3)
    ok &= np.allclose(R[2], [0, -1 / 3, 2 / 3, 2 / 3], atol=1e-14)
    ok &= np.allclose(R[3], [1, 0, 0, 0], atol=1e-14)
    # Algorithm 3 with K = 3 on the star: sum_k c_k r_k with the example's exact r_k.
    c3 = [1 / 3, 1 / 3, 1 / 6, 1 / 12]  # Lemma 2 at alpha = 0.2
    r = [[0, 1, 0, 0], [1, 0, 0, 0], [0, -1 / 3, 2 / 3, 2 / 3], [1, 0, 0, 0]]
    want3 = sum(ck * np.array(rk) for ck, rk in zip(c3, r))
    ok &= np.allclose(M.chebypower(star, 1, "ppr", 0.2, 3, coeffs=np.array(c3)), want3, atol=1e-15)
    g = gg.rmat(9, 16, seed=9)
    s = int(gg.sources(g, 1, 3)[0])
    ok &= bool(np.max(np.abs(M.cheb_basis(g, s, 20).sum(axis=1) - 1.0)) < 1e-9)
    c = M.cheb_coeffs("ppr", 0.2, 10)
    ok &= abs(c[0] - 1 / 3) < 1e-13 and abs(c[1] - 1 / 3) < 1e-13
    n = 64
    cyc = gg.from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    j = np.arange(n)
    fl = M.gp_f("ppr", 0.2, np.cos(2 * np.pi * j / n))
    want = np.array([np.sum(fl * np.cos(2 * np.pi * j * (u - 5) / n)) / n for u in range(n)])
    ok &= bool(np.max(np.abs(M.chebypower(cyc, 5, "ppr", 0.2, 80) - want)) < 1e-12)
    ok &= bool(np.max(np.abs(M.chebypower(g, s, "ppr", 0.2, 80) - M.dense_ppr(g, s, 0.2))) < 1e-12)
    # the stop rule's margin (a query whose ||r_k||_1 grows after the running-max stop)
    gm = gg.rmat(14, 16, seed=2)
    sm = int(gg.sources(gm, 320, 23)[177])
    ym, Km, _ = M.chebypower_tol(gm, sm, "hkpr", 3.0, 1e-6)
    ok &= Km == 12 and bool(np.abs(ym - M.chebypower(gm, sm, "hkpr", 3.0, 150)).sum() <= 1e-6)
    # ChebyPush: the worked example (Section 4) and Theorem 3's degree-normalised bound
    c3e = np.array([0.0, 0.0, 0.0, 1.0])
    _, r3 = M.chebypush(star, 1, "ppr", 0.2, 3, eps=np.full(4, 1 / 3), coeffs=c3e, rule=1, return_r=True)
    ok &= np.allclose(r3, [5 / 3, 0, 0, 0], atol=1e-15)
    _, r3b = M.chebypush(star, 1, "ppr", 0.2, 3, eps=np.full(4, 0.4), coeffs=c3e, rule=0, return_r=True)
    ok &= np.allclose(r3b, [-1, 0, 0, 0], atol=1e-15)
    gs = gg.erdos_renyi(200, 600, 3)
    sh = int(np.argmax(gs.degree))
    cc = M.cheb_coeffs("ppr", 0.2, 120)
    yh = M.chebypush(gs, sh, "ppr", 0.2, 60, eps_a=1e-4, coeffs=cc[:61])
    ok &= bool(np.max(np.abs(M.dense_ppr(gs, sh, 0.2) - yh) / np.maximum(gs.degree, 1)) < 1e-4)
    # alpha-walk endpoints follow PPR; Algorithm 5 is unbiased
    rings = gg.from_edges(7, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 5), (5, 6), (6, 4)])
    ends = np.bincount([M.alpha_walk(rings, 1, 0.3, 11, j) for j in range(20000)], minlength=7) / 20000
    want = M.dense_ppr(rings, 1, 0.3)
    ok &= bool(np.all(np.abs(ends - want) <= 5 * np.sqrt(want * (1 - want) / 20000) + 1e-12))
    ge = gg.erdos_renyi(120, 300, 7)
    se = int(np.argmax(ge.degree))
    runs = [M.bidirectional(ge, se, 0.2, 6, 1.0, 0.5, seed)[0] for seed in range(150)]
    mean, sd = np.mean(runs, axis=0), np.std(runs, axis=0) / np.sqrt(150)
    ok &= bool(np.all(np.abs(mean - M.dense_ppr(ge, se, 0.2)) <= 5 * sd + 1e-12))
    return bool(ok)


def test_unmutated_oracle_passes_pins():
    assert _pins_hold(O)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    M = _load_mutant(tmp_path, name)
    assert not _pins_hold(M), f"mutant {name} passed every pin"
