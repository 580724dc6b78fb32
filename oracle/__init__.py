"""FP64 CPU oracle for ChebyPower (arXiv 2412.10789) -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2412_10789_gb300``) and never imports it.

* ``oracle.c`` (compiled by :func:`build`) holds the sparse algorithms written
  from the paper: Taylor and Chebyshev coefficients (Def. SSPPR/HKPR, Lemma 1),
  P = A D^-1 applied in pull form, Algorithm 1 (PwMethod), Algorithm 3
  (ChebyPower) with a fixed K or with the l1 stopping reading, the Chebyshev
  basis r_k = T_k(P) x, and the error measures.
* This file adds the dense definitions for small graphs: the SSPPR vector
  alpha (I - (1-alpha) P)^-1 e_s (Def. SSPPR) by a linear solve, and the HKPR
  vector e^{-t(I-P)} e_s (Def. HKPR) by a matrix exponential.

Everything is float64.  Graph arguments are any object with ``n``,
``row_ptr`` (int64[n+1]) and ``col_idx`` (int32[nnz]).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

PPR = 0
HKPR = 1
KINDS = {"ppr": PPR, "hkpr": HKPR}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (plain C, no FMA contraction) into liboracle.so."""
    import platform
    stamp = _LIB + ".machine"
    same = os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()
    if (not force and same and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    with open(stamp, "w") as f:
        f.write(platform.machine() + "\n")
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, ci, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_num_threads.restype = ci
        lib.or_set_threads.argtypes = [ci]
        lib.or_set_threads.restype = None
        lib.or_taylor_coeffs.argtypes = [ci, dbl, ci, vp]
        lib.or_taylor_coeffs.restype = None
        lib.or_cheb_coeffs.argtypes = [ci, dbl, ci, ci, vp]
        lib.or_cheb_coeffs.restype = None
        lib.or_P_apply.argtypes = [i64, vp, vp, vp, vp]
        lib.or_P_apply.restype = None
        lib.or_power.argtypes = [i64, vp, vp, vp, vp, ci, vp]
        lib.or_power.restype = ci
        lib.or_chebypower.argtypes = [i64, vp, vp, vp, vp, ci, vp, vp]
        lib.or_chebypower.restype = ci
        lib.or_chebypower_tol.argtypes = [i64, vp, vp, vp, vp, ci, dbl, vp, vp, vp]
        lib.or_chebypower_tol.restype = ci
        lib.or_cheb_basis.argtypes = [i64, vp, vp, vp, ci, vp]
        lib.or_chebypush.argtypes = [i64, vp, vp, i64, vp, ci, vp, ci, vp, vp]
        lib.or_chebypush.restype = ci
        lib.or_bidirectional.argtypes = [i64, vp, vp, i64, dbl, vp, ci, dbl, dbl, ctypes.c_uint64, vp, vp]
        lib.or_bidirectional.restype = ci
        lib.or_walk_seed.argtypes = [ctypes.c_uint64, i64, i64]
        lib.or_walk_seed.restype = ctypes.c_uint64
        lib.or_alpha_walk.argtypes = [vp, vp, i64, dbl, ctypes.c_uint64]
        lib.or_alpha_walk.restype = i64
        lib.or_cheb_basis.restype = ci
        lib.or_errors.argtypes = [i64, vp, vp, vp, vp]
        lib.or_errors.restype = None
        _lib = lib
        return lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_threads(t: int) -> None:
    _load().or_set_threads(int(t))


def _kind(kind) -> int:
    return KINDS[kind] if isinstance(kind, str) else int(kind)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    return rp, ci


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def unit_vector(n: int, s: int) -> np.ndarray:
    e = np.zeros(n, dtype=np.float64)
    e[s] = 1.0
    return e


# ---------------------------------------------------------------- coefficients

def taylor_coeffs(kind, param: float, N: int) -> np.ndarray:
    """zeta_0..zeta_{N-1}: alpha(1-alpha)^k (Def. SSPPR) or e^-t t^k/k! (Def. HKPR)."""
    out = np.zeros(N, dtype=np.float64)
    _load().or_taylor_coeffs(_kind(kind), float(param), int(N), out.ctypes.data)
    return out


def cheb_coeffs(kind, param: float, K: int, M: int = 8192) -> np.ndarray:
    """c_0..c_K of Lemma 1 by trapezoid quadrature of (2/pi) int_0^pi f(cos t) cos(kt) dt."""
    if M < 4 * (K + 1):
        raise ValueError("quadrature needs M well above K")
    out = np.zeros(K + 1, dtype=np.float64)
    _load().or_cheb_coeffs(_kind(kind), float(param), int(K), int(M), out.ctypes.data)
    return out


def gp_f(kind, param: float, x):
    """The GP function on [-1, 1]: alpha/(1-(1-alpha)x) or exp(-t(1-x))."""
    x = np.asarray(x, dtype=np.float64)
    if _kind(kind) == PPR:
        return param / (1.0 - (1.0 - param) * x)
    return np.exp(-param * (1.0 - x))


def ground_truth_steps(kind, param: float) -> int:
    """Truncation used for the paper's ground truth (Section 6): N = ln(1e20)/alpha
    for SSPPR and N = 2 t ln(1e20) for HKPR (natural logarithm)."""
    if _kind(kind) == PPR:
        return int(math.ceil(math.log(1e20) / param))
    return int(math.ceil(2.0 * param * math.log(1e20)))


# ---------------------------------------------------------------- sparse algorithms

def P_apply(g, x: np.ndarray) -> np.ndarray:
    rp, ci = _csr(g)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(g.n, dtype=np.float64)
    _load().or_P_apply(g.n, rp.ctypes.data, ci.ctypes.data, x.ctypes.data, y.ctypes.data)
    return y


def power(g, s_or_x, kind, param: float, N: int | None = None) -> np.ndarray:
    """Algorithm 1 (PwMethod) with N Taylor terms (default: the ground-truth N)."""
    if N is None:
        N = ground_truth_steps(kind, param)
    x = unit_vector(g.n, s_or_x) if np.isscalar(s_or_x) else np.ascontiguousarray(s_or_x, np.float64)
    zeta = taylor_coeffs(kind, param, N)
    rp, ci = _csr(g)
    y = np.empty(g.n, dtype=np.float64)
    _check(_load().or_power(g.n, rp.ctypes.data, ci.ctypes.data, x.ctypes.data, zeta.ctypes.data,
                            int(N), y.ctypes.data), "power")
    return y


def chebypower(g, s_or_x, kind, param: float, K: int, coeffs: np.ndarray | None = None,
               return_norms: bool = False):
    """Algorithm 3 (ChebyPower) with a fixed truncation K >= 1."""
    c = cheb_coeffs(kind, param, K) if coeffs is None else np.ascontiguousarray(coeffs, np.float64)
    x = unit_vector(g.n, s_or_x) if np.isscalar(s_or_x) else np.ascontiguousarray(s_or_x, np.float64)
    rp, ci = _csr(g)
    y = np.empty(g.n, dtype=np.float64)
    nr = np.zeros(K + 1, dtype=np.float64)
    _check(_load().or_chebypower(g.n, rp.ctypes.data, ci.ctypes.data, x.ctypes.data, c.ctypes.data,
                                 int(K), y.ctypes.data, nr.ctypes.data), "chebypower")
    return (y, nr) if return_norms else y


def chebypower_tol(g, s_or_x, kind, param: float, tol: float, Kmax: int = 200):
    """Algorithm 3 stopping at the smallest K with tail(K) * 2 max_{l<=K} ||r_l||_1 <= tol.

    Returns (y, K, norms[0..K])."""
    c = cheb_coeffs(kind, param, Kmax)
    x = unit_vector(g.n, s_or_x) if np.isscalar(s_or_x) else np.ascontiguousarray(s_or_x, np.float64)
    rp, ci = _csr(g)
    y = np.empty(g.n, dtype=np.float64)
    nr = np.zeros(Kmax + 1, dtype=np.float64)
    K = ctypes.c_int(0)
    _check(_load().or_chebypower_tol(g.n, rp.ctypes.data, ci.ctypes.data, x.ctypes.data,
                                     c.ctypes.data, int(Kmax), float(tol), y.ctypes.data,
                                     ctypes.byref(K), nr.ctypes.data), "chebypower_tol")
    return y, int(K.value), nr[: K.value + 1].copy()


def chebypush_eps(c: np.ndarray, K: int, eps_a: float) -> np.ndarray:
    """The thresholds of Algorithm 4: eps_k = eps_a / (4 K sum_{l=k}^K |c_l|), k = 1..K-1 (index 0 unused)."""
    eps = np.zeros(K + 1, dtype=np.float64)
    for k in range(1, K):
        eps[k] = eps_a / (4.0 * K * np.abs(c[k:K + 1]).sum())
    return eps


def chebypush(g, s: int, kind, param: float, K: int, eps_a: float | None = None, eps=None, coeffs=None,
              rule: int = 0, return_r: bool = False):
    """Algorithm 4 (ChebyPush) with truncation K: y = c_0 e_s + sum_{k=1}^{K-1} c_k r^_k|S_k.

    Thresholds: eps_a (the algorithm's eps_k), or an explicit eps[0..K] array.
    rule 0 pushes u when |r(u)| > eps_k d_u (the algorithm), rule 1 when
    r(u)^2 >= eps_k d_u (the decisions of the paper's worked example)."""
    c = cheb_coeffs(kind, param, K) if coeffs is None else np.ascontiguousarray(coeffs, np.float64)
    if eps is None:
        eps = chebypush_eps(c, K, eps_a)
    eps = np.ascontiguousarray(eps, np.float64)
    rp, ci = _csr(g)
    y = np.empty(g.n, dtype=np.float64)
    r = np.empty(g.n, dtype=np.float64)
    _check(_load().or_chebypush(g.n, rp.ctypes.data, ci.ctypes.data, int(s), c.ctypes.data, int(K),
                                eps.ctypes.data, int(rule), y.ctypes.data, r.ctypes.data), "chebypush")
    return (y, r) if return_r else y


def bidirectional(g, s: int, alpha: float, K: int, eps_r: float, delta: float, seed: int, coeffs=None):
    """Algorithm 5 (ChebyPush + alpha-random walks) for SSPPR; returns (pi^, number of walks)."""
    c = cheb_coeffs("ppr", alpha, K) if coeffs is None else np.ascontiguousarray(coeffs, np.float64)
    rp, ci = _csr(g)
    y = np.empty(g.n, dtype=np.float64)
    walks = ctypes.c_int64(0)
    _check(_load().or_bidirectional(g.n, rp.ctypes.data, ci.ctypes.data, int(s), float(alpha), c.ctypes.data, int(K),
                                    float(eps_r), float(delta), ctypes.c_uint64(seed), y.ctypes.data,
                                    ctypes.byref(walks)), "bidirectional")
    return y, int(walks.value)


def alpha_walk(g, v: int, alpha: float, seed: int, j: int) -> int:
    """The node where walk j from v stops (the generator of or_bidirectional)."""
    rp, ci = _csr(g)
    lib = _load()
    return int(lib.or_alpha_walk(rp.ctypes.data, ci.ctypes.data, int(v), float(alpha),
                                 lib.or_walk_seed(ctypes.c_uint64(seed), int(v), int(j))))


def cheb_basis(g, s_or_x, K: int) -> np.ndarray:
    """Rows r_0..r_K of the Chebyshev recurrence r_k = T_k(P) x."""
    x = unit_vector(g.n, s_or_x) if np.isscalar(s_or_x) else np.ascontiguousarray(s_or_x, np.float64)
    rp, ci = _csr(g)
    R = np.empty((K + 1, g.n), dtype=np.float64)
    _check(_load().or_cheb_basis(g.n, rp.ctypes.data, ci.ctypes.data, x.ctypes.data, int(K),
                                 R.ctypes.data), "cheb_basis")
    return R


def errors(g, y: np.ndarray, yh: np.ndarray) -> dict:
    """l1, l2, degree-normalised (max |y-yh|/d_u over d_u >= 1) and max-abs errors."""
    rp, _ = _csr(g)
    y = np.ascontiguousarray(y, dtype=np.float64)
    yh = np.ascontiguousarray(yh, dtype=np.float64)
    out = np.zeros(4, dtype=np.float64)
    _load().or_errors(g.n, rp.ctypes.data, y.ctypes.data, yh.ctypes.data, out.ctypes.data)
    return {"l1": out[0], "l2": out[1], "degnorm": out[2], "maxabs": out[3]}


# ---------------------------------------------------------------- dense definitions

def dense_P(g) -> np.ndarray:
    """P = A D^-1 as a dense matrix, with zero columns for isolated nodes."""
    n = g.n
    A = np.zeros((n, n), dtype=np.float64)
    rp, ci = _csr(g)
    rows = np.repeat(np.arange(n), np.diff(rp))
    A[rows, ci] = 1.0
    d = A.sum(axis=0)
    inv = np.zeros(n)
    inv[d > 0] = 1.0 / d[d > 0]
    return A * inv[None, :]


def dense_ppr(g, s: int, alpha: float, P: np.ndarray | None = None) -> np.ndarray:
    """Def. SSPPR: pi_s = alpha (I - (1-alpha) P)^-1 e_s, by a dense solve."""
    P = dense_P(g) if P is None else P
    M = np.eye(g.n) - (1.0 - alpha) * P
    return np.linalg.solve(M, alpha * unit_vector(g.n, s))


def dense_hkpr(g, s: int, t: float, P: np.ndarray | None = None) -> np.ndarray:
    """Def. HKPR: rho_s = exp(-t (I - P)) e_s, by a dense matrix exponential."""
    from scipy.linalg import expm
    P = dense_P(g) if P is None else P
    E = expm(-t * (np.eye(g.n) - P))
    return E[:, s].copy()


def dense_gp(g, s: int, kind, param: float, P: np.ndarray | None = None) -> np.ndarray:
    return dense_ppr(g, s, param, P) if _kind(kind) == PPR else dense_hkpr(g, s, param, P)
