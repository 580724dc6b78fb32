"""Seeded synthetic graph and source generators (no part of the propagation method).

The graphs stand in for the paper's SNAP datasets (Table 1): Erdos-Renyi for the
small exact-parity case, R-MAT with (a, b, c) = (0.57, 0.19, 0.19) for the
power-law workloads, Chung-Lu for the serving workload.  Every output is a pure
function of its arguments (counter-based random numbers), so the oracle and the
CUDA library see the same arrays.  The C++ source is ``gen.cpp`` beside this file;
``build()`` compiles it with g++ into ``libgraphgen.so`` in this directory.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cpp")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.cpp into libgraphgen.so (skipped when the library is newer)."""
    import platform
    stamp = _LIB + ".machine"
    same = os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()
    if (not force and same and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
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
        i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        pp64 = ctypes.POINTER(ctypes.POINTER(i64))
        pp32 = ctypes.POINTER(ctypes.POINTER(i32))
        p64 = ctypes.POINTER(i64)
        lib.gg_er.argtypes = [i64, i64, u64, pp64, pp32, p64]
        lib.gg_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, pp64, pp32, p64]
        lib.gg_chung_lu.argtypes = [i64, dbl, dbl, dbl, u64, pp64, pp32, p64]
        for f in (lib.gg_er, lib.gg_rmat, lib.gg_chung_lu):
            f.restype = ctypes.c_int
        lib.gg_sources.argtypes = [i64, ctypes.c_void_p, i64, u64, ctypes.c_void_p]
        lib.gg_sources.restype = i64
        lib.gg_uniform.argtypes = [u64, u64, i64, ctypes.c_void_p]
        lib.gg_uniform.restype = None
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_free.restype = None
        lib.gg_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


class _Owned:
    """Keeps a malloc'd buffer alive while numpy views of it exist."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if self.ptr and _lib is not None:
            _lib.gg_free(self.ptr)
            self.ptr = None


def _view(ptr, count, ctype, dtype):
    owner = _Owned(ctypes.cast(ptr, ctypes.c_void_p).value)
    if count == 0:
        return np.zeros(0, dtype=dtype), owner
    buf = (ctype * count).from_address(owner.ptr)
    arr = np.frombuffer(buf, dtype=dtype, count=count)
    return arr, owner


class Graph:
    """Undirected simple graph in CSR form (both directions stored, rows sorted)."""

    def __init__(self, name, n, row_ptr, col_idx, owners=()):
        self.name = name
        self.n = int(n)
        self.row_ptr = row_ptr          # int64[n+1]
        self.col_idx = col_idx          # int32[nnz]
        self._owners = tuple(owners)
        self.nnz = int(row_ptr[-1])
        self.degree = np.diff(row_ptr).astype(np.int32)

    def row_ptr32(self) -> np.ndarray:
        if self.nnz > np.iinfo(np.int32).max:
            raise ValueError("nnz does not fit int32 row_ptr")
        return self.row_ptr.astype(np.int32)

    def digest(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.row_ptr).tobytes())
        h.update(np.ascontiguousarray(self.col_idx).tobytes())
        return h.hexdigest()

    def __repr__(self):
        return f"Graph({self.name}, n={self.n}, nnz={self.nnz})"


def _finish(name, n, rc, rp, ci, nnz):
    if rc != 0:
        raise RuntimeError(f"graph generator {name} failed with code {rc}")
    rpa, o1 = _view(rp, n + 1, ctypes.c_int64, np.int64)
    cia, o2 = _view(ci, nnz.value, ctypes.c_int32, np.int32)
    return Graph(name, n, rpa, cia, (o1, o2))


def erdos_renyi(n: int, m: int, seed: int) -> Graph:
    """G(n, m): m uniform endpoint pairs, self-loops and duplicates dropped."""
    lib = _load()
    rp, ci, nnz = ctypes.POINTER(ctypes.c_int64)(), ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()
    rc = lib.gg_er(n, m, seed, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz))
    return _finish(f"er_n{n}_m{m}_s{seed}", n, rc, rp, ci, nnz)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2) -> Graph:
    """R-MAT with 2^scale nodes and edge_factor * 2^scale edge draws, no noise."""
    lib = _load()
    n = 1 << scale
    rp, ci, nnz = ctypes.POINTER(ctypes.c_int64)(), ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()
    rc = lib.gg_rmat(scale, edge_factor * n, a, b, c, seed, ctypes.byref(rp), ctypes.byref(ci),
                     ctypes.byref(nnz))
    return _finish(f"rmat_s{scale}_ef{edge_factor}_seed{seed}", n, rc, rp, ci, nnz)


def chung_lu(n: int, mean_degree: float = 30.0, exponent: float = 2.1, i0: float = 0.0,
             seed: int = 4) -> Graph:
    """Chung-Lu power-law graph with expected degrees ~ (i+i0+1)^(-1/(exponent-1))."""
    lib = _load()
    rp, ci, nnz = ctypes.POINTER(ctypes.c_int64)(), ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()
    rc = lib.gg_chung_lu(n, mean_degree, exponent, i0, seed, ctypes.byref(rp), ctypes.byref(ci),
                         ctypes.byref(nnz))
    return _finish(f"chunglu_n{n}_d{mean_degree:g}_g{exponent:g}_seed{seed}", n, rc, rp, ci, nnz)


def from_edges(n: int, edges, name: str = "edges") -> Graph:
    """Small hand-written graphs: symmetrise, drop self-loops and duplicates, sort rows."""
    rows = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            rows[u].add(v)
            rows[v].add(u)
    rp = np.zeros(n + 1, dtype=np.int64)
    for u in range(n):
        rp[u + 1] = rp[u] + len(rows[u])
    ci = np.array([v for u in range(n) for v in sorted(rows[u])], dtype=np.int32)
    return Graph(name, n, rp, ci)


def complete(n: int) -> Graph:
    """The complete graph K_n (every pair of distinct nodes, both directions):
    n (n - 1) entries, so n >= 46342 passes 2^31 entries (int64 row offsets)."""
    rp = np.arange(n + 1, dtype=np.int64) * (n - 1)
    ci = np.empty(n * (n - 1), dtype=np.int32)
    j = np.arange(n - 1, dtype=np.int32)[None, :]
    step = max(1, (1 << 26) // max(n, 1))
    for u0 in range(0, n, step):
        u1 = min(n, u0 + step)
        u = np.arange(u0, u1, dtype=np.int32)[:, None]
        ci[u0 * (n - 1):u1 * (n - 1)] = (j + (j >= u)).ravel()  # row u: 0..u-1, u+1..n-1
    return Graph(f"complete_n{n}", n, rp, ci)


def sources(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct sources drawn uniformly among nodes with degree >= 1."""
    lib = _load()
    out = np.zeros(k, dtype=np.int32)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    got = lib.gg_sources(g.n, rp.ctypes.data, k, seed, out.ctypes.data)
    return out[:got]


def top_degree_sources(g: Graph, k: int) -> np.ndarray:
    """The k highest-degree nodes (ties broken by lower id), as in the query-distribution study."""
    order = np.lexsort((np.arange(g.n), -g.degree.astype(np.int64)))
    return order[:k].astype(np.int32)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Counter-based uniform doubles in [0, 1) (used for Poisson arrivals and parameter mixes)."""
    lib = _load()
    out = np.empty(count, dtype=np.float64)
    lib.gg_uniform(seed, stream, count, out.ctypes.data)
    return out


def num_threads() -> int:
    return int(_load().gg_num_threads())
