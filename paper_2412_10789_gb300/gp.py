"""Thin ctypes binding of the C ABI in ``include/gp.h`` (argument marshalling only).

Every computation runs in ``libgpcheby.so``.  PyTorch supplies device memory
(the library's allocations go through torch's caching allocator) and streams
(torch's current stream at graph creation).  Loading fails loudly when the
compiled library is missing; there is no fallback.

The functions keep the C names: ``gp_graph_create``, ``gp_ppr``, ``gp_hkpr``,
``gp_query``, ``gp_power``, ``gp_batch``, ``gp_submit``, ``gp_poll``, ``gp_wait``,
``gp_graph_destroy`` and the helpers.  Vectors are torch tensors (CUDA tensors
for device buffers, CPU tensors -- ideally pinned -- for host buffers) or
numpy arrays for host inputs.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GP_LIB selects another build of the library (e.g. a variant from build.py).
LIB_PATH = os.environ.get("GP_LIB") or os.path.join(_HERE, "libgpcheby.so")

GP_OK, GP_EINVAL, GP_ENOMEM, GP_ECUDA, GP_EAGAIN, GP_ENOTFOUND, GP_ETIMEDOUT, GP_EBUSY, GP_ENOTSUP = range(9)
GP_F32, GP_F64, GP_BF16, GP_F16 = range(4)
GP_FN_PPR, GP_FN_HKPR = 0, 1
GP_K_TAIL, GP_K_PAPER, GP_K_FIXED = 0, 1, 2

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class gp_config(ctypes.Structure):
    _fields_ = [
        ("storage", ctypes.c_int),
        ("block_width", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("k_max", ctypes.c_int32),
        ("validate_symmetry", ctypes.c_int32),
        ("t_heavy", ctypes.c_int32),
        ("row_ptr_64", ctypes.c_int32),
        ("precise_rows", ctypes.c_int32),
        ("warmup_tail", ctypes.c_double),
        ("mem_budget", ctypes.c_size_t),
        ("alloc", _ALLOC_T),
        ("free", _FREE_T),
        ("alloc_ctx", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
    ]


class gp_query_info(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("k16_from", ctypes.c_int32),
        ("tail_bound", ctypes.c_double),
        ("max_r_l1", ctypes.c_double),
        ("ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gp_request(ctypes.Structure):
    _fields_ = [
        ("function", ctypes.c_int32),
        ("source", ctypes.c_int32),
        ("param", ctypes.c_double),
        ("l1_tol", ctypes.c_double),
        ("k_rule", ctypes.c_int32),
        ("k_fixed", ctypes.c_int32),
        ("out_dtype", ctypes.c_int32),
        ("y_on_device", ctypes.c_int32),
        ("y_out", ctypes.c_void_p),
    ]


class GPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def _status_name(s):
    names = ["GP_OK", "GP_EINVAL", "GP_ENOMEM", "GP_ECUDA", "GP_EAGAIN", "GP_ENOTFOUND", "GP_ETIMEDOUT",
             "GP_EBUSY", "GP_ENOTSUP"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def load_library():
    """Load libgpcheby.so (built by ``paper_2412_10789_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2412_10789_gb300.build.build() first "
                               "(the library has no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        pinfo = ctypes.POINTER(gp_query_info)
        sigs = {
            "gp_config_default": (None, [ctypes.POINTER(gp_config)]),
            "gp_graph_create": (ctypes.c_int, [i64, i64, vp, ctypes.c_int, vp, vp, ctypes.c_int,
                                               ctypes.POINTER(gp_config), ctypes.POINTER(vp)]),
            "gp_graph_destroy": (ctypes.c_int, [vp]),
            "gp_graph_info": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                             ctypes.POINTER(i64)]),
            "gp_graph_export": (ctypes.c_int, [vp, vp, vp, vp]),
            "gp_ppr": (ctypes.c_int, [vp, i32, dbl, dbl, ctypes.c_int, vp, ctypes.c_int, pinfo]),
            "gp_hkpr": (ctypes.c_int, [vp, i32, dbl, dbl, ctypes.c_int, vp, ctypes.c_int, pinfo]),
            "gp_query": (ctypes.c_int, [vp, ctypes.POINTER(gp_request), pinfo]),
            "gp_power": (ctypes.c_int, [vp, i32, i32, dbl, dbl, ctypes.c_int, vp, ctypes.c_int, pinfo]),
            "gp_batch": (ctypes.c_int, [vp, i32, ctypes.POINTER(gp_request), pinfo]),
            "gp_batch_clenshaw": (ctypes.c_int, [vp, i32, ctypes.POINTER(gp_request), pinfo]),
            "gp_propagate": (ctypes.c_int, [vp, i32, dbl, dbl, i32, vp, vp, ctypes.c_int, dbl, pinfo]),
            "gp_chebypush": (ctypes.c_int, [vp, i32, i32, dbl, dbl, i32, ctypes.c_int, vp, ctypes.c_int, pinfo]),
            "gp_ppr_bidirectional": (ctypes.c_int, [vp, i32, dbl, dbl, dbl, i32, u64, ctypes.c_int, vp,
                                                    ctypes.c_int, pinfo]),
            "gp_submit": (ctypes.c_int, [vp, ctypes.POINTER(gp_request), ctypes.POINTER(u64)]),
            "gp_poll": (ctypes.c_int, [vp, u64, pinfo]),
            "gp_wait": (ctypes.c_int, [vp, u64, dbl, pinfo]),
            "gp_serve_stats": (ctypes.c_int, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                              ctypes.POINTER(dbl)]),
            "gp_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(i32), i32, ctypes.POINTER(i32),
                                           ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
            "gp_launch_count": (u64, []),
            "gp_profile_enable": (ctypes.c_int, [vp, ctypes.c_int]),
            "gp_profile_read": (ctypes.c_int, [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64), ctypes.POINTER(dbl)]),
            "gp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "gp_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc != GP_OK:
        raise GPError(rc, _lib.gp_last_error().decode(errors="replace"))


def _ptr(x):
    """(address, on_device) of a torch tensor or numpy array (contiguous)."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be contiguous")
        return x.ctypes.data, 0
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(x)}")


def _out_dtype(y):
    if isinstance(y, np.ndarray):
        dt = y.dtype
        if dt == np.float64:
            return GP_F64
        if dt == np.float32:
            return GP_F32
    else:
        import torch
        if y.dtype == torch.float64:
            return GP_F64
        if y.dtype == torch.float32:
            return GP_F32
    raise ValueError("y_out must be float64 or float32")


class TorchAllocator:
    """Device allocations for the library from torch's caching allocator."""

    def __init__(self, stream=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream
        self.c_alloc = _ALLOC_T(self._alloc)
        self.c_free = _FREE_T(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return None

    def _free(self, ptr, ctx):
        if ptr:
            self._torch.cuda.caching_allocator_delete(ptr)


class Graph:
    """Handle of a gp_graph; frees the device graph on close()/destruction."""

    def __init__(self, handle, keepalive):
        self.handle = handle
        self._keepalive = keepalive
        n, nnz, na, md = (ctypes.c_int64() for _ in range(4))
        _check(_lib.gp_graph_info(handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(na), ctypes.byref(md)))
        self.n, self.nnz, self.n_active, self.max_degree = n.value, nnz.value, na.value, md.value
        self.storage = GP_F32

    def close(self):
        if self.handle:
            gp_graph_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def gp_config_default():
    lib = load_library()
    cfg = gp_config()
    lib.gp_config_default(ctypes.byref(cfg))
    return cfg


def gp_graph_create(n, row_ptr, col_idx, degree, cfg=None, use_torch_memory=True, stream=None, **options):
    """Create a device graph from CSR arrays (numpy / CPU tensors, or CUDA tensors).

    ``options`` set gp_config fields by name (k_max, t_light, t_heavy, storage, ...).
    """
    lib = load_library()
    if cfg is None:
        cfg = gp_config_default()
    for k, v in options.items():
        setattr(cfg, k, v)
    keep = []
    if use_torch_memory or stream is not None:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        cfg.stream = st.cuda_stream
        keep.append(st)
    if use_torch_memory:
        a = TorchAllocator(stream=keep[0] if keep else None)
        cfg.alloc = a.c_alloc
        cfg.free = a.c_free
        keep.append(a)
    rp_ptr, rp_dev = _ptr(row_ptr)
    ci_ptr, ci_dev = _ptr(col_idx)
    dg_ptr, dg_dev = _ptr(degree)
    if not (rp_dev == ci_dev == dg_dev):
        raise ValueError("row_ptr, col_idx and degree must all be on the host or all on the device")
    rp64 = 1 if (str(getattr(row_ptr, "dtype", "")).endswith("int64")) else 0
    nnz = int(col_idx.shape[0])
    h = ctypes.c_void_p()
    _check(lib.gp_graph_create(int(n), nnz, rp_ptr, rp64, ci_ptr, dg_ptr, rp_dev, ctypes.byref(cfg),
                               ctypes.byref(h)))
    keep.append(cfg)
    g = Graph(h, keep)
    g.storage = int(cfg.storage)
    return g


def gp_graph_destroy(g: Graph):
    if g.handle:
        h, g.handle = g.handle, None
        _check(_lib.gp_graph_destroy(h))


def gp_graph_export(g: Graph):
    rp = np.empty(g.n + 1, dtype=np.int64)
    ci = np.empty(max(g.nnz, 1), dtype=np.int32)
    dg = np.empty(g.n, dtype=np.int32)
    _check(_lib.gp_graph_export(g.handle, rp.ctypes.data, ci.ctypes.data, dg.ctypes.data))
    return rp, ci[: g.nnz], dg


def _query_call(fn, g, source, param, l1_tol, y_out, want_info):
    ptr, on_dev = _ptr(y_out)
    if int(y_out.shape[0]) != g.n:
        raise ValueError("y_out must have n elements")
    info = gp_query_info() if want_info else None
    _check(fn(g.handle, int(source), float(param), float(l1_tol), _out_dtype(y_out), ptr, on_dev,
              ctypes.byref(info) if info is not None else None))
    return info.as_dict() if info is not None else None


def gp_ppr(g: Graph, source, alpha, l1_tol, y_out, info=True):
    """SSPPR vector of `source` into y_out (n float64/float32, device or host)."""
    return _query_call(_lib.gp_ppr, g, source, alpha, l1_tol, y_out, info)


def gp_hkpr(g: Graph, source, t, l1_tol, y_out, info=True):
    """HKPR vector of `source` into y_out (n float64/float32, device or host)."""
    return _query_call(_lib.gp_hkpr, g, source, t, l1_tol, y_out, info)


def make_request(function, source, param, l1_tol, y_out, k_rule=GP_K_TAIL, k_fixed=0):
    ptr, on_dev = _ptr(y_out)
    r = gp_request()
    r.function = int(function)
    r.source = int(source)
    r.param = float(param)
    r.l1_tol = float(l1_tol)
    r.k_rule = int(k_rule)
    r.k_fixed = int(k_fixed)
    r.out_dtype = _out_dtype(y_out)
    r.y_on_device = on_dev
    r.y_out = ptr
    return r


def gp_query(g: Graph, function, source, param, l1_tol, y_out, k_rule=GP_K_TAIL, k_fixed=0, info=True):
    r = make_request(function, source, param, l1_tol, y_out, k_rule, k_fixed)
    inf = gp_query_info() if info else None
    _check(_lib.gp_query(g.handle, ctypes.byref(r), ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def gp_power(g: Graph, function, source, param, l1_tol, y_out, info=True):
    """GPU PwMethod baseline (Algorithm 1)."""
    ptr, on_dev = _ptr(y_out)
    inf = gp_query_info() if info else None
    _check(_lib.gp_power(g.handle, int(function), int(source), float(param), float(l1_tol), _out_dtype(y_out),
                         ptr, on_dev, ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def gp_batch(g: Graph, requests, info=True):
    """Run a list of gp_request (see make_request) as packed columns."""
    arr = (gp_request * len(requests))(*requests)
    infos = (gp_query_info * len(requests))() if info else None
    _check(_lib.gp_batch(g.handle, len(requests), arr, infos))
    return [i.as_dict() for i in infos] if infos is not None else None


def gp_batch_clenshaw(g: Graph, requests, info=True):
    """The same packed columns in Clenshaw's backward form (K fixed up front)."""
    arr = (gp_request * len(requests))(*requests)
    infos = (gp_query_info * len(requests))() if info else None
    _check(_lib.gp_batch_clenshaw(g.handle, len(requests), arr, infos))
    return [i.as_dict() for i in infos] if infos is not None else None


def gp_propagate(g: Graph, function, param, a, X, Z, l1_tol, info=True):
    """Z = f(D^-a A D^-b) X for an n x F row-major float32 X (numpy or torch, host or CUDA)."""
    for m in (X, Z):
        if str(m.dtype) not in ("float32", "torch.float32") or len(m.shape) != 2:
            raise ValueError("X and Z must be n x F float32 arrays")
    xp, xd = _ptr(X)
    zp, zd = _ptr(Z)
    if xd != zd:
        raise ValueError("X and Z must both be on the host or both on the device")
    F = int(X.shape[1])
    infos = (gp_query_info * F)() if info else None
    _check(_lib.gp_propagate(g.handle, int(function), float(param), float(a), F, xp, zp, xd, float(l1_tol), infos))
    return [i.as_dict() for i in infos] if infos is not None else None


def gp_chebypush(g: Graph, function, source, param, eps_a, y_out, K=0, info=True):
    """ChebyPush (Algorithm 4) from one source; K = 0 picks K from eps_a."""
    ptr, on_dev = _ptr(y_out)
    inf = gp_query_info() if info else None
    _check(_lib.gp_chebypush(g.handle, int(function), int(source), float(param), float(eps_a), int(K),
                             _out_dtype(y_out), ptr, on_dev, ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def gp_ppr_bidirectional(g: Graph, source, alpha, eps_r, delta, y_out, K=0, seed=0, info=True):
    """Algorithm 5 (ChebyPush + alpha-random walks) for SSPPR."""
    ptr, on_dev = _ptr(y_out)
    inf = gp_query_info() if info else None
    _check(_lib.gp_ppr_bidirectional(g.handle, int(source), float(alpha), float(eps_r), float(delta), int(K),
                                     int(seed), _out_dtype(y_out), ptr, on_dev,
                                     ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def gp_submit(g: Graph, request: gp_request) -> int:
    t = ctypes.c_uint64()
    _check(_lib.gp_submit(g.handle, ctypes.byref(request), ctypes.byref(t)))
    return t.value


def gp_poll(g: Graph, ticket: int):
    """Return the info dict when done, None while GP_EAGAIN; raise on other errors."""
    inf = gp_query_info()
    rc = _lib.gp_poll(g.handle, ctypes.c_uint64(ticket), ctypes.byref(inf))
    if rc == GP_EAGAIN:
        return None
    _check(rc)
    return inf.as_dict()


def gp_wait(g: Graph, ticket: int, timeout_ms: float):
    """Block until the ticket completes (info dict) or timeout_ms passes
    (GPError with GP_ETIMEDOUT); other errors raise as well."""
    inf = gp_query_info()
    _check(_lib.gp_wait(g.handle, ctypes.c_uint64(ticket), float(timeout_ms), ctypes.byref(inf)))
    return inf.as_dict()


def gp_serve_stats(g: Graph):
    c, s, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    _check(_lib.gp_serve_stats(g.handle, ctypes.byref(c), ctypes.byref(s), ctypes.byref(m)))
    return {"completed": c.value, "steps": s.value, "mean_active": m.value}


def gp_launch_count() -> int:
    return int(load_library().gp_launch_count())


def gp_profile_enable(g: Graph, on: bool = True):
    _check(_lib.gp_profile_enable(g.handle, 1 if on else 0))


def gp_autotune(g: Graph, storage=None, widths=None):
    """Block width and chunked-row degree threshold with the least device time
    per column and pass on this graph."""
    lib = load_library()
    st = g.storage if storage is None else storage
    arr = (ctypes.c_int32 * len(widths))(*widths) if widths else None
    best, th, us = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(lib.gp_autotune(g.handle, int(st), arr, len(widths) if widths else 0, ctypes.byref(best),
                           ctypes.byref(th), ctypes.byref(us)))
    return {"width": best.value, "t_heavy": th.value, "us_per_column_pass": us.value}


def gp_profile_read(g: Graph):
    ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(_lib.gp_profile_read(g.handle, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)))
    return {"step_ms": ms.value, "step_launches": n.value, "step_bytes": b.value}


def gp_status_string(s: int) -> str:
    return load_library().gp_status_string(int(s)).decode()


def gp_last_error() -> str:
    return load_library().gp_last_error().decode(errors="replace")
