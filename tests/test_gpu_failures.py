"""Failure paths injected on the host (no GPU fault): an allocator callback
that returns NULL at graph creation and inside the running service, a
non-monotone row_ptr, and a bounded wait that runs out (GP_ETIMEDOUT).

Every failure must come back as a status, leave no device allocation behind,
and leave the CUDA context usable.
"""
import ctypes
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch
    from paper_2412_10789_gb300 import build, gp as gpmod
    build.build()
    assert torch.cuda.is_available()
    return gpmod


class FailingAllocator:
    """Device memory from torch's caching allocator that returns NULL once
    `budget` more allocations have been served (None: never), and counts the
    allocations still outstanding."""

    def __init__(self, gp, budget=None):
        import torch
        self.torch = torch
        self.budget = budget
        self.live = set()
        self.failed = 0
        self.c_alloc = gp._ALLOC_T(self._alloc)
        self.c_free = gp._FREE_T(self._free)

    def _alloc(self, nbytes, ctx):
        if self.budget is not None:
            if self.budget <= 0:
                self.failed += 1
                return None
            self.budget -= 1
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), self.torch.cuda.current_device())
        self.live.add(p)
        return p

    def _free(self, ptr, ctx):
        if ptr:
            self.live.discard(ptr)
            self.torch.cuda.caching_allocator_delete(ptr)

    def config(self, gp, **opt):
        cfg = gp.gp_config_default()
        cfg.alloc = self.c_alloc
        cfg.free = self.c_free
        for k, v in opt.items():
            setattr(cfg, k, v)
        return cfg


def _create(gp, g, alloc, **opt):
    return gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, cfg=alloc.config(gp, **opt),
                              use_torch_memory=False)


def test_allocator_null_at_graph_create(gp):
    """NULL from the k-th allocation of gp_graph_create, for every k the
    creation reaches: GP_ENOMEM, nothing left allocated, and the next creation
    with a working allocator answers queries correctly."""
    import torch
    g = gg.rmat(12, 16, seed=2)
    counter = FailingAllocator(gp)
    dg = _create(gp, g, counter)
    dg.close()
    assert not counter.live
    k = 0
    while True:
        fa = FailingAllocator(gp, budget=k)
        try:
            dg = _create(gp, g, fa)
        except gp.GPError as e:
            assert e.status == gp.GP_ENOMEM, e
            assert fa.failed == 1 and not fa.live, (k, len(fa.live))
            k += 1
            continue
        dg.close()
        assert not fa.live
        break
    assert k >= 3  # the creation allocates several buffers; each failure point was reached
    ok = FailingAllocator(gp)
    dg = _create(gp, g, ok)
    try:
        s = int(gg.sources(g, 1, 3)[0])
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        gp.gp_query(dg, 0, s, 0.2, 1e-6, y, k_rule=gp.GP_K_FIXED, k_fixed=20)
        e = O.errors(g, O.chebypower(g, s, "ppr", 0.2, 20), y.cpu().numpy())
        assert e["l1"] <= 1e-6 and e["maxabs"] <= 1e-8, e
    finally:
        dg.close()
    assert not ok.live


def test_allocator_null_inside_the_running_service(gp):
    """The service allocates a host-output staging buffer when it first hands
    a request with a host output to the device.  With the allocator failing by then,
    the service loop stops, every ticket queued or in flight completes with
    GP_ENOMEM, later submissions are refused, and destroy still returns and
    frees everything."""
    import torch
    g = gg.rmat(13, 16, seed=2)
    fa = FailingAllocator(gp)
    dg = _create(gp, g, fa, block_width=16)
    srcs = [int(s) for s in gg.sources(g, 12, 9)]
    try:
        ys = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in srcs]
        # device outputs first: the service starts and answers them
        first = [gp.gp_submit(dg, gp.make_request(0, s, 0.2, 1e-6, ys[i])) for i, s in enumerate(srcs[:4])]
        for t in first:
            info = gp.gp_wait(dg, t, 60000.0)
            assert info["K"] > 0
        fa.budget = 0  # every allocation from now on fails
        host = np.empty(g.n, dtype=np.float64)
        tickets = [gp.gp_submit(dg, gp.make_request(0, s, 0.1, 1e-6, ys[i])) for i, s in enumerate(srcs[5:])]
        tickets.append(gp.gp_submit(dg, gp.make_request(1, srcs[4], 5.0, 1e-6, host)))
        statuses = []
        for t in tickets:
            try:
                gp.gp_wait(dg, t, 60000.0)
                statuses.append(gp.GP_OK)
            except gp.GPError as e:
                statuses.append(e.status)
        assert fa.failed >= 1
        # the host-output ticket and whatever was still queued or running fail; the
        # rest may have finished before the failure
        assert statuses[-1] == gp.GP_ENOMEM, statuses
        assert all(st in (gp.GP_OK, gp.GP_ENOMEM) for st in statuses), statuses
        with pytest.raises(gp.GPError):
            gp.gp_submit(dg, gp.make_request(0, srcs[0], 0.2, 1e-6, ys[0]))
    finally:
        dg.close()
    assert not fa.live


def test_non_monotone_row_ptr_is_rejected(gp):
    g = gg.from_edges(6, [(0, 1), (0, 2), (1, 2), (3, 4), (4, 5)])
    rp = g.row_ptr32().copy()
    ci = g.col_idx.copy()
    deg = g.degree.copy()
    rp[3] = rp[4] + 2        # row 3 would end before it starts
    deg[2] = rp[3] - rp[2]   # keep row 2's degree consistent, so the decrease is what fails
    with pytest.raises(gp.GPError) as ei:
        gp.gp_graph_create(g.n, rp, ci, deg)
    assert ei.value.status == gp.GP_EINVAL
    assert "decreases at row 3" in str(ei.value)


def test_wait_times_out_then_completes(gp):
    import torch
    g = gg.rmat(14, 16, seed=2)
    dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree, block_width=8)
    try:
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        s = int(gg.sources(g, 1, 4)[0])
        t = gp.gp_submit(dg, gp.make_request(0, s, 0.1, 1e-6, y))
        with pytest.raises(gp.GPError) as ei:
            gp.gp_wait(dg, t, 0.0)
        assert ei.value.status == gp.GP_ETIMEDOUT
        t0 = time.perf_counter()
        info = gp.gp_wait(dg, t, 60000.0)
        assert time.perf_counter() - t0 < 60.0 and info["K"] > 0
        e = O.errors(g, O.chebypower(g, s, "ppr", 0.1, 200), y.cpu().numpy())
        assert e["l1"] <= 1e-6
        with pytest.raises(gp.GPError) as ei:  # collected
            gp.gp_wait(dg, t, 10.0)
        assert ei.value.status == gp.GP_ENOTFOUND
    finally:
        dg.close()
