"""Run one small case of a query form, for profilers (ncu) and quick checks.

    python -m paper_2412_10789_gb300.run_case batch  --scale 22 --sources 64 --storage bf16 --width 128 --reps 2
    python -m paper_2412_10789_gb300.run_case single --scale 22 --sources 2

The graph is the seeded R-MAT graph of bench.py (edge factor 16,
(a, b, c) = (0.57, 0.19, 0.19), seed 2); each source gives one SSPPR
(alpha = 0.2) and one HKPR (t = 5) query.  Prints one line with the time of
the last repetition.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("form", choices=["single", "batch"])
    p.add_argument("--scale", type=int, default=22)
    p.add_argument("--sources", type=int, default=64)
    p.add_argument("--storage", default="bf16", choices=["fp32", "bf16", "fp16"])
    p.add_argument("--width", type=int, default=0, help="block width (0: from the query count)")
    p.add_argument("--tol", type=float, default=None, help="l1 tolerance (default 1e-4 batch, 1e-6 single)")
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--k-fixed", type=int, default=0, help="batch: every query runs exactly this K (0: stop rule)")
    args = p.parse_args()

    import torch
    import graphgen as gg
    from paper_2412_10789_gb300 import gp

    g = gg.rmat(args.scale, 16, 0.57, 0.19, 0.19, seed=2)
    srcs = gg.sources(g, args.sources, 2)
    queries = [(0, int(s), 0.2) for s in srcs] + [(1, int(s), 5.0) for s in srcs]
    storage = {"fp32": gp.GP_F32, "bf16": gp.GP_BF16, "fp16": gp.GP_F16}[args.storage]
    if args.form == "batch":
        tol = 1e-4 if args.tol is None else args.tol
        rp = g.row_ptr if g.nnz > 2**31 - 1 else g.row_ptr32()
        dg = gp.gp_graph_create(g.n, rp, g.col_idx, g.degree, storage=storage, block_width=args.width)
        ys = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in queries]
        kw = dict(k_rule=gp.GP_K_FIXED, k_fixed=args.k_fixed) if args.k_fixed > 0 else {}
        reqs = [gp.make_request(fn, s, a, tol, ys[i], **kw) for i, (fn, s, a) in enumerate(queries)]
        for _ in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            infos = gp.gp_batch(dg, reqs)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        ks = [i["K"] for i in infos]
        print(f"batch {args.storage} B={args.width or 'auto'} queries={len(queries)} "
              f"{len(queries) / dt:.1f} q/s, K {min(ks)}..{max(ks)}", flush=True)
    else:
        tol = 1e-6 if args.tol is None else args.tol
        dg = gp.gp_graph_create(g.n, g.row_ptr32(), g.col_idx, g.degree)
        y = torch.empty(g.n, dtype=torch.float64, device="cuda")
        for _ in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for fn, s, a in queries:
                (gp.gp_ppr if fn == 0 else gp.gp_hkpr)(dg, s, a, tol, y, info=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        print(f"single queries={len(queries)} {len(queries) / dt:.1f} q/s", flush=True)
    dg.close()


if __name__ == "__main__":
    main()
