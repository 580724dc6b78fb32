"""The batched form's FP32 neighbour sums, emulated on the CPU (reading 9).

In a 256-column FP32 pass one lane adds a whole 508-entry chunk of a long row
in order.  Emulated with numpy's sequential float32 accumulation, that order
loses two to three times the l1 accuracy of the two-level sums the kernel
uses (blocks of 16 entries, each block added to the running sum); the
chunks' partials are then added in chunk order, and r, Q and y stay FP32 as
on the device.  No GPU and no library code: the oracle and numpy only.
"""
import os
import re

import numpy as np

import graphgen as gg
import oracle as O

F32 = np.float32
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _kernel_constants():
    """The block length of the two-level sums (kBlk) and the chunk length of a
    long row (kBTileCap) as the batched kernel's source defines them, so the
    emulation follows the device code if either changes."""
    with open(os.path.join(ROOT, "paper_2412_10789_gb300", "csrc", "batch.cu")) as f:
        src = f.read()
    blk = int(re.search(r"constexpr int kBlk = (\d+);", src).group(1))
    span = int(re.search(r"#define GP_SPMM_TILE (\d+)", src).group(1))
    cap = span - int(re.search(r"constexpr int kBTileCap = kBTileSpan - (\d+);", src).group(1))
    return blk, cap


BLK, CHUNK = _kernel_constants()


def _seq(x):
    return np.add.accumulate(x, dtype=np.float32)[-1] if x.size else F32(0)


def _lane(x, two_level):
    if not two_level:
        return _seq(x)
    return _seq(np.array([_seq(x[i:i + BLK]) for i in range(0, x.size, BLK)], np.float32))


def _run(g, s, kind, param, two_level):
    rp = np.asarray(g.row_ptr, np.int64)
    ci = np.asarray(g.col_idx, np.int64)
    d = np.diff(rp).astype(np.float64)
    rows = np.nonzero(d > 0)[0]

    def rowsum(q):
        out = np.zeros(g.n, np.float32)
        v = q[ci]
        for u in rows:
            a, b = rp[u], rp[u + 1]
            parts = [_lane(v[c0:min(b, c0 + CHUNK)], two_level) for c0 in range(a, b, CHUNK)]
            out[u] = _seq(np.array(parts, np.float32))
        return out

    _, K, _ = O.chebypower_tol(g, s, kind, param, 1e-6)
    c = O.cheb_coeffs(kind, param, K).astype(np.float32)
    inv = np.where(d > 0, 1.0 / np.maximum(d, 1), 0).astype(np.float32)
    df = d.astype(np.float32)
    e = np.zeros(g.n, np.float32)
    e[s] = 1
    r1 = O.P_apply(g, e.astype(np.float64)).astype(np.float32)
    qp, qc = e * inv, r1 * inv
    y = (c[0] * e + c[1] * r1).astype(np.float32)
    for k in range(1, K):
        r = (F32(2) * rowsum(qc) - df * qp).astype(np.float32)
        y = (y + c[k + 1] * r).astype(np.float32)
        qp, qc = qc, (r * inv).astype(np.float32)
    return np.abs(y.astype(np.float64) - O.chebypower(g, s, kind, param, 150)).sum()


def test_two_level_lane_sums_beat_sequential_ones():
    assert (BLK, CHUNK) == (16, 508), "the kernel's sums changed: re-derive the bars below"
    g = gg.rmat(13, 16, seed=2)  # hubs of up to 2212 entries: several chunks
    seq, two = [], []
    for s in gg.sources(g, 3, 3):
        for kind, param in (("hkpr", 10.0), ("ppr", 0.1)):
            seq.append(_run(g, int(s), kind, param, False))
            two.append(_run(g, int(s), kind, param, True))
    assert max(two) <= 1e-6
    assert max(two) <= 0.7 * max(seq), (two, seq)
