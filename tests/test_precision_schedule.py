"""The 16-bit warm-up schedule as a reading of the paper, checked on the CPU.

A numpy emulation of the batched recurrence with Q stored in BF16 (round to
nearest even) from the switch step on, FP64 sums, compares two switch rules
for slowly decaying expansions (SSPPR alpha = 0.1, HKPR t = 10): the plain
tail sum_{l>k} |c_l| < 1e-2, and the weight W(k) = sum_{m>=0} (m+1)|c_{k+1+m}|
< 1e-2 that accounts for the linear growth (|U_m| <= m + 1) of a rounding
error the recurrence does not compensate (the residual-propagation lemma of
the generalized subset recurrence).  The device uses W(k); its first 16-bit
store is Q_{warm+2}, the pass after the switch.  No GPU and no library code:
the oracle and numpy only.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O


def _bf16(x):
    a = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _f16_scaled(x):
    """FP16 storage of Q * 2^12 (round to nearest even), read back in Q units."""
    return np.asarray(np.asarray(x, np.float32) * np.float32(4096.0), np.float16).astype(np.float64) / 4096.0


def _warm(c, rule, threshold=1e-2):
    for k in range(len(c) - 1):
        if rule == "tail":
            w = np.abs(c[k + 1:]).sum()
        else:
            w = sum((m + 1) * abs(c[k + 1 + m]) for m in range(len(c) - k - 1))
        if w < threshold:
            return k
    return len(c) - 1


def _emulate(g, s, kind, param, rule, tol=1e-4, threshold=1e-2, store=_bf16):
    rp = np.asarray(g.row_ptr, np.int64)
    ci = np.asarray(g.col_idx, np.int64)
    d = np.diff(rp).astype(np.float64)
    ne = d > 0
    inv = np.where(ne, 1.0 / np.maximum(d, 1), 0.0)

    def pull(q):  # (P r)(u) = sum_{v in N(u)} Q(v)
        out = np.zeros(g.n)
        out[ne] = np.add.reduceat(q[ci], rp[:-1][ne])
        return out

    c = O.cheb_coeffs(kind, param, 200)
    _, K, _ = O.chebypower_tol(g, s, kind, param, tol)
    sw = _warm(c, rule, threshold) + 1  # Q_j stored in 16 bits for j > sw
    e = np.zeros(g.n)
    e[s] = 1.0
    r1 = O.P_apply(g, e)
    qp, qc = _f32(e * inv), _f32(r1 * inv)
    y = c[0] * e + c[1] * r1
    for k in range(1, K):
        r = 2.0 * pull(qc) - d * qp
        y = y + c[k + 1] * r
        qp, qc = qc, (_f32 if k + 1 <= sw else store)(r * inv)
    return np.abs(y - O.chebypower(g, s, kind, param, 150)).sum()


@pytest.mark.parametrize("kind,param", [("ppr", 0.1), ("hkpr", 10.0)])
def test_weighted_switch_keeps_bf16_blocks_within_tol(kind, param):
    g = gg.rmat(12, 16, seed=2)
    errs_w = [_emulate(g, int(s), kind, param, "weighted") for s in gg.sources(g, 8, 21)]
    assert max(errs_w) <= 1e-4, errs_w


def test_tail_switch_misses_tol_where_the_weighted_one_does_not():
    # R-MAT 14, an SSPPR alpha = 0.1 source whose rounding errors, stored in
    # BF16 from the plain-tail switch on, push l1 past 1e-4
    g = gg.rmat(14, 16, seed=2)
    s = 14492
    assert s in set(int(v) for v in gg.sources(g, 16, 21))  # one of the seeded uniform sources
    assert _emulate(g, s, "ppr", 0.1, "tail") > 1e-4
    assert _emulate(g, s, "ppr", 0.1, "weighted") <= 0.5e-4


def test_weighted_switch_is_later_than_the_tail_switch():
    for kind, param, later in (("ppr", 0.1, 2), ("ppr", 0.2, 1), ("hkpr", 5.0, 0), ("hkpr", 10.0, 1)):
        c = O.cheb_coeffs(kind, param, 200)
        assert _warm(c, "weighted") - _warm(c, "tail") == later, (kind, param)


# The device's threshold for a column of tolerance tol: the 1e-2 above at
# tol >= 1e-4, scaled with tol below it (the 16-bit rounding error reaching y
# is proportional to the threshold), and four times larger for FP16, whose
# 11-bit significand (Q * 2^12 keeps it clear of the subnormals) rounds eight
# times finer than BF16's 8 bits.
def _threshold(store, tol):
    return (4e-2 if store is _f16_scaled else 1e-2) * min(1.0, tol / 1e-4)


@pytest.mark.parametrize("kind,param", [("ppr", 0.1), ("ppr", 0.2), ("hkpr", 5.0), ("hkpr", 10.0)])
def test_fp16_switch_at_four_times_the_bf16_weight(kind, param):
    g = gg.rmat(12, 16, seed=2)
    errs = [_emulate(g, int(s), kind, param, "weighted", 1e-4, _threshold(_f16_scaled, 1e-4), _f16_scaled)
            for s in gg.sources(g, 6, 23)]
    assert max(errs) <= 1e-4, errs
    c = O.cheb_coeffs(kind, param, 200)
    assert _warm(c, "weighted", 4e-2) <= _warm(c, "weighted", 1e-2)  # fewer FP32 steps


@pytest.mark.parametrize("tol", [1e-5, 1e-6])
@pytest.mark.parametrize("store", [_bf16, _f16_scaled])
def test_threshold_scaled_with_the_tolerance(tol, store):
    g = gg.rmat(12, 16, seed=2)
    errs = [_emulate(g, int(s), kind, param, "weighted", tol, _threshold(store, tol), store)
            for s in gg.sources(g, 3, 29) for kind, param in (("ppr", 0.1), ("hkpr", 10.0))]
    assert max(errs) <= tol, errs
    if store is _bf16:  # the unscaled BF16 threshold would not hold these tolerances
        worst_unscaled = max(_emulate(g, int(s), "ppr", 0.1, "weighted", tol, _threshold(store, 1e-4), store)
                             for s in gg.sources(g, 3, 29))
        assert worst_unscaled > tol
