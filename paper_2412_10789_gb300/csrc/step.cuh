// The fused Chebyshev step kernel (one pass k -> k+1 over all non-isolated
// rows), included by cheb.cu.
//
// Per row u of the relabelled graph the pass computes
//     acc = sum_{v in N(u)} Q_k(v)             (Kahan-compensated FP32)
//     r   = 2 acc - d_u Q_{k-1}(u)             (Eq. res-recurrence; power step: r = acc)
//     Q_{k+1}(u) = r / d_u  over Q_{k-1}(u)    (two-vector form, Eq. 8 / Lemma 6)
//     y(u) += c_{k+1} r                        (float pair, ~48-bit)
//     ||r_{k+1}||_1 partial                   (warp sums, one atomic per CTA)
// so no r_k is read twice.
//
// Work: tiles of at most kTileCap consecutive col_idx entries (schedule.cpp):
// runs of equal-degree rows, or chunks of one long row.  Warps claim tiles
// from a per-pass counter; each warp double-buffers tile indices in shared memory, copying
// the next tile's col_idx with 16-byte cp.async while it gathers and sums the
// current one.  A chunk of a long row only stores its partial sum; a second,
// small kernel (cheb_long_kernel) adds each long row's partials in chunk order
// and updates the row, so the step needs no fences or counters between warps.  Gathers of indices below `hub` read a shared-memory copy of
// the hub rows of Q_k (the most gathered values); the rest go to L2.  The
// kernel is persistent: one CTA of kStepThreads threads per SM.
#pragma once

#include "gp_internal.h"

namespace gp {
namespace {

struct StepArgs {
  const int4* tiles;
  int64_t ntiles;
  const void* rp;
  const int32_t* ci;
  const float* qcur;   // Q_k (gathered)
  float* qprev;        // Q_{k-1} in, Q_{k+1} out
  float2* y;           // y (hi, lo)
  float* norms;        // ||r_l||_1
  int* state;          // [0] = stop K, [2 + k] = tiles claimed in pass k
  const int* poff;     // long rows: first chunk slot
  float2* part;        // long rows: chunk partial sums
  int hub;             // rows of Q_k cached in shared memory
  int nlong;           // long (chunked) rows: relabelled rows 0..nlong-1
  int k;               // this pass computes r_{k+1}
  float c_hi, c_lo;    // c_{k+1} as a float pair
  float tail;          // tail(k) (stop test), negative disables the test
  float tol;           // l1 tolerance over kCMargin
  int cheb;            // 1: Chebyshev recurrence, 0: power step r_{k+1} = P r_k
};

// ---- cache policies, loads and asynchronous copies.  The col_idx stream is
// read once per pass and marked evict-first in L2 so that it does not displace
// Q_k; the gathers of Q_k are marked evict-last.  Own-row reads skip L1.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float ld_own(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_own2(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem_addr(smem)), "l"(gmem),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ float ld_q(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct Ctx {
  const StepArgs* a;
  const float* hub_q;  // shared-memory copy of Q_k[0..hub)
  uint64_t pol_stream, pol_keep;
  float nrm;
};

// One row's update from its neighbour sum acc.
__device__ __forceinline__ void row_update(Ctx& c, int64_t u, int64_t deg, DF acc, float qp, float2 yv) {
  const StepArgs& a = *c.a;
  const float d = (float)deg;
  DF r;
  if (a.cheb) {
    const float p = __fmul_rn(d, qp);  // d * Q_{k-1}(u) exactly, as p + pe
    const float pe = __fmaf_rn(d, qp, -p);
    r = df_add(DF{__fmul_rn(2.0f, acc.hi), __fmul_rn(2.0f, acc.lo)}, DF{-p, -pe});
  } else {
    r = df_norm(acc);
  }
  const float rv = __fadd_rn(r.hi, r.lo);
  a.qprev[u] = __fdiv_rn(rv, d);
  const DF yy = df_add(DF{yv.x, yv.y}, df_mul(r, DF{a.c_hi, a.c_lo}));
  a.y[u] = make_float2(yy.hi, yy.lo);
  c.nrm += fabsf(rv);
}

__device__ __forceinline__ DF shfl_sum_df(DF v, int width) {
  for (int off = width / 2; off > 0; off >>= 1) {
    const DF o{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
    v = df_add(v, o);
  }
  return v;
}

struct TileInfo {
  int64_t row0, e0;
  int kind;   // 0 rows tile, 1 chunk of a long row
  int nrows;  // rows tile: rows; chunk: 1
  int d;      // rows tile: degree of every row; chunk: its entries
  int len;    // entries
  int p;      // chunk index
};

__device__ __forceinline__ TileInfo decode(int4 t) {
  TileInfo ti;
  ti.row0 = t.x;
  ti.e0 = (int64_t)(uint32_t)t.y | ((int64_t)t.z << 32);
  const uint32_t m = (uint32_t)t.w;
  ti.kind = m & 1;
  if (ti.kind == 0) {
    ti.nrows = (m >> 1) & 0xff;
    ti.d = (m >> 9) & 0x3ff;
    ti.len = ti.nrows * ti.d;
    ti.p = 0;
  } else {
    ti.len = (m >> 1) & 0x3ff;
    ti.p = (int)(m >> 11);
    ti.nrows = 1;
    ti.d = ti.len;
  }
  return ti;
}

// Copy a tile's col_idx (16-byte vectors from the 4-entry boundary at or below
// e0) into idx asynchronously.
__device__ __forceinline__ void stage_indices(const Ctx& c, const TileInfo& t, int* idx) {
  const int lane = threadIdx.x & 31;
  const int64_t base = t.e0 & ~int64_t(3);
  const int nvec = (int)((t.e0 - base + t.len + 3) >> 2);
  const int4* src = reinterpret_cast<const int4*>(c.a->ci + base);
  for (int v = lane; v < nvec; v += 32) cp_async16(idx + 4 * v, src + v, c.pol_stream);
}

// Up to N gathers of Q_k at the staged indices idx[start + (i0 + i)*stride],
// i < N and i0 + i < count (hub indices read shared memory); slots past count
// get index -1 and value 0.
template <int N>
__device__ __forceinline__ void gather_batch(const Ctx& c, const int* idx, int start, int stride, int count, int i0,
                                             int id[N], float v[N]) {
  const float* q = c.a->qcur;
  const int hub = c.a->hub;
#pragma unroll
  for (int i = 0; i < N; ++i) id[i] = i0 + i < count ? idx[start + (i0 + i) * stride] : -1;
#pragma unroll
  for (int i = 0; i < N; ++i)
    v[i] = id[i] < 0 ? 0.f : id[i] < hub ? c.hub_q[id[i]] : ld_q(q + id[i], c.pol_keep);
}

// Compensated sum of Q_k over the staged indices idx[start + i*stride],
// i < count: GP_KAHAN_WAYS Kahan accumulators take the entries in turn (a
// shorter chain of dependent adds per accumulator) and are merged as float
// pairs in a fixed order.  With GP_GATHER_PIPE the next batch of N gathers is
// issued before the current batch is added, so two batches are in flight.
#ifndef GP_GATHER_PIPE
#define GP_GATHER_PIPE 0
#endif
#ifndef GP_KAHAN_WAYS
#define GP_KAHAN_WAYS 1
#endif
template <int N>
__device__ __forceinline__ DF gather_sum(const Ctx& c, const int* idx, int start, int stride, int count) {
  constexpr int W = GP_KAHAN_WAYS;
  KSum s[W];
#pragma unroll
  for (int w = 0; w < W; ++w) s[w] = KSum{0.f, 0.f};
#if GP_GATHER_PIPE
  int id[N];
  float v[N];
  gather_batch<N>(c, idx, start, stride, count, 0, id, v);
  for (int i0 = 0; i0 < count; i0 += N) {
    int cid[N];
    float cv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      cid[i] = id[i];
      cv[i] = v[i];
    }
    if (i0 + N < count) gather_batch<N>(c, idx, start, stride, count, i0 + N, id, v);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (cid[i] >= 0) ksum_add(s[i % W], cv[i]);
  }
#else
  for (int i0 = 0; i0 < count; i0 += N) {
    int id[N];
    float v[N];
    gather_batch<N>(c, idx, start, stride, count, i0, id, v);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (id[i] >= 0) ksum_add(s[i % W], v[i]);
  }
#endif
  DF r = ksum_value(s[0]);
#pragma unroll
  for (int w = 1; w < W; ++w) r = df_add(r, ksum_value(s[w]));
  return r;
}

// Rows tile.  With nrows >= 32 (degree <= kTileCap/32) the warp gathers the
// whole tile, writing each value over its index, and lane l sums and updates
// rows l, l+32, ...; with fewer rows G = 32/nrows (rounded down to a power of
// two) lanes share a row, each gathering and summing every G-th entry straight
// from the staged indices, and the row's first lane updates it.  Kahan sums in
// entry order per lane, combined by a fixed shuffle tree.
__device__ __forceinline__ void finish_rows(Ctx& c, const TileInfo& t, int* idx) {
  const StepArgs& a = *c.a;
  const int lane = threadIdx.x & 31;
  const int off0 = (int)(t.e0 & 3);
  if (t.nrows >= 32) {
    float qp[4];
    float2 yv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = lane + 32 * j;
      if (r < t.nrows) {
        qp[j] = a.cheb ? ld_own(a.qprev + t.row0 + r) : 0.f;
        yv[j] = ld_own2(a.y + t.row0 + r);
      }
    }
    constexpr int M = kTileSpan / 32;
    const float* q = a.qcur;
    int id[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int p = lane + 32 * m;
      id[m] = (p >= off0 && p < off0 + t.len) ? idx[p] : -1;
    }
    float v[M];
#pragma unroll
    for (int m = 0; m < M; ++m)
      v[m] = id[m] < 0 ? 0.f : id[m] < a.hub ? c.hub_q[id[m]] : ld_q(q + id[m], c.pol_keep);
#pragma unroll
    for (int m = 0; m < M; ++m)
      if (id[m] >= 0) idx[lane + 32 * m] = __float_as_int(v[m]);
    __syncwarp();
    const float* val = reinterpret_cast<const float*>(idx);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = lane + 32 * j;
      if (r < t.nrows) {
        KSum s{0.f, 0.f};
        const int b = off0 + r * t.d;
        for (int e = 0; e < t.d; ++e) ksum_add(s, val[b + e]);
        row_update(c, t.row0 + r, t.d, ksum_value(s), qp[j], yv[j]);
      }
    }
  } else {
    int G = 32;
    while (G * t.nrows > 32) G >>= 1;
    const int r = lane / G, sub = lane & (G - 1);
    const bool own = r < t.nrows;
    float qp = 0.f;
    float2 yv = make_float2(0.f, 0.f);
    if (own && sub == 0) {
      if (a.cheb) qp = ld_own(a.qprev + t.row0 + r);
      yv = ld_own2(a.y + t.row0 + r);
    }
    DF sv{0.f, 0.f};
    if (own) sv = gather_sum<GP_GATHER_N>(c, idx, off0 + r * t.d + sub, G, (t.d - sub + G - 1) / G);
    const DF v = shfl_sum_df(sv, G);
    if (own && sub == 0) row_update(c, t.row0 + r, t.d, v, qp, yv);
  }
}

// Chunk of a long row: sum it and store the partial (slot poff[row] + p).
__device__ __forceinline__ void finish_chunk(Ctx& c, const TileInfo& t, const int* idx) {
  const StepArgs& a = *c.a;
  const int lane = threadIdx.x & 31;
  const int off0 = (int)(t.e0 & 3);
  const DF v = shfl_sum_df(gather_sum<GP_GATHER_N>(c, idx, off0 + lane, 32, (t.len - lane + 31) / 32), 32);
  if (lane == 0) a.part[a.poff[t.row0] + t.p] = make_float2(v.hi, v.lo);
}

// The stop test at the top of pass k: stop once tail(k) * max_{l<=k} ||r_l||_1
// <= tol, where tol is the caller's l1 tolerance over kCMargin (Theorem 1 with
// Assumption 1's C estimated on the fly).  Thread-local; the caller shares it.
__device__ __forceinline__ int pass_stopped(const StepArgs& a) {
  if (a.tail < 0.f) return 0;
  float C = 0.f;
  for (int l = 0; l <= a.k; ++l) C = fmaxf(C, a.norms[l]);
  return a.tail * C <= a.tol;
}

// Block sum of the warps' ||r_{k+1}||_1 partials, one atomic per CTA.
template <int W>
__device__ __forceinline__ void add_norm(const StepArgs& a, float nrm, float* s_norm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  if (lane == 0) s_norm[warp] = nrm;
  __syncthreads();
  if (warp == 0) {
    float w = lane < W ? s_norm[lane] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
    if (lane == 0 && w != 0.f) atomicAdd(&a.norms[a.k + 1], w);
  }
}

// Long rows after the step: one warp per row adds the row's chunk partials in
// chunk order (lane i takes chunks i, i+32, ...; then a fixed shuffle tree), so
// the sum does not depend on which warp stored which chunk, and applies the
// row update.  Runs after cheb_step_kernel on the same stream and before the
// next pass, whose shared-memory hub reads these rows of Q_{k+1}.
constexpr int kLongWarps = 8;
template <typename RP>
__global__ void __launch_bounds__(32 * kLongWarps) cheb_long_kernel(const __grid_constant__ StepArgs a) {
  __shared__ int s_flag;
  __shared__ float s_norm[kLongWarps];
  if (threadIdx.x == 0) s_flag = pass_stopped(a);
  __syncthreads();
  if (s_flag) return;
  const RP* rp = (const RP*)a.rp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Ctx c;
  c.a = &a;
  c.hub_q = nullptr;
  c.nrm = 0.f;
  for (int64_t row = (int64_t)blockIdx.x * kLongWarps + warp; row < a.nlong;
       row += (int64_t)gridDim.x * kLongWarps) {
    const int slot0 = a.poff[row];
    const int np = a.poff[row + 1] - slot0;
    DF acc{0.f, 0.f};
    for (int i = lane; i < np; i += 32) {
      const float2 pv = __ldcg(a.part + slot0 + i);
      acc = df_add(acc, DF{pv.x, pv.y});
    }
    acc = shfl_sum_df(acc, 32);
    if (lane == 0) {
      const float qp = a.cheb ? ld_own(a.qprev + row) : 0.f;
      const float2 yv = ld_own2(a.y + row);
      row_update(c, row, (int64_t)(rp[row + 1] - rp[row]), acc, qp, yv);
    }
  }
  add_norm<kLongWarps>(a, c.nrm, s_norm);
}

template <typename RP>
__global__ void __launch_bounds__(kStepThreads, 1) cheb_step_kernel(const __grid_constant__ StepArgs a) {
  extern __shared__ __align__(16) int s_dyn[];
  __shared__ int s_flag;
  __shared__ float s_norm[kStepWarps];
  if (threadIdx.x == 0) {
    const int stop = pass_stopped(a);
    if (stop && blockIdx.x == 0) atomicMin(&a.state[0], a.k);
    s_flag = stop;
  }
  __syncthreads();
  if (s_flag) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* wbase = s_dyn + warp * kWarpSmemInts;  // two index buffers of kTileSpan
  float* hub_q = reinterpret_cast<float*>(s_dyn + kStepWarps * kWarpSmemInts);
  Ctx c;
  c.a = &a;
  c.hub_q = hub_q;
  c.pol_stream = policy_evict_first();
  c.pol_keep = policy_evict_last();
  c.nrm = 0.f;
  // Tiles: each warp starts with tiles w, w + W and w + 2W (W warps in the
  // grid), then claims the next unclaimed tile from this pass's counter
  // (state[2 + k], zeroed per query), so no warp is left with a run of costly
  // tiles at the end.  The claim is three tiles ahead: its atomic and the load
  // of its descriptor complete while the warp works on the current tile.
  const int64_t stride = (int64_t)gridDim.x * kStepWarps;
  int64_t t = (int64_t)blockIdx.x * kStepWarps + warp;
  int64_t tn = t + stride, tnn = t + 2 * stride;
  TileInfo cur{};
  if (t < a.ntiles) {
    cur = decode(a.tiles[t]);
    stage_indices(c, cur, wbase);
  }
  cp_async_commit();
  int4 dn = make_int4(0, 0, 0, 0);  // descriptor of tile tn
  if (tn < a.ntiles) dn = a.tiles[tn];
  // fill the hub while the first tile's indices land
  {
    const float4* src = reinterpret_cast<const float4*>(a.qcur);
    float4* dst = reinterpret_cast<float4*>(hub_q);
    for (int i = threadIdx.x; i < a.hub / 4; i += kStepThreads) dst[i] = __ldcg(src + i);
  }
  __syncthreads();
  int b = 0;
  while (t < a.ntiles) {
    TileInfo nxt{};
    if (tn < a.ntiles) {
      nxt = decode(dn);
      stage_indices(c, nxt, wbase + (b ^ 1) * kTileSpan);
    }
    cp_async_commit();
    int claimed = 0;
    if (lane == 0) claimed = atomicAdd(&a.state[2 + a.k], 1);
    int4 dnn = make_int4(0, 0, 0, 0);
    if (tnn < a.ntiles) dnn = a.tiles[tnn];
    cp_async_wait<1>();  // this lane's copies of tile t have landed
    __syncwarp();        // ... and every lane's
    int* idx = wbase + b * kTileSpan;
    if (cur.kind == 0)
      finish_rows(c, cur, idx);
    else
      finish_chunk(c, cur, idx);
    __syncwarp();  // the buffer is free for the copy two tiles ahead
    const int64_t t3 = 3 * stride + __shfl_sync(0xffffffffu, claimed, 0);
    cur = nxt;
    b ^= 1;
    t = tn;
    tn = tnn;
    tnn = t3;
    dn = dnn;
  }
  cp_async_wait<0>();
  add_norm<kStepWarps>(a, c.nrm, s_norm);
}

}  // namespace
}  // namespace gp
