// Float-pair storage path of the single query, for tiny graphs.
//
// With Q_k stored in FP32 the rounding of every stored value (relative 2^-24)
// is carried forward by the recurrence; on graphs whose walk matrix has
// eigenvalues of modulus one that never damp it (a star, a pair, an even
// cycle) and whose vectors have entries near 0.5, it reaches ~1.6e-8 after
// ~15 steps.  Graphs with at most cfg.precise_rows active rows (default 1024)
// therefore keep Q_k as an unevaluated pair of floats (hi + lo, ~48 bits):
// the neighbour sum adds the high parts by cascaded TwoSum summation, and the recurrence,
// the division by d_u and the y update run in pair arithmetic.  A warp per
// row over the relabelled rows; the stop rule is applied on the host between
// passes from the device norms (same rule and precision as the main path).
#include <algorithm>
#include <vector>

#include "gp_internal.h"

namespace gp {

namespace {

__host__ __device__ inline float2 pair_of(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// x / d for an integer-valued d, as a pair: q = hi + lo with hi = fl(x.hi/d)
// and lo the correction from the exact remainder x - hi*d.
__device__ __forceinline__ DF df_div_int(DF x, float d) {
  const float q = __fdiv_rn(x.hi, d);
  const float p = __fmul_rn(q, d);
  const float pe = __fmaf_rn(q, d, -p);  // q*d = p + pe exactly
  const float rem = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
  return df_fast_two_sum(q, __fdiv_rn(rem, d));
}

template <typename RP>
__global__ void precise_init_kernel(const RP* rp, const int32_t* ci, int64_t s, double c0, double c1, int cheb,
                                    float2* q0, float2* q1, float2* y) {
  const int64_t beg = rp[s], end = rp[s + 1];
  const double ds = (double)(end - beg);
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    q0[s] = pair_of(1.0 / ds);
    y[s] = pair_of(c0);
  }
  for (int64_t e = beg + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < end;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = ci[e];
    if (rp[v + 1] == rp[v]) continue;  // a listed node without neighbours: (P e_s)(v) = 0
    q1[v] = pair_of(1.0 / (ds * (double)(rp[v + 1] - rp[v])));
    if (cheb) y[v] = pair_of(c1 / ds);
  }
}

template <typename RP>
__global__ void precise_step_kernel(int64_t na, const RP* rp, const int32_t* ci, const float2* qcur, float2* qprev,
                                    float2* y, float c_hi, float c_lo, int cheb, float* norm_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float nrm = 0.f;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < na; u += nwarps) {
    const int64_t beg = rp[u], end = rp[u + 1];
    S2Sum sh{0.f, 0.f};
    float sl = 0.f;  // the low parts are 2^-24 smaller: a plain sum suffices
    for (int64_t e = beg + lane; e < end; e += 32) {
      const float2 q = qcur[ci[e]];
      s2sum_add(sh, q.x);
      sl = __fadd_rn(sl, q.y);
    }
    DF acc = df_add(s2sum_value(sh), DF{sl, 0.f});
    for (int off = 16; off > 0; off >>= 1) {
      const DF o{__shfl_xor_sync(0xffffffffu, acc.hi, off), __shfl_xor_sync(0xffffffffu, acc.lo, off)};
      acc = df_add(acc, o);
    }
    if (lane == 0) {
      const float d = (float)(end - beg);
      DF r;
      if (cheb) {
        const float2 qp = qprev[u];
        // d * Q_{k-1}(u) as a pair: d*hi exactly (two floats) plus d*lo
        const float p = __fmul_rn(d, qp.x);
        const float pe = __fmaf_rn(d, qp.x, -p);
        const DF prev = df_add(DF{p, pe}, DF{__fmul_rn(d, qp.y), 0.f});
        r = df_add(DF{__fmul_rn(2.0f, acc.hi), __fmul_rn(2.0f, acc.lo)}, DF{-prev.hi, -prev.lo});
      } else {
        r = df_norm(acc);
      }
      const DF qn = df_div_int(r, d);
      qprev[u] = make_float2(qn.hi, qn.lo);
      const float2 yv = y[u];
      const DF yy = df_add(DF{yv.x, yv.y}, df_mul(r, DF{c_hi, c_lo}));
      y[u] = make_float2(yy.hi, yy.lo);
      nrm += fabsf(__fadd_rn(r.hi, r.lo));
    }
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  if (lane == 0 && nrm != 0.f) atomicAdd(norm_out, nrm);
}

}  // namespace

bool use_precise(const Graph& g) {
  const int64_t lim = g.cfg.precise_rows > 0 ? g.cfg.precise_rows : (g.cfg.precise_rows < 0 ? 0 : 1024);
  return g.n_active <= lim;
}

int run_precise(Graph& g, int64_t s, bool cheb, const std::vector<double>& c, const std::vector<double>& tail,
                int k_fixed, double tol, int kcap, double* C_out) {
  const int64_t na = g.n_active;
  Allocator& A = g.alloc;
  float2* qa = (float2*)A.get(sizeof(float2) * g.n);
  float2* qb = (float2*)A.get(sizeof(float2) * g.n);
  float* norms = (float*)A.get(sizeof(float) * 2);
  int K = 0;
  try {
    cudaStream_t st = g.stream;
    GP_CUDA_TRY(cudaMemsetAsync(qa, 0, sizeof(float2) * g.n, st));
    GP_CUDA_TRY(cudaMemsetAsync(qb, 0, sizeof(float2) * g.n, st));
    GP_CUDA_TRY(cudaMemsetAsync(g.qw.y, 0, sizeof(float2) * g.n, st));
    if (g.rp64)
      precise_init_kernel<int64_t><<<4, 256, 0, st>>>((const int64_t*)g.rp, g.ci, s, c[0], cheb ? c[1] : 0.0,
                                                      cheb ? 1 : 0, qa, qb, g.qw.y);
    else
      precise_init_kernel<int32_t><<<4, 256, 0, st>>>((const int32_t*)g.rp, g.ci, s, c[0], cheb ? c[1] : 0.0,
                                                      cheb ? 1 : 0, qa, qb, g.qw.y);
    GP_LAUNCHED();
    float2* bufs[2] = {qa, qb};  // bufs[k & 1] holds Q_k
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((na + 7) / 8, 1024));
    double C = 1.0;  // max ||r_l||_1 so far (||r_0||_1 = ||r_1||_1 = 1)
    // power baseline starts at k = 0 (r_1 = P r_0 is computed on the device)
    int k = cheb ? 1 : 0;
    const int kend = k_fixed >= 1 ? k_fixed : kcap;
    while (k < kend) {
      if (cheb && k_fixed < 1 && tail[k] * C <= tol) break;
      GP_CUDA_TRY(cudaMemsetAsync(norms, 0, sizeof(float), st));
      const float2 ck = pair_of(c[k + 1]);
      if (g.rp64)
        precise_step_kernel<int64_t><<<blocks, 256, 0, st>>>(na, (const int64_t*)g.rp, g.ci, bufs[k & 1],
                                                             bufs[(k + 1) & 1], g.qw.y, ck.x, ck.y, cheb ? 1 : 0,
                                                             norms);
      else
        precise_step_kernel<int32_t><<<blocks, 256, 0, st>>>(na, (const int32_t*)g.rp, g.ci, bufs[k & 1],
                                                             bufs[(k + 1) & 1], g.qw.y, ck.x, ck.y, cheb ? 1 : 0,
                                                             norms);
      GP_LAUNCHED();
      float nr = 0.f;
      GP_CUDA_TRY(cudaMemcpyAsync(&nr, norms, sizeof(float), cudaMemcpyDeviceToHost, st));
      GP_CUDA_TRY(cudaStreamSynchronize(st));
      C = std::max(C, (double)nr);
      ++k;
    }
    K = k;
    *C_out = C;
    GP_CUDA_TRY(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(g.stream);
    A.put(qa);
    A.put(qb);
    A.put(norms);
    throw;
  }
  A.put(qa);
  A.put(qb);
  A.put(norms);
  return K;
}

}  // namespace gp
