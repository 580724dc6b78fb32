// Single-source ChebyPower on the device (Algorithm 3) and the PwMethod
// baseline (Algorithm 1): per-query set-up, the launch sequence of the fused
// step kernel (step.cuh), the device-side stop test, and the output.
//
// Stored form.  The library keeps Q_k = D^{-1} r_k (FP32) instead of r_k, so
// (P r_k)(u) = sum_{v in N(u)} Q_k(v): the edge loop needs no weight or degree
// gather.  y is kept as a float pair (hi + lo) and returned as double or float.
//
// Stopping (Theorem 1 read for l1, Assumption 1's C measured): the pass for
// step k first checks tail(k) * max_{l<=k} ||r_l||_1 <= tol from the norms
// the earlier passes left in device memory; when it holds, the query stopped at
// K = k and the pass returns at once.  The host launches passes in chunks and
// reads K back, so only a few empty passes follow the stop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "gp_internal.h"
#include "step.cuh"

namespace gp {

namespace {

struct InitArgs {
  const void* rp;
  const int32_t* ci;
  float* q0;      // Q_0 buffer (zeroed)
  float* q1;      // Q_1 buffer (zeroed)
  float2* y;      // zeroed
  float* norms;   // zeroed
  int* state;
  int64_t s;      // relabelled source
  double c0, c1;  // coefficients of r_0 and r_1 (c1 = 0 for a power-step start)
  int kcap;
  int cheb;
};

__host__ __device__ inline float2 split_df(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return make_float2(hi, lo);
}

// r_0 = e_s, r_1 = P e_s: Q_0(s) = 1/d_s; for v in N(s) with d_v > 0,
// r_1(v) = 1/d_s and Q_1(v) = 1/(d_s d_v); y = c_0 r_0 + c_1 r_1.  (Algorithm 3,
// first line.)
template <typename RP>
__global__ void cheb_init_kernel(const __grid_constant__ InitArgs a) {
  const RP* rp = (const RP*)a.rp;
  const int64_t beg = rp[a.s], end = rp[a.s + 1];
  const double ds = (double)(end - beg);
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid == 0) {
    a.q0[a.s] = (float)(1.0 / ds);
    a.y[a.s] = split_df(a.c0);
    a.norms[0] = 1.0f;
    a.norms[1] = 1.0f;  // ||P e_s||_1 = d_s * (1/d_s)
    a.state[0] = a.kcap;
  }
  for (int64_t e = beg + tid; e < end; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = a.ci[e];
    // a listed node with an empty row (only an unvalidated asymmetric CSR has
    // one) has (P e_s)(v) = 0: its own row gathers nothing
    if (rp[v + 1] == rp[v]) continue;
    double dv = (double)(rp[v + 1] - rp[v]);
    a.q1[v] = (float)(1.0 / (ds * dv));
    if (a.cheb) a.y[v] = split_df(a.c1 / ds);
  }
}

// y_out[u] = y[newid[u]] in the caller's order, as double or float.  For an
// isolated source (relabelled index >= n_active) the answer is f(0) e_s.
template <typename OUT>
__global__ void finalize_kernel(int64_t n, const int32_t* __restrict__ newid, const float2* __restrict__ y,
                                OUT* __restrict__ out) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    float2 v = y[newid[u]];
    out[u] = (OUT)((double)v.x + (double)v.y);
  }
}

template <typename OUT>
__global__ void point_kernel(int64_t n, int64_t s, double val, OUT* __restrict__ out) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    out[u] = (OUT)(u == s ? val : 0.0);
}

int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// One persistent CTA per SM (the shared-memory hub cache takes the SM's shared memory).
int step_grid(const Graph& g) {
  (void)g;
  return device_sms();
}

// Longest pass sequence any query may run (the power baseline can need
// hundreds of Taylor terms); sizes the per-step norm and counter arrays.
constexpr int kPassCap = 1088;

void ensure_query_work(Graph& g) {
  QueryWork& w = g.qw;
  if (w.qa) return;
  w.kcap = kPassCap;
  // Sized by n, not n_active: with symmetry validation off a listed neighbour
  // may be isolated (id >= n_active); its Q stays zero from this memset.
  w.qa = (float*)g.alloc.get(sizeof(float) * g.n);
  w.qb = (float*)g.alloc.get(sizeof(float) * g.n);
  GP_CUDA_TRY(cudaMemsetAsync(w.qa, 0, sizeof(float) * g.n, g.stream));
  GP_CUDA_TRY(cudaMemsetAsync(w.qb, 0, sizeof(float) * g.n, g.stream));
  w.y = (float2*)g.alloc.get(sizeof(float2) * g.n);
  w.norms = (float*)g.alloc.get(sizeof(float) * (kPassCap + 2));
  w.state = (int*)g.alloc.get(sizeof(int) * (kPassCap + 4));
}

cudaEvent_t pooled_event(Graph& g, size_t i) {
  while (g.ev_pool.size() <= i) {
    cudaEvent_t e;
    GP_CUDA_TRY(cudaEventCreate(&e));
    g.ev_pool.push_back(e);
  }
  return g.ev_pool[i];
}

void validate_request(const Graph& g, const gp_request& r) {
  GP_REQUIRE(r.function == GP_FN_PPR || r.function == GP_FN_HKPR, "function must be GP_FN_PPR or GP_FN_HKPR");
  GP_REQUIRE(r.source >= 0 && (int64_t)r.source < g.n, "source out of range");
  if (r.function == GP_FN_PPR)
    GP_REQUIRE(r.param > 0.0 && r.param < 1.0, "alpha must be in (0, 1)");
  else
    GP_REQUIRE(r.param > 0.0 && r.param <= 1e4, "t must be in (0, 1e4]");
  GP_REQUIRE(r.l1_tol > 0.0 && r.l1_tol < 1.0, "l1_tol must be in (0, 1)");
  GP_REQUIRE(r.out_dtype == GP_F64 || r.out_dtype == GP_F32, "out_dtype must be GP_F64 or GP_F32");
  GP_REQUIRE(r.y_out != nullptr, "y_out is NULL");
  GP_REQUIRE(r.k_rule == GP_K_TAIL || r.k_rule == GP_K_PAPER || r.k_rule == GP_K_FIXED, "bad k_rule");
  if (r.k_rule == GP_K_FIXED) GP_REQUIRE(r.k_fixed >= 1 && r.k_fixed < g.cfg.k_max, "k_fixed must be in [1, k_max)");
}

template <typename OUT>
void launch_finalize(Graph& g, const gp_request& req, OUT* dst) {
  int grid = device_sms() * 4;
  finalize_kernel<OUT><<<grid, 256, 0, g.stream>>>(g.n, g.newid, g.qw.y, dst);
  GP_LAUNCHED();
}

template <typename OUT>
void launch_point(Graph& g, int64_t s, double val, OUT* dst) {
  int grid = device_sms() * 4;
  point_kernel<OUT><<<grid, 256, 0, g.stream>>>(g.n, s, val, dst);
  GP_LAUNCHED();
}

// Write the result into the caller's buffer (device directly, host through a
// staging buffer) in the caller's numbering.
void emit_output(Graph& g, const gp_request& req, bool isolated, double f0) {
  size_t esz = req.out_dtype == GP_F64 ? 8 : 4;
  void* dst = req.y_out;
  if (!req.y_on_device) {
    if (!g.qw.stage) g.qw.stage = g.alloc.get(sizeof(double) * g.n);
    dst = g.qw.stage;
  }
  if (isolated) {
    if (req.out_dtype == GP_F64) launch_point<double>(g, req.source, f0, (double*)dst);
    else launch_point<float>(g, req.source, f0, (float*)dst);
  } else {
    if (req.out_dtype == GP_F64) launch_finalize<double>(g, req, (double*)dst);
    else launch_finalize<float>(g, req, (float*)dst);
  }
  if (!req.y_on_device) {
    GP_CUDA_TRY(cudaMemcpyAsync(req.y_out, dst, esz * g.n, cudaMemcpyDeviceToHost, g.stream));
    GP_CUDA_TRY(cudaStreamSynchronize(g.stream));
  }
}

template <typename RP>
void launch_step(Graph& g, StepArgs& a, int grid) {
  static int configured = 0;  // largest dynamic shared memory size enabled so far
  if (g.sched.smem_bytes > configured) {
    GP_CUDA_TRY(cudaFuncSetAttribute(cheb_step_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     g.sched.smem_bytes));
    GP_CUDA_TRY(cudaFuncSetAttribute(cheb_step_kernel<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     g.sched.smem_bytes));
    configured = g.sched.smem_bytes;
  }
  cheb_step_kernel<RP><<<grid, kStepThreads, g.sched.smem_bytes, g.stream>>>(a);
  GP_LAUNCHED();
  if (a.nlong > 0) {
    const int lgrid = (int)std::min<int64_t>((a.nlong + kLongWarps - 1) / kLongWarps, (int64_t)grid * 16);
    cheb_long_kernel<RP><<<lgrid, 32 * kLongWarps, 0, g.stream>>>(a);
    GP_LAUNCHED();
  }
}

}  // namespace

void free_query_work(Graph& g) {
  QueryWork& w = g.qw;
  g.alloc.put(w.qa);
  g.alloc.put(w.qb);
  g.alloc.put(w.y);
  g.alloc.put(w.norms);
  g.alloc.put(w.state);
  g.alloc.put(w.stage);
  w = QueryWork{};
}

// Shared driver of the Chebyshev query and the power baseline.
static void run_single(Graph& g, const gp_request& req, gp_query_info* info, bool cheb) {
  validate_request(g, req);
  auto t0 = std::chrono::steady_clock::now();
  const int kcap = g.cfg.k_max;
  const int64_t deg_s = g.h_deg[req.source];
  const double f0 = req.function == GP_FN_PPR ? req.param : std::exp(-req.param);
  const bool sync_needed = info != nullptr || !req.y_on_device || g.profiling;
  if (deg_s == 0) {
    // P e_s = 0: r_k = T_k(0) e_s and y = sum_k c_k T_k(0) e_s -> f(0) e_s
    emit_output(g, req, true, f0);
    if (sync_needed) GP_CUDA_TRY(cudaStreamSynchronize(g.stream));
    if (info) {
      info->K = 0;
      info->k16_from = 1;
      info->tail_bound = 0.0;
      info->max_r_l1 = 1.0;
      info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return;
  }
  ensure_query_work(g);
  QueryWork& w = g.qw;
  // ---- coefficients (host FP64)
  std::vector<double> c, tail;
  int k_fixed = -1;  // < 0: stop rule on the device
  if (cheb) {
    cheb_coefficients(req.function, req.param, kcap, c, tail);
    if (req.k_rule == GP_K_PAPER) k_fixed = std::min(kcap - 1, paper_k(req.function, req.param, req.l1_tol));
    if (req.k_rule == GP_K_FIXED) k_fixed = req.k_fixed;
  } else {
    taylor_coefficients(req.function, req.param, req.l1_tol, kPassCap, c);
    tail.assign(kPassCap + 1, -1.0);
  }
  const int64_t s = g.h_newid[req.source];
  if (use_precise(g)) {
    // tiny graph: float-pair storage of Q (precise.cu)
    double C = 1.0;
    const int K = run_precise(g, s, cheb, c, tail, cheb ? k_fixed : (int)c.size() - 1, req.l1_tol / kCMargin, kcap, &C);
    emit_output(g, req, false, f0);
    if (sync_needed) GP_CUDA_TRY(cudaStreamSynchronize(g.stream));
    if (info) {
      info->K = K;
      info->k16_from = K + 1;
      info->max_r_l1 = cheb ? C : 1.0;
      info->tail_bound = cheb && K < (int)tail.size() ? kCMargin * tail[K] * C : 0.0;
      info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return;
  }
  // ---- init
  GP_CUDA_TRY(cudaMemsetAsync(w.qa, 0, sizeof(float) * g.n_active, g.stream));
  GP_CUDA_TRY(cudaMemsetAsync(w.qb, 0, sizeof(float) * g.n_active, g.stream));
  GP_CUDA_TRY(cudaMemsetAsync(w.y, 0, sizeof(float2) * g.n, g.stream));
  GP_CUDA_TRY(cudaMemsetAsync(w.norms, 0, sizeof(float) * (kPassCap + 2), g.stream));
  GP_CUDA_TRY(cudaMemsetAsync(w.state, 0, sizeof(int) * (kPassCap + 4), g.stream));
  InitArgs ia;
  ia.rp = g.rp;
  ia.ci = g.ci;
  ia.q0 = w.qa;
  ia.q1 = w.qb;
  ia.y = w.y;
  ia.norms = w.norms;
  ia.state = w.state;
  ia.s = s;
  ia.c0 = c[0];
  ia.c1 = cheb ? c[1] : 0.0;
  ia.kcap = kcap;
  ia.cheb = cheb ? 1 : 0;
  {
    int blocks = (int)std::min<int64_t>(std::max<int64_t>((deg_s + 255) / 256, 1), device_sms() * 4);
    if (g.rp64) cheb_init_kernel<int64_t><<<blocks, 256, 0, g.stream>>>(ia);
    else cheb_init_kernel<int32_t><<<blocks, 256, 0, g.stream>>>(ia);
    GP_LAUNCHED();
  }
  // ---- passes
  StepArgs a;
  a.tiles = g.sched.tiles;
  a.ntiles = g.sched.ntiles;
  a.poff = g.sched.poff;
  a.part = g.sched.part;
  a.nlong = g.sched.nlong;
  a.hub = g.sched.hub;
  a.rp = g.rp;
  a.ci = g.ci;
  a.y = w.y;
  a.norms = w.norms;
  a.state = w.state;
  a.tol = (float)(req.l1_tol / kCMargin);
  a.cheb = cheb ? 1 : 0;
  const int grid = step_grid(g);
  float* bufs[2] = {w.qa, w.qb};  // bufs[k & 1] holds Q_k
  int K_done = -1;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> prof_marks;  // (k, first event index)
  auto launch_pass = [&](int k, bool test) {
    a.k = k;
    float2 ck = split_df(c[k + 1]);
    a.c_hi = ck.x;
    a.c_lo = ck.y;
    a.tail = test ? (float)tail[k] : -1.0f;
    a.qcur = bufs[k & 1];
    a.qprev = bufs[(k + 1) & 1];
    if (g.profiling) {
      GP_CUDA_TRY(cudaEventRecord(pooled_event(g, ev_used), g.stream));
      prof_marks.push_back({k, ev_used});
      ev_used += 2;
    }
    if (g.rp64) launch_step<int64_t>(g, a, grid);
    else launch_step<int32_t>(g, a, grid);
    if (g.profiling) GP_CUDA_TRY(cudaEventRecord(pooled_event(g, prof_marks.back().second + 1), g.stream));
  };
  if (!cheb) {
    // Power baseline (Algorithm 1): the init left Q_0 = e_s/d_s in bufs[0] and
    // y = zeta_0 e_s; pass k computes r_{k+1} = P r_k over every active row
    // (so every application of P runs through the step kernel) and adds
    // zeta_{k+1} r_{k+1}.  N = c.size() terms -> passes k = 0 .. N-2.
    int N = (int)c.size();
    for (int k = 0; k + 1 < N; ++k) launch_pass(k, false);
    K_done = N - 1;
  } else if (k_fixed >= 1) {
    for (int k = 1; k < k_fixed; ++k) launch_pass(k, false);
    K_done = k_fixed;
  } else {
    // Stop rule: no stop is possible before k_lo (max ||r_l||_1 >= ||r_0||_1 = 1);
    // launch up to k_lo + chunk, then read K back and continue if needed.
    int k_lo = k_lower(tail, req.l1_tol / kCMargin, 1.0);
    const int chunk = 6;
    int k = 1;
    int limit = std::min(kcap - 1, k_lo + chunk);
    int* hstate = nullptr;
    int hbuf = 0;
    hstate = &hbuf;
    for (;;) {
      for (; k <= limit; ++k) launch_pass(k, true);
      GP_CUDA_TRY(cudaMemcpyAsync(hstate, w.state, sizeof(int), cudaMemcpyDeviceToHost, g.stream));
      GP_CUDA_TRY(cudaStreamSynchronize(g.stream));
      if (*hstate < kcap || limit >= kcap - 1) break;
      limit = std::min(kcap - 1, limit + chunk);
    }
    K_done = *hstate < kcap ? *hstate : kcap;  // kcap: the cap was reached
  }
  emit_output(g, req, false, f0);
  if (sync_needed) GP_CUDA_TRY(cudaStreamSynchronize(g.stream));
  if (g.profiling) {
    double bytes = step_bytes_single(g);
    for (auto& m : prof_marks) {
      // passes for k >= K_done returned without work
      if (cheb && k_fixed < 1 && m.first >= K_done) continue;
      float ms = 0.f;
      GP_CUDA_TRY(cudaEventElapsedTime(&ms, g.ev_pool[m.second], g.ev_pool[m.second + 1]));
      g.prof_ms += ms;
      g.prof_launches += 1;
      g.prof_bytes += bytes;
    }
  }
  if (info) {
    std::vector<float> nr(kPassCap + 2);
    GP_CUDA_TRY(cudaMemcpyAsync(nr.data(), w.norms, sizeof(float) * (kPassCap + 2), cudaMemcpyDeviceToHost,
                                g.stream));
    GP_CUDA_TRY(cudaStreamSynchronize(g.stream));
    double C = 0.0;
    int Kr = std::min(K_done, kPassCap);
    for (int l = 0; l <= Kr; ++l) C = std::max(C, (double)nr[l]);
    info->K = K_done;
    info->k16_from = K_done + 1;
    info->max_r_l1 = cheb ? C : 1.0;
    if (cheb) {
      info->tail_bound = Kr < (int)tail.size() ? kCMargin * tail[Kr] * C : 0.0;
    } else {
      double t = 0.0;  // Taylor tail beyond the N terms used, ||P^k e_s||_1 = 1
      std::vector<double> zall;
      taylor_coefficients(req.function, req.param, 0.0, (int)c.size() + 4096, zall);
      for (size_t k2 = c.size(); k2 < zall.size(); ++k2) t += zall[k2];
      info->tail_bound = t;
    }
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
}

void run_query(Graph& g, const gp_request& req, gp_query_info* info) { run_single(g, req, info, true); }
void run_power(Graph& g, const gp_request& req, gp_query_info* info) { run_single(g, req, info, false); }

}  // namespace gp
