// ChebyPush (Algorithm 4) on the device: the subset Chebyshev recurrence of
// Eq. (subset-cheby-implement), carried out by pushes from the nodes whose
// residual exceeds the iteration's threshold.
//
//   y = c_0 e_s; r_cur = P e_s; r_new = -e_s
//   for k = 1 .. K-1:
//     S_k = {u : |r_cur(u)| > eps_k d_u},  eps_k = eps_a / (4 K sum_{l=k}^K |c_l|)
//     for u in S_k: y(u) += c_k r_cur(u); r_new(v) += 2 r_cur(u) / d_u (v in N(u));
//                   r_cur(u) = -r_cur(u)
//     swap(r_cur, r_new)
//
// Each iteration is two kernels over the relabelled graph.  The scan reads
// r_cur over all rows, applies the y update and the sign flip to the
// nodes of S_k, and appends them to a frontier (a row longer than kPushChunk
// entries becomes several frontier entries, so no warp is left with a hub).
// The push scatters 2 r_cur(u) / d_u to the neighbours with FP64 atomic adds,
// a warp per frontier entry.  The pushes of one iteration write r_new only, so
// their order changes only the rounding of r_new; the vectors are FP64 so that
// the threshold decisions follow the FP64 reference.  Scanning every row
// costs 8 bytes per row and iteration; the pushes cost what the frontier
// holds.  The work vectors are allocated at the graph's first push query and
// kept with the graph (PushWork), so a query allocates nothing.  The
// kernels read the query's source and (c_k, eps_k) from a small device block,
// so the whole launch sequence of the push phase (memsets, init, K - 1 scans
// and scatters) is captured once per K into a CUDA graph and replayed: one
// launch per query instead of 2K, which is what bounds a query at large eps_a.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "gp_internal.h"

namespace gp {

namespace {

constexpr int kPushChunk = 2048;  // entries of one frontier item
constexpr int kPushKCap = 1024;   // longest iteration count of a push query

// A query's parameters, read by the kernels from device memory so that one
// captured launch sequence per K serves every source and coefficient set:
// the source (relabelled), the rows the scans cover, and (c_k, eps_k) for
// k = 0..K.  Only rows with neighbours can hold a residual unless the source
// itself is isolated (or an asymmetric CSR lists edges into rows without
// neighbours), so the scans cover the non-isolated prefix of the relabelled
// rows (isolated rows come last), or else all rows.
struct PushParams {
  long long s;
  long long rows;
  double2 ce[kPushKCap + 1];
};

template <typename RP>
__global__ void push_init_kernel(const RP* rp, const int32_t* ci, const PushParams* pp, double* rcur, double* rnew,
                                 double* y) {
  const int64_t s = pp->s;
  const double c0 = pp->ce[0].x;
  const int64_t beg = rp[s], end = rp[s + 1];
  const double inv = 1.0 / (double)(end - beg);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    y[s] = c0;
    rnew[s] = -1.0;
  }
  for (int64_t e = beg + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < end; e += (int64_t)gridDim.x * blockDim.x)
    rcur[ci[e]] = inv;  // (P e_s)(v) = 1 / d_s for v in N(s)
}

// S_k: y += c_k r, r -> -r, and frontier items {u, chunk} with the pushed value.
template <typename RP>
__global__ void push_scan_kernel(const RP* rp, double* rcur, double* y, const PushParams* pp, int k, int2* fr,
                                 double* fval, int* count) {
  const int lane = threadIdx.x & 31;
  const int64_t n = pp->rows;
  const double ck = pp->ce[k].x, eps = pp->ce[k].y;
  for (int64_t u0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; u0 < n;
       u0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = u0 + lane;
    int items = 0;  // a row of degree 0 (a node only an asymmetric CSR lists) pushes nothing
    double r = 0.0, d = 0.0;
    if (u < n) {
      r = rcur[u];
      d = (double)(rp[u + 1] - rp[u]);
      if (fabs(r) > eps * d) {
        y[u] += ck * r;
        rcur[u] = -r;
        items = (int)((rp[u + 1] - rp[u] + kPushChunk - 1) / kPushChunk);
      }
    }
    // warp-aggregated reservation of the frontier slots
    int incl = items;
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(count, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    const int first = base + incl - items;
    for (int j = 0; j < items; ++j) {
      fr[first + j] = make_int2((int)u, j);
      fval[first + j] = 2.0 * r / d;
    }
  }
}

template <typename RP>
__global__ void push_scatter_kernel(const RP* rp, const int32_t* ci, const int2* fr, const double* fval,
                                    const int* count, double* rnew) {
  const int lane = threadIdx.x & 31;
  const int n = *count;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const int2 it = fr[i];
    const double v = fval[i];
    const int64_t beg = rp[it.x] + (int64_t)it.y * kPushChunk;
    const int64_t end = min(beg + (int64_t)kPushChunk, (int64_t)rp[it.x + 1]);
    for (int64_t e = beg + lane; e < end; e += 32) atomicAdd(&rnew[ci[e]], v);
  }
}

// y (relabelled) -> the caller's numbering.
template <typename OUT>
__global__ void push_output_kernel(int64_t n, const int32_t* newid, const double* y, OUT* out) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    out[u] = (OUT)y[newid[u]];
}

// ---- Algorithm 5 (ChebyPush + alpha-random walks) for SSPPR

// SplitMix64 (Steele, Lea and Flood, 2014): state += golden gamma, output =
// the finaliser of the state.  Walk j from node v (caller numbering) draws
// from the stream seeded by mix(seed ^ mix(v * gamma + j)).
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  return sm64_mix(state);
}

// r = e_s - alpha^-1 [I - (1 - alpha) P] pi^ over all rows (FP64, a warp per row).
template <typename RP>
__global__ void bidir_residual_kernel(int64_t n, const RP* rp, const int32_t* ci, int64_t s, double alpha,
                                      const double* y, double* r) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    double acc = 0.0;
    for (int64_t e = rp[u] + lane; e < rp[u + 1]; e += 32) {
      const int32_t v = ci[e];
      const int64_t dv = rp[v + 1] - rp[v];
      if (dv > 0) acc += y[v] / (double)dv;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) r[u] = (u == s ? 1.0 : 0.0) - (y[u] - (1.0 - alpha) * acc) / alpha;
  }
}

// W_v = ceil(|r(v)| W) alpha-random walks from every v with r(v) != 0 (a warp
// per v, its lanes over the walks); each adds r(v) / W_v where it stops.
template <typename RP>
__global__ void bidir_walk_kernel(int64_t n, const RP* rp, const int32_t* ci, const int32_t* order, double alpha,
                                  double W, uint64_t seed, const double* r, double* y,
                                  unsigned long long* walks) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long mine = 0;
  for (int64_t v0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v0 < n; v0 += nw) {
    const double rv = r[v0];
    if (rv == 0.0) continue;
    const int64_t Wv = (int64_t)ceil(fabs(rv) * W);
    const double add = rv / (double)Wv;
    const uint64_t vid = (uint64_t)order[v0];
    for (int64_t j = lane; j < Wv; j += 32) {
      uint64_t state = sm64_mix(seed ^ sm64_mix(vid * 0x9E3779B97F4A7C15ull + (uint64_t)j));
      int64_t v = v0;
      for (;;) {
        const uint64_t z = sm64_next(state);
        const double u01 = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        const int64_t d = rp[v + 1] - rp[v];
        if (u01 < alpha || d == 0) break;
        const uint64_t z2 = sm64_next(state);
        v = ci[rp[v] + (int64_t)(((z2 >> 32) * (uint64_t)d) >> 32)];
      }
      atomicAdd(&y[v], add);
    }
    if (lane == 0) mine += (unsigned long long)Wv;
  }
  if (mine) atomicAdd(walks, mine);
}

int sms() {
  int dev = 0, s = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
  return s > 0 ? s : 1;
}

// The graph's push work vectors (allocated once); the host-output staging
// buffer only when a query writes to host memory.
PushWork& push_work(Graph& g, bool need_stage) {
  PushWork& w = g.pw;
  Allocator& A = g.alloc;
  const int64_t n = std::max<int64_t>(g.n, 1), na = std::max<int64_t>(g.n_active, 1);
  if (!w.ra) {
    // frontier: at most one item per kPushChunk entries plus one per row
    const int64_t cap = na + g.nnz / kPushChunk + 1;
    PushWork t;
    try {
      t.ra = (double*)A.get(sizeof(double) * n);
      t.rb = (double*)A.get(sizeof(double) * n);
      t.y = (double*)A.get(sizeof(double) * n);
      t.fr = (int2*)A.get(sizeof(int2) * cap);
      t.fval = (double*)A.get(sizeof(double) * cap);
      t.counts = (int*)A.get(sizeof(int) * (kPushKCap + 1));
      t.walks = (unsigned long long*)A.get(sizeof(unsigned long long));
    } catch (...) {
      for (void* p : {(void*)t.ra, (void*)t.rb, (void*)t.y, (void*)t.fr, (void*)t.fval, (void*)t.counts,
                      (void*)t.walks})
        A.put(p);
      throw;
    }
    w = t;
  }
  if (need_stage && !w.stage) w.stage = A.get(sizeof(double) * n);
  return w;
}

// Per graph: the pinned and device copies of the query parameters and one
// instantiated CUDA graph per iteration count K (the launch sequence below,
// captured once; the work vectors are the graph's and do not move).  Kept
// beside the graph's PushWork and released with it.
struct PushGraphs {
  PushParams* h = nullptr;  // pinned host
  PushParams* d = nullptr;  // device
  int* h_counts = nullptr;  // pinned host copy of the frontier sizes
  std::map<int, cudaGraphExec_t> exec;
};
std::mutex g_push_mu;
std::map<const Graph*, PushGraphs> g_push;

PushGraphs& push_graphs(Graph& g) {
  std::lock_guard<std::mutex> lk(g_push_mu);
  PushGraphs& pg = g_push[&g];
  if (!pg.h) {
    GP_CUDA_TRY(cudaHostAlloc((void**)&pg.h, sizeof(PushParams), cudaHostAllocDefault));
    GP_CUDA_TRY(cudaHostAlloc((void**)&pg.h_counts, sizeof(int) * (kPushKCap + 1), cudaHostAllocDefault));
    pg.d = (PushParams*)g.alloc.get(sizeof(PushParams));
  }
  return pg;
}

// The push phase of one query: zero the vectors, y = c_0 e_s, r_cur = P e_s,
// r_new = -e_s, then K - 1 iterations of scan + scatter (the vectors swap
// roles each iteration; y ends in w.y).  Stream-ordered on g.stream; no
// allocation and no synchronisation, so it can be captured.
template <typename RP>
void push_sequence(Graph& g, PushWork& w, const PushParams* pp, int K) {
  cudaStream_t st = g.stream;
  const RP* rp = (const RP*)g.rp;
  const int64_t n = std::max<int64_t>(g.n, 1);
  GP_CUDA_TRY(cudaMemsetAsync(w.ra, 0, sizeof(double) * n, st));
  GP_CUDA_TRY(cudaMemsetAsync(w.rb, 0, sizeof(double) * n, st));
  GP_CUDA_TRY(cudaMemsetAsync(w.y, 0, sizeof(double) * n, st));
  GP_CUDA_TRY(cudaMemsetAsync(w.counts, 0, sizeof(int) * (K + 1), st));
  double *rcur = w.ra, *rnew = w.rb;
  push_init_kernel<RP><<<4, 256, 0, st>>>(rp, g.ci, pp, rcur, rnew, w.y);
  GP_CUDA_TRY(cudaGetLastError());
  const int grid = sms() * 8;
  for (int k = 1; k < K; ++k) {
    push_scan_kernel<RP><<<grid, 256, 0, st>>>(rp, rcur, w.y, pp, k, w.fr, w.fval, w.counts + k);
    GP_CUDA_TRY(cudaGetLastError());
    push_scatter_kernel<RP><<<grid, 256, 0, st>>>(rp, g.ci, w.fr, w.fval, w.counts + k, rnew);
    GP_CUDA_TRY(cudaGetLastError());
    std::swap(rcur, rnew);
  }
}

// Run the push phase for source s (relabelled) with thresholds
// eps_k = eps_a / (4 K sum_{l=k}^K |c_l|): upload the parameters, then replay
// the graph captured for this K (capturing it on first use).
void run_push(Graph& g, PushWork& w, int64_t s, const std::vector<double>& c, int K, double eps_a) {
  PushGraphs& pg = push_graphs(g);
  pg.h->s = (long long)s;
  // (an unvalidated asymmetric CSR can push into rows without neighbours)
  pg.h->rows = s < g.n_active && !g.ci_beyond_active ? (long long)g.n_active : (long long)g.n;
  for (int k = 0; k <= K; ++k) {
    double tailK = 0.0;
    for (int l = k; l <= K; ++l) tailK += std::fabs(c[l]);
    pg.h->ce[k] = make_double2(c[k], k >= 1 && tailK > 0.0 ? eps_a / (4.0 * K * tailK) : 0.0);
  }
  cudaStream_t st = g.stream;
  GP_CUDA_TRY(cudaMemcpyAsync(pg.d, pg.h, 16 + sizeof(double2) * (K + 1), cudaMemcpyHostToDevice, st));
  auto it = pg.exec.find(K);
  if (it == pg.exec.end()) {
    cudaGraph_t graph = nullptr;
    GP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      if (g.rp64)
        push_sequence<int64_t>(g, w, pg.d, K);
      else
        push_sequence<int32_t>(g, w, pg.d, K);
    } catch (...) {
      cudaStreamEndCapture(st, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    GP_CUDA_TRY(cudaStreamEndCapture(st, &graph));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    GP_CUDA_TRY(e);
    it = pg.exec.emplace(K, exec).first;
  }
  GP_CUDA_TRY(cudaGraphLaunch(it->second, st));
  count_launch(1 + 2 * (uint64_t)(K - 1));
}

void free_push_graphs(Graph& g) {
  std::lock_guard<std::mutex> lk(g_push_mu);
  auto it = g_push.find(&g);
  if (it == g_push.end()) return;
  PushGraphs& pg = it->second;
  for (auto& kv : pg.exec) cudaGraphExecDestroy(kv.second);
  if (pg.h) cudaFreeHost(pg.h);
  if (pg.h_counts) cudaFreeHost(pg.h_counts);
  g.alloc.put(pg.d);
  g_push.erase(it);
}

}  // namespace

void run_chebypush(Graph& g, int function, int32_t source, double param, double eps_a, int K, gp_dtype out_dtype,
                   void* y_out, int y_on_device, gp_query_info* info) {
  GP_REQUIRE(function == GP_FN_PPR || function == GP_FN_HKPR, "function must be GP_FN_PPR or GP_FN_HKPR");
  GP_REQUIRE(source >= 0 && (int64_t)source < g.n, "source out of range");
  if (function == GP_FN_PPR)
    GP_REQUIRE(param > 0.0 && param < 1.0, "alpha must be in (0, 1)");
  else
    GP_REQUIRE(param > 0.0 && param <= 1e4, "t must be in (0, 1e4]");
  GP_REQUIRE(eps_a > 0.0 && eps_a < 1.0, "eps_a must be in (0, 1)");
  GP_REQUIRE(K >= 0 && K <= 1024, "K must be in [0, 1024] (0: from eps_a)");
  GP_REQUIRE(out_dtype == GP_F64 || out_dtype == GP_F32, "out_dtype must be GP_F64 or GP_F32");
  GP_REQUIRE(y_out != nullptr, "y_out is NULL");
  auto t0 = std::chrono::steady_clock::now();
  // K: Algorithm 4 adds c_0 .. c_{K-1}; by default the smallest K whose
  // truncation tail(K-1) = sum_{l>=K} |c_l| is at most eps_a / 2 (Theorem 3)
  // (coefficients up to 128 first: the usual K is far below, and the table
  // costs host time on every query)
  std::vector<double> c, tail;
  const int kc = K > 0 ? K : 128;
  cheb_coefficients(function, param, kc, c, tail);
  if (K == 0) {
    K = 1;
    while (K < kc && tail[K - 1] > eps_a / 2) ++K;
    if (tail[K - 1] > eps_a / 2) {
      cheb_coefficients(function, param, 1024, c, tail);
      while (K < 1024 && tail[K - 1] > eps_a / 2) ++K;
    }
  }
  const size_t esz = out_dtype == GP_F64 ? 8 : 4;
  cudaStream_t st = g.stream;
  int64_t pushed = 0;
  if (g.h_deg[source] == 0) {
    // an isolated source: r_k = T_k(0) e_s; the sum is f(0) e_s up to the truncation
    double v = 0.0;
    for (int k = 0; k < K; k += 2) v += (k % 4 == 0 ? 1.0 : -1.0) * c[k];
    std::vector<unsigned char> host(esz * g.n, 0);
    if (out_dtype == GP_F64) reinterpret_cast<double*>(host.data())[source] = v;
    else reinterpret_cast<float*>(host.data())[source] = (float)v;
    GP_CUDA_TRY(cudaMemcpyAsync(y_out, host.data(), host.size(),
                                y_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    PushWork& w = push_work(g, !y_on_device);
    try {
      run_push(g, w, g.h_newid[source], c, K, eps_a);
      void* dst = y_on_device ? y_out : w.stage;
      const int grid = sms() * 4;
      if (out_dtype == GP_F64)
        push_output_kernel<double><<<grid, 256, 0, st>>>(g.n, g.newid, w.y, (double*)dst);
      else
        push_output_kernel<float><<<grid, 256, 0, st>>>(g.n, g.newid, w.y, (float*)dst);
      GP_LAUNCHED();
      if (!y_on_device) GP_CUDA_TRY(cudaMemcpyAsync(y_out, w.stage, esz * g.n, cudaMemcpyDeviceToHost, st));
      PushGraphs& pg = push_graphs(g);
      GP_CUDA_TRY(cudaMemcpyAsync(pg.h_counts, w.counts, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, st));
      GP_CUDA_TRY(cudaStreamSynchronize(st));
      for (int k = 1; k < K; ++k) pushed += pg.h_counts[k];
    } catch (...) {
      cudaStreamSynchronize(st);
      throw;
    }
  }
  if (info) {
    info->K = K;
    info->k16_from = K + 1;
    info->tail_bound = tail[K - 1];
    info->max_r_l1 = (double)pushed;  // for ChebyPush: frontier items pushed over all iterations
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
}

void run_bidirectional(Graph& g, int32_t source, double alpha, double eps_r, double delta, int K, uint64_t seed,
                       gp_dtype out_dtype, void* y_out, int y_on_device, gp_query_info* info) {
  GP_REQUIRE(source >= 0 && (int64_t)source < g.n, "source out of range");
  GP_REQUIRE(alpha > 0.0 && alpha < 1.0, "alpha must be in (0, 1)");
  GP_REQUIRE(eps_r > 0.0 && delta > 0.0 && delta <= 1.0, "eps_r must be > 0 and delta in (0, 1]");
  GP_REQUIRE(g.n >= 2, "the graph needs at least two nodes");
  GP_REQUIRE(K >= 0 && K <= 1024, "K must be in [0, 1024] (0: the paper's K)");
  GP_REQUIRE(out_dtype == GP_F64 || out_dtype == GP_F32, "out_dtype must be GP_F64 or GP_F32");
  GP_REQUIRE(y_out != nullptr, "y_out is NULL");
  auto t0 = std::chrono::steady_clock::now();
  const double W = 2.0 * (2.0 * eps_r / 3.0 + 2.0) * std::log((double)g.n) / (eps_r * eps_r * delta);
  const double rmax = std::sqrt(alpha) / W;
  if (K == 0) K = std::max(1, std::min(1024, (int)std::ceil(std::log(1.0 / rmax) / std::sqrt(alpha))));
  std::vector<double> c, tail;
  cheb_coefficients(GP_FN_PPR, alpha, std::max(K, 1), c, tail);
  const size_t esz = out_dtype == GP_F64 ? 8 : 4;
  cudaStream_t st = g.stream;
  PushWork& w = push_work(g, !y_on_device);
  const int64_t n = g.n;
  double *ra = w.ra, *y = w.y;
  unsigned long long h_walks = 0;
  try {
    const int64_t s = g.h_newid[source];
    const int grid = sms() * 8;
    // pi^ = ChebyPush(G, f, s, K, r_max); then r into ra (free after the push)
    run_push(g, w, s, c, K, rmax);
    GP_CUDA_TRY(cudaMemsetAsync(w.walks, 0, sizeof(unsigned long long), st));
    if (g.rp64) {
      bidir_residual_kernel<int64_t><<<grid, 256, 0, st>>>(n, (const int64_t*)g.rp, g.ci, s, alpha, y, ra);
      GP_LAUNCHED();
      bidir_walk_kernel<int64_t><<<grid, 256, 0, st>>>(n, (const int64_t*)g.rp, g.ci, g.order, alpha, W, seed, ra,
                                                       y, w.walks);
    } else {
      bidir_residual_kernel<int32_t><<<grid, 256, 0, st>>>(n, (const int32_t*)g.rp, g.ci, s, alpha, y, ra);
      GP_LAUNCHED();
      bidir_walk_kernel<int32_t><<<grid, 256, 0, st>>>(n, (const int32_t*)g.rp, g.ci, g.order, alpha, W, seed, ra,
                                                       y, w.walks);
    }
    GP_LAUNCHED();
    void* dst = y_on_device ? y_out : w.stage;
    if (out_dtype == GP_F64)
      push_output_kernel<double><<<sms() * 4, 256, 0, st>>>(g.n, g.newid, y, (double*)dst);
    else
      push_output_kernel<float><<<sms() * 4, 256, 0, st>>>(g.n, g.newid, y, (float*)dst);
    GP_LAUNCHED();
    if (!y_on_device) GP_CUDA_TRY(cudaMemcpyAsync(y_out, w.stage, esz * g.n, cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaMemcpyAsync(&h_walks, w.walks, sizeof(h_walks), cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    throw;
  }
  if (info) {
    info->K = K;
    info->k16_from = K + 1;
    info->tail_bound = rmax;            // the push threshold r_max of Algorithm 5
    info->max_r_l1 = (double)h_walks;   // random walks run
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
}

void free_push_work(Graph& g) {
  free_push_graphs(g);
  PushWork& w = g.pw;
  for (void* p : {(void*)w.ra, (void*)w.rb, (void*)w.y, (void*)w.fr, (void*)w.fval, (void*)w.counts,
                  (void*)w.walks, w.stage})
    g.alloc.put(p);
  w = PushWork{};
}

}  // namespace gp
