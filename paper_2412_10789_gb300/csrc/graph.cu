// Graph ingest (gp_graph_create / gp_graph_export / gp_graph_destroy).
//
// The caller's CSR (Section 2.1: undirected, both directions stored) is
// validated and stored relabelled: rows ordered by degree, descending, ties by
// caller id (a stable counting sort on the host, O(n + max degree)).  Column
// ids are rewritten on the device.  With that order the degree buckets of the
// fused step are contiguous row ranges, the most-gathered rows (hubs) share
// cache lines, and isolated rows (degree 0) form a tail the step never visits.
#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "gp_internal.h"

namespace gp {

void* Allocator::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (alloc) {
    p = alloc(bytes, ctx);
    if (!p) throw Error{GP_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{GP_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
    }
  }
  return p;
}

void Allocator::put(void* p) {
  if (!p) return;
  if (free)
    free(p, ctx);
  else
    cudaFree(p);
}

namespace {

// Error word written by the validation kernels: [0] = smallest bad row,
// [1] = OR of the codes below.
enum : unsigned long long {
  V_RANGE = 1,     // col_idx outside [0, n)
  V_SELF = 2,      // self-loop
  V_ORDER = 4,     // row not strictly increasing (unsorted or duplicate)
  V_ASYM = 8,      // (u, v) present without (v, u)
};

template <typename RP>
__global__ void validate_rows_kernel(int64_t n, const RP* __restrict__ rp, const int32_t* __restrict__ ci,
                                     int check_sym, unsigned long long* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    int64_t beg = rp[u], end = rp[u + 1];
    unsigned long long code = 0;
    for (int64_t e = beg + lane; e < end; e += 32) {
      int32_t v = ci[e];
      if (v < 0 || v >= n) { code |= V_RANGE; continue; }
      if (v == u) code |= V_SELF;
      if (e > beg && ci[e - 1] >= v) code |= V_ORDER;
      if (check_sym) {
        // binary search u in row v (rows are sorted when V_ORDER is clear)
        int64_t lo = rp[v], hi = rp[v + 1];
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (ci[mid] < u) lo = mid + 1; else hi = mid;
        }
        if (lo >= rp[v + 1] || ci[lo] != u) code |= V_ASYM;
      }
    }
    for (int off = 16; off > 0; off >>= 1) code |= __shfl_xor_sync(0xffffffffu, code, off);
    if (code && lane == 0) {
      atomicMin(&err[0], (unsigned long long)u);
      atomicOr(&err[1], code);
    }
  }
}

// new_ci[new_rp[i] + j] = newid[ci[rp[order[i]] + j]]  (one warp per new row)
// (*beyond is set when an entry names a node of degree 0, i.e. a relabelled
// id >= n_active: possible only for an unvalidated asymmetric CSR.)
template <typename RP>
__global__ void renumber_kernel(int64_t n, const RP* __restrict__ rp, const int32_t* __restrict__ ci,
                                const RP* __restrict__ new_rp, const int32_t* __restrict__ order,
                                const int32_t* __restrict__ newid, int32_t* __restrict__ new_ci,
                                int64_t n_active, int* beyond) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool far = false;
  for (int64_t i = warp; i < n; i += nwarps) {
    int64_t u = order[i];
    int64_t src = rp[u], dst = new_rp[i], d = new_rp[i + 1] - dst;
    for (int64_t j = lane; j < d; j += 32) {
      const int32_t v = newid[ci[src + j]];
      new_ci[dst + j] = v;
      far |= v >= n_active;
    }
  }
  if (far) *beyond = 1;
}

// Inverse of renumber_kernel: rows back to the caller's numbering.
template <typename RP>
__global__ void export_kernel(int64_t n, const RP* __restrict__ new_rp, const int32_t* __restrict__ new_ci,
                              const int64_t* __restrict__ out_rp, const int32_t* __restrict__ order,
                              const int32_t* __restrict__ newid, int32_t* __restrict__ out_ci) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    int64_t i = newid[u];
    int64_t src = new_rp[i], dst = out_rp[u], d = new_rp[i + 1] - src;
    for (int64_t j = lane; j < d; j += 32) out_ci[dst + j] = order[new_ci[src + j]];
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename T>
struct Tmp {  // device scratch released on scope exit
  Allocator* a;
  T* p = nullptr;
  Tmp(Allocator* al, size_t count) : a(al) { p = (T*)a->get(sizeof(T) * std::max<size_t>(count, 1)); }
  ~Tmp() { a->put(p); }
};

}  // namespace

double step_bytes_single(const Graph& g) {
  // col_idx once, row_ptr of the active rows, Q_k gathered once, Q_{k-1} read,
  // Q_{k+1} written (4 B each), y read + written (8 B each).
  double w_rp = g.rp64 ? 8.0 : 4.0;
  return 4.0 * (double)g.nnz + w_rp * (double)(g.n_active + 1) + 3.0 * 4.0 * (double)g.n_active +
         2.0 * 8.0 * (double)g.n_active;
}

namespace {

template <typename RP>
void ingest(Graph& g, const void* row_ptr_in, int in_rp64, const int32_t* col_idx, const int32_t* degree,
            int on_device) {
  const int64_t n = g.n, nnz = g.nnz;
  cudaStream_t st = g.stream;
  // ---- host copies of row_ptr and degree
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> deg(n);
  if (on_device) {
    if (in_rp64) {
      GP_CUDA_TRY(cudaMemcpyAsync(rp.data(), row_ptr_in, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    } else {
      std::vector<int32_t> r32(n + 1);
      GP_CUDA_TRY(cudaMemcpyAsync(r32.data(), row_ptr_in, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, st));
      GP_CUDA_TRY(cudaStreamSynchronize(st));
      for (int64_t i = 0; i <= n; ++i) rp[i] = r32[i];
    }
    GP_CUDA_TRY(cudaMemcpyAsync(deg.data(), degree, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    if (in_rp64) {
      std::memcpy(rp.data(), row_ptr_in, sizeof(int64_t) * (n + 1));
    } else {
      const int32_t* r32 = (const int32_t*)row_ptr_in;
      for (int64_t i = 0; i <= n; ++i) rp[i] = r32[i];
    }
    std::memcpy(deg.data(), degree, sizeof(int32_t) * n);
  }
  // ---- row-level validation (exact integer comparisons)
  if (rp[0] != 0) throw Error{GP_EINVAL, "row_ptr[0] != 0"};
  if (rp[n] != nnz) throw Error{GP_EINVAL, "row_ptr[n] != nnz"};
  int64_t maxdeg = 0, n_active = 0;
  for (int64_t u = 0; u < n; ++u) {
    int64_t d = rp[u + 1] - rp[u];
    if (d < 0) throw Error{GP_EINVAL, "row_ptr decreases at row " + std::to_string(u)};
    if ((int64_t)deg[u] != d)
      throw Error{GP_EINVAL, "degree[" + std::to_string(u) + "] = " + std::to_string(deg[u]) +
                                 " but the row has " + std::to_string(d) + " entries"};
    maxdeg = std::max(maxdeg, d);
    n_active += d > 0;
  }
  g.max_degree = maxdeg;
  g.n_active = n_active;
  // ---- relabel: stable counting sort by degree, descending
  std::vector<int64_t> start(maxdeg + 2, 0);
  for (int64_t u = 0; u < n; ++u) start[maxdeg - deg[u] + 1]++;
  for (int64_t b = 0; b <= maxdeg; ++b) start[b + 1] += start[b];
  std::vector<int32_t> order(n), newid(n);
  for (int64_t u = 0; u < n; ++u) {
    int64_t i = start[maxdeg - deg[u]]++;
    order[i] = (int32_t)u;
    newid[u] = (int32_t)i;
  }
  std::vector<int64_t> nrp(n + 1);
  nrp[0] = 0;
  for (int64_t i = 0; i < n; ++i) nrp[i + 1] = nrp[i] + deg[order[i]];
  // ---- device copies
  Allocator* A = &g.alloc;
  std::vector<RP> nrp_t(n + 1), rp_t(n + 1);
  for (int64_t i = 0; i <= n; ++i) {
    nrp_t[i] = (RP)nrp[i];
    rp_t[i] = (RP)rp[i];
  }
  g.rp = A->get(sizeof(RP) * (n + 1));
  // col_idx is padded to a whole 16-byte vector plus one: the step kernel reads
  // it as aligned int4 vectors that may extend past the last entry.
  const int64_t ci_alloc = ((nnz + 3) / 4) * 4 + 4;
  g.ci = (int32_t*)A->get(sizeof(int32_t) * ci_alloc);
  GP_CUDA_TRY(cudaMemsetAsync(g.ci + nnz, 0, sizeof(int32_t) * (ci_alloc - nnz), st));
  g.order = (int32_t*)A->get(sizeof(int32_t) * n);
  g.newid = (int32_t*)A->get(sizeof(int32_t) * n);
  GP_CUDA_TRY(cudaMemcpyAsync(g.rp, nrp_t.data(), sizeof(RP) * (n + 1), cudaMemcpyHostToDevice, st));
  GP_CUDA_TRY(cudaMemcpyAsync(g.order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  GP_CUDA_TRY(cudaMemcpyAsync(g.newid, newid.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  Tmp<RP> orp(A, n + 1);
  GP_CUDA_TRY(cudaMemcpyAsync(orp.p, rp_t.data(), sizeof(RP) * (n + 1), cudaMemcpyHostToDevice, st));
  std::unique_ptr<Tmp<int32_t>> oci;
  const int32_t* ci_src = col_idx;
  if (!on_device) {
    oci.reset(new Tmp<int32_t>(A, nnz));
    if (nnz) GP_CUDA_TRY(cudaMemcpyAsync(oci->p, col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
    ci_src = oci->p;
  }
  // ---- column-level validation on the device
  Tmp<unsigned long long> err(A, 2);
  unsigned long long init[2] = {~0ULL, 0ULL};
  GP_CUDA_TRY(cudaMemcpyAsync(err.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
  int grid = sm_count() * 8;
  validate_rows_kernel<RP><<<grid, 256, 0, st>>>(n, orp.p, ci_src, g.cfg.validate_symmetry, err.p);
  GP_LAUNCHED();
  unsigned long long res[2];
  GP_CUDA_TRY(cudaMemcpyAsync(res, err.p, sizeof(res), cudaMemcpyDeviceToHost, st));
  GP_CUDA_TRY(cudaStreamSynchronize(st));
  if (res[1]) {
    std::string what;
    if (res[1] & V_RANGE) what += " column index out of range;";
    if (res[1] & V_SELF) what += " self-loop;";
    if (res[1] & V_ORDER) what += " row not strictly increasing (unsorted or duplicate);";
    if (res[1] & V_ASYM) what += " edge without its reverse (not symmetric);";
    throw Error{GP_EINVAL, "invalid CSR at row " + std::to_string(res[0]) + ":" + what};
  }
  // ---- renumber columns into the relabelled CSR
  Tmp<int> beyond(A, 1);
  GP_CUDA_TRY(cudaMemsetAsync(beyond.p, 0, sizeof(int), st));
  renumber_kernel<RP><<<grid, 256, 0, st>>>(n, orp.p, ci_src, (const RP*)g.rp, g.order, g.newid, g.ci,
                                            g.n_active, beyond.p);
  GP_LAUNCHED();
  int h_beyond = 0;
  GP_CUDA_TRY(cudaMemcpyAsync(&h_beyond, beyond.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA_TRY(cudaStreamSynchronize(st));
  g.ci_beyond_active = h_beyond != 0;
  g.h_newid.swap(newid);
  g.h_deg.swap(deg);
  {
    uint64_t h = 1469598103934665603ull;  // FNV-1a
    auto mix = [&](uint64_t v) {
      for (int i = 0; i < 8; ++i) {
        h ^= (v >> (8 * i)) & 0xff;
        h *= 1099511628211ull;
      }
    };
    mix((uint64_t)n);
    mix((uint64_t)g.nnz);
    for (int32_t d : g.h_deg) mix((uint64_t)(uint32_t)d);
    g.digest = h;
  }
  build_schedule(g, nrp);
  g.h_rp_relabelled.swap(nrp);
}

void destroy_graph(Graph* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  serve_shutdown(*g);
  free_batch_work(*g);
  free_query_work(*g);
  free_push_work(*g);
  free_schedule(*g);
  g->alloc.put(g->rp);
  g->alloc.put(g->ci);
  g->alloc.put(g->order);
  g->alloc.put(g->newid);
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

}  // namespace

}  // namespace gp

using namespace gp;

extern "C" gp_status gp_graph_create(int64_t n, int64_t nnz, const void* row_ptr, int row_ptr_is_64,
                                     const int32_t* col_idx, const int32_t* degree, int inputs_on_device,
                                     const gp_config* cfg, gp_graph** out) {
  return guard([&] {
    GP_REQUIRE(out != nullptr, "out is NULL");
    GP_REQUIRE(n >= 1 && n <= (int64_t)INT32_MAX, "n must be in [1, 2^31-1]");
    GP_REQUIRE(nnz >= 0, "nnz must be >= 0");
    GP_REQUIRE(row_ptr && degree && (col_idx || nnz == 0), "NULL input array");
    GP_REQUIRE(row_ptr_is_64 || nnz <= (int64_t)INT32_MAX, "nnz exceeds int32 row_ptr; pass int64 row_ptr");
    std::unique_ptr<Graph, void (*)(Graph*)> g(new Graph(), destroy_graph);
    if (cfg)
      g->cfg = *cfg;
    else
      gp_config_default(&g->cfg);
    g->alloc.alloc = g->cfg.alloc;
    g->alloc.free = g->cfg.free;
    g->alloc.ctx = g->cfg.alloc_ctx;
    GP_REQUIRE((g->alloc.alloc == nullptr) == (g->alloc.free == nullptr), "alloc and free must be given together");
    if (g->cfg.k_max <= 0) g->cfg.k_max = 96;
    GP_REQUIRE(g->cfg.k_max >= 2 && g->cfg.k_max <= 1024, "k_max must be in [2, 1024]");
    if (g->cfg.stream) {
      g->stream = (cudaStream_t)g->cfg.stream;
    } else {
      GP_CUDA_TRY(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
      g->own_stream = true;
    }
    g->n = n;
    g->nnz = nnz;
    // int32 row offsets whenever they fit; int64 beyond 2^31-1 entries
    g->rp64 = nnz > (int64_t)INT32_MAX || g->cfg.row_ptr_64 != 0;
    if (g->rp64)
      ingest<int64_t>(*g, row_ptr, row_ptr_is_64, col_idx, degree, inputs_on_device);
    else
      ingest<int32_t>(*g, row_ptr, row_ptr_is_64, col_idx, degree, inputs_on_device);
    *out = reinterpret_cast<gp_graph*>(g.release());
  });
}

extern "C" gp_status gp_graph_destroy(gp_graph* gh) {
  return guard([&] { destroy_graph(reinterpret_cast<Graph*>(gh)); });
}

extern "C" gp_status gp_graph_info(const gp_graph* gh, int64_t* n, int64_t* nnz, int64_t* n_active,
                                   int64_t* max_degree) {
  return guard([&] {
    GP_REQUIRE(gh, "graph is NULL");
    const Graph* g = reinterpret_cast<const Graph*>(gh);
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (n_active) *n_active = g->n_active;
    if (max_degree) *max_degree = g->max_degree;
  });
}

extern "C" gp_status gp_graph_export(const gp_graph* gh, int64_t* row_ptr, int32_t* col_idx, int32_t* degree) {
  return guard([&] {
    GP_REQUIRE(gh && row_ptr && degree && col_idx, "NULL argument");
    Graph* g = const_cast<Graph*>(reinterpret_cast<const Graph*>(gh));
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    const int64_t n = g->n;
    row_ptr[0] = 0;
    for (int64_t u = 0; u < n; ++u) row_ptr[u + 1] = row_ptr[u] + g->h_deg[u];
    std::memcpy(degree, g->h_deg.data(), sizeof(int32_t) * n);
    Tmp<int64_t> orp(&g->alloc, n + 1);
    Tmp<int32_t> oci(&g->alloc, g->nnz);
    GP_CUDA_TRY(cudaMemcpyAsync(orp.p, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, g->stream));
    int grid = sm_count() * 8;
    if (g->rp64)
      export_kernel<int64_t><<<grid, 256, 0, g->stream>>>(n, (const int64_t*)g->rp, g->ci, orp.p, g->order,
                                                          g->newid, oci.p);
    else
      export_kernel<int32_t><<<grid, 256, 0, g->stream>>>(n, (const int32_t*)g->rp, g->ci, orp.p, g->order,
                                                          g->newid, oci.p);
    GP_LAUNCHED();
    if (g->nnz)
      GP_CUDA_TRY(cudaMemcpyAsync(col_idx, oci.p, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToHost, g->stream));
    GP_CUDA_TRY(cudaStreamSynchronize(g->stream));
  });
}
