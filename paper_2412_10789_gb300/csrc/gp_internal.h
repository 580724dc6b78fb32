// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gp.h"

namespace gp {

// ----------------------------------------------------------------- errors

struct Error {
  gp_status status;
  std::string msg;
};

void set_last_error(const std::string& msg);
// Run f, turning gp::Error and other exceptions into a status and gp_last_error().
gp_status guard(const std::function<void()>& f);

#define GP_CUDA_TRY(expr)                                                              \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess)                                                             \
      throw ::gp::Error{GP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)}; \
  } while (0)

#define GP_REQUIRE(cond, msg)                                    \
  do {                                                           \
    if (!(cond)) throw ::gp::Error{GP_EINVAL, std::string(msg)}; \
  } while (0)

// A named NVTX range for the lifetime of the object (the calls of the C ABI and
// the service's iterations), so that Nsight timelines group their kernels.
struct TraceRange {
  explicit TraceRange(const char* name);
  ~TraceRange();
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// After a <<<>>> launch: count it and surface launch-configuration errors.
#define GP_LAUNCHED()                           \
  do {                                          \
    ::gp::count_launch();                       \
    GP_CUDA_TRY(cudaGetLastError());            \
  } while (0)

// ----------------------------------------------------------------- coefficients (coeff.cpp)

// Chebyshev coefficients c_0..c_kmax of f (Lemma 2 closed form for SSPPR, Lemma 3
// scaled Bessel values by backward recurrence for HKPR) and tails
// tail[k] = sum_{l>k} |c_l| (the sum continues past kmax until negligible).
void cheb_coefficients(int function, double param, int kmax, std::vector<double>& c,
                       std::vector<double>& tail);
// The same c_0..c_kmax written into c[kmax + 1] without allocating: the HKPR
// recurrence uses `work` (cheb_coefficients_work(...) doubles at least;
// returns false when work_len is smaller).
int cheb_coefficients_work(int function, double param, int kmax);
bool cheb_coefficients_into(int function, double param, int kmax, double* c, double* work, int work_len);
// Taylor coefficients zeta_0..zeta_{N-1} (Def. SSPPR / Def. HKPR) with
// N = smallest count whose tail sum_{k>=N} zeta_k <= tol (capped at nmax).
void taylor_coefficients(int function, double param, double tol, int nmax, std::vector<double>& z);
// K of the paper's experimental rule (Section 6): ceil(alpha^-1/2 ln(1/tol)) or
// ceil(sqrt(t) ln(1/tol)), at least 1.
int paper_k(int function, double param, double tol);
// Smallest k with tail[k] * cmin <= tol (cmin = 1 is the least possible
// max ||r_l||_1), used to size the launch sequence.
int k_lower(const std::vector<double>& tail, double tol, double cmin);
// The l1 stop rule (Theorem 1 with Assumption 1's C estimated on the fly):
// stop at the smallest k with tail(k) * kCMargin * max_{l<=k} ||r_l||_1 <= tol.
// ||r_k||_1 can still grow after k (on power-law graphs the running maximum
// alone let the truncation pass tol by a few percent); the first omitted term
// obeys ||r_{k+1}||_1 <= 2 ||P r_k||_1 + ||r_{k-1}||_1 <= 3 max_{l<=k} ||r_l||_1,
// P being column-stochastic, and the margin read here is 2.
constexpr double kCMargin = 2.0;

// ----------------------------------------------------------------- device memory

struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free)(void*, void*) = nullptr;
  void* ctx = nullptr;
  void* get(size_t bytes);
  void put(void* p);
};

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t count = 0;
};

// ----------------------------------------------------------------- schedule

// Work decomposition of one fused pass over the relabelled (degree-descending)
// rows, built once per graph (schedule.cpp).  The unit is a tile of at most
// kTileCap consecutive entries, described by int4 {row0, e0 low, e0 high, meta}:
//   rows tile  (meta bit 0 = 0): nrows = meta[1..8] consecutive rows that all
//              have degree d = meta[9..18], so entry e belongs to row
//              row0 + (e - e0) / d;
//   chunk tile (meta bit 0 = 1): len = meta[1..10] entries of the long row row0,
//              chunk index p = meta[11..31]; the chunk's partial sum goes to
//              slot poff[row0] + p, and a second kernel adds a row's partials
//              in chunk order.
// Warps claim tiles from a per-pass counter (all tiles move about the same
// number of entries), double-buffering their indices with cp.async (step.cuh).
#ifndef GP_STEP_THREADS
#define GP_STEP_THREADS 768
#endif
#ifndef GP_TILE_VEC
#define GP_TILE_VEC 4
#endif
#ifndef GP_GATHER_N
#define GP_GATHER_N 8
#endif
#ifndef GP_HUB_CACHE
#define GP_HUB_CACHE 1
#endif
constexpr int kStepThreads = GP_STEP_THREADS;  // one persistent CTA per SM
constexpr int kStepWarps = kStepThreads / 32;
constexpr int kTileSpan = 32 * 4 * GP_TILE_VEC;  // entries one tile buffer holds (16-byte vectors)
constexpr int kTileCap = kTileSpan - 4;          // entries of a tile (room for 16-byte alignment)
constexpr int kTileRows = 128;                   // rows of a rows tile
constexpr int kWarpSmemInts = 2 * kTileSpan;     // double-buffered tile indices per warp

struct Schedule {
  int4* tiles = nullptr;   // device
  int64_t ntiles = 0;
  int nlong = 0;           // long rows are relabelled rows 0..nlong-1
  int* poff = nullptr;     // device, nlong+1: first chunk slot of each long row
  float2* part = nullptr;  // device, per-chunk partial sums (hi, lo)
  int hub = 0;             // rows 0..hub-1 of Q_k are cached in shared memory
  int smem_bytes = 0;      // dynamic shared memory of the step kernel
  int t_long = 0;          // rows of this degree or more are chunked
};

// ----------------------------------------------------------------- graph

// ChebyPush / Algorithm 5 work vectors (push.cu), allocated at a graph's first
// push query and kept until the graph is destroyed, so a query allocates
// nothing.
struct PushWork {
  double* ra = nullptr;  // r_cur / r_new pair, n each
  double* rb = nullptr;
  double* y = nullptr;   // n
  int2* fr = nullptr;    // frontier items {row, chunk}
  double* fval = nullptr;
  int* counts = nullptr;                  // frontier items per iteration (1025)
  unsigned long long* walks = nullptr;    // walks taken (Algorithm 5)
  void* stage = nullptr;                  // host-output staging, n doubles (on demand)
};

struct QueryWork {
  float* qa = nullptr;      // Q = D^-1 r, one buffer of the ping-pong pair
  float* qb = nullptr;      // the other
  float2* y = nullptr;      // y as an unevaluated float pair (hi + lo), relabelled order
  float* norms = nullptr;   // ||r_k||_1 per k
  int* state = nullptr;     // [0] = K at which the stop rule fired, [1 + k] = work counter of pass k
  void* stage = nullptr;    // device staging for host outputs (n doubles)
  int kcap = 0;             // length of norms - 2
};

struct Graph {
  int64_t n = 0, nnz = 0, n_active = 0, max_degree = 0;
  uint64_t digest = 0;        // FNV-1a of n, nnz and the degree sequence (autotune cache key)
  bool rp64 = false;          // row_ptr stored as int64
  bool ci_beyond_active = false;  // some col_idx entry names an isolated node (asymmetric input)
  void* rp = nullptr;         // relabelled row_ptr (int32 or int64), device
  int32_t* ci = nullptr;      // relabelled col_idx, device
  int32_t* order = nullptr;   // order[i] = caller id of relabelled row i, device
  int32_t* newid = nullptr;   // newid[u] = relabelled id of caller node u, device
  std::vector<int32_t> h_newid;  // host copy of newid
  std::vector<int32_t> h_deg;    // host copy of the (caller-order) degrees
  std::vector<int64_t> h_rp_relabelled;  // host copy of the relabelled row offsets
  Schedule sched;
  gp_config cfg{};
  Allocator alloc;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::recursive_mutex mu;
  QueryWork qw;
  PushWork pw;
  // kernel timing (gp_profile_*)
  bool profiling = false;
  double prof_ms = 0.0;
  int64_t prof_launches = 0;
  double prof_bytes = 0.0;
  std::vector<cudaEvent_t> ev_pool;
  void* serve = nullptr;      // serving state (serve.cu)
  void* batch = nullptr;      // batched workspace (batch.cu)
};

// schedule.cpp: build the task list from the relabelled row offsets and upload it.
void build_schedule(Graph& g, const std::vector<int64_t>& rp_host_relabelled);
void free_schedule(Graph& g);
// Bytes one fused step must move for one column (algorithmic traffic).
double step_bytes_single(const Graph& g);

// precise.cu: the float-pair storage path for graphs of at most
// cfg.precise_rows active rows; returns K and max_l ||r_l||_1.
bool use_precise(const Graph& g);
int run_precise(Graph& g, int64_t s, bool cheb, const std::vector<double>& c, const std::vector<double>& tail,
                int k_fixed, double tol, int kcap, double* C_out);

// cheb.cu
void run_query(Graph& g, const gp_request& req, gp_query_info* info);
void run_power(Graph& g, const gp_request& req, gp_query_info* info);
void free_query_work(Graph& g);

// batch.cu / serve.cu
void run_batch(Graph& g, int count, const gp_request* reqs, gp_query_info* infos);
void run_clenshaw(Graph& g, int count, const gp_request* reqs, gp_query_info* infos);
void run_propagate(Graph& g, int function, double param, double a, int F, const float* X, float* Z, int on_device,
                   double tol, gp_query_info* infos);
void free_push_work(Graph& g);
// push.cu: ChebyPush (Algorithm 4) for one source.
void run_chebypush(Graph& g, int function, int32_t source, double param, double eps_a, int K, gp_dtype out_dtype,
                   void* y_out, int y_on_device, gp_query_info* info);
// push.cu: Algorithm 5 (ChebyPush + alpha-random walks) for SSPPR.
void run_bidirectional(Graph& g, int32_t source, double alpha, double eps_r, double delta, int K, uint64_t seed,
                       gp_dtype out_dtype, void* y_out, int y_on_device, gp_query_info* info);
// Block width with the least device time per column and pass on this graph
// (cached per graph digest, storage and device unless widths are given).
// The batched form's tuned block: width B, chunk threshold t_long (rows with
// more entries are chunk tiles) and the device time per column and pass.
struct TunedBlock {
  int B;
  int t_long;
  double us;
};
TunedBlock tune_block(Graph& g, gp_dtype storage, std::vector<int> widths);
void free_batch_work(Graph& g);
uint64_t serve_submit(Graph& g, const gp_request& req);
gp_status serve_poll(Graph& g, uint64_t ticket, gp_query_info* info);
gp_status serve_wait(Graph& g, uint64_t ticket, double timeout_ms, gp_query_info* info);
void serve_stats(Graph& g, uint64_t* completed, uint64_t* steps, double* mean_active);
void serve_shutdown(Graph& g);

// ----------------------------------------------------------------- float pairs
#if defined(__CUDACC__)

// Unevaluated sums hi + lo of two floats ("double-float"), built from the
// error-free transformations of Knuth (TwoSum) and Dekker/FMA (TwoProduct).
// The __f*_rn intrinsics keep the compiler from fusing or reordering them.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ DF df_norm(DF x) { return df_fast_two_sum(x.hi, x.lo) ; }
__device__ __forceinline__ DF df_add(DF x, DF y) {
  DF s = df_two_sum(x.hi, y.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return df_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ DF df_mul_f(DF x, float f) {
  float p = __fmul_rn(x.hi, f);
  float e = __fmaf_rn(x.hi, f, -p);
  e = __fmaf_rn(x.lo, f, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
// Kahan-compensated accumulator: sum = s + c.
struct KSum {
  float s, c;
};
__device__ __forceinline__ void ksum_add(KSum& k, float v) {
  float y = __fsub_rn(v, k.c);
  float t = __fadd_rn(k.s, y);
  k.c = __fsub_rn(__fsub_rn(t, k.s), y);
  k.s = t;
}
// Merge two compensated sums into one float pair (hi, lo), value s1 - c1 + s2 - c2.
__device__ __forceinline__ DF ksum_merge(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ DF ksum_value(const KSum& k) { return df_two_sum(k.s, -k.c); }
// Cascaded summation with TwoSum (Ogita, Rump and Oishi's Sum2): the error of
// every addition is captured exactly whatever the signs and magnitudes, so the
// pair (s, c) carries about twice the working precision.
struct S2Sum {
  float s, c;
};
__device__ __forceinline__ void s2sum_add(S2Sum& k, float v) {
  const DF t = df_two_sum(k.s, v);
  k.s = t.hi;
  k.c = __fadd_rn(k.c, t.lo);
}
__device__ __forceinline__ DF s2sum_value(const S2Sum& k) { return df_fast_two_sum(k.s, k.c); }
#endif  // __CUDACC__

}  // namespace gp
