// gp_query_static: a ChebyPower query that allocates nothing.
//
// Some callers cannot allocate device memory when they issue a query: a host
// framework that owns every byte of the GPU and hands out fixed buffers, a
// latency-critical loop that cannot afford cudaFree's device-wide
// synchronisation or a cudaMalloc that may fail under memory pressure, or
// code that must not touch the allocator at all.  For them this entry point
// runs the fused Chebyshev step on the caller's CSR (natural row order, no
// relabelling, no gp_graph) with all of its scratch -- the two Q vectors of
// the recurrence and the float-pair y accumulator -- in one file-scope
// __device__ array of kStaticBytes, which every GPU that loads the library
// holds until the process exits.  The caller still provides the inputs (CSR
// on the device) and the output (y on the device).
//
// Limits and sharing: n <= kStaticMaxN (1,048,576 nodes, 16 MiB of scratch),
// 1 <= K <= kStaticMaxK.  Every call on a device uses the same array and
// leaves its contents behind; each call clears what must start at zero.  Calls
// whose work overlaps on the GPU (different streams, or different host threads)
// race on the array and corrupt each other's results.  The first call on a
// device looks up the array's device address (cudaGetSymbolAddress, with that
// device current) and keeps it for the life of the process; that first call
// should come before any stream capture, and the entry point must not be used
// on a device after cudaDeviceReset (the kept address would be stale).  Every
// later call only enqueues kernels: the source's degree is read on the device,
// so no call waits for the GPU.
//
// The CSR is the caller's and is not checked here: sorted rows without
// duplicates or self-loops, both directions of every edge (Section 2.1), the
// conditions gp_graph_create validates.  A row may list a node whose own row
// is empty; that node contributes nothing (1/d := 0, the reading of P's
// degree-0 columns the rest of the library uses).
#include <cmath>
#include <cstring>
#include <mutex>

#include "gp_internal.h"

constexpr int64_t kStaticMaxN = int64_t(1) << 20;
constexpr int kStaticMaxK = 256;
constexpr int kStaticMaxDevices = 64;
constexpr double kStaticMaxT = 1000.0;
// Work array of the HKPR coefficient recurrence for t <= kStaticMaxT, K <= kStaticMaxK.
constexpr int kStaticCoeffWork = 4096;
// Q_a, Q_b (n floats each) and y (n float pairs): 16 MiB.
constexpr size_t kStaticBytes = (size_t)kStaticMaxN * (4 + 4 + 8);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace gp {
namespace {

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
void* static_scratch(int dev) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    GP_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[dev] = p;
  }
  return g_static_addr[dev];
}

__global__ void static_zero_kernel(int64_t n, float* qa, float* qb, float2* y) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    qa[u] = 0.f;
    qb[u] = 0.f;
    y[u] = make_float2(0.f, 0.f);
  }
}

__host__ __device__ inline float2 static_split(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// r_0 = e_s (Q_0(s) = 1/d_s), r_1 = P e_s (Q_1(v) = 1/(d_s d_v) for v in N(s)),
// y = c_0 r_0 + c_1 r_1.  An isolated source writes nothing (the output kernel
// answers f(0) e_s); a listed neighbour with an empty row keeps r_1(v) = 0.
__global__ void static_init_kernel(const int32_t* rp, const int32_t* ci, int64_t s, double c0, double c1,
                                   float* q0, float* q1, float2* y) {
  const int64_t beg = rp[s], end = rp[s + 1];
  if (beg == end) return;
  const double ds = (double)(end - beg);
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid == 0) {
    q0[s] = (float)(1.0 / ds);
    y[s] = static_split(c0);
  }
  for (int64_t e = beg + tid; e < end; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = ci[e];
    const int32_t dv = rp[v + 1] - rp[v];
    if (dv == 0) continue;
    q1[v] = (float)(1.0 / (ds * (double)dv));
    y[v] = static_split(c1 / ds);
  }
}

// The fused step over the caller's CSR, a warp per row:
// acc = sum_{v in N(u)} Q_k(v) (Kahan per lane, float-pair shuffle tree),
// r = 2 acc - d_u Q_{k-1}(u), Q_{k+1}(u) = r / d_u over Q_{k-1}(u), y += c r.
__global__ void static_step_kernel(int64_t n, const int32_t* rp, const int32_t* ci, const float* qcur, float* qprev,
                                   float2* y, float c_hi, float c_lo) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nwarps) {
    const int64_t beg = rp[u], end = rp[u + 1];
    if (beg == end) continue;
    KSum s{0.f, 0.f};
    for (int64_t e = beg + lane; e < end; e += 32) ksum_add(s, qcur[ci[e]]);
    DF acc = ksum_value(s);
    for (int off = 16; off > 0; off >>= 1) {
      const DF o{__shfl_xor_sync(0xffffffffu, acc.hi, off), __shfl_xor_sync(0xffffffffu, acc.lo, off)};
      acc = df_add(acc, o);
    }
    if (lane == 0) {
      const float d = (float)(end - beg);
      const float qp = qprev[u];
      const float p = __fmul_rn(d, qp), pe = __fmaf_rn(d, qp, -p);
      const DF r = df_add(DF{__fmul_rn(2.0f, acc.hi), __fmul_rn(2.0f, acc.lo)}, DF{-p, -pe});
      const float rv = __fadd_rn(r.hi, r.lo);
      qprev[u] = __fdiv_rn(rv, d);
      const float2 yv = y[u];
      const DF yy = df_add(DF{yv.x, yv.y}, df_mul(r, DF{c_hi, c_lo}));
      y[u] = make_float2(yy.hi, yy.lo);
    }
  }
}

// y_out = y as doubles; for an isolated source (read from row_ptr here) f(0) e_s.
__global__ void static_out_kernel(int64_t n, const int32_t* rp, const float2* y, int64_t s, double f0,
                                  double* out) {
  const bool isolated = rp[s] == rp[s + 1];
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    out[u] = isolated ? (u == s ? f0 : 0.0) : (double)y[u].x + (double)y[u].y;
}

}  // namespace
}  // namespace gp

using namespace gp;

extern "C" gp_status gp_query_static(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                                     int32_t function, int32_t source, double param, int32_t K, double* y_out,
                                     void* stream) {
  return guard([&] {
    GP_REQUIRE(n >= 1, "n must be >= 1");
    if (n > kStaticMaxN)
      throw Error{GP_EINVAL, "gp_query_static: n = " + std::to_string(n) + " exceeds the static scratch limit of " +
                                 std::to_string(kStaticMaxN) + " nodes; use gp_graph_create / gp_query"};
    GP_REQUIRE(nnz >= 0 && nnz <= (int64_t)INT32_MAX, "nnz must be in [0, 2^31-1]");
    GP_REQUIRE(row_ptr && y_out && (col_idx || nnz == 0), "NULL device pointer");
    GP_REQUIRE(function == GP_FN_PPR || function == GP_FN_HKPR, "function must be GP_FN_PPR or GP_FN_HKPR");
    GP_REQUIRE(source >= 0 && (int64_t)source < n, "source out of range");
    if (function == GP_FN_PPR)
      GP_REQUIRE(param > 0.0 && param < 1.0, "alpha must be in (0, 1)");
    else
      GP_REQUIRE(param > 0.0 && param <= kStaticMaxT, "t must be in (0, 1000]");
    GP_REQUIRE(K >= 1 && K <= kStaticMaxK, "K must be in [1, 256]");
    int dev = 0;
    GP_CUDA_TRY(cudaGetDevice(&dev));
    GP_REQUIRE(dev >= 0 && dev < kStaticMaxDevices, "device index out of range");
    unsigned char* base = (unsigned char*)static_scratch(dev);
    float* qa = (float*)base;
    float* qb = qa + kStaticMaxN;
    float2* y = (float2*)(qb + kStaticMaxN);
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 0;
    GP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // c_0..c_K (Lemma 2 / Lemma 3) from the library's coefficient engine, in
    // fixed arrays on the host stack
    double c[kStaticMaxK + 2];
    double work[kStaticCoeffWork];
    if (!cheb_coefficients_into(function, param, K + 1, c, work, kStaticCoeffWork))
      throw Error{GP_EINVAL, "gp_query_static: t too large for the fixed coefficient work array"};
    const double f0 = function == GP_FN_PPR ? param : std::exp(-param);
    static_zero_kernel<<<sms * 4, 256, 0, st>>>(n, qa, qb, y);
    GP_LAUNCHED();
    // the source row has at most n - 1 entries; blocks past its end return at once
    const int init_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 4));
    static_init_kernel<<<init_blocks, 256, 0, st>>>(row_ptr, col_idx, source, c[0], c[1], qa, qb, y);
    GP_LAUNCHED();
    float* bufs[2] = {qa, qb};  // bufs[k & 1] holds Q_k
    for (int k = 1; k < K; ++k) {
      const float2 ck = static_split(c[k + 1]);
      static_step_kernel<<<sms * 8, 256, 0, st>>>(n, row_ptr, col_idx, bufs[k & 1], bufs[(k + 1) & 1], y, ck.x,
                                                  ck.y);
      GP_LAUNCHED();
    }
    static_out_kernel<<<sms * 4, 256, 0, st>>>(n, row_ptr, y, source, f0, y_out);
    GP_LAUNCHED();
  });
}
