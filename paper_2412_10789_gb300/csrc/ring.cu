// Device-resident request loop of the continuous-batching service.
//
// The service's requests and results travel through two rings in pinned,
// mapped host memory that the GPU reads and writes directly:
//   request ring  (host -> device): one RingReq per request, published by
//                 the service thread with a release store of ctl.tail;
//   done ring     (device -> host): one RingDone per finished query, made
//                 visible by a release store of ctl.done after the output
//                 kernel has written the query's y.
// Every iteration is the same fixed sequence of kernels, launched without any
// wait for the device in between:
//   admit    (one block)  takes requests off the request ring into the free
//                          columns of the FP32 block: coefficients, state,
//                          source and output pointer of each new column;
//   reset + init          zero the new columns, r_0 = e_s, r_1 = P e_s;
//   width    (one block)  per block, the pass width from its busiest slot;
//   control + SpMM        the fused pass of each block (Algorithm 3's step
//                          with the per-column stop rule of Theorem 1);
//   retire   (one block)  per block, the columns whose stop rule fired;
//   output                their y into the caller's (or a staging) buffer;
//   complete (one block)  their RingDone records, then frees their columns;
//   migrate               (16-bit storage) columns past their own warm-up
//                          move from the FP32 block to the 16-bit block.
// So admission into free slots, packing as columns of one SpMM, per-column
// retirement and the refill of freed slots are all decided on the device.
// The host thread only publishes requests, launches iterations (at most two
// queued ahead of the GPU) and turns done records into completed tickets.
#include <cuda/atomic>

#include <algorithm>
#include <cstring>

#include "ring.h"

namespace gp {

namespace {

__device__ __forceinline__ uint64_t load_acquire_sys(const uint64_t* p) {
  return cuda::atomic_ref<uint64_t, cuda::thread_scope_system>(*const_cast<uint64_t*>(p))
      .load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void store_release_sys(uint64_t* p, uint64_t v) {
  cuda::atomic_ref<uint64_t, cuda::thread_scope_system>(*p).store(v, cuda::memory_order_release);
}

constexpr int kRingThreads = 256;  // one thread per column slot (blocks of at most 256 columns)

// Exclusive prefix sum of flag over the block; returns the rank, total in *tot.
__device__ __forceinline__ int block_rank(int flag, int* s_scan, int* tot) {
  const int t = threadIdx.x;
  s_scan[t] = flag;
  __syncthreads();
  for (int off = 1; off < kRingThreads; off <<= 1) {
    const int v = t >= off ? s_scan[t - off] : 0;
    __syncthreads();
    s_scan[t] += v;
    __syncthreads();
  }
  const int incl = s_scan[t];
  *tot = s_scan[kRingThreads - 1];
  __syncthreads();
  return incl - flag;
}

// Requests off the ring into free columns of the FP32 block (lowest free
// slots first).  New columns: r_0 = e_s, r_1 = P e_s (set by the init
// kernel), k = 1, ||r_0||_1 = ||r_1||_1 = 1.
__global__ void __launch_bounds__(kRingThreads) ring_admit_kernel(RingCtl* ctl, const RingReq* ring, int cap,
                                                                  RingDev* dev, SlotDev* slots, ColState* col,
                                                                  ColParam* par, ColStat* stat, float* norm, int B,
                                                                  int* new_list) {
  __shared__ int s_scan[kRingThreads];
  __shared__ int s_take;
  __shared__ uint64_t s_head;
  const int j = threadIdx.x;
  const int free_slot = j < B && !slots[j].busy;
  int nfree = 0;
  const int rank = block_rank(free_slot, s_scan, &nfree);
  if (j == 0) {
    const uint64_t tail = load_acquire_sys(&ctl->tail);
    const uint64_t head = dev->head;
    s_head = head;
    s_take = (int)std::min<uint64_t>(tail - head, (uint64_t)nfree);
  }
  __syncthreads();
  const int take = s_take;
  if (free_slot && rank < take) {
    (void)load_acquire_sys(&ctl->tail);  // this thread's reads of the entry follow the host's publication
    const RingReq& r = ring[(s_head + rank) % cap];
    SlotDev sd;
    sd.ticket = r.ticket;
    sd.out = r.out;
    sd.src = r.src;
    sd.busy = 1;
    sd.out_f64 = r.out_f64;
    sd.warm = r.param.warm;
    sd.k16 = -1;
    sd.k_low = r.k_low;
    sd.pad = 0;
    slots[j] = sd;
    col[j] = ColState{1, 0.f};
    stat[j] = ColStat{1, 0, 0, 1.0f};
    norm[j] = 0.f;
    new_list[rank] = j;
  }
  __syncthreads();
  // the coefficient tables, one column at a time by the whole block
  constexpr int kWords = (int)(sizeof(ColParam) / sizeof(float));
  for (int t = 0; t < take; ++t) {
    const float* from = reinterpret_cast<const float*>(&ring[(s_head + t) % cap].param);
    float* to = reinterpret_cast<float*>(par + new_list[t]);
    for (int i = j; i < kWords; i += kRingThreads) to[i] = from[i];
  }
  if (j == 0) {
    dev->new_count = take;
    dev->head = s_head + take;
    dev->active32 += take;
    store_release_sys(&ctl->head, s_head + take);
  }
}

// Calls f(r, t) for every row r < na and item t < nc (a column being reset,
// moved or migrated).  With more than 16 items a warp takes one row at a time,
// its lanes over the items; with fewer, P >= nc lanes take a row and a warp
// covers 32 / P rows at a time, so that more rows' accesses are in flight.
template <typename F>
__device__ __forceinline__ void for_rows_items(int64_t na, int nc, F f) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (nc <= 16) {
    int P = 1;
    while (P < nc) P <<= 1;
    const int rows = 32 / P, t = lane & (P - 1);
    if (t >= nc) return;
    for (int64_t r = w0 * rows + lane / P; r < na; r += nw * rows) f(r, t);
    return;
  }
  for (int64_t r = w0; r < na; r += nw)
    for (int t = lane; t < nc; t += 32) f(r, t);
}

// Zero the new columns of Q_a, Q_b and y over all rows.
__global__ void ring_reset_kernel(int64_t na, int B, const int* new_list, const RingDev* dev, float* fa, float* fb,
                                  float* y) {
  const int nc = dev->new_count;
  if (nc == 0) return;
  for_rows_items(na, nc, [&](int64_t r, int t) {
    const int64_t i = r * B + new_list[t];
    fa[i] = 0.f;
    fb[i] = 0.f;
    y[i] = 0.f;
  });
}

// r_0 = e_s (Q_0 = e_s / d_s), r_1 = P e_s (Q_1(v) = 1 / (d_s d_v) for v in
// N(s) with d_v > 0), y = c_0 r_0 + c_1 r_1, for the new column of this block.
template <typename RP>
__global__ void ring_init_kernel(const void* rpv, const int32_t* ci, int64_t na, int B, const int* new_list,
                                 const RingDev* dev, const SlotDev* slots, const ColParam* par, float* q0, float* q1,
                                 float* y) {
  if ((int)blockIdx.x >= dev->new_count) return;
  const RP* rp = (const RP*)rpv;
  const int j = new_list[blockIdx.x];
  const int64_t s = slots[j].src;
  const int64_t beg = rp[s], end = rp[s + 1];
  const float ds = (float)(end - beg);
  const float c0 = par[j].c[0], c1 = par[j].c[1];
  if (threadIdx.x == 0) {
    q0[s * B + j] = 1.0f / ds;
    y[s * B + j] = c0;
  }
  for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const int32_t v = ci[e];
    if (v >= na) continue;  // only an unvalidated asymmetric CSR lists an isolated row
    const float dv = (float)(rp[v + 1] - rp[v]);
    q1[(int64_t)v * B + j] = (float)(1.0 / ((double)ds * (double)dv));
    y[(int64_t)v * B + j] = c1 / ds;
  }
}

// The pass width of a block: the smallest power of two (at least min_w, at
// most B) that holds its highest busy slot.
__global__ void __launch_bounds__(kRingThreads) ring_width_kernel(const SlotDev* slots, int B, int min_w,
                                                                  int* width) {
  __shared__ int s_max;
  if (threadIdx.x == 0) s_max = -1;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < B && slots[j].busy) atomicMax(&s_max, j);
  __syncthreads();
  if (j == 0) {
    int w = min_w;
    while (w < s_max + 1) w <<= 1;
    *width = std::min(w, B);
  }
}

// Columns of a block whose stop rule fired, as many as the done ring has room
// for (the rest stay until the host has read more records).
__global__ void __launch_bounds__(kRingThreads) ring_retire_kernel(const RingCtl* ctl, const RingDev* dev, int cap,
                                                                   const SlotDev* slots, const ColStat* stat, int B,
                                                                   int* ret_list, int* ret_count) {
  __shared__ int s_scan[kRingThreads];
  const int j = threadIdx.x;
  const int fin = j < B && slots[j].busy && stat[j].done;
  int nfin = 0;
  const int rank = block_rank(fin, s_scan, &nfin);
  const uint64_t used = dev->done - load_acquire_sys(&ctl->consumed);
  const int room = used >= (uint64_t)cap ? 0 : (int)std::min<uint64_t>((uint64_t)cap - used, (uint64_t)nfin);
  if (fin && rank < room) ret_list[rank] = j;
  if (j == 0) *ret_count = room;
}

// y of the retired columns (relabelled rows) into their outputs in the
// caller's numbering, for the columns whose output type is OUT: a thread per
// caller row u reads its relabelled row's values of those columns (the same
// row, so the columns share cached sectors) and writes them coalesced across
// the warp; rows of isolated nodes get 0.
template <typename OUT>
__global__ void ring_output_kernel(int64_t n, int64_t na, const int32_t* newid, const float* y, int B,
                                   const int* ret_list, const int* ret_count, const SlotDev* slots) {
  const int nc = *ret_count;
  if (nc == 0) return;
  __shared__ int s_col[kRingThreads];
  __shared__ OUT* s_out[kRingThreads];
  __shared__ int s_m;
  constexpr int kF64 = sizeof(OUT) == 8;
  if (threadIdx.x == 0) s_m = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    const int j = ret_list[t];
    if (slots[j].out_f64 == kF64) {
      const int at = atomicAdd(&s_m, 1);
      s_col[at] = j;
      s_out[at] = static_cast<OUT*>(slots[j].out);
    }
  }
  __syncthreads();
  const int m = s_m;
  if (m == 0) return;  // no retired column wants this output type
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = newid[u];
    if (i >= na) {
      for (int t = 0; t < m; ++t) s_out[t][u] = (OUT)0;
    } else {
      const float* row = y + i * B;
      for (int t = 0; t < m; ++t) s_out[t][u] = (OUT)__ldg(row + s_col[t]);
    }
  }
}

// Done records of the retired columns (after their outputs), then their
// columns are freed for the next admission.
__global__ void __launch_bounds__(kRingThreads) ring_complete_kernel(RingCtl* ctl, RingDone* done_ring, int cap,
                                                                     RingDev* dev, SlotDev* slots, ColState* col,
                                                                     ColStat* stat, float* norm, const int* ret_list,
                                                                     const int* ret_count, int block16) {
  const int nc = *ret_count;
  if (nc == 0) return;
  const uint64_t base = dev->done;
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    const int j = ret_list[t];
    const ColStat st = stat[j];
    RingDone d;
    d.ticket = slots[j].ticket;
    d.K = st.done ? st.K : st.k;
    d.k16_from = slots[j].k16 >= 0 ? slots[j].k16 : d.K + 1;
    d.C = st.C;
    d.pad = 0;
    done_ring[(base + t) % cap] = d;
    slots[j].busy = 0;
    col[j] = ColState{0, 0.f};
    stat[j] = ColStat{0, 0, 0, 0.f};
    norm[j] = 0.f;
  }
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) {
    dev->done = base + nc;
    if (block16)
      dev->active16 -= nc;
    else
      dev->active32 -= nc;
    store_release_sys(&ctl->done, base + nc);
  }
}

// FP32 columns past their own warm-up (newest term Q_j with j >= warm + 3, so
// every 16-bit term has index >= warm + 2) paired with free 16-bit slots; the
// slot records move with them.  A column moves only while at least
// kMinSteps16 steps are certain to remain (k_low - k), only while the FP32
// block is busy (its busy columns and the requests waiting in the ring fill
// more than half of its slots), and only when the 16-bit block would then hold
// at least kMinCols16 columns (a quarter of its slots at most).  A move frees
// an FP32 slot for the next request and the column's later steps run in 16
// bits.  But every iteration with a column in each block runs two passes, and
// a 16-bit pass over a few columns costs nearly as much as one over many (its
// time is set by the latency of gathering every col_idx entry: at 16 columns
// it costs more per column than a full FP32 pass), so under light load, or
// with too few columns past their warm-up, columns stay in FP32 and each
// iteration stays one pass long.
#ifndef GP_MIN_STEPS16
#define GP_MIN_STEPS16 1
#endif
#ifndef GP_MIN_COLS16
#define GP_MIN_COLS16 64
#endif
constexpr int kMinSteps16 = GP_MIN_STEPS16;
constexpr int kMinCols16 = GP_MIN_COLS16;
__global__ void __launch_bounds__(kRingThreads) ring_migrate_select_kernel(const RingCtl* ctl, RingDev* dev,
                                                                           SlotDev* s32, const ColStat* st32, int B32,
                                                                           SlotDev* s16, int B16, int* from, int* to) {
  __shared__ int s_scan[kRingThreads];
  __shared__ int s_from[kRingThreads];
  __shared__ int s_to[kRingThreads];
  __shared__ int s_busy;
  const int j = threadIdx.x;
  if (j == 0) {
    const uint64_t waiting = load_acquire_sys(&ctl->tail) - dev->head;
    s_busy = 2 * (waiting + (uint64_t)dev->active32) > (uint64_t)B32;
  }
  __syncthreads();
  // after the pass and its control, an active column's newest term is Q_{k-1}
  const int cand = s_busy && j < B32 && s32[j].busy && !st32[j].done && st32[j].k - 1 >= s32[j].warm + 3 &&
                   s32[j].k_low - (st32[j].k - 1) >= kMinSteps16;
  int ncand = 0;
  const int rc = block_rank(cand, s_scan, &ncand);
  if (cand) s_from[rc] = j;
  const int need = kMinCols16 < B16 / 4 ? kMinCols16 : B16 / 4;
  const int go = ncand > 0 && need > 0 && ncand + dev->active16 >= need;
  const int fr = go && j < B16 && !s16[j].busy;
  int nfree = 0;
  const int rf = block_rank(fr, s_scan, &nfree);
  if (fr) s_to[rf] = j;
  __syncthreads();
  const int take = std::min(ncand, nfree);
  if (j < take) {
    const int a = s_from[j], b = s_to[j];
    SlotDev sd = s32[a];
    sd.k16 = st32[a].k - 2;  // Q_{k-1} and Q_{k-2} are rounded: the first 16-bit term is Q_{k-2}
    s16[b] = sd;
    s32[a].busy = 0;
    from[j] = a;
    to[j] = b;
  }
  if (j == 0) {
    dev->mig_count = take;
    dev->active32 -= take;
    dev->active16 += take;
  }
}

template <typename H>
__device__ __forceinline__ H ring_to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 ring_to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half ring_to16<__half>(float x) { return __float2half_rn(x * 4096.0f); }

// Q_k, Q_{k-1} (rounded as the 16-bit passes store them: BF16 round to nearest,
// FP16 of Q * 2^12) and y of the selected columns, rows spread over the warps
// by for_rows_items.
template <typename H>
__global__ void ring_migrate_columns_kernel(int64_t na, int ldb_s, int ldb_d, const int* from, const int* to,
                                            const RingDev* dev, const float* fk, const float* fk1, const float* ys,
                                            H* hk, H* hk1, float* yd) {
  const int nc = dev->mig_count;
  if (nc == 0) return;
  for_rows_items(na, nc, [&](int64_t r, int t) {
    const int64_t a = r * ldb_s + from[t], b = r * ldb_d + to[t];
    hk[b] = ring_to16<H>(fk[a]);
    hk1[b] = ring_to16<H>(fk1[a]);
    yd[b] = ys[a];
  });
}

// The moved columns' coefficients, state and last norm (a block per column);
// the FP32 column is cleared.
__global__ void ring_migrate_state_kernel(const int* from, const int* to, const int* count, ColState* cs_s,
                                          const ColParam* cp_s, ColStat* st_s, float* nm_s, ColState* cs_d,
                                          ColParam* cp_d, ColStat* st_d, float* nm_d) {
  if ((int)blockIdx.x >= *count) return;
  const int a = from[blockIdx.x], b = to[blockIdx.x];
  const float* src = reinterpret_cast<const float*>(cp_s + a);
  float* dst = reinterpret_cast<float*>(cp_d + b);
  for (int i = threadIdx.x; i < (int)(sizeof(ColParam) / sizeof(float)); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    cs_d[b] = cs_s[a];
    st_d[b] = st_s[a];
    nm_d[b] = nm_s[a];
    cs_s[a] = ColState{0, 0.f};
    st_s[a] = ColStat{0, 0, 0, 0.f};
    nm_s[a] = 0.f;
  }
}

// Pack a block's busy columns below the smallest power of two (at least
// min_w) that holds them all, so that the passes of a lightly loaded block
// narrow again (the width follows the highest busy slot): the FP32 block once
// no request waits in the ring (admission refills its free slots first), the
// 16-bit block in every iteration (only moves from the FP32 block fill it, and
// its columns retire at scattered slots).  Columns above that width move into free slots below it; their
// slot records move here, their data and state by the two kernels below.
__global__ void __launch_bounds__(kRingThreads) ring_compact_select_kernel(const RingCtl* ctl, const RingDev* dev,
                                                                           SlotDev* slots, int B, int min_w,
                                                                           int always, int* from, int* to,
                                                                           int* count) {
  __shared__ int s_scan[kRingThreads];
  __shared__ int s_from[kRingThreads];
  __shared__ int s_to[kRingThreads];
  __shared__ int s_quiet;
  const int j = threadIdx.x;
  if (j == 0) s_quiet = always || load_acquire_sys(&ctl->tail) == dev->head;
  const int busy = j < B && slots[j].busy;
  int nb = 0;
  (void)block_rank(busy, s_scan, &nb);
  int w = min_w;
  while (w < nb) w <<= 1;
  w = std::min(w, B);
  const int mover = busy && j >= w;
  int nm = 0;
  const int rm = block_rank(mover, s_scan, &nm);
  if (mover) s_from[rm] = j;
  const int hole = j < w && !busy;
  int nh = 0;
  const int rh = block_rank(hole, s_scan, &nh);
  if (hole) s_to[rh] = j;
  __syncthreads();
  const int take = s_quiet ? std::min(nm, nh) : 0;
  if (j < take) {
    const int a = s_from[j], b = s_to[j];
    slots[b] = slots[a];
    slots[a].busy = 0;
    from[j] = a;
    to[j] = b;
  }
  if (j == 0) *count = take;
}

// Column `from[t]` of every row copied to column `to[t]` of the same block
// (the stored pair and y), rows spread over the warps by for_rows_items.
template <typename T>
__global__ void ring_move_columns_kernel(int64_t na, int B, const int* from, const int* to, const int* count, T* a0,
                                         T* a1, float* y) {
  const int nc = *count;
  if (nc == 0) return;
  for_rows_items(na, nc, [&](int64_t r, int t) {
    const int64_t a = r * B + from[t], b = r * B + to[t];
    a0[b] = a0[a];
    a1[b] = a1[a];
    y[b] = y[a];
  });
}

// Busy columns of both blocks after the iteration, for the host's statistics.
__global__ void ring_stats_kernel(RingCtl* ctl, const RingDev* dev) {
  ctl->active = dev->active32 + dev->active16;
}

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

int ring_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <typename T>
void mapped_alloc(T** host, T** dev, size_t count) {
  GP_CUDA_TRY(cudaHostAlloc((void**)host, sizeof(T) * count, cudaHostAllocMapped | cudaHostAllocPortable));
  std::memset((void*)*host, 0, sizeof(T) * count);
  GP_CUDA_TRY(cudaHostGetDevicePointer((void**)dev, (void*)*host, 0));
}

}  // namespace

RingLoop::RingLoop(Graph& g, int width, gp_dtype storage, cudaStream_t st, int t_long)
    : g_(g), B_(width), st_(st) {
  if (width < 8 || width > kRingThreads) throw Error{GP_EINVAL, "a ring block has 8 to 256 columns"};
  try {
    const bool two = storage == GP_BF16 || storage == GP_F16;
    e32_.reset(new ColumnEngine(g, width, GP_F32, st, t_long));
    if (two) e16_.reset(new ColumnEngine(g, width, storage, st, t_long, true));
    cap_req_ = 1024;
    cap_done_ = 4096;
    mapped_alloc(&ctl_, &ctl_d_, 1);
    mapped_alloc(&req_, &req_d_, (size_t)cap_req_);
    mapped_alloc(&done_, &done_d_, (size_t)cap_done_);
    const size_t bytes = sizeof(RingDev) + 2 * kRingThreads * sizeof(SlotDev) + (5 * kRingThreads + 8) * sizeof(int);
    dmem_ = g.alloc.get(bytes);
    GP_CUDA_TRY(cudaMemsetAsync(dmem_, 0, bytes, st_));
    GP_CUDA_TRY(cudaStreamSynchronize(st_));
    unsigned char* p = static_cast<unsigned char*>(dmem_);
    dev_ = reinterpret_cast<RingDev*>(p);
    p += sizeof(RingDev);
    slots32_ = reinterpret_cast<SlotDev*>(p);
    p += kRingThreads * sizeof(SlotDev);
    slots16_ = reinterpret_cast<SlotDev*>(p);
    p += kRingThreads * sizeof(SlotDev);
    int* ip = reinterpret_cast<int*>(p);
    new_list_ = ip;
    ret32_ = ip + kRingThreads;
    ret16_ = ip + 2 * kRingThreads;
    mig_from_ = ip + 3 * kRingThreads;
    mig_to_ = ip + 4 * kRingThreads;
    cnt_ = ip + 5 * kRingThreads;
  } catch (...) {
    release();
    throw;
  }
}

RingLoop::~RingLoop() { release(); }

void RingLoop::release() {
  if (st_) cudaStreamSynchronize(st_);
  for (cudaGraphExec_t& e : graph_) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  e16_.reset();
  e32_.reset();
  if (ctl_) cudaFreeHost(ctl_);
  if (req_) cudaFreeHost(req_);
  if (done_) cudaFreeHost(done_);
  ctl_ = nullptr;
  req_ = nullptr;
  done_ = nullptr;
  if (dmem_) g_.alloc.put(dmem_);
  dmem_ = nullptr;
}

int RingLoop::room() const {
  const uint64_t head = __atomic_load_n(&ctl_->head, __ATOMIC_ACQUIRE);
  return cap_req_ - (int)(tail_ - head);
}

void RingLoop::publish(const RingReq& r) {
  std::memcpy((void*)&req_[tail_ % (uint64_t)cap_req_], &r, sizeof(RingReq));
  ++tail_;
  __atomic_store_n(&ctl_->tail, tail_, __ATOMIC_RELEASE);
}

void RingLoop::take_done(std::vector<RingDone>& out) {
  const uint64_t done = __atomic_load_n(&ctl_->done, __ATOMIC_ACQUIRE);
  for (uint64_t c = consumed_; c < done; ++c) out.push_back(done_[c % (uint64_t)cap_done_]);
  consumed_ = done;
  __atomic_store_n(&ctl_->consumed, consumed_, __ATOMIC_RELEASE);
}

int RingLoop::active() const { return __atomic_load_n(&ctl_->active, __ATOMIC_RELAXED); }

void RingLoop::iterate() {
  TraceRange trace("gp_serve_iteration");
  const int par = e32_->view().pass & 1;
  if (graph_[par]) {
    GP_CUDA_TRY(cudaGraphLaunch(graph_[par], st_));
    count_launch(graph_launches_[par]);
    e32_->count_pass();
    if (e16_) e16_->count_pass();
    ++iters_;
    return;
  }
  // the first iterations launch directly: they set up the kernels' attributes
  // (lazily, once) outside any capture
  if (iters_ < 2 || graphs_off_) {
    enqueue();
    ++iters_;
    return;
  }
  const uint64_t n0 = g_launches.load();
  cudaGraph_t graph = nullptr;
  GP_CUDA_TRY(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
  try {
    enqueue();
  } catch (...) {
    cudaStreamEndCapture(st_, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  const uint64_t n = g_launches.load() - n0;
  GP_CUDA_TRY(cudaStreamEndCapture(st_, &graph));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    // nothing of the captured iteration ran: undo its pass counts and launch
    // it directly, now and from here on
    (void)cudaGetLastError();
    e32_->count_pass(-1);
    if (e16_) e16_->count_pass(-1);
    g_launches.fetch_sub(n);
    graphs_off_ = true;
    enqueue();
    ++iters_;
    return;
  }
  graph_[par] = exec;
  graph_launches_[par] = n;
  GP_CUDA_TRY(cudaGraphLaunch(exec, st_));
  ++iters_;
}

void RingLoop::enqueue() {
  const int sms = ring_sms();
  const int64_t na = g_.n_active;
  ColumnEngine::View v = e32_->view();
  // admission into the FP32 block: records, reset and r_0, r_1 of the new columns
  ring_admit_kernel<<<1, kRingThreads, 0, st_>>>(ctl_d_, req_d_, cap_req_, dev_, slots32_, v.col, v.par, v.stat,
                                                 v.norm, B_, new_list_);
  GP_LAUNCHED();
  ring_reset_kernel<<<sms * 8, 256, 0, st_>>>(na, B_, new_list_, dev_, v.f[0], v.f[1], v.y);
  GP_LAUNCHED();
  float* q1 = v.f[v.pass & 1];
  float* q0 = v.f[(v.pass + 1) & 1];
  if (g_.rp64)
    ring_init_kernel<int64_t><<<B_, 256, 0, st_>>>(g_.rp, g_.ci, na, B_, new_list_, dev_, slots32_, v.par, q0, q1, v.y);
  else
    ring_init_kernel<int32_t><<<B_, 256, 0, st_>>>(g_.rp, g_.ci, na, B_, new_list_, dev_, slots32_, v.par, q0, q1, v.y);
  GP_LAUNCHED();
  // one fused pass of each block, at the width its busy slots need
  ring_width_kernel<<<1, kRingThreads, 0, st_>>>(slots32_, B_, e32_->min_width(), cnt_ + 2);
  GP_LAUNCHED();
  e32_->pass_device(cnt_ + 2, &dev_->active32);
  if (e16_) {
    ring_width_kernel<<<1, kRingThreads, 0, st_>>>(slots16_, B_, e16_->min_width(), cnt_ + 3);
    GP_LAUNCHED();
    e16_->pass_device(cnt_ + 3, &dev_->active16);
  }
  // the stop rule on the norms of this pass, so finished columns retire now
  e32_->control_after();
  if (e16_) e16_->control_after();
  // retirement: outputs, done records, freed columns
  auto retire = [&](ColumnEngine& e, SlotDev* slots, int* ret, int* count, int block16) {
    const ColumnEngine::View w = e.view();
    ring_retire_kernel<<<1, kRingThreads, 0, st_>>>(ctl_d_, dev_, cap_done_, slots, w.stat, B_, ret, count);
    GP_LAUNCHED();
    ring_output_kernel<double><<<sms * 8, 256, 0, st_>>>(g_.n, na, g_.newid, w.y, B_, ret, count, slots);
    GP_LAUNCHED();
    ring_output_kernel<float><<<sms * 8, 256, 0, st_>>>(g_.n, na, g_.newid, w.y, B_, ret, count, slots);
    GP_LAUNCHED();
    ring_complete_kernel<<<1, kRingThreads, 0, st_>>>(ctl_d_, done_d_, cap_done_, dev_, slots, w.col, w.stat, w.norm,
                                                      ret, count, block16);
    GP_LAUNCHED();
  };
  retire(*e32_, slots32_, ret32_, cnt_ + 0, 0);
  if (e16_) retire(*e16_, slots16_, ret16_, cnt_ + 1, 1);
  // columns past their warm-up move to the 16-bit block (into the buffers each
  // block's next pass gathers and reads)
  if (e16_) {
    const ColumnEngine::View a = e32_->view(), b = e16_->view();
    ring_migrate_select_kernel<<<1, kRingThreads, 0, st_>>>(ctl_d_, dev_, slots32_, a.stat, B_, slots16_, B_, mig_from_,
                                                            mig_to_);
    GP_LAUNCHED();
    const float* fk = a.f[a.pass & 1];
    const float* fk1 = a.f[(a.pass + 1) & 1];
    if (b.storage == GP_F16)
      ring_migrate_columns_kernel<__half><<<sms * 8, 256, 0, st_>>>(na, B_, B_, mig_from_, mig_to_, dev_, fk, fk1, a.y,
                                                                    (__half*)b.h[b.pass & 1],
                                                                    (__half*)b.h[(b.pass + 1) & 1], b.y);
    else
      ring_migrate_columns_kernel<__nv_bfloat16><<<sms * 8, 256, 0, st_>>>(
          na, B_, B_, mig_from_, mig_to_, dev_, fk, fk1, a.y, (__nv_bfloat16*)b.h[b.pass & 1],
          (__nv_bfloat16*)b.h[(b.pass + 1) & 1], b.y);
    GP_LAUNCHED();
    ring_migrate_state_kernel<<<B_, 128, 0, st_>>>(mig_from_, mig_to_, &dev_->mig_count, a.col, a.par, a.stat,
                                                   a.norm, b.col, b.par, b.stat, b.norm);
    GP_LAUNCHED();
  }
  // a lightly loaded block packs its columns so that its passes narrow
  auto compact = [&](ColumnEngine& e, SlotDev* slots) {
    const ColumnEngine::View w = e.view();
    ring_compact_select_kernel<<<1, kRingThreads, 0, st_>>>(ctl_d_, dev_, slots, B_, e.min_width(),
                                                            w.pure16 ? 1 : 0, mig_from_, mig_to_, cnt_ + 4);
    GP_LAUNCHED();
    if (w.pure16)
      ring_move_columns_kernel<uint16_t><<<sms * 8, 256, 0, st_>>>(na, B_, mig_from_, mig_to_, cnt_ + 4,
                                                                   (uint16_t*)w.h[0], (uint16_t*)w.h[1], w.y);
    else
      ring_move_columns_kernel<float><<<sms * 8, 256, 0, st_>>>(na, B_, mig_from_, mig_to_, cnt_ + 4, w.f[0],
                                                                w.f[1], w.y);
    GP_LAUNCHED();
    ring_migrate_state_kernel<<<B_, 128, 0, st_>>>(mig_from_, mig_to_, cnt_ + 4, w.col, w.par, w.stat, w.norm, w.col,
                                                   w.par, w.stat, w.norm);
    GP_LAUNCHED();
  };
  compact(*e32_, slots32_);
  if (e16_) compact(*e16_, slots16_);
  ring_stats_kernel<<<1, 1, 0, st_>>>(ctl_d_, dev_);
  GP_LAUNCHED();
}

}  // namespace gp
