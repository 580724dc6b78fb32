// Batched multi-source ChebyPower (gp_batch) and the column engine the
// serving loop (serve.cpp) runs on.
//
// B queries are the columns of row-major blocks over the relabelled active
// rows: Q_k, Q_{k-1} (storage FP32, BF16 or FP16) and y (FP32), n_active x B.
// One fused SpMM pass advances every active column by one Chebyshev step
// (Eq. res-recurrence): for each row u and column j
//     acc_j = sum_{v in N(u)} Q_k[v][j]            (FP32; one B-wide row gather per edge)
//     r_j   = 2 acc_j - d_u Q_{k-1}[u][j]
//     Q_{k+1}[u][j] = r_j / d_u, y[u][j] += c_j r_j, ||r_j||_1 partial.
// Each edge gathers a whole B*s-byte row, so the block amortises the col_idx
// stream over B columns and uses every byte of the sectors it reads.
//
// The pass is bound by the latency of those gathers, so the kernel keeps many
// of them in flight without holding them in registers: each warp streams
// tiles of consecutive col_idx entries (staged in shared memory one tile
// ahead) and copies the gathered row segments with cp.async into a per-warp
// ring in shared memory, S rounds ahead of the lanes that add them up.  The
// own row's Q_{k-1} and y segments travel through the same ring after the
// row's gathers, so no step of a row waits on a dependent global load.
//
// Columns are independent queries: each has its own function, coefficient
// table, tail, tolerance, step k and stop state (per-column stop rule of
// Theorem 1 read for l1, as in the single query).  A control kernel between
// passes retires columns whose rule fired and sets the next coefficient of the
// others; retired columns are skipped (their y is final).  A column admitted
// at global pass g gets Q_1 in buffer g&1 and Q_0 in buffer (g+1)&1, so every
// pass reads buffer g&1 and writes buffer (g+1)&1 for all columns.
//
// Storage.  BF16/FP16 storage follows a warm-up schedule: passes run in FP32
// while any column's weight W(k) is at least warmup_tail, then two transition
// passes (FP32 -> 16-bit) and 16-bit from there on.  W(k) is the weight with
// which a rounding error of step k reaches y (warm_step below).  FP16 stores Q * 2^12 to
// keep small values of Q = r/d above FP16's subnormal range.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch.h"

namespace gp {

namespace {

constexpr float kF16Scale = 4096.0f;

// ---- schedule of the batched pass
// The pass walks tiles of consecutive col_idx entries (built per engine from
// the relabelled, degree-descending rows):
//   kind 0, rows per group: nrows rows of equal degree d; the lane groups of
//           a warp take one row each (rows g, g + EG, ...), no reduction;
//   kind 1, rows per warp:  nrows rows of equal degree d, each row's entries
//           split over the EG lane groups and combined by shuffles;
//   kind 2, chunk:          len entries of one long row (chunk p); the warp
//           that finishes the row's last chunk adds the chunk partials in
//           chunk order and updates the row.
// Descriptor int4 {row0, e0 low, e0 high, meta}: meta bits 0-1 kind,
// bits 2-16 nrows (kinds 0, 1) or p (kind 2), bits 17-31 d or len.
#ifndef GP_SPMM_TILE
#define GP_SPMM_TILE 512
#endif
constexpr int kBTileSpan = GP_SPMM_TILE;      // staged indices per buffer
constexpr int kBTileCap = kBTileSpan - 4;     // entries of a tile (room for 16-byte alignment)
constexpr int kBTileCost = kBTileSpan;        // rows tiles: nrows * (d + 3) at most
#ifndef GP_SPMM_THREADS
#define GP_SPMM_THREADS 512
#endif
#ifndef GP_SPMM_RING
#define GP_SPMM_RING 256
#endif
constexpr int kBatchThreads = GP_SPMM_THREADS;  // one persistent CTA per SM
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kRingLaneBytes = GP_SPMM_RING;    // per lane: bytes of gathers in flight
constexpr int kHeaderBytes = 256 * 12;          // ColState + norm of up to 256 columns
constexpr size_t kSpmmSmem =
    kHeaderBytes + (size_t)kBatchWarps * (32 * kRingLaneBytes + 2 * kBTileSpan * sizeof(int));

__host__ __device__ inline int4 make_btile(int64_t row0, int64_t e0, int kind, int a, int b) {
  const uint32_t meta = (uint32_t)kind | ((uint32_t)a << 2) | ((uint32_t)b << 17);
  return make_int4((int)row0, (int)(uint32_t)(e0 & 0xffffffffu), (int)(e0 >> 32), (int)meta);
}

struct BTile {
  int64_t row0, e0;
  int kind, a, b;
};

__device__ __forceinline__ BTile decode_btile(int4 t) {
  const uint32_t m = (uint32_t)t.w;
  return BTile{t.x, (int64_t)(uint32_t)t.y | ((int64_t)t.z << 32), (int)(m & 3u), (int)((m >> 2) & 0x7fffu),
               (int)(m >> 17)};
}

// ---- asynchronous-copy groups
__device__ __forceinline__ void bcommit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bwait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Byte offset of 16-byte piece h inside this lane's SB-byte ring slot.  The
// 8 lanes of a quarter-warp read piece h of their slots with one 16-byte
// shared load; with the pieces in order, slots 32 or 64 bytes apart put
// several of those lanes on the same banks.  So with SB = 32 lanes 4-7 (of
// every 8) swap their two pieces, and with SB = 64 the four pieces rotate by
// (lane / 2) % 4: each lane of a quarter-warp then reads a different 16-byte
// bank group, and a slot still holds its own SB bytes.
template <int SB>
__device__ __forceinline__ uint32_t piece(int h) {
  if constexpr (SB == 32) return (uint32_t)(16 * h) ^ (((threadIdx.x >> 2) & 1u) << 4);
  else if constexpr (SB == 64) return 16u * ((uint32_t)h ^ ((threadIdx.x >> 1) & 3u));
  else return 16u * (uint32_t)h;
}

// SB bytes from global to shared memory in 16-byte cp.async copies: global
// piece h of the segment goes to piece(h) of the slot.
template <int SB>
__device__ __forceinline__ void cp_seg(uint32_t dst, const unsigned char* src) {
  if constexpr (SB == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  } else if constexpr (SB == 32) {
    asm volatile(
        "cp.async.cg.shared.global [%0], [%2], 16;\n\t"
        "cp.async.cg.shared.global [%1], [%2+16], 16;" ::"r"(dst + piece<32>(0)),
        "r"(dst + piece<32>(1)), "l"(src)
        : "memory");
  } else {
    asm volatile(
        "cp.async.cg.shared.global [%0], [%4], 16;\n\t"
        "cp.async.cg.shared.global [%1], [%4+16], 16;\n\t"
        "cp.async.cg.shared.global [%2], [%4+32], 16;\n\t"
        "cp.async.cg.shared.global [%3], [%4+48], 16;" ::"r"(dst + piece<64>(0)),
        "r"(dst + piece<64>(1)), "r"(dst + piece<64>(2)), "r"(dst + piece<64>(3)), "l"(src)
        : "memory");
  }
}

// ---- 8-column vectors of each storage type
struct V8 {
  float x[8];
};

template <typename T>
struct Store;

template <>
struct Store<float> {
  static constexpr int bytes = 4;
  template <int N>
  __device__ static __forceinline__ void finish(float*) {}  // sums are in Q units
  struct Raw {
    float4 a, b;
  };
  // pieces h and h + 1 of an SB-byte ring slot
  template <int SB>
  __device__ static __forceinline__ Raw lds(const unsigned char* p, int h) {
    return Raw{*reinterpret_cast<const float4*>(p + piece<SB>(h)),
               *reinterpret_cast<const float4*>(p + piece<SB>(h + 1))};
  }
  __device__ static __forceinline__ void add(const Raw& r, float acc[8]) {
    acc[0] += r.a.x; acc[1] += r.a.y; acc[2] += r.a.z; acc[3] += r.a.w;
    acc[4] += r.b.x; acc[5] += r.b.y; acc[6] += r.b.z; acc[7] += r.b.w;
  }
  __device__ static __forceinline__ V8 load(const void* base, int64_t row, int B, int cg) {
    const float4* p = reinterpret_cast<const float4*>(static_cast<const float*>(base) + row * B + cg * 8);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    return V8{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w}};
  }
  __device__ static __forceinline__ void st8(unsigned char* at, const V8& v) {
    float4* p = reinterpret_cast<float4*>(at);
    p[0] = make_float4(v.x[0], v.x[1], v.x[2], v.x[3]);
    p[1] = make_float4(v.x[4], v.x[5], v.x[6], v.x[7]);
  }
  __device__ static __forceinline__ void st4(unsigned char* at, const float* v) {
    *reinterpret_cast<float4*>(at) = make_float4(v[0], v[1], v[2], v[3]);
  }
  __device__ static __forceinline__ void store(void* base, int64_t row, int B, int cg, const V8& v) {
    st8(reinterpret_cast<unsigned char*>(static_cast<float*>(base) + row * B + cg * 8), v);
  }
};

template <>
struct Store<__nv_bfloat16> {
  static constexpr int bytes = 2;
  template <int N>
  __device__ static __forceinline__ void finish(float*) {}  // sums are in Q units
  using Raw = uint4;
  // piece h of an SB-byte ring slot
  template <int SB>
  __device__ static __forceinline__ Raw lds(const unsigned char* p, int h) {
    return *reinterpret_cast<const uint4*>(p + piece<SB>(h));
  }
  // acc += each bf16 value, widened exactly inside a mixed-precision FP32 add.
  __device__ static __forceinline__ void add(const Raw& w, float acc[8]) {
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %2; add.rn.f32.bf16 %0, lo, %0; add.rn.f32.bf16 %1, hi, %1; }"
          : "+f"(acc[2 * i]), "+f"(acc[2 * i + 1])
          : "r"(u[i]));
  }
  __device__ static __forceinline__ void decode(const Raw& w, float v[8]) {
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      v[2 * i] = __uint_as_float(u[i] << 16);
      v[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
    }
  }
  __device__ static __forceinline__ V8 load(const void* base, int64_t row, int B, int cg) {
    V8 v;
    decode(__ldg(reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(base) + row * B + cg * 8)), v.x);
    return v;
  }
  __device__ static __forceinline__ void st8(unsigned char* at, const V8& v) {
    uint32_t u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v.x[2 * i], v.x[2 * i + 1]);
      u[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(at) = make_uint4(u[0], u[1], u[2], u[3]);
  }
  __device__ static __forceinline__ void st4(unsigned char* at, const float* v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2*>(at) = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
  }
  __device__ static __forceinline__ void store(void* base, int64_t row, int B, int cg, const V8& v) {
    st8(reinterpret_cast<unsigned char*>(static_cast<__nv_bfloat16*>(base) + row * B + cg * 8), v);
  }
};

template <>
struct Store<__half> {
  static constexpr int bytes = 2;
  using Raw = uint4;
  // piece h of an SB-byte ring slot
  template <int SB>
  __device__ static __forceinline__ Raw lds(const unsigned char* p, int h) {
    return *reinterpret_cast<const uint4*>(p + piece<SB>(h));
  }
  // acc += each stored value (Q * 2^12), widened exactly inside a
  // mixed-precision FP32 add; finish() removes the 2^12 once per row.
  __device__ static __forceinline__ void add(const Raw& w, float acc[8]) {
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %2; add.rn.f32.f16 %0, lo, %0; add.rn.f32.f16 %1, hi, %1; }"
          : "+f"(acc[2 * i]), "+f"(acc[2 * i + 1])
          : "r"(u[i]));
  }
  template <int N>
  __device__ static __forceinline__ void finish(float acc[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] *= 1.0f / kF16Scale;  // exact: a power of two
  }
  __device__ static __forceinline__ void decode(const Raw& w, float v[8]) {
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u[i]));
      v[2 * i] = f.x * (1.0f / kF16Scale);
      v[2 * i + 1] = f.y * (1.0f / kF16Scale);
    }
  }
  __device__ static __forceinline__ V8 load(const void* base, int64_t row, int B, int cg) {
    V8 v;
    decode(__ldg(reinterpret_cast<const uint4*>(static_cast<const __half*>(base) + row * B + cg * 8)), v.x);
    return v;
  }
  __device__ static __forceinline__ void st8(unsigned char* at, const V8& v) {
    uint32_t u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __half2 h = __floats2half2_rn(v.x[2 * i] * kF16Scale, v.x[2 * i + 1] * kF16Scale);
      u[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(at) = make_uint4(u[0], u[1], u[2], u[3]);
  }
  __device__ static __forceinline__ void st4(unsigned char* at, const float* v) {
    const __half2 a = __floats2half2_rn(v[0] * kF16Scale, v[1] * kF16Scale);
    const __half2 b = __floats2half2_rn(v[2] * kF16Scale, v[3] * kF16Scale);
    *reinterpret_cast<uint2*>(at) = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
  }
  __device__ static __forceinline__ void store(void* base, int64_t row, int B, int cg, const V8& v) {
    st8(reinterpret_cast<unsigned char*>(static_cast<__half*>(base) + row * B + cg * 8), v);
  }
};

// Update of a row from its neighbour sums acc = (P b)(u) and its own segment
// p of the older vector (Q_{k-1}, or B_{k+2} in Clenshaw's form):
//   forward:         r = 2 acc - d p, Q_{k+1} = r / d, y += c r, ||r||_1
//   Clenshaw step:   b_k = 2 acc - d p (the source term is added after the
//                    pass), B_k = b_k / d; no y
//   Clenshaw final:  y = acc - d p (= P b_1 - b_2; c_0 e_s is added after)
//   first step:      r_1 = acc (= P r_0), Q_1 = r_1 / d written to a fresh
//                    buffer, y += c_1 r_1 (start vectors other than e_s)
constexpr int kModeForward = 0, kModeClenshaw = 1, kModeClenshawFinal = 2, kModeFirst = 3;

struct SpmmArgs {
  const int4* tiles;
  int64_t ntiles;
  const int32_t* ci;
  const void* qcur;     // Q_k  (gather type)
  const void* qprev;    // Q_{k-1} (prev type)
  void* qnext;          // Q_{k+1} (out type); equals qprev when the types match
  float* y;             // n_active x B
  const ColState* col;  // per column: active flag and coefficient of this pass
  float* norm;          // per column ||r_{k+1}||_1 of this pass
  const int* poff;      // long rows: first chunk slot
  const int64_t* ldeg;  // long rows: degree
  float* part;          // long rows: chunk partial sums, [slot][B]
  int* cnt;             // long rows: chunks finished
  const void* zero;     // B zero values: the gather source of a neighbour beyond the active rows
  int64_t na;           // rows of the blocks (nodes with degree >= 1)
  int B;                // columns of this pass (a prefix of each row)
  int ldb;              // row stride of the blocks, in elements
  int check;            // col_idx lists rows beyond the active ones (host: picks the kernel)
  int* tile_ctr;        // tiles claimed past the first three per warp (zeroed by the control kernel)
  int mode;             // kModeForward, kModeClenshaw or kModeClenshawFinal
  const int* Bdev = nullptr;        // non-null: the pass width is read here (set on the device), B is its cap
  const int* active_dev = nullptr;  // non-null: the pass returns at once while this count of busy columns is 0
};

// Combine the entry groups' partial sums (lanes cg, cg + CG, cg + 2 CG, ...).
template <int LC>
__device__ __forceinline__ void reduce_groups(float acc[LC], int CG) {
  for (int off = CG; off < 32; off <<= 1) {
#pragma unroll
    for (int i = 0; i < LC; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
  }
}

// Compile-time geometry of one kernel instance: a lane owns LC consecutive
// columns; one ring round moves SB bytes per lane.
template <typename TG, typename TP, typename TO, int LC>
struct Geo {
  static constexpr int sG = Store<TG>::bytes, sP = Store<TP>::bytes;
  static constexpr int SB = LC * sG;              // bytes of a gathered segment
  static constexpr int S = kRingLaneBytes / SB;   // rounds in flight
  static constexpr int OP = LC * sP / SB;         // rounds of the own Q_{k-1} segment (1 or 2)
  static constexpr int OY = LC * 4 / SB;          // rounds of the own y segment (1 or 2)
  static constexpr int OWN = OP + OY;
  static constexpr uint32_t kStride = 32 * SB;    // ring bytes per round (whole warp)
  static constexpr uint32_t kMask = S * kStride - 1;
  static_assert(S >= 2 && (S & (S - 1)) == 0, "ring depth must be a power of two");
  static_assert(SB == 16 || SB == 32 || SB == 64, "a round moves 16, 32 or 64 bytes per lane");
};

// Per-lane constants of the pass.  The loops read these register copies
// rather than the kernel arguments: the memory clobbers of the cp.async
// statements would force every argument read from memory to be repeated after
// each copy.
struct Lane {
  const SpmmArgs* a;            // (chunk and finisher paths only)
  const ColState* s_col;        // state of this lane's column c at s_col[c * CG] (col())
  uint32_t ring;                // shared address of this lane's slot 0
  const unsigned char* ring_p;  // the same, generic
  const unsigned char* qseg;    // Q_k + this lane's segment offset
  const unsigned char* pseg;    // Q_{k-1} + this lane's segment offset
  unsigned char* nseg;          // Q_{k+1} + this lane's segment offset
  unsigned char* yseg;          // y + this lane's segment offset
  const unsigned char* zero;    // zero segment
  uint32_t rowG, rowP, rowN, rowY;  // row bytes of Q_k, Q_{k-1}, Q_{k+1}, y
  int na;
  int mode;                     // kMode*: which row update the pass applies
  int B;                        // columns of this pass
  int cg, g, CG, EG, lane;
  __device__ __forceinline__ ColState col(int c) const { return s_col[c * CG]; }
};

// Source of the gathered segment of neighbour v.  Rows beyond the active ones,
// which only an unvalidated asymmetric CSR can list, read zeros; the check is
// compiled in only for graphs whose ingest found such entries (CHECK).
template <bool CHECK>
__device__ __forceinline__ const unsigned char* gather_src(const Lane& L, int v) {
  if constexpr (CHECK) return v < L.na ? L.qseg + (uint64_t)(uint32_t)v * L.rowG : L.zero;
  return L.qseg + (uint64_t)(uint32_t)v * L.rowG;
}

// Source of piece o (SB bytes) of row u's own Q_{k-1} segment (o < OP) or y
// segment.
template <int SB, int OP>
__device__ __forceinline__ const unsigned char* own_src(const Lane& L, int64_t u, int o) {
  return o < OP ? L.pseg + (uint64_t)(uint32_t)u * L.rowP + o * SB
                : L.yseg + (uint64_t)(uint32_t)u * L.rowY + (o - OP) * SB;
}

// Add one gathered segment (LC values of TG) from a ring slot.
template <typename TG, int LC>
__device__ __forceinline__ void add_seg(const unsigned char* p, float acc[LC]) {
  constexpr int SB = LC * Store<TG>::bytes;
  constexpr int PG = 8 * Store<TG>::bytes / 16;  // pieces of 8 values
#pragma unroll
  for (int h = 0; h < LC / 8; ++h) Store<TG>::add(Store<TG>::template lds<SB>(p, h * PG), acc + 8 * h);
}

// A lane's neighbour sums.  FP32 gathers add in two levels: rounds go into
// blk, and every kBlk rounds (a warp-uniform count kept by the loop) blk is
// added to acc, so the rounding error of a lane's sum over n entries grows
// like kBlk + n / kBlk ulps instead of n (a lane of a 256-column FP32 pass sums
// a whole 508-entry chunk).  16-bit gathers carry their own storage rounding,
// far above that, and add directly.
constexpr int kBlk = 16;
template <typename TG, int LC>
struct LaneSum {
  static constexpr bool kTwo = Store<TG>::bytes == 4;
  float acc[LC];
  float blk[kTwo ? LC : 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < LC; ++i) acc[i] = 0.f;
    if constexpr (kTwo) {
#pragma unroll
      for (int i = 0; i < LC; ++i) blk[i] = 0.f;
    }
  }
  __device__ __forceinline__ void add(const unsigned char* p) { add_seg<TG, LC>(p, kTwo ? blk : acc); }
  // after round r of a sum (warp-uniform r): close a block every kBlk rounds
  __device__ __forceinline__ void round_done(int r) {
    if constexpr (kTwo) {
      if ((r & (kBlk - 1)) == kBlk - 1) flush();
    }
  }
  // acc = the whole sum (call before acc is read)
  __device__ __forceinline__ void flush() {
    if constexpr (kTwo) {
#pragma unroll
      for (int i = 0; i < LC; ++i) {
        acc[i] += blk[i];
        blk[i] = 0.f;
      }
    }
  }
};

// Copy a tile's col_idx entries [e0, e0 + len) into a warp's staging buffer
// with 16-byte copies from the aligned-down start; entry e0 + i lands at
// index (e0 & 3) + i.  (col_idx is padded so the last vector is in bounds.)
__device__ __forceinline__ void stage_indices(int* buf, const int32_t* ci, int64_t e0, int len, int lane) {
  const int64_t a0 = e0 & ~(int64_t)3;
  const int nvec = (int)((e0 + len - a0 + 3) >> 2);
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
  for (int v = lane; v < nvec; v += 32) cp_seg<16>(base + 16u * v, reinterpret_cast<const unsigned char*>(ci + a0 + 4 * v));
}

__device__ __forceinline__ int tile_len(const BTile& t) { return t.kind == 2 ? t.b : t.a * t.b; }

// The row update, applied as row u's own segments land (after its gathers,
// so acc holds the final neighbour sums).  A Q_{k-1} piece (columns C0 ..
// C0 + PC - 1) turns acc into r = 2 acc - d Q_{k-1} and writes
// Q_{k+1} = r / d; a y piece (columns C0 .. C0 + PW - 1) adds c r to y.
// Retired columns keep their values (Q copied, y final).
template <typename TP, typename TO, int LC, int SB, int PC, int C0>
__device__ __forceinline__ void prev_piece(const Lane& L, int64_t u, float d, const unsigned char* src, float acc[LC],
                                           float nrm[LC]) {
  float prev[PC];
  if constexpr (Store<TP>::bytes == 4) {
#pragma unroll
    for (int q = 0; q < PC / 4; ++q) {
      const float4 x = *reinterpret_cast<const float4*>(src + piece<SB>(q));
      prev[4 * q] = x.x; prev[4 * q + 1] = x.y; prev[4 * q + 2] = x.z; prev[4 * q + 3] = x.w;
    }
  } else {
    static_assert(PC % 8 == 0, "a 16-bit Q_{k-1} segment is one round of whole 8-column groups");
#pragma unroll
    for (int h = 0; h < PC / 8; ++h) Store<TP>::decode(Store<TP>::template lds<SB>(src, h), prev + 8 * h);
  }
  const float inv = 1.0f / d;
  float out[PC];
  if (L.mode == kModeClenshawFinal) {
    // y = P b_1 - b_2 over the piece's columns (FP32 y, written, not read)
#pragma unroll
    for (int i = 0; i < PC; ++i) out[i] = acc[C0 + i] - d * prev[i];
    unsigned char* yd = L.yseg + (uint64_t)(uint32_t)u * L.rowY + C0 * 4;
#pragma unroll
    for (int q = 0; q < PC / 4; ++q)
      *reinterpret_cast<float4*>(yd + 16 * q) = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
    return;
  }
  const bool first = L.mode == kModeFirst;
  const float two = first ? 1.0f : 2.0f, dp = first ? 0.0f : d;
#pragma unroll
  for (int i = 0; i < PC; ++i) {
    const int c = C0 + i;
    const ColState cs = L.col(c);
    const float r = two * acc[c] - dp * prev[i];
    out[i] = cs.active ? r * inv : prev[i];
    acc[c] = cs.active ? r : 0.f;
    if (L.mode == kModeForward || first) nrm[c] += fabsf(acc[c]);
  }
  unsigned char* dst = L.nseg + (uint64_t)(uint32_t)u * L.rowN + C0 * Store<TO>::bytes;
  if constexpr (PC % 8 == 0) {
#pragma unroll
    for (int h = 0; h < PC / 8; ++h) {
      V8 o8;
#pragma unroll
      for (int i = 0; i < 8; ++i) o8.x[i] = out[8 * h + i];
      Store<TO>::st8(dst + h * 8 * Store<TO>::bytes, o8);
    }
  } else {
    static_assert(PC == 4, "a Q_{k-1} piece holds 4, 8 or 16 columns");
    Store<TO>::st4(dst, out);
  }
}

template <int LC, int SB, int PW, int C0>
__device__ __forceinline__ void y_piece(const Lane& L, int64_t u, const unsigned char* src, const float acc[LC]) {
  float4* yrow = reinterpret_cast<float4*>(L.yseg + (uint64_t)(uint32_t)u * L.rowY + C0 * 4);
#pragma unroll
  for (int q = 0; q < PW / 4; ++q) {
    float4 x = *reinterpret_cast<const float4*>(src + piece<SB>(q));
    float* xv = reinterpret_cast<float*>(&x);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = C0 + 4 * q + k;
      const ColState cs = L.col(c);
      xv[k] = fmaf(cs.active ? cs.coef : 0.f, acc[c], xv[k]);
    }
    yrow[q] = x;
  }
}

// Own round o of row u: Q_{k-1} pieces (o < OP), then y pieces.
template <typename TP, typename TO, int LC, int SB, int OP, int OY>
__device__ __forceinline__ void own_round(const Lane& L, int64_t u, float d, int o, const unsigned char* src,
                                          float acc[LC], float nrm[LC]) {
  constexpr int PC = LC / OP, PW = LC / OY;
  if (o < OP) {
    if constexpr (OP == 1) {
      prev_piece<TP, TO, LC, SB, PC, 0>(L, u, d, src, acc, nrm);
    } else {
      if (o == 0)
        prev_piece<TP, TO, LC, SB, PC, 0>(L, u, d, src, acc, nrm);
      else
        prev_piece<TP, TO, LC, SB, PC, PC>(L, u, d, src, acc, nrm);
    }
  } else {
    if constexpr (OY == 1) {
      y_piece<LC, SB, PW, 0>(L, u, src, acc);
    } else {
      if (o == OP)
        y_piece<LC, SB, PW, 0>(L, u, src, acc);
      else
        y_piece<LC, SB, PW, PW>(L, u, src, acc);
    }
  }
}

// Kind 0 tile: lane group g takes rows g, g + EG, ... of the tile; a row is d
// gather rounds, then OP rounds of its Q_{k-1} segment and OY of its y
// segment.  The caller has issued the next tile's index copies, which join
// round 0's copy group.
template <typename TG, typename TP, typename TO, int LC, bool CHECK>
__device__ __forceinline__ void tile_rows_per_group(const Lane& L, const BTile& t, const int* ci_t, float nrm[LC]) {
  using C = Geo<TG, TP, TO, LC>;
  constexpr int S = C::S, SB = C::SB, OP = C::OP;
  const int OWN = L.mode == kModeForward || L.mode == kModeFirst ? C::OWN : OP;  // Clenshaw: no y
  const int d = t.b, nrows = t.a, EG = L.EG;
  const int nseq = (nrows + EG - 1) / EG;
  const int R = nseq * (d + OWN);
  // producer: row sequence, gathers left in the row, own round, next index
  int p_seq = 0, p_left = d, p_own = 0, p_row = L.g;
  const int* p_ci = ci_t + L.g * d;
  uint32_t p_off = 0;
  auto issue = [&]() {
    if (p_seq < nseq) {
      const uint32_t dst = L.ring + p_off;
      if (p_left > 0) {
        if (p_row < nrows) cp_seg<SB>(dst, gather_src<CHECK>(L, *p_ci));
        ++p_ci;
        --p_left;
      } else {
        if (p_row < nrows) cp_seg<SB>(dst, own_src<SB, OP>(L, t.row0 + p_row, p_own));
        if (++p_own == OWN) {
          p_own = 0;
          ++p_seq;
          p_row += EG;
          p_ci += (EG - 1) * d;
          p_left = d;
        }
      }
    }
    p_off = (p_off + C::kStride) & C::kMask;
  };
  LaneSum<TG, LC> sum;
  sum.zero();
#pragma unroll 1
  for (int i = 0; i < S - 1; ++i) {
    issue();
    bcommit();
  }
  int c_left = d, c_own = 0, c_row = L.g;
  uint32_t c_off = 0;
#pragma unroll 1
  for (int rc = 0; rc < R; ++rc) {
    bwait<S - 2>();  // round rc has landed
    const unsigned char* src = L.ring_p + c_off;
    const bool mine = c_row < nrows;
    if (c_left > 0) {
      if (mine) sum.add(src);
      sum.round_done(d - c_left);
      --c_left;
    } else {
      if (c_own == 0) {
        sum.flush();
        Store<TG>::template finish<LC>(sum.acc);
      }
      if (mine) own_round<TP, TO, LC, SB, OP, C::OY>(L, t.row0 + c_row, (float)d, c_own, src, sum.acc, nrm);
      if (++c_own == OWN) {
        sum.zero();
        c_own = 0;
        c_row += EG;
        c_left = d;
      }
    }
    c_off = (c_off + C::kStride) & C::kMask;
    issue();
    bcommit();
  }
}

// Last chunk of a long row: add the chunk partials in chunk order and update
// the row (its own segments are read directly: long rows are few).
template <typename TP, typename TO, int LC>
__device__ __forceinline__ void finish_long_row(const Lane& L, int64_t row, int slot0, int np, float nrm[LC]) {
  const SpmmArgs& a = *L.a;
  __threadfence();
  float tot[LC];
#pragma unroll
  for (int i = 0; i < LC; ++i) tot[i] = 0.f;
  for (int i = L.g; i < np; i += L.EG) {
    const float4* src = reinterpret_cast<const float4*>(a.part + (int64_t)(slot0 + i) * L.B + L.cg * LC);
#pragma unroll
    for (int q = 0; q < LC / 4; ++q) {
      const float4 x = __ldcg(src + q);
      tot[4 * q] += x.x; tot[4 * q + 1] += x.y; tot[4 * q + 2] += x.z; tot[4 * q + 3] += x.w;
    }
  }
  reduce_groups<LC>(tot, L.CG);
  if (L.lane == 0) a.cnt[row] = 0;
  if (L.g == 0) {
    const float d = (float)a.ldeg[row];
    const float inv = 1.0f / d;
    if (L.mode == kModeClenshawFinal) {  // y = P b_1 - b_2
      float* yrow = a.y + row * a.ldb + L.cg * LC;
#pragma unroll
      for (int h = 0; h < LC / 8; ++h) {
        const V8 pv = Store<TP>::load(a.qprev, row, a.ldb, L.cg * (LC / 8) + h);
#pragma unroll
        for (int i = 0; i < 8; ++i) yrow[8 * h + i] = tot[8 * h + i] - d * pv.x[i];
      }
      return;
    }
#pragma unroll
    for (int h = 0; h < LC / 8; ++h) {
      const V8 pv = Store<TP>::load(a.qprev, row, a.ldb, L.cg * (LC / 8) + h);
      V8 out;
      const bool first = L.mode == kModeFirst;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = 8 * h + i;
        const ColState cs = L.col(c);
        const float r = first ? tot[c] : 2.0f * tot[c] - d * pv.x[i];
        out.x[i] = cs.active ? r * inv : pv.x[i];
        tot[c] = cs.active ? r : 0.f;
        if (L.mode == kModeForward || first) nrm[c] += fabsf(tot[c]);
      }
      Store<TO>::store(a.qnext, row, a.ldb, L.cg * (LC / 8) + h, out);
    }
    if (L.mode == kModeClenshaw) return;  // Clenshaw steps: no y
    float4* yrow = reinterpret_cast<float4*>(a.y + row * a.ldb + L.cg * LC);
#pragma unroll
    for (int q = 0; q < LC / 4; ++q) {
      float4 x = yrow[q];
      float* xv = reinterpret_cast<float*>(&x);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const ColState cs = L.col(4 * q + k);
        xv[k] = fmaf(cs.active ? cs.coef : 0.f, tot[4 * q + k], xv[k]);
      }
      yrow[q] = x;
    }
  }
}

// A chunk's neighbour sums are complete: publish its partial; the warp that
// publishes the row's last chunk finishes the row.
template <typename TG, typename TP, typename TO, int LC>
__device__ __forceinline__ void publish_chunk(const Lane& L, const BTile& t, float acc[LC], float nrm[LC]) {
  const SpmmArgs& a = *L.a;
  reduce_groups<LC>(acc, L.CG);
  Store<TG>::template finish<LC>(acc);
  const int64_t row = t.row0;
  const int slot0 = a.poff[row], np = a.poff[row + 1] - slot0;
  if (L.g == 0) {
    float4* dst = reinterpret_cast<float4*>(a.part + (int64_t)(slot0 + t.a) * L.B + L.cg * LC);
#pragma unroll
    for (int i = 0; i < LC / 4; ++i) dst[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
  }
  __threadfence();
  __syncwarp();
  int old = 0;
  if (L.lane == 0) old = atomicAdd(&a.cnt[row], 1);
  old = __shfl_sync(0xffffffffu, old, 0);
  if (old == np - 1) finish_long_row<TP, TO, LC>(L, row, slot0, np, nrm);
}

// Kind 2 tile (a chunk of a long row): pure gather rounds, entry j = r*EG + g
// of the chunk in round r, two rounds per iteration under one wait.
template <typename TG, typename TP, typename TO, int LC, bool CHECK>
__device__ __forceinline__ void tile_chunk(const Lane& L, const BTile& t, const int* ci_t, float nrm[LC]) {
  using C = Geo<TG, TP, TO, LC>;
  constexpr int S = C::S, SB = C::SB;
  static_assert(S >= 3, "two rounds per wait need at least three in the ring");
  const int EG = L.EG, g = L.g;
  const int len = t.b;
  const int G = (len + EG - 1) / EG;
  int pj = g;         // chunk entry of the next round to issue
  uint32_t p_off = 0;
  auto issue = [&]() {
    if (pj < len) cp_seg<SB>(L.ring + p_off, gather_src<CHECK>(L, ci_t[pj]));
    pj += EG;
    p_off = (p_off + C::kStride) & C::kMask;
  };
  LaneSum<TG, LC> sum;
  sum.zero();
#pragma unroll 1
  for (int i = 0; i < S - 1; ++i) {
    issue();
    bcommit();
  }
  int rc = 0, cj = g;
  uint32_t c_off = 0;
#pragma unroll 1
  for (; rc + 1 < G; rc += 2) {
    bwait<S - 3>();  // rounds rc and rc + 1 have landed
    const unsigned char* s0 = L.ring_p + c_off;
    const unsigned char* s1 = L.ring_p + ((c_off + C::kStride) & C::kMask);
    if (cj < len) sum.add(s0);
    if (cj + EG < len) sum.add(s1);
    sum.round_done(rc + 1);
    cj += 2 * EG;
    c_off = (c_off + 2 * C::kStride) & C::kMask;
    issue();
    bcommit();
    issue();
    bcommit();
  }
  if (rc < G) {
    bwait<S - 2>();
    if (cj < len) sum.add(L.ring_p + c_off);
    issue();
    bcommit();
  }
  sum.flush();
  publish_chunk<TG, TP, TO, LC>(L, t, sum.acc, nrm);
}

// Kind 1 tile: the EG lane groups split each row's entries (entry j of a row
// goes to group j % EG) and combine their sums by shuffles; the row then takes
// OP + OY own rounds (group 0).
template <typename TG, typename TP, typename TO, int LC, bool CHECK>
__device__ __forceinline__ void tile_rows_per_warp(const Lane& L, const BTile& t, const int* ci_t, float nrm[LC]) {
  using C = Geo<TG, TP, TO, LC>;
  constexpr int S = C::S, SB = C::SB, OP = C::OP;
  const int OWN = L.mode == kModeForward || L.mode == kModeFirst ? C::OWN : OP;  // Clenshaw: no y
  const int EG = L.EG, g = L.g;
  const int d = t.b;  // entries per row
  const int G = (d + EG - 1) / EG;
  const int nseq = t.a;
  const int R = nseq * (G + OWN);
  int p_seq = 0, p_left = G, p_own = 0, p_j = g;
  const int* p_ci = ci_t + g;
  uint32_t p_off = 0;
  auto issue = [&]() {
    if (p_seq < nseq) {
      const uint32_t dst = L.ring + p_off;
      if (p_left > 0) {
        if (p_j < d) cp_seg<SB>(dst, gather_src<CHECK>(L, *p_ci));
        p_ci += EG;
        p_j += EG;
        --p_left;
      } else {
        if (g == 0) cp_seg<SB>(dst, own_src<SB, OP>(L, t.row0 + p_seq, p_own));
        if (++p_own == OWN) {
          p_own = 0;
          ++p_seq;
          p_left = G;
          p_j = g;
          p_ci = ci_t + p_seq * d + g;
        }
      }
    }
    p_off = (p_off + C::kStride) & C::kMask;
  };
  LaneSum<TG, LC> sum;
  sum.zero();
#pragma unroll 1
  for (int i = 0; i < S - 1; ++i) {
    issue();
    bcommit();
  }
  int c_seq = 0, c_left = G, c_own = 0, c_j = g;
  uint32_t c_off = 0;
#pragma unroll 1
  for (int rc = 0; rc < R; ++rc) {
    bwait<S - 2>();  // round rc has landed
    const unsigned char* src = L.ring_p + c_off;
    if (c_left > 0) {
      if (c_j < d) sum.add(src);
      sum.round_done(G - c_left);
      c_j += EG;
      --c_left;
    } else {
      if (c_own == 0) {  // the row's sums, before its first own piece
        sum.flush();
        reduce_groups<LC>(sum.acc, L.CG);
        Store<TG>::template finish<LC>(sum.acc);
      }
      if (g == 0) own_round<TP, TO, LC, SB, OP, C::OY>(L, t.row0 + c_seq, (float)d, c_own, src, sum.acc, nrm);
      if (++c_own == OWN) {
        sum.zero();
        c_own = 0;
        ++c_seq;
        c_left = G;
        c_j = g;
      }
    }
    c_off = (c_off + C::kStride) & C::kMask;
    issue();
    bcommit();
  }
}

// One fused SpMM pass (see the top of this file).  Per warp, a ring of S
// rounds of cp.async copies in shared memory keeps S row segments per lane in
// flight: round i of a tile is issued S - 1 rounds before it is consumed.  A
// lane group's round copies either one gathered neighbour row segment of
// Q_k, or one piece of its own row's Q_{k-1} and y (fetched through the same
// ring, after the row's gathers, so the update finds them on chip).
template <typename TG, typename TP, typename TO, int LC, bool CHECK>
__global__ void __launch_bounds__(kBatchThreads, 1) spmm_step_kernel(const __grid_constant__ SpmmArgs a) {
  using C = Geo<TG, TP, TO, LC>;
  extern __shared__ __align__(16) unsigned char s_raw[];
  if (a.active_dev && *a.active_dev == 0) return;  // no busy column (set on the device)
  const int B = a.Bdev ? *a.Bdev : a.B;
  ColState* s_col = reinterpret_cast<ColState*>(s_raw);
  float* s_norm = reinterpret_cast<float*>(s_raw + sizeof(ColState) * B);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* ring = s_raw + kHeaderBytes + (size_t)warp * 32 * kRingLaneBytes;
  int* s_ci = reinterpret_cast<int*>(s_raw + kHeaderBytes + (size_t)kBatchWarps * 32 * kRingLaneBytes) +
              warp * 2 * kBTileSpan;
  // column j = cg * LC + i of the pass is stored at i * CG + cg, so that the
  // lane groups of a warp reading column i of their segments read adjacent
  // entries (in column order the reads were LC * 8 bytes apart: one bank)
  for (int j = threadIdx.x; j < B; j += blockDim.x) {
    s_col[(j % LC) * (B / LC) + j / LC] = a.col[j];
    s_norm[j] = 0.f;
  }
  __syncthreads();
  Lane L;
  L.a = &a;
  L.B = B;
  L.CG = B / LC;
  L.EG = 32 / L.CG;
  L.cg = lane % L.CG;
  L.g = lane / L.CG;
  L.lane = lane;
  L.s_col = s_col + L.cg;
  L.ring = (uint32_t)__cvta_generic_to_shared(ring) + lane * C::SB;
  L.ring_p = ring + lane * C::SB;
  L.qseg = static_cast<const unsigned char*>(a.qcur) + (size_t)L.cg * C::SB;
  L.pseg = static_cast<const unsigned char*>(a.qprev) + (size_t)L.cg * LC * C::sP;
  L.nseg = static_cast<unsigned char*>(a.qnext) + (size_t)L.cg * LC * Store<TO>::bytes;
  L.yseg = reinterpret_cast<unsigned char*>(a.y) + (size_t)L.cg * LC * 4;
  L.zero = static_cast<const unsigned char*>(a.zero) + L.cg * C::SB;
  L.rowG = (uint32_t)(a.ldb * C::sG);
  L.rowP = (uint32_t)(a.ldb * C::sP);
  L.rowN = (uint32_t)(a.ldb * Store<TO>::bytes);
  L.rowY = (uint32_t)(a.ldb * 4);
  L.na = (int)a.na;
  L.mode = a.mode;
  float nrm[LC];
#pragma unroll
  for (int i = 0; i < LC; ++i) nrm[i] = 0.f;

  // Tiles: each warp starts with tiles w, w + W and w + 2W (W warps in the
  // grid), then takes the next unclaimed tile from a per-pass counter, so the
  // pass ends when the work does rather than with the warp that drew the
  // costliest tiles.  A claim is three tiles ahead: its atomic completes while
  // the warp works on the current tile, and the claimed tile's descriptor
  // loads during the next one.
  const int64_t nwarps = (int64_t)gridDim.x * kBatchWarps;
  int64_t w = (int64_t)blockIdx.x * kBatchWarps + warp;
  int64_t wn = w + nwarps, wnn = w + 2 * nwarps;
  int4 cur = make_int4(0, 0, 0, 0), nd = make_int4(0, 0, 0, 0);
  if (w < a.ntiles) {
    cur = a.tiles[w];
    const BTile t0 = decode_btile(cur);
    stage_indices(s_ci, a.ci, t0.e0, tile_len(t0), lane);
    bcommit();
    bwait<0>();
    if (wn < a.ntiles) nd = a.tiles[wn];
  }
  for (int buf = 0; w < a.ntiles; buf ^= 1) {
    __syncwarp();  // this tile's staged indices are visible; the other buffer is free
    const BTile t = decode_btile(cur);
    const int* ci_t = s_ci + buf * kBTileSpan + (int)(t.e0 & 3);
    if (wn < a.ntiles) {  // the next tile's indices join this tile's first copy group
      const BTile tn = decode_btile(nd);
      stage_indices(s_ci + (buf ^ 1) * kBTileSpan, a.ci, tn.e0, tile_len(tn), lane);
    }
    int claimed = 0;
    if (lane == 0) claimed = atomicAdd(a.tile_ctr, 1);
    int4 nd2 = make_int4(0, 0, 0, 0);
    if (wnn < a.ntiles) nd2 = a.tiles[wnn];
    if (t.kind == 0)
      tile_rows_per_group<TG, TP, TO, LC, CHECK>(L, t, ci_t, nrm);
    else if (t.kind == 1)
      tile_rows_per_warp<TG, TP, TO, LC, CHECK>(L, t, ci_t, nrm);
    else
      tile_chunk<TG, TP, TO, LC, CHECK>(L, t, ci_t, nrm);
    const int64_t w3 = 3 * nwarps + __shfl_sync(0xffffffffu, claimed, 0);
    cur = nd;
    nd = nd2;
    w = wn;
    wn = wnn;
    wnn = w3;
    bwait<0>();  // only empty groups remain; the next tile restarts the ring at slot 0
  }
#pragma unroll
  for (int i = 0; i < LC; ++i)
    if (nrm[i] != 0.f) atomicAdd(&s_norm[L.cg * LC + i], nrm[i]);
  __syncthreads();
  for (int j = threadIdx.x; j < B; j += blockDim.x)
    if (s_norm[j] != 0.f) atomicAdd(&a.norm[j], s_norm[j]);
}

// Before each pass: fold the last pass's norm into each active column's
// running max, apply its stop rule, and set the coefficient of the next step.
// phase -1 treats every column (before a pass); the service splits it: phase
// 0 before a pass treats only columns that have not run one (k = 1), phase 1
// right after the pass treats the others, so a column whose rule fires on the
// norm of that pass retires before the next pass instead of riding it idle.
__global__ void control_kernel(ColState* col, const ColParam* par, ColStat* stat, float* norm, int B, int kcap,
                               int* tile_ctr, int phase) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0 && phase <= 0) *tile_ctr = 0;
  if (j >= B) return;
  ColState& cs = col[j];
  const ColParam& p = par[j];
  ColStat& st = stat[j];
  if (!cs.active) {
    norm[j] = 0.f;
    return;
  }
  if ((phase == 0 && st.k != 1) || (phase == 1 && st.k < 2)) return;
  if (st.k > 1) st.C = fmaxf(st.C, norm[j]);  // ||r_k||_1 from the last pass
  norm[j] = 0.f;
  const bool stop_rule = p.tol >= 0.f && p.tail[st.k] * st.C <= p.tol;
  const bool stop_fixed = p.kstop > 0 && st.k >= p.kstop;
  if (stop_rule || stop_fixed || st.k >= kcap) {
    cs.active = 0;
    st.K = st.k;
    st.done = 1;
    return;
  }
  cs.coef = p.c[st.k + 1];
  st.k += 1;
}

// Zero the given columns of Q_a, Q_b (and the 16-bit pair) and y over all
// rows: a warp per row, its lanes over the listed columns (one row's writes
// share its cache lines).
__global__ void reset_columns_kernel(int64_t na, int B, const int* cols, int ncols, float* fa, float* fb,
                                     uint16_t* ha, uint16_t* hb, float* y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < na; r += nw) {
    for (int t = lane; t < ncols; t += 32) {
      const int64_t i = r * B + cols[t];
      fa[i] = 0.f;
      fb[i] = 0.f;
      y[i] = 0.f;
      if (ha) {
        ha[i] = 0;  // +0 in BF16 and FP16
        hb[i] = 0;
      }
    }
  }
}

// Move columns perm[0 .. nb) of every row to columns 0 .. nb) in place: a
// warp per row reads all the values it moves before it writes any.
template <typename T>
__device__ __forceinline__ void permute_row(T* base, int64_t r, int ldb, const int* perm, int nb, int lane) {
  T v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = lane + 32 * i;
    if (j < nb) v[i] = base[r * ldb + perm[j]];
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = lane + 32 * i;
    if (j < nb) base[r * ldb + j] = v[i];
  }
  __syncwarp();
}

__global__ void permute_columns_kernel(int64_t na, int ldb, const int* perm, int nb, float* fa, float* fb,
                                       uint16_t* ha, uint16_t* hb, float* y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < na; r += nw) {
    if (fa) {  // a 16-bit engine has no FP32 pair
      permute_row(fa, r, ldb, perm, nb, lane);
      permute_row(fb, r, ldb, perm, nb, lane);
    }
    permute_row(y, r, ldb, perm, nb, lane);
    if (ha) {
      permute_row(ha, r, ldb, perm, nb, lane);
      permute_row(hb, r, ldb, perm, nb, lane);
    }
  }
}

// r_0 = e_s, r_1 = P e_s for column j (FP32 buffers): Q_0 -> q0, Q_1 -> q1,
// y = c_0 r_0 + c_1 r_1.  One block per new column.
template <typename RP>
__global__ void init_columns_kernel(const void* rpv, const int32_t* ci, int64_t na, int B, const int* cols,
                                    const int64_t* src,
                                    const float* c0, const float* c1, float* q0, float* q1, float* y) {
  const RP* rp = (const RP*)rpv;
  const int j = cols[blockIdx.x];
  const int64_t s = src[blockIdx.x];
  const int64_t beg = rp[s], end = rp[s + 1];
  const float ds = (float)(end - beg);
  if (threadIdx.x == 0) {
    q0[s * B + j] = 1.0f / ds;
    y[s * B + j] = c0[blockIdx.x];
  }
  for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const int32_t v = ci[e];
    if (v >= na) continue;  // only an unvalidated asymmetric CSR lists an isolated row
    const float dv = (float)(rp[v + 1] - rp[v]);
    q1[(int64_t)v * B + j] = (float)(1.0 / ((double)ds * (double)dv));
    y[(int64_t)v * B + j] = c1[blockIdx.x] / ds;
  }
}

// y columns (relabelled rows) -> caller order, for the columns listed.  A CTA
// takes 32 caller rows: it copies their 32 y rows (B floats each, contiguous)
// into shared memory, then writes each listed column's 32 values coalesced.
template <typename OUT>
__global__ void output_columns_kernel(int64_t n, int64_t na, const int32_t* newid, const float* y, int B,
                                      const int* cols, int ncols, OUT* const* outs) {
  extern __shared__ __align__(16) float s_tile[];  // 32 x B
  __shared__ int64_t s_row[32];
  for (int64_t u0 = (int64_t)blockIdx.x * 32; u0 < n; u0 += (int64_t)gridDim.x * 32) {
    if (threadIdx.x < 32) {
      const int64_t u = u0 + threadIdx.x;
      s_row[threadIdx.x] = u < n ? (int64_t)newid[u] : -1;
    }
    __syncthreads();
    const int nvec = 32 * (B / 4);
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      const int r = v / (B / 4), c4 = v % (B / 4);
      const int64_t i = s_row[r];
      const float4 val = (i >= 0 && i < na) ? *reinterpret_cast<const float4*>(y + i * B + 4 * c4)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(s_tile + r * B + 4 * c4) = val;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t u = u0 + lane;
    for (int t = warp; t < ncols; t += nw)
      if (u < n) outs[t][u] = (OUT)s_tile[lane * B + cols[t]];
    __syncthreads();
  }
}

// Clenshaw's source term for every busy column j of the block:
// buf[s_j][j] += c_k^(j) / d_{s_j} (a B vector: b_k += c_k e_s, stored as B = b / d),
// or, with to_y, y[s_j][j] += c_0^(j).
__global__ void clenshaw_inject_kernel(float* buf, int ldb, const ColState* col, const ColParam* par,
                                       const int64_t* src, const float* inv_d, int B, int k, int to_y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B || !col[j].active) return;
  const float c = par[j].c[k];
  buf[src[j] * ldb + j] += to_y ? c : c * inv_d[j];
}

// ---- generalized propagation (gp_propagate): Z = f(D^-a A D^-b) X, a + b = 1,
// computed as Z = D^-a f(P) D^a X (Section "Generalizations", the theorem on
// generalized GP vectors), each feature a column of the block.

// x'(u) = d_u^a X[u][f0 + j] over the active rows (relabelled order) into buf,
// and the l1 norm of each column into colnorm.  A warp per row, lanes over
// the columns (nb <= 256: at most 8 per lane).
__global__ void prop_scale_kernel(int64_t na, int B, int nb, int F, int f0, const int32_t* order, const float* degf,
                                  const float* X, float a, float* buf, float* colnorm) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float part[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < na; r += nw) {
    const int64_t u = order[r];
    const float sc = a == 0.f ? 1.f : powf(degf[r], a);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = lane + 32 * i;
      if (j < nb) {
        const float v = sc * X[u * F + f0 + j];
        buf[r * B + j] = v;
        part[i] += fabsf(v);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (lane + 32 * i < nb && part[i] != 0.f) atomicAdd(&colnorm[lane + 32 * i], part[i]);
}

// r_0 = x' / ||x'||_1 (so ||r_0||_1 = 1), Q_0 = r_0 / d over buf, y = c_0 r_0.
__global__ void prop_init_kernel(int64_t na, int B, int nb, const float* degf, const float* colnorm, const float* c0,
                                 float* buf, float* y) {
  const int64_t total = na * (int64_t)nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / nb;
    const int j = (int)(t - r * nb);
    const float nrm = colnorm[j];
    const float x = nrm > 0.f ? buf[r * B + j] / nrm : 0.f;
    buf[r * B + j] = x / degf[r];
    y[r * B + j] = c0[j] * x;
  }
}

// Z[u][feat[t]] = d_u^-a ||x'||_1 y[newid[u]][cols[t]] for the active caller
// rows u (isolated rows are written by prop_isolated_kernel).
__global__ void prop_output_kernel(int64_t n, int64_t na, const int32_t* newid, const float* degf, float a,
                                   const float* y, int B, const int* cols, const int* feat, int ncols,
                                   const float* colnorm, int F, float* Z) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = newid[u];
    if (i >= na) continue;
    const float sc = a == 0.f ? 1.f : powf(degf[i], -a);
    for (int t = 0; t < ncols; ++t) Z[u * F + feat[t]] = sc * colnorm[cols[t]] * y[i * B + cols[t]];
  }
}

// Isolated nodes: D^-a A D^-b has a zero row and column there, so
// Z[u][f] = f(0) X[u][f].
__global__ void prop_isolated_kernel(int64_t n, int64_t na, const int32_t* newid, int F, float f0v, const float* X,
                                     float* Z) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * (int64_t)F;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = t / F;
    if (newid[u] >= na) Z[t] = f0v * X[t];
  }
}

int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename TG, typename TP, typename TO, int LC, bool CHECK>
void launch_spmm_k(const SpmmArgs& a, cudaStream_t st) {
  static const cudaError_t attr = cudaFuncSetAttribute(spmm_step_kernel<TG, TP, TO, LC, CHECK>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpmmSmem);
  GP_CUDA_TRY(attr);
  spmm_step_kernel<TG, TP, TO, LC, CHECK><<<device_sms(), kBatchThreads, kSpmmSmem, st>>>(a);
  GP_LAUNCHED();
}

template <typename TG, typename TP, typename TO, int LC>
void launch_spmm_lc(const SpmmArgs& a, cudaStream_t st) {
  if (a.check)
    launch_spmm_k<TG, TP, TO, LC, true>(a, st);
  else
    launch_spmm_k<TG, TP, TO, LC, false>(a, st);
}

// With 16-bit gathers a lane owns 16 columns (32 bytes per round) when
// B >= 16; FP32 gathers keep 8 columns per lane, so that a round stays 32
// bytes and the ring holds 8 rounds.
template <typename TG, typename TP, typename TO>
void launch_spmm(const SpmmArgs& a, cudaStream_t st) {
  if constexpr (sizeof(TG) == 2) {
    if (a.B >= 16) {
      launch_spmm_lc<TG, TP, TO, 16>(a, st);
      return;
    }
  }
  launch_spmm_lc<TG, TP, TO, 8>(a, st);
}

template <typename H>
void launch_stage(const SpmmArgs& a, int stage, cudaStream_t st) {
  switch (stage) {
    case 0: launch_spmm<float, float, float>(a, st); break;  // FP32
    case 1: launch_spmm<float, float, H>(a, st); break;      // first 16-bit write
    case 2: launch_spmm<H, float, H>(a, st); break;          // first 16-bit gather
    default: launch_spmm<H, H, H>(a, st); break;             // 16-bit
  }
}

}  // namespace

// ------------------------------------------------------------------ engine

double column_warm_tail(double warmup_tail, gp_dtype storage, double tol) {
  const double base = storage == GP_F16 ? 4.0 * warmup_tail : warmup_tail;
  return base * std::min(1.0, tol / 1e-4);
}

// The first step whose Q may be stored in 16 bits: the smallest k with
// W(k) = sum_{m>=0} (m + 1) |c_{k+1+m}| < warmup_tail.  A rounding error that
// the recurrence does not compensate propagates with the second-kind
// polynomials U_m(P) (the residual-propagation lemma of the generalized subset
// recurrence, with no compensation), and |U_m| <= m + 1 on [-1, 1], so an
// error made at step k reaches y weighted by W(k) rather than by the tail
// sum_{l>k} |c_l| (which let slowly decaying expansions, SSPPR alpha = 0.1,
// pass l1 = 1e-4 in 16-bit blocks).  kcap when no step qualifies.
int warm_step(const std::vector<double>& c, int kcap, double warmup_tail) {
  const int last = (int)c.size() - 1;
  for (int k = 0; k <= kcap && k < kMaxColK; ++k) {
    double w = 0.0;
    for (int l = k + 1; l <= last; ++l) w += (double)(l - k) * std::fabs(c[l]);
    if (w < warmup_tail) return k;
  }
  return std::min(kcap, kMaxColK - 1);
}

ColumnEngine::ColumnEngine(Graph& g, int B, gp_dtype storage, cudaStream_t st, int t_long, bool pure16)
    : g_(g), B_(B), bw_(B), storage_(storage), pure16_(pure16), st_(st) {
  if (B < 8 || B > 256 || (B & (B - 1)))
    throw Error{GP_EINVAL, "block width must be a power of two in [8, 256]"};
  if (t_long <= 0) t_long = g.cfg.t_heavy > 0 ? g.cfg.t_heavy - 1 : kBTileCap;
  t_long_ = std::max(1, std::min(t_long, kBTileCap));
  if (storage != GP_F32 && storage != GP_BF16 && storage != GP_F16)
    throw Error{GP_EINVAL, "storage must be GP_F32, GP_BF16 or GP_F16"};
  if (pure16 && storage == GP_F32) throw Error{GP_EINVAL, "a 16-bit engine needs GP_BF16 or GP_F16 storage"};
  kcap_ = std::min(g.cfg.k_max, kMaxColK - 2);
  const int64_t na = std::max<int64_t>(g.n_active, 1);
  Allocator& A = g.alloc;
  try {
    if (!pure16) {
      f_[0] = (float*)A.get(sizeof(float) * na * B);
      f_[1] = (float*)A.get(sizeof(float) * na * B);
    }
    if (storage != GP_F32) {
      h_[0] = A.get(2 * na * B);
      h_[1] = A.get(2 * na * B);
    }
    y_ = (float*)A.get(sizeof(float) * na * B);
    col_ = (ColState*)A.get(sizeof(ColState) * B);
    par_ = (ColParam*)A.get(sizeof(ColParam) * B);
    stat_ = (ColStat*)A.get(sizeof(ColStat) * B);
    norm_ = (float*)A.get(sizeof(float) * B);
    scratch_ = (int*)A.get(sizeof(int) * 4 * B + sizeof(int64_t) * B + sizeof(float) * 2 * B + 16);
    outs_ = A.get(sizeof(void*) * B);
    // tiles of the pass: chunks of the long rows (more than t_long_ entries;
    // the relabelled rows are in descending degree, so they come first), then
    // runs of equal-degree rows
    const std::vector<int64_t>& rp = g.h_rp_relabelled;
    const int EG = 32 / (B / 8);
    std::vector<int4> tiles;
    std::vector<int> poff(1, 0);
    std::vector<int64_t> ldeg;
    int64_t row = 0;
    while (row < g.n_active && rp[row + 1] - rp[row] > t_long_) {
      const int64_t deg = rp[row + 1] - rp[row];
      const int64_t np = (deg + kBTileCap - 1) / kBTileCap;
      if (np > 0x7fff) throw Error{GP_EINVAL, "a row has too many entries for the batched schedule"};
      for (int64_t p = 0; p < np; ++p)
        tiles.push_back(make_btile(row, rp[row] + p * kBTileCap, 2, (int)p,
                                   (int)std::min<int64_t>(kBTileCap, deg - p * kBTileCap)));
      poff.push_back(poff.back() + (int)np);
      ldeg.push_back(deg);
      ++row;
    }
    nlong_ = (int)row;
    while (row < g.n_active) {
      const int64_t d = rp[row + 1] - rp[row];
      int64_t run = row + 1;
      while (run < g.n_active && rp[run + 1] - rp[run] == d) ++run;
      int64_t cap = std::max<int64_t>(1, std::min<int64_t>(kBTileCost / (d + 3), kBTileCap / d));
      if (cap >= EG) cap -= cap % EG;  // whole rounds of the lane groups
      for (; row < run;) {
        const int64_t nr = std::min(cap, run - row);
        tiles.push_back(make_btile(row, rp[row], nr >= EG ? 0 : 1, (int)nr, (int)d));
        row += nr;
      }
    }
    ntiles_ = (int64_t)tiles.size();
    tiles_ = (int4*)A.get(sizeof(int4) * std::max<size_t>(tiles.size(), 1));
    poff_ = (int*)A.get(sizeof(int) * poff.size());
    ldeg_ = (int64_t*)A.get(sizeof(int64_t) * std::max<size_t>(ldeg.size(), 1));
    part_ = (float*)A.get(sizeof(float) * (size_t)std::max(poff.back(), 1) * B);
    cnt_ = (int*)A.get(sizeof(int) * std::max(nlong_, 1));
    zero_ = A.get(sizeof(float) * B);
    tile_ctr_ = (int*)A.get(sizeof(int) * 4);
    if (!tiles.empty())
      GP_CUDA_TRY(cudaMemcpyAsync(tiles_, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, st_));
    GP_CUDA_TRY(cudaMemcpyAsync(poff_, poff.data(), sizeof(int) * poff.size(), cudaMemcpyHostToDevice, st_));
    if (!ldeg.empty())
      GP_CUDA_TRY(cudaMemcpyAsync(ldeg_, ldeg.data(), sizeof(int64_t) * ldeg.size(), cudaMemcpyHostToDevice, st_));
    GP_CUDA_TRY(cudaMemsetAsync(cnt_, 0, sizeof(int) * std::max(nlong_, 1), st_));
    GP_CUDA_TRY(cudaMemsetAsync(zero_, 0, sizeof(float) * B, st_));
    GP_CUDA_TRY(cudaMemsetAsync(col_, 0, sizeof(ColState) * B, st_));
    GP_CUDA_TRY(cudaMemsetAsync(par_, 0, sizeof(ColParam) * B, st_));
    GP_CUDA_TRY(cudaMemsetAsync(stat_, 0, sizeof(ColStat) * B, st_));
    GP_CUDA_TRY(cudaMemsetAsync(norm_, 0, sizeof(float) * B, st_));
    GP_CUDA_TRY(cudaStreamSynchronize(st_));
  } catch (...) {
    release();
    throw;
  }
  slots_.assign(B, Slot{});
}

ColumnEngine::~ColumnEngine() { release(); }

void ColumnEngine::release() {
  if (st_) cudaStreamSynchronize(st_);
  for (cudaEvent_t e : events_) cudaEventDestroy(e);
  events_.clear();
  Allocator& A = g_.alloc;
  for (void* p : {(void*)f_[0], (void*)f_[1], h_[0], h_[1], (void*)y_, (void*)col_, (void*)par_, (void*)stat_,
                  (void*)norm_, (void*)scratch_, outs_, stage_, (void*)tiles_, (void*)poff_, (void*)ldeg_,
                  (void*)part_, (void*)cnt_, zero_, (void*)tile_ctr_, (void*)degf_})
    A.put(p);
  stat_ = nullptr;
  stage_ = nullptr;
  f_[0] = f_[1] = nullptr;
  h_[0] = h_[1] = nullptr;
  y_ = nullptr;
  col_ = nullptr;
  par_ = nullptr;
  norm_ = nullptr;
  scratch_ = nullptr;
  outs_ = nullptr;
  tiles_ = nullptr;
  ldeg_ = nullptr;
  zero_ = nullptr;
  tile_ctr_ = nullptr;
  degf_ = nullptr;
  poff_ = nullptr;
  part_ = nullptr;
  cnt_ = nullptr;
}

size_t ColumnEngine::bytes_per_column(const Graph& g, gp_dtype storage, bool pure16) {
  const size_t na = (size_t)std::max<int64_t>(g.n_active, 1);
  if (pure16) return na * (2 + 2 + 4);
  return na * (4 + 4 + 4 + (storage == GP_F32 ? 0 : 4));
}

int ColumnEngine::free_slots() const {
  int f = 0;
  for (const Slot& s : slots_) f += !s.busy;
  return f;
}

// Admit requests into free slots.  Returns the slots used (one per request, -1
// for an isolated source, which is answered at once).
std::vector<int> ColumnEngine::admit(const std::vector<gp_request>& reqs, std::vector<uint64_t> tags) {
  if (pure16_) throw Error{GP_EINVAL, "a 16-bit engine takes columns only from an FP32 engine"};
  std::vector<int> slots(reqs.size(), -1);
  std::vector<int> cols;
  std::vector<int64_t> srcs;
  std::vector<float> c0, c1;
  std::vector<ColParam> params;
  std::vector<int> tag_of_param;
  const int kcap = kcap_;
  for (size_t i = 0; i < reqs.size(); ++i) {
    const gp_request& r = reqs[i];
    const int64_t deg = g_.h_deg[r.source];
    if (deg == 0) {
      // P e_s = 0: y = f(0) e_s, written directly (no slot)
      const double f0 = r.function == GP_FN_PPR ? r.param : std::exp(-r.param);
      write_point(r, f0);
      continue;
    }
    int slot = -1;
    for (int j = 0; j < B_; ++j)
      if (!slots_[j].busy) {
        slot = j;
        break;
      }
    if (slot < 0) throw Error{GP_EBUSY, "no free column"};
    slots_[slot].busy = true;
    slots_[slot].req = r;
    slots_[slot].tag = i < tags.size() ? tags[i] : 0;
    slots_[slot].t_admit = std::chrono::steady_clock::now();
    slots[i] = slot;
    std::vector<double> c, tail;
    cheb_coefficients(r.function, r.param, kcap, c, tail);
    ColParam p;
    std::memset(&p, 0, sizeof(p));
    slots_[slot].tails.assign(tail.begin(), tail.end());
    slots_[slot].tails.resize(kMaxColK, 0.0);
    for (int k = 0; k <= kcap && k < kMaxColK; ++k) {
      p.c[k] = (float)c[k];
      p.tail[k] = (float)tail[k];
    }
    p.tol = r.k_rule == GP_K_TAIL ? (float)(r.l1_tol / kCMargin) : -1.0f;
    p.kstop = r.k_rule == GP_K_FIXED ? r.k_fixed
              : r.k_rule == GP_K_PAPER ? std::min(kcap - 1, paper_k(r.function, r.param, r.l1_tol))
                                       : 0;
    p.warm = warm_step(c, kcap, column_warm_tail(g_.cfg.warmup_tail, storage_, r.l1_tol));
    params.push_back(p);
    cols.push_back(slot);
    srcs.push_back(g_.h_newid[r.source]);
    c0.push_back((float)c[0]);
    c1.push_back((float)c[1]);
  }
  if (cols.empty()) return slots;
  const int nc = (int)cols.size();
  // upload parameters and init state of the new columns
  int* d_cols = scratch_;
  int64_t* d_src = reinterpret_cast<int64_t*>(scratch_ + 4 * B_);
  float* d_c0 = reinterpret_cast<float*>(d_src + B_);
  float* d_c1 = d_c0 + B_;
  GP_CUDA_TRY(cudaMemcpyAsync(d_cols, cols.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(d_src, srcs.data(), sizeof(int64_t) * nc, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(d_c0, c0.data(), sizeof(float) * nc, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(d_c1, c1.data(), sizeof(float) * nc, cudaMemcpyHostToDevice, st_));
  const ColState cs_on{1, 0.f};
  const ColStat st0{1, 0, 0, 1.0f};  // r_0, r_1 set by the init; ||r_0||_1 = ||r_1||_1 = 1
  for (int t = 0; t < nc; ++t) {
    GP_CUDA_TRY(cudaMemcpyAsync(par_ + cols[t], &params[t], sizeof(ColParam), cudaMemcpyHostToDevice, st_));
    GP_CUDA_TRY(cudaMemcpyAsync(col_ + cols[t], &cs_on, sizeof(ColState), cudaMemcpyHostToDevice, st_));
    GP_CUDA_TRY(cudaMemcpyAsync(stat_ + cols[t], &st0, sizeof(ColStat), cudaMemcpyHostToDevice, st_));
  }
  GP_CUDA_TRY(cudaStreamSynchronize(st_));  // host vectors above are pageable and local
  const int sms = device_sms();
  const size_t cells = (size_t)std::max<int64_t>(g_.n_active, 1) * B_;
  if (nc == B_) {  // a whole new block: clear the buffers outright
    GP_CUDA_TRY(cudaMemsetAsync(f_[0], 0, sizeof(float) * cells, st_));
    GP_CUDA_TRY(cudaMemsetAsync(f_[1], 0, sizeof(float) * cells, st_));
    GP_CUDA_TRY(cudaMemsetAsync(y_, 0, sizeof(float) * cells, st_));
    if (h_[0]) {
      GP_CUDA_TRY(cudaMemsetAsync(h_[0], 0, 2 * cells, st_));
      GP_CUDA_TRY(cudaMemsetAsync(h_[1], 0, 2 * cells, st_));
    }
  } else {
    reset_columns_kernel<<<sms * 8, 256, 0, st_>>>(g_.n_active, B_, d_cols, nc, f_[0], f_[1], (uint16_t*)h_[0],
                                                    (uint16_t*)h_[1], y_);
    GP_LAUNCHED();
  }
  // Q_1 goes to the buffer the next pass gathers (pass_ & 1), Q_0 to the other.
  float* q1 = f_[pass_ & 1];
  float* q0 = f_[(pass_ + 1) & 1];
  if (g_.rp64)
    init_columns_kernel<int64_t><<<nc, 256, 0, st_>>>(g_.rp, g_.ci, g_.n_active, B_, d_cols, d_src, d_c0, d_c1, q0, q1, y_);
  else
    init_columns_kernel<int32_t><<<nc, 256, 0, st_>>>(g_.rp, g_.ci, g_.n_active, B_, d_cols, d_src, d_c0, d_c1, q0, q1, y_);
  GP_LAUNCHED();
  active_ += nc;
  for (const ColParam& p : params) warm_ = std::max(warm_, p.warm);
  return slots;
}

// One fused pass over all active columns (control kernel + SpMM step).  The
// pass covers the smallest power-of-two prefix of the columns (at least 8)
// that holds every busy column, so a lightly loaded engine runs narrow passes.
void ColumnEngine::pass(int force_stage) {
  int last = -1;
  for (int j = 0; j < B_; ++j)
    if (slots_[j].busy) last = j;
  int w = 8;
  while (w < last + 1) w <<= 1;
  bw_ = std::min(w, B_);
  control_kernel<<<(B_ + 127) / 128, 128, 0, st_>>>(col_, par_, stat_, norm_, B_, kcap_, tile_ctr_, -1);
  GP_LAUNCHED();
  // storage stage of this pass: FP32 until every column's warm-up has passed
  int stage = 0;
  if (storage_ != GP_F32) {
    if (h_pass_ < 0 && pass_16_ok()) h_pass_ = pass_;
    if (h_pass_ >= 0) stage = std::min(3, pass_ - h_pass_ + 1);
  }
  if (force_stage >= 0) stage = storage_ == GP_F32 ? 0 : force_stage;  // timing only (autotune)
  if (pure16_) stage = 3;
  SpmmArgs a;
  a.tiles = tiles_;
  a.ntiles = ntiles_;
  a.ci = g_.ci;
  const int cur = pass_ & 1, nxt = (pass_ + 1) & 1;
  a.qcur = stage >= 2 ? h_[cur] : (const void*)f_[cur];
  a.qprev = stage >= 3 ? h_[nxt] : (const void*)f_[nxt];
  a.qnext = stage >= 1 ? h_[nxt] : (void*)f_[nxt];
  a.y = y_;
  a.col = col_;
  a.norm = norm_;
  a.poff = poff_;
  a.ldeg = ldeg_;
  a.part = part_;
  a.cnt = cnt_;
  a.zero = zero_;
  a.na = g_.n_active;
  a.B = bw_;
  a.ldb = B_;
  a.check = g_.ci_beyond_active ? 1 : 0;
  a.tile_ctr = tile_ctr_;
  a.mode = kModeForward;
  const bool prof = profile_;
  if (prof) {
    while (events_.size() < prof_marks_.size() * 2 + 2) {
      cudaEvent_t e;
      GP_CUDA_TRY(cudaEventCreate(&e));
      events_.push_back(e);
    }
    GP_CUDA_TRY(cudaEventRecord(events_[prof_marks_.size() * 2], st_));
  }
  if (storage_ == GP_F16) launch_stage<__half>(a, stage, st_);
  else launch_stage<__nv_bfloat16>(a, stage, st_);
  if (prof) {
    GP_CUDA_TRY(cudaEventRecord(events_[prof_marks_.size() * 2 + 1], st_));
    // algorithmic bytes: col_idx once, Q_k gathered once, Q_{k-1} read,
    // Q_{k+1} written, y read and written, over the pass's columns
    const int sg = stage >= 2 ? 2 : 4, sp = stage >= 3 ? 2 : 4, so = stage >= 1 ? 2 : 4;
    prof_marks_.push_back(4.0 * (double)g_.nnz + (double)g_.n_active * bw_ * (sg + sp + so + 8));
  }
  ++pass_;
  ++passes_total_;
}

// The 16-bit phase may start once every column present has passed its
// warm-up steps (columns admitted later would have to warm up in 16 bits, so
// 16-bit storage is used only by engines that admit all columns at once).
bool ColumnEngine::pass_16_ok() const { return pass_ >= warm_; }

// Columns whose stop rule has fired: read their state, write their outputs,
// and free their slots.  Returns the finished slots.
std::vector<ColumnEngine::Finished> ColumnEngine::collect(bool force_all) {
  std::vector<Finished> fin;
  std::vector<ColStat> stat(B_);
  GP_CUDA_TRY(cudaMemcpyAsync(stat.data(), stat_, sizeof(ColStat) * B_, cudaMemcpyDeviceToHost, st_));
  GP_CUDA_TRY(cudaStreamSynchronize(st_));
  std::vector<int> cols;
  for (int j = 0; j < B_; ++j)
    if (slots_[j].busy && (stat[j].done || force_all)) cols.push_back(j);
  if (cols.empty()) return fin;
  write_outputs(cols);
  for (int j : cols) {
    Finished f;
    f.slot = j;
    f.tag = slots_[j].tag;
    f.req = slots_[j].req;
    f.K = stat[j].done ? stat[j].K : stat[j].k;
    f.C = stat[j].C;
    f.tail_bound = kCMargin * (double)slots_[j].tails[std::min(f.K, kMaxColK - 1)] * stat[j].C;
    f.t_admit = slots_[j].t_admit;
    f.k16_from = h_pass_ >= 0 ? h_pass_ : f.K + 1;
    fin.push_back(f);
    slots_[j].busy = false;
    const ColStat zero{0, 0, 0, 0.f};
    GP_CUDA_TRY(cudaMemcpyAsync(stat_ + j, &zero, sizeof(ColStat), cudaMemcpyHostToDevice, st_));
    ColState cs{0, 0.f};
    GP_CUDA_TRY(cudaMemcpyAsync(col_ + j, &cs, sizeof(ColState), cudaMemcpyHostToDevice, st_));
    --active_;
  }
  GP_CUDA_TRY(cudaStreamSynchronize(st_));
  return fin;
}

void ColumnEngine::write_outputs(const std::vector<int>& cols) {
  if (prop_.on) {
    std::vector<int> feat(cols.size());
    for (size_t t = 0; t < cols.size(); ++t) feat[t] = (int)slots_[cols[t]].tag;
    int* d_cols = scratch_ + 2 * B_;
    int* d_feat = scratch_;
    GP_CUDA_TRY(cudaMemcpyAsync(d_cols, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice, st_));
    GP_CUDA_TRY(cudaMemcpyAsync(d_feat, feat.data(), sizeof(int) * feat.size(), cudaMemcpyHostToDevice, st_));
    prop_output_kernel<<<device_sms() * 8, 256, 0, st_>>>(g_.n, g_.n_active, g_.newid, prop_.degf, (float)prop_.a, y_,
                                                          B_, d_cols, d_feat, (int)cols.size(), prop_.colnorm,
                                                          prop_.F, prop_.Z);
    GP_LAUNCHED();
    GP_CUDA_TRY(cudaStreamSynchronize(st_));  // the host vectors are local
    return;
  }
  // one launch per output type and location; host outputs go through staging
  std::vector<int> dcol64, dcol32;
  std::vector<void*> p64, p32;
  std::vector<std::pair<int, void*>> host;
  for (int j : cols) {
    const gp_request& r = slots_[j].req;
    if (!r.y_on_device) {
      host.push_back({j, r.y_out});
      continue;
    }
    if (r.out_dtype == GP_F64) {
      dcol64.push_back(j);
      p64.push_back(r.y_out);
    } else {
      dcol32.push_back(j);
      p32.push_back(r.y_out);
    }
  }
  auto launch = [&](const std::vector<int>& cl, const std::vector<void*>& ptrs, bool f64) {
    if (cl.empty()) return;
    int* d_cols = scratch_ + 2 * B_;
    GP_CUDA_TRY(cudaMemcpyAsync(d_cols, cl.data(), sizeof(int) * cl.size(), cudaMemcpyHostToDevice, st_));
    GP_CUDA_TRY(cudaMemcpyAsync(outs_, ptrs.data(), sizeof(void*) * ptrs.size(), cudaMemcpyHostToDevice, st_));
    const int grid = device_sms() * 4;
    const size_t smem = sizeof(float) * 32 * B_;
    if (f64)
      output_columns_kernel<double><<<grid, 256, smem, st_>>>(g_.n, g_.n_active, g_.newid, y_, B_, d_cols,
                                                              (int)cl.size(), (double* const*)outs_);
    else
      output_columns_kernel<float><<<grid, 256, smem, st_>>>(g_.n, g_.n_active, g_.newid, y_, B_, d_cols,
                                                             (int)cl.size(), (float* const*)outs_);
    GP_LAUNCHED();
    GP_CUDA_TRY(cudaStreamSynchronize(st_));
  };
  launch(dcol64, p64, true);
  launch(dcol32, p32, false);
  if (!host.empty()) {
    if (!stage_) stage_ = g_.alloc.get(sizeof(double) * g_.n);
    for (auto& h : host) {
      const gp_request& r = slots_[h.first].req;
      std::vector<int> one{h.first};
      std::vector<void*> ptr{stage_};
      launch(one, ptr, r.out_dtype == GP_F64);
      const size_t esz = r.out_dtype == GP_F64 ? 8 : 4;
      GP_CUDA_TRY(cudaMemcpyAsync(h.second, stage_, esz * g_.n, cudaMemcpyDeviceToHost, st_));
      GP_CUDA_TRY(cudaStreamSynchronize(st_));
    }
  }
}

void ColumnEngine::write_point(const gp_request& r, double f0) {
  const size_t esz = r.out_dtype == GP_F64 ? 8 : 4;
  std::vector<unsigned char> host(esz * g_.n, 0);
  if (r.out_dtype == GP_F64)
    reinterpret_cast<double*>(host.data())[r.source] = f0;
  else
    reinterpret_cast<float*>(host.data())[r.source] = (float)f0;
  GP_CUDA_TRY(cudaMemcpyAsync(r.y_out, host.data(), host.size(),
                              r.y_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st_));
  GP_CUDA_TRY(cudaStreamSynchronize(st_));
}

// ------------------------------------------------------------------ gp_batch

void run_batch(Graph& g, int count, const gp_request* reqs, gp_query_info* infos) {
  for (int i = 0; i < count; ++i) {
    const gp_request& r = reqs[i];
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
    if (r.k_rule == GP_K_FIXED)
      GP_REQUIRE(r.k_fixed >= 1 && r.k_fixed < g.cfg.k_max, "k_fixed must be in [1, k_max)");
  }
  if (count == 0) return;
  int B = g.cfg.block_width;
  if (B <= 0) {
    // the next power of two that holds the requests, within [8, 256]; with
    // cfg.autotune, no wider than the tuned width of this graph and storage
    B = std::min(256, std::max(8, (int)(1u << (32 - __builtin_clz((unsigned)std::max(count, 8) - 1)))));
  }
  // cfg.autotune: the tuned width (an upper bound when block_width is 0) and,
  // unless cfg.t_heavy sets it, the tuned chunk threshold
  int t_long = 0;
  if (g.cfg.autotune) {
    const TunedBlock tb = tune_block(g, g.cfg.storage, {});
    if (g.cfg.block_width <= 0) B = std::min(B, tb.B);
    if (g.cfg.t_heavy <= 0) t_long = tb.t_long;
  }
  BatchCache* bc = static_cast<BatchCache*>(g.batch);
  if (!bc) {
    bc = new BatchCache();
    g.batch = bc;
  }
  if (!bc->eng || bc->B != B || bc->storage != g.cfg.storage || bc->t_long != t_long) {
    bc->eng.reset();
    bc->eng.reset(new ColumnEngine(g, B, g.cfg.storage, g.stream, t_long));
    bc->B = B;
    bc->t_long = t_long;
    bc->storage = g.cfg.storage;
  }
  ColumnEngine& eng = *bc->eng;
  eng.restart();
  eng.set_profile(g.profiling);
  auto t0 = std::chrono::steady_clock::now();
  for (int base = 0; base < count; base += B) {
    const int nb = std::min(B, count - base);
    std::vector<gp_request> block(reqs + base, reqs + base + nb);
    std::vector<uint64_t> tags(nb);
    for (int i = 0; i < nb; ++i) tags[i] = (uint64_t)(base + i);
    eng.restart();
    eng.admit(block, tags);
    // isolated sources were answered at admission
    for (int i = 0; i < nb; ++i)
      if (infos && g.h_deg[reqs[base + i].source] == 0) {
        infos[base + i].K = 0;
        infos[base + i].k16_from = 1;
        infos[base + i].tail_bound = 0.0;
        infos[base + i].max_r_l1 = 1.0;
        infos[base + i].ms = 0.0;
      }
    int since_check = 0;
    while (eng.active() > 0) {
      eng.pass();
      if (++since_check >= 4) {
        since_check = 0;
        for (const auto& f : eng.collect(false)) {
          if (infos) {
            gp_query_info& in = infos[f.tag];
            in.K = f.K;
            in.k16_from = f.k16_from;
            in.tail_bound = f.tail_bound;
            in.max_r_l1 = f.C;
            in.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
          }
        }
        while (eng.active() > 0 && eng.compact()) {
        }
      }
    }
    eng.flush_profile();
  }
}

void run_clenshaw(Graph& g, int count, const gp_request* reqs, gp_query_info* infos) {
  for (int i = 0; i < count; ++i) {
    const gp_request& r = reqs[i];
    GP_REQUIRE(r.function == GP_FN_PPR || r.function == GP_FN_HKPR, "function must be GP_FN_PPR or GP_FN_HKPR");
    GP_REQUIRE(r.source >= 0 && (int64_t)r.source < g.n, "source out of range");
    if (r.function == GP_FN_PPR)
      GP_REQUIRE(r.param > 0.0 && r.param < 1.0, "alpha must be in (0, 1)");
    else
      GP_REQUIRE(r.param > 0.0 && r.param <= 1e4, "t must be in (0, 1e4]");
    GP_REQUIRE(r.l1_tol > 0.0 && r.l1_tol < 1.0, "l1_tol must be in (0, 1)");
    GP_REQUIRE(r.out_dtype == GP_F64 || r.out_dtype == GP_F32, "out_dtype must be GP_F64 or GP_F32");
    GP_REQUIRE(r.y_out != nullptr, "y_out is NULL");
    GP_REQUIRE(r.k_rule == GP_K_FIXED || r.k_rule == GP_K_PAPER,
               "Clenshaw's form needs K up front: k_rule must be GP_K_FIXED or GP_K_PAPER");
    if (r.k_rule == GP_K_FIXED)
      GP_REQUIRE(r.k_fixed >= 1 && r.k_fixed <= kMaxColK - 2, "k_fixed must be in [1, 126]");
  }
  if (count == 0) return;
  int B = g.cfg.block_width;
  if (B <= 0) B = std::min(256, std::max(8, (int)(1u << (32 - __builtin_clz((unsigned)std::max(count, 8) - 1)))));
  BatchCache* bc = static_cast<BatchCache*>(g.batch);
  if (!bc) {
    bc = new BatchCache();
    g.batch = bc;
  }
  if (!bc->eng || bc->B != B || bc->storage != g.cfg.storage) {
    bc->eng.reset();
    bc->eng.reset(new ColumnEngine(g, B, g.cfg.storage, g.stream));
    bc->B = B;
    bc->t_long = 0;
    bc->storage = g.cfg.storage;
  }
  ColumnEngine& eng = *bc->eng;
  auto t0 = std::chrono::steady_clock::now();
  for (int base = 0; base < count; base += B) {
    const int nb = std::min(B, count - base);
    std::vector<gp_request> block;
    std::vector<uint64_t> tags;
    for (int i = 0; i < nb; ++i) {
      const gp_request& r = reqs[base + i];
      if (g.h_deg[r.source] == 0) {
        // P e_s = 0: y = f(0) e_s (the same answer as the forward form)
        eng.restart();
        eng.admit({r}, {(uint64_t)(base + i)});
        if (infos) infos[base + i] = gp_query_info{0, 1, 0.0, 1.0, 0.0};
        continue;
      }
      block.push_back(r);
      tags.push_back((uint64_t)(base + i));
    }
    if (block.empty()) continue;
    eng.restart();
    for (const auto& f : eng.clenshaw(block, tags)) {
      if (infos) {
        gp_query_info& in = infos[f.tag];
        in.K = f.K;
        in.k16_from = f.k16_from;
        in.tail_bound = f.tail_bound;
        in.max_r_l1 = 0.0;  // not measured in the backward form
        in.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      }
    }
  }
}

void run_propagate(Graph& g, int function, double param, double a, int F, const float* X, float* Z, int on_device,
                   double tol, gp_query_info* infos) {
  GP_REQUIRE(function == GP_FN_PPR || function == GP_FN_HKPR, "function must be GP_FN_PPR or GP_FN_HKPR");
  if (function == GP_FN_PPR)
    GP_REQUIRE(param > 0.0 && param < 1.0, "alpha must be in (0, 1)");
  else
    GP_REQUIRE(param > 0.0 && param <= 1e4, "t must be in (0, 1e4]");
  GP_REQUIRE(a >= 0.0 && a <= 1.0, "a must be in [0, 1] (b = 1 - a)");
  GP_REQUIRE(F >= 1, "F must be >= 1");
  GP_REQUIRE(X && Z, "X or Z is NULL");
  GP_REQUIRE(tol > 0.0 && tol < 1.0, "l1_tol must be in (0, 1)");
  const size_t bytes = sizeof(float) * (size_t)g.n * F;
  Allocator& A = g.alloc;
  float* dX = const_cast<float*>(X);
  float* dZ = Z;
  if (!on_device) {
    dX = (float*)A.get(bytes);
    dZ = (float*)A.get(bytes);
  }
  try {
    cudaStream_t st = g.stream;
    if (!on_device) GP_CUDA_TRY(cudaMemcpyAsync(dX, X, bytes, cudaMemcpyHostToDevice, st));
    const double f0v = function == GP_FN_PPR ? param : std::exp(-param);
    prop_isolated_kernel<<<device_sms() * 8, 256, 0, st>>>(g.n, g.n_active, g.newid, F, (float)f0v, dX, dZ);
    GP_LAUNCHED();
    if (g.n_active > 0) {
      int B = g.cfg.block_width;
      if (B <= 0) B = std::min(256, std::max(8, (int)(1u << (32 - __builtin_clz((unsigned)std::max(F, 8) - 1)))));
      BatchCache* bc = static_cast<BatchCache*>(g.batch);
      if (!bc) {
        bc = new BatchCache();
        g.batch = bc;
      }
      if (!bc->eng || bc->B != B || bc->storage != g.cfg.storage) {
        bc->eng.reset();
        bc->eng.reset(new ColumnEngine(g, B, g.cfg.storage, st));
        bc->B = B;
        bc->t_long = 0;
        bc->storage = g.cfg.storage;
      }
      auto t0 = std::chrono::steady_clock::now();
      for (int f0 = 0; f0 < F; f0 += B) {
        const int nb = std::min(B, F - f0);
        for (const auto& f : bc->eng->propagate(dX, dZ, F, f0, nb, function, param, a, tol)) {
          if (infos) {
            gp_query_info& in = infos[f.tag];
            in.K = f.K;
            in.k16_from = f.k16_from;
            in.tail_bound = f.tail_bound;
            in.max_r_l1 = f.C;
            in.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
          }
        }
      }
    } else if (infos) {
      for (int f = 0; f < F; ++f) infos[f] = gp_query_info{0, 1, 0.0, 1.0, 0.0};
    }
    if (!on_device) GP_CUDA_TRY(cudaMemcpyAsync(Z, dZ, bytes, cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(g.stream);
    if (!on_device) {
      A.put(dX);
      A.put(dZ);
    }
    throw;
  }
  if (!on_device) {
    A.put(dX);
    A.put(dZ);
  }
}

// ------------------------------------------------------------------ autotune

namespace {
struct TuneKey {
  uint64_t digest;
  int storage, device;
  bool operator<(const TuneKey& o) const {
    return std::tie(digest, storage, device) < std::tie(o.digest, o.storage, o.device);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, TunedBlock> g_tune;

// Mean device time (ms) of `reps` passes of one engine at a forced storage stage.
double time_passes(ColumnEngine& eng, int stage, int reps, cudaStream_t st) {
  eng.pass(stage);  // warm-up (first launch of this instance)
  cudaEvent_t e0, e1;
  GP_CUDA_TRY(cudaEventCreate(&e0));
  GP_CUDA_TRY(cudaEventCreate(&e1));
  GP_CUDA_TRY(cudaEventRecord(e0, st));
  for (int i = 0; i < reps; ++i) eng.pass(stage);
  GP_CUDA_TRY(cudaEventRecord(e1, st));
  GP_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}
}  // namespace

// Time the column engine on this graph (every column a fixed-K query from a
// distinct non-isolated node, so nothing retires) at each candidate width,
// then, at the best width, at each candidate chunk threshold (rows with more
// entries than the threshold are summed as chunk tiles by several warps); keep
// the pair with the least device time per column and pass.  With 16-bit
// storage a block spends about its first half in the FP32 warm-up, so the cost
// is 0.45 of an FP32 pass plus 0.55 of a 16-bit one.
TunedBlock tune_block(Graph& g, gp_dtype storage, std::vector<int> widths) {
  int dev = 0;
  GP_CUDA_TRY(cudaGetDevice(&dev));
  const TuneKey key{g.digest, (int)storage, dev};
  const bool custom = !widths.empty();
  if (!custom) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
    widths = {8, 16, 32, 64, 128, 256};
  }
  for (int B : widths)
    GP_REQUIRE(B >= 8 && B <= 256 && (B & (B - 1)) == 0, "widths must be powers of two in [8, 256]");
  std::vector<int32_t> srcs;
  for (int64_t u = 0; u < g.n && (int)srcs.size() < 256; ++u)
    if (g.h_deg[u] > 0) srcs.push_back((int32_t)u);
  GP_REQUIRE(!srcs.empty(), "the graph has no edges");
  // device time per column and pass of one (width, threshold); < 0 if it does not fit
  auto trial = [&](int B, int t_long) -> double {
    size_t free_b = 0, total_b = 0;
    GP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    if ((size_t)B * ColumnEngine::bytes_per_column(g, storage) > free_b / 2) return -1.0;
    ColumnEngine eng(g, B, storage, g.stream, t_long);
    std::vector<gp_request> reqs(B);
    std::vector<uint64_t> tags(B);
    for (int j = 0; j < B; ++j) {
      gp_request r{};
      r.function = GP_FN_PPR;
      r.source = srcs[j % srcs.size()];
      r.param = 0.2;
      r.l1_tol = 1e-6;
      r.k_rule = GP_K_FIXED;
      r.k_fixed = g.cfg.k_max - 1;  // never retires while timed
      r.out_dtype = GP_F64;
      r.y_on_device = 1;
      r.y_out = nullptr;  // never collected
      reqs[j] = r;
      tags[j] = (uint64_t)j;
    }
    eng.restart();
    eng.admit(reqs, tags);
    const double t32 = time_passes(eng, 0, 2, g.stream);
    const double ms = storage == GP_F32 ? t32 : 0.45 * t32 + 0.55 * time_passes(eng, 3, 2, g.stream);
    return 1000.0 * ms / B;
  };
  TunedBlock best{0, kBTileCap, 0.0};
  for (int B : widths) {
    const double us = trial(B, kBTileCap);
    if (us >= 0.0 && (best.B == 0 || us < best.us)) best = TunedBlock{B, kBTileCap, us};
  }
  GP_REQUIRE(best.B > 0, "no candidate width fits in device memory");
  for (int t : {64, 128, 256}) {
    const double us = trial(best.B, t);
    if (us >= 0.0 && us < best.us) best = TunedBlock{best.B, t, us};
  }
  if (!custom) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  return best;
}

void free_batch_work(Graph& g) {
  BatchCache* bc = static_cast<BatchCache*>(g.batch);
  delete bc;
  g.batch = nullptr;
}

// Halve the pass width once at most half of it is busy: the busy columns move
// to the front of every row (with their state), so later passes gather and
// update only that prefix.  Only between passes; columns admitted later take
// the lowest free slots.
bool ColumnEngine::compact() {
  const int nb = bw_ / 2;
  if (nb < 8) return false;
  std::vector<int> perm;
  for (int j = 0; j < bw_; ++j)
    if (slots_[j].busy) perm.push_back(j);
  if ((int)perm.size() > nb) return false;
  for (int j = 0; j < bw_ && (int)perm.size() < nb; ++j)
    if (!slots_[j].busy) perm.push_back(j);
  int* d_perm = scratch_ + 2 * B_;
  GP_CUDA_TRY(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st_));
  permute_columns_kernel<<<device_sms() * 8, 256, 0, st_>>>(g_.n_active, B_, d_perm, nb, f_[0], f_[1],
                                                            (uint16_t*)h_[0], (uint16_t*)h_[1], y_);
  GP_LAUNCHED();
  // per-column state: through the host (a few hundred KB)
  std::vector<ColState> cs(B_), cs2(B_);
  std::vector<ColParam> cp(B_), cp2(B_);
  std::vector<ColStat> st(B_), st2(B_);
  std::vector<float> nm(B_), nm2(B_);
  GP_CUDA_TRY(cudaMemcpyAsync(cs.data(), col_, sizeof(ColState) * B_, cudaMemcpyDeviceToHost, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(cp.data(), par_, sizeof(ColParam) * B_, cudaMemcpyDeviceToHost, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(st.data(), stat_, sizeof(ColStat) * B_, cudaMemcpyDeviceToHost, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(nm.data(), norm_, sizeof(float) * B_, cudaMemcpyDeviceToHost, st_));
  GP_CUDA_TRY(cudaStreamSynchronize(st_));
  std::vector<Slot> sl(B_);
  for (int j = 0; j < B_; ++j) {
    cs2[j] = ColState{0, 0.f};
    std::memset(&cp2[j], 0, sizeof(ColParam));
    st2[j] = ColStat{0, 0, 0, 0.f};
    nm2[j] = 0.f;
  }
  for (int j = 0; j < nb; ++j) {
    const int o = perm[j];
    cs2[j] = cs[o];
    cp2[j] = cp[o];
    st2[j] = st[o];
    nm2[j] = nm[o];
    sl[j] = slots_[o];
  }
  GP_CUDA_TRY(cudaMemcpyAsync(col_, cs2.data(), sizeof(ColState) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(par_, cp2.data(), sizeof(ColParam) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(stat_, st2.data(), sizeof(ColStat) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(norm_, nm2.data(), sizeof(float) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaStreamSynchronize(st_));  // the host vectors are local
  slots_.swap(sl);
  bw_ = nb;
  return true;
}

// Add the timed passes to the graph's profile counters (gp_profile_read).
void ColumnEngine::flush_profile() {
  if (prof_marks_.empty()) return;
  GP_CUDA_TRY(cudaStreamSynchronize(st_));
  for (size_t i = 0; i < prof_marks_.size(); ++i) {
    float ms = 0.f;
    GP_CUDA_TRY(cudaEventElapsedTime(&ms, events_[2 * i], events_[2 * i + 1]));
    g_.prof_ms += ms;
    g_.prof_launches += 1;
    g_.prof_bytes += prof_marks_[i];
  }
  prof_marks_.clear();
}

// Clenshaw's backward form of the same truncated sum (Lemma 1), for up to B
// queries with K fixed up front: b_{K+1} = b_{K+2} = 0,
// b_k = c_k e_s + 2 P b_{k+1} - b_{k+2} for k = K .. 1, and
// y = c_0 e_s + P b_1 - b_2.  Each step is one fused pass over the FP32 pair
// (B_k = D^-1 b_k written over B_{k+2}); no pass touches y but the last, and
// no norm or stop rule is needed.  Columns with K_j below the block's largest
// K take c_k = 0 above K_j, so their b stay zero until step K_j.
std::vector<ColumnEngine::Finished> ColumnEngine::clenshaw(const std::vector<gp_request>& reqs_in,
                                                           const std::vector<uint64_t>& tags_in) {
  const int nb = (int)reqs_in.size();
  GP_REQUIRE(nb >= 1 && nb <= B_, "a Clenshaw block holds 1 .. B queries");
  // columns in descending K: at backward step k the started columns (K_j >= k)
  // are a prefix, and the step's pass covers only that prefix
  auto k_of = [&](const gp_request& r) {
    const int K = r.k_rule == GP_K_FIXED ? r.k_fixed : paper_k(r.function, r.param, r.l1_tol);
    return std::max(1, std::min(K, kMaxColK - 2));
  };
  std::vector<int> order(nb);
  for (int j = 0; j < nb; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return k_of(reqs_in[x]) > k_of(reqs_in[y]); });
  std::vector<gp_request> reqs(nb);
  std::vector<uint64_t> tags(nb);
  std::vector<int> kcol(nb);
  for (int j = 0; j < nb; ++j) {
    reqs[j] = reqs_in[order[j]];
    tags[j] = tags_in[order[j]];
    kcol[j] = k_of(reqs[j]);
  }
  std::vector<ColState> cs(B_, ColState{0, 0.f});
  std::vector<ColParam> par(B_);
  std::vector<ColStat> st(B_, ColStat{0, 0, 0, 0.f});
  std::vector<int64_t> src(B_, 0);
  std::vector<float> invd(B_, 0.f);
  int kmax = 1;
  for (int j = 0; j < nb; ++j) {
    const gp_request& r = reqs[j];
    const int K = kcol[j];
    std::vector<double> c, tail;
    cheb_coefficients(r.function, r.param, K, c, tail);
    std::memset(&par[j], 0, sizeof(ColParam));
    for (int k = 0; k <= K; ++k) par[j].c[k] = (float)c[k];
    slots_[j].busy = true;
    slots_[j].req = r;
    slots_[j].tag = tags[j];
    slots_[j].t_admit = std::chrono::steady_clock::now();
    slots_[j].tails.assign(kMaxColK, 0.0);
    slots_[j].tails[K] = tail[K];
    cs[j] = ColState{1, 0.f};
    st[j] = ColStat{K, K, 1, 0.f};
    src[j] = g_.h_newid[r.source];
    invd[j] = 1.0f / (float)g_.h_deg[r.source];
    kmax = std::max(kmax, K);
  }
  int64_t* d_src = reinterpret_cast<int64_t*>(scratch_ + 4 * B_);
  float* d_invd = reinterpret_cast<float*>(d_src + B_);
  GP_CUDA_TRY(cudaMemcpyAsync(col_, cs.data(), sizeof(ColState) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(par_, par.data(), sizeof(ColParam) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(stat_, st.data(), sizeof(ColStat) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(d_src, src.data(), sizeof(int64_t) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(d_invd, invd.data(), sizeof(float) * B_, cudaMemcpyHostToDevice, st_));
  const size_t cells = (size_t)std::max<int64_t>(g_.n_active, 1) * B_;
  GP_CUDA_TRY(cudaMemsetAsync(f_[0], 0, sizeof(float) * cells, st_));
  GP_CUDA_TRY(cudaMemsetAsync(f_[1], 0, sizeof(float) * cells, st_));
  GP_CUDA_TRY(cudaMemsetAsync(y_, 0, sizeof(float) * cells, st_));
  auto width_for = [&](int k) {  // the prefix of columns with K_j >= k
    int cnt = 0;
    while (cnt < nb && kcol[cnt] >= k) ++cnt;
    int w = 8;
    while (w < cnt) w <<= 1;
    return std::min(w, B_);
  };
  const int iblk = (B_ + 127) / 128;
  auto inject = [&](float* buf, int k, int to_y) {
    clenshaw_inject_kernel<<<iblk, 128, 0, st_>>>(buf, B_, col_, par_, d_src, d_invd, B_, k, to_y);
    GP_LAUNCHED();
  };
  auto step = [&](int mode, float* cur, float* prv) {
    GP_CUDA_TRY(cudaMemsetAsync(tile_ctr_, 0, sizeof(int), st_));
    SpmmArgs a;
    a.tiles = tiles_;
    a.ntiles = ntiles_;
    a.ci = g_.ci;
    a.qcur = cur;
    a.qprev = prv;
    a.qnext = prv;
    a.y = y_;
    a.col = col_;
    a.norm = norm_;
    a.poff = poff_;
    a.ldeg = ldeg_;
    a.part = part_;
    a.cnt = cnt_;
    a.zero = zero_;
    a.na = g_.n_active;
    a.B = bw_;
    a.ldb = B_;
    a.check = g_.ci_beyond_active ? 1 : 0;
    a.tile_ctr = tile_ctr_;
    a.mode = mode;
    launch_spmm<float, float, float>(a, st_);
  };
  int cur = 0, prv = 1;
  inject(f_[cur], kmax, 0);  // b_K = c_K e_s
  for (int k = kmax - 1; k >= 1; --k) {
    bw_ = width_for(k + 1);  // columns with a nonzero b_{k+1}
    step(kModeClenshaw, f_[cur], f_[prv]);  // b_k over b_{k+2}
    inject(f_[prv], k, 0);
    std::swap(cur, prv);
  }
  bw_ = width_for(1);
  step(kModeClenshawFinal, f_[cur], f_[prv]);  // y = P b_1 - b_2
  inject(y_, 0, 1);
  passes_total_ += kmax;
  std::vector<int> cols(nb);
  for (int j = 0; j < nb; ++j) cols[j] = j;
  write_outputs(cols);
  std::vector<Finished> fin;
  for (int j = 0; j < nb; ++j) {
    Finished f;
    f.slot = j;
    f.tag = slots_[j].tag;
    f.req = slots_[j].req;
    f.K = st[j].K;
    f.C = 0.f;
    f.tail_bound = slots_[j].tails[f.K];
    f.t_admit = slots_[j].t_admit;
    f.k16_from = f.K + 1;
    fin.push_back(f);
    slots_[j].busy = false;
  }
  const std::vector<ColState> off(B_, ColState{0, 0.f});
  GP_CUDA_TRY(cudaMemcpyAsync(col_, off.data(), sizeof(ColState) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaStreamSynchronize(st_));  // the host vectors are local
  return fin;
}

// One block of features f0 .. f0+nb-1 of a generalized propagation: start
// columns r_0 = D^a x / ||D^a x||_1 (relabelled), a first pass r_1 = P r_0,
// then forward passes with each column's own stop rule (relative to
// ||D^a x||_1), compaction as columns retire, and Z written per retired
// column.  X and Z are device arrays (n x F, row-major, caller order).
std::vector<ColumnEngine::Finished> ColumnEngine::propagate(const float* X, float* Z, int F, int f0, int nb,
                                                            int function, double param, double a, double tol) {
  GP_REQUIRE(nb >= 1 && nb <= B_, "a propagation block holds 1 .. B features");
  restart();
  const int64_t na = std::max<int64_t>(g_.n_active, 1);
  if (!degf_) {
    degf_ = (float*)g_.alloc.get(sizeof(float) * na);
    std::vector<float> d(na, 1.f);
    for (int64_t i = 0; i < g_.n_active; ++i) d[i] = (float)(g_.h_rp_relabelled[i + 1] - g_.h_rp_relabelled[i]);
    GP_CUDA_TRY(cudaMemcpyAsync(degf_, d.data(), sizeof(float) * na, cudaMemcpyHostToDevice, st_));
    GP_CUDA_TRY(cudaStreamSynchronize(st_));
  }
  float* colnorm = reinterpret_cast<float*>(reinterpret_cast<int64_t*>(scratch_ + 4 * B_) + B_);  // B floats
  float* c0dev = colnorm + B_;                                                                    // B floats
  prop_ = Prop{true, Z, F, a, degf_, colnorm};
  const size_t cells = (size_t)na * B_;
  GP_CUDA_TRY(cudaMemsetAsync(f_[0], 0, sizeof(float) * cells, st_));
  GP_CUDA_TRY(cudaMemsetAsync(f_[1], 0, sizeof(float) * cells, st_));
  GP_CUDA_TRY(cudaMemsetAsync(y_, 0, sizeof(float) * cells, st_));
  if (h_[0]) {
    GP_CUDA_TRY(cudaMemsetAsync(h_[0], 0, 2 * cells, st_));
    GP_CUDA_TRY(cudaMemsetAsync(h_[1], 0, 2 * cells, st_));
  }
  GP_CUDA_TRY(cudaMemsetAsync(colnorm, 0, sizeof(float) * B_, st_));
  prop_scale_kernel<<<device_sms() * 8, 256, 0, st_>>>(g_.n_active, B_, nb, F, f0, g_.order, degf_, X, (float)a,
                                                       f_[0], colnorm);
  GP_LAUNCHED();
  std::vector<double> c, tail;
  cheb_coefficients(function, param, kcap_, c, tail);
  ColParam p;
  std::memset(&p, 0, sizeof(p));
  for (int k = 0; k <= kcap_ && k < kMaxColK; ++k) {
    p.c[k] = (float)c[k];
    p.tail[k] = (float)tail[k];
  }
  p.tol = (float)(tol / kCMargin);
  p.kstop = 0;
  p.warm = warm_step(c, kcap_, column_warm_tail(g_.cfg.warmup_tail, storage_, tol));
  std::vector<ColState> cs(B_, ColState{0, 0.f});
  std::vector<ColParam> par(B_, p);
  std::vector<ColStat> st(B_, ColStat{0, 0, 0, 0.f});
  std::vector<float> c0(B_, (float)c[0]);
  for (int j = 0; j < nb; ++j) {
    cs[j] = ColState{1, (float)c[1]};
    st[j] = ColStat{1, 0, 0, 1.0f};  // ||r_0||_1 = 1 >= ||r_1||_1
    slots_[j].busy = true;
    std::memset(&slots_[j].req, 0, sizeof(gp_request));
    slots_[j].req.function = function;
    slots_[j].req.param = param;
    slots_[j].req.l1_tol = tol;
    slots_[j].tag = (uint64_t)(f0 + j);
    slots_[j].t_admit = std::chrono::steady_clock::now();
    slots_[j].tails.assign(tail.begin(), tail.end());
    slots_[j].tails.resize(kMaxColK, 0.0);
  }
  GP_CUDA_TRY(cudaMemcpyAsync(col_, cs.data(), sizeof(ColState) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(par_, par.data(), sizeof(ColParam) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(stat_, st.data(), sizeof(ColStat) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemcpyAsync(c0dev, c0.data(), sizeof(float) * B_, cudaMemcpyHostToDevice, st_));
  GP_CUDA_TRY(cudaMemsetAsync(norm_, 0, sizeof(float) * B_, st_));
  prop_init_kernel<<<device_sms() * 8, 256, 0, st_>>>(g_.n_active, B_, nb, degf_, colnorm, c0dev, f_[0], y_);
  GP_LAUNCHED();
  active_ = nb;
  warm_ = p.warm;
  // first pass: r_1 = P r_0 into f_[1], y += c_1 r_1
  {
    int w = 8;
    while (w < nb) w <<= 1;
    bw_ = std::min(w, B_);
    GP_CUDA_TRY(cudaMemsetAsync(tile_ctr_, 0, sizeof(int), st_));
    SpmmArgs a1;
    a1.tiles = tiles_;
    a1.ntiles = ntiles_;
    a1.ci = g_.ci;
    a1.qcur = f_[0];
    a1.qprev = f_[0];
    a1.qnext = f_[1];
    a1.y = y_;
    a1.col = col_;
    a1.norm = norm_;
    a1.poff = poff_;
    a1.ldeg = ldeg_;
    a1.part = part_;
    a1.cnt = cnt_;
    a1.zero = zero_;
    a1.na = g_.n_active;
    a1.B = bw_;
    a1.ldb = B_;
    a1.check = g_.ci_beyond_active ? 1 : 0;
    a1.tile_ctr = tile_ctr_;
    a1.mode = kModeFirst;
    launch_spmm<float, float, float>(a1, st_);
  }
  pass_ = 1;  // Q_1 in f_[1] (the buffer pass 1 gathers), Q_0 in f_[0]
  std::vector<Finished> fin;
  int since = 0;
  while (active_ > 0) {
    pass();
    if (++since >= 4) {
      since = 0;
      for (auto& f : collect(false)) fin.push_back(f);
      while (active_ > 0 && compact()) {
      }
    }
  }
  prop_.on = false;
  return fin;
}

ColumnEngine::View ColumnEngine::view() const {
  View v;
  v.f[0] = f_[0];
  v.f[1] = f_[1];
  v.h[0] = h_[0];
  v.h[1] = h_[1];
  v.y = y_;
  v.col = col_;
  v.par = par_;
  v.stat = stat_;
  v.norm = norm_;
  v.B = B_;
  v.pass = pass_;
  v.storage = storage_;
  v.pure16 = pure16_;
  return v;
}

void ColumnEngine::pass_device(const int* width_dev, const int* active_dev) {
  if (storage_ != GP_F32 && !pure16_) throw Error{GP_EINVAL, "device-width passes run FP32 or pure 16-bit engines"};
  control_kernel<<<(B_ + 127) / 128, 128, 0, st_>>>(col_, par_, stat_, norm_, B_, kcap_, tile_ctr_, 0);
  GP_LAUNCHED();
  SpmmArgs a;
  a.tiles = tiles_;
  a.ntiles = ntiles_;
  a.ci = g_.ci;
  const int cur = pass_ & 1, nxt = (pass_ + 1) & 1;
  a.qcur = pure16_ ? h_[cur] : (const void*)f_[cur];
  a.qprev = pure16_ ? h_[nxt] : (const void*)f_[nxt];
  a.qnext = pure16_ ? h_[nxt] : (void*)f_[nxt];
  a.y = y_;
  a.col = col_;
  a.norm = norm_;
  a.poff = poff_;
  a.ldeg = ldeg_;
  a.part = part_;
  a.cnt = cnt_;
  a.zero = zero_;
  a.na = g_.n_active;
  a.B = B_;  // the cap: it picks the columns per lane, so the device width is at least min_width()
  a.ldb = B_;
  a.check = g_.ci_beyond_active ? 1 : 0;
  a.tile_ctr = tile_ctr_;
  a.mode = kModeForward;
  a.Bdev = width_dev;
  a.active_dev = active_dev;
  if (storage_ == GP_F16) launch_stage<__half>(a, pure16_ ? 3 : 0, st_);
  else launch_stage<__nv_bfloat16>(a, pure16_ ? 3 : 0, st_);
  ++pass_;
  ++passes_total_;
}

void ColumnEngine::control_after() {
  control_kernel<<<(B_ + 127) / 128, 128, 0, st_>>>(col_, par_, stat_, norm_, B_, kcap_, tile_ctr_, 1);
  GP_LAUNCHED();
}

void ColumnEngine::restart() {
  GP_CUDA_TRY(cudaStreamSynchronize(st_));
  bw_ = B_;
  pass_ = 0;
  h_pass_ = -1;
  warm_ = 0;
}

}  // namespace gp
