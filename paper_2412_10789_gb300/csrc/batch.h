// Column engine: B queries as the columns of row-major blocks, advanced
// together by one fused SpMM pass (batch.cu).  Used by gp_batch and by the
// serving loop.
#pragma once

#include <chrono>
#include <memory>
#include <vector>

#include "gp_internal.h"

namespace gp {

constexpr int kMaxColK = 128;  // coefficient table length per column (K <= kMaxColK - 2)

// Per-column values the step kernel reads each pass.
struct ColState {
  int active;
  float coef;  // c_{k+1} of this pass
};

// Per-column constants, written at admission.
struct ColParam {
  float c[kMaxColK];     // Chebyshev coefficients c_0..
  float tail[kMaxColK];  // tail(k) = sum_{l>k} |c_l|
  float tol;             // l1 tolerance over kCMargin: stop at tail(k) * C <= tol (< 0: no rule)
  int kstop;             // fixed K (> 0) or 0
  int warm;              // first k with W(k) < warmup_tail (warm_step in batch.cu)
  int pad;
};

// Per-column progress, updated by the control kernel.
struct ColStat {
  int k;      // r_k is the newest term in y
  int K;      // final K once done
  int done;   // the stop rule (or the fixed K) fired
  float C;    // max_{l<=k} ||r_l||_1
};

class ColumnEngine {
 public:
  struct Finished {
    int slot;
    uint64_t tag;
    gp_request req;
    int K;
    int k16_from;
    float C;
    double tail_bound;
    std::chrono::steady_clock::time_point t_admit;
  };

  // t_long: rows with more entries become chunk tiles (at most kBTileCap;
  // 0: from cfg.t_heavy, else kBTileCap).  pure16: a 16-bit engine (storage
  // GP_BF16 or GP_F16) without the FP32 pair, whose columns come only from an
  // FP32 engine once their warm-up is over (the service's second block, filled
  // by ring.cu); every pass of it gathers, reads and writes 16 bits.
  ColumnEngine(Graph& g, int B, gp_dtype storage, cudaStream_t st, int t_long = 0, bool pure16 = false);
  int t_long() const { return t_long_; }
  ~ColumnEngine();
  ColumnEngine(const ColumnEngine&) = delete;
  ColumnEngine& operator=(const ColumnEngine&) = delete;

  // Device bytes one column occupies (Q pair, 16-bit pair, y).
  static size_t bytes_per_column(const Graph& g, gp_dtype storage, bool pure16 = false);

  int width() const { return B_; }
  int active() const { return active_; }
  int free_slots() const;
  uint64_t passes() const { return passes_total_; }
  // Put requests into free columns (isolated sources are answered at once and
  // take no column).  Returns the column of each request (-1: answered).
  std::vector<int> admit(const std::vector<gp_request>& reqs, std::vector<uint64_t> tags);
  // One fused pass: stop rule and coefficients, then the SpMM step
  // (force_stage >= 0 fixes the storage stage: timing only).
  void pass(int force_stage = -1);
  // Write the outputs of the columns whose rule fired (all busy columns when
  // force_all), free them, and report them.
  std::vector<Finished> collect(bool force_all);
  // Forget the pass count and the 16-bit schedule (no column may be busy).
  void restart();
  bool pure16() const { return pure16_; }
  // Device arrays of the engine, for the device-resident service (ring.cu).
  struct View {
    float* f[2];      // FP32 pair (null in a pure16 engine)
    void* h[2];       // 16-bit pair (null in an FP32 engine)
    float* y;
    ColState* col;
    ColParam* par;
    ColStat* stat;
    float* norm;
    int B;
    int pass;         // index of the next pass: it gathers buffer pass & 1
    gp_dtype storage;
    bool pure16;
  };
  View view() const;
  // One pass whose width and busy-column count are read from device memory
  // (set by the service's kernels): the control kernel for the columns that
  // have not run a pass yet, then the fused SpMM step, which returns at once
  // while no column is busy.
  void pass_device(const int* width_dev, const int* active_dev);
  // The stop rule and next coefficient of the columns that ran the last
  // device-width pass, right after it (pass_device treats only new columns).
  void control_after();
  // Advance (or, with -1, take back) the pass count without launching: a
  // pass_device whose launches a replayed CUDA graph makes.
  void count_pass(int delta = 1) {
    pass_ += delta;
    passes_total_ += delta;
  }
  // Smallest pass width the engine's kernels accept (a 16-bit lane owns 16 columns).
  int min_width() const { return pure16_ && B_ >= 16 ? 16 : 8; }
  // Move the busy columns into the first half of the pass width once at most
  // half of it is busy.  Returns whether the width was halved.
  bool compact();
  // Clenshaw's backward form for a block of up to B requests with K fixed up
  // front (engine restarted, no column busy); writes the outputs and returns
  // the finished columns.
  std::vector<Finished> clenshaw(const std::vector<gp_request>& reqs, const std::vector<uint64_t>& tags);
  // Generalized propagation of features f0 .. f0+nb-1 of X (device, n x F,
  // row-major) into Z: the finished columns (tag = feature index).
  std::vector<Finished> propagate(const float* X, float* Z, int F, int f0, int nb, int function, double param,
                                  double a, double tol);
  // Time each SpMM pass with CUDA events (gp_batch under gp_profile_enable);
  // flush_profile() adds them to the graph's profile counters.
  void set_profile(bool on) { profile_ = on; }
  void flush_profile();

 private:
  void release();
  bool pass_16_ok() const;
  void write_outputs(const std::vector<int>& cols);
  void write_point(const gp_request& r, double f0);

  struct Slot {
    bool busy = false;
    gp_request req{};
    uint64_t tag = 0;
    std::chrono::steady_clock::time_point t_admit;
    std::vector<double> tails;  // FP64 tail(k) for the report
  };

  Graph& g_;
  int B_;
  int t_long_ = 0;  // rows with more entries are chunk tiles
  int bw_ = 0;  // columns of each pass (a prefix of B_)
  gp_dtype storage_;
  bool pure16_ = false;
  cudaStream_t st_;
  int kcap_ = 0;
  float* f_[2] = {nullptr, nullptr};  // FP32 Q pair
  void* h_[2] = {nullptr, nullptr};   // 16-bit Q pair
  float* y_ = nullptr;
  ColState* col_ = nullptr;
  ColParam* par_ = nullptr;
  ColStat* stat_ = nullptr;
  float* norm_ = nullptr;
  int* scratch_ = nullptr;
  void* outs_ = nullptr;
  void* stage_ = nullptr;
  int4* tiles_ = nullptr;     // schedule of the pass (batch.cu)
  int64_t ntiles_ = 0;
  int nlong_ = 0;
  int* poff_ = nullptr;
  int64_t* ldeg_ = nullptr;   // degrees of the long (chunked) rows
  void* zero_ = nullptr;      // B zero floats
  int* tile_ctr_ = nullptr;   // dynamic tile counter of the pass
  float* part_ = nullptr;
  int* cnt_ = nullptr;
  std::vector<Slot> slots_;
  int active_ = 0;
  int pass_ = 0;
  int h_pass_ = -1;
  int warm_ = 0;
  uint64_t passes_total_ = 0;
  bool profile_ = false;
  struct Prop {  // output target while propagate() runs
    bool on;
    float* Z;
    int F;
    double a;
    const float* degf;
    const float* colnorm;
  } prop_{false, nullptr, 0, 0.0, nullptr, nullptr};
  float* degf_ = nullptr;  // degrees of the active rows (relabelled), for propagate()
  std::vector<cudaEvent_t> events_;
  std::vector<double> prof_marks_;  // algorithmic bytes of each timed pass
};

// The W(k) threshold below which a column of tolerance tol may store its Q in
// 16 bits: cfg.warmup_tail for BF16, four times it for FP16 (an 11-bit
// significand against BF16's 8, with Q * 2^12 clear of the subnormals), each
// scaled down in proportion to tol below 1e-4 (the 16-bit rounding error that
// reaches y is proportional to the threshold).
double column_warm_tail(double warmup_tail, gp_dtype storage, double tol);
// The first step k whose W(k) = sum_{m>=0} (m + 1) |c_{k+1+m}| is below the
// threshold (kcap when none): Q_j with j >= k + 2 may be stored in 16 bits.
int warm_step(const std::vector<double>& c, int kcap, double warmup_tail);

struct BatchCache {
  std::unique_ptr<ColumnEngine> eng;
  int B = 0;
  int t_long = 0;
  gp_dtype storage = GP_F32;
};

}  // namespace gp
