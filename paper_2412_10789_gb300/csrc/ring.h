// Data of the device-resident service loop (ring.cu): the request and done
// rings in mapped host memory, the per-slot records and the device counters.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "batch.h"

namespace gp {

// Shared by the service thread and the kernels (mapped host memory).  The
// host writes tail and consumed (release stores); the device writes head and
// done (release stores at system scope) and active.
struct RingCtl {
  uint64_t tail;      // requests published by the host
  uint64_t head;      // requests admitted by the device
  uint64_t done;      // done records written by the device
  uint64_t consumed;  // done records read by the host
  int active;         // busy columns of both blocks after the last iteration
  int pad;
};

// One request as the device admits it: the host computes the coefficients
// (FP64, stored as FP32 tables) and the relabelled source.
struct RingReq {
  ColParam param;
  uint64_t ticket;
  void* out;      // device output: the caller's buffer or a staging buffer
  int64_t src;    // relabelled source (degree >= 1)
  int out_f64;    // 1: double output, 0: float
  int k_low;      // no stop before this step (the stop rule with max ||r_l||_1 at its least, 1)
};

struct RingDone {
  uint64_t ticket;
  int K;
  int k16_from;
  float C;
  int pad;
};

// A column slot's request, on the device.
struct SlotDev {
  uint64_t ticket;
  void* out;
  int64_t src;
  int busy;
  int out_f64;
  int warm;
  int k16;    // first 16-bit term once migrated, else -1
  int k_low;  // no stop before this step
  int pad;
};

// Device counters of the loop.
struct RingDev {
  uint64_t head;
  uint64_t done;
  int new_count;
  int active32;
  int active16;
  int mig_count;
};

}  // namespace gp

namespace gp {

// One FP32 admission block (at most 256 columns) and, with 16-bit storage, a
// 16-bit block of the same width, driven by the device-resident loop.
class RingLoop {
 public:
  // t_long: rows with more entries are chunked (0: the engines' default).
  RingLoop(Graph& g, int width, gp_dtype storage, cudaStream_t st, int t_long = 0);
  ~RingLoop();
  RingLoop(const RingLoop&) = delete;
  RingLoop& operator=(const RingLoop&) = delete;

  int width() const { return B_; }
  // Requests the ring can take now (published but not yet admitted ones use
  // ring entries).
  int room() const;
  // Publish one request (room() must be positive).
  void publish(const RingReq& r);
  // Launch one iteration of the loop (no wait for the device).  After two
  // direct iterations, the launches of an iteration are captured once per
  // pass parity (the only thing that differs between iterations is which of
  // each block's two Q buffers a pass gathers) and replayed as a CUDA graph.
  void iterate();
  // Done records the device has made visible since the last call.
  void take_done(std::vector<RingDone>& out);
  // Busy columns of both blocks after the last finished iteration.
  int active() const;

 private:
  void release();
  void enqueue();               // the launches of one iteration
  cudaGraphExec_t graph_[2] = {nullptr, nullptr};  // iteration launches by pass parity
  uint64_t graph_launches_[2] = {0, 0};            // kernels each graph holds
  uint64_t iters_ = 0;
  bool graphs_off_ = false;     // capture failed once: launch directly
  Graph& g_;
  int B_;
  cudaStream_t st_;
  std::unique_ptr<ColumnEngine> e32_, e16_;
  RingCtl* ctl_ = nullptr;      // mapped host memory
  RingCtl* ctl_d_ = nullptr;    // its device address
  RingReq* req_ = nullptr;
  RingReq* req_d_ = nullptr;
  RingDone* done_ = nullptr;
  RingDone* done_d_ = nullptr;
  int cap_req_ = 0, cap_done_ = 0;
  void* dmem_ = nullptr;        // device block of the lists and counters below
  RingDev* dev_ = nullptr;
  SlotDev* slots32_ = nullptr;
  SlotDev* slots16_ = nullptr;
  int* new_list_ = nullptr;
  int* ret32_ = nullptr;
  int* ret16_ = nullptr;
  int* cnt_ = nullptr;          // [0] retired FP32, [1] retired 16-bit, [2] width FP32, [3] width 16-bit,
                                // [4] columns moved by the compaction
  int* mig_from_ = nullptr;
  int* mig_to_ = nullptr;
  uint64_t tail_ = 0;           // requests published
  uint64_t consumed_ = 0;       // done records read
};

}  // namespace gp
