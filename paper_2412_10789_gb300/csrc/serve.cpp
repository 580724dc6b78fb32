// Continuous-batching service (gp_submit / gp_poll / gp_wait / gp_serve_stats)
// on the device-resident request loop of ring.cu.
//
// gp_submit validates a request, computes its Chebyshev coefficients, tails,
// stop parameters and warm-up step on the host (FP64), and queues it.  One
// service thread per graph publishes queued requests into the request rings
// of its blocks (pinned, mapped host memory the GPU reads), launches
// iterations of the loop back to back (at most two ahead of the GPU, never
// waiting for it otherwise), and turns the done records the GPU writes into
// completed tickets.  Which free column a request takes, when a column
// retires, where its y goes and when its slot is refilled are decided by the
// loop's kernels on the device, one pass at a time, so requests join and
// leave the running block while the others keep going.
//
// The block has as many columns as the memory budget allows (cfg.mem_budget,
// default 80% of the free device memory, at ColumnEngine::bytes_per_column
// each), capped by cfg.block_width (with cfg.autotune and no width, the
// autotuned width; else 256; 512 at most); a block of
// more than 256 columns runs as 256-column halves, each its own loop.  With
// 16-bit storage (cfg.storage GP_BF16 or GP_F16) each half has an FP32 block
// for admission and a 16-bit block of the same width: a column moves to the
// 16-bit block once its own warm-up is over.
//
// Outputs.  The device writes y straight into device outputs.  A request
// with a host output takes one of a few device staging buffers (allocated on
// first use); the service thread copies it to the caller's buffer when the
// done record arrives, and requests wait in the queue while every staging
// buffer is in use.  An isolated source is answered by the service thread
// without a column: y = f(0) e_s.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "ring.h"

namespace gp {

namespace {

constexpr size_t kQueueCap = 1 << 20;
constexpr int kServeMaxWidth = 512;      // query slots of the service's block, at most
constexpr int kServeDefaultWidth = 256;  // ... when cfg.block_width is 0
constexpr int kEngineMaxWidth = 256;     // columns of one loop's block
constexpr int kStaging = 8;              // device staging buffers for host outputs
constexpr int kAhead = 2;                // iterations queued ahead of the GPU

struct Ticket {
  uint64_t id;
  gp_request req;
  RingReq ring;               // the request as the device admits it (out set at publication)
  std::vector<double> tails;  // FP64 tail(k), for the reported bound
  bool isolated = false;
  std::chrono::steady_clock::time_point t_submit;
};

struct InFlight {
  gp_request req;
  std::vector<double> tails;
  int staging;  // staging buffer of a host output, else -1
  std::chrono::steady_clock::time_point t_submit;
};

struct Done {
  gp_status status;
  gp_query_info info;
};

struct Serve {
  Graph* g = nullptr;
  int device = 0;
  gp_dtype storage = GP_F32;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  std::vector<std::unique_ptr<RingLoop>> loops;  // the block's halves
  std::vector<cudaEvent_t> events;
  std::vector<void*> staging;
  std::vector<int> staging_free;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Ticket> pending;
  std::unordered_map<uint64_t, InFlight> inflight;  // published to a ring
  std::unordered_map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::string error;
  std::thread th;
  uint64_t completed = 0, passes = 0;
  double active_sum = 0.0;

  void run() {
    cudaSetDevice(device);
    try {
      loop();
    } catch (const Error& e) {
      fail(e.status, e.msg);
    } catch (const std::exception& e) {
      fail(GP_EINVAL, e.what());
    }
  }

  void fail(gp_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(mu);
    error = msg;
    Done d{st, {}};
    for (auto& kv : inflight) done[kv.first] = d;
    inflight.clear();
    for (auto& t : pending) done[t.id] = d;
    pending.clear();
    stop = true;
    cv.notify_all();
  }

  void* staging_buffer(int i) {
    while ((int)staging.size() <= i) staging.push_back(nullptr);
    if (!staging[i]) staging[i] = g->alloc.get(sizeof(double) * g->n);
    return staging[i];
  }

  // mu held.  Move queued requests into the rings while they have room.
  // Returns the isolated-source tickets to answer outside the lock.
  std::vector<Ticket> publish() {
    std::vector<Ticket> points;
    while (!pending.empty()) {
      Ticket& t = pending.front();
      if (t.isolated) {  // answered by the service thread, tracked as in flight meanwhile
        inflight[t.id] = InFlight{t.req, {}, -1, t.t_submit};
        points.push_back(t);
        pending.pop_front();
        continue;
      }
      RingLoop* best = nullptr;
      for (auto& l : loops)
        if (l->room() > 0 && (!best || l->room() > best->room())) best = l.get();
      if (!best) break;
      int st = -1;
      if (!t.req.y_on_device) {
        if (staging_free.empty()) break;  // waits for a staging buffer
        st = staging_free.back();
        t.ring.out = staging_buffer(st);
        staging_free.pop_back();
      } else {
        t.ring.out = t.req.y_out;
      }
      best->publish(t.ring);
      inflight[t.id] = InFlight{t.req, std::move(t.tails), st, t.t_submit};
      pending.pop_front();
    }
    return points;
  }

  void answer_point(const Ticket& t) {
    const gp_request& r = t.req;
    const double f0 = r.function == GP_FN_PPR ? r.param : std::exp(-r.param);
    const size_t esz = r.out_dtype == GP_F64 ? 8 : 4;
    std::vector<unsigned char> host(esz * g->n, 0);
    if (r.out_dtype == GP_F64)
      reinterpret_cast<double*>(host.data())[r.source] = f0;
    else
      reinterpret_cast<float*>(host.data())[r.source] = (float)f0;
    GP_CUDA_TRY(cudaMemcpyAsync(r.y_out, host.data(), esz * g->n,
                                r.y_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, copy_stream));
    GP_CUDA_TRY(cudaStreamSynchronize(copy_stream));
    std::lock_guard<std::mutex> lk(mu);
    inflight.erase(t.id);
    Done d{GP_OK, {}};
    d.info.K = 0;
    d.info.k16_from = 1;
    d.info.max_r_l1 = 1.0;
    d.info.tail_bound = 0.0;
    d.info.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t.t_submit).count();
    done[t.id] = d;
    ++completed;
    cv.notify_all();
  }

  // A done record: copy a staged output to the caller, complete the ticket.
  void complete(const RingDone& rd) {
    InFlight f;
    {
      // the ticket stays in flight (gp_poll: GP_EAGAIN) until its result is done
      std::lock_guard<std::mutex> lk(mu);
      auto it = inflight.find(rd.ticket);
      if (it == inflight.end()) return;
      f = it->second;
    }
    if (f.staging >= 0) {
      const size_t esz = f.req.out_dtype == GP_F64 ? 8 : 4;
      GP_CUDA_TRY(cudaMemcpyAsync(f.req.y_out, staging[f.staging], esz * g->n, cudaMemcpyDeviceToHost, copy_stream));
      GP_CUDA_TRY(cudaStreamSynchronize(copy_stream));
    }
    std::lock_guard<std::mutex> lk(mu);
    inflight.erase(rd.ticket);
    if (f.staging >= 0) staging_free.push_back(f.staging);
    Done d{GP_OK, {}};
    d.info.K = rd.K;
    d.info.k16_from = rd.k16_from;
    d.info.max_r_l1 = rd.C;
    const int k = std::min(rd.K, (int)f.tails.size() - 1);
    d.info.tail_bound = k >= 0 ? kCMargin * f.tails[k] * rd.C : 0.0;
    d.info.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - f.t_submit).count();
    done[rd.ticket] = d;
    ++completed;
    cv.notify_all();
  }

  void loop() {
    uint64_t it = 0;
    std::vector<RingDone> recs;
    for (;;) {
      std::vector<Ticket> points;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !pending.empty() || !inflight.empty(); });
        if (stop) return;
        points = publish();
      }
      for (const Ticket& t : points) answer_point(t);
      bool busy;
      {
        std::lock_guard<std::mutex> lk(mu);
        busy = !inflight.empty();
      }
      if (busy) {
        for (auto& l : loops) l->iterate();
        GP_CUDA_TRY(cudaEventRecord(events[it % kAhead], stream));
        ++it;
        ++passes;
        // keep at most kAhead iterations queued: wait for the one before
        if (it >= kAhead) GP_CUDA_TRY(cudaEventSynchronize(events[it % kAhead]));
        int act = 0;
        for (auto& l : loops) act += l->active();
        active_sum += act;
      }
      recs.clear();
      for (auto& l : loops) l->take_done(recs);
      for (const RingDone& rd : recs) complete(rd);
    }
  }
};

Serve* get_serve(Graph& g) {
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  if (g.serve) return static_cast<Serve*>(g.serve);
  std::unique_ptr<Serve> s(new Serve());
  s->g = &g;
  GP_CUDA_TRY(cudaGetDevice(&s->device));
  size_t free_b = 0, total_b = 0;
  GP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = g.cfg.mem_budget ? g.cfg.mem_budget : (size_t)(0.8 * (double)free_b);
  const gp_dtype storage = g.cfg.storage;
  const bool two_blocks = storage == GP_BF16 || storage == GP_F16;
  s->storage = two_blocks ? storage : GP_F32;
  const size_t per_col = ColumnEngine::bytes_per_column(g, GP_F32) +
                         (two_blocks ? ColumnEngine::bytes_per_column(g, storage, true) : 0);
  // The width: cfg.block_width, else with cfg.autotune the autotuner's width
  // for this graph (the width of least device time per column and pass; a
  // narrower block also shortens every pass, so latency under load drops
  // too), else 256 (more slots add concurrency, not throughput).
  int cap = kServeDefaultWidth, t_long = 0;
  if (g.cfg.block_width > 0) {
    cap = g.cfg.block_width;
  } else if (g.cfg.autotune) {
    const TunedBlock tb = tune_block(g, GP_F32, {});
    cap = tb.B;
    t_long = tb.t_long;
  }
  cap = std::min(cap, kServeMaxWidth);
  int width = 8;
  while (width * 2 <= cap && (size_t)(width * 2) * per_col <= budget) width *= 2;
  if ((size_t)width * per_col > budget) throw Error{GP_ENOMEM, "memory budget is below eight query columns"};
  GP_CUDA_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  GP_CUDA_TRY(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
  s->events.resize(kAhead, nullptr);
  for (auto& e : s->events) GP_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (int c0 = 0; c0 < width; c0 += kEngineMaxWidth)
    s->loops.emplace_back(new RingLoop(g, std::min(width - c0, kEngineMaxWidth), storage, s->stream, t_long));
  for (int i = kStaging - 1; i >= 0; --i) s->staging_free.push_back(i);
  s->th = std::thread([p = s.get()] { p->run(); });
  g.serve = s.release();
  return static_cast<Serve*>(g.serve);
}

void validate(const Graph& g, const gp_request& r) {
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

// The request as the device admits it: coefficients c_k (Lemma 2 / Lemma 3)
// and tails in FP64, stored as FP32 tables; the stop parameters; the warm-up
// step for the service's 16-bit storage; the relabelled source.
void prepare(const Graph& g, gp_dtype storage, Ticket& t) {
  const gp_request& r = t.req;
  if (g.h_deg[r.source] == 0) {
    t.isolated = true;
    return;
  }
  const int kcap = std::min(g.cfg.k_max, kMaxColK - 2);
  std::vector<double> c, tail;
  cheb_coefficients(r.function, r.param, kcap, c, tail);
  RingReq& q = t.ring;
  std::memset(&q, 0, sizeof(q));
  for (int k = 0; k <= kcap && k < kMaxColK; ++k) {
    q.param.c[k] = (float)c[k];
    q.param.tail[k] = (float)tail[k];
  }
  q.param.tol = r.k_rule == GP_K_TAIL ? (float)(r.l1_tol / kCMargin) : -1.0f;
  q.param.kstop = r.k_rule == GP_K_FIXED ? r.k_fixed
                  : r.k_rule == GP_K_PAPER ? std::min(kcap - 1, paper_k(r.function, r.param, r.l1_tol))
                                           : 0;
  q.param.warm = storage == GP_F32 ? kcap : warm_step(c, kcap, column_warm_tail(g.cfg.warmup_tail, storage, r.l1_tol));
  // with max ||r_l||_1 >= ||r_0||_1 = 1 the tail rule cannot stop before k_lower(.., 1)
  q.k_low = r.k_rule == GP_K_TAIL   ? k_lower(tail, r.l1_tol / kCMargin, 1.0)
            : q.param.kstop > 0 ? q.param.kstop
                                : kcap;
  q.ticket = t.id;
  q.src = g.h_newid[r.source];
  q.out_f64 = r.out_dtype == GP_F64 ? 1 : 0;
  t.tails.assign(tail.begin(), tail.end());
}

}  // namespace

uint64_t serve_submit(Graph& g, const gp_request& req) {
  validate(g, req);
  Serve* s = get_serve(g);
  Ticket t;
  t.req = req;
  t.t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) throw Error{GP_ECUDA, "the service stopped: " + s->error};
    if (s->pending.size() >= kQueueCap) throw Error{GP_EBUSY, "the request queue is full"};
    t.id = s->next_ticket++;
  }
  prepare(g, s->storage, t);  // host FP64 coefficients, outside the lock
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) throw Error{GP_ECUDA, "the service stopped: " + s->error};
  s->pending.push_back(std::move(t));
  s->cv.notify_all();
  return s->pending.back().id;
}

namespace {

// mu held: GP_OK (and *info) once done, GP_EAGAIN while known, else GP_ENOTFOUND.
gp_status ticket_state(Serve* s, uint64_t ticket, gp_query_info* info) {
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    const Done d = it->second;
    s->done.erase(it);
    if (d.status != GP_OK) {
      set_last_error(s->error);
      return d.status;
    }
    if (info) *info = d.info;
    return GP_OK;
  }
  if (s->inflight.count(ticket)) return GP_EAGAIN;
  for (const Ticket& t : s->pending)
    if (t.id == ticket) return GP_EAGAIN;
  set_last_error("unknown ticket");
  return GP_ENOTFOUND;
}

}  // namespace

gp_status serve_poll(Graph& g, uint64_t ticket, gp_query_info* info) {
  Serve* s = static_cast<Serve*>(g.serve);
  if (!s) {
    set_last_error("unknown ticket");
    return GP_ENOTFOUND;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  return ticket_state(s, ticket, info);
}

gp_status serve_wait(Graph& g, uint64_t ticket, double timeout_ms, gp_query_info* info) {
  Serve* s = static_cast<Serve*>(g.serve);
  if (!s) {
    set_last_error("unknown ticket");
    return GP_ENOTFOUND;
  }
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double, std::milli>(std::max(0.0, timeout_ms)));
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    const gp_status st = ticket_state(s, ticket, info);
    if (st != GP_EAGAIN) return st;
    // complete() and fail() notify the condition variable; wake at the deadline otherwise
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && !s->done.count(ticket)) {
      set_last_error("gp_wait: the ticket did not complete within " + std::to_string(timeout_ms) + " ms");
      return GP_ETIMEDOUT;
    }
  }
}

void serve_stats(Graph& g, uint64_t* completed, uint64_t* steps, double* mean_active) {
  Serve* s = static_cast<Serve*>(g.serve);
  uint64_t c = 0, p = 0;
  double m = 0.0;
  if (s) {
    std::lock_guard<std::mutex> lk(s->mu);
    c = s->completed;
    p = s->passes;
    m = p ? s->active_sum / (double)p : 0.0;
  }
  if (completed) *completed = c;
  if (steps) *steps = p;
  if (mean_active) *mean_active = m;
}

void serve_shutdown(Graph& g) {
  Serve* s = static_cast<Serve*>(g.serve);
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  s->loops.clear();
  for (void* p : s->staging)
    if (p) g.alloc.put(p);
  for (cudaEvent_t e : s->events)
    if (e) cudaEventDestroy(e);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  g.serve = nullptr;
}

}  // namespace gp
