// Continuous-batching service (gp_submit / gp_poll / gp_wait / gp_serve_stats).
//
// One service thread per graph owns the column engines (batch.h) of its block
// on its own stream.  The block's width (columns = query slots) is what the
// memory budget allows (cfg.mem_budget, default 80% of the free device
// memory, at ColumnEngine::bytes_per_column each), capped by cfg.block_width
// (256 by default, 512 at most), so a free column is also free memory for one
// more query.  A warp spans at most 256 FP32 columns of a row, so a
// 512-column block is two 256-column engines, each advanced by its own fused
// pass.  Each iteration admits queued requests into free columns (first
// engine first), runs one fused pass over the active columns of each engine
// that has any (the per-column stop rule runs on the device in the pass's
// control kernel), and every few passes collects the retired columns: their y
// is written to the request's y_out, the ticket completes, and the column is
// free for the next request.  Passes cover only the prefix of columns that
// holds the busy ones, and the busy columns are moved to the front when at
// most half of that prefix is busy, so a lightly loaded service runs narrow
// passes.  Requests therefore join and leave the running block while the
// others keep going; their work shares every pass.
//
// 16-bit storage (cfg.storage GP_BF16 or GP_F16).  Columns join at different
// passes, so one block cannot switch its storage for all of them at once.
// The service keeps two blocks of the same width: requests start in an FP32
// block, and once a column's stored terms are past its own warm-up (the
// weighted tail W(k) of its coefficients below its threshold, which scales
// with its tolerance) it moves to a 16-bit block (its Q_k and Q_{k-1} rounded
// to 16 bits, y kept in FP32), where it runs to its stop.  A column whose
// 16-bit block is full stays in FP32 until a slot frees up.
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "batch.h"

namespace gp {

namespace {

constexpr size_t kQueueCap = 1 << 20;
constexpr int kServeMaxWidth = 512;      // query slots of the service's block, at most
constexpr int kServeDefaultWidth = 256;  // ... when cfg.block_width is 0
constexpr int kEngineMaxWidth = 256;     // columns of one engine
constexpr int kCollectEvery = 2;

struct Ticket {
  uint64_t id;
  gp_request req;
  std::chrono::steady_clock::time_point t_submit;
};

struct Done {
  gp_status status;
  gp_query_info info;
};

struct Serve {
  Graph* g = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<std::unique_ptr<ColumnEngine>> engs;  // the FP32 block's column halves (admission)
  std::vector<std::unique_ptr<ColumnEngine>> engs16;  // the 16-bit block's halves (16-bit storage only)
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Ticket> pending;
  std::unordered_map<uint64_t, std::chrono::steady_clock::time_point> inflight;  // admitted
  std::unordered_map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::string error;
  std::thread th;
  uint64_t completed = 0, passes = 0;
  double active_sum = 0.0;

  int active() const {
    int a = 0;
    for (const auto& e : engs) a += e->active();
    for (const auto& e : engs16) a += e->active();
    return a;
  }
  int free_slots() const {
    int f = 0;
    for (const auto& e : engs) f += e->free_slots();
    return f;
  }

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

  void loop() {
    int since_collect = 0;
    for (;;) {
      std::vector<gp_request> reqs;
      std::vector<uint64_t> tags;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !pending.empty() || active() > 0; });
        if (stop) return;
        int free = free_slots();
        while (free > 0 && !pending.empty()) {
          Ticket t = pending.front();
          pending.pop_front();
          reqs.push_back(t.req);
          tags.push_back(t.id);
          inflight[t.id] = t.t_submit;
          --free;
        }
      }
      for (size_t e = 0, i = 0; e < engs.size() && i < reqs.size(); ++e) {
        const size_t take = std::min(reqs.size() - i, (size_t)engs[e]->free_slots());
        if (take == 0) continue;
        std::vector<gp_request> r(reqs.begin() + i, reqs.begin() + i + take);
        std::vector<uint64_t> t(tags.begin() + i, tags.begin() + i + take);
        std::vector<int> slots = engs[e]->admit(r, t);
        i += take;
        // isolated sources are answered at admission
        std::lock_guard<std::mutex> lk(mu);
        for (size_t j = 0; j < slots.size(); ++j)
          if (slots[j] < 0) finish(t[j], 0, 1, 1.0, 0.0);
      }
      if (active() > 0) {
        active_sum += active();
        ++passes;
        for (auto& e : engs)
          if (e->active() > 0) e->pass();
        for (auto& e : engs16)
          if (e->active() > 0) e->pass();
        // columns past their warm-up move from the FP32 block to the 16-bit one
        // (decided from the host's pass counts, so no wait on the device)
        for (auto& e : engs) {
          std::vector<int> warm = e->warm_columns();
          for (auto& h : engs16) {
            if (warm.empty()) break;
            const int moved = h->adopt(*e, warm);
            warm.erase(warm.begin(), warm.begin() + moved);
          }
        }
        if (++since_collect >= kCollectEvery) {
          since_collect = 0;
          bool queued = false;
          {
            std::lock_guard<std::mutex> lk(mu);
            queued = !pending.empty();
          }
          for (auto* list : {&engs, &engs16}) {
            for (auto& e : *list) {
              if (e->active() == 0) continue;
              auto fin = e->collect(false);
              // narrow the passes of a lightly loaded block; with requests
              // waiting, the freed columns refill at once instead
              while (!queued && e->active() > 0 && e->compact()) {
              }
              std::lock_guard<std::mutex> lk(mu);
              for (const auto& f : fin) finish(f.tag, f.K, f.k16_from, f.C, f.tail_bound);
            }
          }
        }
      }
    }
  }

  // mu held
  void finish(uint64_t id, int K, int k16_from, double C, double bound) {
    auto it = inflight.find(id);
    Done d;
    d.status = GP_OK;
    std::memset(&d.info, 0, sizeof(d.info));
    d.info.K = K;
    d.info.k16_from = k16_from;
    d.info.max_r_l1 = C;
    d.info.tail_bound = bound;
    if (it != inflight.end()) {
      d.info.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - it->second).count();
      inflight.erase(it);
    }
    done[id] = d;
    ++completed;
    cv.notify_all();
  }
};

Serve* get_serve(Graph& g) {
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  if (g.serve) return static_cast<Serve*>(g.serve);
  std::unique_ptr<Serve> s(new Serve());
  s->g = &g;
  GP_CUDA_TRY(cudaGetDevice(&s->device));
  GP_CUDA_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  size_t free_b = 0, total_b = 0;
  GP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = g.cfg.mem_budget ? g.cfg.mem_budget : (size_t)(0.8 * (double)free_b);
  const gp_dtype storage = g.cfg.storage;
  const bool two_blocks = storage == GP_BF16 || storage == GP_F16;
  const size_t per_col = ColumnEngine::bytes_per_column(g, GP_F32) +
                         (two_blocks ? ColumnEngine::bytes_per_column(g, storage, true) : 0);
  // 256 slots already keep the GPU busy on large graphs; more slots add
  // concurrency, not throughput, and lengthen every pass (latency under load)
  const int cap = std::min(g.cfg.block_width > 0 ? g.cfg.block_width : kServeDefaultWidth, kServeMaxWidth);
  int width = 8;
  while (width * 2 <= cap && (size_t)(width * 2) * per_col <= budget) width *= 2;
  if ((size_t)width * per_col > budget) throw Error{GP_ENOMEM, "memory budget is below eight query columns"};
  // Columns join at different passes, so they cannot share one 16-bit
  // switch-over: admission is into FP32 blocks, and with 16-bit storage the
  // columns move to 16-bit blocks after their own warm-up.
  for (int c0 = 0; c0 < width; c0 += kEngineMaxWidth) {
    const int w = std::min(width - c0, kEngineMaxWidth);
    s->engs.emplace_back(new ColumnEngine(g, w, GP_F32, s->stream));
    if (two_blocks) {
      s->engs.back()->hand_over_to(storage);
      s->engs16.emplace_back(new ColumnEngine(g, w, storage, s->stream, 0, true));
    }
  }
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

}  // namespace

uint64_t serve_submit(Graph& g, const gp_request& req) {
  validate(g, req);
  Serve* s = get_serve(g);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) throw Error{GP_ECUDA, "the service stopped: " + s->error};
  if (s->pending.size() >= kQueueCap) throw Error{GP_EBUSY, "the request queue is full"};
  const uint64_t id = s->next_ticket++;
  s->pending.push_back(Ticket{id, req, std::chrono::steady_clock::now()});
  s->cv.notify_all();
  return id;
}

gp_status serve_poll(Graph& g, uint64_t ticket, gp_query_info* info) {
  Serve* s = static_cast<Serve*>(g.serve);
  if (!s) {
    set_last_error("unknown ticket");
    return GP_ENOTFOUND;
  }
  std::lock_guard<std::mutex> lk(s->mu);
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
    bool known = s->inflight.count(ticket) > 0;
    for (const Ticket& t : s->pending) known = known || t.id == ticket;
    if (!known) {
      set_last_error("unknown ticket");
      return GP_ENOTFOUND;
    }
    // finish() and fail() notify the condition variable; wake at the deadline otherwise
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
  s->engs.clear();
  s->engs16.clear();
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  g.serve = nullptr;
}

}  // namespace gp
