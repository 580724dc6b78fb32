// C ABI entry points: argument checks, the exception-to-status guard, the
// thread-local error message, and dispatch to the query functions.
#include <cstring>
#include <exception>
#include <functional>
#include <mutex>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "gp_internal.h"

namespace gp {

std::atomic<uint64_t> g_launches{0};

TraceRange::TraceRange(const char* name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

namespace {
thread_local std::string t_last_error;
}

void set_last_error(const std::string& msg) { t_last_error = msg; }

gp_status guard(const std::function<void()>& f) {
  try {
    f();
    return GP_OK;
  } catch (const Error& e) {
    t_last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    t_last_error = "host allocation failed";
    return GP_ENOMEM;
  } catch (const std::exception& e) {
    t_last_error = e.what();
    return GP_EINVAL;
  } catch (...) {
    t_last_error = "unknown error";
    return GP_EINVAL;
  }
}

static Graph* as_graph(gp_graph* g) {
  if (!g) throw Error{GP_EINVAL, "graph is NULL"};
  return reinterpret_cast<Graph*>(g);
}

static gp_request make_request(int function, int32_t source, double param, double tol, gp_dtype out_dtype,
                               void* y_out, int y_on_device) {
  gp_request r;
  std::memset(&r, 0, sizeof(r));
  r.function = function;
  r.source = source;
  r.param = param;
  r.l1_tol = tol;
  r.k_rule = GP_K_TAIL;
  r.k_fixed = 0;
  r.out_dtype = out_dtype;
  r.y_on_device = y_on_device;
  r.y_out = y_out;
  return r;
}

}  // namespace gp

using namespace gp;

extern "C" void gp_config_default(gp_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->storage = GP_F32;
  cfg->block_width = 0;
  cfg->autotune = 0;
  cfg->k_max = 96;
  cfg->validate_symmetry = 1;
  cfg->t_heavy = 0;
  cfg->warmup_tail = 1e-2;
  cfg->mem_budget = 0;
  cfg->alloc = nullptr;
  cfg->free = nullptr;
  cfg->alloc_ctx = nullptr;
  cfg->stream = nullptr;
}

extern "C" gp_status gp_ppr(gp_graph* gh, int32_t source, double alpha, double l1_tol, gp_dtype out_dtype,
                            void* y_out, int y_on_device, gp_query_info* info) {
  TraceRange trace("gp_ppr");
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    gp_request r = make_request(GP_FN_PPR, source, alpha, l1_tol, out_dtype, y_out, y_on_device);
    run_query(*g, r, info);
  });
}

extern "C" gp_status gp_hkpr(gp_graph* gh, int32_t source, double t, double l1_tol, gp_dtype out_dtype,
                             void* y_out, int y_on_device, gp_query_info* info) {
  TraceRange trace("gp_hkpr");
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    gp_request r = make_request(GP_FN_HKPR, source, t, l1_tol, out_dtype, y_out, y_on_device);
    run_query(*g, r, info);
  });
}

extern "C" gp_status gp_query(gp_graph* gh, const gp_request* req, gp_query_info* info) {
  TraceRange trace("gp_query");
  return guard([&] {
    Graph* g = as_graph(gh);
    GP_REQUIRE(req, "request is NULL");
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    run_query(*g, *req, info);
  });
}

extern "C" gp_status gp_power(gp_graph* gh, int32_t function, int32_t source, double param, double l1_tol,
                              gp_dtype out_dtype, void* y_out, int y_on_device, gp_query_info* info) {
  TraceRange trace("gp_power");
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    gp_request r = make_request(function, source, param, l1_tol, out_dtype, y_out, y_on_device);
    run_power(*g, r, info);
  });
}

extern "C" gp_status gp_batch(gp_graph* gh, int32_t count, const gp_request* reqs, gp_query_info* infos) {
  TraceRange trace("gp_batch");
  return guard([&] {
    Graph* g = as_graph(gh);
    GP_REQUIRE(count >= 0, "count must be >= 0");
    GP_REQUIRE(count == 0 || reqs, "requests are NULL");
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    run_batch(*g, count, reqs, infos);
  });
}

extern "C" gp_status gp_submit(gp_graph* gh, const gp_request* req, uint64_t* ticket) {
  return guard([&] {
    Graph* g = as_graph(gh);
    GP_REQUIRE(req && ticket, "NULL argument");
    *ticket = serve_submit(*g, *req);
  });
}

extern "C" gp_status gp_poll(gp_graph* gh, uint64_t ticket, gp_query_info* info) {
  gp_status st = GP_OK;
  gp_status rc = guard([&] {
    Graph* g = as_graph(gh);
    st = serve_poll(*g, ticket, info);
  });
  return rc != GP_OK ? rc : st;
}

extern "C" gp_status gp_wait(gp_graph* gh, uint64_t ticket, double timeout_ms, gp_query_info* info) {
  gp_status st = GP_OK;
  gp_status rc = guard([&] {
    Graph* g = as_graph(gh);
    GP_REQUIRE(timeout_ms >= 0.0, "timeout_ms must be >= 0");
    st = serve_wait(*g, ticket, timeout_ms, info);
  });
  return rc != GP_OK ? rc : st;
}

extern "C" gp_status gp_batch_clenshaw(gp_graph* gh, int32_t count, const gp_request* reqs, gp_query_info* infos) {
  TraceRange trace("gp_batch_clenshaw");
  return guard([&] {
    Graph* g = as_graph(gh);
    GP_REQUIRE(count >= 0, "count must be >= 0");
    GP_REQUIRE(count == 0 || reqs, "requests are NULL");
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    run_clenshaw(*g, count, reqs, infos);
  });
}

extern "C" gp_status gp_propagate(gp_graph* gh, int32_t function, double param, double a, int32_t F, const float* X,
                                   float* Z, int on_device, double l1_tol, gp_query_info* infos) {
  TraceRange trace("gp_propagate");
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    run_propagate(*g, function, param, a, F, X, Z, on_device, l1_tol, infos);
  });
}

extern "C" gp_status gp_chebypush(gp_graph* gh, int32_t function, int32_t source, double param, double eps_a,
                                   int32_t K, gp_dtype out_dtype, void* y_out, int y_on_device, gp_query_info* info) {
  TraceRange trace("gp_chebypush");
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    run_chebypush(*g, function, source, param, eps_a, K, out_dtype, y_out, y_on_device, info);
  });
}

extern "C" gp_status gp_ppr_bidirectional(gp_graph* gh, int32_t source, double alpha, double eps_r, double delta,
                                           int32_t K, uint64_t seed, gp_dtype out_dtype, void* y_out,
                                           int y_on_device, gp_query_info* info) {
  TraceRange trace("gp_ppr_bidirectional");
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    run_bidirectional(*g, source, alpha, eps_r, delta, K, seed, out_dtype, y_out, y_on_device, info);
  });
}

extern "C" gp_status gp_autotune(gp_graph* gh, gp_dtype storage, const int32_t* widths, int32_t nwidths,
                                  int32_t* best_width, int32_t* best_t_heavy, double* us_per_column_pass) {
  TraceRange trace("gp_autotune");
  return guard([&] {
    Graph* g = as_graph(gh);
    GP_REQUIRE(best_width, "best_width is NULL");
    GP_REQUIRE(storage == GP_F32 || storage == GP_BF16 || storage == GP_F16, "storage must be GP_F32, GP_BF16 or GP_F16");
    GP_REQUIRE(nwidths >= 0 && (nwidths == 0 || widths), "widths is NULL");
    std::vector<int> w(widths, widths + nwidths);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    const TunedBlock tb = tune_block(*g, storage, w);
    *best_width = tb.B;
    if (best_t_heavy) *best_t_heavy = tb.t_long + 1;
    if (us_per_column_pass) *us_per_column_pass = tb.us;
  });
}

extern "C" gp_status gp_serve_stats(gp_graph* gh, uint64_t* completed, uint64_t* steps, double* mean_active) {
  return guard([&] { serve_stats(*as_graph(gh), completed, steps, mean_active); });
}

extern "C" uint64_t gp_launch_count(void) { return g_launches.load(); }

extern "C" gp_status gp_profile_enable(gp_graph* gh, int on) {
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    g->profiling = on != 0;
  });
}

extern "C" gp_status gp_profile_read(gp_graph* gh, double* step_ms, int64_t* step_launches, double* step_bytes) {
  return guard([&] {
    Graph* g = as_graph(gh);
    std::lock_guard<std::recursive_mutex> lk(g->mu);
    if (step_ms) *step_ms = g->prof_ms;
    if (step_launches) *step_launches = g->prof_launches;
    if (step_bytes) *step_bytes = g->prof_bytes;
    g->prof_ms = 0.0;
    g->prof_launches = 0;
    g->prof_bytes = 0.0;
  });
}

extern "C" const char* gp_status_string(gp_status s) {
  switch (s) {
    case GP_OK: return "GP_OK";
    case GP_EINVAL: return "GP_EINVAL: invalid argument";
    case GP_ENOMEM: return "GP_ENOMEM: out of memory";
    case GP_ECUDA: return "GP_ECUDA: CUDA error";
    case GP_EAGAIN: return "GP_EAGAIN: not finished";
    case GP_ENOTFOUND: return "GP_ENOTFOUND: unknown ticket";
    case GP_ETIMEDOUT: return "GP_ETIMEDOUT: device wait timed out";
    case GP_EBUSY: return "GP_EBUSY: queue full";
    case GP_ENOTSUP: return "GP_ENOTSUP: not supported";
  }
  return "unknown status";
}

extern "C" const char* gp_last_error(void) { return t_last_error.c_str(); }
