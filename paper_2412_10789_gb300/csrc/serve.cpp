// Continuous-batching service (gp_submit / gp_poll).
#include "gp_internal.h"

namespace gp {

uint64_t serve_submit(Graph& g, const gp_request& req) {
  (void)g; (void)req;
  throw Error{GP_ENOTSUP, "gp_submit is not available in this build"};
}
gp_status serve_poll(Graph& g, uint64_t ticket, gp_query_info* info) {
  (void)g; (void)ticket; (void)info;
  throw Error{GP_ENOTSUP, "gp_poll is not available in this build"};
}
void serve_stats(Graph& g, uint64_t* completed, uint64_t* steps, double* mean_active) {
  (void)g;
  if (completed) *completed = 0;
  if (steps) *steps = 0;
  if (mean_active) *mean_active = 0.0;
}
void serve_shutdown(Graph& g) { (void)g; }

}  // namespace gp
