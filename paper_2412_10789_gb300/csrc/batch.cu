// Batched multi-source ChebyPower (gp_batch).
#include "gp_internal.h"

namespace gp {

void run_batch(Graph& g, int count, const gp_request* reqs, gp_query_info* infos) {
  (void)g; (void)count; (void)reqs; (void)infos;
  throw Error{GP_ENOTSUP, "gp_batch is not available in this build"};
}

void free_batch_work(Graph& g) { (void)g; }

}  // namespace gp
