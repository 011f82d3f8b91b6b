// lgt_server.cu -- continuous-batching job server (see include/lgt.h).
#include "lgt_api_internal.h"

extern "C" lgt_status lgt_server_create(size_t hbm_budget_bytes, int device, lgt_server **out) {
  (void)hbm_budget_bytes; (void)device;
  if (out) *out = nullptr;
  lgt_set_error("server not available in this build");
  return LGT_EINVAL;
}
extern "C" lgt_status lgt_submit(lgt_server *s, const lgt_params *params, const double *links, uint64_t *job_id) {
  (void)s; (void)params; (void)links; (void)job_id;
  lgt_set_error("server not available in this build");
  return LGT_EINVAL;
}
extern "C" lgt_status lgt_poll(lgt_server *s, uint64_t job_id, lgt_result *res, double *links_out) {
  (void)s; (void)job_id; (void)res; (void)links_out;
  lgt_set_error("server not available in this build");
  return LGT_EINVAL;
}
extern "C" lgt_status lgt_cancel(lgt_server *s, uint64_t job_id) {
  (void)s; (void)job_id;
  lgt_set_error("server not available in this build");
  return LGT_EINVAL;
}
extern "C" lgt_status lgt_server_stats(lgt_server *s, uint64_t *a, uint64_t *b, size_t *c) {
  (void)s; (void)a; (void)b; (void)c;
  lgt_set_error("server not available in this build");
  return LGT_EINVAL;
}
extern "C" void lgt_server_destroy(lgt_server *s) { (void)s; }
