// Serving loop: not built yet.
#include "tn_host.h"
extern "C" tn_status tn_server_create(const tn_server_cfg *, tn_server **out) {
  if (out) *out = nullptr;
  return tn_fail(TN_ERR_UNSUPPORTED, "server not built");
}
extern "C" tn_status tn_server_submit(tn_server *, tn_plan *, const uint64_t *, int64_t, tn_precision, tn_c128 *,
                                      uint64_t *) {
  return tn_fail(TN_ERR_UNSUPPORTED, "server not built");
}
extern "C" tn_status tn_server_wait(tn_server *, uint64_t, int64_t) { return TN_ERR_UNSUPPORTED; }
extern "C" tn_status tn_server_stats_get(tn_server *, tn_server_stats *) { return TN_ERR_UNSUPPORTED; }
extern "C" void tn_server_free(tn_server *) {}
