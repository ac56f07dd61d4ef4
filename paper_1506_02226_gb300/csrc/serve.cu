// serve.cu — continuous-batching job server (placeholder until built).
#include <cstring>

#include "plan.h"

extern "C" {
void dbscan_serve_opts_default(dbscan_serve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->slots = 8;
    o->hbm_budget_bytes = (int64_t)120 << 30;
}
int dbscan_serve_create(dbscan_server **out, const dbscan_serve_opts *) {
    if (out) *out = nullptr;
    return DBSCAN_ERR_UNSUPPORTED;
}
int dbscan_serve_submit(dbscan_server *, const dbscan_instance *, uint64_t *) { return DBSCAN_ERR_UNSUPPORTED; }
int dbscan_serve_poll(dbscan_server *, uint64_t, int32_t *) { return DBSCAN_ERR_UNSUPPORTED; }
int dbscan_serve_wait(dbscan_server *, uint64_t, int64_t, double *) { return DBSCAN_ERR_UNSUPPORTED; }
int dbscan_serve_destroy(dbscan_server *) { return DBSCAN_OK; }
}
