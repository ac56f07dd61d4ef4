// extras.cu — lazily allocated plan buffers (host-copy staging) and their release.
#include "plan.h"

int plan_ensure_staging(dbscan_plan *p, int64_t /*n*/, int32_t /*d*/) {
    if (p->stage_in) return DBSCAN_OK;
    const size_t in_bytes = sizeof(float) * (size_t)p->w.cap_n * (size_t)p->opts.max_d;
    const size_t out_bytes = sizeof(int32_t) * (size_t)p->w.cap_n;
    if (cudaMalloc(&p->stage_in, in_bytes) != cudaSuccess) {
        cudaGetLastError();
        p->stage_in = nullptr;
        return DBSCAN_ERR_OOM;
    }
    if (cudaMalloc(&p->stage_out, out_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p->stage_in);
        p->stage_in = nullptr;
        p->stage_out = nullptr;
        return DBSCAN_ERR_OOM;
    }
    p->extra_bytes += in_bytes + out_bytes;
    return DBSCAN_OK;
}

void plan_release_extras(dbscan_plan *p) {
    if (p->stage_in) cudaFree(p->stage_in);
    if (p->stage_out) cudaFree(p->stage_out);
    p->stage_in = nullptr;
    p->stage_out = nullptr;
    if (p->batch) batch_release(p->batch);
    p->batch = nullptr;
    if (p->pp_buf) cudaFree(p->pp_buf);
    p->pp_buf = nullptr;
    p->pp_bytes = 0;
}
