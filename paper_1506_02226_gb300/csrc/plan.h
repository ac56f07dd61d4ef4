// plan.h — host-side state of a dbscan_plan (internal to libdbscan_gb300).
#pragma once

#include "internal.cuh"

struct BatchState;

struct dbscan_plan {
    dbscan_opts opts{};
    cudaStream_t stream = nullptr;
    void *ws_base = nullptr;  // one device allocation, carved into DbWork
    size_t ws_bytes = 0;
    DbWork w{};
    unsigned *h_status = nullptr;          // pinned
    unsigned long long *h_ctr = nullptr;   // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // dbscan_run_host staging (allocated on first use)
    float *stage_in = nullptr;
    int32_t *stage_out = nullptr;
    size_t extra_bytes = 0;
    BatchState *batch = nullptr;  // dbscan_batch state (allocated on first use)
    PhaseMarks marks;             // per-kernel events (opts.profile)
    int test_hook = 0;            // dbscan_plan_test_hook, consumed by the next run it applies to
};

int plan_run(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
             int32_t *labels, int32_t *counts_out, uint8_t *core_out, dbscan_stats *stats);
int plan_read_status(dbscan_plan *plan, bool clear);
int plan_ensure_staging(dbscan_plan *plan, int64_t n, int32_t d);
void plan_release_extras(dbscan_plan *plan);
void batch_release(BatchState *b);
