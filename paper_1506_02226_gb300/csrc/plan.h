// plan.h — host-side state of a dbscan_plan (internal to libdbscan_gb300).
#pragma once

#include "internal.cuh"

struct BatchState;

struct dbscan_plan {
    dbscan_opts opts{};
    cudaStream_t stream = nullptr;
    void *ws_base = nullptr;  // one device allocation, carved into DbWork
    size_t ws_bytes = 0;
    bool owns_ws = false;     // false: the workspace was bound by its owner (a server slot)
    DbWork w{};
    unsigned *h_status = nullptr;          // pinned
    unsigned long long *h_ctr = nullptr;   // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // dbscan_run_host staging (allocated on first use)
    float *stage_in = nullptr;
    int32_t *stage_out = nullptr;
    size_t extra_bytes = 0;
    BatchState *batch = nullptr;  // dbscan_batch state (allocated on first use)
    void *pp_buf = nullptr;       // dbscan_run_paper's matrices (allocated on first use, grown on demand)
    size_t pp_bytes = 0;
    PhaseMarks marks;             // per-kernel events (opts.profile)
    int test_hook = 0;            // dbscan_plan_test_hook, consumed by the next run it applies to
};

int plan_run(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
             int32_t *labels, int32_t *counts_out, uint8_t *core_out, dbscan_stats *stats);
int plan_read_status(dbscan_plan *plan, bool clear);
// Status code of the device error bits of a run.
int plan_status_from_bits(unsigned bits);
// A plan with streams, events and host buffers but no device workspace yet.
int plan_create_unbound(dbscan_plan **out, const dbscan_opts &o);
// Device bytes of the workspace for instances up to (n, d) under o's options
// (exact_d: instances of exactly this d, so no eps-grid arrays when d > 3).
size_t plan_workspace_bytes_for(const dbscan_opts &o, int64_t n, int32_t d, bool exact_d);
// Carves [base, base + bytes) into the plan's workspace for instances up to
// (n, d) (exact_d as above); the plan then accepts such instances.  The memory
// stays the caller's unless the plan owns it (owns_ws).
int plan_bind_workspace(dbscan_plan *p, void *base, size_t bytes, int64_t n, int32_t d, bool exact_d);
int plan_ensure_staging(dbscan_plan *plan, int64_t n, int32_t d);
void plan_release_extras(dbscan_plan *plan);
void batch_release(BatchState *b);
// The paper's materialised pipeline (paper_pipeline.cu): device bytes for n
// points, and the launch of all its stages.
size_t paper_pipeline_bytes(int64_t n);
cudaError_t launch_paper_pipeline(const DbWork &w, void *base, const float *x, int64_t n, int32_t d, int64_t Tc,
                                  int32_t min_pts, int32_t *labels, int *sweeps, cudaStream_t st);
