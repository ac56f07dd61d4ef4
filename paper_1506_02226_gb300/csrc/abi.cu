// abi.cu — the C ABI declared in include/dbscan.h: plans, runs, status codes.
//
// A run enqueues the three steps of Section I on the plan's stream:
//   1-2. pair test fused with neighbour counting -> core flags (Sections IV-A, IV-B)
//   3.   union of core-core eps-edges, border assignment, labels (Section IV-C)
// through either the eps-grid path (d <= 3, grid.cu) or the all-pairs path
// (pairs_simt.cu; tensor-core Gram form in gram_tc.cu).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.cuh"
#include "plan.h"

static_assert(sizeof(dbscan_opts) == 72, "dbscan_opts layout");
static_assert(sizeof(dbscan_stats) == 96, "dbscan_stats layout");
static_assert(sizeof(dbscan_instance) == 40, "dbscan_instance layout");

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carver {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * count;
        return p;
    }
};

// Lays the workspace out (base == nullptr: just measures it).
size_t layout(DbWork &w, const dbscan_opts &o, char *base) {
    Carver c{base};
    const int64_t n = std::max<int64_t>(o.max_n, 1);
    w.cap_n = n;
    w.cap_d = o.max_d;
    w.dp_cap = dp_for(std::min(o.max_d, 64));
    w.P = c.take<float>((size_t)n * w.dp_cap);
    w.count = c.take<int32_t>(n);
    w.core = c.take<uint8_t>(n);
    w.parent = c.take<int32_t>(n);
    w.border = c.take<int32_t>(n);
    w.scan = c.take<int32_t>(n + 1);
    w.scan_part_cap = n / 2048 + 4;
    w.scan_part = c.take<int32_t>(w.scan_part_cap);
    w.status = c.take<unsigned>(4);
    w.ctr = c.take<unsigned long long>(DB_NCTR);
    const bool grid = o.grid != DBSCAN_GRID_OFF && o.max_d >= 1;
    if (grid) {
        int bits = 10;
        while ((int64_t(1) << bits) < 2 * n) ++bits;
        w.hcap = int64_t(1) << bits;
        w.hbits = bits;
        w.hkey = c.take<uint32_t>(w.hcap);
        w.hcount = c.take<int32_t>(w.hcap);
        w.hpack = c.take<int2>(w.hcap);
        w.occ_cap = std::max<int64_t>(int64_t(1) << 15, 4 * n);
        w.occ = c.take<uint32_t>(w.occ_cap);
        w.hcursor = c.take<int32_t>(w.hcap);
        w.slot_of = c.take<int32_t>(n);
        w.pts4 = c.take<float4>(n);
        w.spts = c.take<float4>(n);
        w.sidx = c.take<int32_t>(n);
        w.scell = c.take<int32_t>(n);
        w.score = c.take<uint8_t>(n);
        w.cell_start = c.take<int32_t>(n);
        w.cell_count = c.take<int32_t>(n);
        w.cell_rep = c.take<int32_t>(n);
        w.cell_mid = c.take<float4>(n);
        w.cell_key = c.take<uint32_t>(n);
        const int dg = std::min(o.max_d, 3);
        w.noff_cap = dg == 1 ? 4 : (dg == 2 ? 24 : 124);
        w.nbr = c.take<int32_t>((size_t)n * w.noff_cap);
        w.ncnt = c.take<int32_t>(n);
        w.cell_cand = c.take<int32_t>(n);
    } else {
        w.hcap = 0;
        w.noff_cap = 0;
        w.occ_cap = 0;
    }
    if (o.max_d >= 16) {
        // one more 256-row tile than n needs: the FP16 count's column list leaves
        // a gap of up to 255 rows between its even-norm and odd-norm points
        const int64_t np = (n + 255) / 256 * 256 + 256;
        w.tc_cap_pad = np;
        w.v16 = c.take<int16_t>((size_t)n * 64);
        w.inorm = c.take<int32_t>(n);
        w.opAll = c.take<uint16_t>((size_t)np * 128);
        w.opCore = c.take<uint16_t>((size_t)np * 128);
        w.opNon = c.take<uint16_t>((size_t)np * 128);
        w.metaAll = c.take<char>((size_t)np * 16);
        w.metaCore = c.take<char>((size_t)np * 16);
        w.metaNon = c.take<char>((size_t)np * 16);
        w.list_a = c.take<int32_t>(np);
        w.list_b = c.take<int32_t>(n);
        w.tc_lens = c.take<int32_t>(8);
    } else {
        w.tc_cap_pad = 0;
    }
    return align_up(c.off, 256);
}

}  // namespace

int plan_status_from_bits(unsigned bits) {
    if (bits & DB_EBIT_NOT_QUANTISED) return DBSCAN_ERR_NOT_QUANTISED;
    if (bits & DB_EBIT_TIMEOUT) return DBSCAN_ERR_TIMEOUT;
    if (bits & DB_EBIT_OVERFLOW) return DBSCAN_ERR_CUDA;
    return DBSCAN_OK;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

int plan_read_status(dbscan_plan *plan, bool clear) {
    cudaStream_t st = plan->stream;
    if (cudaMemcpyAsync(plan->h_status, plan->w.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return DBSCAN_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DBSCAN_ERR_CUDA;
    const unsigned bits = *plan->h_status;
    if (clear && bits && cudaMemsetAsync(plan->w.status, 0, sizeof(unsigned), st) != cudaSuccess)
        return DBSCAN_ERR_CUDA;
    return plan_status_from_bits(bits);
}

int plan_run(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
             int32_t *labels, int32_t *counts_out, uint8_t *core_out, dbscan_stats *stats) {
    if (!plan) return DBSCAN_ERR_ARG;
    const dbscan_opts &o = plan->opts;
    if (n < 0 || n > plan->w.cap_n || d < 1 || d > o.max_d || !(eps > 0.0f) || std::isinf(eps) || min_pts < 1)
        return DBSCAN_ERR_ARG;
    if (n > 0 && (!points || !labels)) return DBSCAN_ERR_ARG;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    const double e = (double)eps;
    const int64_t T = (int64_t)std::floor(e * e * 1048576.0);  // exact: 48-bit square, power-of-two scale
    if (stats) stats->threshold = T;
    if (n == 0) return DBSCAN_OK;
    // Index ranges counted in int32: the eps-grid's hash (at least 2n slots)
    // and the all-pairs work items (row tiles x column chunks).
    constexpr int64_t kGridMaxN = int64_t(1) << 29, kAllPairsMaxN = int64_t(1) << 25;
    const bool grid_path = d <= 8 && o.grid != DBSCAN_GRID_OFF && plan->w.hcap > 0;
    if (grid_path ? n > kGridMaxN : n > kAllPairsMaxN) return DBSCAN_ERR_UNSUPPORTED;
    const int64_t Dmax = (int64_t)d * 1023 * 1023;
    const int64_t Tc = std::min(T, Dmax);  // same predicate: no pair is farther than Dmax

    DeviceGuard dg(o.device);
    cudaStream_t st = plan->stream;
    const bool sync = o.synchronous || stats;
    if (o.synchronous && cudaMemsetAsync(plan->w.status, 0, sizeof(unsigned), st) != cudaSuccess)
        return DBSCAN_ERR_CUDA;
    if (cudaMemsetAsync(plan->w.ctr, 0, sizeof(unsigned long long) * DB_NCTR, st) != cudaSuccess)
        return DBSCAN_ERR_CUDA;
    if (stats) cudaEventRecord(plan->ev0, st);
    plan->marks.begin(st);

    const bool exact = counts_out != nullptr;
    int path;
    GridGeom g;
    cudaError_t err;
    const bool want_grid = d <= 3 && o.grid != DBSCAN_GRID_OFF && plan->w.hcap > 0;
    // the projected grid (4 <= d <= 8) needs the eps-grid's arrays and row stride >= 8 (4 for d = 4)
    const bool want_mid = d >= 4 && d <= 8 && o.grid != DBSCAN_GRID_OFF && plan->w.hcap > 0 &&
                          plan->w.dp_cap >= (d <= 4 ? 4 : 8);
    if (o.grid == DBSCAN_GRID_ON && !(want_grid || want_mid)) return DBSCAN_ERR_UNSUPPORTED;
    if (want_grid && grid_geometry(d, Tc, n, &g)) {
        path = DBSCAN_PATH_GRID;
        err = launch_grid_path(plan->w, g, points, n, min_pts, exact, labels, counts_out, core_out, st);
    } else if (want_mid && mid_geometry(d, Tc, n, &g)) {
        path = DBSCAN_PATH_GRID_PROJECTED;
        err = launch_mid_grid_path(plan->w, g, points, n, d, min_pts, exact, labels, counts_out, core_out, st);
    } else {
        if (o.grid == DBSCAN_GRID_ON) return DBSCAN_ERR_UNSUPPORTED;  // eps too large for the cells to prune
        if (n > kAllPairsMaxN) return DBSCAN_ERR_UNSUPPORTED;
        const bool tc_ok = plan->w.tc_cap_pad > 0 && d <= 64 && Tc < (1 << 24);
        const bool want_tc = o.precision == DBSCAN_PREC_FP16_GRAM || o.precision == DBSCAN_PREC_BF16_GRAM ||
                             (o.precision == DBSCAN_PREC_AUTO && d >= 16 && n >= 4096);
        if (want_tc && !tc_ok) {
            if (o.precision != DBSCAN_PREC_AUTO) return DBSCAN_ERR_UNSUPPORTED;
        }
        if (want_tc && tc_ok) {
            path = DBSCAN_PATH_ALLPAIRS_TC;
            const bool stall = plan->test_hook == DBSCAN_HOOK_TC_STALL;
            plan->test_hook = DBSCAN_HOOK_NONE;  // consumed by this run
            err = launch_allpairs_tc(plan->w, points, n, d, Tc, min_pts, o.precision == DBSCAN_PREC_BF16_GRAM, stall,
                                     st);
        } else {
            const int dp = dp_for(d);
            if (dp < 0) return DBSCAN_ERR_UNSUPPORTED;
            path = DBSCAN_PATH_ALLPAIRS_SIMT;
            err = launch_prep_dense(plan->w, points, n, d, dp, st);
            if (!err) err = launch_allpairs_simt(plan->w, n, d, dp, Tc, min_pts, exact, st);
        }
        if (!err) err = launch_labels_allpairs(plan->w, n, labels, counts_out, core_out, st);
    }
    if (!err && o.label_mode == DBSCAN_LABEL_COMPACT) err = launch_compact(plan->w, n, labels, st);
    if (!err && stats && (path == DBSCAN_PATH_GRID || path == DBSCAN_PATH_GRID_PROJECTED))
        err = launch_grid_candidates(plan->w, g, n, path == DBSCAN_PATH_GRID_PROJECTED, st);
    if (err != cudaSuccess) {
        std::fprintf(stderr, "dbscan: launch failed: %s\n", cudaGetErrorString(err));
        return DBSCAN_ERR_CUDA;
    }
    if (stats) cudaEventRecord(plan->ev1, st);
    if (!sync) return DBSCAN_OK;

    if (cudaMemcpyAsync(plan->h_ctr, plan->w.ctr, sizeof(unsigned long long) * DB_NCTR, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return DBSCAN_ERR_CUDA;
    const int s = plan_read_status(plan, !o.synchronous);
    if (s) return s;
    if (stats) {
        const unsigned long long *c = plan->h_ctr;
        stats->n_core = (int64_t)c[2];
        stats->n_border = (int64_t)c[3];
        stats->n_noise = (int64_t)c[4];
        stats->n_clusters = (int64_t)c[5];
        stats->path = path;
        stats->band_pairs = (int64_t)c[6];
        stats->pair_tests =
            (int64_t)(c[DB_CTR_EVAL] + c[DB_CTR_EVAL + 1] + c[DB_CTR_EVAL + 2] + c[DB_CTR_EVAL + 3]);
        if (path == DBSCAN_PATH_GRID || path == DBSCAN_PATH_GRID_PROJECTED) {
            stats->candidate_pairs = (int64_t)c[1];
            stats->cells = (int32_t)(c[0] >> 32);
        } else {
            stats->candidate_pairs = n * n;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, plan->ev0, plan->ev1);
        stats->ms_total = ms;
        stats->kernels = plan->marks.kernels;
    }
    return DBSCAN_OK;
}

int plan_create_unbound(dbscan_plan **out, const dbscan_opts &o) {
    *out = nullptr;
    if (o.max_n < 0 || o.max_n > INT32_MAX / 2 || o.max_d < 1 || o.max_d > 64) return DBSCAN_ERR_ARG;
    if (o.precision < 0 || o.precision > 3 || o.grid < 0 || o.grid > 2 || o.label_mode < 0 || o.label_mode > 1 ||
        o.profile < 0 || o.profile > 1)
        return DBSCAN_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) return DBSCAN_ERR_CUDA;
    DeviceGuard dg(o.device);
    dbscan_plan *p = new (std::nothrow) dbscan_plan();
    if (!p) return DBSCAN_ERR_OOM;
    p->opts = o;
    p->stream = (cudaStream_t)o.stream;
    p->w.marks = &p->marks;
    if (o.profile) {
        p->marks.on = true;
        bool ok = cudaEventCreate(&p->marks.start) == cudaSuccess;
        for (int i = 0; i < PhaseMarks::kMax && ok; ++i) ok = cudaEventCreate(&p->marks.ev[i]) == cudaSuccess;
        if (!ok) {
            dbscan_plan_destroy(p);
            return DBSCAN_ERR_CUDA;
        }
    }
    if (o.grid != DBSCAN_GRID_OFF) {  // grid path: side stream and fork/join events
        bool ok = cudaStreamCreateWithFlags(&p->w.side, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 4 && ok; ++i)
            ok = cudaEventCreateWithFlags(&p->w.fj[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            dbscan_plan_destroy(p);
            return DBSCAN_ERR_CUDA;
        }
    }
    if (cudaMallocHost(&p->h_status, sizeof(unsigned) * 4) != cudaSuccess ||
        cudaMallocHost(&p->h_ctr, sizeof(unsigned long long) * DB_NCTR) != cudaSuccess ||
        cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess) {
        dbscan_plan_destroy(p);
        return DBSCAN_ERR_CUDA;
    }
    *out = p;
    return DBSCAN_OK;
}

// Layout options for instances up to (n, d): with exact_d, d is the only
// dimension the workspace serves, so the grid arrays are left out for d > 8
// (a plan's max_d is only an upper bound, so plans keep them).
static dbscan_opts layout_opts(const dbscan_opts &o, int64_t n, int32_t d, bool exact_d) {
    dbscan_opts q = o;
    q.max_n = n;
    q.max_d = d;
    if (exact_d && d > 8) q.grid = DBSCAN_GRID_OFF;
    return q;
}

size_t plan_workspace_bytes_for(const dbscan_opts &o, int64_t n, int32_t d, bool exact_d) {
    DbWork w{};
    return layout(w, layout_opts(o, n, d, exact_d), nullptr);
}

int plan_bind_workspace(dbscan_plan *p, void *base, size_t bytes, int64_t n, int32_t d, bool exact_d) {
    if (!p || !base || d < 1 || d > 64 || n < 0) return DBSCAN_ERR_ARG;
    const dbscan_opts q = layout_opts(p->opts, n, d, exact_d);
    if (plan_workspace_bytes_for(p->opts, n, d, exact_d) > bytes) return DBSCAN_ERR_ARG;
    PhaseMarks *marks = p->w.marks;
    cudaStream_t side = p->w.side;
    cudaEvent_t fj[4] = {p->w.fj[0], p->w.fj[1], p->w.fj[2], p->w.fj[3]};
    DbWork w{};
    layout(w, q, static_cast<char *>(base));
    w.marks = marks;
    w.side = side;
    for (int i = 0; i < 4; ++i) w.fj[i] = fj[i];
    p->w = w;
    p->opts.max_n = n;
    p->opts.max_d = d;
    p->ws_base = base;
    p->ws_bytes = bytes;
    DeviceGuard dg(p->opts.device);
    if (cudaMemsetAsync(p->w.status, 0, sizeof(unsigned), p->stream) != cudaSuccess) return DBSCAN_ERR_CUDA;
    if (p->owns_ws && cudaStreamSynchronize(p->stream) != cudaSuccess) return DBSCAN_ERR_CUDA;
    return DBSCAN_OK;
}

extern "C" {

void dbscan_opts_default(dbscan_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->device = 0;
    o->synchronous = 1;
    o->stream = nullptr;
    o->max_n = 1 << 20;
    o->max_d = 64;
    o->precision = DBSCAN_PREC_AUTO;
    o->grid = DBSCAN_GRID_AUTO;
    o->label_mode = DBSCAN_LABEL_ROOT_INDEX;
}

int dbscan_plan_create(dbscan_plan **out, const dbscan_opts *opts) {
    if (!out) return DBSCAN_ERR_ARG;
    *out = nullptr;
    dbscan_opts o;
    if (opts) o = *opts;
    else dbscan_opts_default(&o);
    dbscan_plan *p = nullptr;
    int rc = plan_create_unbound(&p, o);
    if (rc) return rc;
    DeviceGuard dg(o.device);
    const size_t bytes = plan_workspace_bytes_for(o, o.max_n, o.max_d, false);
    void *base = nullptr;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        dbscan_plan_destroy(p);
        return DBSCAN_ERR_OOM;
    }
    p->owns_ws = true;
    if ((rc = plan_bind_workspace(p, base, bytes, o.max_n, o.max_d, false)) != DBSCAN_OK) {
        dbscan_plan_destroy(p);
        return rc;
    }
    *out = p;
    return DBSCAN_OK;
}

int dbscan_plan_destroy(dbscan_plan *p) {
    if (!p) return DBSCAN_OK;
    DeviceGuard dg(p->opts.device);
    cudaStreamSynchronize(p->stream);
    plan_release_extras(p);
    if (p->ws_base && p->owns_ws) cudaFree(p->ws_base);
    if (p->h_status) cudaFreeHost(p->h_status);
    if (p->h_ctr) cudaFreeHost(p->h_ctr);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->marks.start) cudaEventDestroy(p->marks.start);
    for (int i = 0; i < PhaseMarks::kMax; ++i)
        if (p->marks.ev[i]) cudaEventDestroy(p->marks.ev[i]);
    if (p->w.side) cudaStreamSynchronize(p->w.side);
    for (int i = 0; i < 4; ++i)
        if (p->w.fj[i]) cudaEventDestroy(p->w.fj[i]);
    if (p->w.side) cudaStreamDestroy(p->w.side);
    delete p;
    return DBSCAN_OK;
}

int dbscan_run(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
               int32_t *labels_out, dbscan_stats *stats) {
    return plan_run(plan, points, n, d, eps, min_pts, labels_out, nullptr, nullptr, stats);
}

int dbscan_run_detail(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t min_pts,
                      int32_t *labels_out, int32_t *counts_out, uint8_t *core_out, dbscan_stats *stats) {
    return plan_run(plan, points, n, d, eps, min_pts, labels_out, counts_out, core_out, stats);
}

int dbscan_run_host(dbscan_plan *plan, const float *host_points, int64_t n, int32_t d, float eps, int32_t min_pts,
                    int32_t *host_labels, dbscan_stats *stats) {
    if (!plan) return DBSCAN_ERR_ARG;
    if (n < 0 || n > plan->w.cap_n || d < 1 || d > plan->opts.max_d) return DBSCAN_ERR_ARG;
    if (n > 0 && (!host_points || !host_labels)) return DBSCAN_ERR_ARG;
    if (n == 0) return plan_run(plan, nullptr, 0, d, eps, min_pts, nullptr, nullptr, nullptr, stats);
    DeviceGuard dg(plan->opts.device);
    int s = plan_ensure_staging(plan, n, d);
    if (s) return s;
    cudaStream_t st = plan->stream;
    if (cudaMemcpyAsync(plan->stage_in, host_points, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return DBSCAN_ERR_CUDA;
    s = plan_run(plan, plan->stage_in, n, d, eps, min_pts, plan->stage_out, nullptr, nullptr, stats);
    if (s) return s;
    if (cudaMemcpyAsync(host_labels, plan->stage_out, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return DBSCAN_ERR_CUDA;
    return plan_read_status(plan, true);
}

int dbscan_plan_sync(dbscan_plan *plan) {
    if (!plan) return DBSCAN_ERR_ARG;
    DeviceGuard dg(plan->opts.device);
    return plan_read_status(plan, true);
}

int dbscan_plan_phase_times(dbscan_plan *plan, int32_t max_phases, float *ms, const char **names, int32_t *count) {
    if (!plan || max_phases < 0) return DBSCAN_ERR_ARG;
    if (count) *count = 0;
    if (!plan->marks.on) return DBSCAN_ERR_UNSUPPORTED;
    DeviceGuard dg(plan->opts.device);
    if (cudaStreamSynchronize(plan->stream) != cudaSuccess) return DBSCAN_ERR_CUDA;
    const int k = std::min<int>(plan->marks.n, max_phases);
    for (int i = 0; i < k; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, i ? plan->marks.ev[i - 1] : plan->marks.start, plan->marks.ev[i]) != cudaSuccess)
            return DBSCAN_ERR_CUDA;
        if (ms) ms[i] = t;
        if (names) names[i] = plan->marks.name[i];
    }
    if (count) *count = plan->marks.n;
    return DBSCAN_OK;
}

int dbscan_tc_verify(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps, int32_t bf16,
                     dbscan_tc_report *out) {
    if (!plan || !out || !points || n < 1 || n > plan->w.cap_n || d < 1 || d > 64 || !(eps > 0.0f) ||
        std::isinf(eps))
        return DBSCAN_ERR_ARG;
    if (plan->w.tc_cap_pad == 0) return DBSCAN_ERR_UNSUPPORTED;
    const double e = (double)eps;
    const int64_t T = std::min<int64_t>((int64_t)std::floor(e * e * 1048576.0), (int64_t)d * 1023 * 1023);
    if (T >= (1 << 24)) return DBSCAN_ERR_UNSUPPORTED;
    DeviceGuard dg(plan->opts.device);
    cudaStream_t st = plan->stream;
    if (cudaMemsetAsync(plan->w.ctr, 0, sizeof(unsigned long long) * DB_NCTR, st) != cudaSuccess)
        return DBSCAN_ERR_CUDA;
    if (cudaMemsetAsync(plan->w.status, 0, sizeof(unsigned), st) != cudaSuccess) return DBSCAN_ERR_CUDA;
    if (launch_tc_verify(plan->w, points, n, d, T, bf16 != 0, st) != cudaSuccess) return DBSCAN_ERR_CUDA;
    if (cudaMemcpyAsync(plan->h_ctr, plan->w.ctr, sizeof(unsigned long long) * DB_NCTR, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return DBSCAN_ERR_CUDA;
    const int s = plan_read_status(plan, true);
    if (s) return s;
    out->pairs = n * n;
    out->band_pairs = (int64_t)plan->h_ctr[6];
    out->wrong_outside_band = (int64_t)plan->h_ctr[7];
    out->max_abs_error_2g = (int64_t)plan->h_ctr[8];
    out->band_halfwidth_2g = bf16 ? 16 * ((d + 15) / 16 * 16) : 0;  // 16 K for the two BF16 terms
    out->threshold = T;
    return DBSCAN_OK;
}

int dbscan_plan_counters(dbscan_plan *plan, uint64_t *out, int32_t n) {
    if (!plan || !out || n < 0) return DBSCAN_ERR_ARG;
    DeviceGuard dg(plan->opts.device);
    const int k = std::min(n, DB_NCTR);
    if (cudaMemcpyAsync(plan->h_ctr, plan->w.ctr, sizeof(unsigned long long) * DB_NCTR, cudaMemcpyDeviceToHost,
                        plan->stream) != cudaSuccess ||
        cudaStreamSynchronize(plan->stream) != cudaSuccess)
        return DBSCAN_ERR_CUDA;
    for (int i = 0; i < k; ++i) out[i] = plan->h_ctr[i];
    return DBSCAN_OK;
}

int dbscan_plan_test_hook(dbscan_plan *plan, int32_t hook) {
    if (!plan || hook < DBSCAN_HOOK_NONE || hook > DBSCAN_HOOK_TC_STALL) return DBSCAN_ERR_ARG;
    plan->test_hook = hook;
    return DBSCAN_OK;
}

int64_t dbscan_plan_workspace_bytes(const dbscan_plan *plan) {
    return plan ? (int64_t)(plan->ws_bytes + plan->extra_bytes) : 0;
}

const char *dbscan_strerror(int s) {
    switch (s) {
        case DBSCAN_OK: return "ok";
        case DBSCAN_ERR_ARG: return "invalid argument";
        case DBSCAN_ERR_NOT_QUANTISED: return "a coordinate is not a multiple of 2^-10 in [0,1)";
        case DBSCAN_ERR_OOM: return "out of memory";
        case DBSCAN_ERR_CUDA: return "CUDA error";
        case DBSCAN_ERR_TIMEOUT: return "bounded wait expired";
        case DBSCAN_ERR_BUSY: return "admission full";
        case DBSCAN_ERR_UNSUPPORTED: return "unsupported option or shape";
        case DBSCAN_ERR_NOT_FOUND: return "unknown job id";
        default: return "unknown status";
    }
}

int32_t dbscan_abi_version(void) { return DBSCAN_ABI_VERSION; }

}  // extern "C"
