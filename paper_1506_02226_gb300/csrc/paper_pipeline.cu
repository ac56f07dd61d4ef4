// paper_pipeline.cu — the paper's own GPU pipeline, kept as a comparison variant.
//
// Section IV builds DBSCAN from three kernels over materialised matrices:
//   distance   the N x N matrix of squared distances (Section IV-A: a thread
//              per row, coalesced writes, the row tile staged in shared
//              memory, the inner loop unrolled);
//   primitive  the `cluster` matrix, cluster[i][j] = 1 iff point j lies in the
//              eps-neighbourhood of point i, and the `valid` vector, valid[i]
//              = 1 iff point i is core (Section IV-B);
//   merge      one launch per target cluster t: every block takes one other
//              valid cluster c and, if the two can be merged, ORs row c into
//              row t and clears valid[c] (Section IV-C; entries only go from 0
//              to 1, so concurrent ORs need no atomics).
// This library's main path never stores either matrix; this variant exists to
// measure the paper's design on the same hardware and inputs.
//
// Readings.  The squared distance is the exact integer D(p,q) of the 2^-10
// grid units (FP32 holds it exactly for d <= 16) and the neighbour test is
// D <= T; a point counts itself, and core means count >= min_pts (Section II).
// Two clusters merge iff some core point lies in both rows: it is an
// eps-neighbour of a core of each, so both belong to one DBSCAN cluster.  The
// paper does not say how often the targets are visited; merges made in one
// launch can enable others, so the sweep over all targets repeats until a
// sweep merges nothing.  Labels then follow this library's canonical form: a
// core point takes the smallest core index of its merged row, a non-core
// point the label of its smallest-index core neighbour, noise -1.
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace {

constexpr int PP_TPB = 128;  // threads per block of the distance kernel (TPB in Section IV-A)

// Distance matrix: a thread per point i keeps its coordinates in registers; the
// block stages PP_TPB points at a time in shared memory.  The matrix is
// symmetric, so thread i writes entry i of row j (column i), which is
// coalesced across the block.
template <int DP>
__global__ void __launch_bounds__(PP_TPB) pp_distance_kernel(const float *__restrict__ x, int n, int d,
                                                             float *__restrict__ dist, unsigned *status) {
    __shared__ float tile[DP][PP_TPB];
    const int i = blockIdx.x * PP_TPB + threadIdx.x;
    float t[DP];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        int u = 0;
        if (i < n && k < d) ok &= db::on_grid(x[(size_t)i * d + k], u);
        t[k] = (float)u;
    }
    if (!ok) atomicOr(status, DB_EBIT_NOT_QUANTISED);
    for (int j0 = 0; j0 < n; j0 += PP_TPB) {
        __syncthreads();
        const int jl = j0 + threadIdx.x;
#pragma unroll
        for (int k = 0; k < DP; ++k) {
            int u = 0;
            if (jl < n && k < d) db::on_grid(x[(size_t)jl * d + k], u);
            tile[k][threadIdx.x] = (float)u;
        }
        __syncthreads();
        if (i >= n) continue;
        const int m = min(PP_TPB, n - j0);
#pragma unroll 8
        for (int jj = 0; jj < m; ++jj) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
                const float df = t[k] - tile[k][jj];
                s = fmaf(df, df, s);  // exact: integers below 16 * 1023^2 < 2^24
            }
            dist[(size_t)(j0 + jj) * n + i] = s;  // symmetric: column i of row j0 + jj
        }
    }
}

// Primitive clusters: a thread per point i scans column i of the distance
// matrix and writes column i of `cluster` (both coalesced across the block);
// before any merge the matrix is symmetric, so column i is also row i, the
// eps-neighbourhood of point i.  valid[i] = (count >= min_pts).
__global__ void pp_primitive_kernel(int n, const float *__restrict__ dist, float T, int min_pts,
                                    uint8_t *__restrict__ cluster, uint8_t *__restrict__ valid,
                                    uint8_t *__restrict__ core) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
        const bool nb = dist[(size_t)j * n + i] <= T;
        cluster[(size_t)j * n + i] = nb;
        cnt += nb;
    }
    valid[i] = cnt >= min_pts;
    core[i] = cnt >= min_pts;
}

// One merge launch for target t: each block tries clusters c (block-strided
// over all rows).  A core point in both rows means the clusters merge; row c
// is then ORed into row t and valid[c] cleared.
__global__ void pp_merge_kernel(int n, int t, uint8_t *cluster, uint8_t *valid, const uint8_t *__restrict__ core,
                                int *changed) {
    __shared__ int hit;
    if (!valid[t]) return;  // merged into an earlier target during this sweep
    uint8_t *rt = cluster + (size_t)t * n;
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        if (c == t || !valid[c]) continue;  // block-uniform
        __syncthreads();
        if (threadIdx.x == 0) hit = 0;
        __syncthreads();
        const uint8_t *rc = cluster + (size_t)c * n;
        int mine = 0;
        for (int j = threadIdx.x; j < n && !mine; j += blockDim.x) mine = rc[j] && rt[j] && core[j];
        if (mine) hit = 1;
        __syncthreads();
        if (!hit) continue;
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            if (rc[j]) rt[j] = 1;
        if (threadIdx.x == 0) {
            valid[c] = 0;
            *changed = 1;
        }
    }
}

// Labels: a core point takes the smallest core index of the valid row that
// holds it (exactly one does once no sweep merges anything); a non-core point
// the label of its smallest-index core neighbour (its own row is its
// neighbourhood: non-core rows are never merged into).
__global__ void pp_root_kernel(int n, const uint8_t *__restrict__ cluster, const uint8_t *__restrict__ valid,
                               const uint8_t *__restrict__ core, int *__restrict__ root) {
    // one block per valid row: its smallest core member, written to every core member
    __shared__ int best;
    const int t = blockIdx.x;
    if (!valid[t]) return;
    if (threadIdx.x == 0) best = INT_MAX;
    __syncthreads();
    const uint8_t *r = cluster + (size_t)t * n;
    int m = INT_MAX;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        if (r[j] && core[j]) m = min(m, j);
    atomicMin(&best, m);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        if (r[j] && core[j]) root[j] = best;
}

__global__ void pp_label_kernel(int n, const uint8_t *__restrict__ cluster, const uint8_t *__restrict__ core,
                                const int *__restrict__ root, int *__restrict__ labels, unsigned long long *ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lab = -1, kind = 2;
    if (core[i]) {
        lab = root[i];
        kind = 0;
    } else {
        const uint8_t *r = cluster + (size_t)i * n;
        for (int j = 0; j < n; ++j)
            if (r[j] && core[j]) {
                lab = root[j];
                kind = 1;
                break;
            }
    }
    labels[i] = lab;
    atomicAdd(ctr + 2 + kind, 1ull);
    if (kind == 0 && lab == i) atomicAdd(ctr + 5, 1ull);
}

}  // namespace

size_t paper_pipeline_bytes(int64_t n) {
    const size_t nn = (size_t)n * (size_t)n;
    return nn * sizeof(float) + nn + 3 * (size_t)n + sizeof(int) * (size_t)n + 256 * 4;
}

// The three stages on `st`, each phase marked (plan profiling); base holds
// paper_pipeline_bytes(n) bytes.  Returns the number of merge sweeps in *sweeps.
cudaError_t launch_paper_pipeline(const DbWork &w, void *base, const float *x, int64_t n64, int32_t d, int64_t Tc,
                                  int32_t min_pts, int32_t *labels, int *sweeps, cudaStream_t st) {
    const int n = (int)n64;
    char *p = static_cast<char *>(base);
    const size_t nn = (size_t)n * (size_t)n;
    float *dist = reinterpret_cast<float *>(p);
    uint8_t *cluster = reinterpret_cast<uint8_t *>(p + nn * sizeof(float));
    uint8_t *valid = cluster + nn;
    uint8_t *core = valid + n;
    int *root = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(core + n) + 15) & ~uintptr_t(15));
    int *changed = root + n;
    int *h_changed = nullptr;
    cudaError_t e;
    const int nb = (n + PP_TPB - 1) / PP_TPB;
    if (d <= 4) pp_distance_kernel<4><<<nb, PP_TPB, 0, st>>>(x, n, d, dist, w.status);
    else if (d <= 8) pp_distance_kernel<8><<<nb, PP_TPB, 0, st>>>(x, n, d, dist, w.status);
    else pp_distance_kernel<16><<<nb, PP_TPB, 0, st>>>(x, n, d, dist, w.status);
    w.marks->kernel("pp_distance", st);
    pp_primitive_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, dist, (float)Tc, min_pts, cluster, valid, core);
    w.marks->kernel("pp_primitive", st);
    if ((e = cudaGetLastError())) return e;
    uint8_t *h_valid = nullptr;
    if ((e = cudaMallocHost(&h_changed, sizeof(int)))) return e;
    if ((e = cudaMallocHost(&h_valid, (size_t)n))) {
        cudaFreeHost(h_changed);
        return e;
    }
    const int mgrid = std::min(n, 152 * 8);
    int s = 0;
    for (;; ++s) {  // sweeps over the targets valid at the sweep's start, until one merges nothing
        if ((e = cudaMemsetAsync(changed, 0, sizeof(int), st))) break;
        if ((e = cudaMemcpyAsync(h_valid, valid, (size_t)n, cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        for (int t = 0; t < n; ++t)
            if (h_valid[t]) pp_merge_kernel<<<mgrid, 128, 0, st>>>(n, t, cluster, valid, core, changed);
        if ((e = cudaMemcpyAsync(h_changed, changed, sizeof(int), cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        if (!*h_changed || s > n) break;
    }
    cudaFreeHost(h_changed);
    cudaFreeHost(h_valid);
    if (e) return e;
    w.marks->kernel("pp_merge", st);
    *sweeps = s + 1;
    pp_root_kernel<<<n, 256, 0, st>>>(n, cluster, valid, core, root);
    w.marks->kernel("pp_root", st);
    pp_label_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, cluster, core, root, labels, w.ctr);
    w.marks->kernel("pp_label", st);
    return cudaGetLastError();
}

#include <cmath>
#include <cstring>

#include "plan.h"

extern "C" int dbscan_run_paper(dbscan_plan *plan, const float *points, int64_t n, int32_t d, float eps,
                                int32_t min_pts, int32_t *labels_out, dbscan_stats *stats) {
    if (!plan) return DBSCAN_ERR_ARG;
    if (n < 0 || n > plan->w.cap_n || n > DBSCAN_PAPER_MAX_N || d < 1 || d > 16 || d > plan->opts.max_d ||
        !(eps > 0.0f) || std::isinf(eps) || min_pts < 1)
        return DBSCAN_ERR_ARG;
    if (n > 0 && (!points || !labels_out)) return DBSCAN_ERR_ARG;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    const double e = (double)eps;
    const int64_t T = (int64_t)std::floor(e * e * 1048576.0);
    const int64_t Tc = std::min<int64_t>(T, (int64_t)d * 1023 * 1023);
    if (stats) stats->threshold = T;
    if (n == 0) return DBSCAN_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != plan->opts.device) cudaSetDevice(plan->opts.device);
    cudaStream_t st = plan->stream;
    int rc = DBSCAN_OK;
    const size_t need = paper_pipeline_bytes(n);
    if (plan->pp_bytes < need) {
        if (plan->pp_buf) cudaFree(plan->pp_buf);
        plan->extra_bytes -= plan->pp_bytes;
        plan->pp_buf = nullptr;
        plan->pp_bytes = 0;
        if (cudaMalloc(&plan->pp_buf, need) != cudaSuccess) {
            cudaGetLastError();
            plan->pp_buf = nullptr;
            rc = DBSCAN_ERR_OOM;
        } else {
            plan->pp_bytes = need;
            plan->extra_bytes += need;
        }
    }
    int sweeps = 0;
    if (!rc) {
        cudaError_t err = cudaMemsetAsync(plan->w.status, 0, sizeof(unsigned), st);
        if (!err) err = cudaMemsetAsync(plan->w.ctr, 0, sizeof(unsigned long long) * DB_NCTR, st);
        if (!err) err = cudaEventRecord(plan->ev0, st);
        plan->marks.begin(st);
        if (!err) err = launch_paper_pipeline(plan->w, plan->pp_buf, points, n, d, Tc, min_pts, labels_out, &sweeps, st);
        if (!err && plan->opts.label_mode == DBSCAN_LABEL_COMPACT) err = launch_compact(plan->w, n, labels_out, st);
        if (!err) err = cudaEventRecord(plan->ev1, st);
        if (!err) err = cudaMemcpyAsync(plan->h_ctr, plan->w.ctr, sizeof(unsigned long long) * DB_NCTR,
                                        cudaMemcpyDeviceToHost, st);
        if (err != cudaSuccess) {
            cudaGetLastError();
            rc = DBSCAN_ERR_CUDA;
        } else {
            rc = plan_read_status(plan, true);
        }
    }
    if (!rc && stats) {
        const unsigned long long *c = plan->h_ctr;
        stats->n_core = (int64_t)c[2];
        stats->n_border = (int64_t)c[3];
        stats->n_noise = (int64_t)c[4];
        stats->n_clusters = (int64_t)c[5];
        stats->path = DBSCAN_PATH_PAPER;
        stats->candidate_pairs = n * n;
        stats->pair_tests = n * n;
        stats->cells = sweeps;  // merge sweeps over the targets (the field is free on this path)
        float ms = 0.f;
        cudaEventElapsedTime(&ms, plan->ev0, plan->ev1);
        stats->ms_total = ms;
        stats->kernels = plan->marks.kernels;
    }
    if (prev >= 0 && prev != plan->opts.device) cudaSetDevice(prev);
    return rc;
}
