// internal.cuh — shared device helpers and launch declarations of libdbscan_gb300.
//
// Notation follows the paper (Wang et al., Sections II and IV): a point p has
// grid units u_p (integers 0..1023), T = floor(eps^2 * 2^20) and q is an
// eps-neighbour of p iff D(p,q) = sum_k (u_pk - u_qk)^2 <= T.
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include "dbscan.h"  // include/ is on the include path

// Device-side error bits, OR-ed into the plan's status word.
#define DB_EBIT_NOT_QUANTISED 1u
#define DB_EBIT_TIMEOUT 2u     // a bounded loop gave up
#define DB_EBIT_OVERFLOW 4u    // a device-side list ran out of room

#define DB_NONE 0x7fffffff     // "no index" (larger than every point index)

// Device counters of a run (DbWork::ctr, DB_NCTR 64-bit slots):
//   0 grid cells|points, 1 grid candidate pairs, 2..5 core/border/noise/clusters,
//   6 band pairs rechecked, 7..8 band verification, 9..13 and 20..29 pipeline
//   diagnostics of the tensor-core count, merge and border passes,
//   15 FP16 tensor-core count ran the folded form (1),
//   16..19 pair tests evaluated by the count, merge, border and (grid path)
//   outer-ring merge passes, 31 work items of the projected grid (int).
#define DB_NCTR 32
#define DB_CTR_EVAL 16
#define DB_CTR_TC_FOLD 15      // 1: the FP16 count ran the folded form
#define DB_CTR_MID_ITEMS 31
#define DB_HASH_EMPTY 0xffffffffu

namespace db {

// ---------------------------------------------------------------------------
// Relaxed, L1-bypassing accesses for data other threads update concurrently.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(int *p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Lock-free union-find over point indices (replaces the paper's per-target
// merge kernel of Section IV-C).  Invariant: parent[x] <= x, and a root is the
// smallest index of its set, because union always links the larger root under
// the smaller one.  Path halving writes only ancestors, so concurrent halving
// and linking keep the invariant.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int uf_find(int *parent, int x) {
    while (true) {
        int p = ld_relaxed(parent + x);
        if (p == x) return x;
        int gp = ld_relaxed(parent + p);
        if (gp == p) return p;
        st_relaxed(parent + x, gp);
        x = gp;
    }
}

// Union of the sets of a and b.  Each failed CAS means another thread linked
// the root first, so the loop makes global progress; the cap only guards
// against a corrupted forest and reports it.
__device__ __forceinline__ void uf_unite(int *parent, int a, int b, unsigned *status) {
    for (int it = 0; it < (1 << 24); ++it) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a > b) {
            int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(parent + b, b, a) == b) return;
    }
    atomicOr(status, DB_EBIT_TIMEOUT);
}

// Union that also returns a root of the merged set (a hint for callers that
// cache it: the value is the set's root at some moment, so any point whose
// parent equals it is in the set).
__device__ __forceinline__ int uf_unite_root(int *parent, int a, int b, unsigned *status) {
    for (int it = 0; it < (1 << 24); ++it) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return a;
        if (a > b) {
            int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(parent + b, b, a) == b) return a;
    }
    atomicOr(status, DB_EBIT_TIMEOUT);
    return -1;
}

// Cell hash slot of the grid paths: four consecutive keys (four cells in a
// row along x) share one 32-byte bucket of the packed table, so the lookups of
// a cell's x-neighbours, made by neighbouring lanes, touch few sectors.
__device__ __forceinline__ unsigned hash_slot(unsigned key, int bits) {
    return ((((key >> 2) * 2654435761u) >> (34 - bits)) << 2) | (key & 3u);
}

// 2^-10 grid check of one coordinate: finite, 0 <= x < 1, 1024 x integral.
__device__ __forceinline__ bool on_grid(float x, int &u) {
    float s = x * 1024.0f;  // exact: scaling by a power of two
    bool ok = (x >= 0.0f) && (x < 1.0f) && (s == floorf(s));
    u = ok ? (int)s : 0;
    return ok;
}

// Sum of v over the block added to *dst by one global atomic.  Every thread
// of the block must call it (it synchronises the block).
__device__ __forceinline__ void block_sum_add(unsigned long long *dst, unsigned long long v) {
    __shared__ unsigned long long part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += part[w];
        if (t) atomicAdd(dst, t);
    }
}

// Programmatic dependent launch.  A kernel started with launch_dependent()
// may be scheduled while the kernel before it in its stream still runs: it
// calls wait_prior_grid() before touching memory, which returns once that
// kernel has completed and its writes are visible (at once for a kernel
// started the plain way).  allow_next_grid() lets the next such kernel of the
// stream be scheduled early; it still waits for this one to complete.  A
// chain of short dependent kernels then overlaps each launch with the tail of
// the kernel before it.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace db

// Starts kern on st as a programmatic dependent of the previous kernel in st
// (kern must call db::wait_prior_grid() before its first memory access).
template <typename... P, typename... A>
inline cudaError_t launch_dependent(void (*kern)(P...), dim3 grid, dim3 block, cudaStream_t st, A &&...args) {
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// ---------------------------------------------------------------------------
// Per-kernel timing: when on, a CUDA event is recorded on the launch stream
// after every kernel, so kernel i took elapsed(ev[i-1] or start, ev[i]).
// ---------------------------------------------------------------------------
struct PhaseMarks {
    static constexpr int kMax = 32;
    bool on = false;
    int n = 0;
    int kernels = 0;
    cudaEvent_t start = nullptr;
    cudaEvent_t ev[kMax] = {};
    const char *name[kMax] = {};
    void begin(cudaStream_t st) {
        n = 0;
        kernels = 0;
        if (on) cudaEventRecord(start, st);
    }
    void kernel(const char *nm, cudaStream_t st) {
        ++kernels;
        if (on && n < kMax) {
            cudaEventRecord(ev[n], st);
            name[n++] = nm;
        }
    }
};

// ---------------------------------------------------------------------------
// Workspace of one clustering run (device pointers carved from one allocation).
// ---------------------------------------------------------------------------
struct DbWork {
    int64_t cap_n;
    int32_t cap_d;
    int32_t dp_cap;         // padded row stride capacity of P
    // all paths
    float *P;               // packed grid units, row stride DP (all-pairs) [cap_n * dp_cap]
    int32_t *count;         // neighbour counts by point index [cap_n]
    uint8_t *core;          // core flags by point index [cap_n]
    int32_t *parent;        // union-find forest by point index [cap_n]
    int32_t *border;        // smallest core neighbour of non-core points [cap_n]
    int32_t *scan;          // exclusive-scan output [cap_n + 1]
    int32_t *scan_part;     // scan partials
    int64_t scan_part_cap;
    unsigned *status;       // device error bits
    unsigned long long *ctr;  // DB_NCTR counters (slots listed beside DB_NCTR)
    // grid path
    int64_t hcap;           // hash slots (power of two >= 2 cap_n)
    int32_t hbits;
    uint32_t *hkey;
    int32_t *hcount;
    int2 *hpack;            // cell hash: {key, cell id} (written after the inserts) [hcap]
    uint32_t *occ;          // occupancy bitmap of all G^d cells, when it fits [occ_cap]
    int64_t occ_cap;        // words (128 bits per point, at least 2^20 bits)
    int32_t *hcursor;
    int32_t *slot_of;       // hash slot of each point [cap_n]
    float4 *pts4;           // {u0,u1,u2,-|u|^2} by point index [cap_n]
    float4 *spts;           // same, grouped by cell [cap_n]
    int32_t *sidx;          // point index of each grouped position [cap_n]
    int32_t *scell;         // cell id of each grouped position [cap_n]
    uint8_t *score;         // core flag of each grouped position [cap_n]
    int32_t *cell_start, *cell_count, *cell_rep;  // [cap_n]
    float4 *cell_mid;       // a core point near each cell's centre [cap_n]
    uint32_t *cell_key;     // [cap_n]
    int32_t *nbr;           // neighbour cell lists, adjacent first [cap_n * noff_cap]
    int32_t *ncnt;          // (adjacent count << 16) | count [cap_n]
    int32_t *cell_cand;     // points in the cells of each neighbour list [cap_n]
    int32_t noff_cap;
    // tensor-core path (max_d >= 16)
    int64_t tc_cap_pad;     // rows of each packed operand (cap_n rounded up to 256, plus 256)
    int16_t *v16;           // centred units v = u - 512 by point index, row stride 64
    int32_t *inorm;         // exact |v|^2 [cap_n]
    uint16_t *opAll, *opCore, *opNon;  // packed FP16 or two-term BF16 operand tiles [tc_cap_pad * 128]
    void *metaAll, *metaCore, *metaNon;  // per-point metadata blocks (16 B per row)
    int32_t *list_a, *list_b;  // core / non-core index lists [tc_cap_pad], [cap_n]
    // [0] cores, [1] non-cores, [2] all, [3] largest |v|^2, [4] even-norm points,
    // [5] length of the FP16 count's column list (even points, gap, odd points)
    int32_t *tc_lens;
    PhaseMarks *marks;      // host-side timing marks of the owning plan
    // second stream of the grid path: independent kernels run beside each
    // other (fork/join by events); unused while per-kernel marks are taken
    cudaStream_t side;
    cudaEvent_t fj[4];
};

// Host-side grid geometry for d <= 3 (see grid.cu).
struct GridGeom {
    int32_t d, c, G, Tc, noff, nnear, hbits;
    int32_t dense;  // 1: cells indexed directly by key (slot = key, G^d slots), 0: hashed (2^hbits slots)
    float Tp1;
    float inv_c;    // 1/c rounded to FP32: floor((u + 1/2) * inv_c) = floor(u / c) for 0 <= u < 2^11
    char4 off[124];
};

// ---- launchers (all enqueue on `st`; return cudaError_t of the launch) ----
cudaError_t launch_prep_dense(const DbWork &w, const float *x, int64_t n, int32_t d, int32_t dp, cudaStream_t st);
cudaError_t launch_allpairs_simt(const DbWork &w, int64_t n, int32_t d, int32_t dp, int64_t Tc, int32_t min_pts,
                                 bool exact_counts, cudaStream_t st);
cudaError_t launch_core_init(const DbWork &w, int64_t n, int32_t min_pts, cudaStream_t st);
cudaError_t launch_allpairs_tc(const DbWork &w, const float *x, int64_t n, int32_t d, int64_t Tc, int32_t min_pts,
                               bool bf16, bool stall, cudaStream_t st);
cudaError_t launch_tc_verify(const DbWork &w, const float *x, int64_t n, int32_t d, int64_t Tc, bool bf16,
                             cudaStream_t st);
cudaError_t launch_labels_allpairs(const DbWork &w, int64_t n, int32_t *labels, int32_t *counts_out,
                                   uint8_t *core_out, cudaStream_t st);
cudaError_t launch_compact(const DbWork &w, int64_t n, int32_t *labels, cudaStream_t st);
cudaError_t launch_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *part, int64_t part_cap,
                                  cudaStream_t st, PhaseMarks *pm);
bool grid_geometry(int32_t d, int64_t Tc, int64_t n, GridGeom *g);
cudaError_t launch_grid_path(const DbWork &w, const GridGeom &g, const float *x, int64_t n, int32_t min_pts,
                             bool exact_counts, int32_t *labels, int32_t *counts_out, uint8_t *core_out,
                             cudaStream_t st);
// Ordered candidate pairs of a grid run (own cell listed: the projected grid).
cudaError_t launch_grid_candidates(const DbWork &w, const GridGeom &g, int64_t n, bool own_cell_listed,
                                   cudaStream_t st);
// Structure kernels shared by the eps-grid and the projected grid (grid_mid.cu):
// occupied slots -> cell table (ids, ranges, keys, occupancy bits), and the
// neighbour-cell lists of g's offsets.
cudaError_t launch_grid_cells(const DbWork &w, const GridGeom &g, unsigned *occ, unsigned long long *midkey,
                              cudaStream_t st);
cudaError_t launch_grid_nbrs(const DbWork &w, const GridGeom &g, const unsigned *occ, cudaStream_t st);
// Projected grid for 4 <= d <= 8 (grid_mid.cu): geometry (false when the
// cells would be too coarse to prune) and the whole path.
bool mid_geometry(int32_t d, int64_t Tc, int64_t n, GridGeom *g);
cudaError_t launch_mid_grid_path(const DbWork &w, const GridGeom &g, const float *x, int64_t n, int32_t d,
                                 int32_t min_pts, bool exact_counts, int32_t *labels, int32_t *counts_out,
                                 uint8_t *core_out, cudaStream_t st);
cudaError_t launch_stats(const DbWork &w, int64_t n, const int32_t *labels, cudaStream_t st);
int32_t dp_for(int32_t d);
