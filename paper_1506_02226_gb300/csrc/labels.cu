// labels.cu — finishing the merge step: labels from the union-find forest,
// optional compaction of cluster ids, an exclusive scan, and run statistics.
//
// After every core-core eps-edge has been united (Section II definition 3;
// Section IV-C's merge), the root of a core point's set is the smallest core
// index of its cluster.  A border point takes the root of its smallest-index
// core neighbour; everything else is noise (-1).  The paper's `valid` vector
// (Section IV-B) corresponds to "is a root" here.
#include <climits>

#include "internal.cuh"

namespace {

constexpr int SCAN_NT = 256, SCAN_IPT = 8, SCAN_TILE = SCAN_NT * SCAN_IPT;

__device__ __forceinline__ int block_sum(int v, int *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    int t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

__global__ void labels_allpairs_kernel(int n, const uint8_t *__restrict__ core, int *parent,
                                       const int *__restrict__ border, const int *__restrict__ count,
                                       int *__restrict__ labels, int *__restrict__ counts_out,
                                       uint8_t *__restrict__ core_out, unsigned long long *ctr) {
    __shared__ int red[32];
    int nc = 0, nb = 0, nn = 0, nr = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lab;
        const bool c = core[i];
        if (c) {
            lab = db::uf_find(parent, i);
            ++nc;
            nr += (lab == i);
        } else if (border[i] != DB_NONE) {
            lab = db::uf_find(parent, border[i]);
            ++nb;
        } else {
            lab = -1;
            ++nn;
        }
        labels[i] = lab;
        if (counts_out) counts_out[i] = count[i];
        if (core_out) core_out[i] = c;
    }
    nc = block_sum(nc, red);
    nb = block_sum(nb, red);
    nn = block_sum(nn, red);
    nr = block_sum(nr, red);
    if (threadIdx.x == 0) {
        if (nc) atomicAdd(ctr + 2, (unsigned long long)nc);
        if (nb) atomicAdd(ctr + 3, (unsigned long long)nb);
        if (nn) atomicAdd(ctr + 4, (unsigned long long)nn);
        if (nr) atomicAdd(ctr + 5, (unsigned long long)nr);
    }
}

// ---- exclusive scan (three passes: tile sums, scan of sums, tile scans) ----
__device__ __forceinline__ int block_excl_scan(int v, int *warp_tot, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    int off = 0;
    total = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
        int t = warp_tot[i];
        if (i < wid) off += t;
        total += t;
    }
    return off + x - v;
}

__global__ void scan_tile_sums(const int *__restrict__ in, int64_t n, int *__restrict__ part) {
    __shared__ int red[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k)
        if (base + k < n) s += in[base + k];
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void scan_partials(int *part, int64_t m) {
    __shared__ int wt[32];
    int carry = 0;
    for (int64_t b = 0; b < m; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        int v = (i < m) ? part[i] : 0;
        int total;
        int ex = block_excl_scan(v, wt, total);
        if (i < m) part[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[m] = carry;
}

__global__ void scan_tiles(const int *__restrict__ in, int64_t n, const int *__restrict__ part,
                           int *__restrict__ out) {
    __shared__ int wt[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    int v[SCAN_IPT];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int ex = block_excl_scan(s, wt, total) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[gridDim.x];
}

__global__ void root_flags_kernel(int n, const int *__restrict__ labels, int *__restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flags[i] = labels[i] == i;
}

__global__ void compact_kernel(int n, int *__restrict__ labels, const int *__restrict__ rank) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int l = labels[i];
        if (l >= 0) labels[i] = rank[l];
    }
}

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

cudaError_t launch_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *part, int64_t part_cap,
                                  cudaStream_t st, PhaseMarks *pm) {
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles + 1 > part_cap) return cudaErrorInvalidValue;
    if (tiles == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), st);
    scan_tile_sums<<<(unsigned)tiles, SCAN_NT, 0, st>>>(in, n, part);
    if (pm) pm->kernel("scan_sums", st);
    scan_partials<<<1, 1024, 0, st>>>(part, tiles);
    if (pm) pm->kernel("scan_partials", st);
    scan_tiles<<<(unsigned)tiles, SCAN_NT, 0, st>>>(in, n, part, out);
    if (pm) pm->kernel("scan_tiles", st);
    return cudaGetLastError();
}

cudaError_t launch_labels_allpairs(const DbWork &w, int64_t n, int32_t *labels, int32_t *counts_out,
                                   uint8_t *core_out, cudaStream_t st) {
    labels_allpairs_kernel<<<grid_for(n), 256, 0, st>>>((int)n, w.core, w.parent, w.border, w.count, labels,
                                                        counts_out, core_out, w.ctr);
    w.marks->kernel("labels", st);
    return cudaGetLastError();
}

cudaError_t launch_compact(const DbWork &w, int64_t n, int32_t *labels, cudaStream_t st) {
    // The border array is free once labels exist; it holds the root flags.
    root_flags_kernel<<<grid_for(n), 256, 0, st>>>((int)n, labels, w.border);
    w.marks->kernel("root_flags", st);
    cudaError_t e = launch_exclusive_scan(w.border, w.scan, n, w.scan_part, w.scan_part_cap, st, w.marks);
    if (e) return e;
    compact_kernel<<<grid_for(n), 256, 0, st>>>((int)n, labels, w.scan);
    w.marks->kernel("compact", st);
    return cudaGetLastError();
}
