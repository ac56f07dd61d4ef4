// batch.cu — many independent instances in one graph-captured launch sequence.
//
// Each instance is one DBSCAN problem (Section II's definitions, the three
// steps of Section IV) with its own n, d, eps and min_pts.  The instances are
// concatenated: point g of the batch is point g - base_i of instance i.  Every
// pass is one persistent kernel whose blocks pull work items (instance, row
// tile of 64 points, chunk of column tiles) from an atomic counter and run the
// same exact all-pairs tile as the single-instance path (ap_tile.cuh), on
// pointers offset to the instance, so each instance keeps its own
// union-find forest and local labels.  The kernel sequence (prep, count, core
// flags, union, border, labels, optional compaction) is captured once into a
// CUDA graph; a batch is then one table upload and one graph launch.
//
// Autotuning: the column chunk per work item (CH) and the number of resident
// blocks per SM are picked on the first call by timing every candidate on the
// caller's batch; the pick is kept by the plan.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ap_tile.cuh"
#include "plan.h"

using namespace aptile;

namespace {

struct BInst {
    const float *x;
    int32_t *labels;
    int n, d, dp, mode;
    int Tc;
    float Tp1;
    int min_pts;
    int base;       // first batch point of this instance
    long long poff; // first float of its packed rows
    int ntiles;     // row tiles of 16 * RM points
    int ctiles;     // column tiles of 64 points
    int nchunks;    // ceil(ctiles / CH)
    int item0;      // first work item of this instance
    int box0[3];    // its first tile box of 32, 64 and 128 rows
    int pad;
};

struct BHdr {  // device-side sizes of the current batch
    int count;
    int total_points;
    int total_items;
    int box_level0[3];  // first box of each level (32, 64, 128 rows) in the box array
    int pad[2];
};

__device__ __forceinline__ int find_inst_by_item(const BInst *__restrict__ t, int count, int item) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t[mid].item0 <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Morton (Z-order) dilation of a 10-bit coordinate: bit b moves to bit 3b.
__device__ __forceinline__ unsigned dilate3(unsigned v) {
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// One block per instance at a time.  An instance of 2 .. sort_cap points is
// put in Z-order of its first three grid coordinates (a bitonic sort of
// {code, index} keys in shared memory), so that a 64-row tile covers a small
// region; larger ones keep their order.  Then the rows are packed in that order
// (centred units v = u - 512: the Gram form is exact up to d = 16), perm gets
// the point of each row, and each 64-row tile its box: the least and greatest
// unit of its rows on every axis.  The reordering changes no result: every
// pass decides the same pairs, and labels are by point index.
__global__ void __launch_bounds__(1024) batch_sortpack_kernel(const BInst *__restrict__ t,
                                                              const BHdr *__restrict__ hdr, int sort_cap,
                                                              int *__restrict__ pinst, int *__restrict__ perm,
                                                              float *__restrict__ P, float *__restrict__ tbox,
                                                              unsigned *status) {
    extern __shared__ unsigned long long keys[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int count = hdr->count;
    bool bad = false;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const BInst I = t[i];
        const int n = I.n, d = I.d, dp = I.dp;
        const bool sorted = n > 1 && n <= sort_cap;
        if (sorted) {
            int npow = 2;
            while (npow < n) npow <<= 1;
            const int dz = d < 3 ? d : 3;
            for (int s = tid; s < npow; s += blockDim.x) {
                unsigned long long k = ~0ull;
                if (s < n) {
                    unsigned code = 0;
                    for (int j = 0; j < dz; ++j) {
                        int u;
                        db::on_grid(I.x[(size_t)s * d + j], u);  // off-grid input is reported below
                        code |= dilate3((unsigned)u) << j;
                    }
                    k = ((unsigned long long)code << 32) | (unsigned)s;
                }
                keys[s] = k;
            }
            __syncthreads();
            for (int k = 2; k <= npow; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int x = tid; x < npow; x += blockDim.x) {
                        const int y = x ^ j;
                        if (y > x) {
                            const unsigned long long kx = keys[x], ky = keys[y];
                            if ((kx > ky) == ((x & k) == 0)) {
                                keys[x] = ky;
                                keys[y] = kx;
                            }
                        }
                    }
                    __syncthreads();
                }
        }
        for (int s = tid; s < n; s += blockDim.x) {
            perm[I.base + s] = sorted ? (int)(unsigned)keys[s] : s;
            pinst[I.base + s] = i;
        }
        for (int e = tid; e < n * dp; e += blockDim.x) {
            const int s = e / dp, k = e - s * dp;
            const int o = sorted ? (int)(unsigned)keys[s] : s;
            float v = 0.f;
            if (k < d) {
                int u;
                bad |= !db::on_grid(I.x[(size_t)o * d + k], u);
                v = (float)(u - 512);
            }
            P[I.poff + (long long)s * dp + k] = v;
        }
        __syncthreads();  // the block's rows are visible to it; keys are free again
        // boxes of the 32-, 64- and 128-row tiles, a warp per tile
        for (int lv = 0; lv < 3; ++lv) {
            const int rows = 32 << lv, nt = (n + rows - 1) / rows;
            float *lvl = tbox + (size_t)(hdr->box_level0[lv] + I.box0[lv]) * 32;
            for (int tt = warp; tt < nt; tt += nwarps) {
                for (int k = 0; k < dp; ++k) {
                    float lo = 3.0e38f, hi = -3.0e38f;
                    for (int r = tt * rows + lane; r < min(n, (tt + 1) * rows); r += 32) {
                        const float v = P[I.poff + (long long)r * dp + k];
                        lo = fminf(lo, v);
                        hi = fmaxf(hi, v);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
                    }
                    if (lane == 0) {
                        lvl[(size_t)tt * 32 + k] = lo;
                        lvl[(size_t)tt * 32 + 16 + k] = hi;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, DB_EBIT_NOT_QUANTISED);
}

template <int PASS, int RM>
__global__ void __launch_bounds__(NT) batch_pass_kernel(const BInst *__restrict__ t, const BHdr *__restrict__ hdr,
                                                        int ch_tiles, int *work, const float *P,
                                                        const int *perm, const float *tbox, int *count,
                                                        const uint8_t *core, int *parent, int *border,
                                                        unsigned *status, unsigned long long *ev) {
    __shared__ int item_s;
    const int nitems = hdr->total_items, ninst = hdr->count;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(work, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= nitems) return;
        const int i = find_inst_by_item(t, ninst, item);
        const BInst &I = t[i];
        const int k = item - I.item0;
        const int rt = k / I.nchunks, chunk = k - rt * I.nchunks;
        int ct0 = chunk * ch_tiles;
        const int ct1 = min(I.ctiles, ct0 + ch_tiles);
        if (PASS == PASS_UNION) ct0 = max(ct0, rt * RM / 4);  // the column tile of the row tile's first row
        if (ct0 >= ct1) continue;
        ApArgs a;
        a.P = P + I.poff;
        a.n = I.n;
        a.Tp1 = I.Tp1;
        a.Tc = I.Tc;
        a.core = core + I.base;
        a.count = count + I.base;
        a.parent = parent + I.base;
        a.border = border + I.base;
        a.status = status;
        a.ntiles = I.ntiles;
        a.splits = 1;
        a.early = I.min_pts;  // batch outputs labels only: counts may stop at min_pts
        a.ev = ev ? ev + 3 * i : nullptr;  // pair tests evaluated by instance i's three passes
        a.perm = perm + I.base;
        constexpr int lv = RM == 2 ? 0 : (RM == 4 ? 1 : 2);  // box level of the row tiles
        a.tbox = tbox + (size_t)(hdr->box_level0[1] + I.box0[1]) * 32;
        a.tbox_rows = tbox + (size_t)(hdr->box_level0[lv] + I.box0[lv]) * 32;
        switch (I.dp) {  // block-uniform: one instance per work item
            case 1: ap_tile_body<1, MODE_GRAM, PASS, RM>(a, rt, ct0, ct1); break;
            case 2: ap_tile_body<2, MODE_GRAM, PASS, RM>(a, rt, ct0, ct1); break;
            case 3: ap_tile_body<3, MODE_GRAM, PASS, RM>(a, rt, ct0, ct1); break;
            case 4: ap_tile_body<4, MODE_GRAM, PASS, RM>(a, rt, ct0, ct1); break;
            case 8: ap_tile_body<8, MODE_GRAM, PASS, RM>(a, rt, ct0, ct1); break;
            default: ap_tile_body<16, MODE_GRAM, PASS, RM>(a, rt, ct0, ct1); break;
        }
    }
}

__global__ void batch_core_init_kernel(const BInst *__restrict__ t, const BHdr *__restrict__ hdr,
                                       const int *__restrict__ pinst, const int *__restrict__ count,
                                       uint8_t *__restrict__ core, int *__restrict__ parent, int *__restrict__ border) {
    const int total = hdr->total_points;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const BInst &I = t[pinst[g]];
        core[g] = count[g] >= I.min_pts;
        parent[g] = g - I.base;
        border[g] = DB_NONE;
    }
}

// Labels in each instance's own index space (a thread per row: core flags
// are by row, the forest and border choices by point); per-instance counts
// (core, border, noise, clusters) when istats != nullptr; root flags for
// compaction, by point.
__global__ void batch_label_kernel(const BInst *__restrict__ t, const BHdr *__restrict__ hdr,
                                   const int *__restrict__ pinst, const int *__restrict__ perm,
                                   const uint8_t *__restrict__ core, int *parent, const int *__restrict__ border,
                                   int *__restrict__ flags, int *istats) {
    const int total = hdr->total_points;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const int i = pinst[g];
        const BInst &I = t[i];
        const int loc = perm[g];  // row g - base holds point loc
        int *par = parent + I.base;
        const int bo = border[I.base + loc];
        int lab, kind;
        if (core[g]) {
            lab = db::uf_find(par, loc);
            kind = 0;
        } else if (bo != DB_NONE) {
            lab = db::uf_find(par, bo);
            kind = 1;
        } else {
            lab = -1;
            kind = 2;
        }
        I.labels[loc] = lab;
        const int root = (kind == 0 && lab == loc);
        flags[I.base + loc] = root;
        if (istats) {
            atomicAdd(istats + 4 * i + kind, 1);
            if (root) atomicAdd(istats + 4 * i + 3, 1);
        }
    }
}

__global__ void batch_compact_kernel(const BInst *__restrict__ t, const BHdr *__restrict__ hdr,
                                     const int *__restrict__ pinst, const int *__restrict__ rank) {
    const int total = hdr->total_points;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const BInst &I = t[pinst[g]];
        const int loc = g - I.base;
        const int l = I.labels[loc];
        if (l >= 0) I.labels[loc] = rank[I.base + l] - rank[I.base];
    }
}

constexpr int kCH[] = {4, 16, 64};
constexpr int kRM[] = {2, 4, 8};  // row tiles of 32, 64 and 128 points (8 rows per thread for the last)
constexpr int kSortMax = 16384;  // largest instance reordered (128 KiB of sort keys in shared memory)
constexpr int kBPS[] = {4, 8};

}  // namespace

struct BatchState {
    int cap_count = 0;
    int64_t cap_points = 0, cap_pfloats = 0, cap_tiles = 0;
    void *dev = nullptr;
    size_t dev_bytes = 0;
    BInst *d_table = nullptr;
    BHdr *d_hdr = nullptr;
    int *d_pinst = nullptr;
    int *d_perm = nullptr;     // point of each row (rows of an instance in Z-order)
    float *d_tbox = nullptr;   // per 64-row tile: least and greatest unit on each axis [tiles][32]
    int sort_cap = 0;          // instances up to this many points are reordered (a power of two)
    float *d_P = nullptr;
    int *d_count = nullptr;
    uint8_t *d_core = nullptr;
    int *d_parent = nullptr, *d_border = nullptr, *d_flags = nullptr, *d_scan = nullptr, *d_part = nullptr;
    int64_t part_cap = 0;
    int *d_work = nullptr;
    unsigned *d_status = nullptr;
    int *d_istats = nullptr;
    unsigned long long *d_ev = nullptr;  // pair tests evaluated per instance and pass [count][3]
    unsigned long long *h_ev = nullptr;
    BInst *h_table = nullptr;
    BHdr *h_hdr = nullptr;
    int *h_istats = nullptr;
    unsigned *h_status = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_ch = -1, graph_bps = -1, graph_rm = -1, graph_stats = -1;
    int ch = 16, bps = 8, rm = 4;  // column tiles per work item, blocks per SM, rows per thread (tile of 16 rm rows)
    bool tuned = false;
    PhaseMarks marks;  // timing off
};

void batch_release(BatchState *b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->dev) cudaFree(b->dev);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->h_hdr) cudaFreeHost(b->h_hdr);
    if (b->h_istats) cudaFreeHost(b->h_istats);
    if (b->h_ev) cudaFreeHost(b->h_ev);
    if (b->h_status) cudaFreeHost(b->h_status);
    delete b;
}

namespace {

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// (Re)allocates the batch workspace for at least these sizes.
int batch_reserve(BatchState *b, int count, int64_t points, int64_t pfloats, int64_t tiles) {
    if (count <= b->cap_count && points <= b->cap_points && pfloats <= b->cap_pfloats && tiles <= b->cap_tiles)
        return DBSCAN_OK;
    const int nc = std::max(count, b->cap_count);
    const int64_t np = std::max<int64_t>(std::max(points, b->cap_points), 1);
    const int64_t nf = std::max<int64_t>(std::max(pfloats, b->cap_pfloats), 1);
    const int64_t nt = std::max<int64_t>(std::max(tiles, b->cap_tiles), 1);
    const int64_t part = np / 2048 + 4;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = al256(off + bytes);
        return o;
    };
    const size_t o_table = take(sizeof(BInst) * nc), o_hdr = take(sizeof(BHdr)), o_pinst = take(4 * np),
                 o_P = take(4 * nf), o_count = take(4 * np), o_core = take(np), o_parent = take(4 * np),
                 o_border = take(4 * np), o_flags = take(4 * np), o_scan = take(4 * (np + 1)),
                 o_part = take(4 * part), o_work = take(4 * 8), o_status = take(16), o_istats = take(16 * nc),
                 o_ev = take(24 * (size_t)nc), o_perm = take(4 * np), o_tbox = take(128 * (size_t)nt);
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->dev) cudaFree(b->dev);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->h_istats) cudaFreeHost(b->h_istats);
    if (b->h_ev) cudaFreeHost(b->h_ev);
    b->dev = nullptr;
    b->h_table = nullptr;
    b->h_istats = nullptr;
    b->h_ev = nullptr;
    if (cudaMalloc(&b->dev, off) != cudaSuccess) {
        cudaGetLastError();
        b->cap_count = 0;
        b->cap_points = b->cap_pfloats = b->cap_tiles = 0;
        return DBSCAN_ERR_OOM;
    }
    if (cudaMallocHost(&b->h_table, sizeof(BInst) * nc) != cudaSuccess ||
        cudaMallocHost(&b->h_istats, 16 * (size_t)nc) != cudaSuccess ||
        cudaMallocHost(&b->h_ev, 24 * (size_t)nc) != cudaSuccess)
        return DBSCAN_ERR_OOM;
    if (!b->h_hdr && cudaMallocHost(&b->h_hdr, sizeof(BHdr)) != cudaSuccess) return DBSCAN_ERR_OOM;
    if (!b->h_status && cudaMallocHost(&b->h_status, 16) != cudaSuccess) return DBSCAN_ERR_OOM;
    char *base = static_cast<char *>(b->dev);
    b->dev_bytes = off;
    b->d_table = reinterpret_cast<BInst *>(base + o_table);
    b->d_hdr = reinterpret_cast<BHdr *>(base + o_hdr);
    b->d_pinst = reinterpret_cast<int *>(base + o_pinst);
    b->d_perm = reinterpret_cast<int *>(base + o_perm);
    b->d_tbox = reinterpret_cast<float *>(base + o_tbox);
    b->d_P = reinterpret_cast<float *>(base + o_P);
    b->d_count = reinterpret_cast<int *>(base + o_count);
    b->d_core = reinterpret_cast<uint8_t *>(base + o_core);
    b->d_parent = reinterpret_cast<int *>(base + o_parent);
    b->d_border = reinterpret_cast<int *>(base + o_border);
    b->d_flags = reinterpret_cast<int *>(base + o_flags);
    b->d_scan = reinterpret_cast<int *>(base + o_scan);
    b->d_part = reinterpret_cast<int *>(base + o_part);
    b->part_cap = part;
    b->d_work = reinterpret_cast<int *>(base + o_work);
    b->d_status = reinterpret_cast<unsigned *>(base + o_status);
    b->d_istats = reinterpret_cast<int *>(base + o_istats);
    b->d_ev = reinterpret_cast<unsigned long long *>(base + o_ev);
    b->cap_count = nc;
    b->cap_points = np;
    b->cap_pfloats = nf;
    b->cap_tiles = nt;
    if (cudaMemset(b->d_status, 0, 16) != cudaSuccess) return DBSCAN_ERR_CUDA;
    return DBSCAN_OK;
}

// Host table for chunk size ch and row tiles of 16 * rm points; returns the
// total work items.  boxes[lv] counts the tile boxes of 32 << lv rows.
int64_t build_table(const dbscan_instance *inst, int count, int ch, int rm, BInst *t, int64_t *points,
                    int64_t *pfloats, int64_t boxes[3], int64_t *max_n) {
    int64_t base = 0, poff = 0, items = 0, mx = 0;
    boxes[0] = boxes[1] = boxes[2] = 0;
    for (int i = 0; i < count; ++i) {
        const dbscan_instance &in = inst[i];
        BInst &I = t[i];
        const double e = (double)in.eps;
        const int64_t T = (int64_t)std::floor(e * e * 1048576.0);
        const int64_t Tc = std::min<int64_t>(T, (int64_t)in.d * 1023 * 1023);
        I.x = in.points;
        I.labels = in.labels_out;
        I.n = (int)in.n;
        I.d = in.d;
        I.dp = dp_for(in.d);  // 1, 2, 3, 4, 8 or 16
        I.mode = MODE_GRAM;
        I.Tc = (int)Tc;
        I.Tp1 = (float)(Tc + 1);
        I.min_pts = in.min_pts;
        I.base = (int)base;
        I.poff = poff;
        I.ntiles = (int)((in.n + 16 * rm - 1) / (16 * rm));
        I.ctiles = (int)((in.n + BN - 1) / BN);
        I.nchunks = (I.ctiles + ch - 1) / ch;
        I.item0 = (int)items;
        for (int lv = 0; lv < 3; ++lv) {
            I.box0[lv] = (int)boxes[lv];
            boxes[lv] += (in.n + (32 << lv) - 1) / (32 << lv);
        }
        I.pad = 0;
        base += in.n;
        poff += (in.n * I.dp + 3) / 4 * 4;  // 16-byte aligned rows of every instance (vector tile loads)
        items += (int64_t)I.ntiles * I.nchunks;
        mx = std::max<int64_t>(mx, in.n);
    }
    *points = base;
    *pfloats = poff;
    *max_n = mx;
    return items;
}

template <int PASS>
void launch_batch_pass(BatchState *b, int rm, int grid, int ch, int *work, bool stats, cudaStream_t st) {
    unsigned long long *ev = stats ? b->d_ev : nullptr;
#define DB_BATCH_PASS(R)                                                                                            \
    batch_pass_kernel<PASS, R><<<grid, NT, 0, st>>>(b->d_table, b->d_hdr, ch, work, b->d_P, b->d_perm, b->d_tbox,  \
                                                    b->d_count, b->d_core, b->d_parent, b->d_border, b->d_status, ev)
    if (rm == 2) DB_BATCH_PASS(2);
    else if (rm == 8) DB_BATCH_PASS(8);
    else DB_BATCH_PASS(4);
#undef DB_BATCH_PASS
}

cudaError_t enqueue_batch(BatchState *b, int label_mode, bool stats, int ch, int bps, int rm, cudaStream_t st,
                          PhaseMarks *pm = nullptr) {
    PhaseMarks off;
    if (!pm) pm = &off;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int pgrid = sms * bps, egrid = sms * 8;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_table, b->h_table, sizeof(BInst) * b->cap_count, cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(BHdr), cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaMemsetAsync(b->d_work, 0, 4 * 8, st))) return e;
    if ((e = cudaMemsetAsync(b->d_count, 0, 4 * (size_t)b->cap_points, st))) return e;
    if (stats && (e = cudaMemsetAsync(b->d_istats, 0, 16 * (size_t)b->cap_count, st))) return e;
    if (stats && (e = cudaMemsetAsync(b->d_ev, 0, 24 * (size_t)b->cap_count, st))) return e;
    batch_sortpack_kernel<<<sms * 2, 1024, sizeof(unsigned long long) * std::max(b->sort_cap, 2), st>>>(
        b->d_table, b->d_hdr, b->sort_cap, b->d_pinst, b->d_perm, b->d_P, b->d_tbox, b->d_status);
    pm->kernel("batch_prep", st);
    launch_batch_pass<PASS_COUNT>(b, rm, pgrid, ch, b->d_work + 0, stats, st);
    pm->kernel("batch_count", st);
    batch_core_init_kernel<<<egrid, 256, 0, st>>>(b->d_table, b->d_hdr, b->d_pinst, b->d_count, b->d_core,
                                                  b->d_parent, b->d_border);
    pm->kernel("batch_core_init", st);
    launch_batch_pass<PASS_UNION>(b, rm, pgrid, ch, b->d_work + 1, stats, st);
    pm->kernel("batch_union", st);
    launch_batch_pass<PASS_BORDER>(b, rm, pgrid, ch, b->d_work + 2, stats, st);
    pm->kernel("batch_border", st);
    batch_label_kernel<<<egrid, 256, 0, st>>>(b->d_table, b->d_hdr, b->d_pinst, b->d_perm, b->d_core, b->d_parent,
                                              b->d_border,
                                              b->d_flags, stats ? b->d_istats : nullptr);
    pm->kernel("batch_label", st);
    if ((e = cudaGetLastError())) return e;
    if (label_mode == DBSCAN_LABEL_COMPACT) {
        if ((e = launch_exclusive_scan(b->d_flags, b->d_scan, b->cap_points, b->d_part, b->part_cap, st, pm)))
            return e;
        batch_compact_kernel<<<egrid, 256, 0, st>>>(b->d_table, b->d_hdr, b->d_pinst, b->d_scan);
        pm->kernel("batch_compact", st);
    }
    if (stats && (e = cudaMemcpyAsync(b->h_istats, b->d_istats, 16 * (size_t)b->cap_count, cudaMemcpyDeviceToHost,
                                      st)))
        return e;
    if (stats && (e = cudaMemcpyAsync(b->h_ev, b->d_ev, 24 * (size_t)b->cap_count, cudaMemcpyDeviceToHost, st)))
        return e;
    if ((e = cudaMemcpyAsync(b->h_status, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), st))) return e;
    return cudaGetLastError();
}

// The whole sequence as one CUDA graph (rebuilt when capacities or the tuned
// configuration change).
int batch_graph_launch(BatchState *b, int label_mode, bool stats, cudaStream_t st) {
    if (!b->graph || b->graph_ch != b->ch || b->graph_bps != b->bps || b->graph_rm != b->rm ||
        b->graph_stats != (int)stats || b->graph_ch < 0) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DBSCAN_ERR_CUDA;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (!e) e = enqueue_batch(b, label_mode, stats, b->ch, b->bps, b->rm, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (e || e2 || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return DBSCAN_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e) {
            cudaGetLastError();
            b->graph = nullptr;
            return DBSCAN_ERR_CUDA;
        }
        b->graph_ch = b->ch;
        b->graph_bps = b->bps;
        b->graph_rm = b->rm;
        b->graph_stats = (int)stats;
    }
    return cudaGraphLaunch(b->graph, st) == cudaSuccess ? DBSCAN_OK : DBSCAN_ERR_CUDA;
}

}  // namespace

extern "C" int dbscan_batch(dbscan_plan *plan, const dbscan_instance *inst, int32_t count, dbscan_stats *per_inst) {
    if (!plan || count < 0 || (count > 0 && !inst)) return DBSCAN_ERR_ARG;
    if (count == 0) return DBSCAN_OK;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        const dbscan_instance &in = inst[i];
        if (in.n < 0 || in.d < 1 || in.d > 16 || !(in.eps > 0.0f) || std::isinf(in.eps) || in.min_pts < 1)
            return in.d > 16 ? DBSCAN_ERR_UNSUPPORTED : DBSCAN_ERR_ARG;
        if (in.n > 0 && (!in.points || !in.labels_out)) return DBSCAN_ERR_ARG;
        total += in.n;
    }
    if (total > INT32_MAX / 2) return DBSCAN_ERR_ARG;
    // work items (instance, row tile, column chunk) are counted in int32: the
    // smallest chunk gives the most items
    int64_t items = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t rows = (inst[i].n + 31) / 32, cols = (inst[i].n + 63) / 64;  // the smallest row tile
        items += rows * ((cols + kCH[0] - 1) / kCH[0]);
    }
    if (items > INT32_MAX) return DBSCAN_ERR_UNSUPPORTED;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != plan->opts.device) cudaSetDevice(plan->opts.device);
    if (!plan->batch) plan->batch = new BatchState();
    BatchState *b = plan->batch;
    const int label_mode = plan->opts.label_mode;
    const bool stats = per_inst != nullptr;
    cudaStream_t st = plan->stream;

    // Sizes for the largest chunk count (smallest CH) so every candidate fits.
    std::vector<BInst> tmp(count);
    int64_t points = 0, pfloats = 0, boxes[3] = {0, 0, 0}, max_n = 0;
    build_table(inst, count, kCH[0], kRM[0], tmp.data(), &points, &pfloats, boxes, &max_n);
    int s = batch_reserve(b, count, points, pfloats, boxes[0] + boxes[1] + boxes[2]);
    if (s) return s;
    // Instances up to kSortMax points are put in Z-order; the sort's shared
    // memory is sized for the largest of them.
    int sort_cap = 2;
    while (sort_cap < std::min<int64_t>(max_n, kSortMax)) sort_cap <<= 1;
    if (sort_cap != b->sort_cap && b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->sort_cap = sort_cap;
    if (sizeof(unsigned long long) * sort_cap > 48 * 1024 &&
        cudaFuncSetAttribute(batch_sortpack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * sort_cap)) != cudaSuccess)
        return DBSCAN_ERR_CUDA;

    auto prepare = [&](int ch, int rm) {
        int64_t pts, pf, bx[3], mn;
        const int64_t items = build_table(inst, count, ch, rm, b->h_table, &pts, &pf, bx, &mn);
        for (int i = count; i < b->cap_count; ++i) std::memset(&b->h_table[i], 0, sizeof(BInst));
        b->h_hdr->count = count;
        b->h_hdr->total_points = (int)pts;
        b->h_hdr->total_items = (int)std::min<int64_t>(items, INT32_MAX);
        b->h_hdr->box_level0[0] = 0;
        b->h_hdr->box_level0[1] = (int)bx[0];
        b->h_hdr->box_level0[2] = (int)(bx[0] + bx[1]);
        b->h_hdr->pad[0] = b->h_hdr->pad[1] = 0;
    };

    if (!b->tuned) {
        // Autotune on this batch: every (row tile, CH, blocks per SM) candidate, best of 2 runs.
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int rm : kRM)
        for (int ch : kCH)
            for (int bps : kBPS) {
                prepare(ch, rm);
                float tbest = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaEventRecord(e0, st);
                    if (enqueue_batch(b, label_mode, false, ch, bps, rm, st)) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return DBSCAN_ERR_CUDA;
                    }
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    tbest = std::min(tbest, ms);
                }
                if (tbest < best) {
                    best = tbest;
                    b->ch = ch;
                    b->bps = bps;
                    b->rm = rm;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->tuned = true;
    }
    prepare(b->ch, b->rm);
    if (plan->opts.profile) {  // per-kernel events: run the sequence uncaptured
        plan->marks.begin(st);
        if (enqueue_batch(b, label_mode, stats, b->ch, b->bps, b->rm, st, &plan->marks)) return DBSCAN_ERR_CUDA;
    } else {
        s = batch_graph_launch(b, label_mode, stats, st);
        if (s) return s;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return DBSCAN_ERR_CUDA;
    if (cur >= 0 && cur != plan->opts.device) cudaSetDevice(cur);
    const unsigned bits = *b->h_status;
    if (bits & DB_EBIT_NOT_QUANTISED) return DBSCAN_ERR_NOT_QUANTISED;
    if (bits & DB_EBIT_TIMEOUT) return DBSCAN_ERR_TIMEOUT;
    if (bits) return DBSCAN_ERR_CUDA;
    if (stats) {
        // the batch's pair tests per pass, also left in the plan's counters 16..18
        unsigned long long tot[4] = {0, 0, 0, 0};
        for (int i = 0; i < count; ++i)
            for (int k = 0; k < 3; ++k) tot[k] += b->h_ev[3 * i + k];
        if (cudaMemcpy(plan->w.ctr + DB_CTR_EVAL, tot, sizeof(tot), cudaMemcpyHostToDevice) != cudaSuccess)
            return DBSCAN_ERR_CUDA;
        for (int i = 0; i < count; ++i) {
            dbscan_stats &o = per_inst[i];
            std::memset(&o, 0, sizeof(o));
            o.n_core = b->h_istats[4 * i + 0];
            o.n_border = b->h_istats[4 * i + 1];
            o.n_noise = b->h_istats[4 * i + 2];
            o.n_clusters = b->h_istats[4 * i + 3];
            o.candidate_pairs = inst[i].n * inst[i].n;
            o.path = DBSCAN_PATH_ALLPAIRS_SIMT;
            const double e = (double)inst[i].eps;
            o.threshold = (int64_t)std::floor(e * e * 1048576.0);
            o.kernels = 6 + (label_mode == DBSCAN_LABEL_COMPACT ? 4 : 0);
            o.pair_tests = (int64_t)(b->h_ev[3 * i] + b->h_ev[3 * i + 1] + b->h_ev[3 * i + 2]);
        }
    }
    return DBSCAN_OK;
}

extern "C" int dbscan_batch_config(dbscan_plan *plan, int32_t *chunk_tiles, int32_t *blocks_per_sm) {
    if (!plan) return DBSCAN_ERR_ARG;
    if (!plan->batch || !plan->batch->tuned) return DBSCAN_ERR_NOT_FOUND;
    if (chunk_tiles) *chunk_tiles = plan->batch->ch;
    if (blocks_per_sm) *blocks_per_sm = plan->batch->bps;
    return DBSCAN_OK;
}

extern "C" int dbscan_batch_tile(dbscan_plan *plan, int32_t *tile_rows, int32_t *tile_cols) {
    if (!plan) return DBSCAN_ERR_ARG;
    if (!plan->batch || !plan->batch->tuned) return DBSCAN_ERR_NOT_FOUND;
    if (tile_rows) *tile_rows = 16 * plan->batch->rm;
    if (tile_cols) *tile_cols = BN;
    return DBSCAN_OK;
}
