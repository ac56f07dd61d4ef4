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
    int ntiles;     // ceil(n / 64)
    int nchunks;    // ceil(ntiles / CH)
    int item0;      // first work item of this instance
    int pad;
};

struct BHdr {  // device-side sizes of the current batch
    int count;
    int total_points;
    int total_items;
    int pad;
};

__device__ __forceinline__ int find_inst_by_base(const BInst *__restrict__ t, int count, int g) {
    int lo = 0, hi = count - 1;  // last instance with base <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t[mid].base <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_inst_by_item(const BInst *__restrict__ t, int count, int item) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t[mid].item0 <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void batch_prep_kernel(const BInst *__restrict__ t, const BHdr *__restrict__ hdr, int *__restrict__ pinst,
                                  float *__restrict__ P, unsigned *status) {
    const int count = hdr->count, total = hdr->total_points;
    bool bad = false;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const int i = find_inst_by_base(t, count, g);
        const BInst &I = t[i];
        const int loc = g - I.base;
        pinst[g] = i;
        float *row = P + I.poff + (long long)loc * I.dp;
        for (int k = 0; k < I.dp; ++k) {
            float v = 0.f;
            if (k < I.d) {
                int u;
                bad |= !db::on_grid(I.x[(size_t)loc * I.d + k], u);
                v = (float)(u - 512);  // centred units: the Gram form is exact up to d = 16
            }
            row[k] = v;
        }
    }
    if (bad) atomicOr(status, DB_EBIT_NOT_QUANTISED);
}

template <int PASS>
__global__ void __launch_bounds__(NT) batch_pass_kernel(const BInst *__restrict__ t, const BHdr *__restrict__ hdr,
                                                        int ch_tiles, int *work, const float *P, int *count,
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
        const int ct1 = min(I.ntiles, ct0 + ch_tiles);
        if (PASS == PASS_UNION) ct0 = max(ct0, rt);
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
        switch (I.dp) {  // block-uniform: one instance per work item
            case 1: ap_tile_body<1, MODE_GRAM, PASS>(a, rt, ct0, ct1); break;
            case 2: ap_tile_body<2, MODE_GRAM, PASS>(a, rt, ct0, ct1); break;
            case 3: ap_tile_body<3, MODE_GRAM, PASS>(a, rt, ct0, ct1); break;
            case 4: ap_tile_body<4, MODE_GRAM, PASS>(a, rt, ct0, ct1); break;
            case 8: ap_tile_body<8, MODE_GRAM, PASS>(a, rt, ct0, ct1); break;
            default: ap_tile_body<16, MODE_GRAM, PASS>(a, rt, ct0, ct1); break;
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

// Labels in each instance's own index space; per-instance counts
// (core, border, noise, clusters) when istats != nullptr; root flags for
// compaction.
__global__ void batch_label_kernel(const BInst *__restrict__ t, const BHdr *__restrict__ hdr,
                                   const int *__restrict__ pinst, const uint8_t *__restrict__ core, int *parent,
                                   const int *__restrict__ border, int *__restrict__ flags, int *istats) {
    const int total = hdr->total_points;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const int i = pinst[g];
        const BInst &I = t[i];
        const int loc = g - I.base;
        int *par = parent + I.base;
        int lab, kind;
        if (core[g]) {
            lab = db::uf_find(par, loc);
            kind = 0;
        } else if (border[g] != DB_NONE) {
            lab = db::uf_find(par, border[g]);
            kind = 1;
        } else {
            lab = -1;
            kind = 2;
        }
        I.labels[loc] = lab;
        const int root = (kind == 0 && lab == loc);
        flags[g] = root;
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
constexpr int kBPS[] = {4, 8};

}  // namespace

struct BatchState {
    int cap_count = 0;
    int64_t cap_points = 0, cap_pfloats = 0;
    void *dev = nullptr;
    size_t dev_bytes = 0;
    BInst *d_table = nullptr;
    BHdr *d_hdr = nullptr;
    int *d_pinst = nullptr;
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
    int graph_ch = -1, graph_bps = -1, graph_stats = -1;
    int ch = 16, bps = 8;
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
int batch_reserve(BatchState *b, int count, int64_t points, int64_t pfloats) {
    if (count <= b->cap_count && points <= b->cap_points && pfloats <= b->cap_pfloats) return DBSCAN_OK;
    const int nc = std::max(count, b->cap_count);
    const int64_t np = std::max<int64_t>(std::max(points, b->cap_points), 1);
    const int64_t nf = std::max<int64_t>(std::max(pfloats, b->cap_pfloats), 1);
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
                 o_ev = take(24 * (size_t)nc);
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
        b->cap_points = b->cap_pfloats = 0;
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
    if (cudaMemset(b->d_status, 0, 16) != cudaSuccess) return DBSCAN_ERR_CUDA;
    return DBSCAN_OK;
}

// Host table for chunk size ch; returns total work items or -1 on a bad instance.
int64_t build_table(const dbscan_instance *inst, int count, int ch, BInst *t, int64_t *points, int64_t *pfloats) {
    int64_t base = 0, poff = 0, items = 0;
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
        I.ntiles = (int)((in.n + BM - 1) / BM);
        I.nchunks = (I.ntiles + ch - 1) / ch;
        I.item0 = (int)items;
        I.pad = 0;
        base += in.n;
        poff += (in.n * I.dp + 3) / 4 * 4;  // 16-byte aligned rows of every instance (vector tile loads)
        items += (int64_t)I.ntiles * I.nchunks;
    }
    *points = base;
    *pfloats = poff;
    return items;
}

cudaError_t enqueue_batch(BatchState *b, int label_mode, bool stats, int ch, int bps, cudaStream_t st,
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
    batch_prep_kernel<<<egrid, 256, 0, st>>>(b->d_table, b->d_hdr, b->d_pinst, b->d_P, b->d_status);
    pm->kernel("batch_prep", st);
    batch_pass_kernel<PASS_COUNT><<<pgrid, NT, 0, st>>>(b->d_table, b->d_hdr, ch, b->d_work + 0, b->d_P, b->d_count,
                                                        b->d_core, b->d_parent, b->d_border, b->d_status, stats ? b->d_ev : nullptr);
    pm->kernel("batch_count", st);
    batch_core_init_kernel<<<egrid, 256, 0, st>>>(b->d_table, b->d_hdr, b->d_pinst, b->d_count, b->d_core,
                                                  b->d_parent, b->d_border);
    pm->kernel("batch_core_init", st);
    batch_pass_kernel<PASS_UNION><<<pgrid, NT, 0, st>>>(b->d_table, b->d_hdr, ch, b->d_work + 1, b->d_P, b->d_count,
                                                        b->d_core, b->d_parent, b->d_border, b->d_status, stats ? b->d_ev : nullptr);
    pm->kernel("batch_union", st);
    batch_pass_kernel<PASS_BORDER><<<pgrid, NT, 0, st>>>(b->d_table, b->d_hdr, ch, b->d_work + 2, b->d_P,
                                                         b->d_count, b->d_core, b->d_parent, b->d_border, b->d_status,
                                                         stats ? b->d_ev : nullptr);
    pm->kernel("batch_border", st);
    batch_label_kernel<<<egrid, 256, 0, st>>>(b->d_table, b->d_hdr, b->d_pinst, b->d_core, b->d_parent, b->d_border,
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
    if (!b->graph || b->graph_ch != b->ch || b->graph_bps != b->bps || b->graph_stats != (int)stats ||
        b->graph_ch < 0) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DBSCAN_ERR_CUDA;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (!e) e = enqueue_batch(b, label_mode, stats, b->ch, b->bps, cs);
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
        const int64_t tiles = (inst[i].n + 63) / 64;
        items += tiles * ((tiles + kCH[0] - 1) / kCH[0]);
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
    int64_t points = 0, pfloats = 0;
    build_table(inst, count, kCH[0], tmp.data(), &points, &pfloats);
    int s = batch_reserve(b, count, points, pfloats);
    if (s) return s;

    auto prepare = [&](int ch) {
        int64_t pts, pf;
        const int64_t items = build_table(inst, count, ch, b->h_table, &pts, &pf);
        for (int i = count; i < b->cap_count; ++i) std::memset(&b->h_table[i], 0, sizeof(BInst));
        b->h_hdr->count = count;
        b->h_hdr->total_points = (int)pts;
        b->h_hdr->total_items = (int)std::min<int64_t>(items, INT32_MAX);
        b->h_hdr->pad = 0;
    };

    if (!b->tuned) {
        // Autotune on this batch: every (CH, blocks per SM) candidate, best of 2 runs.
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int ch : kCH)
            for (int bps : kBPS) {
                prepare(ch);
                float tbest = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaEventRecord(e0, st);
                    if (enqueue_batch(b, label_mode, false, ch, bps, st)) {
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
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->tuned = true;
    }
    prepare(b->ch);
    if (plan->opts.profile) {  // per-kernel events: run the sequence uncaptured
        plan->marks.begin(st);
        if (enqueue_batch(b, label_mode, stats, b->ch, b->bps, st, &plan->marks)) return DBSCAN_ERR_CUDA;
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
