// grid_mid.cu — projected grid candidate path for 4 <= d <= 8.
//
// The paper tests every pair (Section IV-A).  For 4 <= d <= 8 this path bins
// the points on their first three coordinates and tests only pairs whose
// projections lie in adjacent cells, deciding each with the same exact
// predicate D(p,q) <= T over all d coordinates, so it gives the same labels.
//
// Geometry (integer grid units): s = floor(sqrt(T)) bounds |u_pk - u_qk| for
// a neighbour on every axis, so with cell side c = s + 1 every neighbour of p
// lies in p's cell or one of the 26 cells around it in the projection.  Unlike
// the eps-grid of d <= 3 a cell is not a clique (the other coordinates are
// free), so every candidate pair is tested: the predicate runs in the Gram
// form of Section IV-B, T + 1 - |p|^2 - |q|^2 + sum_k 2 u_pk u_qk, whose
// partial sums are integers below 2 d 1023^2 < 2^24 in magnitude for d <= 8,
// so FP32 decides it exactly.
//
// Steps on the device:
//   prep     grid check of all d coordinates, cell key of the first three,
//            hash insert, per-cell count (the eps-grid's hash)
//   cells    cell table (shared with the eps-grid, grid.cu)
//   scatter  rows grouped by cell: units padded to DP (4 or 8), -|u|^2, index
//   nbrs     neighbour lists of the 27 offsets, own cell first (grid.cu)
//   chunks   work items: 32-point chunks of every cell, so a dense cell is
//            spread over many warps
//   count    neighbour counts -> core flags (Section IV-B's fused pass); a
//            chunk stops counting a point once it reaches min_pts unless exact
//            counts are requested
//   merge    union of core-core neighbours (Section IV-C), each unordered pair
//            once (the larger cell id, or the later position in one cell),
//            skipping pairs whose set hints already agree
//   border   smallest-index core neighbour of every non-core point
//   labels   shared with the all-pairs path (labels.cu)
// A chunk's warp walks the candidate cells' points 128 at a time (four loads
// per lane), and tests each batch against every pending point of the chunk,
// broadcast lane by lane.
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid check of all d coordinates, cell key of the first three, hash insert.
__global__ void mid_prep_kernel(const float *__restrict__ x, int n, int d, GridGeom g, unsigned *hkey,
                                int *hcount, int *__restrict__ slot_of, unsigned *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    int slot = -1 - lane;
    if (valid) {
        int u[3] = {0, 0, 0};
        bool ok = true;
        for (int k = 0; k < d; ++k) {
            int uk;
            ok &= db::on_grid(x[(size_t)i * d + k], uk);
            if (k < 3) u[k] = uk;
        }
        if (!ok) atomicOr(status, DB_EBIT_NOT_QUANTISED);
        const unsigned key = ((unsigned)(u[2] / g.c) * (unsigned)g.G + (unsigned)(u[1] / g.c)) * (unsigned)g.G +
                             (unsigned)(u[0] / g.c);
        const unsigned mask = (1u << g.hbits) - 1u;
        unsigned h = db::hash_slot(key, g.hbits);
        bool placed = false;
        for (unsigned probe = 0; probe <= mask; ++probe) {
            const unsigned cur = ld_relaxed_u32(hkey + h);
            if (cur == key) {
                placed = true;
                break;
            }
            if (cur == DB_HASH_EMPTY) {
                const unsigned prev = atomicCAS(hkey + h, DB_HASH_EMPTY, key);
                if (prev == DB_HASH_EMPTY || prev == key) {
                    placed = true;
                    break;
                }
            }
            h = (h + 1) & mask;
        }
        if (!placed) {  // cannot happen with >= 2n slots; keep memory safe if it does
            atomicOr(status, DB_EBIT_OVERFLOW);
            h = 0;
        }
        slot = (int)h;
        slot_of[i] = slot;
    }
    const unsigned peers = __match_any_sync(FULL, slot);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(hcount + slot, __popc(peers));
}

// Rows grouped by cell: P[pos][DP] = units (zero padding), nrm[pos] = -|u|^2,
// sidx[pos] = point index.
template <int DP>
__global__ void mid_scatter_kernel(const float *__restrict__ x, int n, int d, const int *__restrict__ slot_of,
                                   int *hcursor, float *__restrict__ P, float *__restrict__ nrm,
                                   int *__restrict__ sidx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    const int slot = valid ? slot_of[i] : -1 - lane;
    const unsigned peers = __match_any_sync(FULL, slot);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(hcursor + slot, __popc(peers));
    base = __shfl_sync(FULL, base, leader);
    if (!valid) return;
    const int pos = base + __popc(peers & db::lanemask_lt());
    float v[DP];
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        float t = 0.f;
        if (k < d) {
            int uk;
            db::on_grid(x[(size_t)i * d + k], uk);  // prep has flagged any off-grid value
            t = (float)uk;
        }
        v[k] = t;
        s = fmaf(t, t, s);  // exact: integers below 8 * 1023^2
    }
    float4 *dst = reinterpret_cast<float4 *>(P + (size_t)pos * DP);
#pragma unroll
    for (int k = 0; k < DP / 4; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    nrm[pos] = -s;
    sidx[pos] = i;
}

// Chunks per cell (32 points each), zero past the last cell.
__global__ void mid_chunk_count_kernel(int n, const unsigned long long *ctr0, const int *__restrict__ cell_count,
                                       int *__restrict__ cc) {
    const int ncells = (int)(*ctr0 >> 32);
    for (int A = blockIdx.x * blockDim.x + threadIdx.x; A < n; A += gridDim.x * blockDim.x)
        cc[A] = A < ncells ? (cell_count[A] + 31) >> 5 : 0;
}

// Work items (cell, first point of the chunk) from the exclusive scan of the
// chunk counts; *nitems receives the item count.
__global__ void mid_chunk_table_kernel(int n, const unsigned long long *ctr0, const int *__restrict__ cell_count,
                                       const int *__restrict__ scan, int2 *__restrict__ items, int *nitems) {
    const int ncells = (int)(*ctr0 >> 32);
    for (int A = blockIdx.x * blockDim.x + threadIdx.x; A < ncells; A += gridDim.x * blockDim.x) {
        const int k0 = scan[A], nc = (cell_count[A] + 31) >> 5;
        for (int k = 0; k < nc; ++k) items[k0 + k] = make_int2(A, 32 * k);
        if (A == ncells - 1) *nitems = k0 + nc;
    }
}

struct MidArgs {
    GridGeom g;
    const int *cell_start, *cell_count;
    const int *nbr;    // neighbour cell lists (own cell first), row stride g.noff
    const int *ncnt;   // (adjacent count << 16) | count
    const float *P;    // grouped units, row stride DP
    const float *nrm;  // grouped -|u|^2
    const int *sidx;   // grouped point index
    const int2 *items;
    const int *nitems;
    unsigned long long *ev;  // pair tests evaluated: [0] count, [1] merge, [2] border
};

template <int DP>
__device__ __forceinline__ void load_row(const float *P, int pos, float *v) {
    const float4 *src = reinterpret_cast<const float4 *>(P + (size_t)pos * DP);
#pragma unroll
    for (int k = 0; k < DP / 4; ++k) {
        const float4 t = src[k];
        v[4 * k] = t.x;
        v[4 * k + 1] = t.y;
        v[4 * k + 2] = t.z;
        v[4 * k + 3] = t.w;
    }
}

// T + 1 - D(p,q) >= 1 in the Gram form: cp = T + 1 - |p|^2, p2 = 2 u_p,
// q = u_q, qn = -|q|^2 (exact, see the file header).
template <int DP>
__device__ __forceinline__ bool mid_nbr(float cp, const float *p2, const float *q, float qn) {
    float acc = cp + qn;
#pragma unroll
    for (int k = 0; k < DP; ++k) acc = fmaf(p2[k], q[k], acc);
    return acc >= 1.f;
}

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Position of flattened candidate j (smallest lane k with incl[k] > j).
__device__ __forceinline__ int locate(int j, int incl, int c, int s) {
    int k = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
        if (__shfl_sync(FULL, incl, k + step - 1) <= j) k += step;
    k &= 31;
    const int ik = __shfl_sync(FULL, incl, k), ck = __shfl_sync(FULL, c, k), sk = __shfl_sync(FULL, s, k);
    return sk + (j - (ik - ck));
}

// Count pass.  One warp per chunk: lane i holds point i of the chunk; the
// candidates of the cell's list (own cell included, so a point counts
// itself) are tested 128 at a time against every point still below lim.
template <int DP>
__global__ void __launch_bounds__(256) mid_count_kernel(MidArgs a, int min_pts, int exact, int *__restrict__ count,
                                                        uint8_t *__restrict__ core, uint8_t *__restrict__ score,
                                                        int *__restrict__ parent, int *__restrict__ hint) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nitems = *a.nitems;
    const int lim = exact ? INT_MAX : min_pts;
    unsigned ev = 0;
    for (int it = warp; it < nitems; it += nwarps) {
        const int2 item = a.items[it];
        const int A = item.x, i0 = item.y;
        const int sA = a.cell_start[A], cA = a.cell_count[A];
        const bool mine = i0 + lane < cA;
        const int pos = sA + i0 + (mine ? lane : 0);
        float pv[DP];
        load_row<DP>(a.P, pos, pv);
        const float cpm = a.g.Tp1 + a.nrm[pos];
#pragma unroll
        for (int k = 0; k < DP; ++k) pv[k] *= 2.f;
        const int *row = a.nbr + (size_t)A * a.g.noff;
        const int nn = a.ncnt[A] & 0xffff;
        int cnt = 0;
        unsigned pend = __ballot_sync(FULL, mine);
        for (int k0 = 0; k0 < nn && pend; k0 += 32) {
            const int B = (k0 + lane < nn) ? row[k0 + lane] : -1;
            const int s = B >= 0 ? a.cell_start[B] : 0, c = B >= 0 ? a.cell_count[B] : 0;
            const int incl = warp_incl_scan(c), total = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < total && pend; base += 128) {
                float qv[4][DP], qn[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = base + 32 * u + lane;
                    const int q = locate(j, incl, c, s);
                    if (j < total) {
                        load_row<DP>(a.P, q, qv[u]);
                        qn[u] = a.nrm[q];
                    } else {
#pragma unroll
                        for (int k = 0; k < DP; ++k) qv[u][k] = 0.f;
                        qn[u] = -1e30f;
                    }
                }
                if (lane == 0) ev += (unsigned)(__popc(pend) * min(128, total - base));
                for (unsigned m = pend; m; m &= m - 1) {
                    const int i = __ffs(m) - 1;
                    float p2[DP];
#pragma unroll
                    for (int k = 0; k < DP; ++k) p2[k] = __shfl_sync(FULL, pv[k], i);
                    const float cp = __shfl_sync(FULL, cpm, i);
                    int add = 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) add += mid_nbr<DP>(cp, p2, qv[u], qn[u]);
                    const int r = (int)__reduce_add_sync(FULL, (unsigned)add);
                    if (lane == i) cnt += r;
                }
                pend = __ballot_sync(FULL, mine && cnt < lim);
            }
        }
        if (mine) {
            const int o = a.sidx[pos];
            const bool c = cnt >= min_pts;
            count[o] = cnt;
            core[o] = c;
            score[pos] = c;
            parent[o] = o;
            hint[pos] = o;
        }
    }
    db::block_sum_add(a.ev + 0, lane == 0 ? (unsigned long long)ev : 0ull);
}

// Merge pass (Section IV-C): every core point of the chunk against the core
// candidates after it (a larger cell id, or a later position in its own
// cell), uniting the two sets at each eps-pair.  hint[pos] holds a member of
// the point's set (its index, or a root seen later): equal hints mean one set,
// so those pairs need neither a test nor a union.
template <int DP>
__global__ void __launch_bounds__(256) mid_union_kernel(MidArgs a, const uint8_t *__restrict__ score, int *parent,
                                                        int *hint, unsigned *status) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nitems = *a.nitems;
    unsigned ev = 0;
    for (int it = warp; it < nitems; it += nwarps) {
        const int2 item = a.items[it];
        const int A = item.x, i0 = item.y;
        const int sA = a.cell_start[A], cA = a.cell_count[A];
        const bool inr = i0 + lane < cA;
        const int pos = sA + i0 + (inr ? lane : 0);
        const bool mine = inr && score[pos];
        const unsigned cores = __ballot_sync(FULL, mine);
        if (!cores) continue;
        float pv[DP];
        load_row<DP>(a.P, pos, pv);
        const float cpm = a.g.Tp1 + a.nrm[pos];
#pragma unroll
        for (int k = 0; k < DP; ++k) pv[k] *= 2.f;
        const int om = a.sidx[pos];
        int hm = mine ? db::ld_relaxed(hint + pos) : -1;
        const int *row = a.nbr + (size_t)A * a.g.noff;
        const int nn = a.ncnt[A] & 0xffff;
        for (int k0 = 0; k0 < nn; k0 += 32) {
            const int B = (k0 + lane < nn) ? row[k0 + lane] : -1;
            const bool take = B >= A;  // pairs with a smaller cell id come from that cell's side
            const int s = take ? a.cell_start[B] : 0, c = take ? a.cell_count[B] : 0;
            const int incl = warp_incl_scan(c), total = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < total; base += 128) {
                float qv[4][DP], qn[4];
                int qp[4], qo[4], qh[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = base + 32 * u + lane;
                    const int q = locate(j, incl, c, s);
                    qp[u] = -1;
                    if (j < total && score[q]) {
                        qp[u] = q;
                        load_row<DP>(a.P, q, qv[u]);
                        qn[u] = a.nrm[q];
                        qo[u] = a.sidx[q];
                        qh[u] = db::ld_relaxed(hint + q);
                    } else {
#pragma unroll
                        for (int k = 0; k < DP; ++k) qv[u][k] = 0.f;
                        qn[u] = -1e30f;
                        qo[u] = -1;
                        qh[u] = -1;
                    }
                }
                for (unsigned m = cores; m; m &= m - 1) {
                    const int i = __ffs(m) - 1;
                    float p2[DP];
#pragma unroll
                    for (int k = 0; k < DP; ++k) p2[k] = __shfl_sync(FULL, pv[k], i);
                    const float cp = __shfl_sync(FULL, cpm, i);
                    const int pi = __shfl_sync(FULL, pos, i), oi = __shfl_sync(FULL, om, i);
                    int h = __shfl_sync(FULL, hm, i);
                    int root = INT_MAX;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (qp[u] <= pi || qh[u] == h) continue;  // not after p, padding, or one set already
                        ++ev;
                        if (!mid_nbr<DP>(cp, p2, qv[u], qn[u])) continue;
                        const int r = db::uf_unite_root(parent, oi, qo[u], status);
                        if (r >= 0) {
                            qh[u] = r;
                            db::st_relaxed(hint + qp[u], r);
                            root = min(root, r);
                        }
                    }
                    root = (int)__reduce_min_sync(FULL, (unsigned)root);
                    if (root != INT_MAX && lane == i) {
                        hm = root;
                        db::st_relaxed(hint + pos, root);
                    }
                }
            }
        }
    }
    db::block_sum_add(a.ev + 1, (unsigned long long)ev);
}

// Border pass: every non-core point of the chunk takes its smallest-index
// core neighbour (DB_NONE if it has none).  A candidate whose index is not
// below the point's best so far needs no test.
template <int DP>
__global__ void __launch_bounds__(256) mid_border_kernel(MidArgs a, const uint8_t *__restrict__ score,
                                                         int *__restrict__ border) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nitems = *a.nitems;
    unsigned ev = 0;
    for (int it = warp; it < nitems; it += nwarps) {
        const int2 item = a.items[it];
        const int A = item.x, i0 = item.y;
        const int sA = a.cell_start[A], cA = a.cell_count[A];
        const bool inr = i0 + lane < cA;
        const int pos = sA + i0 + (inr ? lane : 0);
        const bool mine = inr && !score[pos];
        const unsigned pend = __ballot_sync(FULL, mine);
        if (!pend) continue;
        float pv[DP];
        load_row<DP>(a.P, pos, pv);
        const float cpm = a.g.Tp1 + a.nrm[pos];
#pragma unroll
        for (int k = 0; k < DP; ++k) pv[k] *= 2.f;
        int b = DB_NONE;
        const int *row = a.nbr + (size_t)A * a.g.noff;
        const int nn = a.ncnt[A] & 0xffff;
        for (int k0 = 0; k0 < nn; k0 += 32) {
            const int B = (k0 + lane < nn) ? row[k0 + lane] : -1;
            const int s = B >= 0 ? a.cell_start[B] : 0, c = B >= 0 ? a.cell_count[B] : 0;
            const int incl = warp_incl_scan(c), total = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < total; base += 128) {
                float qv[4][DP], qn[4];
                int qi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = base + 32 * u + lane;
                    const int q = locate(j, incl, c, s);
                    qi[u] = DB_NONE;
                    if (j < total && score[q]) {
                        qi[u] = a.sidx[q];
                        load_row<DP>(a.P, q, qv[u]);
                        qn[u] = a.nrm[q];
                    } else {
#pragma unroll
                        for (int k = 0; k < DP; ++k) qv[u][k] = 0.f;
                        qn[u] = -1e30f;
                    }
                }
                for (unsigned m = pend; m; m &= m - 1) {
                    const int i = __ffs(m) - 1;
                    float p2[DP];
#pragma unroll
                    for (int k = 0; k < DP; ++k) p2[k] = __shfl_sync(FULL, pv[k], i);
                    const float cp = __shfl_sync(FULL, cpm, i);
                    int best = __shfl_sync(FULL, b, i);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool better = qi[u] < best;  // else the pair needs no test
                        ev += better;
                        if (better && mid_nbr<DP>(cp, p2, qv[u], qn[u])) best = qi[u];
                    }
                    best = (int)__reduce_min_sync(FULL, (unsigned)best);
                    if (lane == i) b = best;
                }
            }
        }
        if (mine) border[a.sidx[pos]] = b;
    }
    db::block_sum_add(a.ev + 2, (unsigned long long)ev);
}

int64_t isqrt64(int64_t v) {
    if (v <= 0) return 0;
    int64_t r = (int64_t)std::sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

template <int DP>
cudaError_t mid_passes(const DbWork &w, const GridGeom &g, const float *x, int n, int d, int min_pts, bool exact,
                       int32_t *labels, int32_t *counts_out, uint8_t *core_out, const unsigned *occ,
                       cudaStream_t st) {
    // Arrays of the eps-grid's workspace the projected path reuses: P holds the
    // grouped rows (stride DP <= the plan's row stride), pts4 the grouped
    // -|u|^2, cell_mid the chunk table, cell_rep the chunks per cell, slot_of
    // (free after the scatter) the set hints.
    float *nrm = reinterpret_cast<float *>(w.pts4);
    int2 *items = reinterpret_cast<int2 *>(w.cell_mid);
    int *nitems = reinterpret_cast<int *>(w.ctr + DB_CTR_MID_ITEMS);
    int *cc = w.cell_rep;
    int *hint = w.slot_of;
    const int nb = (n + 255) / 256;
    mid_scatter_kernel<DP><<<nb, 256, 0, st>>>(x, n, d, w.slot_of, w.hcursor, w.P, nrm, w.sidx);
    w.marks->kernel("mid_scatter", st);
    cudaError_t e;
    if ((e = launch_grid_nbrs(w, g, occ, st))) return e;
    mid_chunk_count_kernel<<<std::min(nb, 152 * 8), 256, 0, st>>>(n, w.ctr, w.cell_count, cc);
    w.marks->kernel("mid_chunks", st);
    if ((e = launch_exclusive_scan(cc, w.scan, n, w.scan_part, w.scan_part_cap, st, w.marks))) return e;
    mid_chunk_table_kernel<<<std::min(nb, 152 * 8), 256, 0, st>>>(n, w.ctr, w.cell_count, w.scan, items, nitems);
    w.marks->kernel("mid_chunk_table", st);
    MidArgs a{g, w.cell_start, w.cell_count, w.nbr, w.ncnt, w.P, nrm, w.sidx, items, nitems, w.ctr + DB_CTR_EVAL};
    const int wgrid = 152 * 16;  // 8 warps per block, warps stride over the chunks
    mid_count_kernel<DP><<<wgrid, 256, 0, st>>>(a, min_pts, exact ? 1 : 0, w.count, w.core, w.score, w.parent, hint);
    w.marks->kernel("mid_count", st);
    mid_union_kernel<DP><<<wgrid, 256, 0, st>>>(a, w.score, w.parent, hint, w.status);
    w.marks->kernel("mid_union", st);
    mid_border_kernel<DP><<<wgrid, 256, 0, st>>>(a, w.score, w.border);
    w.marks->kernel("mid_border", st);
    if ((e = cudaGetLastError())) return e;
    return launch_labels_allpairs(w, n, labels, counts_out, core_out, st);
}

}  // namespace

bool mid_geometry(int32_t d, int64_t Tc, int64_t n, GridGeom *g) {
    if (d < 4 || d > 8) return false;
    const int64_t s = isqrt64(Tc);
    const int64_t c = s + 1;
    const int64_t G = (1024 + c - 1) / c;
    if (G < 4) return false;  // cells this coarse prune little: all pairs instead
    g->d = 3;  // key dimensions
    g->c = (int32_t)c;
    g->G = (int32_t)G;
    g->Tc = (int32_t)Tc;
    g->Tp1 = (float)(Tc + 1);
    g->inv_c = (float)(1.0 / (double)g->c);
    int bits = 10;
    while ((int64_t(1) << bits) < 2 * n) ++bits;
    g->hbits = bits;
    g->dense = 0;  // hashed cell table
    int k = 0;
    g->off[k++] = make_char4(0, 0, 0, 0);  // own cell first
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox)
                if (ox || oy || oz) g->off[k++] = make_char4((signed char)ox, (signed char)oy, (signed char)oz, 0);
    g->noff = k;  // 27
    g->nnear = k;
    return true;
}

cudaError_t launch_mid_grid_path(const DbWork &w, const GridGeom &g, const float *x, int64_t n64, int32_t d,
                                 int32_t min_pts, bool exact, int32_t *labels, int32_t *counts_out,
                                 uint8_t *core_out, cudaStream_t st) {
    const int n = (int)n64;
    const int64_t H = int64_t(1) << g.hbits;
    const int DP = d <= 4 ? 4 : 8;
    if (H > w.hcap || g.noff > w.noff_cap || w.dp_cap < DP) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.hkey, 0xff, sizeof(unsigned) * H, st))) return e;
    if ((e = cudaMemsetAsync(w.hcount, 0, sizeof(int) * H, st))) return e;
    const int64_t all_cells = (int64_t)g.G * g.G * g.G;
    const int64_t occ_words = (all_cells + 31) / 32;
    unsigned *occ = occ_words <= w.occ_cap ? w.occ : nullptr;
    if (occ && (e = cudaMemsetAsync(occ, 0, sizeof(unsigned) * occ_words, st))) return e;
    const int nb = (n + 255) / 256;
    mid_prep_kernel<<<nb, 256, 0, st>>>(x, n, d, g, w.hkey, w.hcount, w.slot_of, w.status);
    w.marks->kernel("mid_prep", st);
    if ((e = launch_grid_cells(w, g, occ, nullptr, st))) return e;
    return DP == 4 ? mid_passes<4>(w, g, x, n, d, min_pts, exact, labels, counts_out, core_out, occ, st)
                   : mid_passes<8>(w, g, x, n, d, min_pts, exact, labels, counts_out, core_out, occ, st);
}
