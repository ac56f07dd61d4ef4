// grid.cu — eps-grid candidate path for d <= 3.
//
// The paper tests every pair (Section IV-A).  For d <= 3 this path tests only
// pairs in nearby grid cells, and decides each with the same exact predicate
// D(p,q) <= T, so it gives the same labels.
//
// Geometry (all in integer grid units):
//   m = floor(sqrt(floor(T/d))), cell side c = m + 1.  Two points in one cell
//   differ by at most m per axis, so D <= d*m^2 <= T: every cell is a clique of
//   mutual eps-neighbours.
//   s = floor(sqrt(T)) bounds |u_pk - u_qk| for a neighbour, so neighbours lie
//   within r = ceil(s/c) <= 2 cells per axis; an offset o is kept when its two
//   cells can hold a pair with D <= T: sum_k [o_k != 0] ((|o_k|-1) c + 1)^2 <= T.
//
// Cells are found through an open-addressing hash of the cell key, so no sort
// is needed: points are counted per cell, each occupied cell reserves a
// contiguous range, and points are scattered into their cell's range.
//
// Steps on the device, each a kernel:
//   prep     grid check, cell key, hash insert, per-cell count
//   cells    occupied slot -> cell id and point range (block-aggregated)
//   scatter  points grouped by cell
//   nbrs     neighbour lists: the occupied cells at the kept offsets,
//            compacted, adjacent offsets first
//   count    neighbour counts -> core flags (Section IV-B).  A cell with at
//            least min_pts points makes all its points core with no test; other
//            points stop counting once they reach min_pts unless exact counts
//            are requested.  Each cell records its smallest core index (rep).
//            Each core point then hangs under its cell's rep (cells are cliques).
//   union    neighbouring cells whose cores contain one eps-pair are united
//            (Section IV-C's merge), adjacent cells in one launch and the
//            outer ring in a second; a cell pair already in one set is skipped
//   border   each non-core point finds its smallest-index core neighbour
//   root     the union-find root of every cell with cores
//   label    labels (a thread per point)
// nbrs runs beside scatter, and border beside union, on the plan's second
// stream: each pair is independent and latency-bound.  Every kernel starts as
// a programmatic dependent of the one before it in its stream, so its launch
// overlaps that kernel's tail.
// The count and border kernels give a thread to each grouped point, which
// walks its cell's neighbour list (four entries and their ranges loaded at
// once); the merge kernel gives a warp to one cell at a time, a lane to each
// neighbouring cell, and searches a cell pair 32 lanes wide.
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

using db::hash_slot;

__device__ __forceinline__ unsigned cell_key_of(const int *u, const GridGeom &g) {
    unsigned cx = (unsigned)(u[0] / g.c);
    unsigned cy = g.d > 1 ? (unsigned)(u[1] / g.c) : 0u;
    unsigned cz = g.d > 2 ? (unsigned)(u[2] / g.c) : 0u;
    return (cz * (unsigned)g.G + cy) * (unsigned)g.G + cx;
}

__global__ void grid_prep_kernel(const float *__restrict__ x, int n, GridGeom g, unsigned *hkey, int *hcount,
                                 int *__restrict__ slot_of, float4 *__restrict__ pts4, int *__restrict__ parent,
                                 unsigned *status) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    int slot = -1 - lane;
    if (valid) {
        int u[3] = {0, 0, 0};
        bool ok = true;
        for (int k = 0; k < g.d; ++k) {
            int uk;
            ok &= db::on_grid(x[(size_t)i * g.d + k], uk);
            u[k] = uk;
        }
        if (!ok) atomicOr(status, DB_EBIT_NOT_QUANTISED);
        const unsigned key = cell_key_of(u, g);
        const unsigned mask = (1u << g.hbits) - 1u;
        unsigned h = g.dense ? key : hash_slot(key, g.hbits);
        bool placed = g.dense != 0;  // a dense table needs no probe
        for (unsigned probe = 0; probe <= mask && !placed; ++probe) {
            unsigned cur = ld_relaxed_u32(hkey + h);
            if (cur == key) { placed = true; break; }
            if (cur == DB_HASH_EMPTY) {
                unsigned prev = atomicCAS(hkey + h, DB_HASH_EMPTY, key);
                if (prev == DB_HASH_EMPTY || prev == key) { placed = true; break; }
            }
            h = (h + 1) & mask;
        }
        if (!placed) {  // cannot happen with >= 2n slots; keep memory safe if it does
            atomicOr(status, DB_EBIT_OVERFLOW);
            h = 0;
        }
        slot = (int)h;
        slot_of[i] = slot;
        parent[i] = i;  // every point starts as its own set; only cell representatives are ever linked
        const float f0 = (float)u[0], f1 = (float)u[1], f2 = (float)u[2];
        pts4[i] = make_float4(f0, f1, f2, -(f0 * f0 + f1 * f1 + f2 * f2));
    }
    // One atomic per distinct cell in the warp.
    const unsigned peers = __match_any_sync(0xffffffffu, slot);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(hcount + slot, __popc(peers));
}

constexpr int CELLS_PER_THREAD = 4;

__global__ void grid_cells_kernel(int H, int dense, const unsigned *__restrict__ hkey, const int *__restrict__ hcount,
                                  int2 *__restrict__ hpack, int *__restrict__ hcursor, int *__restrict__ cell_start,
                                  int *__restrict__ cell_count, unsigned *__restrict__ cell_key,
                                  int *__restrict__ cell_rep, unsigned long long *__restrict__ midkey,
                                  unsigned *__restrict__ occ, unsigned long long *ctr0) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    __shared__ int wocc[32], wcnt[32];
    __shared__ unsigned long long base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int s0 = (blockIdx.x * blockDim.x + threadIdx.x) * CELLS_PER_THREAD;
    int cnt[CELLS_PER_THREAD];
    int tocc = 0, tcnt = 0;
#pragma unroll
    for (int k = 0; k < CELLS_PER_THREAD; ++k) {
        cnt[k] = (s0 + k < H) ? hcount[s0 + k] : 0;
        tocc += cnt[k] > 0;
        tcnt += cnt[k];
    }
    int xo = tocc, xc = tcnt;
    for (int o = 1; o < 32; o <<= 1) {
        int yo = __shfl_up_sync(0xffffffffu, xo, o), yc = __shfl_up_sync(0xffffffffu, xc, o);
        if (lane >= o) { xo += yo; xc += yc; }
    }
    if (lane == 31) { wocc[wid] = xo; wcnt[wid] = xc; }
    __syncthreads();
    int offo = 0, offc = 0, toto = 0, totc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < wid) { offo += wocc[w]; offc += wcnt[w]; }
        toto += wocc[w];
        totc += wcnt[w];
    }
    if (threadIdx.x == 0)
        base = (toto || totc) ? atomicAdd(ctr0, ((unsigned long long)toto << 32) | (unsigned)totc) : 0ull;
    __syncthreads();
    int cid = (int)(base >> 32) + offo + xo - tocc;
    int start = (int)(base & 0xffffffffull) + offc + xc - tcnt;
#pragma unroll
    for (int k = 0; k < CELLS_PER_THREAD; ++k) {
        const int s = s0 + k;
        if (cnt[k] > 0) {
            const unsigned key = dense ? (unsigned)s : hkey[s];
            cell_start[cid] = start;
            cell_count[cid] = cnt[k];
            cell_key[cid] = key;
            cell_rep[cid] = DB_NONE;
            if (midkey) midkey[cid] = ~0ull;
            hpack[s] = make_int2((int)key, cid);
            hcursor[s] = start;
            if (occ) atomicOr(occ + (key >> 5), 1u << (key & 31u));
            ++cid;
            start += cnt[k];
        } else if (s < H) {
            hpack[s] = make_int2((int)DB_HASH_EMPTY, -1);
        }
    }
}

__global__ void grid_scatter_kernel(int n, const int *__restrict__ slot_of, int *hcursor, const int2 *__restrict__ hpack,
                                    const float4 *__restrict__ pts4, float4 *__restrict__ spts, int *__restrict__ sidx,
                                    int *__restrict__ scell) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    const int slot = valid ? slot_of[i] : -1 - lane;
    const unsigned peers = __match_any_sync(0xffffffffu, slot);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(hcursor + slot, __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!valid) return;
    const int pos = base + __popc(peers & db::lanemask_lt());
    spts[pos] = pts4[i];
    sidx[pos] = i;
    scell[pos] = hpack[slot].y;
}

// Neighbour lists, a warp per cell: lane l looks up offsets l, l+32, l+64 and
// l+96 (all loads independent), and the cells found are written compacted,
// adjacent offsets first; ncnt[A] = (adjacent count << 16) | total count, and
// cell_cand[A] = the points in the listed cells.
// When the occupancy bitmap of all G^d cells fits its buffer (occ != null),
// an empty neighbour costs one bit test and no hash probe.
__global__ void grid_nbr_kernel(GridGeom g, const unsigned long long *ctr0, const unsigned *__restrict__ cell_key,
                                const int2 *__restrict__ hpack, const unsigned *__restrict__ occ,
                                const int *__restrict__ cell_count, int *__restrict__ nbr, int *__restrict__ ncnt,
                                int *__restrict__ cell_cand) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    // Offsets go through shared memory into registers once: lanes indexing the
    // parameter array with different offsets would serialise on every read.
    __shared__ char4 soff[128];
    for (int o = threadIdx.x; o < 128; o += blockDim.x) soff[o] = o < g.noff ? g.off[o] : make_char4(0, 0, 0, 0);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    char4 offr[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) offr[u] = soff[32 * u + lane];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int ncells = (int)(*ctr0 >> 32);
    const unsigned mask = (1u << g.hbits) - 1u;
    const int G = g.G;
    for (int A = warp; A < ncells; A += nwarps) {
        const unsigned key = cell_key[A];
        const int c[3] = {(int)(key % G), (int)((key / G) % G), (int)(key / ((unsigned)G * G))};
        unsigned k2[4];
        bool in[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int o = 32 * u + lane;
            in[u] = false;
            k2[u] = 0;
            if (o < g.noff) {
                const char4 off = offr[u];
                const int nc[3] = {c[0] + off.x, c[1] + off.y, c[2] + off.z};
                in[u] = nc[0] >= 0 && nc[0] < G && nc[1] >= 0 && nc[1] < G && nc[2] >= 0 && nc[2] < G;
                k2[u] = ((unsigned)nc[2] * G + (unsigned)nc[1]) * G + (unsigned)nc[0];
            }
        }
        if (occ) {
            unsigned wbits[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) wbits[u] = in[u] ? occ[k2[u] >> 5] : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) in[u] = (wbits[u] >> (k2[u] & 31u)) & 1u;
        }
        int2 e[4];
        unsigned h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            h[u] = g.dense ? k2[u] : hash_slot(k2[u], g.hbits);
            e[u] = in[u] ? hpack[h[u]] : make_int2((int)DB_HASH_EMPTY, -1);
        }
        int res[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            res[u] = -1;
            if (g.dense) {  // the slot of a key is the key: found or empty, no probe
                if ((unsigned)e[u].x == k2[u]) res[u] = e[u].y;
                continue;
            }
            // continue probing past other keys (rare at load factor <= 1/2)
            for (unsigned probe = 0; probe <= mask; ++probe) {
                if ((unsigned)e[u].x == k2[u]) { res[u] = e[u].y; break; }
                if ((unsigned)e[u].x == DB_HASH_EMPTY) break;
                h[u] = (h[u] + 1) & mask;
                e[u] = hpack[h[u]];
            }
        }
        int *row = nbr + (size_t)A * g.noff;
        int nn = 0, nnear = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (32 * u >= g.noff) break;
            const unsigned hits = __ballot_sync(FULL, res[u] >= 0);
            if (res[u] >= 0) row[nn + __popc(hits & db::lanemask_lt())] = res[u];
            const int nl = g.nnear - 32 * u;  // lanes of this chunk with adjacent offsets
            const unsigned near_lanes = nl <= 0 ? 0u : (nl >= 32 ? FULL : ((1u << nl) - 1u));
            nnear += __popc(hits & near_lanes);
            nn += __popc(hits);
        }
        // points in the listed cells: the candidates of each point of A
        int tc = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) tc += res[u] >= 0 ? cell_count[res[u]] : 0;
        tc = (int)__reduce_add_sync(FULL, (unsigned)tc);
        if (lane == 0) {
            ncnt[A] = (nnear << 16) | nn;
            cell_cand[A] = tc;
        }
    }
}

// Exact score T + 1 - D(p,q) in the Gram form of Section IV-B: every partial
// sum is an integer below 2*3*1023^2 < 2^24 in magnitude, so FP32 is exact.
template <int D>
__device__ __forceinline__ bool is_nbr(float cp, float px2, float py2, float pz2, float4 q) {
    float acc = cp + q.w;
    acc = fmaf(px2, q.x, acc);
    if (D > 1) acc = fmaf(py2, q.y, acc);
    if (D > 2) acc = fmaf(pz2, q.z, acc);
    return acc >= 1.f;
}

struct PairArgs {
    GridGeom g;
    const unsigned long long *ctr0;
    int n;
    const float4 *spts;
    const int *sidx;
    const int *scell;  // cell of each grouped position
    const int *cell_start, *cell_count, *cell_rep;
    const unsigned long long *cell_mid;  // per cell: (squared distance to the centre << 32) | packed point
    const unsigned *cell_key;
    const int *nbr;   // neighbour cell lists, row stride g.noff
    const int *ncnt;  // (adjacent count << 16) | count
    const int *cell_cand;  // points in the cells of each neighbour list
    unsigned long long *ev;  // pair tests evaluated: [0] count, [1] merge, [2] border, [3] outer-ring merge
};

// A point whose neighbour cells hold at most this many points walks them in
// its own thread; the points of a cell with more are walked by the whole warp,
// 32 candidates a step (a cell next to a tight blob can hold thousands).
constexpr int kThreadWalkMax = 96;

// ---- warp-cooperative candidate walk ---------------------------------------
// The neighbour list of a cell is read 32 entries at a time: lane l holds
// (start, size) of one neighbour cell and an inclusive prefix of the sizes, so
// the candidates of those cells form one flattened range that the 32 lanes
// walk together.

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Lane k holding flattened candidate j: the smallest lane with incl[k] > j (a
// 5-step binary search over the lanes' prefixes); its position is then
// start[k] + (j - exclusive[k]).  All 32 lanes must call it; the result is
// meaningless when j >= total.
__device__ __forceinline__ int locate_lane(int j, int incl) {
    int k = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
        if (__shfl_sync(FULL, incl, k + step - 1) <= j) k += step;
    return k & 31;
}

// A point of the grid as {u0, u1, u2, -|u|^2} from its packed form
// u0 | u1 << 10 | u2 << 20 (low 30 bits of a cell_mid entry).
__device__ __forceinline__ float4 unpack_point(unsigned long long key) {
    const unsigned v = (unsigned)key;
    const float x = (float)(v & 1023u), y = (float)((v >> 10) & 1023u), z = (float)((v >> 20) & 1023u);
    return make_float4(x, y, z, -(x * x + y * y + z * z));
}

// Segmented minimum over a warp whose lanes hold consecutive grouped
// positions (so equal cell ids are contiguous): afterwards the first lane of
// each run of equal `cell` holds the minimum of `v` over its run.
template <typename V>
__device__ __forceinline__ V seg_min_down(V v, int cell) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_down_sync(FULL, v, o);
        const int cy = __shfl_down_sync(FULL, cell, o);
        if (lane + o < 32 && cy == cell) v = y < v ? y : v;
    }
    return v;
}

// Count pass (Section IV-B, fused pair test + count), a thread per grouped
// position p in cell A.  The points of A are all neighbours (A is a clique),
// so p starts at |A|; when |A| >= min_pts and no exact counts are asked for
// p is core with no pair test.  Otherwise p tests the points of A's neighbour
// cells, and stops once it has min_pts neighbours unless exact counts are
// asked for: in its own thread when they are few (four list entries and their
// ranges loaded at once), else together with the warp's other points of A,
// the warp walking the candidates 128 a step with four independent loads per
// lane.  Lanes of a warp hold consecutive positions, mostly of one cell, so
// their loads coalesce.  Per cell, the smallest core index goes to
// cell_rep[A] and the core point nearest A's centre (the merge pass tries it
// first) to cell_mid[A], both by a segmented warp minimum and one atomic per
// run of the cell's points in the warp.
template <int D>
__global__ void __launch_bounds__(256) grid_count_kernel(PairArgs a, int min_pts, int exact, uint8_t *score,
                                                         int *cell_rep, unsigned long long *cell_mid,
                                                         int *counts_out, uint8_t *core_out) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < a.n;
    const int lim = exact ? INT_MAX : min_pts;
    const int A = valid ? a.scell[p] : -1 - lane;  // no two invalid lanes share a cell
    unsigned long long ev = 0;  // pair tests of this thread
    int cnt = 0, o = DB_NONE;
    bool heavy = false;
    float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        cnt = a.cell_count[A];
        pt = a.spts[p];
        o = a.sidx[p];
    }
    const float cp = a.g.Tp1 + pt.w, px2 = 2.f * pt.x, py2 = 2.f * pt.y, pz2 = 2.f * pt.z;
    if (valid && cnt < lim) {
        heavy = a.cell_cand[A] > kThreadWalkMax;
        if (!heavy) {
            const int *row = a.nbr + (size_t)A * a.g.noff;
            const int nn = a.ncnt[A] & 0xffff;
            for (int k0 = 0; k0 < nn && cnt < lim; k0 += 4) {
                int s[4], e[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) s[u] = k0 + u < nn ? row[k0 + u] : -1;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int B = s[u];
                    s[u] = B >= 0 ? a.cell_start[B] : 0;
                    e[u] = B >= 0 ? s[u] + a.cell_count[B] : 0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    ev += (unsigned)(e[u] - s[u]);
#pragma unroll 4
                    for (int q = s[u]; q < e[u]; ++q) cnt += is_nbr<D>(cp, px2, py2, pz2, a.spts[q]);
                }
            }
        }
    }
    // cells with many candidates: the warp walks each one's candidates for its
    // lanes of that cell still below the limit
    unsigned hv = __ballot_sync(FULL, heavy);
    while (hv) {
        const int H = __shfl_sync(FULL, A, __ffs(hv) - 1);
        const unsigned mine = __ballot_sync(FULL, heavy && A == H);
        hv &= ~mine;
        const int *row = a.nbr + (size_t)H * a.g.noff;
        const int nn = a.ncnt[H] & 0xffff;
        unsigned pend = mine;
        for (int k0 = 0; k0 < nn && pend; k0 += 32) {
            const int B = (k0 + lane < nn) ? row[k0 + lane] : -1;
            const int s = B >= 0 ? a.cell_start[B] : 0, c = B >= 0 ? a.cell_count[B] : 0;
            const int incl = warp_incl_scan(c), total = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < total && pend; base += 128) {
                float4 qq[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = base + 32 * u + lane;
                    const int k = locate_lane(j, incl);
                    const int ex = __shfl_sync(FULL, incl, k) - __shfl_sync(FULL, c, k);  // lane k's first j
                    const int q = __shfl_sync(FULL, s, k) + (j - ex);
                    qq[u] = j < total ? a.spts[q] : make_float4(0.f, 0.f, 0.f, -1e30f);
                }
                if (lane == 0) ev += (unsigned long long)__popc(pend) * (unsigned)min(128, total - base);
                for (unsigned m = pend; m; m &= m - 1) {
                    const int i = __ffs(m) - 1;
                    const float cpi = __shfl_sync(FULL, cp, i), px2i = __shfl_sync(FULL, px2, i);
                    const float py2i = D > 1 ? __shfl_sync(FULL, py2, i) : 0.f;
                    const float pz2i = D > 2 ? __shfl_sync(FULL, pz2, i) : 0.f;
                    int add = 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) add += is_nbr<D>(cpi, px2i, py2i, pz2i, qq[u]);
                    const int r = (int)__reduce_add_sync(FULL, (unsigned)add);
                    if (lane == i) cnt += r;
                }
                pend = __ballot_sync(FULL, ((mine >> lane) & 1u) && cnt < lim);
            }
        }
    }
    if (valid) {
        const bool core = cnt >= min_pts;
        score[p] = core;
        if (counts_out) counts_out[o] = cnt;
        if (core_out) core_out[o] = core;
        if (!core) o = DB_NONE;
    }
    // the core point nearest A's centre, in doubled grid units (cell coordinate
    // floor(u / c) from the exact float form of GridGeom.inv_c)
    unsigned long long mid = ~0ull;
    if (o != DB_NONE) {
        const int c = a.g.c;
        const int ux = (int)pt.x, uy = (int)pt.y, uz = (int)pt.z;
        const int dx = 2 * ux - (2 * (int)((pt.x + 0.5f) * a.g.inv_c) * c + c - 1);
        const int dy = D > 1 ? 2 * uy - (2 * (int)((pt.y + 0.5f) * a.g.inv_c) * c + c - 1) : 0;
        const int dz = D > 2 ? 2 * uz - (2 * (int)((pt.z + 0.5f) * a.g.inv_c) * c + c - 1) : 0;
        mid = ((unsigned long long)(unsigned)(dx * dx + dy * dy + dz * dz) << 32) |
              (unsigned)(ux | (uy << 10) | (uz << 20));
    }
    o = seg_min_down(o, A);
    mid = seg_min_down(mid, A);
    const int Aprev = __shfl_up_sync(FULL, A, 1);
    if (valid && (lane == 0 || Aprev != A) && o != DB_NONE) {
        atomicMin(cell_rep + A, o);
        atomicMin(cell_mid + A, mid);
    }
    db::block_sum_add(a.ev + 0, ev);
}

// Merge pass (Section IV-C).  The core points of one cell are already one set
// (cells are cliques).  A warp takes one cell A at a time; its lanes look at
// up to 32 neighbouring cells B of A at once (the adjacent part of A's
// neighbour list in one launch, the outer ring in a second; each cell pair
// from its smaller key).  In the adjacent launch,
// a lane whose two central core points (cell_mid) are within eps unites the
// two sets at once; for every other B with cores that is not yet in A's set,
// the warp searches for one core pair within eps and unites the two sets at
// the first hit.  The search
// stages up to 128 points of the smaller cell in the warp's shared memory
// (coalesced loads) and runs the lanes over the larger cell against them.
template <int D>
__global__ void __launch_bounds__(256) grid_union_kernel(PairArgs a, const uint8_t *__restrict__ score, int *parent,
                                                         unsigned *status, bool far_ring,
                                                         const int *__restrict__ croot) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    __shared__ float4 ybuf[8][128];
    __shared__ uint8_t ycore[8][128];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int ncells = (int)(*a.ctr0 >> 32);
    float4 *yb = ybuf[wib];
    uint8_t *yc = ycore[wib];
    unsigned long long ev = 0;  // pair tests this lane accounts for
    const bool use_mid = !far_ring;
    for (int A = warp; A < ncells; A += nwarps) {
        // A's entries in one round of independent loads (wasted on a cell without cores)
        const int repA = a.cell_rep[A];
        const unsigned keyA = a.cell_key[A];
        const int sA = a.cell_start[A], cA = a.cell_count[A];
        const int nc = a.ncnt[A];
        const unsigned long long mkA = use_mid ? a.cell_mid[A] : 0ull;
        const int crA = croot ? croot[A] : -1;
        if (repA == DB_NONE) continue;
        const int *row = a.nbr + (size_t)A * a.g.noff;
        const int k_begin = far_ring ? (nc >> 16) : 0, k_end = far_ring ? (nc & 0xffff) : (nc >> 16);
        const float4 mA = unpack_point(mkA);
        const float cmA = a.g.Tp1 + mA.w, mx2 = 2.f * mA.x, my2 = 2.f * mA.y, mz2 = 2.f * mA.z;
        for (int k0 = k_begin; k0 < k_end; k0 += 32) {
            const int k = k0 + lane;
            const int B = k < k_end ? row[k] : -1;
            // B's entries in one round of independent loads; each cell pair is
            // examined from its smaller key
            const unsigned keyB = B >= 0 ? a.cell_key[B] : 0u;
            int repB = B >= 0 ? a.cell_rep[B] : DB_NONE;
            const unsigned long long mkB = (use_mid && B >= 0) ? a.cell_mid[B] : 0ull;
            const int crB = (croot && B >= 0) ? croot[B] : -2;
            if (keyB <= keyA) repB = DB_NONE;
            const float4 mB = repB != DB_NONE ? unpack_point(mkB) : make_float4(0.f, 0.f, 0.f, -1e30f);
            bool need = repB != DB_NONE;
            // cells whose snapshot roots agree are in one set already (sets only merge)
            if (need && croot) need = crB != crA;
            if (need) need = db::uf_find(parent, repA) != db::uf_find(parent, repB);
            // the two central core points first: a hit unites at once, lanes in parallel
            const bool hit = need && use_mid && is_nbr<D>(cmA, mx2, my2, mz2, mB);
            ev += need && use_mid;
            if (hit) db::uf_unite(parent, repA, repB, status);
            need = need && !hit;
            unsigned todo = __ballot_sync(FULL, need);
            bool first = true;
            while (todo) {
                const int l = __ffs(todo) - 1;
                todo &= todo - 1;
                const int Bl = __shfl_sync(FULL, B, l), rB = __shfl_sync(FULL, repB, l);
                if (!first) {  // an earlier union may have joined them
                    int same = 0;
                    if (lane == 0) same = db::uf_find(parent, repA) == db::uf_find(parent, rB);
                    if (__shfl_sync(FULL, same, 0)) continue;
                }
                first = false;
                const int sB = a.cell_start[Bl], cB = a.cell_count[Bl];
                const bool swap = cB > cA;  // lanes over the larger cell
                const int sX = swap ? sB : sA, cX = swap ? cB : cA, sY = swap ? sA : sB, cY = swap ? cA : cB;
                bool found = false;
                for (int y0 = 0; y0 < cY && !found; y0 += 128) {
                    const int ny = min(128, cY - y0);
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = lane + 32 * u;
                        if (k < ny) {
                            yb[k] = a.spts[sY + y0 + k];
                            yc[k] = score[sY + y0 + k];
                        }
                    }
                    __syncwarp();
                    for (int x0 = 0; x0 < cX && !found; x0 += 32) {
                        const int xi = x0 + lane;
                        const bool vx = xi < cX && score[sX + xi];
                        const unsigned vxm = __ballot_sync(FULL, vx);
                        if (!vxm) continue;
                        const float4 px = a.spts[sX + (xi < cX ? xi : 0)];
                        const float cp = a.g.Tp1 + px.w, px2 = 2.f * px.x, py2 = 2.f * px.y, pz2 = 2.f * px.z;
                        for (int k = 0; k < ny; ++k) {
                            if (!yc[k]) continue;
                            if (lane == 0) ev += (unsigned)__popc(vxm);
                            if (__any_sync(FULL, vx && is_nbr<D>(cp, px2, py2, pz2, yb[k]))) {
                                found = true;
                                break;
                            }
                        }
                    }
                }
                if (found && lane == 0) db::uf_unite(parent, repA, rB, status);
                __syncwarp();
            }
        }
    }
    db::block_sum_add(a.ev + (far_ring ? 3 : 1), ev);  // the outer ring has a counter of its own
}

// Border pass: each non-core point takes its smallest-index core neighbour
// (the reading used for points reachable from several clusters), a thread per
// grouped position; core positions have nothing to do.  The own cell's
// representative (its smallest core index) is a neighbour (cells are
// cliques); a neighbour cell is walked only when its representative can beat
// the current best, and a candidate is tested only when it is core with a
// smaller index.  As in the count pass, a point with few candidates walks them
// in its own thread, and the warp walks together for the points of a cell
// with many.  bord[p] gets the cell of the chosen core point (DB_NONE for
// noise): the point's label is that cell's root.
template <int D>
__global__ void __launch_bounds__(256) grid_border_kernel(PairArgs a, const uint8_t *__restrict__ score,
                                                          int *__restrict__ bord) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < a.n;
    const bool mine = valid && !score[p];
    const int A = valid ? a.scell[p] : -1 - lane;
    unsigned long long ev = 0;  // pair tests of this thread
    int best = DB_NONE, bc = DB_NONE;
    bool heavy = false;
    float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mine) {
        best = a.cell_rep[A];
        bc = best != DB_NONE ? A : DB_NONE;
        pt = a.spts[p];
        heavy = a.cell_cand[A] > kThreadWalkMax;
    }
    const float cp = a.g.Tp1 + pt.w, px2 = 2.f * pt.x, py2 = 2.f * pt.y, pz2 = 2.f * pt.z;
    if (mine && !heavy) {
        const int *row = a.nbr + (size_t)A * a.g.noff;
        const int nn = a.ncnt[A] & 0xffff;
        for (int k0 = 0; k0 < nn; k0 += 4) {
            int B[4], r[4], s[4], e[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) B[u] = k0 + u < nn ? row[k0 + u] : -1;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                r[u] = B[u] >= 0 ? a.cell_rep[B[u]] : DB_NONE;
                s[u] = B[u] >= 0 ? a.cell_start[B[u]] : 0;
                e[u] = B[u] >= 0 ? s[u] + a.cell_count[B[u]] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (r[u] >= best) continue;  // no core index of B can beat the current best
                for (int q = s[u]; q < e[u]; ++q) {
                    const uint8_t sc = score[q];  // three independent loads
                    const int qi = a.sidx[q];
                    const float4 pq = a.spts[q];
                    if (sc && qi < best) {
                        ++ev;
                        if (is_nbr<D>(cp, px2, py2, pz2, pq)) {
                            best = qi;
                            bc = B[u];
                        }
                    }
                }
            }
        }
    }
    unsigned hv = __ballot_sync(FULL, heavy);
    while (hv) {
        const int H = __shfl_sync(FULL, A, __ffs(hv) - 1);
        const unsigned mineH = __ballot_sync(FULL, heavy && A == H);
        hv &= ~mineH;
        const bool inH = (mineH >> lane) & 1u;
        const int *row = a.nbr + (size_t)H * a.g.noff;
        const int nn = a.ncnt[H] & 0xffff;
        for (int k0 = 0; k0 < nn; k0 += 32) {
            const int B = (k0 + lane < nn) ? row[k0 + lane] : -1;
            const int r = B >= 0 ? a.cell_rep[B] : DB_NONE;
            const int s = B >= 0 ? a.cell_start[B] : 0;
            int c = B >= 0 ? a.cell_count[B] : 0;
            const int bmax = (int)__reduce_max_sync(FULL, inH ? (unsigned)best : 0u);
            if (r >= bmax) c = 0;  // cannot beat any point's current best
            const int incl = warp_incl_scan(c), total = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < total; base += 128) {
                float4 qq[4];
                int qi[4], qc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = base + 32 * u + lane;
                    const int k = locate_lane(j, incl);
                    const int ex = __shfl_sync(FULL, incl, k) - __shfl_sync(FULL, c, k);  // lane k's first j
                    const int q = __shfl_sync(FULL, s, k) + (j - ex);
                    qc[u] = __shfl_sync(FULL, B, k);
                    const bool v = j < total;
                    const uint8_t scq = v ? score[q] : 0;  // three independent loads
                    const int qv = v ? a.sidx[q] : DB_NONE;
                    qq[u] = v ? a.spts[q] : make_float4(0.f, 0.f, 0.f, -1e30f);
                    qi[u] = scq ? qv : DB_NONE;
                }
                for (unsigned m = mineH; m; m &= m - 1) {
                    const int i = __ffs(m) - 1;
                    const float cpi = __shfl_sync(FULL, cp, i), px2i = __shfl_sync(FULL, px2, i);
                    const float py2i = D > 1 ? __shfl_sync(FULL, py2, i) : 0.f;
                    const float pz2i = D > 2 ? __shfl_sync(FULL, pz2, i) : 0.f;
                    const int bi = __shfl_sync(FULL, best, i);
                    int lb = bi, lc = DB_NONE;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool better = qi[u] < lb;  // else the pair needs no test
                        ev += better;
                        if (better && is_nbr<D>(cpi, px2i, py2i, pz2i, qq[u])) {
                            lb = qi[u];
                            lc = qc[u];
                        }
                    }
                    const int nb = (int)__reduce_min_sync(FULL, (unsigned)lb);
                    if (nb < bi) {  // warp-uniform: the one lane holding nb has its cell
                        const int w = __ffs(__ballot_sync(FULL, lb == nb)) - 1;
                        const int cw = __shfl_sync(FULL, lc, w);
                        if (lane == i) {
                            best = nb;
                            bc = cw;
                        }
                    }
                }
            }
        }
    }
    if (mine) bord[p] = bc;
    db::block_sum_add(a.ev + 2, ev);
}

// Root of every cell with cores, once per cell (a thread per cell), and the
// number of clusters: a cluster's root is the representative of its own cell.
// With ctr == null it only takes a snapshot of the roots (for the outer ring).
__global__ void grid_cell_root_kernel(const unsigned long long *ctr0, const int *__restrict__ cell_rep, int *parent,
                                      int *__restrict__ cell_root, unsigned long long *ctr) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    __shared__ int red[8];
    const int ncells = (int)(*ctr0 >> 32);
    int nr = 0;
    for (int A = blockIdx.x * blockDim.x + threadIdx.x; A < ncells; A += gridDim.x * blockDim.x) {
        const int rep = cell_rep[A];
        int root = -1;
        if (rep != DB_NONE) {
            root = db::uf_find(parent, rep);
            nr += root == rep;
        }
        cell_root[A] = root;
    }
    if (!ctr) return;  // a snapshot only (block-uniform)
    for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(FULL, nr, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nr;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (t) atomicAdd(ctr + 5, (unsigned long long)t);
    }
}

// Labels, a thread per grouped point: core points take their cell's root (the
// cluster's smallest core index), border points the root of the cell of their
// chosen core neighbour, noise -1.  Also counts core / border / noise points.
__global__ void grid_label_kernel(int n, const int *__restrict__ sidx, const int *__restrict__ scell,
                                  const uint8_t *__restrict__ score, const int *__restrict__ cell_root,
                                  const int *__restrict__ bord, int *__restrict__ labels, unsigned long long *ctr) {
    db::wait_prior_grid();  // started as a programmatic dependent
    db::allow_next_grid();
    __shared__ int red[3][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nc = 0, nb = 0, nn = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int orig = sidx[p];
        int lab;
        if (score[p]) {
            lab = cell_root[scell[p]];
            ++nc;
        } else {
            const int bc = bord[p];  // the cell of the chosen core neighbour
            if (bc == DB_NONE) {
                lab = -1;
                ++nn;
            } else {
                lab = cell_root[bc];
                ++nb;
            }
        }
        labels[orig] = lab;
    }
    int v[3] = {nc, nb, nn};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], o);
        if (lane == 0) red[k][wid] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        if (t) atomicAdd(ctr + 2 + threadIdx.x, (unsigned long long)t);
    }
}

__global__ void grid_candidates_kernel(GridGeom g, const unsigned long long *ctr0, const int *__restrict__ cell_count,
                                       const int *__restrict__ nbr, const int *__restrict__ ncnt, int own_listed,
                                       unsigned long long *out) {
    __shared__ unsigned long long red[32];
    const int ncells = (int)(*ctr0 >> 32);
    unsigned long long s = 0;
    for (int A = blockIdx.x * blockDim.x + threadIdx.x; A < ncells; A += gridDim.x * blockDim.x) {
        const long long ca = cell_count[A];
        long long t = own_listed ? 0 : ca;
        const int nn = ncnt[A] & 0xffff;
        for (int k = 0; k < nn; ++k) t += cell_count[nbr[(size_t)A * g.noff + k]];
        s += (unsigned long long)(ca * t);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (t) atomicAdd(out, t);
    }
}

int64_t isqrt64(int64_t v) {
    if (v <= 0) return 0;
    int64_t r = (int64_t)std::sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// Fork: work enqueued on the returned stream may run beside later work on st
// (the side stream, except while per-kernel marks are taken); join: st waits
// for it.
cudaStream_t fork(const DbWork &w, cudaStream_t st, int k) {
    if (!w.side || w.marks->on) return st;
    cudaEventRecord(w.fj[k], st);
    cudaStreamWaitEvent(w.side, w.fj[k], 0);
    return w.side;
}

void join(const DbWork &w, cudaStream_t st, cudaStream_t s2, int k) {
    if (s2 == st) return;
    cudaEventRecord(w.fj[k], s2);
    cudaStreamWaitEvent(st, w.fj[k], 0);
}

template <int D>
cudaError_t grid_pair_passes(const DbWork &w, const GridGeom &g, int n, int min_pts, bool exact, int32_t *labels,
                             int32_t *counts_out, uint8_t *core_out, cudaStream_t st) {
    unsigned long long *mid = reinterpret_cast<unsigned long long *>(w.cell_mid);  // 8 of its 16 bytes per cell
    PairArgs a{g,          w.ctr, n,          w.spts, w.sidx, w.scell,       w.cell_start, w.cell_count,
               w.cell_rep, mid,   w.cell_key, w.nbr,  w.ncnt, w.cell_cand, w.ctr + DB_CTR_EVAL};
    const int wgrid = 152 * 16;  // merge: 8 warps per block, warps stride over the cells
    const int pgrid = (n + 255) / 256;  // count, border: a thread per grouped position
    launch_dependent(grid_count_kernel<D>, pgrid, 256, st, a, min_pts, exact ? 1 : 0, w.score, w.cell_rep, mid,
                     counts_out, core_out);
    w.marks->kernel("grid_count", st);
    // The border pass needs the core flags but not the merge: it runs beside it.
    cudaStream_t s2 = fork(w, st, 2);
    launch_dependent(grid_border_kernel<D>, pgrid, 256, s2, a, w.score, w.border);
    w.marks->kernel("grid_border", s2);
    launch_dependent(grid_union_kernel<D>, wgrid, 256, st, a, w.score, w.parent, w.status, false, nullptr);
    w.marks->kernel("grid_union_near", st);
    if (g.noff > g.nnear) {
        // With a wide outer ring (3-D: 98 offsets), the roots after the adjacent
        // merge (into the hash counts, free after the cells kernel) let it skip
        // the cell pairs already joined without two finds each.
        const int *croot = nullptr;
        if (g.noff - g.nnear > 32) {
            launch_dependent(grid_cell_root_kernel, 152 * 4, 256, st, w.ctr, w.cell_rep, w.parent, w.hcount,
                             nullptr);
            w.marks->kernel("grid_root_snapshot", st);
            croot = w.hcount;
        }
        launch_dependent(grid_union_kernel<D>, wgrid, 256, st, a, w.score, w.parent, w.status, true, croot);
        w.marks->kernel("grid_union_far", st);
    }
    join(w, st, s2, 3);
    // the hash cursors are free after the scatter: they hold the cell roots
    launch_dependent(grid_cell_root_kernel, 152 * 4, 256, st, w.ctr, w.cell_rep, w.parent, w.hcursor, w.ctr);
    w.marks->kernel("grid_cell_root", st);
    launch_dependent(grid_label_kernel, pgrid, 256, st, n, w.sidx, w.scell, w.score, w.hcursor, w.border, labels,
                     w.ctr);
    w.marks->kernel("grid_label", st);
    return cudaGetLastError();
}

}  // namespace

bool grid_geometry(int32_t d, int64_t Tc, int64_t n, GridGeom *g) {
    if (d < 1 || d > 3) return false;
    const int64_t m = isqrt64(Tc / d);
    const int64_t c = m + 1;
    const int64_t s = isqrt64(Tc);
    const int64_t r = (s + c - 1) / c;
    if (r > 2) return false;  // cannot happen for d <= 3 (s < sqrt(3) c)
    g->d = d;
    g->c = (int32_t)c;
    g->G = (int32_t)((1024 + c - 1) / c);
    g->Tc = (int32_t)Tc;
    g->Tp1 = (float)(Tc + 1);
    g->inv_c = (float)(1.0 / (double)c);
    int bits = 10;
    while ((int64_t(1) << bits) < 2 * n) ++bits;
    g->hbits = bits;
    g->dense = 0;  // the launch may switch to a direct table
    int k = 0;
    const int rz = d > 2 ? (int)r : 0, ry = d > 1 ? (int)r : 0, rx = (int)r;
    for (int oz = -rz; oz <= rz; ++oz)
        for (int oy = -ry; oy <= ry; ++oy)
            for (int ox = -rx; ox <= rx; ++ox) {
                if (!ox && !oy && !oz) continue;
                int64_t md = 0;
                for (int o : {ox, oy, oz})
                    if (o) {
                        int64_t gap = (int64_t)(std::abs(o) - 1) * c + 1;
                        md += gap * gap;
                    }
                if (md > Tc) continue;
                g->off[k++] = make_char4((signed char)ox, (signed char)oy, (signed char)oz, 0);
            }
    g->noff = k;
    // Adjacent cells (every |o_k| <= 1) first: the merge pass runs them before the
    // outer ring, which then mostly finds its cell pairs already united.
    std::stable_partition(g->off, g->off + k, [](char4 o) {
        return std::abs(o.x) <= 1 && std::abs(o.y) <= 1 && std::abs(o.z) <= 1;
    });
    int nn = 0;
    while (nn < k && std::abs(g->off[nn].x) <= 1 && std::abs(g->off[nn].y) <= 1 && std::abs(g->off[nn].z) <= 1) ++nn;
    g->nnear = nn;
    return true;
}

cudaError_t launch_grid_path(const DbWork &w, const GridGeom &g0, const float *x, int64_t n64, int32_t min_pts,
                             bool exact, int32_t *labels, int32_t *counts_out, uint8_t *core_out, cudaStream_t st) {
    const int n = (int)n64;
    if ((int64_t(1) << g0.hbits) > w.hcap || g0.noff > w.noff_cap) return cudaErrorInvalidValue;
    // When all G^d cells fit the table, a cell's slot is its key: no hashing,
    // and the cells pass scans G^d slots instead of 2^hbits (2-D: 65,536 cells
    // at eps = 0.005 against 2^20 slots for 500,000 points).
    int64_t all_cells = 1;
    for (int k = 0; k < g0.d; ++k) all_cells *= g0.G;
    GridGeom g = g0;
    g.dense = all_cells <= w.hcap ? 1 : 0;
    const int64_t H = g.dense ? all_cells : (int64_t(1) << g.hbits);
    cudaError_t e;
    if (!g.dense && (e = cudaMemsetAsync(w.hkey, 0xff, sizeof(unsigned) * H, st))) return e;
    if ((e = cudaMemsetAsync(w.hcount, 0, sizeof(int) * H, st))) return e;
    // occupancy bitmap of all G^d cells for the hashed table, when it fits its buffer
    const int64_t occ_words = (all_cells + 31) / 32;
    unsigned *occ = (!g.dense && occ_words <= w.occ_cap) ? w.occ : nullptr;
    if (occ && (e = cudaMemsetAsync(occ, 0, sizeof(unsigned) * occ_words, st))) return e;
    const int nb = (n + 255) / 256;
    launch_dependent(grid_prep_kernel, nb, 256, st, x, n, g, w.hkey, w.hcount, w.slot_of, w.pts4, w.parent,
                     w.status);
    w.marks->kernel("grid_prep", st);
    if ((e = launch_grid_cells(w, g, occ, reinterpret_cast<unsigned long long *>(w.cell_mid), st))) return e;
    // The neighbour lists need the cell table but not the grouped points.
    cudaStream_t s2 = fork(w, st, 0);
    if ((e = launch_grid_nbrs(w, g, occ, s2))) return e;
    launch_dependent(grid_scatter_kernel, nb, 256, st, n, w.slot_of, w.hcursor, w.hpack, w.pts4, w.spts, w.sidx,
                     w.scell);
    w.marks->kernel("grid_scatter", st);
    join(w, st, s2, 1);
    if ((e = cudaGetLastError())) return e;
    switch (g.d) {
        case 1: return grid_pair_passes<1>(w, g, n, min_pts, exact, labels, counts_out, core_out, st);
        case 2: return grid_pair_passes<2>(w, g, n, min_pts, exact, labels, counts_out, core_out, st);
        default: return grid_pair_passes<3>(w, g, n, min_pts, exact, labels, counts_out, core_out, st);
    }
}

cudaError_t launch_grid_cells(const DbWork &w, const GridGeom &g, unsigned *occ, unsigned long long *midkey,
                              cudaStream_t st) {
    int64_t H = int64_t(1) << g.hbits;
    if (g.dense) {
        H = 1;
        for (int k = 0; k < g.d; ++k) H *= g.G;
    }
    const int cells_per_block = 256 * CELLS_PER_THREAD;
    launch_dependent(grid_cells_kernel, (unsigned)((H + cells_per_block - 1) / cells_per_block), 256, st, (int)H,
                     g.dense, w.hkey, w.hcount, w.hpack, w.hcursor, w.cell_start, w.cell_count, w.cell_key,
                     w.cell_rep, midkey, occ, w.ctr);
    w.marks->kernel("grid_cells", st);
    return cudaGetLastError();
}

cudaError_t launch_grid_nbrs(const DbWork &w, const GridGeom &g, const unsigned *occ, cudaStream_t st) {
    launch_dependent(grid_nbr_kernel, 152 * 16, 256, st, g, w.ctr, w.cell_key, w.hpack, occ, w.cell_count, w.nbr,
                     w.ncnt, w.cell_cand);
    w.marks->kernel("grid_nbrs", st);
    return cudaGetLastError();
}

cudaError_t launch_grid_candidates(const DbWork &w, const GridGeom &g, int64_t /*n*/, bool own_cell_listed,
                                   cudaStream_t st) {
    grid_candidates_kernel<<<152 * 4, 256, 0, st>>>(g, w.ctr, w.cell_count, w.nbr, w.ncnt, own_cell_listed ? 1 : 0,
                                                    w.ctr + 1);
    w.marks->kernel("grid_candidates", st);
    return cudaGetLastError();
}
