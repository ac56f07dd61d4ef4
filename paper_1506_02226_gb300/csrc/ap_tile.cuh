// ap_tile.cuh — the all-pairs SIMT tile (Section IV-A/IV-B), shared by the
// single-instance kernels (pairs_simt.cu) and the batched kernels (batch.cu).
//
// The score of a pair is T + 1 - D(p,q), an integer, and q is a neighbour
// iff score >= 1; __saturatef(score) is then exactly 0 or 1.
// Rows hold centred units v = u - 512 in [-512, 511] (D is unchanged).
//   MODE_GRAM   (d <= 16): score = (T+1 - |p|^2) - |q|^2 + sum_k (2v_pk) v_qk
//               in FP32 (Section IV-B's hoisted form).  After k terms the
//               partial sum lies in [T+1 - sum_i (|v_pi| + |v_qi|)^2, T+1] (the
//               terms not yet added are sums of squares, and each one added is
//               at least -(|v_pi| + |v_qi|)^2 + v_pi^2 + v_qi^2), and
//               (|v_pi| + |v_qi|)^2 <= 1023^2, so every partial sum is an
//               integer of magnitude below 16 * 1023^2 < 2^24: FP32 is exact.
//   MODE_DIRECT (FP32, T + 1 <= 2^24): score = (T+1) - sum (v_pk-v_qk)^2.
//               Partial sums only decrease; they are exact while >= -2^24, and
//               once below that they stay below 1, so the decision is exact.
//   MODE_INT    otherwise: the same in int32.
#pragma once

#include <climits>

#include "internal.cuh"

namespace aptile {

constexpr int BM = 64, BN = 64, NT = 256;  // the single-instance tile; batched row tiles are 16 * RM rows
enum { PASS_COUNT = 0, PASS_UNION = 1, PASS_BORDER = 2 };
enum { MODE_GRAM = 0, MODE_DIRECT = 1, MODE_INT = 2 };

struct ApArgs {
    const float *P;  // packed units, row stride DP
    int n;
    float Tp1;       // T + 1 (exact: T + 1 <= 2^24 whenever a float mode is used)
    int Tc;          // T clamped to d*1023^2
    const uint8_t *core;
    int *count;
    int *parent;
    int *border;
    unsigned *status;
    int ntiles;
    int splits;
    int early;  // count pass: stop a row tile once every row has this many (0: exact counts)
    unsigned long long *ev;  // pair tests evaluated, [0] count, [1] merge, [2] border pass (nullable)
    // Rows reordered (nullable: rows in index order).  Row j is point perm[j];
    // count and core stay by row, parent and border by point index.
    const int *perm = nullptr;
    // Per 64-row column tile and per row tile (16 * RM rows), the least and
    // greatest unit of its rows on each of the DP axes: lo[0..15], hi[16..31]
    // (nullable: no tile pruning).  Two tiles whose boxes lie more than eps
    // apart hold no neighbour pair.
    const float *tbox = nullptr;
    const float *tbox_rows = nullptr;
};

// RM consecutive floats of a shared-memory row at a multiple of RM (vector loads).
template <int RM>
__device__ __forceinline__ void load_rows(const float *src, float (&v)[RM]) {
    if constexpr (RM == 2) {
        const float2 a = *reinterpret_cast<const float2 *>(src);
        v[0] = a.x;
        v[1] = a.y;
    } else {
#pragma unroll
        for (int h = 0; h < RM / 4; ++h) {
            const float4 a = *reinterpret_cast<const float4 *>(src + 4 * h);
            v[4 * h] = a.x;
            v[4 * h + 1] = a.y;
            v[4 * h + 2] = a.z;
            v[4 * h + 3] = a.w;
        }
    }
}


// One block's work: row tile rt (16 * RM rows; RM rows by 4 columns per
// thread) against column tiles [ct_begin, ct_end) of 64 columns.  Called by
// the all-pairs kernel below (RM = 4) and, once per work item, by the batched
// kernel (batch.cu, RM chosen by its autotuner).  All branches that return
// are block-uniform.
template <int DP, int MODE, int PASS, int RM = 4>
__device__ __forceinline__ void ap_tile_body(const ApArgs &a, int rt, int ct_begin, int ct_end) {
    constexpr int BMr = 16 * RM;
    __shared__ __align__(16) float As[DP][BMr];
    __shared__ __align__(16) float Bs[DP][BN];
    __shared__ float An[BMr], Bn[BN];
    __shared__ uint8_t Ac[BMr], Bc[BN];
    __shared__ uint8_t Aiso[BMr];  // border: the row has no neighbour but itself
    __shared__ int Aperm[BMr], Bperm[BN];
    __shared__ float Abox[32];

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = rt * BMr;
    __syncthreads();  // the previous work item of this block is done with the tiles

    // ---- the row tile stays in shared memory for the whole block (Section IV-A) ----
    if constexpr (DP % 4 == 0) {  // rows of 4, 8 or 16 units: 16-byte vector loads (rows are 16-byte aligned)
        for (int e = tid; e < BMr * (DP / 4); e += NT) {
            const int r = e / (DP / 4), k4 = e - r * (DP / 4);
            const int row = row0 + r;
            const float4 v = (row < a.n) ? reinterpret_cast<const float4 *>(a.P + (size_t)row * DP)[k4]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
            As[4 * k4][r] = v.x;
            As[4 * k4 + 1][r] = v.y;
            As[4 * k4 + 2][r] = v.z;
            As[4 * k4 + 3][r] = v.w;
        }
    } else {
        for (int e = tid; e < BMr * DP; e += NT) {
            int r = e / DP, k = e - (e / DP) * DP;
            int row = row0 + r;
            As[k][r] = (row < a.n) ? a.P[(size_t)row * DP + k] : 0.f;
        }
    }
    if (PASS != PASS_COUNT)
        for (int r = tid; r < BMr; r += NT) Ac[r] = (row0 + r < a.n) ? a.core[row0 + r] : 0;
    if (PASS != PASS_COUNT && a.perm)
        for (int r = tid; r < BMr; r += NT) Aperm[r] = (row0 + r < a.n) ? a.perm[row0 + r] : 0;
    if (a.tbox && tid < 32) Abox[tid] = a.tbox_rows[(size_t)rt * 32 + tid];
    // A non-core point's count is exact (the count pass never stops early on a
    // tile holding one), so a count of 1 means no neighbour but itself.
    if (PASS == PASS_BORDER)
        for (int r = tid; r < BMr; r += NT) Aiso[r] = (row0 + r < a.n) && !Ac[r] && a.count[row0 + r] <= 1;
    __syncthreads();
    if (MODE == MODE_GRAM) {
        // Per-row terms hoisted out of the pair loop (Section IV-B): T+1-|p|^2 and 2p.
        for (int r = tid; r < BMr; r += NT) {
            float nrm = 0.f;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
                float v = As[k][r];
                nrm = fmaf(v, v, nrm);
                As[k][r] = 2.f * v;
            }
            An[r] = a.Tp1 - nrm;
        }
    }
    int want_rows = 1;
    if (PASS == PASS_UNION || PASS == PASS_BORDER) {
        int mine = 0;
        for (int r = tid; r < BMr; r += NT)
            if (row0 + r < a.n) mine |= (PASS == PASS_UNION) ? (Ac[r] != 0) : (Ac[r] == 0 && !Aiso[r]);
        want_rows = __syncthreads_or(mine);
    } else {
        __syncthreads();
    }
    if (!want_rows) return;

    float rc[RM];
    int prior[RM];  // count pass with early exit: counts other work already added
    int bm[RM];
    int rootp[RM];  // union: last known root of each row's set
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        rc[i] = 0.f;
        prior[i] = 0;
        bm[i] = INT_MAX;
        rootp[i] = -2;
    }
    if (PASS == PASS_COUNT && a.early > 0) {
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const int p = row0 + ty * RM + i;
            prior[i] = p < a.n ? a.count[p] : INT_MAX / 2;
        }
        int done = 1;
#pragma unroll
        for (int i = 0; i < RM; ++i) done &= prior[i] >= a.early;
        if (__syncthreads_and(done)) return;  // every row is already core
    }
    const int rows_in = min(BMr, a.n - row0);
    unsigned long long evaluated = 0;  // pairs of the tiles scored (thread 0's count)

    for (int ct = ct_begin; ct < ct_end; ++ct) {
        if (a.tbox) {
            // squared gap between the two tiles' boxes (integers below 2^24 in
            // FP32: exact); every thread finds the same, so the skip is uniform
            const float *cb = a.tbox + (size_t)ct * 32;
            float gap2 = 0.f;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
                const float g = fmaxf(fmaxf(cb[k] - Abox[16 + k], Abox[k] - cb[16 + k]), 0.f);
                gap2 = fmaf(g, g, gap2);
            }
            if (gap2 > (float)a.Tc) continue;  // no pair of the two tiles is within eps
        }
        const int col0 = ct * BN;
        __syncthreads();
        if (MODE == MODE_GRAM) {
            if (tid < BN) {
                const int col = col0 + tid;
                float nrm = 0.f;
                if (col < a.n) {
                    if constexpr (DP % 4 == 0) {  // 16-byte vector loads of the column's units
#pragma unroll
                        for (int k4 = 0; k4 < DP / 4; ++k4) {
                            const float4 v = reinterpret_cast<const float4 *>(a.P + (size_t)col * DP)[k4];
                            Bs[4 * k4][tid] = v.x;
                            Bs[4 * k4 + 1][tid] = v.y;
                            Bs[4 * k4 + 2][tid] = v.z;
                            Bs[4 * k4 + 3][tid] = v.w;
                            nrm = fmaf(v.x, v.x, nrm);
                            nrm = fmaf(v.y, v.y, nrm);
                            nrm = fmaf(v.z, v.z, nrm);
                            nrm = fmaf(v.w, v.w, nrm);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < DP; ++k) {
                            float v = a.P[(size_t)col * DP + k];
                            Bs[k][tid] = v;
                            nrm = fmaf(v, v, nrm);
                        }
                    }
                    Bn[tid] = -nrm;
                } else {
#pragma unroll
                    for (int k = 0; k < DP; ++k) Bs[k][tid] = 0.f;
                    Bn[tid] = -1e30f;  // padding column: never a neighbour
                }
            }
        } else {
            for (int e = tid; e < BN * DP; e += NT) {
                int c = e / DP, k = e - (e / DP) * DP;
                int col = col0 + c;
                Bs[k][c] = (col < a.n) ? a.P[(size_t)col * DP + k] : (MODE == MODE_INT ? 0.f : 1e18f);
            }
        }
        int want_cols = 1;
        if (PASS != PASS_COUNT) {
            int mine = 0;
            for (int c = tid; c < BN; c += NT) {
                int col = col0 + c;
                uint8_t f = (col < a.n) ? a.core[col] : 0;
                Bc[c] = f;
                if (a.perm) Bperm[c] = (col < a.n) ? a.perm[col] : 0;
                mine |= f;
            }
            want_cols = __syncthreads_or(mine);
        } else {
            __syncthreads();
        }
        if (!want_cols) continue;
        if (tid == 0) evaluated += (unsigned long long)rows_in * min(BN, a.n - col0);

        float acc[RM][4];
        int iacc[RM][4];
        if (MODE == MODE_GRAM) {
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = An[ty * RM + i] + Bn[tx * 4 + j];
        } else if (MODE == MODE_DIRECT) {
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = a.Tp1;
        } else {
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) iacc[i][j] = a.Tc;
        }
#pragma unroll
        for (int k = 0; k < DP; ++k) {
            float ar[RM];
            load_rows<RM>(&As[k][ty * RM], ar);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (MODE == MODE_GRAM) {
                        acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
                    } else if (MODE == MODE_DIRECT) {
                        float df = ar[i] - br[j];
                        acc[i][j] = fmaf(-df, df, acc[i][j]);
                    } else {
                        int di = (int)ar[i] - (int)br[j];
                        iacc[i][j] -= di * di;
                    }
                }
        }
        // ---- fused consumer (Section IV-B: no distance is stored) ----
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const int r = ty * RM + i, p = row0 + r;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = tx * 4 + j, q = col0 + c;
                bool nb;
                if (MODE == MODE_INT) nb = (iacc[i][j] >= 0) && (q < a.n);
                else nb = acc[i][j] >= 1.f;
                if (PASS == PASS_COUNT) {
                    if (MODE == MODE_INT) rc[i] += nb ? 1.f : 0.f;
                    else rc[i] += __saturatef(acc[i][j]);
                } else if (PASS == PASS_UNION) {
                    if (nb && p < q && Ac[r] && Bc[c]) {
                        const int po = a.perm ? Aperm[r] : p, qo = a.perm ? Bperm[c] : q;
                        // q already hangs under p's last known root: same set, skip
                        // (a plain, possibly stale read is enough: a stale parent
                        // equal to the root still means the same set)
                        if (a.parent[qo] != rootp[i])
                            rootp[i] = db::uf_unite_root(a.parent, po, qo, a.status);
                    }
                } else {
                    if (nb && p < a.n && !Ac[r] && Bc[c]) bm[i] = min(bm[i], a.perm ? Bperm[c] : q);
                }
            }
        }
        if (PASS == PASS_COUNT && a.early > 0 && ((ct - ct_begin) & 3) == 3) {
            // every 4 tiles: stop once every row of the tile has min_pts neighbours
            int done = 1;
#pragma unroll
            for (int i = 0; i < RM; ++i) {
                int v = (int)rc[i];
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                done &= prior[i] + v >= a.early;
            }
            if (__syncthreads_and(done)) break;  // counts are flushed after the loop
        }
        if (PASS == PASS_BORDER && !a.perm) {
            // Columns grow with ct, so a row's first hit is its smallest core
            // neighbour in this block's range: stop once every row has one (or
            // needs none).  (Reordered rows have no such order.)
            int done = 1;
#pragma unroll
            for (int i = 0; i < RM; ++i) {
                int v = bm[i];
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
                const int r = ty * RM + i;
                done &= (v != INT_MAX) || (row0 + r >= a.n) || Ac[r] || Aiso[r];
            }
            if (__syncthreads_and(done)) break;
        }
    }

    if (tid == 0 && a.ev && evaluated) atomicAdd(a.ev + PASS, evaluated);
    if (PASS == PASS_COUNT) {
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            int v = (int)rc[i];
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const int p = row0 + ty * RM + i;
            if (tx == 0 && p < a.n && v) atomicAdd(a.count + p, v);
        }
    } else if (PASS == PASS_BORDER) {
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            int v = bm[i];
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
            const int p = row0 + ty * RM + i;
            if (tx == 0 && p < a.n && v != INT_MAX) atomicMin(a.border + (a.perm ? Aperm[ty * RM + i] : p), v);
        }
    }
}

}  // namespace aptile
