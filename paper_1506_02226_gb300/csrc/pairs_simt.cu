// pairs_simt.cu — all-pairs eps-test on the CUDA cores, fused with its consumer.
//
// Section IV-A tiles the pair loop through shared memory (each thread keeps its
// own point in registers, a block stages TPB points at a time) and unrolls the
// inner loop; Section IV-B fuses the distance test with the neighbour count, so
// the distance matrix is never stored; Section IV-B's last step moves the
// per-row terms out of the loop (the Gram form
// dist = |t|^2 + |p|^2 - 2 t.p), used here up to d = 16.  Here a 256-thread block owns a 64x64 tile of
// (row, column) pairs; each thread scores a 4x4 micro-tile from shared memory.
// The same tile loop feeds three consumers:
//   PASS_COUNT   neighbour counts (step 2, core detection)
//   PASS_UNION   union of core-core eps-edges (step 3, merging; Section IV-C)
//   PASS_BORDER  smallest core neighbour of each non-core point
//
// Exact arithmetic.  The score of a pair is T + 1 - D(p,q), an integer, and q
// is a neighbour iff score >= 1; __saturatef(score) is then exactly 0 or 1.
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
#include <climits>

#include "ap_tile.cuh"

using namespace aptile;

namespace {
__global__ void prep_dense_kernel(const float *__restrict__ x, int64_t n, int d, int dp, float *__restrict__ P,
                                  unsigned *status) {
    const int64_t total = n * dp;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / dp;
        int k = (int)(i - r * dp);
        float v = 0.f;
        if (k < d) {
            int u;
            bad |= !db::on_grid(x[r * d + k], u);
            v = (float)(u - 512);  // centred: exact Gram form up to d = 16
        }
        P[i] = v;
    }
    if (bad) atomicOr(status, DB_EBIT_NOT_QUANTISED);
}

template <int DP, int MODE, int PASS>
__global__ void __launch_bounds__(NT) ap_tile_kernel(ApArgs a) {
    const int rt = blockIdx.x;
    const int first = (PASS == PASS_UNION) ? rt : 0;  // union: upper triangle only
    const int span = a.ntiles - first;
    const int per = (span + a.splits - 1) / a.splits;
    const int ct_begin = first + blockIdx.y * per;
    const int ct_end = min(a.ntiles, ct_begin + per);
    if (ct_begin >= ct_end) return;
    ap_tile_body<DP, MODE, PASS>(a, rt, ct_begin, ct_end);
}

__global__ void core_init_kernel(int n, int min_pts, const int *__restrict__ count, uint8_t *__restrict__ core,
                                 int *__restrict__ parent, int *__restrict__ border) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        core[i] = count[i] >= min_pts;
        parent[i] = i;
        border[i] = DB_NONE;
    }
}

template <int DP, int MODE, int PASS>
cudaError_t launch_pass(const ApArgs &a, const DbWork &w, cudaStream_t st) {
    dim3 grid(a.ntiles, a.splits);
    ap_tile_kernel<DP, MODE, PASS><<<grid, NT, 0, st>>>(a);
    w.marks->kernel(PASS == PASS_COUNT ? "ap_count" : (PASS == PASS_UNION ? "ap_union" : "ap_border"), st);
    return cudaGetLastError();
}

template <int DP, int MODE>
cudaError_t run_passes(ApArgs a, const DbWork &w, int n, int min_pts, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(int32_t) * (size_t)n, st);
    if (e) return e;
    if ((e = launch_pass<DP, MODE, PASS_COUNT>(a, w, st))) return e;
    core_init_kernel<<<min((n + 255) / 256, 4096), 256, 0, st>>>(n, min_pts, w.count, w.core, w.parent, w.border);
    w.marks->kernel("core_init", st);
    if ((e = cudaGetLastError())) return e;
    if ((e = launch_pass<DP, MODE, PASS_UNION>(a, w, st))) return e;
    return launch_pass<DP, MODE, PASS_BORDER>(a, w, st);
}

template <int DP>
cudaError_t dispatch_mode(int mode, ApArgs a, const DbWork &w, int n, int min_pts, cudaStream_t st) {
    if constexpr (DP <= 16) {
        return run_passes<DP, MODE_GRAM>(a, w, n, min_pts, st);
    } else {
        if (mode == MODE_DIRECT) return run_passes<DP, MODE_DIRECT>(a, w, n, min_pts, st);
        return run_passes<DP, MODE_INT>(a, w, n, min_pts, st);
    }
}

}  // namespace

int32_t dp_for(int32_t d) {
    if (d <= 4) return d == 4 ? 4 : d;  // 1, 2, 3, 4
    if (d <= 8) return 8;
    if (d <= 16) return 16;
    if (d <= 32) return 32;
    if (d <= 64) return 64;
    return -1;
}

cudaError_t launch_prep_dense(const DbWork &w, const float *x, int64_t n, int32_t d, int32_t dp, cudaStream_t st) {
    int64_t total = n * dp;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    if (blocks < 1) blocks = 1;
    prep_dense_kernel<<<blocks, 256, 0, st>>>(x, n, d, dp, w.P, w.status);
    w.marks->kernel("prep_dense", st);
    return cudaGetLastError();
}

cudaError_t launch_core_init(const DbWork &w, int64_t n, int32_t min_pts, cudaStream_t st) {
    core_init_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>((int)n, min_pts, w.count, w.core,
                                                                                  w.parent, w.border);
    w.marks->kernel("core_init", st);
    return cudaGetLastError();
}

cudaError_t launch_allpairs_simt(const DbWork &w, int64_t n64, int32_t d, int32_t dp, int64_t Tc, int32_t min_pts,
                                 bool exact_counts, cudaStream_t st) {
    const int n = (int)n64;
    ApArgs a;
    a.P = w.P;
    a.n = n;
    a.Tc = (int)Tc;
    a.Tp1 = (float)(Tc + 1);
    a.core = w.core;
    a.count = w.count;
    a.parent = w.parent;
    a.border = w.border;
    a.status = w.status;
    a.ntiles = (n + BM - 1) / BM;
    a.early = exact_counts ? 0 : min_pts;
    a.ev = w.ctr + DB_CTR_EVAL;
    // Enough blocks to fill 152 SMs a few times over, splitting the column range.
    int splits = (4 * 152 + a.ntiles - 1) / a.ntiles;
    a.splits = std::max(1, std::min(splits, a.ntiles));
    int mode = (d <= 16) ? MODE_GRAM : ((Tc + 1 <= (1 << 24)) ? MODE_DIRECT : MODE_INT);
    switch (dp) {
        case 1: return dispatch_mode<1>(mode, a, w, n, min_pts, st);
        case 2: return dispatch_mode<2>(mode, a, w, n, min_pts, st);
        case 3: return dispatch_mode<3>(mode, a, w, n, min_pts, st);
        case 4: return dispatch_mode<4>(mode, a, w, n, min_pts, st);
        case 8: return dispatch_mode<8>(mode, a, w, n, min_pts, st);
        case 16: return dispatch_mode<16>(mode, a, w, n, min_pts, st);
        case 32: return dispatch_mode<32>(mode, a, w, n, min_pts, st);
        case 64: return dispatch_mode<64>(mode, a, w, n, min_pts, st);
        default: return cudaErrorInvalidValue;
    }
}
