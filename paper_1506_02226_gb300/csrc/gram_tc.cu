// gram_tc.cu — tensor-core Gram form of the pair test (tcgen05, sm_103a).
//
// Section IV-B of the paper rewrites the squared distance as
//   dist(t, p) = |t|^2 + |p|^2 - 2 t.p
// and hoists the per-point terms out of the loop.  For d >= 16 the dot
// products t.p of a 128 x 256 tile of pairs are one dense contraction, so they
// run on the 5th-generation tensor cores: tcgen05.mma with FP16 or BF16
// operands staged in shared memory and an FP32 accumulator in tensor memory.
//
// Exactness.  Coordinates are centred, v = u - 512 in [-512, 511]:
//   FP16 holds every v exactly, products are exact, and for d <= 64 every
//   partial sum of G = v_p . v_q is an integer of magnitude <= 64 * 2^18 =
//   2^24, so FP32 accumulation leaves G exact.  Then, with beta_q = |v_q|^2 and
//   alpha_p = |v_p|^2 - T (both exact integers, |.| <= 2^24 because T < 2^24),
//   w = fma(2, G, -beta_q) rounds at most once, and w >= alpha_p decides
//   D(p,q) <= T exactly: when |2G - beta| > 2^24 the rounded w stays on the
//   same side of alpha.  The stated FP16 band is therefore 0; the diagnostic
//   pass (TC_VERIFY, dbscan_tc_verify) recomputes every pair exactly on the
//   device and reports max |2G - 2G_exact| = 0 and no pair decided wrongly.
//   BF16 (8-bit significand) cannot hold every v, so each is split into two
//   BF16 terms, v = hi + lo with hi = bf16(v) and lo = v - hi in {-1, 0, 1}
//   (both exact), and the MMA sums hi.hi + hi.lo + lo.hi over K, i.e. G minus
//   sum(lo_p lo_q), |sum| <= K.  Its partial sums stay below
//   K (512^2 + 2 * 512) < 2^25, so each of the 3K accumulations beyond 2^24
//   rounds by at most 2: |G_bf16 - G| <= 7K.  With the roundings of w (at most
//   4 each), a pair is decided directly when |w - alpha| > 16K, and rechecked
//   exactly otherwise (rho = sqrt(16K) (1 + 2^-10) per row and column, so that
//   rho_p rho_q covers the band).  The band holds only pairs within 16K
//   squared units of the threshold.
//
// Folded FP16 count.  The count pass appends one 16-column chunk to each
// operand row so that the MMA also subtracts the column term: rows carry
// 1, 2^11, 2^15 and columns the negated digits of h_q = ceil(|v_q|^2 / 2)
// (integers FP16 holds exactly), and the accumulator holds G - h_q.  Every
// term of that sum is an integer and their magnitudes add up to at most
// |v_p||v_q| + h_q <= (|v_p|^2 + 2|v_q|^2 + 1) / 2, so when
// 3 max|v|^2 + 1 <= 2^25 every partial sum, in any order of accumulation, is
// an integer of magnitude <= 2^24 and the accumulator is exact.  The columns
// are ordered even |v_q|^2 first (odd ones from the next 256-column tile on),
// so each tile has one parity f and each row one threshold per parity:
// D <= T iff G - h_q >= ceil((|v_p|^2 - T - f) / 2).  The epilogue then needs
// one saturating add per pair and no column data.  Inputs with larger norms
// (only the extreme corners of the grid reach them at d = 64) run the same
// pass on G alone with the column norms; the pass decides on the device.
//
// Data layout.  Each operand list (all points, core points, non-core points)
// is packed once into 128-row tiles in the canonical K-major layout without
// swizzle: 8 x 8 core matrices of 128 contiguous bytes, K-adjacent core
// matrices 128 B apart (leading byte offset) and 8-row groups KG*128 B apart
// (stride byte offset).  A 128-row A tile or a 256-row B tile is therefore one
// contiguous block, fetched by a single cp.async.bulk (TMA) copy.  Per-point
// metadata {beta, rho, index} rides along in the same copy group.
//
// CTA roles (320 threads for the FP16 count and the verification, 576
// otherwise; one CTA per SM, persistent over work items of one row unit and
// a chunk of column tiles):
//   warp 0      producer: bulk copies of A tiles (2 buffers, each holding the
//               item's row tiles: two for the FP16 count and border, one
//               otherwise), B tiles (a ring of 3 stages for the FP16 count, 4
//               for the FP16 border, 5 for the merge, 2 for BF16, each freed by
//               the MMA commit of its tile) and their metadata (a ring of 4 to
//               6 stages, freed by the epilogue), completion via mbarrier
//               transaction counts
//   warp 1      TMEM owner (alloc/dealloc of 512 columns) and MMA issuer:
//               K/16 tcgen05.mma (M=128, N=256, K=16) per MMA tile into one of
//               two 256-column accumulators (with two row tiles, each B tile
//               feeds one MMA tile per row tile, one per accumulator);
//               tcgen05.commit signals the epilogue
//   warps 2..   epilogue: tcgen05.ld of the accumulator (one TMEM lane = one
//               row; with two row tiles a group of warps per row tile and
//               accumulator, in the FP16 count one warp per lane quadrant,
//               otherwise two or four warps per lane quadrant split the 256
//               columns), the exact decision above, and the pass's consumer:
//               neighbour count, union of core-core neighbours, or smallest
//               core neighbour.
// Every wait is bounded (about two seconds of %globaltimer); on expiry the CTA
// records DB_EBIT_TIMEOUT, stops issuing work, waits for its own copies and
// MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int TM = 128, TN = 256;
constexpr int FP16_BAND = 0;  // FP16 Gram products are exact (see above): no band
// BF16 candidate filter: lowering of its threshold that covers the rounding
// difference between the filter score and the rare path's score (below 16).
constexpr float kBf16FilterSlack = 16.f;
// BF16 band in units of w = 2G - |v_q|^2 for padded dimension K (see above).
__host__ __device__ constexpr int bf16_band(int K) { return 16 * K; }

enum { TC_COUNT = 0, TC_UNION = 1, TC_BORDER = 2, TC_VERIFY = 3 };

// Epilogue warps per CTA.  The FP16 count: two groups of four warps (one per
// TMEM lane quadrant), one group per row tile of the item and accumulator
// buffer, and each warp decides all 256 columns of its rows, loading 32
// columns ahead of the ones it decides (measured against the alternatives,
// with one row tile per item: four warps of 64 columns per quadrant 6.75 ms,
// two of 128 on every tile 6.27, this 6.14, sixteen warps in two groups 6.30).
// FP16 border: two groups of eight, two warps per quadrant of 128 columns
// each.  Merge and BF16: four per quadrant (64 columns each).  Groups of 32
// columns in both (the candidate scores and the accumulator copy fit the
// 16-warp register budget).  Verification: two per quadrant, groups of 64.
template <int PASS, bool BF16>
constexpr int epi_warps() {
    return (PASS == TC_COUNT && !BF16) ? 8 : (PASS != TC_VERIFY ? 16 : 8);
}
template <int PASS, bool BF16>
constexpr int group_cols() {
    return (PASS == TC_COUNT && !BF16) ? 128 : (PASS == TC_VERIFY ? 64 : 32);
}
template <int PASS, bool BF16>
constexpr int tc_threads() {
    return 32 * (2 + epi_warps<PASS, BF16>());
}

// Per-point metadata, in list order, stored as one 2 KB block per 128 points:
// beta[128] (|v|^2), rho[128] (BF16 band factor), idx[128] (point index, -1
// for padding), pad[128].  A 128-row A tile takes one block, a 256-column B
// tile two consecutive blocks; each epilogue warp reads one of them.
struct MetaBlock {
    float beta[TM];
    float rho[TM];
    int idx[TM];
    float beta_f[TM];  // the candidate filter's column term: beta (FP16), beta - rho^2 rounded (BF16)
};

struct TcArgs {
    const uint16_t *opR;  // packed row operand (tiles of 128 rows)
    const MetaBlock *metaR;
    const uint16_t *opC;  // packed column operand (tiles of 256 rows)
    const MetaBlock *metaC;
    const int *nR_ptr;    // device-side list lengths
    const int *nC_ptr;
    int K;                // padded dimension (multiple of 16, <= 64)
    int ks;               // stored operand columns per row: K, 2K (BF16 terms) or K + 16 (FP16 count)
    int T;                // threshold (< 2^24)
    int bf16;
    int pass;
    int upper;                   // union: only pairs i < j of one list
    unsigned long long wait_ns;  // budget of every barrier wait
    const int *bmax_ptr;  // FP16 count: largest |v|^2 of the input (decides the folded form)
    const int *nE_ptr;    // FP16 count: even-norm points at the head of the column list
    int stall;                   // test hook: the MMA issuer issues nothing
    const int16_t *v16;   // centred units by point index, row stride K (exact recheck)
    int *count;
    int *parent;
    int *border;
    unsigned *status;
    unsigned long long *ctr;  // [6] band pairs, [7] verify: disagreements outside the band, [8] max |w - exact|
    int col_chunk;            // column tiles per work item
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps (issuing nothing) until the phase completes or about 0.5 ms pass.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(500000u)
        : "memory");
    return ok != 0;
}

// Bounded wait: about two seconds, or until another role has given up.
// Waiting threads sleep inside try_wait, so they take no issue slots from the
// epilogue warps sharing their SM sub-partition.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                       unsigned long long budget_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        for (int i = 0; i < 8; ++i)
            if (mbar_try_wait_sleep(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > budget_ns) {
            *abort_flag = 1;
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag: the abort path uses it to let a
// role's own copies or MMAs in flight land before the CTA's memory goes away.
__device__ __noinline__ bool mbar_wait_quiet(uint64_t *bar, uint32_t parity, unsigned long long budget_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (globaltimer() - t0 <= budget_ns)
        if (mbar_try_wait_sleep(bar, parity)) return true;
    return false;
}
constexpr unsigned long long kDrainNs = 100000000ull;  // 100 ms: copies and MMAs land in microseconds

// Packed FP32 pairs (sm_100 and later): two lanes of arithmetic per
// instruction, each rounded exactly as its scalar counterpart.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Optional pipeline diagnostics (compile with -DDB_TC_WAIT_STATS): cycles each
// role spends blocked on each barrier, summed per pass into the counters
// listed at the end of the kernel.
#ifdef DB_TC_WAIT_STATS
#define TC_WAIT(acc, expr) ({ long long _t0 = clock64(); bool _r = (expr); acc += clock64() - _t0; _r; })
#else
#define TC_WAIT(acc, expr) (expr)
#endif

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, M=128, N=256, K=16, FP32 accumulate.
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Waits for this thread's TMEM loads; the registers of r pass through the
// statement, so no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld_dep(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Shared-memory matrix descriptor: no swizzle, K-major, LBO = 128 B (next core
// matrix along K), SBO = KG * 128 B (next 8-row group), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo_bytes) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A/B = F16 or BF16, both K-major,
// N = 256 (bits 17..22 hold N/8), M = 128 (bits 24..28 hold M/16).
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(TN >> 3) << 17) |
           ((uint32_t)(TM >> 4) << 24);
}

// Exact D(p,q) <= T from the centred int16 rows (the recheck of band pairs).
__device__ __noinline__ int exact_sqdist(const int16_t *__restrict__ v16, int K, int p, int q) {
    const int4 *a = reinterpret_cast<const int4 *>(v16 + (size_t)p * K);
    const int4 *b = reinterpret_cast<const int4 *>(v16 + (size_t)q * K);
    int s = 0;
    for (int c = 0; c < K / 8; ++c) {
        int4 x = a[c], y = b[c];
        const int xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            int d0 = (int)(int16_t)(xs[h] & 0xffff) - (int)(int16_t)(ys[h] & 0xffff);
            int d1 = (xs[h] >> 16) - (ys[h] >> 16);
            s += d0 * d0 + d1 * d1;
        }
    }
    return s;
}

// Shared memory of one CTA: KC stored operand columns per row (64 for FP16,
// 128 for the two BF16 terms), NS stages of B tiles (5 for FP16: 32 KB each;
// 2 for BF16: 64 KB each) and NM stages of their metadata.  A B stage is free
// again once its MMAs have completed; the epilogue holds only the tile's
// metadata, in a ring of its own, so the operand ring runs up to NS tiles
// ahead of the MMAs whatever the epilogue's pace.
template <int KC, int NS, int NM, int RTN, int CR, int NA = 2>
struct __align__(16) SmemT {
    static constexpr int NSTAGE = NS;
    static constexpr int NMETA = NM;
    static constexpr int NABUF = NA;
    uint16_t A[NA * RTN][TM * KC];   // NA buffers of RTN row tiles (16 KB each for FP16, 32 KB for BF16)
    uint16_t B[NS][TN * KC];
    MetaBlock metaA[NA * RTN];       // 2 KB per row tile
    MetaBlock metaB[NM][2];          // NM x 4 KB
    uint64_t a_full[NA], a_empty[NA];
    uint64_t b_full[NS], b_empty[NS];
    uint64_t m_empty[NM];            // metadata stage released by the epilogue warps of its tile
    uint64_t t_full[2], t_empty[2];
    uint64_t drain;                  // abort path: one more MMA commit, waited for by the issuer
    uint32_t tmem_base;
    int abort_flag;
    int drain_failed;                // a role's bounded drain wait gave up
    // union pass (CR = 512): hints of the column points' sets, per accumulator
    // buffer and column half (128 each, shared by the four warps of a half; a
    // buffer is refilled only after all its epilogue warps have released it)
    int colroot[CR];
};

// Shared memory of each pass.  FP16 count: two row tiles per item of K + 16
// stored columns (the folded chunk, below), 3 B stages of 40 KB and 4 metadata
// stages; FP16 border: two row tiles, 4 and 5; FP16 merge and verification 5
// and 6; BF16 2 and 6.
// Compile-time knobs of the FP16 count (the defaults measured best or within
// noise of the alternatives): column tiles per work item, A buffers, B stages
// and metadata stages.
#ifndef DB_TC_COUNT_CHUNK
#define DB_TC_COUNT_CHUNK 32
#endif
#ifndef DB_TC_C16_NA
#define DB_TC_C16_NA 2
#endif
#ifndef DB_TC_C16_NS
#define DB_TC_C16_NS 3
#endif
#ifndef DB_TC_C16_NM
#define DB_TC_C16_NM 4
#endif
template <int PASS, bool BF16>
struct TcSmem {
    static constexpr bool RT2 = !BF16 && (PASS == TC_COUNT || PASS == TC_BORDER);
    static constexpr bool C16 = !BF16 && PASS == TC_COUNT;
    using type = SmemT<BF16 ? 128 : (C16 ? 80 : 64), BF16 ? 2 : (C16 ? DB_TC_C16_NS : (RT2 ? 4 : 5)),
                       C16 ? DB_TC_C16_NM : (RT2 ? 5 : 6), RT2 ? 2 : 1, PASS == TC_UNION ? 512 : 1,
                       C16 ? DB_TC_C16_NA : 2>;
};

// Work item w covers row unit rt (TMU rows: one 128-row tile, or two for the
// FP16 count and border) and column tiles [c0, c1) of one column chunk.
// Count and border passes: ch = w / nrt, rt = w % nrt, so the CTAs running at
// one time share their column chunk and its B tiles come from L2.  Merge pass
// (a.upper): rt = w / nchunk and the chunk rotates with the row tile, so the
// CTAs running at one time work on different column chunks: the first visit to
// a chunk's points unites and flattens them, and later visits find them in
// their cluster's set (the core operand, at most n x 128 bytes, stays in L2).
template <int TMU>
__device__ __forceinline__ bool item_range(const TcArgs &a, int w, int nR, int nC, int &rt, int &c0, int &c1) {
    const int nrt = (nR + TMU - 1) / TMU, nct = (nC + TN - 1) / TN;
    const int nchunk = (nct + a.col_chunk - 1) / a.col_chunk;
    if (w >= nrt * nchunk) return false;
    int ch;
    if (a.upper) {
        rt = w / nchunk;
        ch = (w - rt * nchunk + rt) % nchunk;
    } else {
        ch = w / nrt;
        rt = w - ch * nrt;
    }
    c0 = ch * a.col_chunk;
    c1 = min(nct, c0 + a.col_chunk);
    if (a.upper) c0 = max(c0, (rt * TMU) / TN);  // pairs i < j only: skip tiles left of the diagonal
    return true;
}

// Rare path of the epilogue: a pair that may be a neighbour.  Returns bit 0 =
// neighbour, bit 1 = it was inside the rounding band and was rechecked.
template <bool BF16>
__device__ __noinline__ int decide_candidate(float wv, float alpha, float rho_p, float rho_q, const int16_t *v16,
                                             int K, int p, int q, int T) {
    const bool sure = BF16 ? (fmaf(-rho_p, rho_q, wv) >= alpha) : (wv > alpha + (float)FP16_BAND);
    if (sure) return 1;
    return (exact_sqdist(v16, K, p, q) <= T ? 1 : 0) | 2;
}

// Union of p's and q's sets; returns a root the merged set had at some moment
// (out of line: keeps the union-find loop out of the epilogue's registers).
__device__ __noinline__ int unite_root(int *parent, int p, int q, unsigned *status) {
    return db::uf_unite_root(parent, p, q, status);
}


template <int PASS, bool BF16>
__global__ void __launch_bounds__(tc_threads<PASS, BF16>(), 1) tc_pass_kernel(TcArgs a) {
    constexpr int EPI_WARPS = epi_warps<PASS, BF16>();
    // FP16 count and border: each work item holds two row tiles, so every B
    // tile feeds two MMA tiles, one per accumulator buffer, and two groups of
    // epilogue warps drain them, a group per buffer (and row tile).
    constexpr int RTN = (!BF16 && (PASS == TC_COUNT || PASS == TC_BORDER)) ? 2 : 1;
    constexpr int TMU = TM * RTN;
    constexpr int EPI_GROUPS = (PASS == TC_COUNT && !BF16) || RTN == 2 ? 2 : 1;
    constexpr int TILE_WARPS = EPI_WARPS / EPI_GROUPS;  // epilogue warps that read one tile
    constexpr int GW = group_cols<PASS, BF16>();    // columns per group
    constexpr int WPQ = TILE_WARPS / 4;             // warps per lane quadrant on one tile
    constexpr int NG = (TN / WPQ) / GW;             // groups per epilogue warp and tile
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // Align by pointer arithmetic on the shared array (not through an integer),
    // so the compiler keeps shared-space loads, stores and atomics.
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    using Smem = typename TcSmem<PASS, BF16>::type;
    constexpr int NSTAGE = Smem::NSTAGE, NMETA = Smem::NMETA, NA = Smem::NABUF;
    Smem &S = *reinterpret_cast<Smem *>(smem_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nR = *a.nR_ptr, nC = *a.nC_ptr;
    const int nrt = (nR + TMU - 1) / TMU, nct = (nC + TN - 1) / TN;
    const int nchunk = (nct + a.col_chunk - 1) / a.col_chunk;
    const int nitems = nrt * nchunk;
    if ((int)blockIdx.x >= nitems) return;  // nothing for this CTA (before any TMEM use)

    volatile int *abort_flag = &S.abort_flag;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(&S.a_full[i], 1);
            mbar_init(&S.a_empty[i], 1 + EPI_WARPS);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.t_full[i], 1);
            mbar_init(&S.t_empty[i], TILE_WARPS);
        }
        for (int i = 0; i < NSTAGE; ++i) {
            mbar_init(&S.b_full[i], 1);
            mbar_init(&S.b_empty[i], 1);  // the MMA commit of the tile
        }
        for (int i = 0; i < NMETA; ++i) mbar_init(&S.m_empty[i], RTN == 2 ? EPI_WARPS : TILE_WARPS);
        mbar_init(&S.drain, 1);
        S.abort_flag = 0;
        S.drain_failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(&S.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const int K = a.K;
    const int KS = a.ks;  // stored columns per row: v, [hi | lo] (BF16) or [v | folded chunk] (FP16 count)
    const int KG = KS / 8;
    // FP16 count: the column term folded into the MMA when the input's norms
    // keep it exact (3 max|v|^2 + 1 <= 2^25, see the count epilogue), and the
    // column tiles [0, ctE) that hold the even-norm points.
    bool fold = false;
    int nE = 0, ctE = 0;
    if constexpr (PASS == TC_COUNT && !BF16) {
        fold = 3ll * (long long)*a.bmax_ptr + 1 <= (1ll << 25);
        nE = *a.nE_ptr;
        ctE = (nE + TN - 1) / TN;
    }
    long long w_prod = 0, w_mma_b = 0, w_mma_t = 0, w_epi = 0, t_start = clock64();
    (void)w_prod, (void)w_mma_b, (void)w_mma_t, (void)w_epi, (void)t_start;
    const uint32_t a_bytes = (uint32_t)(TM * KS * 2), b_bytes = (uint32_t)(TN * KS * 2);

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int t = 0, ia = 0;
            int last_b[NSTAGE], last_a[NA];  // phase of each buffer's last copy (-1: none)
            for (int i = 0; i < NA; ++i) last_a[i] = -1;
            for (int s = 0; s < NSTAGE; ++s) last_b[s] = -1;
            for (int w = blockIdx.x; w < nitems && !*abort_flag; w += gridDim.x, ++ia) {
                int rt, c0, c1;
                item_range<TMU>(a, w, nR, nC, rt, c0, c1);
                const int ab = ia % NA;
                if (!mbar_wait(&S.a_empty[ab], ((ia / NA) & 1) ^ 1, abort_flag, a.wait_ns)) break;
                // RTN consecutive row tiles (the packed list holds whole 256-row tiles)
                mbar_arrive_expect_tx(&S.a_full[ab], RTN * (a_bytes + (uint32_t)sizeof(MetaBlock)));
                bulk_g2s(S.A[ab * RTN], a.opR + (size_t)rt * RTN * TM * KS, RTN * a_bytes, &S.a_full[ab]);
                bulk_g2s(&S.metaA[ab * RTN], a.metaR + rt * RTN, RTN * (uint32_t)sizeof(MetaBlock), &S.a_full[ab]);
                last_a[ab] = ia / NA;
                for (int ct = c0; ct < c1; ++ct, ++t) {
                    const int s = t % NSTAGE, m = t % NMETA;
                    if (!TC_WAIT(w_prod, mbar_wait(&S.b_empty[s], ((t / NSTAGE) & 1) ^ 1, abort_flag, a.wait_ns)) ||
                        !TC_WAIT(w_prod, mbar_wait(&S.m_empty[m], ((t / NMETA) & 1) ^ 1, abort_flag, a.wait_ns)))
                        break;
                    // the metadata lands in its own ring, counted by the tile's b_full
                    mbar_arrive_expect_tx(&S.b_full[s], b_bytes + 2 * sizeof(MetaBlock));
                    bulk_g2s(S.B[s], a.opC + (size_t)ct * TN * KS, b_bytes, &S.b_full[s]);
                    bulk_g2s(&S.metaB[m][0], a.metaC + 2 * ct, 2 * sizeof(MetaBlock), &S.b_full[s]);
                    last_b[s] = t / NSTAGE;
                }
            }
            // On a clean finish every copy has been consumed, so it has landed.
            // After an abort, wait (bounded) until the last copy into each buffer
            // has landed: a buffer holds at most one copy in flight, so the
            // parity of its last phase identifies it.
            if (*abort_flag) {
                bool ok = true;
                for (int s = 0; s < NSTAGE; ++s)
                    if (last_b[s] >= 0) ok &= mbar_wait_quiet(&S.b_full[s], last_b[s] & 1, kDrainNs);
                for (int ab = 0; ab < NA; ++ab)
                    if (last_a[ab] >= 0) ok &= mbar_wait_quiet(&S.a_full[ab], last_a[ab] & 1, kDrainNs);
                if (!ok) S.drain_failed = 1;
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        // (test hook a.stall: it issues nothing, so the other roles' bounded
        // waits expire and the CTA takes the abort path with no MMA in flight)
        if (lane == 0 && !a.stall) {
            const uint32_t idesc = idesc_f16(BF16);
            int t = 0, ia = 0;
            bool clean = true;
            unsigned long long evaluated = 0;  // pairs of the tiles multiplied
            for (int w = blockIdx.x; w < nitems && !*abort_flag; w += gridDim.x, ++ia) {
                int rt, c0, c1;
                item_range<TMU>(a, w, nR, nC, rt, c0, c1);
                const int ab = ia % NA;
                if (!mbar_wait(&S.a_full[ab], (ia / NA) & 1, abort_flag, a.wait_ns)) break;
                bool ok = true;
                for (int ct = c0; ct < c1 && ok; ++ct, ++t) {
                    const int s = t % NSTAGE;
                    if (!TC_WAIT(w_mma_b, mbar_wait(&S.b_full[s], (t / NSTAGE) & 1, abort_flag, a.wait_ns))) {
                        ok = false;
                        break;
                    }
                    const uint32_t b_addr = smem_u32(S.B[s]);
                    for (int r = 0; r < RTN; ++r) {
                        // accumulator buffer and its use count: with two row tiles each
                        // buffer serves one of them on every B tile; otherwise the
                        // buffers alternate between tiles
                        const int b = RTN == 2 ? r : (t & 1), use = RTN == 2 ? t : (t >> 1);
                        if (!TC_WAIT(w_mma_t, mbar_wait(&S.t_empty[b], (use & 1) ^ 1, abort_flag, a.wait_ns))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        // the RTN row tiles lie back to back (a_bytes each) from the buffer's start
                        const uint32_t a_addr = smem_u32(S.A[ab * RTN]) + (uint32_t)r * a_bytes;
                        // FP16: sum over K of v_p v_q.  BF16: hi.hi + hi.lo + lo.hi, the
                        // lo columns K/16 chunks after the hi ones (256 B per chunk).
                        const int kch = K / 16;
                        const int kmma = fold ? KS / 16 : kch;  // the folded chunk follows the K columns of v
                        for (int kk = 0; kk < kmma; ++kk) {
                            const uint64_t ad = smem_desc(a_addr + kk * 256, KG * 128);
                            const uint64_t bd = smem_desc(b_addr + kk * 256, KG * 128);
                            mma_f16(tmem + (uint32_t)(b * TN), ad, bd, idesc, kk > 0 ? 1u : 0u);
                            if (BF16) {
                                const uint64_t bl = smem_desc(b_addr + (kch + kk) * 256, KG * 128);
                                const uint64_t al = smem_desc(a_addr + (kch + kk) * 256, KG * 128);
                                mma_f16(tmem + (uint32_t)(b * TN), ad, bl, idesc, 1u);
                                mma_f16(tmem + (uint32_t)(b * TN), al, bd, idesc, 1u);
                            }
                        }
                        mma_commit(&S.t_full[b]);  // accumulator ready for the epilogue
                        // (FP16 count: the gap between the even and odd points holds no pairs)
                        const int ncols = (PASS == TC_COUNT && !BF16 && ct < ctE) ? min(TN, nE - ct * TN)
                                                                                 : min(TN, nC - ct * TN);
                        evaluated += (unsigned long long)max(0, min(TM, nR - (rt * RTN + r) * TM)) * ncols;
                    }
                    if (!ok) break;
                    mma_commit(&S.b_empty[s]);  // operands of this stage consumed
                }
                mma_commit(&S.a_empty[ab]);
                if (!ok) {
                    clean = false;
                    break;
                }
            }
            // Wait for the arrivals of the last commits, so that none lands after
            // the CTA has exited.  Stage s was last used by tile t_s (its phase
            // t_s / NSTAGE); A buffer ab by item ia_ab (phase ia_ab / NA).
            if (clean && !*abort_flag) {
                for (int s = 0; s < NSTAGE && s < t; ++s) {
                    const int ts = s + ((t - 1 - s) / NSTAGE) * NSTAGE;
                    mbar_wait(&S.b_empty[s], (ts / NSTAGE) & 1, abort_flag, a.wait_ns);
                }
                for (int ab = 0; ab < NA && ab < ia; ++ab) {
                    const int il = ab + ((ia - 1 - ab) / NA) * NA;
                    mbar_wait(&S.a_empty[ab], (il / NA) & 1, abort_flag, a.wait_ns);
                }
            }
            if (a.pass != TC_VERIFY && evaluated) atomicAdd(a.ctr + DB_CTR_EVAL + a.pass, evaluated);
            if (PASS == TC_COUNT && !BF16 && fold && blockIdx.x == 0) a.ctr[DB_CTR_TC_FOLD] = 1ull;
            // After an abort: one more commit, which arrives once every MMA this
            // thread issued has completed, and a bounded wait for it.
            if (*abort_flag && t > 0) {
                mma_commit(&S.drain);
                if (!mbar_wait_quiet(&S.drain, 0, kDrainNs)) S.drain_failed = 1;
            }
        }
    } else {
        // ---------------- epilogue ----------------
        const int ew = warp - 2;                  // 0..EPI_WARPS-1
        const int quad = warp & 3;                // TMEM lane quadrant this warp may access
        const int colbase = ((ew >> 2) % WPQ) * (TN / WPQ);  // first column of this warp in the tile
        const int half = colbase >> 7;            // 128-column metadata block holding it
        const int moff = colbase & 127;           // its offset in that block
        const int r = quad * 32 + lane;           // row within the tile
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        int t = 0, ia = 0;
        unsigned long long band_cnt = 0, bad_cnt = 0;
        unsigned maxerr = 0;
        for (int w = blockIdx.x; w < nitems; w += gridDim.x, ++ia) {
            int rt, c0, c1;
            item_range<TMU>(a, w, nR, nC, rt, c0, c1);
            const int ab = ia % NA;
            // the row tile of the item this warp serves (its group's, with two)
            const int rsel = RTN == 2 ? ew / TILE_WARPS : 0;
            if (!__all_sync(0xffffffffu, mbar_wait(&S.a_full[ab], (ia / NA) & 1, abort_flag, a.wait_ns))) break;
            const MetaBlock &ma = S.metaA[ab * RTN + rsel];
            const float beta_p = ma.beta[r], rho_p = ma.rho[r];
            const int p = ma.idx[r];
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.a_empty[ab]);
            const int i_row = (rt * RTN + rsel) * TM + r;  // list index of this row
            const bool row_ok = i_row < nR && p >= 0;
            const float alpha = beta_p - (float)a.T;  // |v_p|^2 - T, exact
            // folded FP16 count: 1 - thr_f for the even (f = 0) and odd (f = 1)
            // column tiles, thr_f = ceil((|v_p|^2 - T - f) / 2) = (a_p - f + 1) >> 1
            const int a_p = row_ok ? (int)beta_p - a.T : 0;
            const float c_even = (float)(1 - ((a_p + 1) >> 1)), c_odd = (float)(1 - (a_p >> 1));
            (void)c_even, (void)c_odd;
            int cnt = 0, bmin = INT_MAX;
            // union: a member of p's set (its parent, then the last root seen)
            int rootp = (PASS == TC_UNION && row_ok) ? db::ld_relaxed(a.parent + p) : -2;
            bool ok = true;
            for (int ct = c0; ct < c1; ++ct, ++t) {
                // accumulator buffer of this warp's tile and its use count (see the MMA issuer)
                const int m = t % NMETA, b = RTN == 2 ? rsel : (t & 1), use = RTN == 2 ? t : (t >> 1);
                if (RTN == 1 && EPI_GROUPS == 2 && b != ew / TILE_WARPS) continue;  // the other group's tile
                // warp-uniform outcome: the accumulator loads below are warp-collective
                // the accumulator is usually ready: test once inline before the bounded wait
                if (!__all_sync(0xffffffffu,
                                mbar_try_wait(&S.t_full[b], use & 1) ||
                                    TC_WAIT(w_epi, mbar_wait(&S.t_full[b], use & 1, abort_flag, a.wait_ns)))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const MetaBlock &mc = S.metaB[m][half];
                int *colroot = S.colroot + (PASS == TC_UNION ? (b * 2 + half) * 128 : 0);
                bool hints = false;  // union: colroot filled for this tile
                // union: the parents of this warp's GW * NG column points of the
                // tile, loaded now so that their latency hides behind the
                // accumulator loads and scores
                int pr[NG];
                if (PASS == TC_UNION) {
#pragma unroll
                    for (int k = 0; k < NG; ++k) {
                        const int q = mc.idx[moff + lane + GW * k];
                        pr[k] = q >= 0 ? db::ld_relaxed(a.parent + q) : -1;
                    }
                }
                if constexpr (PASS == TC_COUNT && !BF16) {
                    // all 256 columns in eight groups of 32: the next group's TMEM load
                    // is in flight while this group is decided
                    const uint32_t tb = tmem + lane_base + (uint32_t)(b * TN);
                    unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};  // +0.0f in both halves
                    uint32_t ga[32], gb[32];
                    auto all_groups = [&](auto &&decide) {
                        tmem_ld32_nowait(tb, ga);
                        tmem_wait_ld_dep(ga);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            uint32_t(&cur)[32] = (i & 1) ? gb : ga;
                            uint32_t(&nxt)[32] = (i & 1) ? ga : gb;
                            if (i + 1 < 8) tmem_ld32_nowait(tb + (uint32_t)(32 * (i + 1)), nxt);
                            decide(cur, 32 * i);
                            if (i + 1 < 8) tmem_wait_ld_dep(nxt);
                        }
                    };
                    if (fold) {
                        // Folded form: the accumulator holds G - h_q exactly, with
                        // h_q = ceil(|v_q|^2 / 2) (see the count's operands), and this
                        // tile's columns share the parity f of |v_q|^2.  D <= T iff
                        // G - h_q >= thr_f = ceil((|v_p|^2 - T - f) / 2), so
                        // sat(acc + 1 - thr_f) is exactly 1 for a neighbour and 0
                        // otherwise: one saturating add per pair, one packed add per
                        // two pairs, no column data.
                        const float cf = ct < ctE ? c_even : c_odd;
                        all_groups([&](uint32_t(&g)[32], int) {
#pragma unroll
                            for (int h = 0; h < 16; ++h)
                                acc[h & 3] = f2_add(acc[h & 3], f2_pack(__saturatef(__uint_as_float(g[2 * h]) + cf),
                                                                        __saturatef(__uint_as_float(g[2 * h + 1]) + cf)));
                        });
                    } else {
                        // G alone (exact), so sat(2G - |v_q|^2 + 1 - alpha) is exactly
                        // 1 for a neighbour (T - D + 1 >= 1) and 0 otherwise.  Two
                        // pairs per packed FFMA (w' = |v_q|^2 - 2G, the exact negation
                        // of fma(2, G, -|v_q|^2): round-to-nearest is symmetric), one
                        // saturating subtract per pair (c1 - w' = c1 + w, the same
                        // rounding as before) and one packed add per two pairs.
                        const float c1 = 1.f - alpha;
                        const unsigned long long m2 = f2_pack(-2.f, -2.f);
                        all_groups([&](uint32_t(&g)[32], int col) {
                            const float *bet = S.metaB[m][col >> 7].beta + (col & 127);
#pragma unroll
                            for (int j8 = 0; j8 < 4; ++j8) {
                                const float4 ba = *reinterpret_cast<const float4 *>(bet + 8 * j8);
                                const float4 bb = *reinterpret_cast<const float4 *>(bet + 8 * j8 + 4);
                                const float bq[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                                for (int h = 0; h < 4; ++h) {
                                    const unsigned long long w = f2_fma(
                                        f2_pack(__uint_as_float(g[8 * j8 + 2 * h]), __uint_as_float(g[8 * j8 + 2 * h + 1])),
                                        m2, f2_pack(bq[2 * h], bq[2 * h + 1]));
                                    float w0, w1;
                                    f2_unpack(w, w0, w1);
                                    acc[h] = f2_add(acc[h], f2_pack(__saturatef(c1 - w0), __saturatef(c1 - w1)));
                                }
                            }
                        });
                    }
                    float sm[8];
#pragma unroll
                    for (int h = 0; h < 4; ++h) f2_unpack(acc[h], sm[2 * h], sm[2 * h + 1]);
                    if (row_ok) cnt += (int)(((sm[0] + sm[1]) + (sm[2] + sm[3])) + ((sm[4] + sm[5]) + (sm[6] + sm[7])));
                } else
#pragma unroll 1
                for (int hc = 0; hc < NG; ++hc) {
                    const int cb = moff + hc * GW;  // column within the 128-column block
                    uint32_t g[GW];
                    const uint32_t taddr = tmem + lane_base + (uint32_t)(b * TN + half * 128 + cb);
                    tmem_ld32_nowait(taddr, g);
                    if constexpr (GW >= 64) tmem_ld32_nowait(taddr + 32, g + 32);
                    if constexpr (GW >= 128) {
                        tmem_ld32_nowait(taddr + 64, g + 64);
                        tmem_ld32_nowait(taddr + 96, g + 96);
                    }
                    tmem_wait_ld();
                    if (PASS == TC_VERIFY) {
                        if (!row_ok) continue;
#pragma unroll 1
                        for (int j = 0; j < GW; ++j) {
                            const int q = mc.idx[cb + j];
                            if (q < 0) continue;
                            const float gv = __uint_as_float(g[j & (GW - 1)]);
                            const float wv = fmaf(2.f, gv, -mc.beta[cb + j]);
                            const int D = exact_sqdist(a.v16, K, p, q);
                            // 2G exactly, from integers: |v_p|^2 + |v_q|^2 - D (the betas are exact)
                            const long long two_g = (long long)beta_p + (long long)mc.beta[cb + j] - D;
                            const double err = fabs(2.0 * (double)gv - (double)two_g);
                            maxerr = max(maxerr, (unsigned)fmin(err, 4.0e9));
                            const bool nb_exact = D <= a.T;
                            const float del = BF16 ? rho_p * mc.rho[cb + j] : (float)FP16_BAND;
                            const bool in_band = fabsf(wv - alpha) <= del;
                            band_cnt += in_band;
                            if (!in_band && ((wv >= alpha) != nb_exact)) ++bad_cnt;
                            cnt += nb_exact;
                        }
                        continue;
                    }
                    // Union / border / BF16: one FFMA per pair; the maxima of the
                    // eight strided column groups (j mod 8) come from the first
                    // three levels of an FMNMX tree.  Only groups whose maximum can
                    // reach the threshold are rescanned.
                    // Candidate score per pair: 2G - beta_f, computed as the exact
                    // negation beta_f - 2G two pairs per packed FFMA (round-to-nearest
                    // is symmetric), minus its minimum.  FP16: beta_f = |v_q|^2.
                    // BF16: beta_f = |v_q|^2 - rho^2 (rho is the same for every point),
                    // so the score is the rare path's 2G - |v_q|^2 + rho_p rho_q up to
                    // a few units of rounding (at most 2 per rounding at magnitudes
                    // below 2^25, two roundings on each side); the threshold is lowered
                    // by kBf16FilterSlack to cover them, and the rare path decides.
                    const float thr = BF16 ? alpha - kBf16FilterSlack : alpha - (float)FP16_BAND;
                    float mx;
                    float nv[GW];  // after the tree, nv[i] = minimum over the columns j = i (mod 8)
                    {
                        const unsigned long long m2 = f2_pack(-2.f, -2.f);
#pragma unroll
                        for (int j4 = 0; j4 < GW / 4; ++j4) {
                            const float4 b4 = *reinterpret_cast<const float4 *>(&mc.beta_f[cb + 4 * j4]);
                            const unsigned long long w01 =
                                f2_fma(f2_pack(__uint_as_float(g[4 * j4 + 0]), __uint_as_float(g[4 * j4 + 1])), m2,
                                       f2_pack(b4.x, b4.y));
                            const unsigned long long w23 =
                                f2_fma(f2_pack(__uint_as_float(g[4 * j4 + 2]), __uint_as_float(g[4 * j4 + 3])), m2,
                                       f2_pack(b4.z, b4.w));
                            f2_unpack(w01, nv[4 * j4 + 0], nv[4 * j4 + 1]);
                            f2_unpack(w23, nv[4 * j4 + 2], nv[4 * j4 + 3]);
                        }
#pragma unroll
                        for (int w2 = GW / 2; w2 >= 8; w2 >>= 1)
#pragma unroll
                            for (int j = 0; j < w2; ++j) nv[j] = fminf(nv[j], nv[j + w2]);
                        mx = -fminf(fminf(fminf(nv[0], nv[1]), fminf(nv[2], nv[3])),
                                    fminf(fminf(nv[4], nv[5]), fminf(nv[6], nv[7])));
                    }
                    // Border: the columns are core points in ascending index order,
                    // so a group whose first index is not below the best so far
                    // cannot improve it.
                    const bool need = row_ok && mx >= thr && (PASS != TC_BORDER || mc.idx[cb] < bmin);
                    if (!__any_sync(0xffffffffu, need)) continue;
                    if (PASS == TC_UNION && !hints) {
                        // the parents loaded at the tile's start, for this warp's columns
                        // (the warps of the other lane quadrants that share them write
                        // them too: any value is a member of the column point's set)
#pragma unroll
                        for (int k = 0; k < NG; ++k) colroot[moff + lane + GW * k] = pr[k];
                        __syncwarp();
                        hints = true;
                    }
                    // Rare path: the lanes that need it build the mask of
                    // possible neighbours (for FP16 exactly the neighbours; padding
                    // columns never pass, their beta is 1e30).  The merge pass also
                    // drops the columns whose set hint equals the row's: those pairs
                    // need no union.
                    // Only the residues j mod 8 whose minimum passes the filter in
                    // some lane of the warp are scanned (warp-uniform branches, so the
                    // column indices stay compile-time constants).
                    uint64_t mask = 0;
                    {
                        unsigned rm = 0;
                        if (need) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) rm |= (unsigned)(-nv[i] >= thr) << i;
                        }
                        const unsigned um = __reduce_or_sync(0xffffffffu, rm);
                        const int col_lim = a.upper ? (i_row - (ct * TN + half * 128)) : -1;  // cols <= this: j <= i
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            if (!((um >> i) & 1u)) continue;
#pragma unroll
                            for (int u = 0; u < GW / 8; ++u) {
                                const int j = i + 8 * u;
                                const float w1 = fmaf(2.f, __uint_as_float(g[j]), -mc.beta[cb + j]);
                                bool c = need && (BF16 ? (fmaf(rho_p, mc.rho[cb + j], w1) >= alpha) : (w1 >= alpha));
                                if (PASS == TC_UNION) c = c && colroot[cb + j] != rootp;
                                mask |= (uint64_t)(c && (cb + j) > col_lim) << j;
                            }
                        }
                    }
                    uint64_t nbm = mask;  // confirmed neighbours among the mask
                    if (BF16) {
                        nbm = 0;
                        for (uint64_t mm = mask; mm; mm &= mm - 1) {
                            const int j = __ffsll((long long)mm) - 1;
                            const int q = mc.idx[cb + j];
                            // recompute 2G - |v_q|^2 for column j from the accumulator copy in g
                            float gj = 0.f;
#pragma unroll
                            for (int k = 0; k < GW; ++k)
                                if (k == j) gj = __uint_as_float(g[k]);
                            const float wj = fmaf(2.f, gj, -mc.beta[cb + j]);
                            const int res = decide_candidate<BF16>(wj, alpha, rho_p, mc.rho[cb + j], a.v16, K, p, q, a.T);
                            band_cnt += res >> 1;
                            if (!(res & 1)) continue;
                            nbm |= 1ull << j;
                            if (PASS == TC_BORDER) break;  // ascending columns: the first is the smallest
                        }
                    }
                    if (PASS == TC_COUNT) cnt += __popcll(nbm);
                    if (PASS == TC_BORDER && nbm) bmin = min(bmin, mc.idx[cb + __ffsll((long long)nbm) - 1]);
                    if (PASS == TC_UNION) {
                        // Skip a neighbour whose set p is known to be in: colroot[j]
                        // holds a member of column j's set (its parent, or the root
                        // of a later union), rootp a member of p's.  Equal members
                        // mean one set, so only pairs from different-looking sets
                        // reach the atomics.  After a union both endpoints point
                        // straight at the returned root (a valid ancestor; never
                        // written on the root itself, whose link another thread may
                        // have set), so later tiles find the forest flat and a
                        // converged cluster costs one shared-memory compare per pair.
                        for (uint64_t mm = nbm; mm; mm &= mm - 1) {
                            const int j = cb + __ffsll((long long)mm) - 1;
                            if (colroot[j] == rootp) continue;
                            const int q = mc.idx[j];
                            const int r = unite_root(a.parent, p, q, a.status);
                            if (r >= 0) {
                                if (q != r) db::st_relaxed(a.parent + q, r);
                                if (p != r && r != rootp) db::st_relaxed(a.parent + p, r);
                            }
                            rootp = r;
                            colroot[j] = r;
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&S.t_empty[b]);
                    mbar_arrive(&S.m_empty[m]);
                }
            }
            if (row_ok) {
                if ((PASS == TC_COUNT || PASS == TC_VERIFY) && cnt) atomicAdd(a.count + p, cnt);
                if (PASS == TC_BORDER && bmin != INT_MAX) atomicMin(a.border + p, bmin);
            }
            if (!ok) break;
        }
        if (band_cnt) atomicAdd(a.ctr + 6, band_cnt);
        if (bad_cnt) atomicAdd(a.ctr + 7, bad_cnt);
        if (maxerr) atomicMax(a.ctr + 8, (unsigned long long)maxerr);
    }

#ifdef DB_TC_WAIT_STATS
    // slots 9..13 (count), 20..24 (merge), 25..29 (border): producer, MMA issuer
    // on B tiles, MMA issuer on accumulators, one epilogue warp, issuer total
    {
        unsigned long long *ws = a.ctr + (PASS == TC_COUNT ? 9 : (PASS == TC_UNION ? 20 : 25));
        if (PASS != TC_VERIFY && threadIdx.x == 0) atomicAdd(ws, (unsigned long long)w_prod);
        if (PASS != TC_VERIFY && threadIdx.x == 32) {
            atomicAdd(ws + 1, (unsigned long long)w_mma_b);
            atomicAdd(ws + 2, (unsigned long long)w_mma_t);
            atomicAdd(ws + 4, (unsigned long long)(clock64() - t_start));
        }
        if (PASS != TC_VERIFY && threadIdx.x == 64) atomicAdd(ws + 3, (unsigned long long)w_epi);
    }
#endif
    // ---------------- teardown ----------------
    tc_fence_before();
    __syncthreads();
    if (S.abort_flag) {
        if (threadIdx.x == 0) atomicOr(a.status, DB_EBIT_TIMEOUT);
        // The producer has waited (bounded) for the last copy into each buffer
        // and the MMA issuer for a final commit that follows all its MMAs, so
        // nothing of this CTA is in flight.  Only if one of those waits gave up
        // does thread 0 also spin 20 ms before the tensor memory is freed.
        if (threadIdx.x == 0 && S.drain_failed) {
            const uint64_t t0 = globaltimer();
            while (globaltimer() - t0 < 20000000ull) {
            }
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 512);
}


// ---------------- preparation kernels ----------------

// Grid check and centred integer rows: v16[i][k] = u - 512 (pads 0), |v|^2,
// and the largest |v|^2 into *bmax (which starts at 0).  A warp per row (lane
// k reads coordinate k, then k + 32), so the input rows are read coalesced.
__global__ void tc_prep_kernel(const float *__restrict__ x, int n, int d, int K, int16_t *__restrict__ v16,
                               int *__restrict__ nrm, unsigned *status, int *bmax) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    int wmax = 0;
    bool ok = true;
    for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < n; i += nwarps) {
        int s = 0;
        for (int k = lane; k < K; k += 32) {
            int v = 0;
            if (k < d) {
                int u;
                ok &= db::on_grid(x[(size_t)i * d + k], u);
                v = u - 512;
            }
            v16[(size_t)i * K + k] = (int16_t)v;
            s += v * v;
        }
        s = __reduce_add_sync(0xffffffffu, s);
        if (lane == 0) nrm[i] = s;
        wmax = max(wmax, s);
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(status, DB_EBIT_NOT_QUANTISED);
    if (lane == 0 && wmax > 0) atomicMax(bmax, wmax);
}

// Blocks of 256 threads for tc_prep_kernel: a warp per row, at most 16 blocks per SM.
int tc_prep_blocks(int n) { return (int)std::min<int64_t>(((int64_t)n + 7) / 8, 152 * 16); }

__device__ __forceinline__ uint16_t fp16_bits(int v) {
    __half h = __int2half_rn(v);
    return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ uint16_t bf16_bits_rn(int v) {
    __nv_bfloat16 h = __float2bfloat16_rn((float)v);
    return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ int bf16_value(uint16_t bits) {
    return (int)__uint_as_float((uint32_t)bits << 16);  // an integer for every |v| <= 512
}

// Operand modes of tc_pack_kernel: plain v (or the BF16 terms), and the two
// sides of the folded FP16 count, which append one 16-column chunk to v.
enum { PACK_PLAIN = 0, PACK_FOLD_ROWS = 1, PACK_FOLD_COLS = 2 };

// The folded chunk.  Row side: 1, 2^11, 2^15 (then zeros).  Column side: the
// digits of h_q = ceil(|v_q|^2 / 2) = q0 + 2^11 q1 + 2^22 q2 (q0, q1 < 2^11),
// negated, as -q0, -q1, -2^7 q2 (then zeros); a padding column takes
// h = 2^24.  Every entry is an integer FP16 holds exactly, and the chunk's
// products sum to -h_q, so the MMA accumulates G - h_q.
__device__ __forceinline__ int fold_entry(int mode, int kk, bool valid, int nrm_q) {
    if (mode == PACK_FOLD_ROWS) return kk == 0 ? 1 : (kk == 1 ? 2048 : (kk == 2 ? 32768 : 0));
    const int h = valid ? (nrm_q + 1) >> 1 : (1 << 24);
    return kk == 0 ? -(h & 2047) : (kk == 1 ? -((h >> 11) & 2047) : (kk == 2 ? -((h >> 22) << 7) : 0));
}

// Packs list entries (list == nullptr: identity; an entry of -1 is padding)
// into the tiled operand layout and writes their metadata; padding rows and
// rows past the list length up to the padded length become zero rows with
// index -1 and beta = 1e30 (never neighbours).
__global__ void tc_pack_kernel(const int *__restrict__ list, const int *__restrict__ len_ptr, int n_pad, int K,
                               int bf16, int mode, const int16_t *__restrict__ v16, const int *__restrict__ nrm,
                               uint16_t *__restrict__ op, MetaBlock *__restrict__ meta) {
    const int len = *len_ptr;
    // stored columns: v (FP16), [hi | lo] (BF16) or [v | folded chunk] (FP16 count)
    const int KS = bf16 ? 2 * K : (mode != PACK_PLAIN ? K + 16 : K);
    const int KG = KS / 8, KH = K / 8;
    const float rho_c = sqrtf((float)bf16_band(K)) * (1.f + 1.f / 1024.f);
    const int64_t total = (int64_t)n_pad * KG;  // one thread per (row, 8-element group)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / KG), kg = (int)(e - (int64_t)i * KG);
        const int tile = i / TM, r = i - tile * TM;
        const int rg = r >> 3, ri = r & 7;
        uint16_t h[8];
        const int p = i < len ? (list ? list[i] : i) : -1;
        const bool valid = p >= 0;
        const bool lo = kg >= KH;  // BF16: the remainder columns; folded modes: the extra chunk
        const int k0 = (lo ? kg - KH : kg) * 8;
        if (lo && mode != PACK_PLAIN) {
            const int nq = valid ? nrm[p] : 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) h[k] = fp16_bits(fold_entry(mode, k0 + k, valid, nq));
        } else
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (!valid) {
                h[k] = 0;
                continue;
            }
            const int v = v16[(size_t)p * K + k0 + k];
            if (!bf16) {
                h[k] = fp16_bits(v);
            } else {
                const uint16_t hi = bf16_bits_rn(v);
                h[k] = lo ? bf16_bits_rn(v - bf16_value(hi)) : hi;  // v - hi is -1, 0 or 1: exact
            }
        }
        const size_t off = (size_t)tile * TM * KS + ((size_t)(rg * KG + kg) * 64) + ri * 8;
        uint4 pk;
        pk.x = h[0] | ((uint32_t)h[1] << 16);
        pk.y = h[2] | ((uint32_t)h[3] << 16);
        pk.z = h[4] | ((uint32_t)h[5] << 16);
        pk.w = h[6] | ((uint32_t)h[7] << 16);
        *reinterpret_cast<uint4 *>(op + off) = pk;
        if (kg == 0) {
            MetaBlock &m = meta[tile];
            if (valid) {
                m.beta[r] = (float)nrm[p];
                m.rho[r] = bf16 ? rho_c : 0.f;
                m.idx[r] = p;
            } else {
                m.beta[r] = 1e30f;
                m.rho[r] = 0.f;
                m.idx[r] = -1;
            }
            m.beta_f[r] = valid ? (bf16 ? (float)nrm[p] - rho_c * rho_c : (float)nrm[p]) : 1e30f;
        }
    }
}

// Core and non-core lists in increasing index order (from an exclusive scan of
// the core flags): lists[0..ncore) = cores, noncore list separately.
__global__ void tc_split_kernel(int n, const uint8_t *__restrict__ core, const int *__restrict__ scan,
                                int *__restrict__ core_list, int *__restrict__ non_list, int *__restrict__ lens) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = scan[i];
        if (core[i]) core_list[c] = i;
        else non_list[i - c] = i;
        if (i == n - 1) {
            lens[0] = c + core[i];
            lens[1] = n - lens[0];
        }
    }
}

// lens[2] = n (the all-points list), lens[3] = 0 (the running max of |v|^2).
__global__ void tc_init_lens_kernel(int *lens, int n) {
    lens[2] = n;
    lens[3] = 0;
}

// Column list of the FP16 count: the points of even |v|^2 in index order, then,
// from the next 256-row tile on, those of odd |v|^2; the gap holds -1.  flags
// is the parity of each |v|^2 and scan its exclusive scan.  lens[4] = even
// points, lens[5] = the list's length.
__global__ void tc_parity_list_kernel(int n, const int *__restrict__ flags, const int *__restrict__ scan,
                                      int *__restrict__ list, int *__restrict__ lens) {
    const int n_odd = scan[n - 1] + flags[n - 1];
    const int nE = n - n_odd, nEp = (nE + TN - 1) / TN * TN;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = g; i < n; i += gridDim.x * blockDim.x) list[flags[i] ? nEp + scan[i] : i - scan[i]] = i;
    if (g < nEp - nE) list[nE + g] = -1;
    if (g == 0) {
        lens[4] = nE;
        lens[5] = nEp + n_odd;
    }
}

__global__ void tc_parity_flags_kernel(int n, const int *__restrict__ nrm, int *__restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flags[i] = nrm[i] & 1;
}

__global__ void core_flags_kernel(int n, const uint8_t *__restrict__ core, int *__restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flags[i] = core[i];
}

template <int PASS, bool BF16>
size_t tc_smem_bytes() {
    return sizeof(typename TcSmem<PASS, BF16>::type) + 1024;
}

template <int PASS, bool BF16>
cudaError_t launch_pass_t(const TcArgs &a, int sms, cudaStream_t st) {
    // the shared-memory attribute, set once per device (plans may live on
    // several devices of one process; setting it twice is harmless)
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!(attr_set.load(std::memory_order_relaxed) & bit) || !bit) {
        cudaError_t e = cudaFuncSetAttribute(tc_pass_kernel<PASS, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tc_smem_bytes<PASS, BF16>());
        if (e) return e;
        attr_set.fetch_or(bit, std::memory_order_relaxed);
    }
    tc_pass_kernel<PASS, BF16><<<sms, tc_threads<PASS, BF16>(), tc_smem_bytes<PASS, BF16>(), st>>>(a);
    return cudaGetLastError();
}

template <int PASS>
cudaError_t launch_pass(const TcArgs &a, int sms, cudaStream_t st) {
    return a.bf16 ? launch_pass_t<PASS, true>(a, sms, st) : launch_pass_t<PASS, false>(a, sms, st);
}

}  // namespace

// Host launcher of the whole tensor-core all-pairs pipeline.
cudaError_t launch_allpairs_tc(const DbWork &w, const float *x, int64_t n64, int32_t d, int64_t Tc, int32_t min_pts,
                               bool bf16, bool stall, cudaStream_t st) {
    const int n = (int)n64;
    const int K = ((d + 15) / 16) * 16;
    const int n_pad = ((n + TN - 1) / TN) * TN;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = (n + 255) / 256;
    int *lens = w.tc_lens;  // [0] cores, [1] non-cores, [2] all, [3] max |v|^2, [4] even, [5] count columns
    tc_init_lens_kernel<<<1, 1, 0, st>>>(lens, n);
    tc_prep_kernel<<<tc_prep_blocks(n), 256, 0, st>>>(x, n, d, K, w.v16, w.inorm, w.status, lens + 3);
    w.marks->kernel("tc_prep", st);
    const int pack_blocks = (int)std::min<int64_t>(((int64_t)n_pad * (K / 8) + 255) / 256, 152 * 32);
    cudaError_t e;
    if (!bf16) {
        // FP16 count operands: rows [v | 1, 2^11, 2^15], columns [v | -digits of
        // ceil(|v|^2 / 2)] with the even-norm points first (see fold_entry)
        tc_parity_flags_kernel<<<std::min(nb, 152 * 16), 256, 0, st>>>(n, w.inorm, w.list_b);
        if ((e = launch_exclusive_scan(w.list_b, w.scan, n, w.scan_part, w.scan_part_cap, st, w.marks))) return e;
        tc_parity_list_kernel<<<std::min(nb, 152 * 16), 256, 0, st>>>(n, w.list_b, w.scan, w.list_a, lens);
        tc_pack_kernel<<<pack_blocks, 256, 0, st>>>(nullptr, lens + 2, n_pad, K, 0, PACK_FOLD_ROWS, w.v16, w.inorm,
                                                    w.opAll, reinterpret_cast<MetaBlock *>(w.metaAll));
        tc_pack_kernel<<<pack_blocks, 256, 0, st>>>(w.list_a, lens + 5, n_pad + TN, K, 0, PACK_FOLD_COLS, w.v16,
                                                    w.inorm, w.opCore, reinterpret_cast<MetaBlock *>(w.metaCore));
    } else {
        tc_pack_kernel<<<pack_blocks, 256, 0, st>>>(nullptr, lens + 2, n_pad, K, 1, PACK_PLAIN, w.v16, w.inorm,
                                                    w.opAll, reinterpret_cast<MetaBlock *>(w.metaAll));
    }
    w.marks->kernel("tc_pack_all", st);
    if ((e = cudaMemsetAsync(w.count, 0, sizeof(int) * (size_t)n, st))) return e;

    TcArgs a{};
    a.K = K;
    a.ks = bf16 ? 2 * K : K;
    a.T = (int)Tc;
    a.bf16 = bf16 ? 1 : 0;
    a.v16 = w.v16;
    a.count = w.count;
    a.parent = w.parent;
    a.border = w.border;
    a.status = w.status;
    a.ctr = w.ctr;
    a.col_chunk = DB_TC_COUNT_CHUNK;
    a.wait_ns = 2000000000ull;  // about two seconds per barrier wait
    // pass 1: all x all -> neighbour counts (the stall hook: a 50 ms budget the
    // waits exhaust, since no MMA completes)
    a.stall = stall ? 1 : 0;
    if (stall) a.wait_ns = 50000000ull;
    a.opR = a.opC = w.opAll;
    a.metaR = a.metaC = reinterpret_cast<const MetaBlock *>(w.metaAll);
    a.nR_ptr = a.nC_ptr = lens + 2;
    if (!bf16) {
        a.ks = K + 16;
        a.opC = w.opCore;
        a.metaC = reinterpret_cast<const MetaBlock *>(w.metaCore);
        a.nC_ptr = lens + 5;
        a.nE_ptr = lens + 4;
        a.bmax_ptr = lens + 3;
    }
    a.pass = TC_COUNT;
    a.upper = 0;
    if ((e = launch_pass<TC_COUNT>(a, sms, st))) return e;
    a.col_chunk = 32;
    w.marks->kernel("tc_count", st);
    a.ks = bf16 ? 2 * K : K;
    a.stall = 0;
    a.wait_ns = 2000000000ull;
    // core flags, parent, border init (shared with the SIMT path)
    launch_core_init(w, n, min_pts, st);
    // core / non-core lists
    core_flags_kernel<<<std::min(nb, 152 * 16), 256, 0, st>>>(n, w.core, w.list_b);
    w.marks->kernel("tc_core_flags", st);
    {
        cudaError_t e2 = launch_exclusive_scan(w.list_b, w.scan, n, w.scan_part, w.scan_part_cap, st, w.marks);
        if (e2) return e2;
    }
    tc_split_kernel<<<std::min(nb, 152 * 16), 256, 0, st>>>(n, w.core, w.scan, w.list_a, w.list_b, lens);
    w.marks->kernel("tc_split", st);
    tc_pack_kernel<<<pack_blocks, 256, 0, st>>>(w.list_a, lens + 0, n_pad, K, bf16, PACK_PLAIN, w.v16, w.inorm,
                                                w.opCore, reinterpret_cast<MetaBlock *>(w.metaCore));
    w.marks->kernel("tc_pack_core", st);
    tc_pack_kernel<<<pack_blocks, 256, 0, st>>>(w.list_b, lens + 1, n_pad, K, bf16, PACK_PLAIN, w.v16, w.inorm,
                                                w.opNon, reinterpret_cast<MetaBlock *>(w.metaNon));
    w.marks->kernel("tc_pack_noncore", st);
    // pass 2: core x core (i < j) -> union
    a.opR = a.opC = w.opCore;
    a.metaR = a.metaC = reinterpret_cast<const MetaBlock *>(w.metaCore);
    a.nR_ptr = a.nC_ptr = lens + 0;
    a.pass = TC_UNION;
    a.upper = 1;
    if ((e = launch_pass<TC_UNION>(a, sms, st))) return e;
    w.marks->kernel("tc_union", st);
    // pass 3: non-core x core -> smallest core neighbour
    a.opR = w.opNon;
    a.metaR = reinterpret_cast<const MetaBlock *>(w.metaNon);
    a.nR_ptr = lens + 1;
    a.opC = w.opCore;
    a.metaC = reinterpret_cast<const MetaBlock *>(w.metaCore);
    a.nC_ptr = lens + 0;
    a.pass = TC_BORDER;
    a.upper = 0;
    if ((e = launch_pass<TC_BORDER>(a, sms, st))) return e;
    w.marks->kernel("tc_border", st);
    return cudaGetLastError();
}

// Diagnostic: the count pass with every pair also decided exactly; records in
// ctr[6] the band pairs, ctr[7] the pairs outside the band whose fast decision
// disagrees with the exact one (must be 0), ctr[8] the largest |2G - exact|.
cudaError_t launch_tc_verify(const DbWork &w, const float *x, int64_t n64, int32_t d, int64_t Tc, bool bf16,
                             cudaStream_t st) {
    const int n = (int)n64;
    const int K = ((d + 15) / 16) * 16;
    const int n_pad = ((n + TN - 1) / TN) * TN;
    cudaError_t e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int *lens = w.tc_lens;
    tc_init_lens_kernel<<<1, 1, 0, st>>>(lens, n);
    tc_prep_kernel<<<tc_prep_blocks(n), 256, 0, st>>>(x, n, d, K, w.v16, w.inorm, w.status, lens + 3);
    const int pack_blocks = (int)std::min<int64_t>(((int64_t)n_pad * (K / 8) + 255) / 256, 152 * 32);
    tc_pack_kernel<<<pack_blocks, 256, 0, st>>>(nullptr, lens + 2, n_pad, K, bf16, PACK_PLAIN, w.v16, w.inorm,
                                                w.opAll, reinterpret_cast<MetaBlock *>(w.metaAll));
    if ((e = cudaMemsetAsync(w.count, 0, sizeof(int) * (size_t)n, st))) return e;
    TcArgs a{};
    a.K = K;
    a.ks = bf16 ? 2 * K : K;
    a.T = (int)Tc;
    a.bf16 = bf16 ? 1 : 0;
    a.v16 = w.v16;
    a.count = w.count;
    a.status = w.status;
    a.ctr = w.ctr;
    a.col_chunk = 32;
    a.wait_ns = 2000000000ull;
    a.opR = a.opC = w.opAll;
    a.metaR = a.metaC = reinterpret_cast<const MetaBlock *>(w.metaAll);
    a.nR_ptr = a.nC_ptr = lens + 2;
    a.pass = TC_VERIFY;
    return launch_pass<TC_VERIFY>(a, sms, st);
}
