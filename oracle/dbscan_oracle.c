/*
 * Exact brute-force DBSCAN — the correctness oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which
 * only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load.  It shares no code, header, table or helper with the CUDA library, and
 * the CUDA library never calls it.
 *
 * What it computes (Wang et al., "Design and optimization of DBSCAN Algorithm
 * based on CUDA", Section II; the serial three-step outline at the end of
 * Section II; the eps^2 comparison of Section IV-A and the "<= eps^2" test of
 * Section IV-B):
 *
 *   1. Coordinates are multiples of 2^-10 in [0, 1).  u = 1024 x is an integer
 *      in 0..1023; anything else is rejected (status 2).
 *   2. T = floor(eps * eps * 2^20) in double.  eps is a float, so its square is
 *      exact in double (24 + 24 <= 53 bits) and so is the scaling by 2^20.
 *   3. D(p,q) = sum_k (u_pk - u_qk)^2, an exact integer.  q is an
 *      eps-neighbour of p iff D(p,q) <= T, i.e. the real squared distance
 *      D * 2^-20 <= eps^2 (Section II, definition 1; Section IV-B's "<=").
 *   4. count[p] = #{q : D(p,q) <= T}, p itself included.  p is a core point
 *      iff count[p] >= min_pts (Section II, definition 2: "at least MinPts").
 *   5. Core points that are eps-neighbours are directly reachable from each
 *      other; a cluster's core points are the connected components of that
 *      graph (Section II, definition 3 and the cluster definition).  The
 *      cluster id is the smallest core index in the component.
 *   6. A non-core point with at least one core neighbour is a border point.
 *      It may be reachable from several clusters; it is given the cluster of
 *      its smallest-index core neighbour (a fixed reading: the paper leaves the
 *      choice open).
 *   7. Every other point is noise, label -1.
 *   8. Label mode 1 renumbers the cluster ids to 0..k-1 in increasing order of
 *      their smallest core index.
 *
 * Parallelism: rows of the count (4), edge discovery (5) and border (6) loops
 * are spread over OpenMP threads; each row's result is the plain definition.
 * The unions of step 5 are applied sequentially, in row order.
 *
 * Planted mistakes (``mutation`` bits) exist only so that the tests can show
 * that the pins catch them; production callers pass 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_QUANTISED 2
#define OR_ERR_OOM 3

#define MUT_STRICT_LESS 1   /* use D < T instead of D <= T */
#define MUT_NO_SELF 2       /* leave p out of its own count */
#define MUT_BORDER_MAX 4    /* give a border point its largest-index core neighbour */
#define MUT_NO_UNION 8      /* never merge: every core point is its own cluster */

int oracle_max_dim(void) { return 2048; } /* D fits in int32 up to here */

int oracle_quantise(const float *x, int64_t n, int32_t d, int32_t *u) {
    if (n < 0 || d < 1 || d > 2048 || (n > 0 && (!x || !u))) return OR_ERR_ARG;
    for (int64_t i = 0; i < n * (int64_t)d; ++i) {
        float v = x[i];
        if (!(v >= 0.0f && v < 1.0f)) return OR_ERR_NOT_QUANTISED; /* also NaN */
        double s = (double)v * 1024.0;
        double f = floor(s);
        if (f != s) return OR_ERR_NOT_QUANTISED;
        u[i] = (int32_t)f;
    }
    return OR_OK;
}

int64_t oracle_threshold(float eps) {
    double e = (double)eps;
    return (int64_t)floor(e * e * 1048576.0);
}

static int32_t sqdist(const int32_t *a, const int32_t *b, int32_t d) {
    int32_t s = 0;
    for (int32_t k = 0; k < d; ++k) {
        int32_t t = a[k] - b[k];
        s += t * t;
    }
    return s;
}

static int is_nbr(int32_t D, int64_t T, int mutation) {
    if (mutation & MUT_STRICT_LESS) return (int64_t)D < T;
    return (int64_t)D <= T;
}

/* Step 4: neighbour counts of rows [row0, row1) against all n points. */
int oracle_counts(const int32_t *u, int64_t n, int32_t d, int64_t T, int64_t row0, int64_t row1,
                  int32_t *counts, int32_t nthreads, int32_t mutation) {
    if (row0 < 0 || row1 > n || row0 > row1) return OR_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = row0; p < row1; ++p) {
        int32_t c = 0;
        for (int64_t q = 0; q < n; ++q) {
            if (q == p && (mutation & MUT_NO_SELF)) continue;
            c += is_nbr(sqdist(u + p * d, u + q * d, d), T, mutation);
        }
        counts[p - row0] = c;
    }
    return OR_OK;
}

static int32_t uf_find(int32_t *parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]]; /* path halving */
        x = parent[x];
    }
    return x;
}

/* Link the larger root under the smaller, so every root is its set's minimum. */
static void uf_union(int32_t *parent, int32_t a, int32_t b) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) parent[b] = a;
    else parent[a] = b;
}

int oracle_dbscan(const float *x, int64_t n, int32_t d, float eps, int32_t min_pts, int32_t label_mode,
                  int32_t *labels, int32_t *counts_out, uint8_t *core_out, int32_t nthreads,
                  int32_t mutation) {
    if (n < 0 || d < 1 || d > 2048 || min_pts < 1 || !(eps > 0.0f) || isinf(eps) || !labels)
        return OR_ERR_ARG;
    if (n == 0) return OR_OK;
    if (n > INT32_MAX) return OR_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int st = OR_OK;
    int32_t *u = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)d);
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *core = (uint8_t *)malloc((size_t)n);
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *border = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!u || !cnt || !core || !parent || !border) { st = OR_ERR_OOM; goto done; }

    /* Steps 1-2. */
    st = oracle_quantise(x, n, d, u);
    if (st != OR_OK) goto done;
    const int64_t T = oracle_threshold(eps);

    /* Step 4: counts and core flags. */
    oracle_counts(u, n, d, T, 0, n, cnt, nthreads, mutation);
    for (int64_t p = 0; p < n; ++p) core[p] = cnt[p] >= min_pts;

    /* Step 5: union every core-core eps-edge (q < p), rows discovered in
     * parallel in blocks, unions applied in row order. */
    for (int64_t p = 0; p < n; ++p) parent[p] = (int32_t)p;
    if (!(mutation & MUT_NO_UNION)) {
        const int64_t B = 1024;
        int32_t **lists = (int32_t **)calloc((size_t)B, sizeof(int32_t *));
        int64_t *lens = (int64_t *)calloc((size_t)B, sizeof(int64_t));
        if (!lists || !lens) { free(lists); free(lens); st = OR_ERR_OOM; goto done; }
        int oom = 0;
        for (int64_t p0 = 0; p0 < n && !oom; p0 += B) {
            int64_t p1 = p0 + B < n ? p0 + B : n;
#pragma omp parallel for schedule(dynamic, 4)
            for (int64_t p = p0; p < p1; ++p) {
                int64_t cap = 0, len = 0;
                int32_t *l = NULL;
                if (core[p]) {
                    for (int64_t q = 0; q < p; ++q) {
                        if (!core[q] || !is_nbr(sqdist(u + p * d, u + q * d, d), T, mutation)) continue;
                        if (len == cap) {
                            cap = cap ? 2 * cap : 64;
                            int32_t *nl = (int32_t *)realloc(l, sizeof(int32_t) * (size_t)cap);
                            if (!nl) { oom = 1; break; }
                            l = nl;
                        }
                        l[len++] = (int32_t)q;
                    }
                }
                lists[p - p0] = l;
                lens[p - p0] = len;
            }
            for (int64_t p = p0; p < p1; ++p) {
                for (int64_t j = 0; j < lens[p - p0]; ++j) uf_union(parent, (int32_t)p, lists[p - p0][j]);
                free(lists[p - p0]);
                lists[p - p0] = NULL;
            }
        }
        free(lists);
        free(lens);
        if (oom) { st = OR_ERR_OOM; goto done; }
    }

    /* Step 6: border points take their smallest-index core neighbour. */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        int32_t b = -1;
        if (!core[p]) {
            for (int64_t q = 0; q < n; ++q) {
                if (!core[q] || !is_nbr(sqdist(u + p * d, u + q * d, d), T, mutation)) continue;
                b = (int32_t)q;
                if (!(mutation & MUT_BORDER_MAX)) break;
            }
        }
        border[p] = b;
    }

    /* Steps 5-7: labels. */
    for (int64_t p = 0; p < n; ++p) {
        if (core[p]) labels[p] = uf_find(parent, (int32_t)p);
        else if (border[p] >= 0) labels[p] = uf_find(parent, border[p]);
        else labels[p] = -1;
    }

    /* Step 8: compact ids 0..k-1 in increasing order of the root index. */
    if (label_mode == 1) {
        int32_t *rank = parent; /* roots are fixed now; reuse as rank table */
        int32_t k = 0;
        for (int64_t p = 0; p < n; ++p) {
            /* p is a root iff it is core and its label is itself */
            rank[p] = (core[p] && labels[p] == p) ? k++ : -1;
        }
        for (int64_t p = 0; p < n; ++p)
            if (labels[p] >= 0) labels[p] = rank[labels[p]];
    }

    if (counts_out) memcpy(counts_out, cnt, sizeof(int32_t) * (size_t)n);
    if (core_out) memcpy(core_out, core, (size_t)n);
done:
    free(u);
    free(cnt);
    free(core);
    free(parent);
    free(border);
    return st;
}
