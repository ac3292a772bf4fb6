/*
 * domagg_oracle.c -- CPU oracle for aggregation over dominated points.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, the smoke check of __graft_entry__ and the
 * CPU-baseline leg of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library; it is plain, slow and meant to be read
 * against the paper.
 *
 * What is computed (Sroka & Tyszkiewicz, "Aggregating over Dominated Points
 * by Sorting, Scanning, Zip and Flat Maps", Sec. 1.2): for every query q,
 *     out(q) = F over { w(d) : d in D, d < q },
 * where d < q means d_i < q_i in EVERY coordinate (strict), and F is an
 * associative, commutative operation with unit e (Sec. 1, Sec. 1.2).
 *
 * Three independent routes are provided:
 *   oracle_brute       -- the definition written out: O(|D||Q|m) loops
 *                         (oracle_brute_ns: the same with chosen coordinates
 *                         compared non-strictly, d_i <= q_i).
 *   oracle_sortscan    -- the paper's algorithm in list form, Sec. 4 with the
 *                         one-logarithm improvement of Sec. 5: dense ranks,
 *                         P0/P1 flat map, lexicographic sort, segmented scan,
 *                         then the ID sort + ID-segmented scan of Sec. 4
 *                         (instructions 6m+4, 6m+5) to collect each query.
 *   oracle_brute_transpose -- the adjoint with respect to the weights:
 *                         grad(d) = sum over { g(q) : q in Q, d < q }.
 *   oracle_sweep2      -- m = 2 only: a sweep over the last coordinate with
 *                         a Fenwick tree over the first coordinate's ranks,
 *                         O(n log n), so full-size inputs can be checked on
 *                         every query (oracle_sweep2_transpose: its adjoint).
 *                         It is not the paper's algorithm; it is pinned to
 *                         the brute force above by the tests.
 * plus the small primitives the tests pin against the paper's worked
 * examples: the segmented scan (Definition "Segmented scan", Sec. 2.2) and
 * the prefix sets P0/P1 (Sec. 3).
 *
 * Conventions (the oracle's own; the Python test wrapper maps them):
 *   coordinate dtype: 0 = int32, 2 = float32; row-major [n][m].
 *   weight dtype    : 0 = int32, 1 = int64, 2 = float32.
 *   op              : 0 = sum, 1 = max, 2 = count, 3 = min.
 *   out             : int64[nQ] for integer results (sum of int32/int64,
 *                     max / min of int32, count) and double[nQ] for float
 *                     results (sum / max / min of float32).  Empty set -> e:
 *                     0 for sums and counts, INT32_MIN / -inf for max,
 *                     INT32_MAX / +inf for min.
 *   Sums of integers wrap modulo 2^64 (associative and commutative, so the
 *   result does not depend on order).  Sums of float32 are accumulated in
 *   double.  S (optional, double[nQ]) receives sum |w(d)| over the dominated
 *   set, the scale of the float32 tolerance.
 *   Return value: 0 = ok, 1 = bad argument, 6 = NaN coordinate.
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   - ranks are 0-based dense ranks r in [0, U); each is written with
 *     b = ceil(log2 U) binary digits (b = 0 when U = 1);
 *   - D and Q are concatenated instead of zipped, so |D| != |Q| is allowed;
 *   - in the Sec. 5 variant queries precede data points when all
 *     coordinates tie, and the segments are the m-1 bitstring coordinates;
 *   - -0.0 and +0.0 are the same coordinate; a NaN coordinate is an error.
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
#define OR_ERR_NAN 6

#define CT_I32 0
#define CT_F32 2
#define WT_I32 0
#define WT_I64 1
#define WT_F32 2
#define OP_SUM 0
#define OP_MAX 1
#define OP_COUNT 2
#define OP_MIN 3

/* ORACLE_PLANT selects a deliberately wrong variant, built only by the tests
 * that check that the pins catch such mistakes.  0 = the real oracle. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

/* ------------------------------------------------------------------ */
/* coordinates                                                        */
/* ------------------------------------------------------------------ */

static double coord_at(const void* base, int ct, int64_t row, int m, int i) {
    if (ct == CT_I32) return (double)((const int32_t*)base)[row * m + i];
    float f = ((const float*)base)[row * m + i];
    if (f == 0.0f) f = 0.0f; /* -0.0 and +0.0 are one coordinate */
    return (double)f;
}

/* Both int32 and float32 values are represented exactly in double, so the
 * comparisons below are the comparisons of the original values. */
static int any_nan(const void* base, int ct, int64_t n, int m) {
    if (ct != CT_F32) return 0;
    const float* f = (const float*)base;
    for (int64_t k = 0; k < n * (int64_t)m; ++k)
        if (f[k] != f[k]) return 1;
    return 0;
}

/* d < q coordinate-wise, strict in every coordinate (Sec. 1.2); with bit i
 * of `nonstrict` set, coordinate i is compared as d_i <= q_i instead (an
 * extension: the paper defines the strict order only). */
static int dominated_ns(const void* D, int64_t d, const void* Q, int64_t q, int ct, int m, unsigned nonstrict) {
    for (int i = 0; i < m; ++i) {
        double x = coord_at(D, ct, d, m, i), y = coord_at(Q, ct, q, m, i);
        if ((nonstrict >> i) & 1u) {
            if (!(x <= y)) return 0;
            continue;
        }
#if ORACLE_PLANT == 1
        if (!(x <= y)) return 0; /* planted: non-strict dominance */
#else
        if (!(x < y)) return 0;
#endif
    }
    return 1;
}
static int dominated(const void* D, int64_t d, const void* Q, int64_t q, int ct, int m) {
    return dominated_ns(D, d, Q, q, ct, m, 0u);
}

/* ------------------------------------------------------------------ */
/* the aggregation F with its unit e (Sec. 1)                         */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t i; /* integer results: sums wrap modulo 2^64 */
    double f;  /* float results */
} agg_t;

static int result_is_float(int wt, int op) { return op != OP_COUNT && wt == WT_F32; }

static agg_t agg_unit(int wt, int op) {
    agg_t a;
    a.i = 0;
    a.f = 0.0;
    if (op == OP_MAX) {
        a.i = INT32_MIN;
        a.f = -INFINITY;
    }
    if (op == OP_MIN) {
        a.i = INT32_MAX;
        a.f = INFINITY;
    }
    (void)wt;
    return a;
}

static agg_t weight_of(const void* W, int wt, int op, int64_t d) {
    agg_t a;
    a.i = 0;
    a.f = 0.0;
    if (op == OP_COUNT) {
        a.i = 1;
        return a;
    }
    if (wt == WT_I32) a.i = ((const int32_t*)W)[d];
    else if (wt == WT_I64) a.i = ((const int64_t*)W)[d];
    else a.f = (double)((const float*)W)[d];
    return a;
}

static double abs_weight(const void* W, int wt, int op, int64_t d) {
    if (op == OP_COUNT) return 1.0;
    if (wt == WT_I32) return fabs((double)((const int32_t*)W)[d]);
    if (wt == WT_I64) return fabs((double)((const int64_t*)W)[d]);
    return fabs((double)((const float*)W)[d]);
}

static agg_t agg_F(agg_t a, agg_t b, int op) {
    agg_t r;
    if (op == OP_MAX) {
        r.i = a.i > b.i ? a.i : b.i;
        r.f = a.f > b.f ? a.f : b.f;
        if (a.f != a.f) r.f = b.f; /* NaN weights never win a max */
        if (b.f != b.f) r.f = a.f;
    } else if (op == OP_MIN) {
        r.i = a.i < b.i ? a.i : b.i;
        r.f = a.f < b.f ? a.f : b.f;
        if (a.f != a.f) r.f = b.f; /* NaN weights never win a min */
        if (b.f != b.f) r.f = a.f;
    } else { /* sum and count */
        r.i = (int64_t)((uint64_t)a.i + (uint64_t)b.i);
        r.f = a.f + b.f;
    }
    return r;
}

static void store_out(void* out, int wt, int op, int64_t q, agg_t a) {
    if (result_is_float(wt, op)) ((double*)out)[q] = a.f;
    else ((int64_t*)out)[q] = a.i;
}

static int check_args(int m, int64_t nD, int64_t nQ, int ct, int wt, int op) {
    if (m < 1 || m > 8 || nD < 0 || nQ < 0) return OR_ERR_ARG;
    if (ct != CT_I32 && ct != CT_F32) return OR_ERR_ARG;
    if (op < OP_SUM || op > OP_MIN) return OR_ERR_ARG;
    if (op != OP_COUNT && wt != WT_I32 && wt != WT_I64 && wt != WT_F32) return OR_ERR_ARG;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 1. brute force: the definition (Sec. 1.2)                          */
/* ------------------------------------------------------------------ */

int oracle_brute_ns(int m, const void* D, int64_t nD, const void* Q, int64_t nQ, int ct, const void* W, int wt,
                    int op, unsigned nonstrict, void* out, double* S, int nthreads) {
    int st = check_args(m, nD, nQ, ct, wt, op);
    if (st) return st;
    if (any_nan(D, ct, nD, m) || any_nan(Q, ct, nQ, m)) return OR_ERR_NAN;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t q = 0; q < nQ; ++q) {
        agg_t acc = agg_unit(wt, op);
        double s = 0.0;
        for (int64_t d = 0; d < nD; ++d) {
            if (!dominated_ns(D, d, Q, q, ct, m, nonstrict)) continue;
            acc = agg_F(acc, weight_of(W, wt, op, d), op);
            s += abs_weight(W, wt, op, d);
        }
        store_out(out, wt, op, q, acc);
        if (S) S[q] = s;
    }
    (void)nthreads;
    return OR_OK;
}

int oracle_brute(int m, const void* D, int64_t nD, const void* Q, int64_t nQ, int ct,
                 const void* W, int wt, int op, void* out, double* S, int nthreads) {
    return oracle_brute_ns(m, D, nD, Q, nQ, ct, W, wt, op, 0u, out, S, nthreads);
}

/* Adjoint of the float32 dominance sum with respect to the weights:
 * out(q) = sum_{d<q} w(d) is linear in w, so dL/dw(d) = sum_{q : d<q} g(q)
 * with g = dL/dout.  Accumulated in double; S receives sum |g(q)|. */
int oracle_brute_transpose(int m, const void* D, int64_t nD, const void* Q, int64_t nQ, int ct,
                           const float* G, double* grad, double* S, int nthreads) {
    if (m < 1 || m > 8 || nD < 0 || nQ < 0 || (ct != CT_I32 && ct != CT_F32)) return OR_ERR_ARG;
    if (any_nan(D, ct, nD, m) || any_nan(Q, ct, nQ, m)) return OR_ERR_NAN;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t d = 0; d < nD; ++d) {
        double acc = 0.0, s = 0.0;
        for (int64_t q = 0; q < nQ; ++q) {
            if (!dominated(D, d, Q, q, ct, m)) continue;
            acc += (double)G[q];
            s += fabs((double)G[q]);
        }
        grad[d] = acc;
        if (S) S[d] = s;
    }
    (void)nthreads;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 2. primitives of Sec. 2.2 and Sec. 3                               */
/* ------------------------------------------------------------------ */

/* sscan(a, t, +) of Definition "Segmented scan" (Sec. 2.2): out_k is the sum
 * of a_i over i <= k with t_i = t_k, for a sorted tag list t. */
void oracle_sscan_i64(const int64_t* a, const int64_t* t, int64_t n, int64_t* out) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t s = 0;
        for (int64_t i = 0; i <= k; ++i)
            if (t[i] == t[k]) s += a[i];
        out[k] = s;
    }
}

/* Bit k (0 = most significant) of x written with b binary digits. */
static int bit_msb(uint64_t x, int b, int k) { return (int)((x >> (b - 1 - k)) & 1u); }

/* P0(x) (which = 0) or P1(x) (which = 1) of Sec. 3 for the b-digit binary
 * expansion of x: all bitstrings v such that v0 (resp. v1) is a prefix of x.
 * A prefix is returned as (length, value): the first `length` digits of x
 * read as a number.  Returns the number of prefixes written. */
int oracle_prefix_set(uint64_t x, int b, int which, int* len_out, uint64_t* val_out) {
    int n = 0;
    for (int k = 0; k < b; ++k) {
        if (bit_msb(x, b, k) != which) continue;
        len_out[n] = k;
        val_out[n] = k == 0 ? 0 : (x >> (b - k));
        ++n;
    }
    return n;
}

/* ------------------------------------------------------------------ */
/* 3. the algorithm of Sec. 4 with the improvement of Sec. 5          */
/* ------------------------------------------------------------------ */

#define MAXM 8

typedef struct {
    int len[MAXM - 1];       /* bitstring coordinates: prefix length ... */
    uint64_t val[MAXM - 1];  /* ... and prefix value */
    double last;             /* the m-th coordinate, kept as a number (Sec. 5) */
    int is_query;
    int64_t id;              /* data: index into D; query: nD + index into Q */
} record_t;

static int g_m; /* record comparators need m */

/* Lexicographic order of two bitstrings given as (length, value). */
static int cmp_bits(int la, uint64_t va, int lb, uint64_t vb) {
    int l = la < lb ? la : lb;
    uint64_t pa = l == 0 ? 0 : (va >> (la - l)), pb = l == 0 ? 0 : (vb >> (lb - l));
    if (pa != pb) return pa < pb ? -1 : 1;
    if (la != lb) return la < lb ? -1 : 1;
    return 0;
}

/* The doubly lexicographic order of Sec. 4 (instruction 6m+2) as modified in
 * Sec. 5: bitstring coordinates first, then the numeric last coordinate, and
 * on a complete tie queries precede data points.  IDs finish the order so the
 * result does not depend on the sort's stability. */
static int cmp_record(const void* pa, const void* pb) {
    const record_t* a = (const record_t*)pa;
    const record_t* b = (const record_t*)pb;
    for (int i = 0; i < g_m - 1; ++i) {
        int c = cmp_bits(a->len[i], a->val[i], b->len[i], b->val[i]);
        if (c) return c;
    }
    if (a->last != b->last) return a->last < b->last ? -1 : 1;
    if (a->is_query != b->is_query) {
#if ORACLE_PLANT == 2
        return a->is_query ? 1 : -1; /* planted: data before queries */
#else
        return a->is_query ? -1 : 1;
#endif
    }
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

static int same_segment(const record_t* a, const record_t* b) {
    for (int i = 0; i < g_m - 1; ++i)
        if (a->len[i] != b->len[i] || a->val[i] != b->val[i]) return 0;
#if ORACLE_PLANT == 4
    if (a->last != b->last) return 0; /* planted: last coordinate also tags segments */
#endif
    return 1;
}

static int cmp_double(const void* pa, const void* pb) {
    double a = *(const double*)pa, b = *(const double*)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Digits needed for 0-based ranks in [0, U): ceil(log2 U), 0 when U <= 1. */
static int digits_for(int64_t U) {
    int b = 0;
    while (((int64_t)1 << b) < U) ++b;
#if ORACLE_PLANT == 3
    if (b > 0) --b; /* planted: one binary digit too few */
#endif
    return b;
}

/* Dense 0-based rank of v among the sorted distinct values u[0..U). */
static int64_t rank_of(const double* u, int64_t U, double v) {
    int64_t lo = 0, hi = U; /* first index with u[idx] >= v */
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (u[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

typedef struct {
    int64_t id;
    agg_t a;
} idval_t;

static int cmp_id_desc(const void* pa, const void* pb) {
    const idval_t* a = (const idval_t*)pa;
    const idval_t* b = (const idval_t*)pb;
    return a->id > b->id ? -1 : (a->id < b->id ? 1 : 0);
}

/* Runs the pipeline.  If T_out is not NULL it receives the number of records
 * of the flat map (instruction 6m+1 as reduced by Sec. 5).  If out is NULL only
 * the record count is computed. */
int oracle_sortscan(int m, const void* D, int64_t nD, const void* Q, int64_t nQ, int ct,
                    const void* W, int wt, int op, void* out, int64_t* T_out) {
    int st = check_args(m, nD, nQ, ct, wt, op);
    if (st) return st;
    if (m > MAXM) return OR_ERR_ARG;
    if (any_nan(D, ct, nD, m) || any_nan(Q, ct, nQ, m)) return OR_ERR_NAN;
    int64_t N = nD + nQ;

    /* Instruction 0: DQ, here the concatenation of D and Q; point k < nD is
     * data point k, point k >= nD is query k - nD. */
#define DQ_COORD(k, i) ((k) < nD ? coord_at(D, ct, (k), m, (i)) : coord_at(Q, ct, (k) - nD, m, (i)))

    /* Instructions 5i-4 .. 5i and 5m+i for the first m-1 dimensions: sort the
     * coordinate, count distinct values (U_i), rank every point densely and
     * write the rank with b_i binary digits. */
    int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1) * (size_t)(m > 1 ? m - 1 : 1));
    int b[MAXM];
    double* col = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!rank || !col) {
        free(rank);
        free(col);
        return OR_ERR_ARG;
    }
    for (int i = 0; i < m - 1; ++i) {
        for (int64_t k = 0; k < N; ++k) col[k] = DQ_COORD(k, i);
        qsort(col, (size_t)N, sizeof(double), cmp_double);
        int64_t U = 0;
        for (int64_t k = 0; k < N; ++k)
            if (k == 0 || col[k] != col[k - 1]) col[U++] = col[k];
        b[i] = digits_for(U);
        for (int64_t k = 0; k < N; ++k) rank[k * (m - 1) + i] = rank_of(col, U, DQ_COORD(k, i));
    }
    free(col);

    /* Instruction 6m+1 with Sec. 5: every data point is replaced by the
     * product P0(r_1) x ... x P0(r_{m-1}), every query by the product of its
     * P1 sets; the last coordinate stays a number, IDs are inherited. */
    int64_t T = 0;
    for (int64_t k = 0; k < N; ++k) {
        int64_t c = 1;
        for (int i = 0; i < m - 1; ++i) {
            int lens[64];
            uint64_t vals[64];
            c *= oracle_prefix_set((uint64_t)rank[k * (m - 1) + i], b[i], k < nD ? 0 : 1, lens, vals);
        }
        T += c;
    }
    if (T_out) *T_out = T;
    if (!out) {
        free(rank);
        return OR_OK;
    }
    record_t* rec = (record_t*)malloc(sizeof(record_t) * (size_t)(T > 0 ? T : 1));
    if (!rec) {
        free(rank);
        return OR_ERR_ARG;
    }
    int64_t t = 0;
    for (int64_t k = 0; k < N; ++k) {
        int which = k < nD ? 0 : 1;
        int cnt[MAXM], lens[MAXM][64];
        uint64_t vals[MAXM][64];
        int64_t c = 1;
        for (int i = 0; i < m - 1; ++i) {
            cnt[i] = oracle_prefix_set((uint64_t)rank[k * (m - 1) + i], b[i], which, lens[i], vals[i]);
            c *= cnt[i];
        }
        for (int64_t e = 0; e < c; ++e) { /* mixed-radix walk over the product */
            int64_t rest = e;
            record_t* r = &rec[t++];
            memset(r, 0, sizeof(*r));
            for (int i = m - 2; i >= 0; --i) {
                int pick = (int)(rest % cnt[i]);
                rest /= cnt[i];
                r->len[i] = lens[i][pick];
                r->val[i] = vals[i][pick];
            }
            r->last = DQ_COORD(k, m - 1);
            r->is_query = which;
            r->id = k;
        }
    }
    free(rank);

    /* Instruction 6m+2: SEDQ = sort(EDQ, doubly lexicographic). */
    g_m = m;
    qsort(rec, (size_t)T, sizeof(record_t), cmp_record);

    /* Instruction 6m+3: A_1 = sscan(weights, tags, F); a query weighs e. */
    idval_t* A = (idval_t*)malloc(sizeof(idval_t) * (size_t)(T > 0 ? T : 1));
    if (!A) {
        free(rec);
        return OR_ERR_ARG;
    }
    agg_t e = agg_unit(wt, op);
    agg_t run = e;
    for (int64_t k = 0; k < T; ++k) {
        if (k == 0 || !same_segment(&rec[k - 1], &rec[k])) run = e;
        agg_t w = rec[k].is_query ? e : weight_of(W, wt, op, rec[k].id);
        run = agg_F(run, w, op);
        A[k].id = rec[k].id;
        A[k].a = run;
    }
    free(rec);

    /* Instructions 6m+4, 6m+5: sort A_1 by ID (non-increasing) and run a
     * segmented scan with the IDs as tags; each query's total ends at the last
     * element of its ID segment.  (Instructions 6m+6 .. 6m+9 only copy that
     * total back to every tuple of the query; one value per query is kept.) */
    qsort(A, (size_t)T, sizeof(idval_t), cmp_id_desc);
    for (int64_t q = 0; q < nQ; ++q) store_out(out, wt, op, q, e);
    run = e;
    for (int64_t k = 0; k < T; ++k) {
        if (k == 0 || A[k].id != A[k - 1].id) run = e;
        run = agg_F(run, A[k].a, op);
        int last_of_segment = (k + 1 == T) || A[k + 1].id != A[k].id;
        if (last_of_segment && A[k].id >= nD) store_out(out, wt, op, A[k].id - nD, run);
    }
    free(A);
#undef DQ_COORD
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 4. m = 2 by a sweep over the last coordinate with a Fenwick tree    */
/* ------------------------------------------------------------------ */

/* A classical O(n log n) route to the definition of Sec. 1.2 for m = 2,
 * independent of the paper's pipeline: visit the points in the order of the
 * last coordinate; a data point is added to a Fenwick (binary indexed) tree
 * at the dense rank of its first coordinate, and a query reads F over the
 * tree's prefix of smaller ranks.  A tied last coordinate puts queries first
 * (the query must not see a datum with an equal last coordinate); with
 * bit 1 of `nonstrict` set (d_1 <= q_1) data go first.  With bit 0 set
 * (d_0 <= q_0) the query reads the prefix up to and including its own rank.
 * Sums of float32 weights are accumulated in double: the tree adds them in a
 * different order than the definition does, so the result may differ from
 * the exact sum by a few units of 2^-53 times sum |w|, far below the float32
 * tolerance the tests use.  Integer sums wrap modulo 2^64 and max / min are
 * exact, so those results are identical to the definition's. */

typedef struct {
    double x0, x1; /* the two coordinates (-0.0 folded into +0.0) */
    int64_t idx;   /* data: index into D; query: nD + index into Q */
    int64_t rank;  /* dense 0-based rank of x0 among all points */
} sweep_pt;

static int g_sweep_data_first; /* tie order of the last coordinate */
static int64_t g_sweep_nD;

static int cmp_sweep_x0(const void* pa, const void* pb) {
    const sweep_pt* a = (const sweep_pt*)pa;
    const sweep_pt* b = (const sweep_pt*)pb;
    if (a->x0 != b->x0) return a->x0 < b->x0 ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

static int cmp_sweep(const void* pa, const void* pb) {
    const sweep_pt* a = (const sweep_pt*)pa;
    const sweep_pt* b = (const sweep_pt*)pb;
    if (a->x1 != b->x1) return a->x1 < b->x1 ? -1 : 1;
    int aq = a->idx >= g_sweep_nD, bq = b->idx >= g_sweep_nD;
    if (aq != bq) {
        int q_first = aq ? -1 : 1;
#if ORACLE_PLANT == 5
        return -q_first; /* planted: data before queries on a tie */
#else
        return g_sweep_data_first ? -q_first : q_first;
#endif
    }
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* A node of the Fenwick tree: F over its range, and the sum of |w| there. */
typedef struct {
    agg_t a;
    double s;
} fen_t;

/* Core of the sweep over points given as doubles.  xd/xq are [n][2]; the
 * weight of data point d is taken by weight_of(W, wt, op, d). */
static int sweep2(const double* xd, int64_t nD, const double* xq, int64_t nQ, const void* W, int wt, int op,
                  unsigned nonstrict, void* out, double* S) {
    int64_t N = nD + nQ;
    sweep_pt* P = (sweep_pt*)malloc(sizeof(sweep_pt) * (size_t)(N > 0 ? N : 1));
    if (!P) return OR_ERR_ARG;
    for (int64_t k = 0; k < N; ++k) {
        const double* x = k < nD ? xd + 2 * k : xq + 2 * (k - nD);
        P[k].x0 = x[0];
        P[k].x1 = x[1];
        P[k].idx = k;
    }
    /* dense 0-based ranks of the first coordinate: sort by it, count changes */
    qsort(P, (size_t)N, sizeof(sweep_pt), cmp_sweep_x0);
    int64_t U = 0;
    for (int64_t k = 0; k < N; ++k) {
        if (k > 0 && P[k].x0 != P[k - 1].x0) ++U;
        P[k].rank = U;
    }
    if (N > 0) ++U;
    /* the order of the last coordinate */
    g_sweep_nD = nD;
    g_sweep_data_first = (int)((nonstrict >> 1) & 1u);
    qsort(P, (size_t)N, sizeof(sweep_pt), cmp_sweep);
    /* Fenwick tree over ranks 1..U (1-based inside the tree) */
    fen_t* tree = (fen_t*)malloc(sizeof(fen_t) * (size_t)(U + 1));
    if (!tree) {
        free(P);
        return OR_ERR_ARG;
    }
    agg_t e = agg_unit(wt, op);
    for (int64_t k = 0; k <= U; ++k) {
        tree[k].a = e;
        tree[k].s = 0.0;
    }
#if ORACLE_PLANT == 6
    const int incl = 1; /* planted: the query's own rank is included */
#else
    const int incl = (int)(nonstrict & 1u);
#endif
    for (int64_t k = 0; k < N; ++k) {
        if (P[k].idx < nD) {
            agg_t w = weight_of(W, wt, op, P[k].idx);
            double aw = abs_weight(W, wt, op, P[k].idx);
            for (int64_t j = P[k].rank + 1; j <= U; j += j & (-j)) {
                tree[j].a = agg_F(tree[j].a, w, op);
                tree[j].s += aw;
            }
        } else {
            /* F over ranks [0, rank) (strict) or [0, rank] (non-strict) */
            agg_t acc = e;
            double s = 0.0;
            for (int64_t j = P[k].rank + (incl ? 1 : 0); j > 0; j -= j & (-j)) {
                acc = agg_F(acc, tree[j].a, op);
                s += tree[j].s;
            }
            store_out(out, wt, op, P[k].idx - nD, acc);
            if (S) S[P[k].idx - nD] = s;
        }
    }
    free(P);
    free(tree);
    return OR_OK;
}

static double* coords_as_double(const void* base, int ct, int64_t n, double sign) {
    double* x = (double*)malloc(sizeof(double) * (size_t)(2 * n > 0 ? 2 * n : 1));
    if (!x) return NULL;
    for (int64_t k = 0; k < n; ++k)
        for (int i = 0; i < 2; ++i) {
            double v = sign * coord_at(base, ct, k, 2, i);
            x[2 * k + i] = v == 0.0 ? 0.0 : v; /* -0.0 is +0.0 */
        }
    return x;
}

/* out(q) = F over { w(d) : d < q } for m = 2 (bit i of nonstrict: d_i <= q_i),
 * by the sweep above.  Same conventions as oracle_brute_ns. */
int oracle_sweep2(const void* D, int64_t nD, const void* Q, int64_t nQ, int ct, const void* W, int wt, int op,
                  unsigned nonstrict, void* out, double* S) {
    int st = check_args(2, nD, nQ, ct, wt, op);
    if (st) return st;
    if (nonstrict > 3u) return OR_ERR_ARG;
    if (any_nan(D, ct, nD, 2) || any_nan(Q, ct, nQ, 2)) return OR_ERR_NAN;
    double* xd = coords_as_double(D, ct, nD, 1.0);
    double* xq = coords_as_double(Q, ct, nQ, 1.0);
    st = (xd && xq) ? sweep2(xd, nD, xq, nQ, W, wt, op, nonstrict, out, S) : OR_ERR_ARG;
    free(xd);
    free(xq);
    return st;
}

/* The adjoint of the float32 sum for m = 2: grad(d) = sum of g(q) over
 * queries q with d < q (bit i of nonstrict: d_i <= q_i), by the sweep on the
 * negated problem: with every coordinate negated, q plays a data point of
 * weight g(q) and d a query (d_i < q_i  <=>  -q_i < -d_i; negation is exact
 * in double for int32 and float32 values). */
int oracle_sweep2_transpose(const void* D, int64_t nD, const void* Q, int64_t nQ, int ct, const float* G,
                            unsigned nonstrict, double* grad, double* S) {
    if (nD < 0 || nQ < 0 || (ct != CT_I32 && ct != CT_F32) || nonstrict > 3u) return OR_ERR_ARG;
    if (any_nan(D, ct, nD, 2) || any_nan(Q, ct, nQ, 2)) return OR_ERR_NAN;
    double* xq = coords_as_double(Q, ct, nQ, -1.0); /* the new data points */
    double* xd = coords_as_double(D, ct, nD, -1.0); /* the new queries */
    int st = (xd && xq) ? sweep2(xq, nQ, xd, nD, G, WT_F32, OP_SUM, nonstrict, grad, S) : OR_ERR_ARG;
    free(xd);
    free(xq);
    return st;
}

/* Number of threads OpenMP would use (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
