/*
 * bdc_oracle.c -- plain, slow, FP64 CPU oracle for Blahut-Arimoto on the
 * finite-length binary deletion channel BDC_d (inputs {0,1}^n, outputs
 * {0,1}^{<=n}).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this file.  It shares no
 * code, header, table or helper with the CUDA library: it is written from the
 * paper's definitions, in the paper's order, with no blocking or fusion.
 *
 * Encoding (the paper indexes strings from 0, Sec. 2.1):
 *   - a string s of length L is the integer whose most significant of L bits
 *     is s_0, so lexicographic order is numeric order;
 *   - an output y of length k has code (1<<k)|y; the empty output has code 1;
 *   - logarithms are base 2 (Sec. 2.1).
 *
 * Parity status: every function below is pinned by a -m "not gpu" test
 * against closed forms, brute force or a library routine; see the test files
 * named in each comment.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXN 32

/* s_i, the i-th symbol (0-indexed from the left) of the length-L string s. */
static int sym(uint64_t s, int L, int i) { return (int)((s >> (L - 1 - i)) & 1u); }

static double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; i++) r = r * (double)(n - k + i) / (double)i;
    return floor(r + 0.5);
}

/* Probability of keeping exactly k of n symbols with a fixed keep set under
 * BDC_d: d^(n-k) (1-d)^k, with 0^0 = 1 (C pow already gives pow(0,0) = 1). */
static double keep_weight(int n, int k, double d) {
    return pow(d, (double)(n - k)) * pow(1.0 - d, (double)k);
}

/* ---------------------------------------------------------------------------
 * Channel rule (Sec. 2.2): P_{n,k}(y|x) = (#times y appears as a subsequence
 * of x) / C(n,k), and BDC_d gives W(y|x) = #emb * d^(n-k) (1-d)^k.
 * ------------------------------------------------------------------------- */

/* #embeddings of y (length k) into x (length n): textbook DP, M[j] = number of
 * ways to embed y_0..y_{j-1} into the prefix of x scanned so far. */
uint64_t orc_embed_count(int n, uint64_t x, int k, uint64_t y) {
    uint64_t M[ORC_MAXN + 2];
    if (k > n) return 0;
    memset(M, 0, sizeof M);
    M[0] = 1;
    for (int i = 0; i < n; i++) {
        int b = sym(x, n, i);
        for (int j = k; j >= 1; j--)
            if (sym(y, k, j - 1) == b) M[j] += M[j - 1];
    }
    return M[k];
}

/* Brute force over all 2^n deletion patterns of x (a keep mask m, symbol i
 * kept iff bit i from the left of m is 1).  counts[code] += 1 and
 * W[code] += d^(n-|m|)(1-d)^|m|.  Arrays have 2^(n+1) entries, zeroed here. */
void orc_channel_row_bruteforce(int n, uint64_t x, double d, uint64_t *counts, double *W) {
    uint64_t nout = 1ull << (n + 1);
    if (counts) memset(counts, 0, nout * sizeof(uint64_t));
    if (W) memset(W, 0, nout * sizeof(double));
    for (uint64_t m = 0; m < (1ull << n); m++) {
        uint64_t y = 0;
        int k = 0;
        for (int i = 0; i < n; i++)
            if (sym(m, n, i)) { y = (y << 1) | (uint64_t)sym(x, n, i); k++; }
        uint64_t code = (1ull << k) | y;
        if (counts) counts[code] += 1;
        if (W) W[code] += keep_weight(n, k, d);
    }
}

/* ---------------------------------------------------------------------------
 * Distinct subsequences of x with their multiplicities.  Depth-first walk of
 * the subsequence trie; a child y.b exists iff its embedding count is > 0.
 * The count of a child comes from the same textbook DP as orc_embed_count,
 * evaluated one column at a time: col_j[i] = #embeddings of y_0..y_{j-1} into
 * x_0..x_{i-1}; col_{j+1}[i] = col_{j+1}[i-1] + [x_{i-1} = y_j] col_j[i-1].
 * The visitor receives (code, length, count) for every nonempty distinct y,
 * in depth-first (lexicographic prefix) order.
 * ------------------------------------------------------------------------- */
typedef void (*orc_visit_fn)(void *ctx, uint64_t code, int k, uint64_t count);

static void subseq_walk(int n, uint64_t x, orc_visit_fn visit, void *ctx) {
    uint64_t col[ORC_MAXN + 1][ORC_MAXN + 1];
    uint64_t code[ORC_MAXN + 1];
    int next_b[ORC_MAXN + 1];
    for (int i = 0; i <= n; i++) col[0][i] = 1; /* the empty string embeds once */
    code[0] = 1;
    next_b[0] = 0;
    int t = 0;
    while (t >= 0) {
        if (t == n || next_b[t] > 1) { t--; continue; }
        int b = next_b[t]++;
        uint64_t *c = col[t], *cn = col[t + 1];
        cn[0] = 0;
        for (int i = 1; i <= n; i++)
            cn[i] = cn[i - 1] + ((uint64_t)sym(x, n, i - 1) == (uint64_t)b ? c[i - 1] : 0);
        if (cn[n] == 0) continue;
        code[t + 1] = (code[t] << 1) | (uint64_t)b;
        visit(ctx, code[t + 1], t + 1, cn[n]);
        next_b[t + 1] = 0;
        t++;
    }
}

typedef struct { uint64_t *N; double *S; uint64_t *sumc; } stats_ctx;
static void stats_visit(void *vctx, uint64_t code, int k, uint64_t count) {
    stats_ctx *c = (stats_ctx *)vctx;
    (void)code;
    c->N[k] += 1;
    c->sumc[k] += count;
    c->S[k] += (double)count * log2((double)count);
}

/* Per length k: N_k = #distinct length-k subsequences (the paper's N_{x,k},
 * Sec. 4.1 Cnt[0][k]); S_k = sum over them of count*log2(count);
 * sumc_k = sum of counts (= C(n,k)).  k = 0 is the empty string. */
void orc_subseq_stats(int n, uint64_t x, uint64_t *N, double *S, uint64_t *sumc) {
    for (int k = 0; k <= n; k++) { N[k] = 0; S[k] = 0.0; sumc[k] = 0; }
    N[0] = 1; sumc[0] = 1; /* empty subsequence: one embedding, log2(1) = 0 */
    stats_ctx c = {N, S, sumc};
    subseq_walk(n, x, stats_visit, &c);
}

typedef struct { uint64_t *codes; uint64_t *counts; int64_t m; } list_ctx;
static void list_visit(void *vctx, uint64_t code, int k, uint64_t count) {
    list_ctx *c = (list_ctx *)vctx;
    (void)k;
    if (c->codes) c->codes[c->m] = code;
    if (c->counts) c->counts[c->m] = count;
    c->m++;
}

/* All nonempty distinct subsequences of x (codes, counts) in walk order;
 * returns how many.  Pass NULL arrays to only count them. */
int64_t orc_subseq_list(int n, uint64_t x, uint64_t *codes, uint64_t *counts) {
    list_ctx c = {codes, counts, 0};
    subseq_walk(n, x, list_visit, &c);
    return c.m;
}

/* ---------------------------------------------------------------------------
 * Output marginal and divergence, straight from their definitions (Sec. 2.3):
 *   q(y)  = sum_x p(x) W(y|x)
 *   D_x   = sum_y W(y|x) log2(W(y|x) / q(y))
 * ------------------------------------------------------------------------- */

typedef struct { double *q; double px; const double *kw; } qctx;
static void q_visit(void *vctx, uint64_t code, int k, uint64_t count) {
    qctx *c = (qctx *)vctx;
    c->q[code] += c->px * (double)count * c->kw[k];
}

/* q over all 2^(n+1) codes (slot 0 unused, set to 0).  Plain scatter over
 * every (x, distinct y) pair; the empty output gets sum_x p(x) d^n. */
void orc_q_full(int n, double d, const double *p, double *q) {
    double kw[ORC_MAXN + 1];
    for (int k = 0; k <= n; k++) kw[k] = keep_weight(n, k, d);
    memset(q, 0, (1ull << (n + 1)) * sizeof(double));
    for (uint64_t x = 0; x < (1ull << n); x++) {
        qctx c = {q, p[x], kw};
        q[1] += p[x] * kw[0];
        subseq_walk(n, x, q_visit, &c);
    }
}

/* q at one code, summing over every input x in {0,1}^n (count by DP). */
double orc_q_point(int n, double d, const double *p, uint64_t code) {
    int k = 63 - __builtin_clzll(code);
    uint64_t y = code ^ (1ull << k);
    double w = keep_weight(n, k, d), acc = 0.0;
    for (uint64_t x = 0; x < (1ull << n); x++) {
        uint64_t c = orc_embed_count(n, x, k, y);
        if (c) acc += p[x] * (double)c * w;
    }
    return acc;
}

typedef struct { const double *q; const double *kw; double acc; int bad; } dctx;
static void d_visit(void *vctx, uint64_t code, int k, uint64_t count) {
    dctx *c = (dctx *)vctx;
    double w = (double)count * c->kw[k];
    if (w == 0.0) return;
    if (!(c->q[code] > 0.0)) { c->bad = 1; return; }
    c->acc += w * log2(w / c->q[code]);
}

/* D_x for q indexed by code.  Returns +INFINITY if some y with W(y|x) > 0 has
 * q(y) <= 0. */
double orc_D_point(int n, double d, const double *q, uint64_t x) {
    double kw[ORC_MAXN + 1];
    for (int k = 0; k <= n; k++) kw[k] = keep_weight(n, k, d);
    dctx c = {q, kw, 0.0, 0};
    double w0 = kw[0];
    if (w0 > 0.0) {
        if (!(q[1] > 0.0)) return INFINITY;
        c.acc += w0 * log2(w0 / q[1]);
    }
    subseq_walk(n, x, d_visit, &c);
    return c.bad ? INFINITY : c.acc;
}

/* D_x for every x (OpenMP over x when compiled with it). */
void orc_D_full(int n, double d, const double *q, double *D) {
    int64_t nx = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t x = 0; x < nx; x++) D[x] = orc_D_point(n, d, q, (uint64_t)x);
}

/* D_x for a list of inputs (OpenMP over the list).  Used to time the oracle
 * on a sample (orc_pairs_list counts the pairs it enumerates, separately). */
void orc_D_list(int n, double d, const double *q, const uint64_t *xs, int64_t count, double *D) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < count; i++) D[i] = orc_D_point(n, d, q, xs[i]);
}

/* Number of (x, distinct y) pairs, the empty output included, over a list
 * of inputs (OpenMP). */
int64_t orc_pairs_list(int n, const uint64_t *xs, int64_t count) {
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : pairs)
    for (int64_t i = 0; i < count; i++) pairs += orc_subseq_list(n, xs[i], NULL, NULL) + 1;
    return pairs;
}

/* Threads of the OpenMP loops (<= 0: leave the runtime's default); returns
 * the number the loops will use. */
int orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

/* Dual (minimax) upper bound for any positive q: max_x D(W_x || q/sum q)
 * = max_x D_x(q) + log2 sum_y q(y).  Also returns argmax. */
double orc_certify(int n, double d, const double *q, int64_t *argmax) {
    int64_t nx = (int64_t)1 << n;
    double s = 0.0;
    for (uint64_t c = 1; c < (1ull << (n + 1)); c++) s += q[c];
    double best = -INFINITY;
    int64_t arg = 0;
    double *D = (double *)malloc((size_t)nx * sizeof(double));
    orc_D_full(n, d, q, D);
    for (int64_t x = 0; x < nx; x++)
        if (D[x] > best) { best = D[x]; arg = x; }
    free(D);
    if (argmax) *argmax = arg;
    return best + log2(s);
}

/* ---------------------------------------------------------------------------
 * Generic Blahut-Arimoto on a DMC given as sparse rows (Sec. 2.3), in the
 * paper's order: output distribution, refined input distribution,
 * normalisation, stopping test.  In log2 form (Sec. 3): with
 * D_x = sum_y P(y|x) log2(P(y|x)/Y(y)), the refined input is X(x) 2^{D_x}.
 * At iteration t (using X^(t) and its Y^(t)) it records
 *   lower_t = log2 sum_x X^(t)(x) 2^{D_x}   (Blahut's lower bound)
 *   upper_t = max_x D_x                      (the dual upper bound)
 *   stat_t  = max_x log2(X^(t+1)(x)/X^(t)(x)) (the stopping statistic)
 * and stops once stat_t < tol (the paper's test) or after max_iters updates.
 * p is read as X^(0) and overwritten by the final X.  Returns iterations run.
 * ------------------------------------------------------------------------- */
int orc_ba_sparse(int64_t nx, int64_t ny, const int64_t *rowptr, const int64_t *col,
                  const double *val, double *p, int max_iters, double tol,
                  double *lower, double *upper, double *stat) {
    double *q = (double *)malloc((size_t)ny * sizeof(double));
    double *D = (double *)malloc((size_t)nx * sizeof(double));
    int t;
    for (t = 0; t < max_iters; t++) {
        for (int64_t y = 0; y < ny; y++) q[y] = 0.0;
        for (int64_t x = 0; x < nx; x++)
            for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++) q[col[e]] += p[x] * val[e];
        double up = -INFINITY;
        for (int64_t x = 0; x < nx; x++) {
            double acc = 0.0;
            for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++)
                if (val[e] > 0.0) acc += val[e] * log2(val[e] / q[col[e]]);
            D[x] = acc;
            if (acc > up) up = acc;
        }
        double Z = 0.0;
        for (int64_t x = 0; x < nx; x++) Z += p[x] * exp2(D[x]);
        double st = -INFINITY;
        for (int64_t x = 0; x < nx; x++) {
            double pn = p[x] * exp2(D[x]) / Z;
            if (p[x] > 0.0) {
                double r = log2(pn / p[x]);
                if (r > st) st = r;
            }
            p[x] = pn;
        }
        if (lower) lower[t] = log2(Z);
        if (upper) upper[t] = up;
        if (stat) stat[t] = st;
        if (st < tol) { t++; break; }
    }
    free(q);
    free(D);
    return t;
}

/* Sparse rows of BDC_d for inputs of length n, built by brute force over all
 * deletion patterns (n <= 14).  Columns are codes.  Returns nnz; call with
 * NULL arrays first to size them. */
int64_t orc_bdc_rows(int n, double d, int64_t *rowptr, int64_t *col, double *val) {
    uint64_t nout = 1ull << (n + 1);
    uint64_t *cnt = (uint64_t *)malloc(nout * sizeof(uint64_t));
    double *W = (double *)malloc(nout * sizeof(double));
    int64_t e = 0;
    for (uint64_t x = 0; x < (1ull << n); x++) {
        if (rowptr) rowptr[x] = e;
        orc_channel_row_bruteforce(n, x, d, cnt, W);
        for (uint64_t c = 1; c < nout; c++)
            if (cnt[c]) {
                if (col) { col[e] = (int64_t)c; val[e] = W[c]; }
                e++;
            }
    }
    if (rowptr) rowptr[1ull << n] = e;
    free(cnt);
    free(W);
    return e;
}

/* Sparse rows of the exact deletion channel BDC_{n,k} (Sec. 2.2): outputs are
 * the 2^k strings of length k (column = y, not the code). */
int64_t orc_exact_rows(int n, int k, int64_t *rowptr, int64_t *col, double *val) {
    double ck = binom(n, k);
    int64_t e = 0;
    for (uint64_t x = 0; x < (1ull << n); x++) {
        if (rowptr) rowptr[x] = e;
        for (uint64_t y = 0; y < (1ull << k); y++) {
            uint64_t c = orc_embed_count(n, x, k, y);
            if (c) {
                if (col) { col[e] = (int64_t)y; val[e] = (double)c / ck; }
                e++;
            }
        }
    }
    if (rowptr) rowptr[1ull << n] = e;
    return e;
}

/* ---------------------------------------------------------------------------
 * Paper algorithms kept as pinned references (Sec. 4 and Sec. 5).
 * ------------------------------------------------------------------------- */

/* Sec. 4.1: NextPos[i][b] = smallest p >= i with x_p = b, else n (scan from
 * right to left), and Cnt[i][t] = #distinct length-t subsequences of x[i:]
 * by the four-case recursion on NextPos.  Tables are (n+1) x 2 and
 * (n+1) x (kmax+1), row-major. */
void orc_nextpos_cnt(int n, uint64_t x, int kmax, int32_t *nextpos, uint64_t *cnt) {
    for (int b = 0; b < 2; b++) nextpos[2 * n + b] = n;
    for (int i = n - 1; i >= 0; i--) {
        nextpos[2 * i + 0] = nextpos[2 * (i + 1) + 0];
        nextpos[2 * i + 1] = nextpos[2 * (i + 1) + 1];
        nextpos[2 * i + sym(x, n, i)] = i;
    }
    int W = kmax + 1;
    for (int i = 0; i <= n; i++) cnt[i * W + 0] = 1;
    for (int t = 1; t <= kmax; t++) cnt[n * W + t] = 0;
    for (int i = n - 1; i >= 0; i--) {
        int j0 = nextpos[2 * i], j1 = nextpos[2 * i + 1];
        for (int t = 1; t <= kmax; t++) {
            uint64_t v = 0;
            if (j0 < n) v += cnt[(j0 + 1) * W + (t - 1)];
            if (j1 < n) v += cnt[(j1 + 1) * W + (t - 1)];
            cnt[i * W + t] = v;
        }
    }
}

/* Sec. 4.2, Alg. unrank(x,k,j): the j-th (0-based) lexicographically
 * smallest distinct length-k subsequence of x.  Returns 0 and writes y, or -1
 * if j >= Cnt[0][k]. */
int orc_unrank(int n, uint64_t x, int k, uint64_t j, uint64_t *y_out) {
    int32_t np[2 * (ORC_MAXN + 1)];
    uint64_t cnt[(ORC_MAXN + 1) * (ORC_MAXN + 1)];
    orc_nextpos_cnt(n, x, k, np, cnt);
    int W = k + 1;
    if (j >= cnt[0 * W + k]) return -1;
    int i = 0, rem = k;
    uint64_t y = 0;
    while (rem > 0) {
        int j0 = np[2 * i + 0];
        uint64_t c0 = (j0 < n) ? cnt[(j0 + 1) * W + (rem - 1)] : 0;
        if (j < c0) { y = y << 1; i = j0 + 1; rem--; continue; }
        j -= c0;
        int j1 = np[2 * i + 1];
        uint64_t c1 = (j1 < n) ? cnt[(j1 + 1) * W + (rem - 1)] : 0;
        if (j < c1) { y = (y << 1) | 1u; i = j1 + 1; rem--; continue; }
        return -1; /* unreachable when j < Cnt[0][k] */
    }
    *y_out = y;
    return 0;
}

/* Sec. 5.1, Alg. subsetUnrank(n,w,j): scan t = 0..n-1 over the 0-based
 * ground set; c = C(n-t-1, w-1) subsets take t as their next element.
 * Writes the w chosen elements in increasing order; returns w. */
int orc_subset_unrank(int n, int w, uint64_t j, int32_t *subset) {
    int m = 0;
    for (int t = 0; t < n; t++) {
        if (w == 0) break;
        uint64_t c = (uint64_t)binom(n - t - 1, w - 1);
        if (j < c) { subset[m++] = t; w--; }
        else j -= c;
    }
    return m;
}

/* Sec. 5.2, Alg. RecSuperSeq(i,n,k,y): the i-th length-n supersequence of y.
 * w is the smallest with i < C(n,<=w); S = subsetUnrank(n, w, i - C(n,<=w-1))
 * are the unmatched positions.  Positions in S get the complement of the next
 * unmatched symbol of y (of y_{k-1} once y is exhausted).  Positions outside S
 * copy the next symbol of y; once y is exhausted the printed algorithm sets
 * them "arbitrarily (e.g. 0)" (fixed = 0), which is not injective; the
 * reading used here (fixed = 1) sets them to y_{k-1}, so that they cannot
 * be confused with a position of S.  k >= 1.  Returns the string x. */
uint64_t orc_recsuperseq(uint64_t i, int n, int k, uint64_t y, int fixed) {
    int w = 0;
    uint64_t below = 0; /* C(n, <= w-1) */
    while (w <= n - k) {
        uint64_t cw = (uint64_t)binom(n, w);
        if (i < below + cw) break;
        below += cw;
        w++;
    }
    int32_t S[ORC_MAXN + 1];
    int m = orc_subset_unrank(n, w, i - below, S);
    int inS[ORC_MAXN + 1];
    memset(inS, 0, sizeof inS);
    for (int a = 0; a < m; a++) inS[S[a]] = 1;
    uint64_t x = 0;
    int r = 0;
    for (int p = 0; p < n; p++) {
        int b;
        if (inS[p]) b = (r < k) ? 1 - sym(y, k, r) : 1 - sym(y, k, k - 1);
        else if (r < k) { b = sym(y, k, r); r++; }
        else b = fixed ? sym(y, k, k - 1) : 0;
        x = (x << 1) | (uint64_t)b;
    }
    return x;
}

/* ---------------------------------------------------------------------------
 * Orbits under complement and reversal (Appendix A).
 * ------------------------------------------------------------------------- */
static uint64_t rev_bits(uint64_t s, int L) {
    uint64_t r = 0;
    for (int i = 0; i < L; i++) r |= (uint64_t)sym(s, L, i) << i;
    return r;
}
/* Representative = lexicographically smallest member of {s, cpl s, rev s,
 * cpl rev s}; *osize receives the orbit size (number of distinct members). */
uint64_t orc_orbit_rep(uint64_t s, int L, int *osize) {
    uint64_t mask = (L == 64) ? ~0ull : ((1ull << L) - 1);
    uint64_t m[4] = {s, s ^ mask, rev_bits(s, L), rev_bits(s, L) ^ mask};
    uint64_t best = m[0];
    int distinct = 0;
    for (int a = 0; a < 4; a++) {
        if (m[a] < best) best = m[a];
        int seen = 0;
        for (int b = 0; b < a; b++) if (m[b] == m[a]) seen = 1;
        if (!seen) distinct++;
    }
    if (osize) *osize = distinct;
    return best;
}

/* ---------------------------------------------------------------------------
 * Smoothed dual bound (tau-log-sum-exp of D_x over all inputs) and its
 * gradient, for q = softmax over output orbit classes.
 *   q(c)    = exp(theta[cls(c)]) / sum_c' exp(theta[cls(c')])
 *   F       = tau log2 sum_x 2^{D_x(q)/tau}
 *   dF/dL_c = -sum_x pi_x W(c|x),  pi = softmax_x(D/tau), L = log2 q
 *   dF/dtheta_r = (sum_{c in class r} dF/dL_c + |class r| q_r) / ln 2
 *   dF/dd   = sum_x pi_x sum_y dW/dd log2(W/q),  dW/dd = W((n-k)/d - k/(1-d))
 * cls maps every code in [1, 2^(n+1)) to its class index (slot 0 unused).
 * Dense over all pairs; n <= 12.  grad_theta has ncls entries.
 * ------------------------------------------------------------------------- */
double orc_dual_bound(int n, double d, double tau, const double *theta, const int64_t *cls,
                      int64_t ncls, double *grad_theta, double *grad_d) {
    uint64_t nout = 1ull << (n + 1);
    int64_t nx = (int64_t)1 << n;
    double *q = (double *)calloc(nout, sizeof(double));
    double *g = (double *)calloc(nout, sizeof(double));
    double *Dx = (double *)malloc((size_t)nx * sizeof(double));
    double *dD = (double *)malloc((size_t)nx * sizeof(double));
    uint64_t *cnt = (uint64_t *)malloc(nout * sizeof(uint64_t));
    double *W = (double *)malloc(nout * sizeof(double));
    double tmax = -INFINITY;
    for (uint64_t c = 1; c < nout; c++) if (theta[cls[c]] > tmax) tmax = theta[cls[c]];
    double Zt = 0.0;
    for (uint64_t c = 1; c < nout; c++) Zt += exp(theta[cls[c]] - tmax);
    for (uint64_t c = 1; c < nout; c++) q[c] = exp(theta[cls[c]] - tmax) / Zt;
    double Dmax = -INFINITY;
    for (int64_t x = 0; x < nx; x++) {
        orc_channel_row_bruteforce(n, (uint64_t)x, d, cnt, W);
        double acc = 0.0, dacc = 0.0;
        for (uint64_t c = 1; c < nout; c++) {
            if (W[c] <= 0.0) continue;
            int k = 63 - __builtin_clzll(c);
            double lr = log2(W[c] / q[c]);
            acc += W[c] * lr;
            dacc += W[c] * ((double)(n - k) / d - (double)k / (1.0 - d)) * lr;
        }
        Dx[x] = acc;
        dD[x] = dacc;
        if (acc > Dmax) Dmax = acc;
    }
    double Zx = 0.0;
    for (int64_t x = 0; x < nx; x++) Zx += exp2((Dx[x] - Dmax) / tau);
    double F = Dmax + tau * log2(Zx);
    double gd = 0.0;
    for (int64_t x = 0; x < nx; x++) {
        double pi = exp2((Dx[x] - Dmax) / tau) / Zx;
        gd += pi * dD[x];
        if (grad_theta) {
            orc_channel_row_bruteforce(n, (uint64_t)x, d, cnt, W);
            for (uint64_t c = 1; c < nout; c++) g[c] -= pi * W[c];
        }
    }
    if (grad_theta) {
        for (int64_t r = 0; r < ncls; r++) grad_theta[r] = 0.0;
        for (uint64_t c = 1; c < nout; c++) grad_theta[cls[c]] += g[c] + q[c];
        for (int64_t r = 0; r < ncls; r++) grad_theta[r] /= log(2.0);
    }
    if (grad_d) *grad_d = gd;
    free(q); free(g); free(Dx); free(dD); free(cnt); free(W);
    return F;
}

/* ---------------------------------------------------------------------------
 * O2: the factorised sweep in plain FP64 (a second CPU implementation of the
 * output marginal and of the divergence's cross term, written from the
 * prefix recursion of the channel rule of Sec. 2.2; no blocking, no fusion).
 * It is the same-algorithm CPU baseline and the full-iteration reference at
 * sizes where the definitions above take too long; it is pinned against them
 * (q_full, D_full, embed_count) by the -m "not gpu" tests.
 *
 * Read x = r s left to right, r the first i symbols, s the other n - i.
 * W_i(u|r) is the probability that the first i symbols leave u; appending b
 * to r either deletes b (weight a) or keeps it, matched to u's last symbol
 * (weight c):  W_{i+1}(u | r b) = a W_i(u|r) + c [u ends in b] W_i(u^-|r),
 * with u^- = u without its last symbol.  For BDC_d, (a, c) = (d, 1 - d);
 * with (a, c) = (1, 1) the recursion counts embeddings (Count(u, r)).  The
 * partial sums F_i(u, s) = sum_r p(r s) W_i(u|r) then obey
 *     F_{i+1}(u, s') = a (F_i(u, 0 s') + F_i(u, 1 s')) + c F_i(u^-, u_last s')
 * from F_0(empty, x) = p(x) to F_n(u, empty) = sum_x p(x) W(u|x) = q(u).
 * Level i stores F_i(u, s) at index (code(u) << (n - i)) | s, code(u) =
 * (1 << |u|) | u, so every level lives in [1, 2^(n+1)).
 * The transpose runs the other way: from Gbar_n(u) = L(u),
 *     Gbar_i(v, b s') = a Gbar_{i+1}(v, s') + c Gbar_{i+1}(v b, s'),
 * and Gbar_0(empty, x) = sum_y W(y|x) L(y).
 * ------------------------------------------------------------------------- */
static int bitlen_u64(uint64_t v) { return v ? 64 - __builtin_clzll(v) : 0; }

/* q[c] = sum_x p(x) W(y|x) over all codes (slot 0 = 0). */
void orc_sweep_forward(int n, double a, double c, const double *p, double *q) {
    uint64_t M = 1ull << (n + 1);
    double *cur = (double *)calloc(M, sizeof(double));
    double *nxt = (double *)calloc(M, sizeof(double));
    for (uint64_t x = 0; x < (1ull << n); x++) cur[(1ull << n) | x] = p[x];
    for (int i = 0; i < n; i++) {
        int rest = n - i - 1; /* length of s' */
        uint64_t ncodes = 1ull << (i + 2); /* u of length 0 .. i+1 */
        memset(nxt, 0, M * sizeof(double));
#pragma omp parallel for schedule(static)
        for (int64_t cu = 1; cu < (int64_t)ncodes; cu++) {
            int k = bitlen_u64((uint64_t)cu) - 1;
            for (uint64_t s = 0; s < (1ull << rest); s++) {
                double v = 0.0;
                if (k <= i) {
                    uint64_t base = ((uint64_t)cu << (rest + 1)) | s;
                    v += a * (cur[base] + cur[base | (1ull << rest)]);
                }
                if (k >= 1) {
                    uint64_t b = (uint64_t)cu & 1u, cp = (uint64_t)cu >> 1;
                    v += c * cur[(cp << (rest + 1)) | (b << rest) | s];
                }
                nxt[((uint64_t)cu << rest) | s] = v;
            }
        }
        double *t = cur; cur = nxt; nxt = t;
    }
    memcpy(q, cur, M * sizeof(double));
    q[0] = 0.0;
    free(cur);
    free(nxt);
}

/* G[x] = sum_y W(y|x) L[code(y)] for every x (L indexed by code, slot 0
 * ignored). */
void orc_sweep_adjoint(int n, double a, double c, const double *L, double *G) {
    uint64_t M = 1ull << (n + 1);
    double *cur = (double *)calloc(M, sizeof(double));
    double *nxt = (double *)calloc(M, sizeof(double));
    memcpy(cur, L, M * sizeof(double));
    cur[0] = 0.0;
    for (int i = n - 1; i >= 0; i--) {
        int rest = n - i - 1;
        uint64_t nv = 1ull << (i + 1); /* v of length 0 .. i */
        memset(nxt, 0, M * sizeof(double));
#pragma omp parallel for schedule(static)
        for (int64_t cv = 1; cv < (int64_t)nv; cv++) {
            for (uint64_t b = 0; b < 2; b++)
                for (uint64_t s = 0; s < (1ull << rest); s++) {
                    double v = a * cur[((uint64_t)cv << rest) | s] + c * cur[((((uint64_t)cv << 1) | b) << rest) | s];
                    nxt[((uint64_t)cv << (rest + 1)) | (b << rest) | s] = v;
                }
        }
        double *t = cur; cur = nxt; nxt = t;
    }
    for (uint64_t x = 0; x < (1ull << n); x++) G[x] = cur[(1ull << n) | x];
    free(cur);
    free(nxt);
}

/* S_k(x) = sum over distinct length-k subsequences y of x of
 * Count(y,x) log2 Count(y,x), for a list of inputs (OpenMP over the list);
 * S is [count][n+1]. */
void orc_subseq_S_list(int n, const uint64_t *xs, int64_t count, double *S) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < count; i++) {
        uint64_t N[ORC_MAXN + 1], sc[ORC_MAXN + 1];
        orc_subseq_stats(n, xs[i], N, S + (size_t)i * (n + 1), sc);
    }
}
