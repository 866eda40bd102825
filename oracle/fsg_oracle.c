/*
 * FP64 CPU oracle for the FastSimilarityGraph hot path
 * (Macgregor & Sun, "Fast Approximation of Similarity Graphs with Kernel
 * Density Estimation", NeurIPS 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
 * restatement of what the method computes.  It is used by the tests, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline leg, and by nothing
 * else.  It shares no code, header, table or constant with the CUDA library
 * under paper_2310_13870_gb300/csrc; neither side includes the other.
 *
 * What it computes (paper section / equation / algorithm in brackets):
 *   - Gaussian kernel k(x_i,x_j) = exp(-gamma * ||x_i - x_j||^2)   [Sec. 2.1]
 *     with gamma = 1/(2 sigma^2) (default) or 1/sigma^2 (the form printed in
 *     Sec. 2.1); all arithmetic in FP64 with direct coordinate differences.
 *   - the two other kernels Sec. 2.1 names: Laplacian exp(-c ||x_i - x_j||_1)
 *     and exponential exp(-c ||x_i - x_j||_2), c = 1/sigma (a reading: the
 *     paper gives the norm in the exponent, not the scale).
 *   - KDE over a contiguous range of tree positions, g_[a,b)(y_i)  [Eq. 1]
 *     with Neumaier-compensated summation.
 *   - The recursive halving descent of Algorithm 1 / Sec. 4.1: the left half
 *     holds floor(|X|/2) points; at every level both halves' KDEs are
 *     computed afresh and the query moves left iff u < g_left/(g_left+g_right).
 *   - Degrees g_[1,n](x_i)                                       [Algorithm 2]
 *   - Re-weighting w = k/p_hat, p_hat = p_i + p_j - p_i p_j,
 *     p_i = min(L k / g_[1,n](x_i), 1)                     [Eq. 2, Algorithm 2]
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
 *     numbers: as easy as 1, 2, 3"), written from that paper's definition.
 *
 * Readings where the paper is silent (the project's design notes list each):
 *   - self term: EXCLUDE (default) omits j == i from every sum, matching the
 *     fully connected graph of Sec. 2.1 which has no self loops; INCLUDE keeps
 *     it (k(i,i) = 1) as literally written in Algorithm 1;
 *   - draw for (seed, point i, sample l, level lev): one Philox4x32-10 call with
 *     counter (i, l, lev / 4, 0) and key (seed low 32 bits, seed high 32 bits);
 *     output word (lev % 4) divided by 2^32 is u in [0,1);
 *   - comparison: strict u < ratio (Algorithm 1 prints <=; the two differ on a
 *     set of measure zero and strict never enters a zero-mass half);
 *   - if a query's degree is 0 it has no samples (index -1).
 */
#include "fsg_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al. (SC'11), Sec. 3/4:     */
/* each round multiplies words 0 and 2 by the two round multipliers, and the */
/* high halves are xored with the other words and the key; the key is bumped */
/* by the two Weyl constants between rounds.                                 */
/* ------------------------------------------------------------------------ */
#define ORA_PHILOX_M0 0xD2511F53u
#define ORA_PHILOX_M1 0xCD9E8D57u
#define ORA_PHILOX_W0 0x9E3779B9u
#define ORA_PHILOX_W1 0xBB67AE85u

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORA_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORA_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += ORA_PHILOX_W0; k1 += ORA_PHILOX_W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint32_t ora_draw_u32(uint64_t seed, uint32_t i, uint32_t l, uint32_t level) {
    uint32_t ctr[4] = {i, l, level >> 2, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    ora_philox4x32_10(ctr, key, out);
    return out[level & 3u];
}

double ora_uniform(uint64_t seed, uint32_t i, uint32_t l, uint32_t level) {
    return (double)ora_draw_u32(seed, i, l, level) * 0x1p-32;
}

/* ------------------------------------------------------------------------ */
/* Kernel function (Sec. 2.1).                                               */
/* ------------------------------------------------------------------------ */
double ora_gamma(double sigma, int scale_conv) {
    if (scale_conv == ORA_SIGMA_SQ) return 1.0 / (sigma * sigma);
    return 1.0 / (2.0 * sigma * sigma);
}

double ora_scale(double sigma, int scale_conv, int family) {
    if (family != ORA_GAUSSIAN) return 1.0 / sigma;
    return ora_gamma(sigma, scale_conv);
}

/* k(a, b) of the family: the exponent is -scale times the squared Euclidean
 * distance (Gaussian), the l1 distance (Laplacian) or the Euclidean distance
 * (exponential). */
double ora_kernel(const float* a, const float* b, int d, double gamma, int family) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double diff = (double)a[t] - (double)b[t];
        if (family == ORA_LAPLACIAN) s += fabs(diff);
        else s += diff * diff;
    }
    if (family == ORA_EXPONENTIAL) s = sqrt(s);
    return exp(-gamma * s);
}

/* ------------------------------------------------------------------------ */
/* Tree: node [lo,hi) of size >= 2 splits at lo + floor((hi-lo)/2), so the    */
/* left half holds floor(|X|/2) points (Sec. 4.1).                           */
/* ------------------------------------------------------------------------ */
int64_t ora_split(int64_t lo, int64_t hi) { return lo + (hi - lo) / 2; }

/* KDE of query point i (original index) over tree positions [lo,hi) (Eq. 1). */
double ora_kde(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family,
               int self_mode, int64_t i, int64_t lo, int64_t hi) {
    (void)n;
    const float* xi = X + (size_t)i * (size_t)d;
    double sum = 0.0, comp = 0.0; /* Neumaier compensated sum */
    for (int64_t p = lo; p < hi; ++p) {
        int64_t j = perm ? perm[p] : p;
        if (j == i && self_mode == ORA_SELF_EXCLUDE) continue;
        double v = ora_kernel(xi, X + (size_t)j * (size_t)d, d, gamma, family);
        double t = sum + v;
        if (fabs(sum) >= fabs(v)) comp += (sum - t) + v;
        else comp += (v - t) + sum;
        sum = t;
    }
    return sum + comp;
}

/* ------------------------------------------------------------------------ */
/* Threading helper: run fn(ctx, q) for q in [0, nq) on nthreads threads.    */
/* ------------------------------------------------------------------------ */
typedef void (*ora_task_fn)(void* ctx, int64_t q);
typedef struct { ora_task_fn fn; void* ctx; int64_t nq; int64_t next; pthread_mutex_t mu; } ora_pool;

static void* ora_worker(void* arg) {
    ora_pool* p = (ora_pool*)arg;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t q = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (q >= p->nq) break;
        p->fn(p->ctx, q);
    }
    return NULL;
}

int ora_num_threads(int requested) {
    if (requested > 0) return requested;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

static void ora_parallel_for(int64_t nq, int nthreads, ora_task_fn fn, void* ctx) {
    int nt = ora_num_threads(nthreads);
    if (nt > 256) nt = 256;
    if ((int64_t)nt > nq) nt = (int)(nq > 0 ? nq : 1);
    ora_pool pool;
    pool.fn = fn; pool.ctx = ctx; pool.nq = nq; pool.next = 0;
    pthread_mutex_init(&pool.mu, NULL);
    if (nt <= 1) {
        ora_worker(&pool);
    } else {
        pthread_t th[256];
        for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, ora_worker, &pool);
        for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    }
    pthread_mutex_destroy(&pool.mu);
}

/* ------------------------------------------------------------------------ */
/* Degrees g_[1,n](x_i) (Algorithm 2).                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const float* X; int64_t n; int d; double gamma; int family; int self_mode;
    const int64_t* queries; double* deg;
} ora_deg_ctx;

static void ora_deg_task(void* c, int64_t q) {
    ora_deg_ctx* x = (ora_deg_ctx*)c;
    int64_t i = x->queries ? x->queries[q] : q;
    x->deg[q] = ora_kde(x->X, x->n, x->d, NULL, x->gamma, x->family, x->self_mode, i, 0, x->n);
}

int ora_degrees(const float* X, int64_t n, int d, double gamma, int family, int self_mode,
                const int64_t* queries, int64_t nq, double* deg, int nthreads) {
    if (!X || n < 1 || d < 1 || !deg || !(gamma > 0)) return -1;
    ora_deg_ctx c = {X, n, d, gamma, family, self_mode, queries, deg};
    ora_parallel_for(nq, nthreads, ora_deg_task, &c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The descent of Algorithm 1 for one query point and L samples.             */
/* Node KDEs are memoised per query (the same (i, node) value is reused by    */
/* every sample passing through that node); every value is the fresh Eq. 1    */
/* sum over the node range, as in Algorithm 1.                                */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t lo, hi; double g; } ora_memo_entry;
typedef struct { ora_memo_entry* e; int64_t len, cap; } ora_memo;

static double ora_memo_kde(ora_memo* m, const float* X, int64_t n, int d, const int64_t* perm,
                           double gamma, int family, int self_mode, int64_t i, int64_t lo, int64_t hi) {
    for (int64_t t = 0; t < m->len; ++t)
        if (m->e[t].lo == lo && m->e[t].hi == hi) return m->e[t].g;
    double g = ora_kde(X, n, d, perm, gamma, family, self_mode, i, lo, hi);
    if (m->len == m->cap) {
        m->cap = m->cap ? 2 * m->cap : 256;
        m->e = (ora_memo_entry*)realloc(m->e, (size_t)m->cap * sizeof(ora_memo_entry));
    }
    m->e[m->len].lo = lo; m->e[m->len].hi = hi; m->e[m->len].g = g; m->len++;
    return g;
}

typedef struct {
    const float* X; int64_t n; int d; const int64_t* perm;
    double gamma; int family; int self_mode; int L; uint64_t seed;
    const int64_t* queries; int64_t* samples; double* margin; int32_t* levels;
} ora_sample_ctx;

static void ora_sample_task(void* c, int64_t q) {
    ora_sample_ctx* x = (ora_sample_ctx*)c;
    int64_t i = x->queries ? x->queries[q] : q;
    ora_memo memo = {NULL, 0, 0};
    double root = ora_memo_kde(&memo, x->X, x->n, x->d, x->perm, x->gamma, x->family, x->self_mode, i, 0, x->n);
    for (int l = 0; l < x->L; ++l) {
        size_t o = (size_t)q * (size_t)x->L + (size_t)l;
        double mrg = INFINITY;
        int32_t nlev = 0;
        if (!(root > 0.0)) {            /* no mass: no sample */
            x->samples[o] = -1;
            if (x->margin) x->margin[o] = mrg;
            if (x->levels) x->levels[o] = 0;
            continue;
        }
        int64_t lo = 0, hi = x->n;
        uint32_t lev = 0;
        while (hi - lo > 1) {
            int64_t mid = ora_split(lo, hi);
            double gl = ora_memo_kde(&memo, x->X, x->n, x->d, x->perm, x->gamma, x->family, x->self_mode, i, lo, mid);
            double gr = ora_memo_kde(&memo, x->X, x->n, x->d, x->perm, x->gamma, x->family, x->self_mode, i, mid, hi);
            double r = gl / (gl + gr);
            double u = ora_uniform(x->seed, (uint32_t)i, (uint32_t)l, lev);
            double dm = fabs(u - r);
            if (dm < mrg) mrg = dm;
            if (u < r) hi = mid; else lo = mid;
            ++lev; ++nlev;
        }
        x->samples[o] = x->perm ? x->perm[lo] : lo;
        if (x->margin) x->margin[o] = mrg;
        if (x->levels) x->levels[o] = nlev;
    }
    free(memo.e);
}

int ora_sample(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family, int self_mode,
               int L, uint64_t seed, const int64_t* queries, int64_t nq,
               int64_t* samples, double* margin, int32_t* levels, int nthreads) {
    if (!X || n < 1 || d < 1 || L < 1 || !samples || !(gamma > 0)) return -1;
    ora_sample_ctx c = {X, n, d, perm, gamma, family, self_mode, L, seed, queries, samples, margin, levels};
    ora_parallel_for(nq, nthreads, ora_sample_task, &c);
    return 0;
}

/* Probability that the descent of query i ends at tree position p: the      */
/* product, over the levels on the path to p, of the chosen half's share.     */
double ora_path_prob(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family,
                     int self_mode, int64_t i, int64_t p) {
    int64_t lo = 0, hi = n;
    double prob = 1.0;
    while (hi - lo > 1) {
        int64_t mid = ora_split(lo, hi);
        double gl = ora_kde(X, n, d, perm, gamma, family, self_mode, i, lo, mid);
        double gr = ora_kde(X, n, d, perm, gamma, family, self_mode, i, mid, hi);
        if (gl + gr <= 0.0) return 0.0;
        if (p < mid) { prob *= gl / (gl + gr); hi = mid; }
        else { prob *= gr / (gl + gr); lo = mid; }
    }
    return prob;
}

/* ------------------------------------------------------------------------ */
/* Re-weighting of Algorithm 2 / Eq. 2 for given sampled pairs.              */
/* deg is indexed by original point index and holds g_[1,n] for every point  */
/* that appears in src or dst.                                               */
/* ------------------------------------------------------------------------ */
int ora_weights(const float* X, int64_t n, int d, double gamma, int family, int L, const double* deg,
                int64_t m, const int64_t* src, const int64_t* dst, double* k_out, double* w_out) {
    (void)n;
    if (!X || !deg || (m > 0 && (!src || !dst || !w_out))) return -1;
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double k = ora_kernel(X + (size_t)i * (size_t)d, X + (size_t)j * (size_t)d, d, gamma, family);
        double pi = fmin((double)L * k / deg[i], 1.0);
        double pj = fmin((double)L * k / deg[j], 1.0);
        double ph = pi + pj - pi * pj;
        if (k_out) k_out[e] = k;
        w_out[e] = k / ph;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole of Algorithm 2 for every point (small n): L samples per point,       */
/* degrees, re-weighting, and the edge list.                                  */
/*   edge_mode SET  : one edge per unordered pair {i,j}, i != j, sampled from */
/*                    either side (the set union of Algorithm 2);           */
/*   edge_mode MULTI: one edge per sample with j != i (i = source).           */
/* SET edges are written with src < dst, sorted by (src, dst).                */
/* ------------------------------------------------------------------------ */
static int ora_cmp_pair(const void* a, const void* b) {
    const int64_t* x = (const int64_t*)a; const int64_t* y = (const int64_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

int ora_build_graph(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family,
                    int self_mode, int L, uint64_t seed, int edge_mode,
                    int64_t* src, int64_t* dst, double* w, int64_t cap, int64_t* m_out,
                    double* deg_out, int64_t* samples_out, int64_t* n_self_out, int nthreads) {
    if (!X || n < 1 || d < 1 || L < 1 || !src || !dst || !w || !m_out || !(gamma > 0)) return -1;
    double* deg = (double*)malloc((size_t)n * sizeof(double));
    int64_t* smp = (int64_t*)malloc((size_t)n * (size_t)L * sizeof(int64_t));
    if (!deg || !smp) { free(deg); free(smp); return -2; }
    ora_degrees(X, n, d, gamma, family, self_mode, NULL, n, deg, nthreads);
    ora_sample(X, n, d, perm, gamma, family, self_mode, L, seed, NULL, n, smp, NULL, NULL, nthreads);
    int64_t cnt = 0, nself = 0;
    int64_t* pairs = (int64_t*)malloc((size_t)n * (size_t)L * 2 * sizeof(int64_t));
    if (!pairs) { free(deg); free(smp); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        for (int l = 0; l < L; ++l) {
            int64_t j = smp[(size_t)i * (size_t)L + (size_t)l];
            if (j < 0) continue;
            if (j == i) { ++nself; continue; }
            if (edge_mode == ORA_EDGES_SET) {
                pairs[2 * cnt] = i < j ? i : j;
                pairs[2 * cnt + 1] = i < j ? j : i;
            } else {
                pairs[2 * cnt] = i;
                pairs[2 * cnt + 1] = j;
            }
            ++cnt;
        }
    }
    if (edge_mode == ORA_EDGES_SET) {
        qsort(pairs, (size_t)cnt, 2 * sizeof(int64_t), ora_cmp_pair);
        int64_t u = 0;
        for (int64_t e = 0; e < cnt; ++e) {
            if (u > 0 && pairs[2 * (u - 1)] == pairs[2 * e] && pairs[2 * (u - 1) + 1] == pairs[2 * e + 1])
                continue;
            pairs[2 * u] = pairs[2 * e]; pairs[2 * u + 1] = pairs[2 * e + 1]; ++u;
        }
        cnt = u;
    }
    int rc = 0;
    if (cnt > cap) {
        rc = -3;
    } else {
        for (int64_t e = 0; e < cnt; ++e) { src[e] = pairs[2 * e]; dst[e] = pairs[2 * e + 1]; }
        ora_weights(X, n, d, gamma, family, L, deg, cnt, src, dst, NULL, w);
    }
    *m_out = cnt;
    if (deg_out) memcpy(deg_out, deg, (size_t)n * sizeof(double));
    if (samples_out) memcpy(samples_out, smp, (size_t)n * (size_t)L * sizeof(int64_t));
    if (n_self_out) *n_self_out = nself;
    free(pairs); free(deg); free(smp);
    return rc;
}
