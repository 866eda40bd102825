/*
 * FP64 CPU oracle for the FastSimilarityGraph hot path -- TEST INFRASTRUCTURE.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
 * It shares nothing with the CUDA library; see fsg_oracle.c for what each
 * function follows in the paper.
 *
 * Points X are [n][d] float32 row-major, indexed by ORIGINAL point index.
 * perm (may be NULL = identity) maps tree position p -> original index.
 * Every function returning int returns 0 on success, < 0 on bad arguments.
 */
#ifndef FSG_ORACLE_H
#define FSG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_TWO_SIGMA_SQ = 0, ORA_SIGMA_SQ = 1 };
enum { ORA_SELF_EXCLUDE = 0, ORA_SELF_INCLUDE = 1 };
enum { ORA_EDGES_SET = 0, ORA_EDGES_MULTI = 1 };
/* kernel family (Sec. 2.1): the exponent is -scale times ||.||_2^2, ||.||_1 or ||.||_2 */
enum { ORA_GAUSSIAN = 0, ORA_LAPLACIAN = 1, ORA_EXPONENTIAL = 2 };

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t ora_draw_u32(uint64_t seed, uint32_t i, uint32_t l, uint32_t level);
double ora_uniform(uint64_t seed, uint32_t i, uint32_t l, uint32_t level);

double ora_gamma(double sigma, int scale_conv);
/* the scale of the family: gamma for the Gaussian, 1/sigma for the others */
double ora_scale(double sigma, int scale_conv, int family);
double ora_kernel(const float* a, const float* b, int d, double gamma, int family);
int64_t ora_split(int64_t lo, int64_t hi);
double ora_kde(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family,
               int self_mode, int64_t i, int64_t lo, int64_t hi);
int ora_num_threads(int requested);

int ora_degrees(const float* X, int64_t n, int d, double gamma, int family, int self_mode,
                const int64_t* queries, int64_t nq, double* deg, int nthreads);

/* samples[q][l]: original index of the sampled neighbour of queries[q]
 * (queries NULL = all points), -1 if the query has zero degree.
 * margin[q][l] (optional): min over the descent's decisions of |u - ratio|.
 * levels[q][l] (optional): number of decisions taken. */
int ora_sample(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family, int self_mode,
               int L, uint64_t seed, const int64_t* queries, int64_t nq,
               int64_t* samples, double* margin, int32_t* levels, int nthreads);

double ora_path_prob(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family,
                     int self_mode, int64_t i, int64_t p);

int ora_weights(const float* X, int64_t n, int d, double gamma, int family, int L, const double* deg,
                int64_t m, const int64_t* src, const int64_t* dst, double* k_out, double* w_out);

int ora_build_graph(const float* X, int64_t n, int d, const int64_t* perm, double gamma, int family,
                    int self_mode, int L, uint64_t seed, int edge_mode,
                    int64_t* src, int64_t* dst, double* w, int64_t cap, int64_t* m_out,
                    double* deg_out, int64_t* samples_out, int64_t* n_self_out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
