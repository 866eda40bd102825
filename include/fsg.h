/*
 * fsg.h -- C ABI of the GB300 (sm_103a) FastSimilarityGraph hot path.
 *
 * The library computes, on one GPU, the data-parallel core of the algorithm of
 * Macgregor & Sun, "Fast Approximation of Similarity Graphs with Kernel
 * Density Estimation" (NeurIPS 2023):
 *   - Gaussian kernel k(x_i,x_j) = exp(-gamma ||x_i-x_j||^2), and the
 *     Laplacian and exponential kernels of the same section       (Sec. 2.1)
 *   - KDE sums g_[a,b](y_i) = sum_{j=a..b} k(y_i,x_j), computed exactly, or
 *     within a stated relative bound (approximate KDE, fsg_params.kde_eps)
 *                                                                      (Eq. 1)
 *   - degrees g_[1,n](x_i)                                          (Algorithm 2)
 *   - L neighbour samples per point by recursive halving of the point set,
 *     moving left with probability g_left/(g_left+g_right)   (Algorithm 1, Sec. 4.1)
 *   - the re-weighted sparse edge list w = k / p_hat                 (Eq. 2, Algorithm 2)
 *
 * Conventions shared by every call
 *   - Every function returns an int status: FSG_OK (0) or one of FSG_ERR_*.
 *     fsg_error_string() describes a status.  Invalid arguments are refused
 *     before anything is enqueued.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued asynchronously on that stream; outputs are
 *     valid once the stream reaches that point.  Device-side faults of the
 *     library's own checks (a bounded wait that ran out) are recorded in a
 *     per-tree status word that fsg_sync() reads and returns.
 *   - Device pointers (d_*) are CUDA global-memory addresses on the current
 *     device; host pointers (h_*) are ordinary host memory (pinned memory makes
 *     the copies of the host entry point asynchronous).
 *   - Points are float32, row-major [n][d], indexed by ORIGINAL point index.
 *     Outputs indexed by point use original indices as well.
 *   - The caller owns every buffer it passes; the library never frees them.
 *     fsg_tree objects are owned by the library and released by fsg_free_tree.
 *   - No host fallback exists: without a usable sm_103a GPU every compute call
 *     fails with FSG_ERR_CUDA.
 */
#ifndef FSG_H
#define FSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FSG_OK 0
#define FSG_ERR_INVALID_ARG 1   /* bad size, NULL pointer, sigma <= 0, ...      */
#define FSG_ERR_OOM 2           /* a device allocation failed                     */
#define FSG_ERR_CUDA 3          /* a CUDA runtime call failed                     */
#define FSG_ERR_TIMEOUT 4       /* a bounded device wait ran out                  */
#define FSG_ERR_UNSUPPORTED 5   /* option not implemented for these sizes        */
#define FSG_ERR_BUSY 6          /* server: no slot or budget for the request      */
#define FSG_ERR_CAPACITY 7      /* an output buffer is too small                  */
#define FSG_ERR_SCRATCH 8       /* problem too large for fsg_degrees_noalloc      */
#define FSG_ERR_CANCELLED 9     /* server: the request was cancelled              */
#define FSG_ERR_BOUNDS 10       /* bounds-checking build: an index check failed   */

/* ---- option values ----------------------------------------------------- */
/* Bandwidth convention: gamma = 1/(2 sigma^2) (default) or 1/sigma^2, the form
 * printed in Sec. 2.1. */
#define FSG_TWO_SIGMA_SQ 0
#define FSG_SIGMA_SQ 1
/* Self term: EXCLUDE omits j == i from every KDE sum (the fully connected
 * graph of Sec. 2.1 has no self loops, so g_[1,n](x_i) equals the degree);
 * INCLUDE keeps k(i,i) = 1 as Algorithm 1 literally sums over all of X. */
#define FSG_SELF_EXCLUDE 0
#define FSG_SELF_INCLUDE 1
/* Arithmetic of the kernel evaluations. */
#define FSG_PREC_AUTO 0         /* FP32 for d <= 16; tensor-core form for large d */
#define FSG_PREC_FP32 1         /* FP32 direct differences + ex2 on every d       */
#define FSG_PREC_SPLIT_BF16 2   /* FP32 data as 3-part BF16, six tcgen05        */
                                /* products per coordinate, FP32 accumulate.     */
                                /* d <= 64: tiles centred at their mean; use     */
                                /* with fsg_spatial_order (the leaf phase too    */
                                /* for d in 17..64; FP32 for d <= 16); the only  */
                                /* form with the approximate bin pass            */
                                /* (fsg_params.kde_eps).  d > 64: uncentred      */
                                /* ||x||^2 + ||y||^2 - 2 x.y (norms from FP64    */
                                /* sums) on the tensor-core bin pass and leaf    */
                                /* kernel; a value is within relative            */
                                /* gamma (6 dpad / 16 + 1) 2^-22 (|x|^2 + |y|^2) */
                                /* + 2^-22 (dpad = d rounded up to 64)           */
#define FSG_PREC_EXACT_INT 3    /* tcgen05 BF16 on data that are k/255 exactly    */
/* Kernel family (Sec. 2.1): the exponent of k(x, y) is minus the scale times
 * the squared Euclidean distance (Gaussian, scale gamma of scale_conv), the
 * l1 distance (Laplacian, scale 1/sigma) or the Euclidean distance
 * (exponential, scale 1/sigma).  The Laplacian and exponential kernels run on
 * the fused schedule's FP32 paths: for d <= 16 with bins of 65..128 points
 * (the default tree for most n from 65 to 262,144 at d <= 16), and for any
 * d > 16.  The exponential also runs on the exact 8-bit tensor-core path
 * (FSG_PREC_EXACT_INT, or AUTO on 8-bit data with d >= 64: the square root of
 * the exact integer squared distance); for the Laplacian AUTO means FP32.
 * Elsewhere (levelwise schedules, the split precision, fsg_params.resolve,
 * weight_f64) FSG_ERR_UNSUPPORTED. */
#define FSG_KERNEL_GAUSSIAN 0
#define FSG_KERNEL_LAPLACIAN 1
#define FSG_KERNEL_EXPONENTIAL 2
/* Edge semantics of Algorithm 2's set union. */
#define FSG_EDGES_SET 0         /* one edge per unordered pair {i,j} sampled      */
#define FSG_EDGES_MULTI 1       /* one edge per (non-self) sample                 */
/* Sampling schedule. */
#define FSG_SCHED_FUSED 0       /* top levels from one bin pass, then leaf finish */
#define FSG_SCHED_LEVELWISE 1   /* literal per-level KDE of both halves           */
#define FSG_SCHED_CARRIED 2     /* per level the left half only, g_R = g - g_L    */
                                /* carried from the parent (decisions flagged    */
                                /* within the carried error bound)               */

typedef struct fsg_tree fsg_tree; /* opaque */

/* Tree order (fsg_tree_opts.order). */
#define FSG_ORDER_IDENTITY 0    /* position p holds point p (or d_perm[p])         */
#define FSG_ORDER_SPATIAL 1     /* computed on the GPU from the points, at build   */
                                /* and at every fsg_tree_update: each node above   */
                                /* 32 points split at the tree's midpoint along    */
                                /* its widest coordinate (to one of 256 buckets)   */

typedef struct {
    /* Device int32 [n]: tree position p -> original point index (a
     * permutation), or NULL for the identity order.  Copied at build time. */
    const int32_t* d_perm;
    /* Largest node handled by the leaf-finish kernel (power of two in
     * [64, 1024]); 0 selects 128 (raised automatically for very large n).
     * Smaller values run more levels through the bin pass. */
    int32_t leaf_max;
    /* FSG_ORDER_IDENTITY | FSG_ORDER_SPATIAL (then d_perm must be NULL).  The
     * order changes which points share a node, not the sampling distribution
     * (Sec. 4.1); the split form and the approximate bin pass rely on compact
     * nodes. */
    int32_t order;
    int32_t reserved[4];
} fsg_tree_opts;

typedef struct {
    double sigma;          /* kernel bandwidth, > 0 and finite                 */
    int32_t scale_conv;    /* FSG_TWO_SIGMA_SQ | FSG_SIGMA_SQ                   */
    int32_t self_mode;     /* FSG_SELF_EXCLUDE | FSG_SELF_INCLUDE               */
    int32_t precision;     /* FSG_PREC_*                                        */
    int32_t schedule;      /* FSG_SCHED_*                                       */
    /* Relative error bound eps of the GPU's KDE sums used to flag near-threshold
     * decisions: a level is flagged when |u - r| < 2 eps r (1-r) + 2^-22 with
     * r = g_left/(g_left+g_right).  0 selects 2^-13, or 2^-10 for
     * FSG_PREC_SPLIT_BF16 (whose sums carry up to about 4e-4 relative error
     * from the tensor cores' FP32 accumulation). */
    float flag_eps;
    /* Approximate KDE (tree-pruned bin pass), 0 = exact.  With kde_eps in
     * (0, 0.5] the bin pass skips every point tile whose largest possible
     * contribution to a query tile's sums, count * exp(-gamma gap^2) with gap
     * the distance between the two tiles' bounding boxes, is at most
     * kde_eps / T of a lower bound of those queries' degrees (their exact sums
     * over their own tile; T = the point tiles of one query's sweep), so
     * every degree and every node sum above the bins loses at most
     * kde_eps * degree of its mass (a one-sided error, before rounding).
     * Decisions on those sums are flagged with the extra tolerance
     * kde_eps * degree, so unflagged samples still equal the exact method's.
     * Values inside a bin are not approximated.  FSG_PREC_SPLIT_BF16 with
     * d <= 64 only (FSG_ERR_UNSUPPORTED otherwise); negative, non-finite or > 0.5:
     * FSG_ERR_INVALID_ARG.  The paper's bound for the method is
     * eps <= 1/(6 log n). */
    float kde_eps;
    int32_t kernel;        /* FSG_KERNEL_* (0: Gaussian)                         */
    /* High-precision re-decision of flagged descents (0 = off, 1 = on):
     * after the fused schedule, every sample with a decision inside the flag
     * band is taken again from the root; each such decision is made on sums
     * of kernel values within relative error 2^-20 of the exact ones
     * (double-single squared distances, FP64 accumulation), compared in FP64
     * with the full 32-bit draw (u = word 2^-32), and the levels inside the
     * bin reached are all decided that way.  A sample stays flagged only if a
     * high-precision margin is itself within 2^-20; every other sample
     * equals the exact method's (Algorithm 1).  fsg_stats.n_resolved counts
     * the samples taken again and n_flagged the ones still flagged.
     * Gaussian kernel, FSG_SCHED_FUSED, bins of at most 1024 points;
     * FSG_ERR_UNSUPPORTED otherwise. */
    int32_t resolve;
    /* 1: fsg_build_graph writes d_w as double [cap]: w = k / p_hat (Eq. 2)
     * formed in FP64 from a high-precision k(x_i, x_j) (relative error
     * 2^-20) and the FP32-accumulated degrees; 0: float [cap]. */
    int32_t weight_f64;
    int32_t reserved[1];
} fsg_params;

/* Device-side statistics of one fsg_build_graph call (all int64). */
typedef struct {
    int64_t n_samples;     /* n * L descents run                               */
    int64_t n_flagged;     /* samples with >= 1 near-threshold decision         */
    int64_t n_self;        /* samples that returned the query itself (INCLUDE)  */
    int64_t n_empty;       /* samples of zero-degree queries (index -1)         */
    int64_t n_evals;       /* kernel evaluations executed                        */
    int64_t n_items;       /* distinct (query, node) pairs in the leaf finish   */
    int64_t n_edges;       /* edges written                                     */
    int64_t status;        /* device status word (FSG_OK or FSG_ERR_TIMEOUT)    */
    int64_t n_bin_evals;   /* of n_evals, those of the bin pass (the split pass */
                           /* skips tile pairs whose values are all zero)       */
    int64_t n_resolved;    /* samples re-decided in high precision (resolve)    */
} fsg_stats;

/* Library version string and a description of a status code. */
const char* fsg_version(void);
const char* fsg_error_string(int status);

/*
 * Builds the device-resident tree of n points (Sec. 4.1: the point set is split
 * recursively into a left half of floor(|X|/2) points and a right half).
 *   d_points : device float32 [n][d] row-major, read only during this call.
 *   n        : 1 <= n <= 2^31 - 1;  d : 1 <= d <= 4096.
 *   opts     : may be NULL (identity order, automatic leaf_max).
 * Writes *out.  The tree holds a tree-ordered, padded copy of the points and
 * grows a workspace on first use; fsg_free_tree releases both.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int fsg_build_tree(const float* d_points, int64_t n, int32_t d, const fsg_tree_opts* opts,
                   void* stream, fsg_tree** out);

/*
 * Spatial tree order (host, synchronous): a permutation for
 * fsg_tree_opts.d_perm under which every node of the tree is a compact group
 * of points.  Each node [lo, hi) of tree positions is split where the tree
 * splits it (its left floor(|X|/2) positions, Sec. 4.1) along the coordinate
 * of largest spread among its points, the smaller values going left (ties by
 * original index); nodes of at most `leaf` points keep original-index order.
 * The KDE, the degrees and the sampling distribution do not depend on the
 * order (Eq. 1); sample identities under given Philox draws do, as they do on
 * any permutation.  FSG_PREC_SPLIT_BF16 centres each query tile at its mean,
 * which cancels less when the tile is a compact group.
 *   h_points : host float32 [n][d], finite.   h_perm : host int32 [n] out,
 *   position -> original index.   Deterministic.
 * Errors: INVALID_ARG (null pointer, n or d out of range, leaf < 1, a
 * non-finite coordinate).
 */
int fsg_spatial_order(const float* h_points, int64_t n, int32_t d, int32_t leaf, int32_t* h_perm);

/*
 * The tree's order: d_perm_out[p] = original index of the point at tree
 * position p (device int32 [n], caller-owned), asynchronous on the stream.
 * Lets a caller (or a checker) reproduce the tree of FSG_ORDER_SPATIAL.
 */
int fsg_tree_perm(const fsg_tree* tree, int32_t* d_perm_out, void* stream);
void fsg_free_tree(fsg_tree* tree);

/* Number of points, dimension and depth ceil(log2 n) of a tree. */
int fsg_tree_info(const fsg_tree* tree, int64_t* n, int32_t* d, int32_t* depth);

/*
 * Kernel evaluations k(x_q, x_p) that the bin pass of the fused schedule
 * executes on this tree with these parameters (a diagnostic for roofline
 * accounting; Eq. 1 needs n^2 of them).  The symmetric passes evaluate each
 * pair once off their diagonal blocks: (n^2 + sum_k S_k^2) / 2 for the
 * d <= 16 FP32 pass and the tensor-core pass (also in the split form above
 * d = 64), S_k the point counts of their blocks or chunks of bins, and
 * T (T + 1) / 2 tiles of 128 x 128 for the d > 16 FP32 pass (T = ceil(n /
 * 128)); n^2 for the two-order forms (other bin sizes); for the d <= 64
 * split pass n^2 is an upper bound (it skips tile pairs whose values are
 * all zero in FP32 and counts what it executes in fsg_stats.n_bin_evals).  0 for the levelwise
 * schedules, which count their own evaluations on the device
 * (fsg_stats.n_evals).
 *   evals : host int64, written on success.
 * Errors: INVALID_ARG.
 */
int fsg_bin_pass_evals(const fsg_tree* tree, const fsg_params* params, int64_t* evals);

/*
 * Launch shapes of the fused schedule's kernels; 0 selects the built-in
 * heuristic.  They change how work is split among CTAs, not what is
 * computed: results stay within the stated tolerances, and samples can differ
 * only where a decision is flagged (the grouping of FP32 partial sums of the
 * bin passes depends on sym_bins / tc_bins; leaf_splits changes nothing).
 */
typedef struct {
    int32_t sym_bins;     /* bins per block of the symmetric d <= 16 bin pass   */
    int32_t tc_bins;      /* bins per chunk of the tensor-core bin pass (<= 24; */
                          /* 8..16 in its symmetric form)                      */
    int32_t leaf_splits;  /* CTAs per bin of the leaf finish                   */
    int32_t reserved[5];
} fsg_tuning;

/*
 * Autotuner: times the candidate launch shapes of the bin pass that this tree
 * and these parameters select (symmetric FP32: 4..16 bins per block;
 * tensor-core: 8..24 bins per chunk) and of the leaf finish (the heuristic
 * split count x 1/4 .. 4), each the best of `reps` runs on `stream`, keeps the
 * fastest on the tree and writes it to *out (if not NULL).  The choice is
 * cached per (d, n, L, bin layout, path) for the process: a second call for
 * the same shape reuses it without timing.  Synchronizes `stream`; not for
 * use during CUDA-graph capture.  The paper has no counterpart (launch shapes
 * of this implementation).
 * Errors: INVALID_ARG, OOM, CUDA, UNSUPPORTED.
 */
int fsg_autotune(fsg_tree* tree, const fsg_params* params, int32_t L, uint64_t seed, int32_t reps, fsg_tuning* out,
                 void* stream);

/* Sets (tuning != NULL) and/or reads (out != NULL) the tree's launch shapes.
 * Negative fields are refused with INVALID_ARG. */
int fsg_tree_tuning(fsg_tree* tree, const fsg_tuning* tuning, fsg_tuning* out);

/*
 * Replaces the tree's points by new values of the same shape (n, d) in the
 * same tree order, without allocating (Sec. 4.1's tree is rebuilt in place).
 *   d_points : device float32 [n][d], read only during this call.
 * Errors: INVALID_ARG, CUDA.
 */
int fsg_tree_update(fsg_tree* tree, const float* d_points, void* stream);

/*
 * Degrees g_[1,n](x_i) of Algorithm 2 (Eq. 1 over all points) for every point.
 *   d_deg : device float64 [n], indexed by original point index.
 * Errors: INVALID_ARG (params), OOM, CUDA, UNSUPPORTED.
 */
int fsg_degrees(fsg_tree* tree, const fsg_params* params, double* d_deg, void* stream);

/*
 * Degrees without any device allocation.  (The paper has no counterpart:
 * this is a service for callers, computing the same values as fsg_degrees.)
 *
 * Some callers cannot call cudaMalloc: an application whose device memory is
 * owned entirely by its own pool allocator (a framework's caching allocator,
 * a serving runtime that reserves its HBM budget up front) must not have a
 * library allocate behind its back, and latency-critical callers cannot pay
 * for cudaMalloc/cudaFree, which may synchronize the device.  This entry
 * point needs no tree object and no workspace: its scratch (a tree-ordered
 * copy of the points, bin boundaries, per-bin partial sums) lives in one
 * statically sized array in the library's device memory, which every GPU
 * that loads the library holds until the process exits.
 *   d_points : device float32 [n][d] row-major, read only.
 *   d_deg    : device float64 [n], original index order (same values as
 *              fsg_degrees to FP32 accuracy).
 *   Limits   : 1 <= d <= 16, and the scratch (about 270 bytes per point at
 *              d = 16) must fit FSG_NOALLOC_SCRATCH_BYTES; larger problems are
 *              refused with FSG_ERR_SCRATCH before anything is enqueued.
 * The first call on a device looks up that device's address of the array
 * (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture.  Every call, on any stream, shares the one
 * array and leaves its contents behind: calls that overlap on the GPU race
 * and give wrong results, so serialize them (one stream, or events).  Each
 * call clears what it reads before writing it (the status word and the
 * position map) and overwrites every partial sum it uses, so a call does not
 * depend on what an earlier one left.
 * Device-side failure: there is no tree whose status word fsg_sync could
 * read, so when a bounded wait of the bin pass runs out (the condition the
 * other calls report as FSG_ERR_TIMEOUT) every entry of d_deg is set to NaN.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: INVALID_ARG, UNSUPPORTED (d > 16), SCRATCH, CUDA.
 */
#define FSG_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int fsg_degrees_noalloc(const float* d_points, int64_t n, int32_t d, const fsg_params* params, double* d_deg,
                        void* stream);

/*
 * L samples per point by the descent of Algorithm 1 (Sec. 4.1).  The uniform
 * u of (point i, sample l, level lev) is word (lev mod 4) of Philox4x32-10
 * (Salmon et al., SC'11) at counter (i, l, lev/4, 0) with key (seed low 32
 * bits, seed high 32 bits), divided by 2^32; the descent goes left iff
 * u < g_left/(g_left+g_right).
 *   L         : 1..64.
 *   d_samples : device int32 [n][L]: original index of the neighbour, or -1
 *               when the point has zero degree.
 *   d_flags   : device uint8 [n][L] or NULL: bit 0 = some decision was within
 *               the flag tolerance (see fsg_params.flag_eps), bit 1 = some
 *               node had zero FP32 mass.
 * Errors: INVALID_ARG, OOM, CUDA, UNSUPPORTED.
 */
int fsg_sample_edges(fsg_tree* tree, const fsg_params* params, int32_t L, uint64_t seed,
                     int32_t* d_samples, uint8_t* d_flags, void* stream);

/*
 * The whole of Algorithm 2: L samples per point, degrees, and the sparse
 * edge list with weights w(i,j) = k(x_i,x_j) / p_hat(i,j),
 * p_hat = p_i + p_j - p_i p_j, p_i = min(L k / g_[1,n](x_i), 1)    (Eq. 2).
 *   edge_mode  : FSG_EDGES_SET or FSG_EDGES_MULTI.
 *   d_src,d_dst: device int32 [cap] original indices (SET: the point that
 *                sampled the edge first in (point, sample) order is src).
 *   d_w        : device float32 [cap], or float64 [cap] with
 *                params->weight_f64.
 *   cap        : >= n*L (an upper bound of the edge count in either mode).
 *   d_m_out    : device int64, number of edges written.
 *   d_deg, d_samples, d_flags, d_stats : optional device outputs (NULL to
 *                skip): float64 [n], int32 [n][L], uint8 [n][L], fsg_stats.
 * Errors: INVALID_ARG, CAPACITY, OOM, CUDA, UNSUPPORTED.
 */
int fsg_build_graph(fsg_tree* tree, const fsg_params* params, int32_t L, uint64_t seed,
                    int32_t edge_mode, int32_t* d_src, int32_t* d_dst, void* d_w, int64_t cap,
                    int64_t* d_m_out, double* d_deg, int32_t* d_samples, uint8_t* d_flags,
                    fsg_stats* d_stats, void* stream);

/*
 * Algorithm 2 in steps over ranges of query points, for long runs that are
 * checkpointed and resumed (the paper has no counterpart; Sec. 4.1's
 * descents are independent per query given the KDE values and the draws).
 * fsg_graph_begin validates the call exactly as fsg_build_graph does, runs
 * the bin pass for every query and keeps its sums in the tree; each
 * fsg_graph_step samples the queries at tree positions [q_begin, q_end)
 * (tree position = original index under the identity order; fsg_tree_perm
 * gives the map otherwise): degrees, descents, bucketing, leaf finish and,
 * with params->resolve, the re-decision, overwriting that range's sampling
 * state in the tree.  A step reads only the bin sums and its queries' own
 * draws, so steps may come in any order, be repeated (after a failed
 * fsg_sync, say) and be resumed from any position: the device-resident
 * state of the other ranges is the checkpoint, fsg_graph_cursor the first
 * position not yet stepped.  fsg_graph_end forms the edge list and the
 * optional outputs (arguments as in fsg_build_graph) once every position
 * has been stepped.  For any split into steps the results are bit for bit
 * those of fsg_build_graph with the same arguments (with params->resolve:
 * while each call's flagged samples fit the re-decision's batched scratch,
 * max(65,536, n L / 64); beyond it the per-sample fallback sums in another
 * order); statistics count the work done (a repeated step counts twice).
 * Any other call on the tree (fsg_build_graph, fsg_degrees,
 * fsg_tree_update, ...) ends the run.  The steps share the tree's
 * workspace: issue them one after another on one stream, or order them with
 * events (steps that overlap on the GPU race).  Fused schedule only.
 *   q_begin, q_end : 0 <= q_begin < q_end <= n.
 *   cursor         : host int64: smallest position not yet stepped (n when
 *                    every position was).
 * Errors: INVALID_ARG (no run begun, bad range, end before every position
 * was stepped), UNSUPPORTED (levelwise schedules), and those of
 * fsg_build_graph.
 */
int fsg_graph_begin(fsg_tree* tree, const fsg_params* params, int32_t L, uint64_t seed, void* stream);
int fsg_graph_step(fsg_tree* tree, int64_t q_begin, int64_t q_end, void* stream);
int fsg_graph_cursor(const fsg_tree* tree, int64_t* cursor);
int fsg_graph_end(fsg_tree* tree, int32_t edge_mode, int32_t* d_src, int32_t* d_dst, void* d_w, int64_t cap,
                  int64_t* d_m_out, double* d_deg, int32_t* d_samples, uint8_t* d_flags, fsg_stats* d_stats,
                  void* stream);

/*
 * Per-phase timing with CUDA events recorded on the call's stream (not part
 * of the paper's method; used to report kernel durations).
 * fsg_profile(tree, 1) makes later calls record an event at each phase
 * boundary; fsg_profile_read() waits for the last profiled call and writes
 * the duration in milliseconds of each phase into ms[FSG_NUM_PHASES] (0 for
 * phases that did not run) and the total number of the library's kernel
 * launches made on this tree since it was built into *launches.
 */
#define FSG_PHASE_TREE 0        /* tree build / update                         */
#define FSG_PHASE_KDE_BINS 1    /* bin pass: every query against every point   */
#define FSG_PHASE_DESCEND_TOP 2 /* degrees and the top s0 levels               */
#define FSG_PHASE_BUCKET 3      /* grouping of (query, node) items per node    */
#define FSG_PHASE_LEAF 4        /* leaf finish: remaining levels and weights   */
#define FSG_PHASE_EDGES 5       /* edge list                                   */
#define FSG_PHASE_OUTPUTS 6     /* per-sample outputs and statistics           */
#define FSG_PHASE_RESOLVE 7     /* high-precision re-decision (params.resolve) */
#define FSG_NUM_PHASES 8
int fsg_profile(fsg_tree* tree, int enable);
int fsg_profile_read(fsg_tree* tree, float* ms, int64_t* launches);

/*
 * Batched graph construction over many independent point sets (for example
 * the pixel features of many images): every set runs the whole of
 * Algorithm 2 with its own parameters.  fsg_batch_create builds one tree per
 * set (allocating); fsg_batch_run refreshes every tree from its d_points and
 * enqueues every set's graph build on `streams` internal streams forked from
 * (and joined back into) the caller's stream.  When every set takes the
 * symmetric FP32 bin pass (the same d <= 16 and kernel family, the fused
 * schedule, exact KDE), the bin passes of all sets are one launch over the
 * sets' block pairs (Sec. 4.2: one level's KDE calls over all sets add up
 * to one KDE of their total size), between the trees' refresh and the rest of
 * each set's build; otherwise each set keeps its own launches.  Results are
 * the same either way.  With capture != 0 the first run records the whole
 * launch sequence into a CUDA graph and later runs replay it (inputs and
 * outputs are read and written through the pointers given at creation, so
 * new point values of the same shapes are picked up).
 */
typedef struct {
    const float* d_points;  /* device float32 [n][d], read at every run       */
    int64_t n;
    int32_t d;
    int32_t L;              /* 1..64                                          */
    fsg_params params;
    uint64_t seed;
    int32_t edge_mode;      /* FSG_EDGES_SET | FSG_EDGES_MULTI                */
    int32_t reserved0;
    int32_t* d_src;         /* device int32 [cap]                             */
    int32_t* d_dst;         /* device int32 [cap]                             */
    float* d_w;             /* device float32 [cap] (params.weight_f64 = 0)   */
    int64_t cap;            /* >= n * L                                       */
    int64_t* d_m_out;       /* device int64: edges written                    */
    double* d_deg;          /* optional device float64 [n]                    */
    fsg_stats* d_stats;     /* optional device statistics                     */
} fsg_batch_item;

typedef struct fsg_batch fsg_batch; /* opaque */

/* Errors: INVALID_ARG (any item), OOM, CUDA, UNSUPPORTED, CAPACITY. */
int fsg_batch_create(const fsg_batch_item* items, int32_t count, int32_t streams, int32_t capture,
                     void* stream, fsg_batch** out);
int fsg_batch_run(fsg_batch* batch, void* stream);
void fsg_batch_destroy(fsg_batch* batch);

/*
 * Serving: a request loop inside the library.  Graph-build requests (host
 * points, host outputs) of different n and d are queued; a worker thread
 * admits them (in arrival order, or by response ratio: see admission below)
 * whenever a slot (a stream) is free and the request's device memory
 * estimate fits the HBM budget next to the requests in flight.  Admitted requests run concurrently on their slots' streams, so
 * their kernels overlap on the GPU; device memory comes from the server's own
 * stream-ordered pool, so admitting and retiring requests never synchronizes
 * the device.  A request's result (edge list in its host buffers, latency) is
 * reported by fsg_server_poll once its edges are on the host.  Each result is
 * the one fsg_build_graph_host gives for the same request alone.
 */
typedef struct {
    int64_t hbm_budget_bytes;        /* device bytes for requests in flight (> 0)    */
    int32_t max_slots;               /* requests in flight at once, 1..64            */
    int32_t queue_cap;               /* pending requests before BUSY (0 = 65536)     */
    int32_t inject_alloc_fail_every; /* testing: every k-th admission fails with OOM */
    int32_t admission;               /* FSG_ADMIT_ARRIVAL (0) | FSG_ADMIT_RESPONSE_RATIO */
    int32_t reserved[4];
} fsg_server_opts;

/* Admission order.  ARRIVAL: strict arrival order.  RESPONSE_RATIO: highest
 * response ratio next (Brinch Hansen, 1971): the queued request with the
 * largest (waiting time + estimated run time) / estimated run time goes
 * first, so short requests overtake long ones while a long request's ratio
 * grows with its wait and it is never starved.  The run-time estimate is
 * proportional to the n^2 (d + 6) pair work of the request plus a fixed
 * launch cost.  In both orders the chosen request waits at the head until the
 * budget has room for it; results do not depend on the order. */
enum { FSG_ADMIT_ARRIVAL = 0, FSG_ADMIT_RESPONSE_RATIO = 1 };

typedef struct {
    const float* h_points;  /* host float32 [n][d]; valid until the result is polled */
    int64_t n;
    int32_t d;
    int32_t L;              /* 1..64                                          */
    fsg_params params;
    uint64_t seed;
    int32_t edge_mode;
    int32_t reserved0;
    int32_t* h_src;         /* host int32 [cap] (pinned memory is faster)     */
    int32_t* h_dst;         /* host int32 [cap]                               */
    float* h_w;             /* host float32 [cap] (params.weight_f64 = 0)     */
    int64_t cap;            /* >= n * L                                       */
} fsg_request;

typedef struct {
    uint64_t id;
    int32_t status;         /* FSG_OK or an FSG_ERR_* code                     */
    int32_t reserved0;
    int64_t n_edges;
    int64_t n_flagged;
    double latency_ms;      /* submission -> edges on the host                */
    double queue_ms;        /* submission -> admission                        */
} fsg_result;

typedef struct fsg_server fsg_server; /* opaque */

/* Errors: INVALID_ARG, OOM, CUDA. */
int fsg_server_create(const fsg_server_opts* opts, fsg_server** out);
/* Errors: INVALID_ARG (malformed request), CAPACITY (cap < n L),
 * BUSY (queue full, or the request alone exceeds the HBM budget). */
int fsg_server_submit(fsg_server* server, const fsg_request* req, uint64_t* id_out);
/* Up to max finished results into out; waits up to wait_ms for the first. */
int fsg_server_poll(fsg_server* server, fsg_result* out, int32_t max, int32_t* count_out, int32_t wait_ms);
/* A pending request is dropped (its result has status FSG_ERR_CANCELLED); a
 * request in flight completes and is then reported as cancelled. */
int fsg_server_cancel(fsg_server* server, uint64_t id);
int fsg_server_info(fsg_server* server, int64_t* pending, int64_t* in_flight, int64_t* bytes_in_use);
/* Waits for requests in flight, drops pending ones, frees everything. */
void fsg_server_destroy(fsg_server* server);

/*
 * Self-test of the failure path: launches a kernel that waits, the way every
 * pipeline of the library does, on an mbarrier that nothing completes, with
 * a wall-clock limit of limit_ns (1e3 .. 1e10).  Returns FSG_ERR_TIMEOUT when
 * the wait ran out and the kernel reported it through its status word as
 * designed (no trap; the context stays usable), FSG_OK if the wait completed
 * (a failure of the test), INVALID_ARG or CUDA otherwise.  Synchronous.
 */
int fsg_selftest_wait_timeout(int64_t limit_ns, void* stream);

/*
 * Waits for the stream and returns the tree's device status word
 * (FSG_OK or FSG_ERR_TIMEOUT), then clears it.  In a library built with
 * FSG_BOUNDS_CHECK (FSG_BOUNDS_CHECK=1 python -m paper_2310_13870_gb300.build,
 * into _build_bounds/) it also returns FSG_ERR_BOUNDS when an index check of
 * any kernel failed since the last call.  Errors: CUDA.
 */
int fsg_sync(fsg_tree* tree, void* stream);

/*
 * Bounds-checking build only (see fsg_sync): the first failed index check
 * since the last call (out[0] = 1, out[1] = the check's site number, out[2] =
 * the index, out[3] = its limit; all 0 when none failed), then cleared.
 * Synchronizes the device.  Other builds: FSG_ERR_UNSUPPORTED.  The paper has
 * no counterpart (a debugging aid of this library).
 */
int fsg_bounds_error(int64_t* out);

/*
 * End-to-end entry point on HOST buffers: copies h_points to the device,
 * builds the tree (FSG_ORDER_SPATIAL for FSG_PREC_SPLIT_BF16 up to d = 64,
 * identity otherwise), runs fsg_build_graph, and copies the edge list back.  The
 * server builds its trees the same way.
 *   h_src, h_dst (int32 [cap]), h_w (float32 [cap]; params->weight_f64 must
 *   be 0), *h_m_out (edge count).
 * Blocks until the result is on the host.  The device buffers live in an
 * internal per-thread cache that grows to the largest (n, d, L) seen.
 * Errors: as fsg_build_graph, plus CAPACITY when cap < n*L.
 */
int fsg_build_graph_host(const float* h_points, int64_t n, int32_t d, const fsg_params* params,
                         int32_t L, uint64_t seed, int32_t edge_mode, int32_t* h_src,
                         int32_t* h_dst, float* h_w, int64_t cap, int64_t* h_m_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FSG_H */
