// Internal declarations of the sm_103a FastSimilarityGraph library.
// Device helpers shared by the kernels: Philox4x32-10, packed FP32x2
// arithmetic, ex2, 1-D bulk copies (TMA engine) with mbarriers whose waits are
// bounded, and the descent decision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "fsg.h"

namespace fsg {

constexpr int kMaxL = 64;
// Item counters/cursors per bin are split into this many sub-slots (chosen by
// the query index) so that concurrent atomics spread over more addresses.
constexpr int kBinSlots = 16;
constexpr int kMaxFmaDim = 16;       // FP32 FMA tiles are compiled for d <= 16
constexpr int kStatusTimeout = FSG_ERR_TIMEOUT;
// Time limit of every bounded device wait (an mbarrier phase that does not
// complete within it is reported as FSG_ERR_TIMEOUT).
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------------------------
// Tree and workspace
// ---------------------------------------------------------------------------
struct Workspace {
    size_t bytes = 0;
    void* base = nullptr;
    // carve-outs (valid after ensure_workspace)
    float* binsum = nullptr;        // [n][nb]   bin sums per query (tree order)
    float* degf = nullptr;          // [n]       FP32 degree per position
    uint8_t* flags = nullptr;       // [n][L]    per-sample flags (tree order)
    int32_t* leaf_pos = nullptr;    // [n][L]    sampled neighbour position or -1
    float* ksmp = nullptr;          // [n][L]    kernel value k(x_i, x_j) of each sample
    uint8_t* lflags = nullptr;      // [n][L]    flags of the leaf-finish decisions
    int32_t* qitem_bin = nullptr;   // [n][L]     per query: distinct bins its samples reached
    uint64_t* qitem_mask = nullptr; // [n][L]     per query: mask of its samples at each
    int32_t* qitem_cnt = nullptr;   // [n]        per query: number of such bins
    int32_t* bin_count = nullptr;   // [nb][kBinSlots]   items per (bin, sub-slot)
    int32_t* bin_cursor = nullptr;  // [nb][kBinSlots]   scatter cursors
    int32_t* bin_off = nullptr;     // [nb*kBinSlots+1]  segment offsets
    int32_t* items_q = nullptr;     // [max_items] query position, grouped by bin
    uint64_t* items_mask = nullptr; // [max_items] samples of that query at the bin
    float* leafv = nullptr;         // [max_items][2^dm] leaf values (d > 16 only)
    int32_t* uniq = nullptr;        // [n][L]    per-query sorted distinct neighbours
    float* uniq_w = nullptr;        // [n][L]
    int32_t* ucnt = nullptr;        // [n]
    uint64_t* emit_mask = nullptr;  // [n]
    int64_t* ecount = nullptr;      // [n+1]     edges per query, scanned in place
    int64_t* scan_tmp = nullptr;    // [blocks]
    fsg_stats* stats = nullptr;     // device statistics of the last call
    int32_t* misc = nullptr;        // [8] n_tiles, ...
    int64_t cap_n = 0, cap_L = 0;
};

// Scratch of the high-precision re-decision (fsg_params.resolve), allocated
// on first use: the flagged levels of every sample, the flagged samples, the
// (sample, level) jobs grouped by node and their high-precision sums.
struct ResolveWs {
    void* base = nullptr;
    size_t bytes = 0;
    int64_t cap_nl = 0;             // n * L the arrays are sized for
    int32_t fcap = 0, jcap = 0;     // flagged samples and jobs of the batched path
    uint16_t* flev = nullptr;       // [n][L]  bit t: the FP32 decision at level t was flagged
    int32_t* list = nullptr;        // [n L]   flagged samples
    int32_t* sbin = nullptr;        // [fcap]  bin of each flagged sample's FP32 path
    int32_t* node_cnt = nullptr;    // [nb]    jobs per node (heap index)
    int32_t* node_cur = nullptr;    // [nb]
    int32_t* node_off = nullptr;    // [nb+1]  job offsets per node
    int32_t* cta_off = nullptr;     // [nb+1]  work items per node (32 jobs x a chunk of points)
    int32_t* part_off = nullptr;    // [nb+1]  partial-sum offsets per node
    int32_t* job_s = nullptr;       // [jcap]  flagged sample of a job
    int32_t* job_t = nullptr;       // [jcap]  level of a job
    int32_t* slot_of = nullptr;     // [fcap][kRsMaxLevels] job slot of (flagged sample, level)
    double* part = nullptr;         // [pcap][2] high-precision (g_left, g_right) per (job, point chunk)
    int32_t pcap = 0;
    int32_t* wlist = nullptr;       // [n L]   samples left to the per-sample walker (| mode << 30)
    int32_t* cnt = nullptr;         // [8]     flagged, jobs, walker entries, overflow
};
constexpr int kRsMaxLevels = 13;    // s0 <= 12 bin-pass levels

// Launch shapes (0: the built-in heuristic), chosen by fsg_autotune.
struct LaunchTuning {
    int32_t sym_bins = 0;     // bins per block of the symmetric d <= 16 bin pass
    int32_t tc_bins = 0;      // bins per chunk of the tensor-core bin pass
    int32_t leaf_splits = 0;  // CTAs per bin of the leaf finish
};

}  // namespace fsg

struct fsg_tree {
    int64_t n = 0;
    int32_t d = 0;
    int32_t dp = 0;          // padded dimension (multiple of 4)
    int32_t depth = 0;       // ceil(log2 n)
    int32_t leaf_max = 256;
    int32_t s0 = 0;          // levels decided from the bin pass
    int32_t nb = 1;          // bins = 2^s0
    int32_t mmax = 1;        // largest bin size = ceil(n / nb)
    int32_t dm = 0;          // ceil(log2 mmax): levels in the leaf finish
    int64_t n_pad = 0;       // rows allocated in the point arrays
    int device = 0;
    float* Xt = nullptr;     // [n_pad][dp]     tree-ordered points
    float* Xdup = nullptr;   // [n_pad][dp][2]  same, each coordinate twice (d <= 16)
    int32_t* perm = nullptr; // [n]  position -> original index
    void* ord = nullptr;     // scratch of the GPU spatial order (FSG_ORDER_SPATIAL)
    int32_t* inv = nullptr;  // [n]  original index -> position
    int32_t* bnd = nullptr;  // [nb+1] level-s0 node boundaries
    int32_t* status = nullptr;  // device status word
    int exact_int = 0;       // points are multiples of 1/255 in [0,1]
    // tensor-core path (d >= 64, exact 8-bit data): BF16 copy of 255 x,
    // squared norms in integer units, TMA descriptors (A: 128 rows, B: 256 rows,
    // P: 16 rows)
    void* Xb = nullptr;
    float* norms = nullptr;
    int32_t dpad = 0;
    // FP32 path for d > 16: the points as transposed 128-position tiles (query
    // layout [k][132] and duplicated point layout [k][130][2] per tile, k
    // padded to a multiple of 32), refreshed by every generic bin pass
    float* Xtt = nullptr;
    // split-precision pass: per bin, the bounding box of its points ([nb][2][64])
    float* sboxes = nullptr;
    alignas(64) unsigned char tmap_a[128] = {};
    alignas(64) unsigned char tmap_b[128] = {};
    alignas(64) unsigned char tmap_p[128] = {};  // 16-row boxes: point rows of the tensor-core leaf kernel
    // split-precision tensor-core path for d > 64 (FSG_PREC_SPLIT_BF16, made
    // on first use): every coordinate as three BF16 parts, [n_pad][3 dpad]
    // (all hi, then all mid, then all lo), the squared norms (FP64 sums
    // rounded once) and TMA descriptors with the same boxes as above
    void* Xs = nullptr;
    float* snorms = nullptr;
    alignas(64) unsigned char tmap_sa[128] = {};
    alignas(64) unsigned char tmap_sb[128] = {};
    alignas(64) unsigned char tmap_sp[128] = {};
    fsg::Workspace ws;
    fsg::ResolveWs rs;
    // stepped graph build (fsg_graph_begin / step / end): the call's
    // parameters and the stepped position ranges (sorted, disjoint, merged);
    // any other call on the tree ends it
    struct GraphRun {
        bool active = false;
        fsg_params p{};
        int32_t L = 0;
        uint64_t seed = 0;
        std::vector<std::pair<int64_t, int64_t>> done;
    } run;
    fsg::LaunchTuning tune;
    // per-phase timing (fsg_profile) and kernel-launch count
    bool profiling = false;
    cudaEvent_t ev_start[FSG_NUM_PHASES] = {};
    cudaEvent_t ev_end[FSG_NUM_PHASES] = {};
    bool ev_used[FSG_NUM_PHASES] = {};
    int64_t launches = 0;
    // Stream-ordered allocation (used by the server): when set, every device
    // buffer of this tree comes from `pool` on `alloc_stream` and is returned
    // with cudaFreeAsync, so creating and freeing trees never synchronizes.
    cudaMemPool_t pool = nullptr;
    cudaStream_t alloc_stream = nullptr;
};

namespace fsg {

// ---------------------------------------------------------------------------
// Host-side launchers (one per .cu file)
// ---------------------------------------------------------------------------
struct KernelParams {
    int precision;    // FSG_PREC_*
    float neg_c;      // -gamma * log2(e): k = ex2(neg_c * ||x-y||^2)
    float gamma;
    int self_exclude;
    int L;
    uint64_t seed;
    float flag_eps;
    float kde_eps;    // approximate bin pass: skipped mass <= kde_eps * degree (0 = exact)
    int family;       // FSG_KERNEL_*
    float hp_ch, hp_cl;  // gamma log2 e as a pair of FP32 numbers (high-precision values)
    int resolve;      // re-decide flagged descents in high precision
    int weight_f64;   // d_w is double: weights in FP64 from high-precision kernel values
};

// Raises the dynamic shared-memory limit of `kernel` on the current device to
// at least `bytes` (cudaFuncSetAttribute), once per (kernel, device) and
// value; safe to call from several threads and for several devices.
cudaError_t set_smem_limit_fn(const void* kernel, size_t bytes);
template <typename K>
inline cudaError_t set_smem_limit(K* kernel, size_t bytes) {
    return set_smem_limit_fn(reinterpret_cast<const void*>(kernel), bytes);
}

int ensure_workspace(fsg_tree* t, int L, cudaStream_t s);
int build_tree_internal(const float* d_points, int64_t n, int32_t d, const fsg_tree_opts* opts, cudaStream_t s,
                        cudaMemPool_t pool, fsg_tree** out);
size_t tree_bytes_estimate(int64_t n, int32_t d, int32_t L);
cudaError_t launch_tree_prep(fsg_tree* t, const float* d_points, const int32_t* d_perm, cudaStream_t s);
cudaError_t launch_kde_bins(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
bool kde_bins_supported(const fsg_tree* t);
cudaError_t launch_kde_bins_sym(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
// The symmetric d <= 16 pass of many trees in one launch: one descriptor per
// tree (device table, pair_off = the tree's first block pair in the launch).
struct SymPackDesc {
    const float* Xdup;
    const float* Xt;
    const int32_t* bnd;
    float* binsum;
    int32_t* status;
    int nb, G, nblk, pair_off;
    float neg_c;
    int self_exclude;
};
constexpr int kSymPackMax = 64;
struct SymPackTable {  // descriptors passed by value (a kernel parameter)
    SymPackDesc d[kSymPackMax];
    int count;
};
// Fills the tree's descriptor; returns its block pairs.
int sym_pack_fill(const fsg_tree* t, const KernelParams& kp, int pair_off, SymPackDesc* out);
cudaError_t launch_kde_bins_sym_packed(const SymPackDesc* d_descs, int count, int total, int d, int family,
                                       cudaStream_t s);
cudaError_t launch_kde_bins_sym_packed(const SymPackTable& tab, int total, int d, int family, cudaStream_t s);
// Argument and path checks of a graph build, and its kernel parameters.
int check_graph_call(const fsg_tree* t, const fsg_params* p);
KernelParams kernel_params_of(const fsg_params* p, int L, uint64_t seed);
// fsg_build_graph; with skip_bins the tree's bin sums are taken as already
// computed (by a packed bin pass of the batch).
int build_graph_internal(fsg_tree* t, const fsg_params* p, int32_t L, uint64_t seed, int32_t edge_mode,
                         int32_t* d_src, int32_t* d_dst, void* d_w, int64_t cap, int64_t* d_m_out, double* d_deg,
                         int32_t* d_samples, uint8_t* d_flags, fsg_stats* d_stats, cudaStream_t s, bool skip_bins);
bool kde_bins_sym_supported(const fsg_tree* t);
int64_t kde_bins_sym_evals(const fsg_tree* t);
// The descent above the bins and the bucketing for the queries at tree
// positions [q_lo, q_hi) (q_hi < 0: every query).
cudaError_t launch_descend_top(const fsg_tree* t, const KernelParams& kp, double* d_deg, int with_samples,
                               cudaStream_t s, int64_t q_lo = 0, int64_t q_hi = -1);
cudaError_t launch_bucket(const fsg_tree* t, const KernelParams& kp, cudaStream_t s, int64_t q_lo = 0,
                          int64_t q_hi = -1);
cudaError_t launch_leaf_finish(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
int leaf_queries_per_tile(const fsg_tree* t);
int64_t leaf_default_splits(const fsg_tree* t, int L);
// The 128-point leaf kernel applies: d <= 16, every bin of 65..128 points.
bool use_leaf128(const fsg_tree* t);
cudaError_t launch_edges(const fsg_tree* t, const KernelParams& kp, int edge_mode, int32_t* d_src,
                         int32_t* d_dst, void* d_w, int64_t cap, int64_t* d_m_out, cudaStream_t s);
// High-precision re-decision of flagged samples (scratch t->rs, allocated by
// ensure_resolve before the call's first launch).
bool resolve_supported(const fsg_tree* t);
int ensure_resolve(fsg_tree* t, int L, cudaStream_t s);
// Re-decides the flagged samples of the queries at tree positions
// [q_lo, q_hi) (q_hi < 0: every query).
cudaError_t launch_resolve(const fsg_tree* t, const KernelParams& kp, cudaStream_t s, int64_t q_lo = 0,
                           int64_t q_hi = -1);
cudaError_t launch_outputs(const fsg_tree* t, const KernelParams& kp, int32_t* d_samples, uint8_t* d_flags,
                           fsg_stats* d_stats, cudaStream_t s);
cudaError_t launch_kde_bins_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
bool kde_bins_generic_sym_supported(const fsg_tree* t);
size_t generic_tile_bytes(int64_t n, int32_t d);
int64_t kde_bins_generic_sym_evals(const fsg_tree* t);
int tc_prepare(fsg_tree* t, cudaStream_t s);
// The three-part BF16 image of the points for the split form at d > 64
// (allocated and described on the first call, refilled on every call).
int splitk_prepare(fsg_tree* t, cudaStream_t s);
// The split form at d > 64 runs the tensor-core bin pass and leaf kernel on
// the three-part image (bins of at least 33 points).
bool splitk_supported(const fsg_tree* t);
bool kde_bins_tc_supported(const fsg_tree* t);
// Pairs the tensor-core bin pass evaluates (symmetric form: each pair once
// outside the diagonal chunks).
int64_t kde_bins_tc_evals(const fsg_tree* t);
bool kde_bins_split_supported(const fsg_tree* t);
// Bytes of the split-precision pass's per-tree workspace (boxes, query-tile
// images, and the bins' images when the split leaf phase runs).
size_t split_workspace_bytes(int64_t n, int64_t nb, bool bin_images);
// GPU spatial order of d_points ([n][d]) in the scratch buf
// (spatial_order_scratch_bytes); *out = the array holding it.
size_t spatial_order_scratch_bytes(int64_t n, int d);
cudaError_t launch_spatial_order(const float* d_points, int64_t n, int d, int leaf, void* buf, const int32_t** out,
                                 cudaStream_t s);
constexpr int kSpatialLeaf = 32;
// Split-precision leaf phase on the tensor cores: d in 17..64, bins of at
// most 128 points (after the split bin pass, whose workspace it shares).
bool leaf_split_tc_supported(const fsg_tree* t);
cudaError_t launch_leaf_split_tc(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
bool leaf_fused_generic_supported(const fsg_tree* t);
cudaError_t launch_leaf_fused_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
cudaError_t launch_kde_bins_split(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
cudaError_t launch_kde_bins_tc(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
cudaError_t launch_leaf_values_tc(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
cudaError_t launch_leaf_values_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s);
cudaError_t launch_levelwise(const fsg_tree* t, const KernelParams& kp, double* d_deg, int with_samples,
                             int carried, cudaStream_t s, int64_t* launches);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplications whose high halves are xored into the other words and the
// round key; the key advances by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r < 9) { k.x += W0; k.y += W1; }
    }
    return c;
}

// Four consecutive levels (4m .. 4m+3) of one (point, sample) share one block.
__device__ __forceinline__ uint4 draw_block(uint64_t seed, uint32_t i, uint32_t l, uint32_t level) {
    return philox4x32_10(make_uint4(i, l, level >> 2, 0u),
                         make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)));
}
__device__ __forceinline__ uint32_t block_word(const uint4& b, uint32_t level) {
    const uint32_t w = level & 3u;
    return w == 0 ? b.x : (w == 1 ? b.y : (w == 2 ? b.z : b.w));
}

// One level of the descent of Algorithm 1: returns 1 for the right half.
// The exact rule is "left iff u < g_left / (g_left + g_right)", i.e.
// u * S - g_left < 0 with S = g_left + g_right, evaluated here with one fused
// multiply-add.  u is the draw truncated to 24 bits (exact in FP32, at most
// 2^-24 below the 32-bit value).  The decision is flagged when
// |u S - g_left| < 2 eps min(g_left, g_right) + 2^-22 S: with both sums
// within relative error eps of the exact ones, an unflagged decision equals
// the exact one (min(r, 1-r) >= r (1-r) bounds the ratio's error).
// abs_tol: a further absolute error of gl and gr together (sums that may miss
// up to that much mass, as the approximate bin pass's do): u S - gl moves by
// at most that much.
__device__ __forceinline__ int descend_decide(float gl, float gr, uint32_t word, float eps, uint8_t& flag,
                                              float abs_tol = 0.f) {
    const float S = gl + gr;
    if (!(S > 0.f)) { flag |= 2; return 1; }
    const float u = __uint2float_rz(word >> 8) * 0x1p-24f;
    const float dlt = fmaf(u, S, -gl);
    const float tol = 2.f * eps * fminf(gl, gr) + 0x1p-22f * S + abs_tol;
    if (fabsf(dlt) < tol) flag |= 1;
    return dlt < 0.f ? 0 : 1;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32x2 arithmetic (sm_100+): both lanes rounded to nearest, IEEE.
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d; asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c)); return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t d; asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi)); return d;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
    float2 r; asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v)); return r;
}

// ---------------------------------------------------------------------------
// High-precision kernel values (the re-decision of flagged descents and the
// FP64 weights).  The squared distance of two FP32 points is accumulated as
// an unevaluated pair of FP32 numbers (hi + lo): each coordinate difference
// is split exactly into its rounded value and rounding error (two-sum,
// Knuth), its square exactly into product and error (fused multiply-add),
// and the terms are added with two-sum, so ||x - y||^2 carries a relative
// error of a few 2^-46.  The exponent c ||x - y||^2 (c = gamma log2 e, also
// as a pair) is split into an integer and a fraction f, |f| <= 1/2 + 2^-20,
// and k = 2^-f 2^-i with 2^-f from ex2.approx (relative error below 2^-22)
// and f rounded to FP32 (2^-25 absolute, 2^-25.5 relative in k).  Every
// value is therefore within relative error kHpEta of exp(-gamma ||x-y||^2)
// computed exactly, or below 2^-126 where FP32 flushes it to zero.
// ---------------------------------------------------------------------------
constexpr double kHpEta = 0x1p-20;  // relative error bound used by the re-decision (a 3x margin)

__device__ __forceinline__ void hp_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Adds the square of x - y (both FP32) to the pair (sh, sl).
__device__ __forceinline__ void hp_acc_sq(float x, float y, float& sh, float& sl) {
    float dh, dl;
    hp_two_sum(x, -y, dh, dl);            // x - y = dh + dl exactly
    const float ph = __fmul_rn(dh, dh);
    float pl = __fmaf_rn(dh, dh, -ph);    // dh^2 = ph + pl exactly
    pl = __fmaf_rn(__fmul_rn(2.f, dh), dl, pl);  // + 2 dh dl (dl^2 < 2^-48 dh^2)
    float th, te;
    hp_two_sum(sh, ph, th, te);
    sh = th;
    sl = __fadd_rn(sl, __fadd_rn(te, pl));
}

// 2^-(th + tl) for th >= 0 (the pair of the exponent in base 2).
__device__ __forceinline__ float hp_exp2_neg(float th, float tl) {
    const float ti = rintf(th);
    if (ti > 150.f) return 0.f;
    const float f = __fadd_rn(__fsub_rn(th, ti), tl);  // th - ti is exact
    const float m = ex2_approx(-f);
    const int e = 127 - (int)ti;                       // 2^-ti as an FP32 power of two
    return e >= 1 ? __fmul_rn(m, __int_as_float(e << 23)) : 0.f;
}

// k from the pair (sh, sl) = ||x - y||^2 and (ch, cl) = gamma log2 e.
__device__ __forceinline__ float hp_finish(float sh, float sl, float ch, float cl) {
    const float th = __fmul_rn(sh, ch);
    const float tl = __fadd_rn(__fmaf_rn(sh, ch, -th), __fmaf_rn(sh, cl, __fmul_rn(sl, ch)));
    return hp_exp2_neg(th, tl);
}

// k(x, y) = exp(-gamma ||x - y||^2) to relative error kHpEta (see above);
// (ch, cl) = gamma log2 e as a pair.  x: dp coordinates (any memory), y: a
// 16-byte aligned row of dp coordinates (dp a multiple of 4, zero padding on
// both sides), read 16 coordinates at a time with the loads issued together.
__device__ __forceinline__ float hp_gauss(const float* __restrict__ x, const float* __restrict__ y, int dp, float ch,
                                          float cl) {
    float sh = 0.f, sl = 0.f;
    const float4* y4 = reinterpret_cast<const float4*>(y);
    for (int t0 = 0; t0 < dp; t0 += 16) {
        float4 c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t0 + 4 * k < dp) c[k] = __ldg(y4 + (t0 >> 2) + k);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (t0 + 4 * k < dp) {
                const float* xx = x + t0 + 4 * k;
                hp_acc_sq(xx[0], c[k].x, sh, sl);
                hp_acc_sq(xx[1], c[k].y, sh, sl);
                hp_acc_sq(xx[2], c[k].z, sh, sl);
                hp_acc_sq(xx[3], c[k].w, sh, sl);
            }
        }
    }
    return hp_finish(sh, sl, ch, cl);
}

// hp_gauss, first testing the pair in FP32: where ch ||x - y||^2 > 127 the
// high-precision value would be flushed to zero (2^-f 2^-i with i >= 127,
// i.e. an exponent of at least 126.5), so 0 is returned without the
// high-precision work.  The FP32 exponent (direct differences, relative error
// about (d + 2) 2^-24) is within 0.04 of the pair's for d <= 4096, so the
// test never drops a value the high-precision path keeps.
__device__ __forceinline__ float hp_gauss_far0(const float* __restrict__ x, const float* __restrict__ y, int dp,
                                               float ch, float cl) {
    const float4* y4 = reinterpret_cast<const float4*>(y);
    float s = 0.f;
    for (int t0 = 0; t0 < dp; t0 += 16) {
        float4 c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t0 + 4 * k < dp) c[k] = __ldg(y4 + (t0 >> 2) + k);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (t0 + 4 * k < dp) {
                const float* xx = x + t0 + 4 * k;
                float dd = xx[0] - c[k].x; s = fmaf(dd, dd, s);
                dd = xx[1] - c[k].y; s = fmaf(dd, dd, s);
                dd = xx[2] - c[k].z; s = fmaf(dd, dd, s);
                dd = xx[3] - c[k].w; s = fmaf(dd, dd, s);
            }
        }
    }
    if (s * ch > 127.f) return 0.f;
    return hp_gauss(x, y, dp, ch, cl);
}

// Kernel families (Sec. 2.1): the exponent is neg_c times the squared
// Euclidean distance (Gaussian), the l1 distance (Laplacian) or the Euclidean
// distance (exponential).  A distance is accumulated term by term from the
// coordinate differences dd (first, acc) and finished (fin) before the scale;
// the packed (two lanes) and the scalar forms round identically per lane.
constexpr int kFamGauss = FSG_KERNEL_GAUSSIAN;
constexpr int kFamLaplace = FSG_KERNEL_LAPLACIAN;
constexpr int kFamExp = FSG_KERNEL_EXPONENTIAL;
__device__ __forceinline__ uint64_t f2_abs(uint64_t a) { return a & 0x7fffffff7fffffffull; }
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <int F> __device__ __forceinline__ uint64_t fam_first2(uint64_t dd) {
    return F == kFamLaplace ? f2_abs(dd) : f2_mul(dd, dd);
}
template <int F> __device__ __forceinline__ uint64_t fam_acc2(uint64_t dd, uint64_t s) {
    return F == kFamLaplace ? f2_add(s, f2_abs(dd)) : f2_fma(dd, dd, s);
}
template <int F> __device__ __forceinline__ uint64_t fam_fin2(uint64_t s) {
    if (F != kFamExp) return s;
    const float2 v = f2_unpack(s);
    return f2_pack(sqrt_approx(v.x), sqrt_approx(v.y));
}
template <int F> __device__ __forceinline__ float fam_first1(float dd) {
    return F == kFamLaplace ? fabsf(dd) : __fmul_rn(dd, dd);
}
template <int F> __device__ __forceinline__ float fam_acc1(float dd, float s) {
    return F == kFamLaplace ? __fadd_rn(s, fabsf(dd)) : __fmaf_rn(dd, dd, s);
}
template <int F> __device__ __forceinline__ float fam_fin1(float s) {
    return F == kFamExp ? sqrt_approx(s) : s;
}

// --- mbarrier + 1-D bulk copy (TMA engine) --------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// The first 1024-byte boundary at or after p (dynamic shared memory), by
// pointer arithmetic on p itself, so accesses through the result stay
// shared-memory instructions (a round trip through an integer would make
// them generic loads and stores).
__device__ __forceinline__ unsigned char* smem_align1024(unsigned char* p) {
    return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bulk copy of `bytes` (multiple of 16, 16-byte aligned on both sides) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// The same test, but the thread may be suspended (up to about ns nanoseconds)
// until the phase completes instead of returning at once: waiting threads
// then take no issue slots from the working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: returns false (and records FSG_ERR_TIMEOUT) if the phase did
// not complete within kWaitLimitNs of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int32_t* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_sleep(bar, parity, 1u << 20)) return true;
        if ((it & 31u) == 0u && global_ns() - t0 > kWaitLimitNs) {
            atomicExch(status, kStatusTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ int ceil_log2_dev(int m) {
    return m <= 1 ? 0 : 32 - __clz(m - 1);
}

// Start of node k (0..15) at depth 4 of a bin of m points, by the halving
// rule (k = 16: the end).  Shared by the leaf kernels that keep a bin's row
// of values.
__device__ __forceinline__ int depth4_start(int k, int m) {
    if (k >= 16) return m;
    int a = 0, c = m;
    for (int t = 3; t >= 0; --t) {
        const int mid = a + (c - a) / 2;
        if ((k >> t) & 1) a = mid; else c = mid;
    }
    return a;
}

// One sample's remaining decisions inside a bin of m points (dm = ceil(log2 m)
// levels, the first at tree level s0), from the item's row of values vi
// (vi[j] = k(query, point j of the bin)) and the tree bi of its depth-4 node
// sums (bi[16 + k] = node k, bi[h] = bi[2h] + bi[2h+1]): the four top levels
// read bi, deeper ones sum the values of the node's two halves.  Returns the
// leaf's offset in the bin and sets the flags.
__device__ __forceinline__ int descend_bin_row(const float* __restrict__ vi, const float* __restrict__ bi, int m,
                                               int dm, int s0, uint64_t seed, uint32_t qi, uint32_t l, float eps,
                                               uint8_t& f) {
    int a = 0, c = m, h = 1;
    uint4 blk = make_uint4(0, 0, 0, 0);
    int blk_id = -1;
    for (int t = 0; t < dm; ++t) {
        int right = 1;  // a single point sits in the right half
        if (c - a >= 2) {
            const int mid = a + (c - a) / 2;
            float gl, gr;
            if (t < 4) {  // both halves are nodes of the depth-4 tree
                gl = bi[2 * h];
                gr = bi[2 * h + 1];
            } else {
                gl = 0.f;
                gr = 0.f;
                for (int j = a; j < mid; ++j) gl += vi[j];
                for (int j = mid; j < c; ++j) gr += vi[j];
            }
            const uint32_t lev = (uint32_t)(s0 + t);
            if ((int)(lev >> 2) != blk_id) {
                blk_id = (int)(lev >> 2);
                blk = draw_block(seed, qi, l, lev);
            }
            right = descend_decide(gl, gr, block_word(blk, lev), eps, f);
            if (right) a = mid; else c = mid;
        }
        h = 2 * h + right;
    }
    return a;
}

#endif  // __CUDACC__

// ---------------------------------------------------------------------------
// Bounds-checking build (-DFSG_BOUNDS_CHECK; FSG_BOUNDS_CHECK=1 python -m
// paper_2310_13870_gb300.build).  FSG_INB(i, lim, site) tests an index before
// a global access; a failure is recorded once per translation unit (site,
// index, limit) in that unit's device error words and the access is skipped
// instead of going out of bounds.  fsg_sync then returns FSG_ERR_BOUNDS and
// fsg_bounds_error reads and clears the record.  Other builds compile every
// check to `true`.
// ---------------------------------------------------------------------------
#ifdef FSG_BOUNDS_CHECK
#define FSG_BOUNDS_TU(name)                                                                         \
    static __device__ unsigned long long g_fsg_bounds[4];                                           \
    static __device__ __forceinline__ bool fsg_inb(long long i, long long lim, int site) {          \
        if (i >= 0 && i < lim) return true;                                                         \
        if (atomicCAS(&g_fsg_bounds[0], 0ull, 1ull) == 0ull) {                                      \
            g_fsg_bounds[1] = (unsigned long long)site;                                             \
            g_fsg_bounds[2] = (unsigned long long)i;                                                \
            g_fsg_bounds[3] = (unsigned long long)lim;                                              \
        }                                                                                           \
        return false;                                                                               \
    }                                                                                               \
    namespace fsg {                                                                                 \
    int bounds_read_##name(long long* out) {                                                        \
        if (cudaMemcpyFromSymbol(out, g_fsg_bounds, sizeof(g_fsg_bounds)) != cudaSuccess) return -1; \
        if (out[0]) {                                                                               \
            const unsigned long long z[4] = {0, 0, 0, 0};                                           \
            cudaMemcpyToSymbol(g_fsg_bounds, z, sizeof(z));                                         \
        }                                                                                           \
        return out[0] ? 1 : 0;                                                                      \
    }                                                                                               \
    }
#define FSG_INB(i, lim, site) fsg_inb((long long)(i), (long long)(lim), (site))
#else
#define FSG_BOUNDS_TU(name)
#define FSG_INB(i, lim, site) true
#endif
// Check sites (FSG_INB's third argument).
enum {
    kSiteSymRow = 1, kSiteSymMirror, kSitePlainRow, kSiteTopItem, kSiteScatter, kSiteLeaf128, kSiteLeafFinish,
    kSiteTcRow, kSiteTcCol, kSiteResolveWalk, kSiteResolvePart, kSiteResolveList
};
#ifdef FSG_BOUNDS_CHECK
int bounds_read_fma(long long* out);
int bounds_read_descend(long long* out);
int bounds_read_tc(long long* out);
int bounds_read_resolve(long long* out);
#endif

inline int ceil_log2_host(int64_t m) {
    int r = 0;
    while ((int64_t(1) << r) < m) ++r;
    return r;
}

}  // namespace fsg
