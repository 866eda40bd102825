// C ABI entry points (include/fsg.h): argument checks, the tree object and
// its workspace, and the fixed launch sequence of each call.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "fsg_internal.cuh"

namespace fsg {

int leaf_queries_per_tile(const fsg_tree* t);

namespace {

constexpr double kLog2e = 1.4426950408889634073599246810019;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return FSG_OK;
    if (e == cudaErrorMemoryAllocation) return FSG_ERR_OOM;
    return FSG_ERR_CUDA;
}

int check_params(const fsg_params* p) {
    if (!p) return FSG_ERR_INVALID_ARG;
    if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return FSG_ERR_INVALID_ARG;
    if (p->scale_conv != FSG_TWO_SIGMA_SQ && p->scale_conv != FSG_SIGMA_SQ) return FSG_ERR_INVALID_ARG;
    if (p->self_mode != FSG_SELF_EXCLUDE && p->self_mode != FSG_SELF_INCLUDE) return FSG_ERR_INVALID_ARG;
    if (p->precision < FSG_PREC_AUTO || p->precision > FSG_PREC_EXACT_INT) return FSG_ERR_INVALID_ARG;
    if (p->schedule != FSG_SCHED_FUSED && p->schedule != FSG_SCHED_LEVELWISE && p->schedule != FSG_SCHED_CARRIED)
        return FSG_ERR_INVALID_ARG;
    if (!(p->flag_eps >= 0.f) || !std::isfinite(p->flag_eps) || p->flag_eps > 0.25f) return FSG_ERR_INVALID_ARG;
    if (!(p->kde_eps >= 0.f) || !std::isfinite(p->kde_eps) || p->kde_eps > 0.5f) return FSG_ERR_INVALID_ARG;
    if (p->kernel != FSG_KERNEL_GAUSSIAN && p->kernel != FSG_KERNEL_LAPLACIAN && p->kernel != FSG_KERNEL_EXPONENTIAL)
        return FSG_ERR_INVALID_ARG;
    if ((p->resolve != 0 && p->resolve != 1) || (p->weight_f64 != 0 && p->weight_f64 != 1)) return FSG_ERR_INVALID_ARG;
    return FSG_OK;
}

// The arithmetic a call runs.  The tensor-core forms get the squared
// distance from the expanded dot product: the Gaussian's exponent, and the
// exponential's after a square root (exact integers on 8-bit data).  The
// Laplacian's l1 distance has no such form, so for it AUTO means FP32.
int eff_precision(const fsg_params* p) {
    return p->kernel == FSG_KERNEL_LAPLACIAN && p->precision == FSG_PREC_AUTO ? FSG_PREC_FP32 : p->precision;
}

KernelParams make_kernel_params(const fsg_params* p, int L, uint64_t seed) {
    // Gaussian: gamma of the bandwidth convention; Laplacian and exponential:
    // 1/sigma times their distance
    const double gamma = p->kernel != FSG_KERNEL_GAUSSIAN ? 1.0 / p->sigma
                         : p->scale_conv == FSG_SIGMA_SQ  ? 1.0 / (p->sigma * p->sigma)
                                                          : 1.0 / (2.0 * p->sigma * p->sigma);
    KernelParams kp{};
    kp.precision = eff_precision(p);
    kp.gamma = (float)gamma;
    kp.neg_c = (float)(-gamma * kLog2e);
    if (kp.neg_c > -1e-30f) kp.neg_c = -1e-30f;  // keeps far-away padding at exactly 0
    kp.self_exclude = p->self_mode == FSG_SELF_EXCLUDE ? 1 : 0;
    kp.L = L;
    kp.seed = seed;
    // default: the relative error bound of the sums of the chosen form (the
    // split form's FP32 tensor-core accumulation adds up to about 4e-4)
    kp.flag_eps = p->flag_eps > 0.f ? p->flag_eps : (p->precision == FSG_PREC_SPLIT_BF16 ? 0x1p-10f : 0x1p-13f);
    kp.kde_eps = p->kde_eps;
    kp.family = p->kernel;
    // gamma log2 e as an unevaluated pair of FP32 numbers (high-precision values)
    const double c = gamma * kLog2e;
    kp.hp_ch = (float)c;
    kp.hp_cl = (float)(c - (double)kp.hp_ch);
    kp.resolve = p->resolve;
    kp.weight_f64 = p->weight_f64;
    return kp;
}

// Records the start/end event of a phase when profiling is on.
// One phase of a call: CUDA events around it when profiling (fsg_profile),
// and always an NVTX range with the phase's name on the host timeline, for
// tracing tools such as Nsight Systems (without a tool attached the NVTX
// calls return at once).
constexpr const char* kPhaseNames[FSG_NUM_PHASES] = {"fsg:tree",  "fsg:kde_bins", "fsg:descend_top",
                                                     "fsg:bucket", "fsg:leaf",    "fsg:edges",
                                                     "fsg:outputs", "fsg:resolve"};
struct PhaseScope {
    fsg_tree* t;
    int phase;
    cudaStream_t s;
    PhaseScope(fsg_tree* t_, int phase_, cudaStream_t s_) : t(t_), phase(phase_), s(s_) {
        nvtxRangePushA(kPhaseNames[phase]);
        if (t->profiling) cudaEventRecord(t->ev_start[phase], s);
    }
    ~PhaseScope() {
        if (t->profiling) {
            cudaEventRecord(t->ev_end[phase], s);
            t->ev_used[phase] = true;
        }
        nvtxRangePop();
    }
};

// Every call on a tree starts here; it ends a stepped build in progress
// (the call reuses the workspace that holds the run's state).
void begin_call(fsg_tree* t) {
    for (int k = 0; k < FSG_NUM_PHASES; ++k) t->ev_used[k] = false;
    t->run.active = false;
}

// Bin pass: the symmetric kernel (each pair once) when bins hold 61..128 points.
bool use_tc(const fsg_tree* t, int precision) {
    return precision == FSG_PREC_EXACT_INT || (precision == FSG_PREC_AUTO && kde_bins_tc_supported(t));
}
// The split form at d > 64: the tensor-core kernels on the three-part image.
bool use_splitk(const fsg_tree* t, int precision) { return precision == FSG_PREC_SPLIT_BF16 && t->d > 64; }

cudaError_t run_kde_bins(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    if (use_splitk(t, kp.precision)) return launch_kde_bins_tc(t, kp, s);
    if (kp.precision == FSG_PREC_SPLIT_BF16) return launch_kde_bins_split(t, kp, s);
    if (use_tc(t, kp.precision)) return launch_kde_bins_tc(t, kp, s);
    if (t->d > kMaxFmaDim) return launch_kde_bins_generic(t, kp, s);
    if (kde_bins_sym_supported(t)) return launch_kde_bins_sym(t, kp, s);
    return launch_kde_bins(t, kp, s);
}

// The remaining levels of every sample inside its bin.  Tensor-core path and
// d > 16 with bins of <= 128 points: one fused kernel (values and descent);
// other d > 16 bins: leaf values, then the leaf finish; d <= 16: the leaf
// finish evaluates its own values.
cudaError_t run_leaf_phase(fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    if (t->d > kMaxFmaDim && (use_tc(t, kp.precision) || use_splitk(t, kp.precision)) && (1 << t->dm) <= 256) {
        t->launches += 1;
        return launch_leaf_values_tc(t, kp, s);
    }
    if (kp.precision == FSG_PREC_SPLIT_BF16 && leaf_split_tc_supported(t)) {  // the split mode's arithmetic
        t->launches += 2;
        return launch_leaf_split_tc(t, kp, s);
    }
    if (leaf_fused_generic_supported(t)) {  // d > 16, bins of <= 128 points: values stay on chip
        t->launches += 1;
        return launch_leaf_fused_generic(t, kp, s);
    }
    cudaError_t e = cudaSuccess;
    if (t->d > kMaxFmaDim) {
        e = launch_leaf_values_generic(t, kp, s);
        t->launches += 1;
    }
    if (e == cudaSuccess) e = launch_leaf_finish(t, kp, s);
    t->launches += 1;
    return e;
}

// Kernel evaluations the bin pass executes (n^2, or about n^2/2 when symmetric).
int64_t bin_pass_evals(const fsg_tree* t, int precision) {
    if (use_tc(t, precision) || use_splitk(t, precision)) return kde_bins_tc_evals(t);
    if (precision == FSG_PREC_SPLIT_BF16) return t->n * t->n;
    if (t->d <= kMaxFmaDim) return kde_bins_sym_supported(t) ? kde_bins_sym_evals(t) : t->n * t->n;
    return kde_bins_generic_sym_supported(t) ? kde_bins_generic_sym_evals(t) : t->n * t->n;
}

int check_path(const fsg_tree* t, const fsg_params* p) {
    if (p->precision == FSG_PREC_SPLIT_BF16 && !kde_bins_split_supported(t) && !splitk_supported(t))
        return FSG_ERR_UNSUPPORTED;
    // the Laplacian and exponential kernels: the fused schedule's FP32 paths
    // (d <= 16: the symmetric bin pass and the 128-point leaf kernel; d > 16:
    // the generic passes and leaf kernels); the exponential also on the exact
    // 8-bit tensor-core path
    if (p->kernel != FSG_KERNEL_GAUSSIAN &&
        ((p->precision != FSG_PREC_AUTO && p->precision != FSG_PREC_FP32 &&
          !(p->precision == FSG_PREC_EXACT_INT && p->kernel == FSG_KERNEL_EXPONENTIAL)) ||
         p->schedule != FSG_SCHED_FUSED || (t->d <= kMaxFmaDim && (!kde_bins_sym_supported(t) || !use_leaf128(t)))))
        return FSG_ERR_UNSUPPORTED;
    // the approximate bin pass is the split form's tile pruning (d <= 64)
    if (p->kde_eps > 0.f && (p->precision != FSG_PREC_SPLIT_BF16 || p->schedule != FSG_SCHED_FUSED ||
                             !kde_bins_split_supported(t)))
        return FSG_ERR_UNSUPPORTED;
    if (p->precision == FSG_PREC_EXACT_INT && !kde_bins_tc_supported(t)) return FSG_ERR_UNSUPPORTED;
    // the high-precision re-decision re-reads the fused schedule's bin sums (Gaussian kernel)
    if (p->resolve && (p->schedule != FSG_SCHED_FUSED || p->kernel != FSG_KERNEL_GAUSSIAN ||
                       !resolve_supported(t)))
        return FSG_ERR_UNSUPPORTED;
    if (p->weight_f64 && p->kernel != FSG_KERNEL_GAUSSIAN) return FSG_ERR_UNSUPPORTED;
    // the levelwise schedules are plain FP32 paths only
    if (p->schedule != FSG_SCHED_FUSED && p->precision != FSG_PREC_AUTO && p->precision != FSG_PREC_FP32)
        return FSG_ERR_UNSUPPORTED;
    return FSG_OK;
}

cudaError_t tree_malloc(fsg_tree* t, void** p, size_t bytes, cudaStream_t s) {
    if (t->pool) return cudaMallocFromPoolAsync(p, bytes, t->pool, s);
    return cudaMalloc(p, bytes);
}

void tree_free(fsg_tree* t, void* p) {
    if (!p) return;
    if (t->pool) cudaFreeAsync(p, t->alloc_stream);
    else cudaFree(p);
}

}  // namespace

namespace {
std::mutex g_attr_mu;
std::map<std::pair<const void*, int>, size_t> g_attr_set;  // (kernel, device) -> limit set
}  // namespace

cudaError_t set_smem_limit_fn(const void* kernel, size_t bytes) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    size_t& cur = g_attr_set[{kernel, dev}];
    if (cur >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// Byte sizes of the workspace carve-outs, in carve order (shared by the
// allocation and the server's admission estimate).
namespace {
constexpr int kWsParts = 23;
void workspace_sizes(int64_t n, int d, int dm, int nb, int64_t Lc, size_t (&sz)[kWsParts]) {
    const int64_t max_items = n * (Lc < nb ? Lc : nb);  // distinct (query, bin) pairs
    const int64_t nblocks = (n + 1023) / 1024 + 2;
    const size_t v[kWsParts] = {
        sizeof(float) * (size_t)n * nb,                       // binsum
        sizeof(float) * (size_t)n,                            // degf
        sizeof(uint8_t) * (size_t)n * Lc,                     // flags
        sizeof(int32_t) * (size_t)n * Lc,                     // leaf_pos
        sizeof(float) * (size_t)n * Lc,                       // ksmp
        sizeof(uint8_t) * (size_t)n * Lc,                     // lflags
        sizeof(int32_t) * (size_t)n * Lc,                     // qitem_bin
        sizeof(uint64_t) * (size_t)n * Lc,                    // qitem_mask
        sizeof(int32_t) * (size_t)n,                          // qitem_cnt
        sizeof(int32_t) * (size_t)nb * kBinSlots,             // bin_count
        sizeof(int32_t) * (size_t)nb * kBinSlots,             // bin_cursor
        sizeof(int32_t) * (size_t)(nb * kBinSlots + 1),       // bin_off
        sizeof(int32_t) * (size_t)max_items,                  // items_q
        sizeof(uint64_t) * (size_t)max_items,                 // items_mask
        d > kMaxFmaDim ? sizeof(float) * (size_t)max_items * ((size_t)1 << dm) : 0,  // leafv
        sizeof(int32_t) * (size_t)n * Lc,                     // uniq
        sizeof(float) * (size_t)n * Lc,                       // uniq_w
        sizeof(int32_t) * (size_t)n,                          // ucnt
        sizeof(uint64_t) * (size_t)n,                         // emit_mask
        sizeof(int64_t) * (size_t)(n + 1),                    // ecount
        sizeof(int64_t) * (size_t)nblocks,                    // scan_tmp
        sizeof(fsg_stats),                                    // stats
        sizeof(int32_t) * 8,                                  // misc
    };
    for (int k = 0; k < kWsParts; ++k) sz[k] = v[k];
}
}  // namespace

// The split-precision pass's workspace (allocated on first use): for d <= 64
// bin and tile boxes and the query tiles' split images; for d > 64 the
// three-part image of the points (refilled by fsg_tree_update).
int ensure_split(fsg_tree* t, const fsg_params* p, cudaStream_t s) {
    if (p->precision != FSG_PREC_SPLIT_BF16 || p->schedule != FSG_SCHED_FUSED) return FSG_OK;
    if (t->d > 64) {
        if (t->Xs) return FSG_OK;
        const int dpad = (t->d + 63) / 64 * 64;
        const size_t xbytes = sizeof(uint16_t) * 3 * (size_t)dpad * (size_t)t->n_pad;
        if (tree_malloc(t, &t->Xs, xbytes, s) != cudaSuccess ||
            tree_malloc(t, (void**)&t->snorms, sizeof(float) * (size_t)t->n_pad, s) != cudaSuccess) {
            cudaGetLastError();
            tree_free(t, t->Xs);
            t->Xs = nullptr;
            return FSG_ERR_OOM;
        }
        if (cudaMemsetAsync(t->Xs, 0, xbytes, s) != cudaSuccess) return FSG_ERR_CUDA;
        const int rc = splitk_prepare(t, s);
        if (rc != FSG_OK) {
            tree_free(t, t->Xs);
            tree_free(t, t->snorms);
            t->Xs = nullptr;
            t->snorms = nullptr;
        }
        return rc;
    }
    if (t->sboxes) return FSG_OK;
    if (tree_malloc(t, (void**)&t->sboxes, split_workspace_bytes(t->n, t->nb, leaf_split_tc_supported(t)), s) !=
        cudaSuccess) {
        cudaGetLastError();
        t->sboxes = nullptr;
        return FSG_ERR_OOM;
    }
    return FSG_OK;
}

int ensure_workspace(fsg_tree* t, int L, cudaStream_t s) {
    Workspace& ws = t->ws;
    if (ws.base && ws.cap_n >= t->n && ws.cap_L >= L) return FSG_OK;
    const int64_t Lc = L > ws.cap_L ? L : ws.cap_L;
    size_t sz[kWsParts];
    workspace_sizes(t->n, t->d, t->dm, t->nb, Lc, sz);
    void** ptrs[kWsParts] = {
        (void**)&ws.binsum, (void**)&ws.degf, (void**)&ws.flags, (void**)&ws.leaf_pos, (void**)&ws.ksmp,
        (void**)&ws.lflags, (void**)&ws.qitem_bin, (void**)&ws.qitem_mask, (void**)&ws.qitem_cnt,
        (void**)&ws.bin_count, (void**)&ws.bin_cursor, (void**)&ws.bin_off, (void**)&ws.items_q,
        (void**)&ws.items_mask, (void**)&ws.leafv, (void**)&ws.uniq, (void**)&ws.uniq_w, (void**)&ws.ucnt,
        (void**)&ws.emit_mask, (void**)&ws.ecount, (void**)&ws.scan_tmp, (void**)&ws.stats, (void**)&ws.misc,
    };
    size_t offs[kWsParts];
    size_t off = 0;
    for (int k = 0; k < kWsParts; ++k) {
        offs[k] = off;
        off = align_up(off + sz[k], 256);
    }
    if (ws.base) {
        if (!t->pool) cudaStreamSynchronize(s);
        tree_free(t, ws.base);
        ws.base = nullptr;
    }
    void* base = nullptr;
    cudaError_t e = tree_malloc(t, &base, off, t->pool ? t->alloc_stream : s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ws.cap_n = ws.cap_L = 0;
        return status_of(e);
    }
    ws.base = base;
    ws.bytes = off;
    for (int k = 0; k < kWsParts; ++k) *ptrs[k] = static_cast<char*>(base) + offs[k];
    ws.cap_n = t->n;
    ws.cap_L = Lc;
    return FSG_OK;
}

// Device bytes a tree of n points in d dimensions and its workspace for L
// samples take (the geometry of build_tree_internal with automatic leaf_max).
size_t tree_bytes_estimate(int64_t n, int32_t d, int32_t L) {
    int leaf_max = 128;
    auto pick = [&](int lm) {
        int s0 = 0;
        while ((n + (int64_t(1) << s0) - 1) >> s0 > lm) ++s0;
        return s0;
    };
    int s0 = pick(leaf_max);
    while (s0 > 11 && leaf_max < 1024) { leaf_max *= 2; s0 = pick(leaf_max); }
    const int nb = 1 << s0;
    const int mmax = (int)((n + nb - 1) / nb);
    const int dm = ceil_log2_host(mmax);
    const int64_t n_pad = (n + 127) / 128 * 128;
    const int dp = (d + 3) & ~3;
    size_t tot = sizeof(float) * (size_t)n_pad * dp * (d <= kMaxFmaDim ? 3 : 1) + sizeof(int32_t) * 2 * (size_t)n +
                 sizeof(int32_t) * (size_t)(nb + 1) + 64;
    if (d > kMaxFmaDim && mmax <= 128) tot += generic_tile_bytes(n, d);
    size_t sz[kWsParts];
    workspace_sizes(n, d, dm, nb, L, sz);
    for (int k = 0; k < kWsParts; ++k) tot += align_up(sz[k], 256);
    return tot + 4096 * 8;
}

}  // namespace fsg

using namespace fsg;

extern "C" {

const char* fsg_version(void) { return "fsg-gb300 0.1 (sm_103a)"; }

const char* fsg_error_string(int status) {
    switch (status) {
        case FSG_OK: return "ok";
        case FSG_ERR_INVALID_ARG: return "invalid argument";
        case FSG_ERR_OOM: return "device allocation failed";
        case FSG_ERR_CUDA: return "CUDA runtime error";
        case FSG_ERR_TIMEOUT: return "a bounded device wait ran out";
        case FSG_ERR_UNSUPPORTED: return "option not supported for these sizes";
        case FSG_ERR_BUSY: return "no slot or memory budget available";
        case FSG_ERR_CAPACITY: return "output buffer too small";
        case FSG_ERR_SCRATCH: return "problem too large for the fixed scratch of fsg_degrees_noalloc";
        case FSG_ERR_CANCELLED: return "request cancelled";
        case FSG_ERR_BOUNDS: return "an index check of the bounds-checking build failed";
        default: return "unknown status";
    }
}

int fsg_build_tree(const float* d_points, int64_t n, int32_t d, const fsg_tree_opts* opts, void* stream,
                   fsg_tree** out) {
    return fsg::build_tree_internal(d_points, n, d, opts, (cudaStream_t)stream, nullptr, out);
}

}  // extern "C"

int fsg::build_tree_internal(const float* d_points, int64_t n, int32_t d, const fsg_tree_opts* opts, cudaStream_t s,
                             cudaMemPool_t pool, fsg_tree** out) {
    if (!out) return FSG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d_points || n < 1 || n > (int64_t)0x7fffffff - 4096 || d < 1 || d > 4096) return FSG_ERR_INVALID_ARG;
    int leaf_max = opts && opts->leaf_max ? opts->leaf_max : 0;
    if (leaf_max && (leaf_max < 64 || leaf_max > 1024 || (leaf_max & (leaf_max - 1)))) return FSG_ERR_INVALID_ARG;
    const int order = opts ? opts->order : FSG_ORDER_IDENTITY;
    if (order != FSG_ORDER_IDENTITY && order != FSG_ORDER_SPATIAL) return FSG_ERR_INVALID_ARG;
    if (order == FSG_ORDER_SPATIAL && opts->d_perm) return FSG_ERR_INVALID_ARG;
    const bool auto_leaf = leaf_max == 0;
    if (auto_leaf) leaf_max = 128;
    if (d > kMaxFmaDim && leaf_max < 128) leaf_max = 128;  // the d > 16 tiles assume bins of > 64 points
    auto pick = [&](int lm, int& s0) {
        s0 = 0;
        while ((n + (int64_t(1) << s0) - 1) >> s0 > lm) ++s0;
    };
    int s0 = 0;
    pick(leaf_max, s0);
    while (auto_leaf && s0 > 11 && leaf_max < 1024) { leaf_max *= 2; pick(leaf_max, s0); }
    if (s0 > 12) return FSG_ERR_UNSUPPORTED;
    fsg_tree* t = new (std::nothrow) fsg_tree();
    if (!t) return FSG_ERR_OOM;
    t->pool = pool;
    t->alloc_stream = s;
    t->n = n;
    t->d = d;
    t->dp = (d + 3) & ~3;
    t->depth = ceil_log2_host(n);
    t->leaf_max = leaf_max;
    t->s0 = s0;
    t->nb = 1 << s0;
    t->mmax = (int)((n + t->nb - 1) / t->nb);
    t->dm = ceil_log2_host(t->mmax);
    t->n_pad = (n + 127) / 128 * 128;
    cudaGetDevice(&t->device);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = tree_malloc(t, p, bytes, s);
    };
    alloc((void**)&t->Xt, sizeof(float) * (size_t)t->n_pad * t->dp);
    if (d <= kMaxFmaDim) alloc((void**)&t->Xdup, sizeof(float) * 2 * (size_t)t->n_pad * t->dp);
    alloc((void**)&t->perm, sizeof(int32_t) * (size_t)n);
    alloc((void**)&t->inv, sizeof(int32_t) * (size_t)n);
    alloc((void**)&t->bnd, sizeof(int32_t) * (size_t)(t->nb + 1));
    alloc((void**)&t->status, sizeof(int32_t) * 8);
    if (order == FSG_ORDER_SPATIAL) alloc(&t->ord, spatial_order_scratch_bytes(n, d));
    const int32_t* perm_in = opts ? opts->d_perm : nullptr;
    if (e == cudaSuccess && t->ord) e = launch_spatial_order(d_points, n, d, kSpatialLeaf, t->ord, &perm_in, s);
    if (e == cudaSuccess) {
        e = launch_tree_prep(t, d_points, perm_in, s);
        t->launches += 2;
    }
    int rc = status_of(e);
    if (rc == FSG_OK && d >= 64 && !pool) {
        // 8-bit data: prepare the tensor-core path (BF16 copy, norms, TMA maps)
        int32_t st[2] = {0, 0};
        e = cudaMemcpyAsync(st, t->status, sizeof(st), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rc = status_of(e);
        if (rc == FSG_OK && st[1] == 0) {
            t->exact_int = 1;
            rc = tc_prepare(t, s);
        }
    }
    if (rc == FSG_OK && opts && opts->d_perm) {
        // a caller-given order is validated before the tree is handed out
        int32_t st[2] = {0, 0};
        e = cudaMemcpyAsync(st, t->status, sizeof(st), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rc = status_of(e);
        if (rc == FSG_OK && st[0] != 0) rc = FSG_ERR_INVALID_ARG;
    }
    if (rc == FSG_OK && d > kMaxFmaDim && !t->exact_int && t->mmax <= 128) {
        // transposed tiles of the symmetric FP32 pass (allocated here, never during a capture)
        e = tree_malloc(t, (void**)&t->Xtt, generic_tile_bytes(n, d), s);
        rc = status_of(e);
    }
    if (rc != FSG_OK) {
        cudaGetLastError();
        fsg_free_tree(t);
        return rc;
    }
    *out = t;
    return FSG_OK;
}

extern "C" {

void fsg_free_tree(fsg_tree* t) {
    if (!t) return;
    for (int k = 0; k < FSG_NUM_PHASES; ++k) {
        if (t->ev_start[k]) cudaEventDestroy(t->ev_start[k]);
        if (t->ev_end[k]) cudaEventDestroy(t->ev_end[k]);
    }
    tree_free(t, t->Xt);
    tree_free(t, t->Xdup);
    tree_free(t, t->perm);
    tree_free(t, t->inv);
    tree_free(t, t->bnd);
    tree_free(t, t->status);
    tree_free(t, t->ws.base);
    tree_free(t, t->Xtt);
    tree_free(t, t->sboxes);
    tree_free(t, t->ord);
    tree_free(t, t->rs.base);
    tree_free(t, t->Xs);
    tree_free(t, t->snorms);
    if (t->Xb) cudaFree(t->Xb);
    if (t->norms) cudaFree(t->norms);
    delete t;
}

int fsg_tree_info(const fsg_tree* t, int64_t* n, int32_t* d, int32_t* depth) {
    if (!t) return FSG_ERR_INVALID_ARG;
    if (n) *n = t->n;
    if (d) *d = t->d;
    if (depth) *depth = t->depth;
    return FSG_OK;
}

static int run_sampling(fsg_tree* t, const KernelParams& kp, int schedule, double* d_deg, cudaStream_t s,
                        bool skip_bins = false);

namespace {
struct TuneKey {
    int64_t n;
    int32_t d, L, s0, mmax, path;
    bool operator<(const TuneKey& o) const {
        return std::tie(n, d, L, s0, mmax, path) < std::tie(o.n, o.d, o.L, o.s0, o.mmax, o.path);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, LaunchTuning> g_tune_cache;

void to_public(const LaunchTuning& lt, fsg_tuning* out) {
    if (!out) return;
    std::memset(out, 0, sizeof(*out));
    out->sym_bins = lt.sym_bins;
    out->tc_bins = lt.tc_bins;
    out->leaf_splits = lt.leaf_splits;
}
}  // namespace

int fsg_tree_tuning(fsg_tree* t, const fsg_tuning* tuning, fsg_tuning* out) {
    if (!t) return FSG_ERR_INVALID_ARG;
    if (tuning) {
        if (tuning->sym_bins < 0 || tuning->tc_bins < 0 || tuning->leaf_splits < 0 || tuning->leaf_splits > 65535)
            return FSG_ERR_INVALID_ARG;
        t->tune.sym_bins = tuning->sym_bins;
        t->tune.tc_bins = tuning->tc_bins;
        t->tune.leaf_splits = tuning->leaf_splits;
    }
    to_public(t->tune, out);
    return FSG_OK;
}

int fsg_autotune(fsg_tree* t, const fsg_params* p, int32_t L, uint64_t seed, int32_t reps, fsg_tuning* out,
                 void* stream) {
    if (!t || L < 1 || L > kMaxL || reps < 1 || reps > 100) return FSG_ERR_INVALID_ARG;
    int rc = check_params(p);
    if (rc != FSG_OK) return rc;
    if ((rc = check_path(t, p)) != FSG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_workspace(t, L, s)) != FSG_OK) return rc;
    if ((rc = ensure_split(t, p, s)) != FSG_OK) return rc;
    if (p->resolve && (rc = ensure_resolve(t, L, s)) != FSG_OK) return rc;
    if (p->schedule != FSG_SCHED_FUSED) {  // the levelwise schedule has no shapes to choose
        to_public(t->tune, out);
        return FSG_OK;
    }
    const bool tc = use_tc(t, eff_precision(p)) || use_splitk(t, eff_precision(p));
    const int path = use_splitk(t, eff_precision(p)) ? 3 : tc ? 2
                     : (t->d <= kMaxFmaDim && kde_bins_sym_supported(t)) ? 1 : 0;
    const TuneKey key{t->n, t->d, L, t->s0, t->mmax, path};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            t->tune = it->second;
            to_public(t->tune, out);
            return FSG_OK;
        }
    }
    const KernelParams kp = make_kernel_params(p, L, seed);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const bool was_profiling = t->profiling;
    t->profiling = false;
    // best of `reps` runs of fn(), in ms (a huge value on a CUDA error)
    auto time_it = [&](auto fn) -> float {
        float best = 1e30f;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = fn();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best) best = ms;
        }
        return best;
    };
    LaunchTuning best = t->tune;
    if (e == cudaSuccess && path != 0) {
        std::vector<int> cand;
        if (path == 1) {
            const int gmax = 256 / ((t->mmax + 3) / 4);
            for (int g : {4, 6, 8, 10, 12, 14, 16})
                if (g <= gmax) cand.push_back(g);
        } else {
            for (int g : {8, 12, 16, 20, 24}) cand.push_back(g);
        }
        float tbest = 1e30f;
        for (int g : cand) {
            if (path == 1) t->tune.sym_bins = g; else t->tune.tc_bins = g;
            const float ms = time_it([&] { return run_kde_bins(t, kp, s); });
            if (ms < tbest) {
                tbest = ms;
                if (path == 1) best.sym_bins = g; else best.tc_bins = g;
            }
        }
        t->tune = best;
    }
    if (e == cudaSuccess) {  // leaf finish: one full sampling pass sets up its inputs
        begin_call(t);
        rc = run_sampling(t, kp, FSG_SCHED_FUSED, nullptr, s);
        if (rc != FSG_OK) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) {
        const int64_t items_est = t->n * (int64_t)(L < t->nb ? L : t->nb);
        const bool fused_tc = t->d > kMaxFmaDim && tc && (1 << t->dm) <= 256;  // the heuristics of each launcher
        int64_t S0 = leaf_default_splits(t, L);
        if (fused_tc) {
            S0 = (152 * 2 * 8 + t->nb - 1) / t->nb;
            const int64_t cpb = (items_est / t->nb + 127) / 128 + 1;
            if (S0 > cpb) S0 = cpb;
            if (S0 < 1) S0 = 1;
        }
        float tbest = 1e30f;
        for (int64_t S : {S0 / 4, S0 / 2, S0, 2 * S0, 4 * S0}) {
            if (S < 1 || S > 65535) continue;
            t->tune.leaf_splits = (int32_t)S;
            const float ms = time_it([&] { return run_leaf_phase(t, kp, s); });
            if (ms < tbest) {
                tbest = ms;
                best.leaf_splits = (int32_t)S;
            }
        }
        t->tune = best;
    }
    t->profiling = was_profiling;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != FSG_OK) return rc;
    if (e != cudaSuccess) return status_of(e);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = best;
    }
    to_public(best, out);
    return FSG_OK;
}

int fsg_bin_pass_evals(const fsg_tree* t, const fsg_params* p, int64_t* evals) {
    if (!t || !evals) return FSG_ERR_INVALID_ARG;
    const int rc = check_params(p);
    if (rc != FSG_OK) return rc;
    *evals = p->schedule != FSG_SCHED_FUSED ? 0 : bin_pass_evals(t, eff_precision(p));
    return FSG_OK;
}

int fsg_tree_update(fsg_tree* t, const float* d_points, void* stream) {
    if (!t || !d_points) return FSG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    begin_call(t);
    PhaseScope ph(t, FSG_PHASE_TREE, s);
    // the stored order is reused (tree_prep reads perm[p] before rewriting
    // it), or, for FSG_ORDER_SPATIAL, computed again from the new points
    const int32_t* perm_in = t->perm;
    cudaError_t e = cudaSuccess;
    if (t->ord) e = launch_spatial_order(d_points, t->n, t->d, kSpatialLeaf, t->ord, &perm_in, s);
    if (e == cudaSuccess) e = launch_tree_prep(t, d_points, perm_in, s);
    t->launches += 2;
    int rc = status_of(e);
    if (rc == FSG_OK && t->Xb) {  // refresh the tensor-core copy (exactness re-checked on the device)
        rc = tc_prepare(t, s);
        t->launches += 1;
    }
    if (rc == FSG_OK && t->Xs) {  // refresh the split form's three-part image
        rc = splitk_prepare(t, s);
        t->launches += 1;
    }
    return rc;
}

int fsg_tree_perm(const fsg_tree* t, int32_t* d_perm_out, void* stream) {
    if (!t || !d_perm_out) return FSG_ERR_INVALID_ARG;
    return status_of(cudaMemcpyAsync(d_perm_out, t->perm, sizeof(int32_t) * (size_t)t->n, cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream));
}

int fsg_profile(fsg_tree* t, int enable) {
    if (!t) return FSG_ERR_INVALID_ARG;
    if (enable && !t->ev_start[0]) {
        for (int k = 0; k < FSG_NUM_PHASES; ++k) {
            if (cudaEventCreate(&t->ev_start[k]) != cudaSuccess || cudaEventCreate(&t->ev_end[k]) != cudaSuccess)
                return FSG_ERR_CUDA;
        }
    }
    t->profiling = enable != 0;
    return FSG_OK;
}

int fsg_profile_read(fsg_tree* t, float* ms, int64_t* launches) {
    if (!t) return FSG_ERR_INVALID_ARG;
    if (launches) *launches = t->launches;
    if (!ms) return FSG_OK;
    for (int k = 0; k < FSG_NUM_PHASES; ++k) {
        ms[k] = 0.f;
        if (t->ev_used[k] && t->ev_start[k]) {
            if (cudaEventSynchronize(t->ev_end[k]) != cudaSuccess) return FSG_ERR_CUDA;
            if (cudaEventElapsedTime(&ms[k], t->ev_start[k], t->ev_end[k]) != cudaSuccess) return FSG_ERR_CUDA;
        }
    }
    return FSG_OK;
}

static int run_sampling(fsg_tree* t, const KernelParams& kp, int schedule, double* d_deg, cudaStream_t s,
                        bool skip_bins) {
    Workspace& ws = t->ws;
    if (schedule != FSG_SCHED_FUSED) {
        cudaError_t e = cudaMemsetAsync(ws.stats, 0, sizeof(fsg_stats), s);
        if (e == cudaSuccess) {
            PhaseScope ph(t, FSG_PHASE_KDE_BINS, s);
            e = launch_levelwise(t, kp, d_deg, 1, schedule == FSG_SCHED_CARRIED, s, &t->launches);
        }
        return status_of(e);
    }
    cudaError_t e = cudaMemsetAsync(ws.bin_count, 0, sizeof(int32_t) * t->nb * kBinSlots, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.bin_cursor, 0, sizeof(int32_t) * t->nb * kBinSlots, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.stats, 0, sizeof(fsg_stats), s);
    if (e == cudaSuccess && !skip_bins) {
        PhaseScope ph(t, FSG_PHASE_KDE_BINS, s);
        e = run_kde_bins(t, kp, s);
        t->launches += 1;
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_DESCEND_TOP, s);
        e = launch_descend_top(t, kp, d_deg, 1, s);
        t->launches += 1;
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_BUCKET, s);
        e = launch_bucket(t, kp, s);
        t->launches += 2;
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_LEAF, s);
        e = run_leaf_phase(t, kp, s);
    }
    if (e == cudaSuccess && kp.resolve) {
        PhaseScope ph(t, FSG_PHASE_RESOLVE, s);
        e = launch_resolve(t, kp, s);
        t->launches += 8;
    }
    return status_of(e);
}

// Evaluations of the bin pass (every query against every point), counted on
// the host; the levelwise schedule and the split pass for d <= 64 (which
// skips tiles) count their own on the device.
static int64_t bin_evals(const fsg_tree* t, const fsg_params* p) {
    if (p->schedule != FSG_SCHED_FUSED || (p->precision == FSG_PREC_SPLIT_BF16 && !use_splitk(t, p->precision)))
        return 0;
    return bin_pass_evals(t, eff_precision(p));
}

// Statistics known on the host: samples run, bin-pass evaluations.
// (keep_resolved: n_resolved was accumulated by the steps of a stepped build)
__global__ static void stats_finish_kernel(fsg_stats* st, int64_t n_samples, int64_t bin_evals,
                                           const int32_t* status, const int32_t* n_resolved, fsg_stats* out,
                                           int keep_resolved = 0) {
    st->n_samples = n_samples;
    st->n_evals += bin_evals;       // the split pass for d <= 64 counts its own on the device
    st->n_bin_evals += bin_evals;
    st->status = status[0];
    if (!keep_resolved) st->n_resolved = n_resolved ? *n_resolved : 0;
    if (out) *out = *st;
}

// A stepped build: the samples one step re-decided, added to the statistics.
__global__ static void add_resolved_kernel(fsg_stats* st, const int32_t* cnt) { st->n_resolved += cnt[0]; }

// A stepped build: every position's FP32 degree to the caller's array in
// original index order (the value descend_top writes in a whole build).
__global__ static void degrees_out_kernel(const float* __restrict__ degf, const int32_t* __restrict__ perm,
                                          int64_t n, double* __restrict__ d_deg) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        d_deg[perm[q]] = (double)degf[q];
}

int fsg_degrees(fsg_tree* t, const fsg_params* p, double* d_deg, void* stream) {
    if (!t || !d_deg) return FSG_ERR_INVALID_ARG;
    int rc = check_params(p);
    if (rc != FSG_OK) return rc;
    if ((rc = check_path(t, p)) != FSG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_workspace(t, 1, s)) != FSG_OK) return rc;
    if ((rc = ensure_split(t, p, s)) != FSG_OK) return rc;
    const KernelParams kp = make_kernel_params(p, 1, 0);
    begin_call(t);
    cudaError_t e;
    if (p->schedule != FSG_SCHED_FUSED) {  // both levelwise schedules: the root pass
        e = cudaMemsetAsync(t->ws.stats, 0, sizeof(fsg_stats), s);
        PhaseScope ph(t, FSG_PHASE_KDE_BINS, s);
        if (e == cudaSuccess) e = launch_levelwise(t, kp, d_deg, 0, 0, s, &t->launches);
        return status_of(e);
    }
    {
        PhaseScope ph(t, FSG_PHASE_KDE_BINS, s);
        e = run_kde_bins(t, kp, s);
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_DESCEND_TOP, s);
        e = launch_descend_top(t, kp, d_deg, 0, s);
    }
    t->launches += 2;
    return status_of(e);
}

int fsg_sample_edges(fsg_tree* t, const fsg_params* p, int32_t L, uint64_t seed, int32_t* d_samples,
                     uint8_t* d_flags, void* stream) {
    if (!t || !d_samples || L < 1 || L > kMaxL) return FSG_ERR_INVALID_ARG;
    int rc = check_params(p);
    if (rc != FSG_OK) return rc;
    if ((rc = check_path(t, p)) != FSG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_workspace(t, L, s)) != FSG_OK) return rc;
    if ((rc = ensure_split(t, p, s)) != FSG_OK) return rc;
    if (p->resolve && (rc = ensure_resolve(t, L, s)) != FSG_OK) return rc;
    const KernelParams kp = make_kernel_params(p, L, seed);
    begin_call(t);
    if ((rc = run_sampling(t, kp, p->schedule, nullptr, s)) != FSG_OK) return rc;
    cudaError_t e;
    {
        PhaseScope ph(t, FSG_PHASE_OUTPUTS, s);
        e = launch_outputs(t, kp, d_samples, d_flags, nullptr, s);
        if (e == cudaSuccess) {
            stats_finish_kernel<<<1, 1, 0, s>>>(t->ws.stats, t->n * L, bin_evals(t, p), t->status,
                                                p->resolve ? t->rs.cnt : nullptr, nullptr);
            e = cudaGetLastError();
        }
        t->launches += 2;
    }
    return status_of(e);
}

int fsg_build_graph(fsg_tree* t, const fsg_params* p, int32_t L, uint64_t seed, int32_t edge_mode, int32_t* d_src,
                    int32_t* d_dst, void* d_w, int64_t cap, int64_t* d_m_out, double* d_deg, int32_t* d_samples,
                    uint8_t* d_flags, fsg_stats* d_stats, void* stream) {
    return fsg::build_graph_internal(t, p, L, seed, edge_mode, d_src, d_dst, d_w, cap, d_m_out, d_deg, d_samples,
                                     d_flags, d_stats, (cudaStream_t)stream, false);
}

// Stepped build: the bin pass of every query, kept in the tree's workspace.
int fsg_graph_begin(fsg_tree* t, const fsg_params* p, int32_t L, uint64_t seed, void* stream) {
    if (!t || L < 1 || L > kMaxL) return FSG_ERR_INVALID_ARG;
    int rc = check_params(p);
    if (rc != FSG_OK) return rc;
    if ((rc = check_path(t, p)) != FSG_OK) return rc;
    if (p->schedule != FSG_SCHED_FUSED) return FSG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_workspace(t, L, s)) != FSG_OK) return rc;
    if ((rc = ensure_split(t, p, s)) != FSG_OK) return rc;
    if (p->resolve && (rc = ensure_resolve(t, L, s)) != FSG_OK) return rc;
    const KernelParams kp = make_kernel_params(p, L, seed);
    begin_call(t);  // ends any earlier run
    cudaError_t e = cudaMemsetAsync(t->ws.stats, 0, sizeof(fsg_stats), s);
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_KDE_BINS, s);
        e = run_kde_bins(t, kp, s);
        t->launches += 1;
    }
    if (e != cudaSuccess) return status_of(e);
    t->run.p = *p;
    t->run.L = L;
    t->run.seed = seed;
    t->run.done.clear();
    t->run.active = true;
    return FSG_OK;
}

// Stepped build: sampling of the queries at tree positions [q0, q1).
int fsg_graph_step(fsg_tree* t, int64_t q0, int64_t q1, void* stream) {
    if (!t || !t->run.active || q0 < 0 || q1 > t->n || q0 >= q1) return FSG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const fsg_params& p = t->run.p;
    const KernelParams kp = make_kernel_params(&p, t->run.L, t->run.seed);
    Workspace& ws = t->ws;
    cudaError_t e = cudaMemsetAsync(ws.bin_count, 0, sizeof(int32_t) * t->nb * kBinSlots, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.bin_cursor, 0, sizeof(int32_t) * t->nb * kBinSlots, s);
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_DESCEND_TOP, s);
        e = launch_descend_top(t, kp, nullptr, 1, s, q0, q1);
        t->launches += 1;
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_BUCKET, s);
        e = launch_bucket(t, kp, s, q0, q1);
        t->launches += 2;
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_LEAF, s);
        e = run_leaf_phase(t, kp, s);
    }
    if (e == cudaSuccess && kp.resolve) {
        PhaseScope ph(t, FSG_PHASE_RESOLVE, s);
        e = launch_resolve(t, kp, s, q0, q1);
        if (e == cudaSuccess) {
            add_resolved_kernel<<<1, 1, 0, s>>>(ws.stats, t->rs.cnt);
            e = cudaGetLastError();
        }
        t->launches += 9;
    }
    if (e != cudaSuccess) return status_of(e);
    // record [q0, q1) among the stepped ranges (sorted, merged)
    auto& done = t->run.done;
    done.emplace_back(q0, q1);
    std::sort(done.begin(), done.end());
    std::vector<std::pair<int64_t, int64_t>> merged;
    for (const auto& r : done) {
        if (!merged.empty() && r.first <= merged.back().second)
            merged.back().second = std::max(merged.back().second, r.second);
        else
            merged.push_back(r);
    }
    done.swap(merged);
    return FSG_OK;
}

int fsg_graph_cursor(const fsg_tree* t, int64_t* cursor) {
    if (!t || !cursor || !t->run.active) return FSG_ERR_INVALID_ARG;
    const auto& done = t->run.done;
    *cursor = (done.empty() || done[0].first > 0) ? 0 : done[0].second;
    return FSG_OK;
}

// Stepped build: the edge list and outputs once every position was stepped.
int fsg_graph_end(fsg_tree* t, int32_t edge_mode, int32_t* d_src, int32_t* d_dst, void* d_w, int64_t cap,
                  int64_t* d_m_out, double* d_deg, int32_t* d_samples, uint8_t* d_flags, fsg_stats* d_stats,
                  void* stream) {
    if (!t || !t->run.active || !d_src || !d_dst || !d_w || !d_m_out) return FSG_ERR_INVALID_ARG;
    if (edge_mode != FSG_EDGES_SET && edge_mode != FSG_EDGES_MULTI) return FSG_ERR_INVALID_ARG;
    const int32_t L = t->run.L;
    if (cap < t->n * (int64_t)L) return FSG_ERR_CAPACITY;
    const auto& done = t->run.done;
    if (done.size() != 1 || done[0].first != 0 || done[0].second != t->n) return FSG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const fsg_params& p = t->run.p;
    const KernelParams kp = make_kernel_params(&p, L, t->run.seed);
    cudaError_t e;
    {
        PhaseScope ph(t, FSG_PHASE_EDGES, s);
        e = launch_edges(t, kp, edge_mode, d_src, d_dst, d_w, cap, d_m_out, s);
        t->launches += edge_mode == FSG_EDGES_SET ? 6 : 5;
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_OUTPUTS, s);
        e = launch_outputs(t, kp, d_samples, d_flags, d_stats, s);
        if (e == cudaSuccess && d_deg) {
            int64_t blocks = (t->n + 255) / 256;
            if (blocks > 152 * 8) blocks = 152 * 8;
            degrees_out_kernel<<<(int)blocks, 256, 0, s>>>(t->ws.degf, t->perm, t->n, d_deg);
            e = cudaGetLastError();
            t->launches += 1;
        }
        if (e == cudaSuccess) {
            stats_finish_kernel<<<1, 1, 0, s>>>(t->ws.stats, t->n * L, bin_evals(t, &p), t->status, nullptr, d_stats,
                                                1);
            e = cudaGetLastError();
        }
        t->launches += 2;
    }
    if (e == cudaSuccess) t->run.active = false;
    return status_of(e);
}

}  // extern "C"

int fsg::check_graph_call(const fsg_tree* t, const fsg_params* p) {
    const int rc = check_params(p);
    return rc != FSG_OK ? rc : check_path(t, p);
}

fsg::KernelParams fsg::kernel_params_of(const fsg_params* p, int L, uint64_t seed) {
    return make_kernel_params(p, L, seed);
}

int fsg::build_graph_internal(fsg_tree* t, const fsg_params* p, int32_t L, uint64_t seed, int32_t edge_mode,
                              int32_t* d_src, int32_t* d_dst, void* d_w, int64_t cap, int64_t* d_m_out,
                              double* d_deg, int32_t* d_samples, uint8_t* d_flags, fsg_stats* d_stats,
                              cudaStream_t s, bool skip_bins) {
    if (!t || L < 1 || L > kMaxL || !d_src || !d_dst || !d_w || !d_m_out) return FSG_ERR_INVALID_ARG;
    if (edge_mode != FSG_EDGES_SET && edge_mode != FSG_EDGES_MULTI) return FSG_ERR_INVALID_ARG;
    if (cap < t->n * (int64_t)L) return FSG_ERR_CAPACITY;
    int rc = check_params(p);
    if (rc != FSG_OK) return rc;
    if ((rc = check_path(t, p)) != FSG_OK) return rc;
    if ((rc = ensure_workspace(t, L, s)) != FSG_OK) return rc;
    if ((rc = ensure_split(t, p, s)) != FSG_OK) return rc;
    if (p->resolve && (rc = ensure_resolve(t, L, s)) != FSG_OK) return rc;
    const KernelParams kp = make_kernel_params(p, L, seed);
    begin_call(t);
    if ((rc = run_sampling(t, kp, p->schedule, d_deg, s, skip_bins)) != FSG_OK) return rc;
    cudaError_t e;
    {
        PhaseScope ph(t, FSG_PHASE_EDGES, s);
        e = launch_edges(t, kp, edge_mode, d_src, d_dst, d_w, cap, d_m_out, s);
        t->launches += edge_mode == FSG_EDGES_SET ? 6 : 5;
    }
    if (e == cudaSuccess) {
        PhaseScope ph(t, FSG_PHASE_OUTPUTS, s);
        e = launch_outputs(t, kp, d_samples, d_flags, d_stats, s);
        if (e == cudaSuccess) {
            stats_finish_kernel<<<1, 1, 0, s>>>(t->ws.stats, t->n * L, bin_evals(t, p), t->status,
                                                p->resolve ? t->rs.cnt : nullptr, d_stats);
            e = cudaGetLastError();
        }
        t->launches += 2;
    }
    return status_of(e);
}

extern "C" {

int fsg_bounds_error(int64_t* out) {
    if (!out) return FSG_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) out[k] = 0;
#ifdef FSG_BOUNDS_CHECK
    if (cudaDeviceSynchronize() != cudaSuccess) return FSG_ERR_CUDA;
    int (*readers[])(long long*) = {bounds_read_fma, bounds_read_descend, bounds_read_tc, bounds_read_resolve};
    for (auto rd : readers) {
        long long v[4] = {0, 0, 0, 0};
        const int r = rd(v);
        if (r < 0) return FSG_ERR_CUDA;
        if (r > 0 && out[0] == 0)
            for (int k = 0; k < 4; ++k) out[k] = v[k];
    }
    return FSG_OK;
#else
    return FSG_ERR_UNSUPPORTED;
#endif
}

int fsg_sync(fsg_tree* t, void* stream) {
    if (!t) return FSG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_of(e);
#ifdef FSG_BOUNDS_CHECK
    {
        int64_t be[4];
        const int rb = fsg_bounds_error(be);
        if (rb != FSG_OK) return rb;
        if (be[0]) return FSG_ERR_BOUNDS;
    }
#endif
    if (st != 0) {
        cudaMemsetAsync(t->status, 0, sizeof(int32_t), s);
        cudaStreamSynchronize(s);
        return st;
    }
    return FSG_OK;
}

// ---------------------------------------------------------------------------
// Host-buffer entry point: device buffers cached per calling thread.
// ---------------------------------------------------------------------------
namespace {
struct HostCache {
    float* d_points = nullptr;
    int32_t* d_src = nullptr;
    int32_t* d_dst = nullptr;
    float* d_w = nullptr;
    int64_t* d_m = nullptr;
    int64_t cap_pts = 0, cap_edges = 0;
    fsg_tree* tree = nullptr;  // reused while (n, d) stay the same
    ~HostCache() {
        fsg_free_tree(tree);
        cudaFree(d_points); cudaFree(d_src); cudaFree(d_dst); cudaFree(d_w); cudaFree(d_m);
    }
};
thread_local HostCache g_host_cache;
}  // namespace

int fsg_build_graph_host(const float* h_points, int64_t n, int32_t d, const fsg_params* p, int32_t L, uint64_t seed,
                         int32_t edge_mode, int32_t* h_src, int32_t* h_dst, float* h_w, int64_t cap,
                         int64_t* h_m_out, void* stream) {
    if (!h_points || !h_src || !h_dst || !h_w || !h_m_out || n < 1 || d < 1 || L < 1 || L > kMaxL)
        return FSG_ERR_INVALID_ARG;
    if (p && p->weight_f64) return FSG_ERR_INVALID_ARG;  // h_w is float32
    if (cap < n * (int64_t)L) return FSG_ERR_CAPACITY;
    int rc = check_params(p);
    if (rc != FSG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    HostCache& hc = g_host_cache;
    cudaError_t e = cudaSuccess;
    if (hc.cap_pts < n * (int64_t)d) {
        cudaFree(hc.d_points);
        hc.d_points = nullptr;
        hc.cap_pts = 0;
        e = cudaMalloc(&hc.d_points, sizeof(float) * (size_t)n * d);
        if (e != cudaSuccess) return status_of(e);
        hc.cap_pts = n * (int64_t)d;
    }
    const int64_t ecap = n * (int64_t)L;
    if (hc.cap_edges < ecap) {
        cudaFree(hc.d_src); cudaFree(hc.d_dst); cudaFree(hc.d_w); cudaFree(hc.d_m);
        hc.d_src = hc.d_dst = nullptr; hc.d_w = nullptr; hc.d_m = nullptr; hc.cap_edges = 0;
        e = cudaMalloc(&hc.d_src, sizeof(int32_t) * (size_t)ecap);
        if (e == cudaSuccess) e = cudaMalloc(&hc.d_dst, sizeof(int32_t) * (size_t)ecap);
        if (e == cudaSuccess) e = cudaMalloc(&hc.d_w, sizeof(float) * (size_t)ecap);
        if (e == cudaSuccess) e = cudaMalloc(&hc.d_m, sizeof(int64_t));
        if (e != cudaSuccess) return status_of(e);
        hc.cap_edges = ecap;
    }
    e = cudaMemcpyAsync(hc.d_points, h_points, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return status_of(e);
    // the split form up to d = 64 takes the spatial tree order (compact tiles
    // for its centring; above d = 64 it centres nothing)
    const bool spatial = p->precision == FSG_PREC_SPLIT_BF16 && d <= 64;
    fsg_tree* t = hc.tree;
    if (t && t->n == n && t->d == d && (t->ord != nullptr) == spatial) {
        rc = fsg_tree_update(t, hc.d_points, stream);
        if (rc != FSG_OK) return rc;
    } else {
        fsg_free_tree(hc.tree);
        hc.tree = nullptr;
        fsg_tree_opts o{};
        o.order = spatial ? FSG_ORDER_SPATIAL : FSG_ORDER_IDENTITY;
        rc = fsg_build_tree(hc.d_points, n, d, &o, stream, &t);
        if (rc != FSG_OK) return rc;
        hc.tree = t;
    }
    rc = fsg_build_graph(t, p, L, seed, edge_mode, hc.d_src, hc.d_dst, hc.d_w, ecap, hc.d_m, nullptr, nullptr,
                         nullptr, nullptr, stream);
    int64_t m = 0;
    if (rc == FSG_OK) {
        e = cudaMemcpyAsync(&m, hc.d_m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rc = status_of(e);
    }
    if (rc == FSG_OK) {
        if (m > cap) m = cap;
        e = cudaMemcpyAsync(h_src, hc.d_src, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_dst, hc.d_dst, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_w, hc.d_w, sizeof(float) * (size_t)m, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rc = status_of(e);
        *h_m_out = m;
    }
    if (rc == FSG_OK) rc = fsg_sync(t, stream);
    return rc;
}

}  // extern "C"
