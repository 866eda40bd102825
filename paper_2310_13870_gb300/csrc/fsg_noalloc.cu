// Allocation-free degree computation (fsg_degrees_noalloc): the same bin
// pass and per-query sums as fsg_degrees, with every scratch array carved out
// of one statically sized __device__ array instead of cudaMalloc'ed memory.
// For callers that must not allocate device memory (their pool allocator
// owns the device, or they cannot afford cudaMalloc's synchronization).
#include <cmath>
#include <mutex>

#include "fsg_internal.cuh"

namespace {

// The scratch.  In host code `g_noalloc_scratch` names a host-side stand-in,
// not device memory: kernels only ever receive the device address looked up
// by cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FSG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
int noalloc_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSG_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FSG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return FSG_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FSG_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// The caller's only view of a device-side failure: when a bounded wait of the
// bin pass ran out (status word set), every degree of the call becomes NaN.
__global__ void noalloc_finish_kernel(const int32_t* __restrict__ status, int64_t n, double* __restrict__ d_deg) {
    if (status[0] == FSG_OK) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d_deg[i] = nan;
}

// Scratch layout for n points of dimension d with nb bins.
struct NoallocLayout {
    size_t xt, xdup, perm, inv, bnd, binsum, degf, status, total;
    NoallocLayout(int64_t n, int64_t n_pad, int dp, int nb) {
        xt = 0;
        xdup = up256(xt + sizeof(float) * (size_t)n_pad * dp);
        perm = up256(xdup + sizeof(float) * 2 * (size_t)n_pad * dp);
        inv = up256(perm + sizeof(int32_t) * (size_t)n);
        bnd = up256(inv + sizeof(int32_t) * (size_t)n);
        binsum = up256(bnd + sizeof(int32_t) * (size_t)(nb + 1));
        degf = up256(binsum + sizeof(float) * (size_t)n * nb);
        status = up256(degf + sizeof(float) * (size_t)n);
        total = up256(status + sizeof(int32_t) * 8);
    }
};

}  // namespace

extern "C" int fsg_degrees_noalloc(const float* d_points, int64_t n, int32_t d, const fsg_params* p, double* d_deg,
                                   void* stream) {
    if (!d_points || !d_deg || !p || n < 1 || n > (int64_t)0x7fffffff - 4096 || d < 1) return FSG_ERR_INVALID_ARG;
    if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return FSG_ERR_INVALID_ARG;
    if (p->scale_conv != FSG_TWO_SIGMA_SQ && p->scale_conv != FSG_SIGMA_SQ) return FSG_ERR_INVALID_ARG;
    if (p->self_mode != FSG_SELF_EXCLUDE && p->self_mode != FSG_SELF_INCLUDE) return FSG_ERR_INVALID_ARG;
    if (!(p->kde_eps >= 0.f) || !std::isfinite(p->kde_eps) || p->kde_eps > 0.5f) return FSG_ERR_INVALID_ARG;
    if (p->kernel != FSG_KERNEL_GAUSSIAN && p->kernel != FSG_KERNEL_LAPLACIAN && p->kernel != FSG_KERNEL_EXPONENTIAL)
        return FSG_ERR_INVALID_ARG;
    // the exact FP32 pass of the Gaussian kernel only
    if (d > fsg::kMaxFmaDim || p->kde_eps > 0.f || p->kernel != FSG_KERNEL_GAUSSIAN) return FSG_ERR_UNSUPPORTED;
    // Geometry: 16 bins (or fewer for tiny n) only to spread the bin pass over
    // the GPU; the degree is the sum of a query's bins.
    int s0 = 0;
    while (s0 < 4 && (int64_t(1) << (s0 + 1)) <= n) ++s0;
    const int nb = 1 << s0;
    const int dp = (d + 3) & ~3;
    const int64_t n_pad = (n + 127) / 128 * 128;
    const NoallocLayout lay(n, n_pad, dp, nb);
    if (lay.total > (size_t)FSG_NOALLOC_SCRATCH_BYTES) return FSG_ERR_SCRATCH;
    void* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != FSG_OK) return rc;
    char* base = static_cast<char*>(scratch);

    fsg_tree t;  // host description only: every pointer is into the scratch
    t.n = n;
    t.d = d;
    t.dp = dp;
    t.depth = fsg::ceil_log2_host(n);
    t.s0 = s0;
    t.nb = nb;
    t.mmax = (int)((n + nb - 1) / nb);
    t.dm = fsg::ceil_log2_host(t.mmax);
    t.leaf_max = t.mmax;
    t.n_pad = n_pad;
    cudaGetDevice(&t.device);
    t.Xt = reinterpret_cast<float*>(base + lay.xt);
    t.Xdup = reinterpret_cast<float*>(base + lay.xdup);
    t.perm = reinterpret_cast<int32_t*>(base + lay.perm);
    t.inv = reinterpret_cast<int32_t*>(base + lay.inv);
    t.bnd = reinterpret_cast<int32_t*>(base + lay.bnd);
    t.status = reinterpret_cast<int32_t*>(base + lay.status);
    t.ws.binsum = reinterpret_cast<float*>(base + lay.binsum);
    t.ws.degf = reinterpret_cast<float*>(base + lay.degf);

    const double gamma = p->scale_conv == FSG_SIGMA_SQ ? 1.0 / (p->sigma * p->sigma)
                                                       : 1.0 / (2.0 * p->sigma * p->sigma);
    fsg::KernelParams kp{};
    kp.family = FSG_KERNEL_GAUSSIAN;
    kp.kde_eps = 0.f;
    kp.precision = FSG_PREC_FP32;
    kp.gamma = (float)gamma;
    kp.neg_c = (float)(-gamma * 1.4426950408889634073599246810019);
    if (kp.neg_c > -1e-30f) kp.neg_c = -1e-30f;
    kp.self_exclude = p->self_mode == FSG_SELF_EXCLUDE ? 1 : 0;
    kp.L = 1;
    kp.seed = 0;
    kp.flag_eps = 0x1p-13f;

    cudaStream_t s = (cudaStream_t)stream;
    // tree_prep clears the inverse map and the status word it reuses; the bin
    // pass writes every (query, bin) entry and descend_top every degree; the
    // last kernel turns a timed-out bin pass into NaN degrees.
    cudaError_t e = fsg::launch_tree_prep(&t, d_points, nullptr, s);
    if (e == cudaSuccess) e = fsg::launch_kde_bins(&t, kp, s);
    if (e == cudaSuccess) e = fsg::launch_descend_top(&t, kp, d_deg, 0, s);
    if (e == cudaSuccess) {
        const int64_t blocks = (n + 255) / 256;
        noalloc_finish_kernel<<<(int)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(t.status, n, d_deg);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? FSG_ERR_OOM : FSG_ERR_CUDA;
    }
    return FSG_OK;
}
