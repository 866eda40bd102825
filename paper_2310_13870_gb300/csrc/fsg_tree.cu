// Tree build: points gathered into tree order (so every node of the halving
// tree of Sec. 4.1 is a contiguous range of positions), padded to a multiple
// of four coordinates, plus the position<->index maps and the boundaries of
// the nodes at the bin level s0.
#include "fsg_internal.cuh"

namespace fsg {
namespace {

// One warp per tree position p (lanes over the padded coordinates): row
// perm_in[p] of X into row p of Xt (and of Xdup, each value twice), the
// position<->index maps, and the 8-bit test of the tensor-core path (one
// flag write per warp, not per value).
__global__ void tree_prep_kernel(const float* __restrict__ X, int64_t n, int d, int dp,
                                 const int32_t* __restrict__ perm_in, int32_t* __restrict__ perm,
                                 int32_t* __restrict__ inv, float* __restrict__ Xt, float* __restrict__ Xdup,
                                 int64_t n_pad, int32_t* __restrict__ status, int32_t* __restrict__ not_exact) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    bool inexact = false;
    for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < n_pad; p += warps) {
        int64_t j = -1;
        if (p < n) {
            j = perm_in ? (int64_t)perm_in[p] : p;
            if (j < 0 || j >= n) {  // not a permutation: record and read nothing
                if (lane == 0) atomicExch(status, FSG_ERR_INVALID_ARG);
                j = -1;
            }
            if (lane == 0) {
                perm[p] = (int32_t)j;
                if (j >= 0 && atomicExch(&inv[j], (int32_t)p) != -1) atomicExch(status, FSG_ERR_INVALID_ARG);
            }
        }
        const float* xr = X + (j >= 0 ? j : 0) * (int64_t)d;
        float* tr = Xt + p * (int64_t)dp;
        for (int t = lane; t < dp; t += 32) {
            float v = 0.f;
            if (t < d && j >= 0) {
                v = xr[t];
                // 8-bit test for the tensor-core path: v within float rounding of k/255, 0 <= k <= 255
                const float sv = v * 255.f;
                if (!(v >= 0.f && v <= 1.f && fabsf(sv - rintf(sv)) <= 1e-3f)) inexact = true;
            }
            tr[t] = v;
            if (Xdup) reinterpret_cast<float2*>(Xdup)[p * (int64_t)dp + t] = make_float2(v, v);
        }
    }
    if (__any_sync(0xffffffffu, inexact) && lane == 0) *not_exact = 1;
}

// Boundary b of level s0: walk s0 halvings from the root, left = floor(size/2).
__global__ void bounds_kernel(int64_t n, int s0, int nb, int32_t* __restrict__ bnd) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nb) return;
    if (b == nb) { bnd[b] = (int32_t)n; return; }
    int64_t lo = 0, hi = n;
    for (int t = s0 - 1; t >= 0; --t) {
        const int64_t mid = lo + (hi - lo) / 2;
        if ((b >> t) & 1) lo = mid; else hi = mid;
    }
    bnd[b] = (int32_t)lo;
}

}  // namespace

cudaError_t launch_tree_prep(fsg_tree* t, const float* d_points, const int32_t* d_perm, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(t->inv, 0xff, sizeof(int32_t) * t->n, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(t->status, 0, sizeof(int32_t) * 2, s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (t->n_pad + 7) / 8;  // 8 warps of 256 threads, one position each
    if (blocks > 152 * 16) blocks = 152 * 16;
    tree_prep_kernel<<<(int)blocks, 256, 0, s>>>(d_points, t->n, t->d, t->dp, d_perm, t->perm, t->inv, t->Xt, t->Xdup,
                                            t->n_pad, t->status, t->status + 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bounds_kernel<<<(t->nb + 1 + 255) / 256, 256, 0, s>>>(t->n, t->s0, t->nb, t->bnd);
    return cudaGetLastError();
}

}  // namespace fsg
