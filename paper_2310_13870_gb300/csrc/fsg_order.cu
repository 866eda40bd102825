// Spatial tree order (host): a permutation under which every node of the
// halving tree of Sec. 4.1 is a compact group of points.  Node [lo, hi) of
// tree positions is split at its own midpoint lo + floor((hi - lo) / 2), as
// the tree splits it, along the coordinate of largest spread among the
// node's points: the floor(|X|/2) points with the smallest values of that
// coordinate go left (ties broken by original index).  Nodes of at most
// `leaf` points keep original-index order.  The KDE and the sampling
// distribution do not depend on the order (Eq. 1 sums over the node's
// points whatever their positions); the order only decides which points
// share a bin, and so how far a bin's points lie from its centre, which the
// centred split-precision bin pass relies on.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "fsg.h"

namespace {

struct OrderState {
    const float* X;
    int64_t d;
    int32_t leaf;
    std::vector<int32_t>* idx;
};

void split_node(OrderState& st, int64_t lo, int64_t hi) {
    std::vector<int32_t>& idx = *st.idx;
    while (hi - lo > st.leaf) {
        // axis of largest spread among the node's points
        int64_t axis = 0;
        float best = -1.f;
        for (int64_t t = 0; t < st.d; ++t) {
            float mn = st.X[(int64_t)idx[lo] * st.d + t], mx = mn;
            for (int64_t p = lo + 1; p < hi; ++p) {
                const float v = st.X[(int64_t)idx[p] * st.d + t];
                mn = std::min(mn, v);
                mx = std::max(mx, v);
            }
            if (mx - mn > best) {
                best = mx - mn;
                axis = t;
            }
        }
        const int64_t mid = lo + (hi - lo) / 2;
        const float* X = st.X;
        const int64_t d = st.d;
        auto less = [X, d, axis](int32_t a, int32_t b) {
            const float va = X[(int64_t)a * d + axis], vb = X[(int64_t)b * d + axis];
            return va < vb || (va == vb && a < b);
        };
        std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, less);
        split_node(st, lo, mid);
        lo = mid;  // the right half, without another stack frame
    }
    std::sort(idx.begin() + lo, idx.begin() + hi);
}

}  // namespace

extern "C" int fsg_spatial_order(const float* h_points, int64_t n, int32_t d, int32_t leaf, int32_t* h_perm) {
    if (!h_points || !h_perm || n < 1 || n > INT32_MAX || d < 1 || d > 4096 || leaf < 1)
        return FSG_ERR_INVALID_ARG;
    for (int64_t e = 0; e < n * (int64_t)d; ++e)
        if (!(h_points[e] == h_points[e]) || h_points[e] > 3.0e38f || h_points[e] < -3.0e38f)
            return FSG_ERR_INVALID_ARG;  // NaN or infinite coordinate
    std::vector<int32_t> idx((size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[(size_t)i] = (int32_t)i;
    OrderState st{h_points, d, leaf, &idx};
    split_node(st, 0, n);
    std::copy(idx.begin(), idx.end(), h_perm);
    return FSG_OK;
}

// ---------------------------------------------------------------------------
// Spatial tree order on the GPU (fsg_tree_opts.order = FSG_ORDER_SPATIAL), the
// same construction level by level: at level lev every node [lo, hi) of more
// than `leaf` points (the tree's midpoint rule) is split by one CTA.
//   1. the widest coordinate: per-coordinate min and max over the node's
//      points (eight coordinates per pass);
//   2. a 256-bucket histogram of that coordinate over [min, max]; the bucket
//      holding rank floor(m/2) is the median bucket;
//   3. a scan-based partition in position order: points of lower buckets go
//      left, of higher buckets right, and the median bucket's points fill the
//      left half's remaining slots in position order, the rest going right.
// So the left floor(m/2) positions hold the smaller values of the node's
// widest coordinate up to the width of one bucket, and the result depends
// only on the points (no atomics decide a position).  Nodes of at most
// `leaf` points are copied.  Runs in the build and in every fsg_tree_update.
// ---------------------------------------------------------------------------
#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr int kOrdThreads = 256;
constexpr int kOrdBuckets = 256;
constexpr int kOrdE = 16;  // positions per thread per partition chunk

__device__ __forceinline__ void node_range(int64_t n, int lev, int64_t k, int64_t& lo, int64_t& hi) {
    lo = 0;
    hi = n;
    for (int t = lev - 1; t >= 0; --t) {
        const int64_t mid = lo + (hi - lo) / 2;
        if ((k >> t) & 1) lo = mid; else hi = mid;
    }
}

__device__ __forceinline__ int bucket_of(float key, float mn, float scale) {
    const int b = (int)((key - mn) * scale);
    return b < 0 ? 0 : (b >= kOrdBuckets ? kOrdBuckets - 1 : b);
}

__global__ void iota_kernel(int64_t n, int32_t* __restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

__global__ void __launch_bounds__(kOrdThreads)
order_level_kernel(const float* __restrict__ X, int d, int64_t n, int lev, int leaf, const int32_t* __restrict__ pin,
                   int32_t* __restrict__ pout) {
    __shared__ float rmin[kOrdThreads / 32][8], rmax[kOrdThreads / 32][8];
    __shared__ int hist[kOrdBuckets];
    __shared__ int wsum[3][kOrdThreads / 32];
    __shared__ float s_best[2];  // min, scale of the chosen coordinate
    __shared__ int s_axis;
    __shared__ int s_split[4];   // median bucket, lower count, taken from the median bucket, median count
    __shared__ int s_run[3];     // running L, M, H counts over the chunks
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int64_t lo, hi;
    node_range(n, lev, blockIdx.x, lo, hi);
    const int64_t m = hi - lo;
    if (m <= leaf) {
        for (int64_t p = lo + tid; p < hi; p += kOrdThreads) pout[p] = pin[p];
        return;
    }
    const int64_t need = m / 2;  // the left child's size
    // 1. widest coordinate
    float best_spread = -1.f, best_min = 0.f;
    int best_t = 0;
    for (int c0 = 0; c0 < d; c0 += 8) {
        float mn[8], mx[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { mn[u] = 3.0e38f; mx[u] = -3.0e38f; }
        for (int64_t p = lo + tid; p < hi; p += kOrdThreads) {
            const float* row = X + (int64_t)pin[p] * d;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (c0 + u < d) {
                    const float v = row[c0 + u];
                    mn[u] = fminf(mn[u], v);
                    mx[u] = fmaxf(mx[u], v);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn[u] = fminf(mn[u], __shfl_xor_sync(0xffffffffu, mn[u], o));
                mx[u] = fmaxf(mx[u], __shfl_xor_sync(0xffffffffu, mx[u], o));
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 8; ++u) { rmin[warp][u] = mn[u]; rmax[warp][u] = mx[u]; }
        }
        __syncthreads();
        if (tid == 0) {
            for (int u = 0; u < 8 && c0 + u < d; ++u) {
                float a = rmin[0][u], b = rmax[0][u];
                for (int w = 1; w < kOrdThreads / 32; ++w) { a = fminf(a, rmin[w][u]); b = fmaxf(b, rmax[w][u]); }
                if (b - a > best_spread) { best_spread = b - a; best_min = a; best_t = c0 + u; }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        s_axis = best_t;
        s_best[0] = best_min;
        s_best[1] = best_spread > 0.f ? (float)kOrdBuckets / best_spread : 0.f;
    }
    for (int b = tid; b < kOrdBuckets; b += kOrdThreads) hist[b] = 0;
    __syncthreads();
    const int axis = s_axis;
    const float kmin = s_best[0], scale = s_best[1];
    // 2. histogram and the median bucket
    for (int64_t p = lo + tid; p < hi; p += kOrdThreads)
        atomicAdd(&hist[bucket_of(X[(int64_t)pin[p] * d + axis], kmin, scale)], 1);
    __syncthreads();
    if (tid == 0) {
        int64_t cum = 0;
        int mb = kOrdBuckets - 1;
        for (int b = 0; b < kOrdBuckets; ++b) {
            if (cum + hist[b] > need) { mb = b; break; }
            cum += hist[b];
        }
        s_split[0] = mb;
        s_split[1] = (int)cum;           // points in lower buckets (<= need)
        s_split[2] = (int)(need - cum);  // median-bucket points that go left
        s_split[3] = hist[mb];
        s_run[0] = s_run[1] = s_run[2] = 0;
    }
    __syncthreads();
    const int mb = s_split[0], n_lower = s_split[1], take = s_split[2], n_med = s_split[3];
    // 3. partition, chunks of kOrdThreads * kOrdE positions, thread = kOrdE consecutive positions
    for (int64_t base = lo; base < hi; base += (int64_t)kOrdThreads * kOrdE) {
        const int64_t p0 = base + (int64_t)tid * kOrdE;
        uint32_t cat = 0;  // 2 bits per position: 0 lower, 1 median, 2 higher, 3 none
        int cnt[3] = {0, 0, 0};
#pragma unroll
        for (int e = 0; e < kOrdE; ++e) {
            const int64_t p = p0 + e;
            int c = 3;
            if (p < hi) {
                const int b = bucket_of(X[(int64_t)pin[p] * d + axis], kmin, scale);
                c = b < mb ? 0 : (b == mb ? 1 : 2);
                ++cnt[c];
            }
            cat |= (uint32_t)c << (2 * e);
        }
        // exclusive scan of the three counts over the CTA's threads
        int inc[3] = {cnt[0], cnt[1], cnt[2]};
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int y = __shfl_up_sync(0xffffffffu, inc[c], o);
                if (lane >= o) inc[c] += y;
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int c = 0; c < 3; ++c) wsum[c][warp] = inc[c];
        }
        __syncthreads();
        int off[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int before = 0;
            for (int w = 0; w < warp; ++w) before += wsum[c][w];
            off[c] = s_run[c] + before + inc[c] - cnt[c];
        }
#pragma unroll
        for (int e = 0; e < kOrdE; ++e) {
            const int c = (int)((cat >> (2 * e)) & 3u);
            if (c == 3) continue;
            int64_t dst;
            if (c == 0) {
                dst = lo + off[0]++;
            } else if (c == 1) {
                const int r = off[1]++;
                dst = r < take ? lo + n_lower + r : lo + need + (r - take);
            } else {
                dst = lo + need + (n_med - take) + off[2]++;
            }
            pout[dst] = pin[p0 + e];
        }
        __syncthreads();  // every thread has read s_run and wsum
        if (tid == kOrdThreads - 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int tot = 0;
                for (int w = 0; w < kOrdThreads / 32; ++w) tot += wsum[c][w];
                s_run[c] += tot;
            }
        }
        __syncthreads();
    }
}

}  // namespace

// Levels until every node holds at most `leaf` points.
int spatial_order_levels(int64_t n, int leaf) {
    int lev = 0;
    while ((n + (int64_t(1) << lev) - 1) >> lev > leaf) ++lev;
    return lev;
}

// The order of d_points into buf (2 n int32 of scratch); returns the array
// that holds it (buf or buf + n).
cudaError_t launch_spatial_order(const float* d_points, int64_t n, int d, int leaf, int32_t* buf,
                                 const int32_t** out, cudaStream_t s) {
    int32_t* a = buf;
    int32_t* b = buf + n;
    iota_kernel<<<(int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(n, a);
    cudaError_t e = cudaGetLastError();
    const int levels = spatial_order_levels(n, leaf);
    for (int lev = 0; lev < levels && e == cudaSuccess; ++lev) {
        order_level_kernel<<<(unsigned)(int64_t(1) << lev), kOrdThreads, 0, s>>>(d_points, d, n, lev, leaf, a, b);
        e = cudaGetLastError();
        int32_t* t = a;
        a = b;
        b = t;
    }
    *out = a;
    return e;
}

}  // namespace fsg
