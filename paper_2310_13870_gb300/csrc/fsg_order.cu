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

constexpr int kOrdThreads = 512;
constexpr int kOrdU = 4;   // points per thread and iteration (their loads issued together)
constexpr int kOrdC = 16;  // coordinates per min/max pass
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
    __shared__ float rmin[kOrdThreads / 32][kOrdC], rmax[kOrdThreads / 32][kOrdC];
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
    for (int c0 = 0; c0 < d; c0 += kOrdC) {
        float mn[kOrdC], mx[kOrdC];
#pragma unroll
        for (int u = 0; u < kOrdC; ++u) { mn[u] = 3.0e38f; mx[u] = -3.0e38f; }
        for (int64_t p = lo + tid; p < hi; p += (int64_t)kOrdThreads * kOrdU) {
            const float* row[kOrdU];
#pragma unroll
            for (int k = 0; k < kOrdU; ++k) {
                const int64_t pk = p + (int64_t)k * kOrdThreads;
                row[k] = pk < hi ? X + (int64_t)pin[pk] * d : nullptr;
            }
#pragma unroll
            for (int k = 0; k < kOrdU; ++k) {
                if (!row[k]) continue;
#pragma unroll
                for (int u = 0; u < kOrdC; ++u) {
                    if (c0 + u < d) {
                        const float v = row[k][c0 + u];
                        mn[u] = fminf(mn[u], v);
                        mx[u] = fmaxf(mx[u], v);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kOrdC; ++u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn[u] = fminf(mn[u], __shfl_xor_sync(0xffffffffu, mn[u], o));
                mx[u] = fmaxf(mx[u], __shfl_xor_sync(0xffffffffu, mx[u], o));
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < kOrdC; ++u) { rmin[warp][u] = mn[u]; rmax[warp][u] = mx[u]; }
        }
        __syncthreads();
        if (warp == 0) {  // lane u < kOrdC reduces coordinate c0 + u over the warps
            float a = 3.0e38f, b = -3.0e38f;
            if (lane < kOrdC) {
                a = rmin[0][lane];
                b = rmax[0][lane];
                for (int w = 1; w < kOrdThreads / 32; ++w) { a = fminf(a, rmin[w][lane]); b = fmaxf(b, rmax[w][lane]); }
            }
            float sp = (lane < kOrdC && c0 + lane < d) ? b - a : -2.f;
            int t = c0 + lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {  // widest, lowest coordinate on ties
                const float sp2 = __shfl_xor_sync(0xffffffffu, sp, o);
                const int t2 = __shfl_xor_sync(0xffffffffu, t, o);
                const float a2 = __shfl_xor_sync(0xffffffffu, a, o);
                if (sp2 > sp || (sp2 == sp && t2 < t)) { sp = sp2; t = t2; a = a2; }
            }
            if (lane == 0 && sp > best_spread) { best_spread = sp; best_min = a; best_t = t; }
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
    for (int64_t p = lo + tid; p < hi; p += (int64_t)kOrdThreads * kOrdU) {
        float key[kOrdU];
#pragma unroll
        for (int k = 0; k < kOrdU; ++k) {
            const int64_t pk = p + (int64_t)k * kOrdThreads;
            key[k] = pk < hi ? X[(int64_t)pin[pk] * d + axis] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kOrdU; ++k)
            if (p + (int64_t)k * kOrdThreads < hi) atomicAdd(&hist[bucket_of(key[k], kmin, scale)], 1);
    }
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
        int c0 = 0, c1 = 0, c2 = 0;
        int key_b[kOrdE];
#pragma unroll
        for (int e = 0; e < kOrdE; ++e) {
            const int64_t p = p0 + e;
            key_b[e] = p < hi ? bucket_of(X[(int64_t)pin[p] * d + axis], kmin, scale) : -1;
        }
#pragma unroll
        for (int e = 0; e < kOrdE; ++e) {
            const int b = key_b[e];
            const uint32_t c = b < 0 ? 3u : (b < mb ? 0u : (b == mb ? 1u : 2u));
            c0 += c == 0u;
            c1 += c == 1u;
            c2 += c == 2u;
            cat |= c << (2 * e);
        }
        // exclusive scan of the three counts over the CTA's threads
        int i0 = c0, i1 = c1, i2 = c2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y0 = __shfl_up_sync(0xffffffffu, i0, o);
            const int y1 = __shfl_up_sync(0xffffffffu, i1, o);
            const int y2 = __shfl_up_sync(0xffffffffu, i2, o);
            if (lane >= o) { i0 += y0; i1 += y1; i2 += y2; }
        }
        if (lane == 31) {
            wsum[0][warp] = i0;
            wsum[1][warp] = i1;
            wsum[2][warp] = i2;
        }
        __syncthreads();
        int b0 = 0, b1 = 0, b2 = 0;
        for (int w = 0; w < warp; ++w) { b0 += wsum[0][w]; b1 += wsum[1][w]; b2 += wsum[2][w]; }
        int o0 = s_run[0] + b0 + i0 - c0, o1 = s_run[1] + b1 + i1 - c1, o2 = s_run[2] + b2 + i2 - c2;
#pragma unroll
        for (int e = 0; e < kOrdE; ++e) {
            const uint32_t c = (cat >> (2 * e)) & 3u;
            if (c == 3u) continue;
            int64_t dst;
            if (c == 0u) {
                dst = lo + o0++;
            } else if (c == 1u) {
                const int r = o1++;
                dst = r < take ? lo + n_lower + r : lo + need + (r - take);
            } else {
                dst = lo + need + (n_med - take) + o2++;
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


// ---- wide levels (fewer than kWideNodes nodes): a node's work spread over
// CTAs of kWideChunk positions, four kernels per level: min/max by ordered
// integer atomics, the histogram by atomic adds (both independent of the
// order of the additions), counts per chunk with each position's category,
// and the scatter at offsets from the earlier chunks' counts.
constexpr int kWideNodes = 256;
constexpr int kWideChunk = 512;
constexpr int kWideThreads = 256;  // two consecutive positions per thread

__device__ __forceinline__ uint32_t f2o(float v) {  // order-preserving float -> uint
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

struct WideCtx {
    int64_t lo, hi, clo, chi;  // node, chunk
    int k;
};
__device__ __forceinline__ WideCtx wide_ctx(int64_t n, int lev, int cpn) {
    WideCtx c;
    c.k = (int)(blockIdx.x / cpn);
    const int ci = (int)(blockIdx.x % cpn);
    node_range(n, lev, c.k, c.lo, c.hi);
    c.clo = c.lo + (int64_t)ci * kWideChunk;
    c.chi = c.clo + kWideChunk < c.hi ? c.clo + kWideChunk : c.hi;
    return c;
}

__global__ void wide_reset_kernel(int nodes, int d, uint32_t* __restrict__ omin, uint32_t* __restrict__ omax,
                                  int32_t* __restrict__ hist) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nodes * d) {
        omin[i] = 0xffffffffu;
        omax[i] = 0u;
    }
    if (i < nodes * kOrdBuckets) hist[i] = 0;
}

__global__ void __launch_bounds__(kWideThreads)
wide_minmax_kernel(const float* __restrict__ X, int d, int64_t n, int lev, int cpn, int leaf,
                   const int32_t* __restrict__ pin, uint32_t* __restrict__ omin, uint32_t* __restrict__ omax) {
    __shared__ float rmin[kWideThreads / 32][kOrdC], rmax[kWideThreads / 32][kOrdC];
    const WideCtx c = wide_ctx(n, lev, cpn);
    if (c.hi - c.lo <= leaf || c.clo >= c.chi) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t p0 = c.clo + 2 * tid;
    const float* r0 = p0 < c.chi ? X + (int64_t)pin[p0] * d : nullptr;
    const float* r1 = p0 + 1 < c.chi ? X + (int64_t)pin[p0 + 1] * d : nullptr;
    for (int c0 = 0; c0 < d; c0 += kOrdC) {
        float mn[kOrdC], mx[kOrdC];
#pragma unroll
        for (int u = 0; u < kOrdC; ++u) {
            mn[u] = 3.0e38f;
            mx[u] = -3.0e38f;
            if (c0 + u < d) {
                if (r0) { mn[u] = fminf(mn[u], r0[c0 + u]); mx[u] = fmaxf(mx[u], r0[c0 + u]); }
                if (r1) { mn[u] = fminf(mn[u], r1[c0 + u]); mx[u] = fmaxf(mx[u], r1[c0 + u]); }
            }
        }
#pragma unroll
        for (int u = 0; u < kOrdC; ++u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn[u] = fminf(mn[u], __shfl_xor_sync(0xffffffffu, mn[u], o));
                mx[u] = fmaxf(mx[u], __shfl_xor_sync(0xffffffffu, mx[u], o));
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < kOrdC; ++u) { rmin[warp][u] = mn[u]; rmax[warp][u] = mx[u]; }
        }
        __syncthreads();
        if (warp == 0 && lane < kOrdC && c0 + lane < d) {
            float a = rmin[0][lane], b = rmax[0][lane];
            for (int w = 1; w < kWideThreads / 32; ++w) { a = fminf(a, rmin[w][lane]); b = fmaxf(b, rmax[w][lane]); }
            atomicMin(&omin[(int64_t)c.k * d + c0 + lane], f2o(a));
            atomicMax(&omax[(int64_t)c.k * d + c0 + lane], f2o(b));
        }
        __syncthreads();
    }
}

// The node's widest coordinate (lowest on ties), its minimum and bucket scale.
__device__ __forceinline__ void wide_axis(int d, int k, const uint32_t* __restrict__ omin,
                                          const uint32_t* __restrict__ omax, int& axis, float& kmin, float& scale) {
    __shared__ int s_axis;
    __shared__ float s_min, s_scale;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        float sp = -2.f, a = 0.f;
        int t = 0x7fffffff;
        for (int c = lane; c < d; c += 32) {
            const float lo = o2f(omin[(int64_t)k * d + c]), hi = o2f(omax[(int64_t)k * d + c]);
            if (hi - lo > sp) { sp = hi - lo; a = lo; t = c; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float sp2 = __shfl_xor_sync(0xffffffffu, sp, o);
            const int t2 = __shfl_xor_sync(0xffffffffu, t, o);
            const float a2 = __shfl_xor_sync(0xffffffffu, a, o);
            if (sp2 > sp || (sp2 == sp && t2 < t)) { sp = sp2; t = t2; a = a2; }
        }
        if (lane == 0) {
            s_axis = t;
            s_min = a;
            s_scale = sp > 0.f ? (float)kOrdBuckets / sp : 0.f;
        }
    }
    __syncthreads();
    axis = s_axis;
    kmin = s_min;
    scale = s_scale;
}

__global__ void __launch_bounds__(kWideThreads)
wide_hist_kernel(const float* __restrict__ X, int d, int64_t n, int lev, int cpn, int leaf,
                 const int32_t* __restrict__ pin, const uint32_t* __restrict__ omin,
                 const uint32_t* __restrict__ omax, int32_t* __restrict__ hist) {
    __shared__ int h[kOrdBuckets];
    const WideCtx c = wide_ctx(n, lev, cpn);
    if (c.hi - c.lo <= leaf || c.clo >= c.chi) return;
    int axis;
    float kmin, scale;
    wide_axis(d, c.k, omin, omax, axis, kmin, scale);
    for (int b = threadIdx.x; b < kOrdBuckets; b += kWideThreads) h[b] = 0;
    __syncthreads();
    for (int e = 0; e < 2; ++e) {
        const int64_t p = c.clo + 2 * threadIdx.x + e;
        if (p < c.chi) atomicAdd(&h[bucket_of(X[(int64_t)pin[p] * d + axis], kmin, scale)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kOrdBuckets; b += kWideThreads)
        if (h[b]) atomicAdd(&hist[c.k * kOrdBuckets + b], h[b]);
}

// The node's split from its histogram: median bucket, lower count, taken from
// the median bucket, median count.
__device__ __forceinline__ void wide_split(const int32_t* __restrict__ hist, int k, int64_t need, int (&sp)[4]) {
    __shared__ int s[4];
    if (threadIdx.x == 0) {
        int64_t cum = 0;
        int mb = kOrdBuckets - 1;
        for (int b = 0; b < kOrdBuckets; ++b) {
            const int hb = hist[k * kOrdBuckets + b];
            if (cum + hb > need) { mb = b; break; }
            cum += hb;
        }
        s[0] = mb;
        s[1] = (int)cum;
        s[2] = (int)(need - cum);
        s[3] = hist[k * kOrdBuckets + mb];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) sp[i] = s[i];
}

__global__ void __launch_bounds__(kWideThreads)
wide_count_kernel(const float* __restrict__ X, int d, int64_t n, int lev, int cpn, int leaf,
                  const int32_t* __restrict__ pin, const uint32_t* __restrict__ omin,
                  const uint32_t* __restrict__ omax, const int32_t* __restrict__ hist, uint8_t* __restrict__ cat,
                  int32_t* __restrict__ ccount) {
    __shared__ int cnt[3];
    const WideCtx c = wide_ctx(n, lev, cpn);
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    if (c.hi - c.lo <= leaf || c.clo >= c.chi) {
        if (threadIdx.x < 3) ccount[blockIdx.x * 3 + threadIdx.x] = 0;
        return;
    }
    int axis;
    float kmin, scale;
    wide_axis(d, c.k, omin, omax, axis, kmin, scale);
    int sp[4];
    wide_split(hist, c.k, (c.hi - c.lo) / 2, sp);
    int l0 = 0, l1 = 0, l2 = 0;
    for (int e = 0; e < 2; ++e) {
        const int64_t p = c.clo + 2 * threadIdx.x + e;
        if (p < c.chi) {
            const int b = bucket_of(X[(int64_t)pin[p] * d + axis], kmin, scale);
            const uint8_t g = b < sp[0] ? 0 : (b == sp[0] ? 1 : 2);
            cat[p] = g;
            l0 += g == 0;
            l1 += g == 1;
            l2 += g == 2;
        }
    }
    if (l0) atomicAdd(&cnt[0], l0);  // integer counts: any order gives the same total
    if (l1) atomicAdd(&cnt[1], l1);
    if (l2) atomicAdd(&cnt[2], l2);
    __syncthreads();
    if (threadIdx.x < 3) ccount[blockIdx.x * 3 + threadIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kWideThreads)
wide_scatter_kernel(int64_t n, int lev, int cpn, int leaf, const int32_t* __restrict__ pin,
                    const int32_t* __restrict__ hist, const uint8_t* __restrict__ cat,
                    const int32_t* __restrict__ ccount, int32_t* __restrict__ pout) {
    __shared__ int wsum[3][kWideThreads / 32];
    __shared__ int before[3];
    const WideCtx c = wide_ctx(n, lev, cpn);
    if (c.clo >= c.chi) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (c.hi - c.lo <= leaf) {  // a node not split at this level: copied
        for (int64_t p = c.clo + tid; p < c.chi; p += kWideThreads) pout[p] = pin[p];
        return;
    }
    const int64_t need = (c.hi - c.lo) / 2;
    int sp[4];
    wide_split(hist, c.k, need, sp);
    const int take = sp[2], n_lower = sp[1], n_med = sp[3];
    // counts of the node's earlier chunks
    const int ci = (int)(blockIdx.x % cpn), cbase = (int)(blockIdx.x - ci);
    if (warp == 0) {
        int s0 = 0, s1 = 0, s2 = 0;
        for (int j = lane; j < ci; j += 32) {
            s0 += ccount[(cbase + j) * 3 + 0];
            s1 += ccount[(cbase + j) * 3 + 1];
            s2 += ccount[(cbase + j) * 3 + 2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) { before[0] = s0; before[1] = s1; before[2] = s2; }
    }
    // this thread's two positions, in position order
    int g[2] = {3, 3};
    int c0 = 0, c1 = 0, c2 = 0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int64_t p = c.clo + 2 * tid + e;
        if (p < c.chi) {
            g[e] = cat[p];
            c0 += g[e] == 0;
            c1 += g[e] == 1;
            c2 += g[e] == 2;
        }
    }
    int i0 = c0, i1 = c1, i2 = c2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y0 = __shfl_up_sync(0xffffffffu, i0, o);
        const int y1 = __shfl_up_sync(0xffffffffu, i1, o);
        const int y2 = __shfl_up_sync(0xffffffffu, i2, o);
        if (lane >= o) { i0 += y0; i1 += y1; i2 += y2; }
    }
    if (lane == 31) { wsum[0][warp] = i0; wsum[1][warp] = i1; wsum[2][warp] = i2; }
    __syncthreads();
    int b0 = before[0], b1 = before[1], b2 = before[2];
    for (int w = 0; w < warp; ++w) { b0 += wsum[0][w]; b1 += wsum[1][w]; b2 += wsum[2][w]; }
    int o0 = b0 + i0 - c0, o1 = b1 + i1 - c1, o2 = b2 + i2 - c2;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (g[e] == 3) continue;
        int64_t dst;
        if (g[e] == 0) {
            dst = c.lo + o0++;
        } else if (g[e] == 1) {
            const int r = o1++;
            dst = r < take ? c.lo + n_lower + r : c.lo + need + (r - take);
        } else {
            dst = c.lo + need + (n_med - take) + o2++;
        }
        pout[dst] = pin[c.clo + 2 * tid + e];
    }
}

}  // namespace

// Levels until every node holds at most `leaf` points.
int spatial_order_levels(int64_t n, int leaf) {
    int lev = 0;
    while ((n + (int64_t(1) << lev) - 1) >> lev > leaf) ++lev;
    return lev;
}

// Scratch of launch_spatial_order: two position arrays, a category byte per
// position, and the wide levels' per-node min/max, histograms and per-chunk
// counts.
struct OrdScratch {
    int32_t* a;
    int32_t* b;
    uint8_t* cat;
    uint32_t* omin;
    uint32_t* omax;
    int32_t* hist;
    int32_t* ccount;
    size_t bytes;
    OrdScratch(void* base, int64_t n, int d) {
        auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
        const size_t chunks = (size_t)(n / kWideChunk) + 2 * kWideNodes + 1;
        size_t off = 0;
        unsigned char* p = static_cast<unsigned char*>(base);
        a = reinterpret_cast<int32_t*>(p + off); off += up(sizeof(int32_t) * (size_t)n);
        b = reinterpret_cast<int32_t*>(p + off); off += up(sizeof(int32_t) * (size_t)n);
        cat = p + off; off += up((size_t)n);
        omin = reinterpret_cast<uint32_t*>(p + off); off += up(sizeof(uint32_t) * kWideNodes * (size_t)d);
        omax = reinterpret_cast<uint32_t*>(p + off); off += up(sizeof(uint32_t) * kWideNodes * (size_t)d);
        hist = reinterpret_cast<int32_t*>(p + off); off += up(sizeof(int32_t) * kWideNodes * kOrdBuckets);
        ccount = reinterpret_cast<int32_t*>(p + off); off += up(sizeof(int32_t) * 3 * chunks);
        bytes = off;
    }
};

size_t spatial_order_scratch_bytes(int64_t n, int d) { return OrdScratch(nullptr, n, d).bytes; }

// The order of d_points into the scratch at buf; *out = the array holding it.
cudaError_t launch_spatial_order(const float* d_points, int64_t n, int d, int leaf, void* buf, const int32_t** out,
                                 cudaStream_t s) {
    const OrdScratch sc(buf, n, d);
    int32_t* a = sc.a;
    int32_t* b = sc.b;
    iota_kernel<<<(int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(n, a);
    cudaError_t e = cudaGetLastError();
    const int levels = spatial_order_levels(n, leaf);
    for (int lev = 0; lev < levels && e == cudaSuccess; ++lev) {
        const int nodes = 1 << lev;
        const int64_t maxsize = (n + nodes - 1) / nodes;
        if (nodes < kWideNodes) {
            const int cpn = (int)((maxsize + kWideChunk - 1) / kWideChunk);
            const int grid = nodes * cpn;
            const int rs = nodes * (d > kOrdBuckets ? d : kOrdBuckets);
            wide_reset_kernel<<<(rs + 255) / 256, 256, 0, s>>>(nodes, d, sc.omin, sc.omax, sc.hist);
            wide_minmax_kernel<<<grid, kWideThreads, 0, s>>>(d_points, d, n, lev, cpn, leaf, a, sc.omin, sc.omax);
            wide_hist_kernel<<<grid, kWideThreads, 0, s>>>(d_points, d, n, lev, cpn, leaf, a, sc.omin, sc.omax,
                                                           sc.hist);
            wide_count_kernel<<<grid, kWideThreads, 0, s>>>(d_points, d, n, lev, cpn, leaf, a, sc.omin, sc.omax,
                                                            sc.hist, sc.cat, sc.ccount);
            wide_scatter_kernel<<<grid, kWideThreads, 0, s>>>(n, lev, cpn, leaf, a, sc.hist, sc.cat, sc.ccount, b);
        } else {
            order_level_kernel<<<(unsigned)nodes, kOrdThreads, 0, s>>>(d_points, d, n, lev, leaf, a, b);
        }
        e = cudaGetLastError();
        int32_t* t = a;
        a = b;
        b = t;
    }
    *out = a;
    return e;
}

}  // namespace fsg
