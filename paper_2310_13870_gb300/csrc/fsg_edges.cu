// Edge list of Algorithm 2: the union over all points of the sampled pairs,
// with the weights of Eq. 2, w = k / p_hat, p_hat = p_i + p_j - p_i p_j,
// p_i = min(L k / g_[1,n](x_i), 1), formed here from each sample's kernel
// value k (kept by the leaf finish) and the two endpoints' degrees.
//
//   SET   : each unordered pair {i,j} (i != j) appears once.  Per query, the
//           distinct sampled neighbours are sorted in-warp (bitonic network);
//           the pair is written by i unless j also sampled i and j has the
//           smaller original index.  Membership is a binary search in j's
//           sorted list, so no global sort is needed.
//   MULTI : every non-self sample is an edge (i = the sampling point).
// Counts per query are scanned (three-kernel exclusive scan) into offsets.
#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int32_t kSentinel = 0x7fffffff;

// Weight of Eq. 2 in FP32; symmetric in (i, j) bit for bit.
__device__ __forceinline__ float edge_weight(float k, float deg_i, float deg_j, int L) {
    if (!(k > 0.f)) return 0.f;
    const float Lk = (float)L * k;
    const float pi = fminf(__fdiv_rn(Lk, deg_i), 1.f);
    const float pj = fminf(__fdiv_rn(Lk, deg_j), 1.f);
    return __fdiv_rn(k, pi + pj - pi * pj);
}

// Weight of Eq. 2 in FP64 from a high-precision kernel value of the pair at
// tree positions (a, b) and the two FP32-accumulated degrees; symmetric in
// (a, b) bit for bit.
__device__ __forceinline__ double edge_weight_f64(const float* __restrict__ Xt, int dp, int d, int a, int b,
                                                  float deg_a, float deg_b, int L, float ch, float cl) {
    const double k = (double)hp_gauss(Xt + (size_t)a * dp, Xt + (size_t)b * dp, dp, ch, cl);
    if (!(k > 0.0)) return 0.0;
    const double Lk = (double)L * k;
    const double pa = fmin(Lk / (double)deg_a, 1.0);
    const double pb = fmin(Lk / (double)deg_b, 1.0);
    return k / (pa + pb - pa * pb);
}

// Bitonic sort of the warp's 64 (key, value) pairs: element index lane holds
// (k0, v0), index lane+32 holds (k1, v1).  Ascending by key.
__device__ __forceinline__ void warp_sort64(int32_t& k0, float& v0, int32_t& k1, float& v1, int lane) {
    for (int k = 2; k <= 64; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                if (k1 < k0) {  // k == 64: ascending across the two halves
                    int32_t tk = k0; k0 = k1; k1 = tk;
                    float tv = v0; v0 = v1; v1 = tv;
                }
            } else {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    int32_t& kk = r ? k1 : k0;
                    float& vv = r ? v1 : v0;
                    const int idx = lane + 32 * r;
                    const int32_t pk = __shfl_xor_sync(kFull, kk, j);
                    const float pv = __shfl_xor_sync(kFull, vv, j);
                    const bool up = (idx & k) == 0;
                    const bool lower = (idx & j) == 0;
                    const bool take_min = (up == lower);
                    if (take_min ? (pk < kk) : (pk > kk)) { kk = pk; vv = pv; }
                }
            }
        }
    }
}

// SET, step 1: per query, the sorted distinct neighbours (self and -1 dropped).
__global__ void __launch_bounds__(128)
unique_neighbours_kernel(const int32_t* __restrict__ leaf_pos, const float* __restrict__ ksmp,
                         const float* __restrict__ degf, int n, int L, int32_t* __restrict__ uniq,
                         float* __restrict__ uniq_w, int32_t* __restrict__ ucnt) {
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = blockIdx.x * warps + w; q < n; q += gridDim.x * warps) {
        int32_t k0 = kSentinel, k1 = kSentinel;
        float v0 = 0.f, v1 = 0.f;
        const float dq = degf[q];
        if (lane < L) {
            const int32_t j = leaf_pos[(size_t)q * L + lane];
            if (j >= 0 && j != q) { k0 = j; v0 = edge_weight(ksmp[(size_t)q * L + lane], dq, degf[j], L); }
        }
        if (lane + 32 < L) {
            const int32_t j = leaf_pos[(size_t)q * L + lane + 32];
            if (j >= 0 && j != q) { k1 = j; v1 = edge_weight(ksmp[(size_t)q * L + lane + 32], dq, degf[j], L); }
        }
        warp_sort64(k0, v0, k1, v1, lane);
        // previous element of index lane (k0) and lane+32 (k1)
        int32_t prev0 = __shfl_up_sync(kFull, k0, 1);
        int32_t prev1 = __shfl_up_sync(kFull, k1, 1);
        const int32_t last0 = __shfl_sync(kFull, k0, 31);
        if (lane == 0) { prev0 = -1; prev1 = last0; }
        const bool u0 = k0 != kSentinel && k0 != prev0;
        const bool u1 = k1 != kSentinel && k1 != prev1;
        const uint32_t b0 = __ballot_sync(kFull, u0), b1 = __ballot_sync(kFull, u1);
        const int c0 = __popc(b0);
        const uint32_t below = (1u << lane) - 1u;
        if (u0) {
            const int r = __popc(b0 & below);
            uniq[(size_t)q * L + r] = k0;
            uniq_w[(size_t)q * L + r] = v0;
        }
        if (u1) {
            const int r = c0 + __popc(b1 & below);
            uniq[(size_t)q * L + r] = k1;
            uniq_w[(size_t)q * L + r] = v1;
        }
        if (lane == 0) ucnt[q] = c0 + __popc(b1);
    }
}

__device__ __forceinline__ bool sorted_contains(const int32_t* __restrict__ a, int len, int32_t x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = a[mid];
        if (v == x) return true;
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

// SET, step 2: which of q's distinct neighbours q writes, and how many.
__global__ void __launch_bounds__(128)
owner_kernel(const int32_t* __restrict__ uniq, const int32_t* __restrict__ ucnt, const int32_t* __restrict__ perm,
             int n, int L, uint64_t* __restrict__ emit_mask, int64_t* __restrict__ ecount) {
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = blockIdx.x * warps + w; q < n; q += gridDim.x * warps) {
        const int c = ucnt[q];
        const int32_t iq = perm[q];
        uint64_t mask = 0;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int k = lane + 32 * r;
            bool emit = false;
            if (k < c) {
                const int32_t j = uniq[(size_t)q * L + k];
                emit = true;
                if (perm[j] < iq && sorted_contains(uniq + (size_t)j * L, ucnt[j], q)) emit = false;
            }
            const uint32_t bal = __ballot_sync(kFull, emit);
            mask |= (uint64_t)bal << (32 * r);
        }
        if (lane == 0) {
            emit_mask[q] = mask;
            ecount[q] = __popcll(mask);
        }
    }
}

// MULTI: edges per query = its non-self, non-empty samples.
__global__ void multi_count_kernel(const int32_t* __restrict__ leaf_pos, int n, int L, int64_t* __restrict__ ecount) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int c = 0;
        for (int l = 0; l < L; ++l) {
            const int32_t j = leaf_pos[(size_t)q * L + l];
            c += (j >= 0 && j != q) ? 1 : 0;
        }
        ecount[q] = c;
    }
}

// --- exclusive scan of int64 counts (n elements, in place, total at [n]) ---
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int64_t block_inclusive_scan(int64_t v, int64_t* sh) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < (kScanBlock >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    if (w > 0) v += sh[w - 1];
    return v;
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const int64_t* __restrict__ x, int n,
                                                                int64_t* __restrict__ sums) {
    __shared__ int64_t sh[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    int64_t v = i < n ? x[i] : 0;
    v = block_inclusive_scan(v, sh);
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kScanBlock) scan_top_kernel(int64_t* __restrict__ sums, int nblocks) {
    __shared__ int64_t sh[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += kScanBlock) {
        const int i = base + threadIdx.x;
        const int64_t v0 = i < nblocks ? sums[i] : 0;
        const int64_t inc = block_inclusive_scan(v0, sh);
        const int64_t c = carry;
        if (i < nblocks) sums[i] = c + inc - v0;  // exclusive
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry = c + inc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_apply_kernel(int64_t* __restrict__ x, int n,
                                                               const int64_t* __restrict__ sums,
                                                               int64_t* __restrict__ m_out,
                                                               fsg_stats* __restrict__ stats) {
    __shared__ int64_t sh[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int64_t v = i < n ? x[i] : 0;
    const int64_t inc = block_inclusive_scan(v, sh) + sums[blockIdx.x];
    if (i < n) x[i] = inc - v;
    if (i == n - 1) {
        x[n] = inc;
        *m_out = inc;
        stats->n_edges = inc;
    }
}

// F64: weights in FP64 from high-precision kernel values (wout is double).
template <bool F64>
__global__ void __launch_bounds__(128)
set_write_kernel(const int32_t* __restrict__ uniq, const float* __restrict__ uniq_w,
                 const uint64_t* __restrict__ emit_mask, const int64_t* __restrict__ eoff,
                 const int32_t* __restrict__ perm, int n, int L, int64_t cap, int32_t* __restrict__ src,
                 int32_t* __restrict__ dst, void* __restrict__ wout, const float* __restrict__ Xt, int dp, int d,
                 const float* __restrict__ degf, float ch, float cl) {
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = blockIdx.x * warps + w; q < n; q += gridDim.x * warps) {
        const uint64_t mk = emit_mask[q];
        const int64_t base = eoff[q];
        const int32_t iq = perm[q];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int k = lane + 32 * r;
            if ((mk >> k) & 1ull) {
                const int64_t o = base + __popcll(mk & ((1ull << k) - 1ull));
                if (o < cap) {
                    const int32_t j = uniq[(size_t)q * L + k];
                    src[o] = iq;
                    dst[o] = perm[j];
                    if (F64)
                        static_cast<double*>(wout)[o] = edge_weight_f64(Xt, dp, d, q, j, degf[q], degf[j], L, ch, cl);
                    else
                        static_cast<float*>(wout)[o] = uniq_w[(size_t)q * L + k];
                }
            }
        }
    }
}

template <bool F64>
__global__ void multi_write_kernel(const int32_t* __restrict__ leaf_pos, const float* __restrict__ ksmp,
                                   const float* __restrict__ degf, const int64_t* __restrict__ eoff,
                                   const int32_t* __restrict__ perm, int n, int L,
                                   int64_t cap, int32_t* __restrict__ src, int32_t* __restrict__ dst,
                                   void* __restrict__ wout, const float* __restrict__ Xt, int dp, int d, float ch,
                                   float cl) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int64_t o = eoff[q];
        const int32_t iq = perm[q];
        for (int l = 0; l < L; ++l) {
            const int32_t j = leaf_pos[(size_t)q * L + l];
            if (j >= 0 && j != q) {
                if (o < cap) {
                    src[o] = iq;
                    dst[o] = perm[j];
                    if (F64)
                        static_cast<double*>(wout)[o] = edge_weight_f64(Xt, dp, d, q, j, degf[q], degf[j], L,
                                                                        ch, cl);
                    else
                        static_cast<float*>(wout)[o] = edge_weight(ksmp[(size_t)q * L + l], degf[q], degf[j], L);
                }
                ++o;
            }
        }
    }
}

// Per-sample outputs in original index order, and sample statistics.
__global__ void outputs_kernel(const int32_t* __restrict__ leaf_pos, const uint8_t* __restrict__ flags,
                               const uint8_t* __restrict__ lflags, const int32_t* __restrict__ perm, int n, int L,
                               int32_t* __restrict__ d_samples,
                               uint8_t* __restrict__ d_flags, fsg_stats* __restrict__ stats) {
    // one warp per query position q, lanes over its L samples
    unsigned long long fl = 0, sf = 0, em = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); q < n; q += warps) {
        const size_t orow = (size_t)perm[q] * L;
        for (int l = lane; l < L; l += 32) {
            const size_t e = (size_t)q * L + l;
            const int32_t pos = leaf_pos[e];
            const uint8_t f = flags[e] | (pos >= 0 ? lflags[e] : (uint8_t)0);
            if (d_samples) d_samples[orow + l] = pos >= 0 ? perm[pos] : -1;
            if (d_flags) d_flags[orow + l] = f;
            fl += f != 0;
            sf += pos == q;
            em += pos < 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fl += __shfl_down_sync(kFull, fl, o);
        sf += __shfl_down_sync(kFull, sf, o);
        em += __shfl_down_sync(kFull, em, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (fl) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->n_flagged), fl);
        if (sf) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->n_self), sf);
        if (em) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->n_empty), em);
    }
}

int grid_for(int64_t work, int per_block) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_edges(const fsg_tree* t, const KernelParams& kp, int edge_mode, int32_t* d_src, int32_t* d_dst,
                         void* d_w, int64_t cap, int64_t* d_m_out, cudaStream_t s) {
    const auto& ws = t->ws;
    const int n = (int)t->n, L = kp.L;
    if (edge_mode == FSG_EDGES_SET) {
        unique_neighbours_kernel<<<grid_for(n, 4), 128, 0, s>>>(ws.leaf_pos, ws.ksmp, ws.degf, n, L, ws.uniq,
                                                               ws.uniq_w, ws.ucnt);
        owner_kernel<<<grid_for(n, 4), 128, 0, s>>>(ws.uniq, ws.ucnt, t->perm, n, L, ws.emit_mask, ws.ecount);
    } else {
        multi_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(ws.leaf_pos, n, L, ws.ecount);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nblocks = (n + kScanBlock - 1) / kScanBlock;
    scan_reduce_kernel<<<nblocks, kScanBlock, 0, s>>>(ws.ecount, n, ws.scan_tmp);
    scan_top_kernel<<<1, kScanBlock, 0, s>>>(ws.scan_tmp, nblocks);
    scan_apply_kernel<<<nblocks, kScanBlock, 0, s>>>(ws.ecount, n, ws.scan_tmp, d_m_out, ws.stats);
    if (edge_mode == FSG_EDGES_SET) {
        auto k = kp.weight_f64 ? set_write_kernel<true> : set_write_kernel<false>;
        k<<<grid_for(n, 4), 128, 0, s>>>(ws.uniq, ws.uniq_w, ws.emit_mask, ws.ecount, t->perm, n, L, cap, d_src,
                                         d_dst, d_w, t->Xt, t->dp, t->d, ws.degf, kp.hp_ch, kp.hp_cl);
    } else {
        auto k = kp.weight_f64 ? multi_write_kernel<true> : multi_write_kernel<false>;
        k<<<grid_for(n, 256), 256, 0, s>>>(ws.leaf_pos, ws.ksmp, ws.degf, ws.ecount, t->perm, n, L, cap, d_src,
                                           d_dst, d_w, t->Xt, t->dp, t->d, kp.hp_ch, kp.hp_cl);
    }
    return cudaGetLastError();
}

cudaError_t launch_outputs(const fsg_tree* t, const KernelParams& kp, int32_t* d_samples, uint8_t* d_flags,
                           fsg_stats* d_stats, cudaStream_t s) {
    (void)d_stats;
    const auto& ws = t->ws;
    outputs_kernel<<<grid_for(t->n * 32, 256), 256, 0, s>>>(ws.leaf_pos, ws.flags, ws.lflags, t->perm, (int)t->n,
                                                              kp.L, d_samples, d_flags, ws.stats);
    return cudaGetLastError();
}

}  // namespace fsg
