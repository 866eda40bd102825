// Re-decision of flagged descents in high precision (fsg_params.resolve).
//
// A descent decision of Algorithm 1 compares the draw u with the ratio
// g_left / (g_left + g_right).  The fused schedule takes it on FP32 sums and
// flags it when |u - ratio| falls inside the sums' error bound, so a flagged
// sample may differ from the exact method's.  This pass takes every flagged
// sample again from the root:
//   * levels above the bins: the FP32 node sums are rebuilt from the query's
//     bin sums in the order descend_top used (bit-identical), and each level
//     is tested as before; a level inside the FP32 band is decided on
//     high-precision sums of both halves (double-single squared distances,
//     values within relative error 2^-20, FP64 accumulation) compared in
//     FP64 with the full 32-bit draw, u = word 2^-32;
//   * the levels inside the bin reached: all of them on high-precision values
//     of the bin's points, summed pairwise in FP64 over the halving tree.
// A decision whose high-precision margin |u S - g_left| is still within the
// high-precision bound stays flagged; every other one equals the exact
// method's.  The sample's neighbour, its kernel value and its flags are
// overwritten in place, before the edge list is formed.
#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr int kRsThreads = 256;

__global__ void resolve_compact_kernel(const uint8_t* __restrict__ flags, const uint8_t* __restrict__ lflags,
                                       const int32_t* __restrict__ leaf_pos, int64_t total,
                                       int32_t* __restrict__ list, int32_t* __restrict__ count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pos = leaf_pos[e];
        if (pos >= 0 && ((flags[e] | lflags[e]) & 1)) list[atomicAdd(count, 1)] = (int32_t)e;
    }
}

// Sum over the CTA of one double per thread (every thread gets the result).
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // red is free
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kRsThreads / 32; ++k) s += red[k];
    return s;
}

// High-precision sum of k(query, point) over tree positions [a, c), the
// query's own position left out when self_exclude.
__device__ __forceinline__ double hp_range(const float* __restrict__ Xt, int dp, int d, const float* __restrict__ xq,
                                           int a, int c, int qpos, int self_exclude, float ch, float cl,
                                           double* red) {
    double s = 0.0;
    for (int p = a + (int)threadIdx.x; p < c; p += kRsThreads) {
        if (self_exclude && p == qpos) continue;
        s += (double)hp_gauss(xq, Xt + (size_t)p * dp, d, ch, cl);
    }
    return block_sum(s, red);
}

// FP64 decision on high-precision sums: 1 = right.  hp_flag: the margin is
// within the sums' error bound (relative kHpEta each, plus the FP64 rounding
// of the accumulation and of u S - g_left).
__device__ __forceinline__ int hp_decide(double gl, double gr, uint32_t word, uint8_t& f) {
    const double S = gl + gr;
    if (!(S > 0.0)) { f |= 2; return 1; }
    const double u = (double)word * 0x1p-32;
    const double dlt = u * S - gl;
    if (fabs(dlt) <= (kHpEta + 0x1p-40) * S) f |= 1;
    return dlt < 0.0 ? 0 : 1;
}

__global__ void __launch_bounds__(kRsThreads)
resolve_kernel(const float* __restrict__ Xt, int dp, int d, const int32_t* __restrict__ perm,
               const int32_t* __restrict__ bnd, int nb, int s0, const float* __restrict__ binsum,
               const int32_t* __restrict__ list, const int32_t* __restrict__ count, KernelParams kp, int leafmax,
               int32_t* __restrict__ leaf_pos, float* __restrict__ ksmp, uint8_t* __restrict__ flags,
               uint8_t* __restrict__ lflags) {
    extern __shared__ __align__(16) unsigned char smem_r[];
    float* tree = reinterpret_cast<float*>(smem_r);                       // [2 nb]
    double* V = reinterpret_cast<double*>(tree + 2 * nb + 2);             // [2 leafmax] halving-tree sums
    int32_t* spos = reinterpret_cast<int32_t*>(V + 2 * leafmax);          // [leafmax] slot -> position
    float* xq = reinterpret_cast<float*>(spos + leafmax);                 // [d] query coordinates
    __shared__ double red[kRsThreads / 32];
    const int tid = threadIdx.x;
    const int L = kp.L;
    const int cnt = *count;
    for (int it = blockIdx.x; it < cnt; it += gridDim.x) {
        const int e = list[it];
        const int q = e / L, l = e - q * L;
        const uint32_t i = (uint32_t)perm[q];
        __syncthreads();  // the previous sample's shared data are no longer read
        for (int b = tid; b < nb; b += kRsThreads) tree[nb + b] = binsum[(size_t)q * nb + b];
        for (int t = tid; t < d; t += kRsThreads) xq[t] = Xt[(size_t)q * dp + t];
        __syncthreads();
        // node sums of levels s0-1 .. 0, pairwise, as descend_top formed them
        for (int lev = s0 - 1; lev >= 0; --lev) {
            for (int h = (1 << lev) + tid; h < (2 << lev); h += kRsThreads) tree[h] = tree[2 * h] + tree[2 * h + 1];
            __syncthreads();
        }
        const float root = tree[1];
        const float abs_tol = kp.kde_eps > 0.f ? kp.kde_eps * root / (1.f - kp.kde_eps) : 0.f;
        uint8_t f = 0;
        int h = 1, a = 0, c = bnd[nb];
        uint4 blk = make_uint4(0, 0, 0, 0);
        int blk_id = -1;
        for (int t = 0; t < s0; ++t) {
            if ((t >> 2) != blk_id) {
                blk_id = t >> 2;
                blk = draw_block(kp.seed, i, (uint32_t)l, (uint32_t)t);
            }
            const uint32_t word = block_word(blk, (uint32_t)t);
            uint8_t f32 = 0;
            int right = descend_decide(tree[2 * h], tree[2 * h + 1], word, kp.flag_eps, f32, abs_tol);
            const int mid = a + (c - a) / 2;
            if (f32 & 1) {  // inside the FP32 band: both halves in high precision
                const double gl = hp_range(Xt, dp, d, xq, a, mid, q, kp.self_exclude, kp.hp_ch, kp.hp_cl, red);
                const double gr = hp_range(Xt, dp, d, xq, mid, c, q, kp.self_exclude, kp.hp_ch, kp.hp_cl, red);
                right = hp_decide(gl, gr, word, f);
            } else {
                f |= f32;
            }
            if (right) a = mid; else c = mid;
            h = 2 * h + right;
        }
        // the bin reached: high-precision values in the slots of its halving tree
        const int m = c - a;
        const int dm = ceil_log2_dev(m);
        const int leaf0 = 1 << dm;
        for (int sl = tid; sl < leaf0; sl += kRsThreads) {
            int lo = 0, hi = m;
            for (int t = dm - 1; t >= 0; --t) {
                const int md = lo + (hi - lo) / 2;
                if ((sl >> t) & 1) lo = md; else hi = md;
            }
            const int pos = hi - lo == 1 ? a + lo : -1;
            spos[sl] = pos;
            double v = 0.0;
            if (pos >= 0 && !(kp.self_exclude && pos == q))
                v = (double)hp_gauss(xq, Xt + (size_t)pos * dp, d, kp.hp_ch, kp.hp_cl);
            V[leaf0 + sl] = v;
        }
        __syncthreads();
        for (int lev = dm - 1; lev >= 0; --lev) {
            for (int x = (1 << lev) + tid; x < (2 << lev); x += kRsThreads) V[x] = V[2 * x] + V[2 * x + 1];
            __syncthreads();
        }
        if (tid == 0) {
            int hh = 1, lo = 0, hi = m;
            for (int t = 0; t < dm; ++t) {
                int right = 1;  // a single point sits in the right half
                if (hi - lo >= 2) {
                    const uint32_t lev = (uint32_t)(s0 + t);
                    if ((int)(lev >> 2) != blk_id) {
                        blk_id = (int)(lev >> 2);
                        blk = draw_block(kp.seed, i, (uint32_t)l, lev);
                    }
                    right = hp_decide(V[2 * hh], V[2 * hh + 1], block_word(blk, lev), f);
                    const int md = lo + (hi - lo) / 2;
                    if (right) lo = md; else hi = md;
                }
                hh = 2 * hh + right;
            }
            leaf_pos[e] = spos[hh - leaf0];
            ksmp[e] = (float)V[hh];
            flags[e] = f;
            lflags[e] = 0;
        }
    }
}

}  // namespace

bool resolve_supported(const fsg_tree* t) { return t->d <= 4096 && t->nb <= 4096 && (1 << t->dm) <= 1024; }

size_t resolve_smem(const fsg_tree* t) {
    const int leafmax = 1 << t->dm;
    return (size_t)(2 * t->nb + 2) * 4 + (size_t)2 * leafmax * 8 + (size_t)leafmax * 4 + (size_t)t->d * 4 + 16;
}

cudaError_t launch_resolve(const fsg_tree* t, const KernelParams& kp, int32_t* list, int32_t* count,
                           cudaStream_t s) {
    const auto& ws = t->ws;
    const int64_t total = t->n * (int64_t)kp.L;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    resolve_compact_kernel<<<(int)blocks, 256, 0, s>>>(ws.flags, ws.lflags, ws.leaf_pos, total, list, count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = resolve_smem(t);
    e = set_smem_limit(resolve_kernel, smem);
    if (e != cudaSuccess) return e;
    resolve_kernel<<<152 * 4, kRsThreads, smem, s>>>(t->Xt, t->dp, t->d, t->perm, t->bnd, t->nb, t->s0, ws.binsum,
                                                    list, count, kp, 1 << t->dm, ws.leaf_pos, ws.ksmp, ws.flags,
                                                    ws.lflags);
    return cudaGetLastError();
}

}  // namespace fsg
