// The descent of Algorithm 1 (Sec. 4.1) for all L samples of every point.
//
//  descend_top  : per query, the bin sums of level s0 are summed pairwise into
//                 the query's node sums of levels 0..s0 (a segment tree in
//                 shared memory); the root is the degree g_[1,n] (Algorithm 2).
//                 Each sample then takes its first s0 decisions, comparing the
//                 Philox draw with g_left/(g_left+g_right) at every level.
//                 The distinct (query, bin) pairs reached go straight into
//                 per-bin item lists (bin-major, capacity n per bin), each
//                 item carrying the 64-bit mask of the query's samples there.
//  leaf_finish  : per (bin, batch of items): the kernel value of every (query,
//                 point) pair of the bin, the query's segment tree over the
//                 bin's sub-nodes, and the remaining decisions of every
//                 sample down to a single point; the sample's weight
//                 w = k / p_hat of Eq. 2 is formed from that point's value.
#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Per query (one warp): segment tree of the query's node sums over levels
// 0..s0 built from its bin sums, the degree (the root), the first s0
// decisions of each of the query's L samples, and the compact list of the
// distinct bins its samples reached with the mask of samples at each.
__global__ void __launch_bounds__(256)
descend_top_kernel(const float* __restrict__ binsum, int n, int nb, int s0, const int32_t* __restrict__ perm,
                   KernelParams kp, int with_samples, double* __restrict__ d_deg, float* __restrict__ degf,
                   uint8_t* __restrict__ flags, int32_t* __restrict__ leaf_pos, float* __restrict__ wsmp,
                   int32_t* __restrict__ bin_count, int32_t* __restrict__ items_q,
                   uint64_t* __restrict__ items_mask) {
    extern __shared__ __align__(16) unsigned char smem_b[];
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t* sbin = reinterpret_cast<int32_t*>(smem_b) + (size_t)w * 64;             // [64] per warp
    float* tree = reinterpret_cast<float*>(reinterpret_cast<int32_t*>(smem_b) + (size_t)warps * 64) +
                  (size_t)w * 2 * nb;                                                 // [2 nb] per warp
    const int L = kp.L;
    for (int q = blockIdx.x * warps + w; q < n; q += gridDim.x * warps) {
        const float* row = binsum + (size_t)q * nb;
        for (int b = lane; b < nb; b += 32) tree[nb + b] = row[b];
        __syncwarp();
        for (int lev = s0 - 1; lev >= 0; --lev) {
            for (int h = (1 << lev) + lane; h < (2 << lev); h += 32) tree[h] = tree[2 * h] + tree[2 * h + 1];
            __syncwarp();
        }
        const float root = tree[1];
        const int i = perm[q];
        if (lane == 0) {
            degf[q] = root;
            if (d_deg) d_deg[i] = (double)root;
        }
        if (with_samples) {
            int binv[2] = {-1, -1};
            if (root > 0.f) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int l = lane + 32 * r;
                    if (l < L) {
                        uint8_t f = 0;
                        int h = 1;
                        uint4 blk = make_uint4(0, 0, 0, 0);
                        for (int t = 0; t < s0; ++t) {
                            if ((t & 3) == 0) blk = draw_block(kp.seed, (uint32_t)i, (uint32_t)l, (uint32_t)t);
                            h = 2 * h + descend_decide(tree[2 * h], tree[2 * h + 1], block_word(blk, (uint32_t)t),
                                                       kp.flag_eps, f);
                        }
                        binv[r] = h - nb;
                        flags[(size_t)q * L + l] = f;
                    }
                    sbin[l] = binv[r];
                }
                __syncwarp();
                // Group the samples by bin: sample l's mask holds every sample at its bin.
                uint64_t M[2] = {0ull, 0ull};
                for (int e = 0; e < 64; e += 4) {
                    const int4 v = *reinterpret_cast<const int4*>(sbin + e);
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        M[r] |= (uint64_t)(v.x == binv[r]) << e;
                        M[r] |= (uint64_t)(v.y == binv[r]) << (e + 1);
                        M[r] |= (uint64_t)(v.z == binv[r]) << (e + 2);
                        M[r] |= (uint64_t)(v.w == binv[r]) << (e + 3);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int l = lane + 32 * r;
                    // the lowest sample of each bin writes the (query, mask) item
                    if (binv[r] >= 0 && (M[r] & ((1ull << l) - 1ull)) == 0ull) {
                        const int b = binv[r];
                        const int slot = atomicAdd(&bin_count[b], 1);
                        items_q[(size_t)b * n + slot] = q;
                        items_mask[(size_t)b * n + slot] = M[r];
                    }
                }
            } else {
                // zero FP32 mass: no sample; flag unless no other point exists
                const uint8_t f = (n > 1 || !kp.self_exclude) ? 2 : 0;
                for (int l = lane; l < L; l += 32) {
                    leaf_pos[(size_t)q * L + l] = -1;
                    wsmp[(size_t)q * L + l] = 0.f;
                    flags[(size_t)q * L + l] = f;
                }
            }
        }
        __syncwarp();
    }
}

constexpr int kThreadsC = 256;

// Leaf finish: CTA (b, y) handles chunks y, y + gridDim.y, ... of bin b's
// item list, qt items per chunk.  Thread t owns leaf slots t, t + 256, ... of
// the bin's perfect binary tree (slot = the path bits of the halving descent;
// slots of empty nodes hold 0) -- or, when the tree has fewer than 256
// leaves, slot t mod 2^dm for every G-th query.  Each chunk: kernel value of
// every (query, slot), per-query trees summed upwards in shared memory, then
// one thread per (query, sample) takes the remaining decisions and forms the
// weight w = k / p_hat of Eq. 2.
template <int D, int SPT>
__global__ void __launch_bounds__(kThreadsC)
leaf_finish_kernel(const float* __restrict__ Xt, const int32_t* __restrict__ perm, const int32_t* __restrict__ bnd,
                   int n, int s0, const int32_t* __restrict__ bin_count, const int32_t* __restrict__ items_q,
                   const uint64_t* __restrict__ items_mask, const float* __restrict__ degf, KernelParams kp, int qt,
                   int dm_max, int32_t* __restrict__ leaf_pos, float* __restrict__ wsmp, uint8_t* __restrict__ flags,
                   unsigned long long* __restrict__ n_evals, unsigned long long* __restrict__ n_items) {
    constexpr int DP = (D + 3) & ~3;
    const int b = blockIdx.x;
    const int cnt = bin_count[b];
    const int nchunks = (cnt + qt - 1) / qt;
    if ((int)blockIdx.y >= nchunks) return;

    extern __shared__ __align__(16) unsigned char smem_c[];
    const int vs = 2 << dm_max;  // row stride of the per-query trees
    float* V = reinterpret_cast<float*>(smem_c);
    float* qs = V + (size_t)qt * vs;
    uint64_t* qmask = reinterpret_cast<uint64_t*>(qs + (size_t)qt * DP);
    int32_t* qpos = reinterpret_cast<int32_t*>(qmask + qt);
    int32_t* qidx = qpos + qt;
    float* qdeg = reinterpret_cast<float*>(qidx + qt);
    int32_t* loff = reinterpret_cast<int32_t*>(qdeg + qt);   // qt + 1
    int32_t* list = loff + qt + 1;                            // qt * 64

    const int tid = threadIdx.x;
    const int L = kp.L;
    const int p_lo = bnd[b];
    const int m = bnd[b + 1] - p_lo;
    const int dm = ceil_log2_dev(m);
    const int leaf0 = 1 << dm;
    const int G = leaf0 >= kThreadsC ? 1 : kThreadsC / leaf0;
    const int g = leaf0 >= kThreadsC ? 0 : tid / leaf0;
    const int s_first = leaf0 >= kThreadsC ? tid : tid % leaf0;
    // This thread's slots: point coordinates kept in registers for every chunk.
    float pc[SPT][D];
    int ppos[SPT];
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
        const int sl = s_first + u * kThreadsC;
        ppos[u] = -1;
        if (sl < leaf0) {
            int a = 0, c = m;  // walk the slot's path bits from the root
            for (int t = dm - 1; t >= 0; --t) {
                const int mid = a + (c - a) / 2;
                if ((sl >> t) & 1) a = mid; else c = mid;
            }
            if (c - a == 1) ppos[u] = p_lo + a;
        }
#pragma unroll
        for (int t = 0; t < D; ++t) pc[u][t] = ppos[u] >= 0 ? Xt[(size_t)ppos[u] * DP + t] : 0.f;
    }
    const size_t base = (size_t)b * n;
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int it0 = chunk * qt;
        const int qcnt = min(qt, cnt - it0);
        for (int e = tid; e < qcnt; e += kThreadsC) {
            const int q = items_q[base + it0 + e];
            qpos[e] = q;
            qidx[e] = perm[q];
            qmask[e] = items_mask[base + it0 + e];
            qdeg[e] = degf[q];
        }
        for (int e = tid; e < qcnt * DP; e += kThreadsC) {
            const int qq = e / DP;
            qs[e] = Xt[(size_t)items_q[base + it0 + qq] * DP + (e - qq * DP)];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
            const int sl = s_first + u * kThreadsC;
            if (sl < leaf0) {
                for (int qq = g; qq < qcnt; qq += G) {
                    float k = 0.f;
                    if (ppos[u] >= 0) {
                        const float* qc = qs + qq * DP;
                        float dd = qc[0] - pc[u][0];
                        float acc = dd * dd;
#pragma unroll
                        for (int t = 1; t < D; ++t) {
                            dd = qc[t] - pc[u][t];
                            acc = fmaf(dd, dd, acc);
                        }
                        k = ex2_approx(acc * kp.neg_c);
                        if (kp.self_exclude && ppos[u] == qpos[qq]) k = 0.f;
                    }
                    V[(size_t)qq * vs + leaf0 + sl] = k;
                }
            }
        }
        __syncthreads();
        for (int lev = dm - 1; lev >= 0; --lev) {
            const int cn = qcnt << lev;
            for (int e = tid; e < cn; e += kThreadsC) {
                const int qq = e >> lev;
                const int h = (1 << lev) + (e & ((1 << lev) - 1));
                float* row = V + (size_t)qq * vs;
                row[h] = row[2 * h] + row[2 * h + 1];
            }
            __syncthreads();
        }
        // List of (query, sample) pairs of this chunk (warp 0: popcount prefix).
        if (tid < 32) {
            int c0 = 0, c1 = 0;
            if (tid < qcnt) c0 = __popcll(qmask[tid]);
            if (tid + 32 < qcnt) c1 = __popcll(qmask[tid + 32]);
            int s0v = c0, s1v = c1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y0 = __shfl_up_sync(0xffffffffu, s0v, o);
                const int y1 = __shfl_up_sync(0xffffffffu, s1v, o);
                if (tid >= o) { s0v += y0; s1v += y1; }
            }
            const int tot0 = __shfl_sync(0xffffffffu, s0v, 31);
            if (tid < qcnt) loff[tid] = s0v - c0;
            if (tid + 32 < qcnt) loff[tid + 32] = tot0 + s1v - c1;
            if (tid == 31) loff[qcnt] = tot0 + s1v;
        }
        __syncthreads();
        for (int e = tid; e < qcnt * 64; e += kThreadsC) {
            const int qq = e >> 6, l = e & 63;
            const uint64_t mk = qmask[qq];
            if ((mk >> l) & 1ull) list[loff[qq] + __popcll(mk & ((1ull << l) - 1ull))] = (qq << 6) | l;
        }
        __syncthreads();
        const int nsamp = loff[qcnt];
        for (int e = tid; e < nsamp; e += kThreadsC) {
            const int qq = list[e] >> 6, l = list[e] & 63;
            const float* row = V + (size_t)qq * vs;
            const uint32_t i = (uint32_t)qidx[qq];
            int a = 0, c = m, h = 1;
            uint8_t f = 0;
            uint4 blk = make_uint4(0, 0, 0, 0);
            int blk_id = -1;
            for (int t = 0; t < dm; ++t) {
                if (c - a >= 2) {
                    const uint32_t lev = (uint32_t)(s0 + t);
                    if ((int)(lev >> 2) != blk_id) {
                        blk = draw_block(kp.seed, i, (uint32_t)l, lev);
                        blk_id = (int)(lev >> 2);
                    }
                    const int mid = a + (c - a) / 2;
                    const int right = descend_decide(row[2 * h], row[2 * h + 1], block_word(blk, lev), kp.flag_eps, f);
                    if (right) a = mid; else c = mid;
                    h = 2 * h + right;
                } else {
                    h = 2 * h + 1;  // a single point sits in the right half
                }
            }
            const int pos = p_lo + a;
            const float k = row[h];
            const float Lk = (float)L * k;
            const float pi = fminf(__fdiv_rn(Lk, qdeg[qq]), 1.f);
            const float pj = fminf(__fdiv_rn(Lk, degf[pos]), 1.f);
            const float ph = pi + pj - pi * pj;
            const size_t o = (size_t)qpos[qq] * L + l;
            leaf_pos[o] = pos;
            wsmp[o] = k > 0.f ? __fdiv_rn(k, ph) : 0.f;
            flags[o] |= f;
        }
        if (tid == 0) {
            atomicAdd(n_evals, (unsigned long long)qcnt * (unsigned long long)m);
            atomicAdd(n_items, (unsigned long long)qcnt);
        }
        __syncthreads();
    }
}

template <int D, int SPT>
cudaError_t launch_leaf_ds(const fsg_tree* t, const KernelParams& kp, int qt, cudaStream_t s) {
    constexpr int DP = (D + 3) & ~3;
    const int vs = 2 << t->dm;
    const size_t smem = (size_t)qt * vs * 4 + (size_t)qt * DP * 4 + (size_t)qt * 8 + (size_t)qt * 12 +
                        (size_t)(qt + 1) * 4 + (size_t)qt * 64 * 4;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(leaf_finish_kernel<D, SPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // Splits per bin: about 8 waves of CTAs over the expected items.
    const int64_t items_est = t->n * (int64_t)(kp.L < t->nb ? kp.L : t->nb);
    const int64_t chunks_per_bin = (items_est / t->nb + qt - 1) / qt + 1;
    int64_t S = (152 * 4 * 8 + t->nb - 1) / t->nb;
    if (S > chunks_per_bin) S = chunks_per_bin;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    dim3 grid(t->nb, (unsigned)S);
    const auto& ws = t->ws;
    leaf_finish_kernel<D, SPT><<<grid, kThreadsC, smem, s>>>(
        t->Xt, t->perm, t->bnd, (int)t->n, t->s0, ws.bin_count, ws.items_q, ws.items_mask, ws.degf, kp, qt, t->dm,
        ws.leaf_pos, ws.wsmp, ws.flags, reinterpret_cast<unsigned long long*>(&ws.stats->n_evals),
        reinterpret_cast<unsigned long long*>(&ws.stats->n_items));
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_leaf_d(const fsg_tree* t, const KernelParams& kp, int qt, cudaStream_t s) {
    const int leaf0 = 1 << t->dm;
    if (leaf0 <= kThreadsC) return launch_leaf_ds<D, 1>(t, kp, qt, s);
    if (leaf0 <= 2 * kThreadsC) return launch_leaf_ds<D, 2>(t, kp, qt, s);
    return launch_leaf_ds<D, 4>(t, kp, qt, s);
}

}  // namespace

int leaf_queries_per_tile(const fsg_tree* t) {
    int qt = 8192 / (2 << t->dm);  // 32 KB of per-query trees
    if (qt > 64) qt = 64;
    if (qt < 4) qt = 4;
    return qt;
}

cudaError_t launch_descend_top(const fsg_tree* t, const KernelParams& kp, double* d_deg, int with_samples,
                               cudaStream_t s) {
    int warps = 8;
    while (warps > 1 && (size_t)warps * (256 + 8 * t->nb) > 96 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * (256 + 8 * t->nb);  // per warp: 64 sample bins + 2 nb tree nodes
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(descend_top_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(smem < 48 * 1024 ? 48 * 1024 : smem));
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    int64_t blocks = (t->n + warps - 1) / warps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const auto& ws = t->ws;
    descend_top_kernel<<<(int)blocks, warps * 32, smem, s>>>(ws.binsum, (int)t->n, t->nb, t->s0, t->perm, kp,
                                                            with_samples, d_deg, ws.degf, ws.flags, ws.leaf_pos,
                                                            ws.wsmp, ws.bin_count, ws.items_q, ws.items_mask);
    return cudaGetLastError();
}

cudaError_t launch_leaf_finish(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const int qt = leaf_queries_per_tile(t);
    switch (t->d) {
        case 1: return launch_leaf_d<1>(t, kp, qt, s);
        case 2: return launch_leaf_d<2>(t, kp, qt, s);
        case 3: return launch_leaf_d<3>(t, kp, qt, s);
        case 4: return launch_leaf_d<4>(t, kp, qt, s);
        case 5: return launch_leaf_d<5>(t, kp, qt, s);
        case 6: return launch_leaf_d<6>(t, kp, qt, s);
        case 7: return launch_leaf_d<7>(t, kp, qt, s);
        case 8: return launch_leaf_d<8>(t, kp, qt, s);
        case 9: return launch_leaf_d<9>(t, kp, qt, s);
        case 10: return launch_leaf_d<10>(t, kp, qt, s);
        case 11: return launch_leaf_d<11>(t, kp, qt, s);
        case 12: return launch_leaf_d<12>(t, kp, qt, s);
        case 13: return launch_leaf_d<13>(t, kp, qt, s);
        case 14: return launch_leaf_d<14>(t, kp, qt, s);
        case 15: return launch_leaf_d<15>(t, kp, qt, s);
        case 16: return launch_leaf_d<16>(t, kp, qt, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsg
