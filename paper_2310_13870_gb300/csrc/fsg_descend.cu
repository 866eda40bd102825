// The descent of Algorithm 1 (Sec. 4.1) for all L samples of every point.
//
//  descend_top  : per query, the bin sums of level s0 are summed pairwise into
//                 the query's node sums of levels 0..s0 (a segment tree in
//                 shared memory); the root is the degree g_[1,n] (Algorithm 2).
//                 Each sample then takes its first s0 decisions, comparing the
//                 Philox draw with g_left/(g_left+g_right) at every level.
//  bucket       : the distinct (query, bin) pairs reached are counted per bin,
//                 scanned, and scattered into per-bin item lists, each item
//                 carrying the 64-bit mask of the query's samples at that bin.
//  leaf_finish  : per (bin, batch of items): the kernel value of every (query,
//                 point) pair of the bin, the query's segment tree over the
//                 bin's sub-nodes, and the remaining decisions of every
//                 sample down to a single point; the sample's weight
//                 w = k / p_hat of Eq. 2 is formed from that point's value.
#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Group the warp's (up to 64) samples by bin: returns the mask of samples at
// the same bin as sample `lane` (Ma) and as sample `lane + 32` (Mb).
__device__ __forceinline__ void sample_groups(int a, int b, int lane, uint64_t& Ma, uint64_t& Mb) {
    const uint32_t ma = __match_any_sync(kFull, a);
    const uint32_t mb = __match_any_sync(kFull, b);
    uint32_t xa = 0, xb = 0;
#pragma unroll 4
    for (int m = 0; m < 32; ++m) {
        const int bm = __shfl_sync(kFull, b, m);
        const int am = __shfl_sync(kFull, a, m);
        if (bm == a) xa |= 1u << m;
        if (am == b) xb |= 1u << m;
    }
    Ma = (uint64_t)ma | ((uint64_t)xa << 32);
    Mb = (uint64_t)xb | ((uint64_t)mb << 32);
    (void)lane;
}

__global__ void __launch_bounds__(128)
descend_top_kernel(const float* __restrict__ binsum, int n, int nb, int s0, const int32_t* __restrict__ perm,
                   KernelParams kp, int with_samples, double* __restrict__ d_deg, float* __restrict__ degf,
                   int32_t* __restrict__ node_bin, uint8_t* __restrict__ flags, int32_t* __restrict__ leaf_pos,
                   float* __restrict__ wsmp, int32_t* __restrict__ bin_count) {
    extern __shared__ float tree_s[];
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* tree = tree_s + (size_t)w * 2 * nb;
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
            int binv[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int l = lane + 32 * r;
                binv[r] = -1;
                if (l < L) {
                    uint8_t f = 0;
                    int bin = -1;
                    if (root > 0.f) {
                        int h = 1;
                        uint4 blk = make_uint4(0, 0, 0, 0);
                        for (int t = 0; t < s0; ++t) {
                            if ((t & 3) == 0) blk = draw_block(kp.seed, (uint32_t)i, (uint32_t)l, (uint32_t)t);
                            h = 2 * h + descend_decide(tree[2 * h], tree[2 * h + 1], block_word(blk, (uint32_t)t),
                                                       kp.flag_eps, f);
                        }
                        bin = h - nb;
                    } else {
                        // zero FP32 mass: no sample; flag unless no other point exists
                        if (n > 1 || !kp.self_exclude) f |= 2;
                        leaf_pos[(size_t)q * L + l] = -1;
                        wsmp[(size_t)q * L + l] = 0.f;
                    }
                    node_bin[(size_t)q * L + l] = bin;
                    flags[(size_t)q * L + l] = f;
                    binv[r] = bin;
                }
            }
            uint64_t Ma, Mb;
            sample_groups(binv[0], binv[1], lane, Ma, Mb);
            if (binv[0] >= 0 && (Ma & ((1ull << lane) - 1ull)) == 0ull) atomicAdd(&bin_count[binv[0]], 1);
            if (binv[1] >= 0 && (Mb & ((1ull << (lane + 32)) - 1ull)) == 0ull) atomicAdd(&bin_count[binv[1]], 1);
        }
        __syncwarp();
    }
}

// Exclusive scan of the per-bin item counts (single CTA), tile counts per bin.
__global__ void __launch_bounds__(1024)
scan_bins_kernel(const int32_t* __restrict__ bin_count, int nb, int qt, int32_t* __restrict__ bin_off,
                 int32_t* __restrict__ tile_prefix, int32_t* __restrict__ misc, fsg_stats* __restrict__ stats) {
    __shared__ int32_t s_items[1024], s_tiles[1024];
    const int tid = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    int ci = 0, ct = 0;
    for (int u = 0; u < per; ++u) {
        const int b = tid * per + u;
        if (b < nb) { ci += bin_count[b]; ct += (bin_count[b] + qt - 1) / qt; }
    }
    s_items[tid] = ci;
    s_tiles[tid] = ct;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int vi = tid >= off ? s_items[tid - off] : 0;
        const int vt = tid >= off ? s_tiles[tid - off] : 0;
        __syncthreads();
        s_items[tid] += vi;
        s_tiles[tid] += vt;
        __syncthreads();
    }
    int ri = s_items[tid] - ci, rt = s_tiles[tid] - ct;  // exclusive prefix of this thread's range
    for (int u = 0; u < per; ++u) {
        const int b = tid * per + u;
        if (b < nb) {
            bin_off[b] = ri;
            tile_prefix[b] = rt;
            ri += bin_count[b];
            rt += (bin_count[b] + qt - 1) / qt;
        }
    }
    if (tid == 1023) {
        bin_off[nb] = s_items[1023];
        tile_prefix[nb] = s_tiles[1023];
        misc[0] = s_tiles[1023];
        stats->n_items = s_items[1023];
    }
}

__global__ void __launch_bounds__(128)
scatter_items_kernel(const int32_t* __restrict__ node_bin, int n, int L, const int32_t* __restrict__ bin_off,
                     int32_t* __restrict__ bin_cursor, int32_t* __restrict__ items_q,
                     uint64_t* __restrict__ items_mask) {
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = blockIdx.x * warps + w; q < n; q += gridDim.x * warps) {
        const int a = lane < L ? node_bin[(size_t)q * L + lane] : -1;
        const int b = lane + 32 < L ? node_bin[(size_t)q * L + lane + 32] : -1;
        uint64_t Ma, Mb;
        sample_groups(a, b, lane, Ma, Mb);
        if (a >= 0 && (Ma & ((1ull << lane) - 1ull)) == 0ull) {
            const int slot = bin_off[a] + atomicAdd(&bin_cursor[a], 1);
            items_q[slot] = q;
            items_mask[slot] = Ma;
        }
        if (b >= 0 && (Mb & ((1ull << (lane + 32)) - 1ull)) == 0ull) {
            const int slot = bin_off[b] + atomicAdd(&bin_cursor[b], 1);
            items_q[slot] = q;
            items_mask[slot] = Mb;
        }
    }
}

constexpr int kThreadsC = 256;

template <int D, int PPT>
__global__ void __launch_bounds__(kThreadsC)
leaf_finish_kernel(const float* __restrict__ Xt, const int32_t* __restrict__ perm, const int32_t* __restrict__ bnd,
                   int nb, int s0, const int32_t* __restrict__ bin_off, const int32_t* __restrict__ bin_count,
                   const int32_t* __restrict__ tile_prefix, const int32_t* __restrict__ misc,
                   const int32_t* __restrict__ items_q, const uint64_t* __restrict__ items_mask,
                   const float* __restrict__ degf, KernelParams kp, int qt, int dm_max,
                   int32_t* __restrict__ leaf_pos, float* __restrict__ wsmp, uint8_t* __restrict__ flags,
                   unsigned long long* __restrict__ n_evals) {
    constexpr int DP = (D + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smem_c[];
    const int vs = 2 << dm_max;  // row stride of the per-query segment trees
    float* V = reinterpret_cast<float*>(smem_c);
    float* qs = V + (size_t)qt * vs;
    uint64_t* qmask = reinterpret_cast<uint64_t*>(qs + (size_t)qt * DP);
    int32_t* qpos = reinterpret_cast<int32_t*>(qmask + qt);
    int32_t* qidx = qpos + qt;
    float* qdeg = reinterpret_cast<float*>(qidx + qt);
    int32_t* loff = reinterpret_cast<int32_t*>(qdeg + qt);   // qt + 1
    int32_t* list = loff + qt + 1;                            // qt * 64

    const int tid = threadIdx.x;
    const int ntiles = misc[0];
    const int L = kp.L;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int lo = 0, hi = nb;  // largest b with tile_prefix[b] <= tile
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tile_prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        const int b = lo;
        const int j0 = (tile - tile_prefix[b]) * qt;
        const int qcnt = min(qt, bin_count[b] - j0);
        const int it0 = bin_off[b] + j0;
        const int p_lo = bnd[b];
        const int m = bnd[b + 1] - p_lo;
        const int dm = ceil_log2_dev(m);
        const int leaf0 = 1 << dm;

        for (int e = tid; e < qcnt; e += kThreadsC) {
            const int q = items_q[it0 + e];
            qpos[e] = q;
            qidx[e] = perm[q];
            qmask[e] = items_mask[it0 + e];
            qdeg[e] = degf[q];
        }
        for (int e = tid; e < qcnt * DP; e += kThreadsC) {
            const int qq = e / DP;
            qs[e] = Xt[(size_t)items_q[it0 + qq] * DP + (e - qq * DP)];
        }
        for (int e = tid; e < qcnt * leaf0; e += kThreadsC) {
            const int qq = e >> dm;
            V[(size_t)qq * vs + leaf0 + (e & (leaf0 - 1))] = 0.f;
        }
        // This thread's points and their leaf slots (path bits, 1 = right half).
        float pc[PPT][D];
        int slot[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int p = tid + u * kThreadsC;
            slot[u] = -1;
            if (p < m) {
#pragma unroll
                for (int t = 0; t < D; ++t) pc[u][t] = Xt[(size_t)(p_lo + p) * DP + t];
                int a = 0, c = m, sl = 0;
                for (int t = 0; t < dm; ++t) {
                    const int mid = a + (c - a) / 2;
                    const int right = p >= mid ? 1 : 0;
                    if (right) a = mid; else c = mid;
                    sl = 2 * sl + right;
                }
                slot[u] = sl;
            } else {
#pragma unroll
                for (int t = 0; t < D; ++t) pc[u][t] = 0.f;
            }
        }
        __syncthreads();
        // Kernel values of every (query, point) pair of the tile.
        for (int qq = 0; qq < qcnt; ++qq) {
            float qc[D];
#pragma unroll
            for (int t = 0; t < D; ++t) qc[t] = qs[qq * DP + t];
            const int qp = qpos[qq];
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                if (slot[u] >= 0) {
                    float dd = qc[0] - pc[u][0];
                    float s = dd * dd;
#pragma unroll
                    for (int t = 1; t < D; ++t) {
                        dd = qc[t] - pc[u][t];
                        s = fmaf(dd, dd, s);
                    }
                    float k = ex2_approx(s * kp.neg_c);
                    if (kp.self_exclude && p_lo + tid + u * kThreadsC == qp) k = 0.f;
                    V[(size_t)qq * vs + leaf0 + slot[u]] = k;
                }
            }
        }
        __syncthreads();
        for (int lev = dm - 1; lev >= 0; --lev) {
            const int cnt = qcnt << lev;
            for (int e = tid; e < cnt; e += kThreadsC) {
                const int qq = e >> lev;
                const int h = (1 << lev) + (e & ((1 << lev) - 1));
                float* row = V + (size_t)qq * vs;
                row[h] = row[2 * h] + row[2 * h + 1];
            }
            __syncthreads();
        }
        // List of (query, sample) pairs of this tile.
        if (tid == 0) {
            int acc = 0;
            for (int qq = 0; qq < qcnt; ++qq) { loff[qq] = acc; acc += __popcll(qmask[qq]); }
            loff[qcnt] = acc;
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
        if (tid == 0) atomicAdd(n_evals, (unsigned long long)qcnt * (unsigned long long)m);
        __syncthreads();
    }
}

template <int D>
cudaError_t launch_leaf_d(const fsg_tree* t, const KernelParams& kp, int qt, cudaStream_t s) {
    constexpr int DP = (D + 3) & ~3;
    const int vs = 2 << t->dm;
    const size_t smem = (size_t)qt * vs * 4 + (size_t)qt * DP * 4 + (size_t)qt * 8 + (size_t)qt * 12 +
                        (size_t)(qt + 1) * 4 + (size_t)qt * 64 * 4;
    const int ppt = (t->mmax + kThreadsC - 1) / kThreadsC;
    int64_t max_items = t->n * (int64_t)(kp.L < t->nb ? kp.L : t->nb);
    int64_t tiles_ub = (max_items + qt - 1) / qt + t->nb;
    int grid = 152 * 3;
    if (tiles_ub < grid) grid = (int)tiles_ub;
    if (grid < 1) grid = 1;
    auto* ws = &t->ws;
#define FSG_LEAF_LAUNCH(PPT)                                                                                      \
    {                                                                                                             \
        cudaError_t e = cudaFuncSetAttribute(leaf_finish_kernel<D, PPT>,                                          \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);            \
        if (e != cudaSuccess) return e;                                                                           \
        leaf_finish_kernel<D, PPT><<<grid, kThreadsC, smem, s>>>(                                                 \
            t->Xt, t->perm, t->bnd, t->nb, t->s0, ws->bin_off, ws->bin_count, ws->tile_prefix, ws->misc,           \
            ws->items_q, ws->items_mask, ws->degf, kp, qt, t->dm, ws->leaf_pos, ws->wsmp, ws->flags,               \
            reinterpret_cast<unsigned long long*>(&ws->stats->n_evals));                                          \
        return cudaGetLastError();                                                                                \
    }
    if (ppt <= 1) FSG_LEAF_LAUNCH(1)
    if (ppt <= 2) FSG_LEAF_LAUNCH(2)
    FSG_LEAF_LAUNCH(4)
#undef FSG_LEAF_LAUNCH
}

}  // namespace

int leaf_queries_per_tile(const fsg_tree* t) {
    int qt = 16384 / (2 << t->dm);
    if (qt > 64) qt = 64;
    if (qt < 4) qt = 4;
    return qt;
}

cudaError_t launch_descend_top(const fsg_tree* t, const KernelParams& kp, double* d_deg, int with_samples,
                               cudaStream_t s) {
    int warps = 4;
    while (warps > 1 && (size_t)warps * 2 * t->nb * 4 > 64 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * 2 * t->nb * 4;
    cudaError_t e = cudaFuncSetAttribute(descend_top_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem < 48 * 1024 ? 48 * 1024 : smem));
    if (e != cudaSuccess) return e;
    int64_t blocks = (t->n + warps - 1) / warps;
    if (blocks > 152 * 32) blocks = 152 * 32;
    const auto& ws = t->ws;
    descend_top_kernel<<<(int)blocks, warps * 32, smem, s>>>(ws.binsum, (int)t->n, t->nb, t->s0, t->perm, kp,
                                                            with_samples, d_deg, ws.degf, ws.node_bin, ws.flags,
                                                            ws.leaf_pos, ws.wsmp, ws.bin_count);
    return cudaGetLastError();
}

cudaError_t launch_bucket(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const auto& ws = t->ws;
    const int qt = leaf_queries_per_tile(t);
    scan_bins_kernel<<<1, 1024, 0, s>>>(ws.bin_count, t->nb, qt, ws.bin_off, ws.tile_prefix, ws.misc, ws.stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t blocks = (t->n + 3) / 4;
    if (blocks > 152 * 32) blocks = 152 * 32;
    scatter_items_kernel<<<(int)blocks, 128, 0, s>>>(ws.node_bin, (int)t->n, kp.L, ws.bin_off, ws.bin_cursor,
                                                     ws.items_q, ws.items_mask);
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
