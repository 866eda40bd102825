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
//                 sample down to a single point, whose kernel value is kept
//                 for the weight of Eq. 2 (formed by the edge kernels).
#include "fsg_internal.cuh"

FSG_BOUNDS_TU(descend)

namespace fsg {
namespace {

__device__ __forceinline__ int k_of(int r, uint32_t b0, uint32_t b1, uint32_t below) {
    return r == 0 ? __popc(b0 & below) : __popc(b0) + __popc(b1 & below);
}

// Per query (one warp): segment tree of the query's node sums over levels
// 0..s0 built from its bin sums, the degree (the root), the first s0
// decisions of each of the query's L samples, and the compact list of the
// distinct bins its samples reached with the mask of samples at each.
__global__ void __launch_bounds__(256)
descend_top_kernel(const float* __restrict__ binsum, int n, int q_lo, int q_hi, int nb, int s0,
                   const int32_t* __restrict__ perm, KernelParams kp, int with_samples, double* __restrict__ d_deg,
                   float* __restrict__ degf,
                   uint8_t* __restrict__ flags, int32_t* __restrict__ leaf_pos, float* __restrict__ ksmp,
                   int32_t* __restrict__ bin_count, int32_t* __restrict__ qitem_bin,
                   uint64_t* __restrict__ qitem_mask, int32_t* __restrict__ qitem_cnt, uint16_t* __restrict__ flev) {
    extern __shared__ __align__(16) unsigned char smem_b[];
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* tree = reinterpret_cast<float*>(smem_b) + (size_t)w * 2 * nb;  // [2 nb] per warp
    const int L = kp.L;
    // Rows of 128..1024 bins move as float4 (one row = nb/128 per lane), the
    // next query's row in flight while the current one is processed; other
    // bin counts load one float per lane and iteration.
    const bool vec = (nb & 127) == 0 && nb <= 1024;
    const int nv = nb >> 7;
    const int qstride = gridDim.x * warps;
    float4 v[8];
    auto load_row = [&](int qq) {
        const float4* r4 = reinterpret_cast<const float4*>(binsum + (size_t)qq * nb);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < nv) v[k] = __ldcs(r4 + k * 32 + lane);
    };
    if (vec && q_lo + (int)blockIdx.x * warps + w < q_hi) load_row(q_lo + blockIdx.x * warps + w);
    for (int q = q_lo + blockIdx.x * warps + w; q < q_hi; q += qstride) {
        if (vec) {
            float4* t4 = reinterpret_cast<float4*>(tree + nb);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < nv) t4[k * 32 + lane] = v[k];
            if (q + qstride < q_hi) load_row(q + qstride);
        } else {
            const float* row = binsum + (size_t)q * nb;
            for (int b = lane; b < nb; b += 32) tree[nb + b] = row[b];
        }
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
                        // approximate bin sums miss at most kde_eps of the exact degree
                        // (root >= (1 - kde_eps) degree)
                        const float abs_tol = kp.kde_eps > 0.f ? kp.kde_eps * root / (1.f - kp.kde_eps) : 0.f;
                        uint32_t flev_m = 0;  // levels whose decision was flagged (re-decision)
                        for (int t = 0; t < s0; ++t) {
                            if ((t & 3) == 0) blk = draw_block(kp.seed, (uint32_t)i, (uint32_t)l, (uint32_t)t);
                            uint8_t ft = 0;
                            h = 2 * h + descend_decide(tree[2 * h], tree[2 * h + 1], block_word(blk, (uint32_t)t),
                                                       kp.flag_eps, ft, abs_tol);
                            flev_m |= (uint32_t)(ft & 1) << t;
                            f |= ft;
                        }
                        binv[r] = h - nb;
                        flags[(size_t)q * L + l] = f;
                        if (flev) flev[(size_t)q * L + l] = (uint16_t)flev_m;
                    }
                }
                __syncwarp();
                // Group the samples by bin: sample l's mask holds every sample
                // at its bin, gathered in a per-bin table that reuses the tree
                // storage (nb 64-bit words; the tree is no longer read).
                uint64_t* group = reinterpret_cast<uint64_t*>(tree);
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    if (binv[r] >= 0) group[binv[r]] = 0ull;
                __syncwarp();
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    if (binv[r] >= 0) atomicOr(reinterpret_cast<unsigned long long*>(group + binv[r]),
                                               1ull << (lane + 32 * r));
                __syncwarp();
                uint64_t M[2] = {0ull, 0ull};
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    if (binv[r] >= 0) M[r] = group[binv[r]];
                __syncwarp();
                // The lowest sample of each bin writes the (bin, mask) item of
                // this query; items are packed per query and counted per bin.
                bool lead[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int l = lane + 32 * r;
                    lead[r] = binv[r] >= 0 && (M[r] & ((1ull << l) - 1ull)) == 0ull;
                }
                const uint32_t b0 = __ballot_sync(0xffffffffu, lead[0]), b1 = __ballot_sync(0xffffffffu, lead[1]);
                const uint32_t below = (1u << lane) - 1u;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    if (lead[r] && FSG_INB(k_of(r, b0, b1, below), L, kSiteTopItem) && FSG_INB(binv[r], nb, kSiteTopItem)) {
                        const int k = r == 0 ? __popc(b0 & below) : __popc(b0) + __popc(b1 & below);
                        qitem_bin[(size_t)q * L + k] = binv[r];
                        qitem_mask[(size_t)q * L + k] = M[r];
                        atomicAdd(&bin_count[binv[r] * kBinSlots + (q & (kBinSlots - 1))], 1);
                    }
                }
                if (lane == 0) qitem_cnt[q] = __popc(b0) + __popc(b1);
            } else {
                // zero FP32 mass: no sample; flag unless no other point exists
                const uint8_t f = (n > 1 || !kp.self_exclude) ? 2 : 0;
                for (int l = lane; l < L; l += 32) {
                    leaf_pos[(size_t)q * L + l] = -1;
                    ksmp[(size_t)q * L + l] = 0.f;
                    flags[(size_t)q * L + l] = f;
                }
                if (lane == 0) qitem_cnt[q] = 0;
            }
        }
        __syncwarp();
    }
}

// Exclusive scan of the per-(bin, sub-slot) item counts (single CTA).  Bin b's
// segment is [bin_off[b * kBinSlots], bin_off[(b + 1) * kBinSlots]).
__global__ void __launch_bounds__(1024)
scan_bins_kernel(const int32_t* __restrict__ bin_count, int nb, int32_t* __restrict__ bin_off) {
    __shared__ int32_t s_items[1024];
    const int tid = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    int ci = 0;
    for (int u = 0; u < per; ++u) {
        const int b = tid * per + u;
        if (b < nb) ci += bin_count[b];
    }
    s_items[tid] = ci;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int vi = tid >= off ? s_items[tid - off] : 0;
        __syncthreads();
        s_items[tid] += vi;
        __syncthreads();
    }
    int ri = s_items[tid] - ci;
    for (int u = 0; u < per; ++u) {
        const int b = tid * per + u;
        if (b < nb) {
            bin_off[b] = ri;
            ri += bin_count[b];
        }
    }
    if (tid == 1023) bin_off[nb] = s_items[1023];
}

// Items of every query into their bin's segment [bin_off[b], bin_off[b+1]).
__global__ void __launch_bounds__(128)
scatter_items_kernel(const int32_t* __restrict__ qitem_bin, const uint64_t* __restrict__ qitem_mask,
                     const int32_t* __restrict__ qitem_cnt, int q_lo, int q_hi, int L,
                     const int32_t* __restrict__ bin_off, int32_t* __restrict__ bin_cursor,
                     int32_t* __restrict__ items_q, uint64_t* __restrict__ items_mask, long long max_items) {
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = q_lo + blockIdx.x * warps + w; q < q_hi; q += gridDim.x * warps) {
        const int cnt = qitem_cnt[q];
        for (int k = lane; k < cnt; k += 32) {
            const int b = qitem_bin[(size_t)q * L + k] * kBinSlots + (q & (kBinSlots - 1));
            const int slot = bin_off[b] + atomicAdd(&bin_cursor[b], 1);
            if (!FSG_INB(slot, max_items, kSiteScatter)) continue;
            items_q[slot] = q;
            items_mask[slot] = qitem_mask[(size_t)q * L + k];
        }
    }
}

constexpr int kThreadsC = 256;

constexpr int kLeafWords = 256;   // Philox blocks precomputed per chunk (more: computed inline)

// Shared-memory layout of the leaf finish (same arithmetic on host and device).
struct LeafSmem {
    size_t P, spos, V, qmask, qpos, qidx, qdeg, loff, list, W, total;
    __host__ __device__ static size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
    __host__ __device__ LeafSmem(int leafmax, int dh, int qc) {
        const size_t vs = 2 * (size_t)leafmax + 1;
        P = 0;
        spos = up16(P + (size_t)(leafmax / 2 + 2) * dh * 16);
        V = up16(spos + (size_t)(leafmax + 4) * 4);
        qmask = up16(V + (size_t)qc * vs * 4);
        qpos = up16(qmask + (size_t)qc * 8);
        qidx = up16(qpos + (size_t)qc * 4);
        qdeg = up16(qidx + (size_t)qc * 4);            // query coordinates [qc][16]
        loff = up16(qdeg + (size_t)qc * 16 * 4);
        list = up16(loff + (size_t)(qc + 1) * 4);
        W = up16(list + (size_t)qc * 64 * 4);
        total = up16(W + (size_t)kLeafWords * 16);
    }
};

// Leaf finish: CTA (b, y) handles chunks y, y + gridDim.y, ... of bin b's
// item list, qc <= 32 items (queries) per chunk, lane = query.  The bin's
// points are laid out in shared memory by leaf slot of the bin's perfect
// binary tree (slot = path bits of the halving descent), two slots
// interleaved per 16-byte word so that one load yields FP32x2 operands for
// two slots; empty slots hold coordinate 1e19 and evaluate to exactly 0.
// Warp w evaluates slot pairs w, w+8, ... for every query of the chunk; the
// per-query trees are summed upwards in shared memory (rows of odd stride, so
// the lanes' stores hit distinct banks); then one thread per (query, sample)
// takes the remaining decisions and forms the weight w = k / p_hat (Eq. 2).
// FROM_GLOBAL: the leaf values were computed by another kernel (any d) and
// are read from leafv[item][slot] instead of being evaluated here.
template <int D, bool FROM_GLOBAL>
__global__ void __launch_bounds__(kThreadsC, 4)
leaf_finish_kernel(const float* __restrict__ Xt, const int32_t* __restrict__ perm, const int32_t* __restrict__ bnd,
                   int n, int s0, const int32_t* __restrict__ bin_off, const int32_t* __restrict__ items_q,
                   const uint64_t* __restrict__ items_mask, const float* __restrict__ leafv, KernelParams kp,
                   int qc_max, int dm_max,
                   int32_t* __restrict__ leaf_pos, float* __restrict__ ksmp, uint8_t* __restrict__ lflags,
                   unsigned long long* __restrict__ n_evals, unsigned long long* __restrict__ n_items) {
    constexpr int DP = (D + 3) & ~3;
    constexpr int DH = (D + 1) / 2;  // 16-byte words per slot pair
    const int b = blockIdx.x;
    const int cnt = bin_off[(b + 1) * kBinSlots] - bin_off[b * kBinSlots];
    const int nchunks = (cnt + qc_max - 1) / qc_max;
    if ((int)blockIdx.y >= nchunks) return;

    extern __shared__ __align__(16) unsigned char smem_c[];
    const int leafmax = 1 << dm_max;
    const int vs = 2 * leafmax + 1;  // odd row stride
    const LeafSmem lay(leafmax, DH, qc_max);
    float4* P = reinterpret_cast<float4*>(smem_c + lay.P);           // [leafmax/2 + 2][DH] slot pairs
    int32_t* spos = reinterpret_cast<int32_t*>(smem_c + lay.spos);   // [leafmax + 4] slot -> position
    float* V = reinterpret_cast<float*>(smem_c + lay.V);             // [qc_max][vs] per-query trees
    uint64_t* qmask = reinterpret_cast<uint64_t*>(smem_c + lay.qmask);
    int32_t* qpos = reinterpret_cast<int32_t*>(smem_c + lay.qpos);
    int32_t* qidx = reinterpret_cast<int32_t*>(smem_c + lay.qidx);
    float* qco = reinterpret_cast<float*>(smem_c + lay.qdeg);        // [qc_max][DP] query coordinates
    int32_t* loff = reinterpret_cast<int32_t*>(smem_c + lay.loff);   // qc_max + 1
    int32_t* list = reinterpret_cast<int32_t*>(smem_c + lay.list);   // qc_max * 64
    uint4* W = reinterpret_cast<uint4*>(smem_c + lay.W);              // [kLeafWords] Philox blocks

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int L = kp.L;
    const int p_lo = bnd[b];
    const int m = bnd[b + 1] - p_lo;
    const int dm = ceil_log2_dev(m);
    const int leaf0 = 1 << dm;
    // Slot table and pair-interleaved point coordinates.
    for (int sl = tid; !FROM_GLOBAL && sl < 4 * ((leaf0 + 3) / 4); sl += kThreadsC) {
        int a = 0, c = m;  // walk the slot's path bits from the root
        for (int t = dm - 1; t >= 0; --t) {
            const int mid = a + (c - a) / 2;
            if ((sl >> t) & 1) a = mid; else c = mid;
        }
        const int pos = (sl < leaf0 && c - a == 1) ? p_lo + a : -1;
        spos[sl] = pos;
        float* Pw = reinterpret_cast<float*>(P + (size_t)(sl >> 1) * DH);
#pragma unroll
        for (int u = 0; u < DH; ++u) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = 2 * u + h;
                const float v = (t < D) ? (pos >= 0 ? Xt[(size_t)pos * DP + t] : 1e19f) : 0.f;
                Pw[4 * u + 2 * h + (sl & 1)] = v;
            }
        }
    }
    const uint64_t nc2 = f2_pack(kp.neg_c, kp.neg_c);
    const size_t base = (size_t)bin_off[b * kBinSlots];
    // Warp 0 holds the next chunk's items (query, mask, index, coordinates) in
    // registers: their global loads overlap the current chunk's work.
    int nx_q = -1, nx_i = 0;
    uint64_t nx_m = 0ull;
    float nx_x[D];
    auto fetch = [&](int chunk) {
        const int it = chunk * qc_max + lane;
        nx_q = -1;
        if (chunk < nchunks && lane < qc_max && it < cnt) {
            nx_q = items_q[base + it];
            nx_m = items_mask[base + it];
            nx_i = perm[nx_q];
            if (!FROM_GLOBAL) {
#pragma unroll
                for (int t = 0; t < D; ++t) nx_x[t] = Xt[(size_t)nx_q * DP + t];
            }
        }
    };
    if (tid < 32) fetch(blockIdx.y);
    unsigned long long ev_acc = 0, it_acc = 0;
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int it0 = chunk * qc_max;
        const int qcnt = min(qc_max, cnt - it0);
        if (tid < 32) {
            if (lane < qcnt) {
                qpos[lane] = nx_q;
                qidx[lane] = nx_i;
                qmask[lane] = nx_m;
                if (!FROM_GLOBAL) {
#pragma unroll
                    for (int t = 0; t < D; ++t) qco[lane * DP + t] = nx_x[t];
                }
            }
            fetch(chunk + gridDim.y);
        }
        __syncthreads();
        if (FROM_GLOBAL) {
            for (int e = tid; e < qcnt * leaf0; e += kThreadsC) {
                const int qq = e >> dm, sl = e & (leaf0 - 1);
                V[(size_t)qq * vs + leaf0 + sl] = leafv[(base + it0 + qq) * (size_t)leafmax + sl];
            }
        }
        // List of (query, sample) pairs of this chunk (warp 0, lane = query),
        // built before warp 0's share of the kernel values.
        if (tid < 32) {
            const uint64_t mk0 = tid < qcnt ? qmask[tid] : 0ull;
            const int c0 = __popcll(mk0);
            int sv = c0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, sv, o);
                if (tid >= o) sv += y;
            }
            int off = sv - c0;
            if (tid < qcnt) loff[tid] = off;
            if (tid == 31) loff[qcnt] = sv;
            for (uint64_t mk = mk0; mk; mk &= mk - 1ull) list[off++] = (tid << 6) | (__ffsll((long long)mk) - 1);
        }
        // Kernel values: lane = query.  Bins of 128 leaf slots: warp w takes the
        // contiguous slots 16 w .. 16 w + 15 and sums that subtree in registers
        // (no barrier between its levels).  Other sizes: warp w takes slot
        // pairs w, w + 8, ... and the levels are summed in shared memory.
        const bool sub16 = !FROM_GLOBAL && leaf0 == 128;
        if (!FROM_GLOBAL && lane < qc_max) {
            const bool qv = lane < qcnt;
            const int my_pos = qv ? qpos[lane] : -2;
            uint64_t qd[D];
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const float x = qv ? qco[lane * DP + t] : 1e19f;
                qd[t] = f2_pack(x, x);
            }
            float* row = V + (size_t)lane * vs;
            // kernel values of slot pair pp (two slots), masked at the query itself
            auto pair_values = [&](int pp, float& k0, float& k1) {
                const float4* Pp = P + (size_t)pp * DH;
                uint64_t s2 = 0ull, s3 = 0ull;
#pragma unroll
                for (int u = 0; u < DH; ++u) {
                    const float4 c4 = Pp[u];
                    const uint64_t ca = f2_pack(c4.x, c4.y), cb = f2_pack(c4.z, c4.w);
                    uint64_t dd = f2_sub(qd[2 * u], ca);
                    s2 = u == 0 ? f2_mul(dd, dd) : f2_fma(dd, dd, s2);
                    if (2 * u + 1 < D) {
                        dd = f2_sub(qd[2 * u + 1], cb);
                        s3 = u == 0 ? f2_mul(dd, dd) : f2_fma(dd, dd, s3);
                    }
                }
                if (D > 1) s2 = f2_add(s2, s3);
                const float2 sv = f2_unpack(f2_mul(s2, nc2));
                k0 = ex2_approx(sv.x);
                k1 = ex2_approx(sv.y);
                if (kp.self_exclude) {
                    if (spos[2 * pp] == my_pos) k0 = 0.f;
                    if (spos[2 * pp + 1] == my_pos) k1 = 0.f;
                }
            };
            if (sub16) {
                float lv[16];
#pragma unroll
                for (int j = 0; j < 8; ++j) pair_values(8 * w + j, lv[2 * j], lv[2 * j + 1]);
                // heap positions: leaves 128 + 16 w + i, then halves up to the subtree root 8 + w
#pragma unroll
                for (int i = 0; i < 16; ++i) row[128 + 16 * w + i] = lv[i];
#pragma unroll
                for (int width = 8; width >= 1; width >>= 1) {
#pragma unroll
                    for (int i = 0; i < width; ++i) {
                        lv[i] = lv[2 * i] + lv[2 * i + 1];
                        row[8 * width + width * w + i] = lv[i];
                    }
                }
            } else {
                // Quads of 4 consecutive slots (two slot pairs): leaves, their two
                // parents and their grandparent are formed here, in registers.
                const int nquad = (leaf0 + 3) / 4;
                for (int j = w; j < nquad; j += kThreadsC / 32) {
                    float kq[4];
                    pair_values(2 * j, kq[0], kq[1]);
                    pair_values(2 * j + 1, kq[2], kq[3]);
                    const int s4 = 4 * j;
                    if (leaf0 >= 4) {
                        row[leaf0 + s4] = kq[0];
                        row[leaf0 + s4 + 1] = kq[1];
                        row[leaf0 + s4 + 2] = kq[2];
                        row[leaf0 + s4 + 3] = kq[3];
                        const float p0 = kq[0] + kq[1], p1 = kq[2] + kq[3];
                        row[(leaf0 + s4) / 2] = p0;
                        row[(leaf0 + s4) / 2 + 1] = p1;
                        row[(leaf0 + s4) / 4] = p0 + p1;
                    } else {
                        for (int x = 0; x < leaf0; ++x) row[leaf0 + x] = kq[x];
                        if (leaf0 == 2) row[1] = kq[0] + kq[1];
                    }
                }
            }
        }
        __syncthreads();
        if (sub16) {  // the top three levels over the eight subtree roots, one thread per query
            if (tid < qcnt) {
                float* r = V + (size_t)tid * vs;
                float l2[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    l2[i] = r[8 + 2 * i] + r[9 + 2 * i];
                    r[4 + i] = l2[i];
                }
                const float a2 = l2[0] + l2[1], b2 = l2[2] + l2[3];
                r[2] = a2;
                r[3] = b2;
                r[1] = a2 + b2;
            }
        } else {
            for (int lev = FROM_GLOBAL ? dm - 1 : dm - 3; lev >= 0; --lev) {
                const int cn = qcnt << lev;
                for (int e = tid; e < cn; e += kThreadsC) {
                    const int qq = e >> lev;
                    const int h = (1 << lev) + (e & ((1 << lev) - 1));
                    float* r = V + (size_t)qq * vs;
                    r[h] = r[2 * h] + r[2 * h + 1];
                }
                if (lev > 0) __syncthreads();
            }
        }
        // (the Philox blocks below are drawn in the same phase as the last tree level)
        // Philox blocks of every sample's remaining levels, one per thread.
        const int nsamp = loff[qcnt];
        const int blk0 = s0 >> 2;
        const int nblk = dm > 0 ? ((s0 + dm - 1) >> 2) - blk0 + 1 : 0;
        const bool pre = nsamp * nblk <= kLeafWords;
        if (pre) {
            for (int e = tid; e < nsamp * nblk; e += kThreadsC) {
                const int sidx = e / nblk, jb = e - sidx * nblk;
                const int qq = list[sidx] >> 6, l = list[sidx] & 63;
                W[e] = draw_block(kp.seed, (uint32_t)qidx[qq], (uint32_t)l, (uint32_t)(4 * (blk0 + jb)));
            }
        }
        __syncthreads();  // tree and Philox blocks complete
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
                        blk_id = (int)(lev >> 2);
                        blk = pre ? W[e * nblk + (blk_id - blk0)] : draw_block(kp.seed, i, (uint32_t)l, lev);
                    }
                    const int mid = a + (c - a) / 2;
                    const int right = descend_decide(row[2 * h], row[2 * h + 1], block_word(blk, lev), kp.flag_eps, f);
                    if (right) a = mid; else c = mid;
                    h = 2 * h + right;
                } else {
                    h = 2 * h + 1;  // a single point sits in the right half
                }
            }
            const size_t o = (size_t)qpos[qq] * L + l;
            if (FSG_INB(o, (long long)n * L, kSiteLeafFinish)) {
                leaf_pos[o] = p_lo + a;
                ksmp[o] = row[h];
                lflags[o] = f;
            }
        }
        ev_acc += (unsigned long long)qcnt * (unsigned long long)m;
        it_acc += (unsigned long long)qcnt;
        __syncthreads();
    }
    if (tid == 0) {
        atomicAdd(n_evals, ev_acc);
        atomicAdd(n_items, it_acc);
    }
}

template <int D, bool FROM_GLOBAL = false>
cudaError_t launch_leaf_d(const fsg_tree* t, const KernelParams& kp, int qc, cudaStream_t s) {
    constexpr int DH = (D + 1) / 2;
    const size_t smem = LeafSmem(1 << t->dm, DH, qc).total;
    {
        const cudaError_t e = set_smem_limit(leaf_finish_kernel<D, FROM_GLOBAL>, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    int64_t S = leaf_default_splits(t, kp.L);
    if (t->tune.leaf_splits > 0) S = t->tune.leaf_splits;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    dim3 grid(t->nb, (unsigned)S);
    const auto& ws = t->ws;
    leaf_finish_kernel<D, FROM_GLOBAL><<<grid, kThreadsC, smem, s>>>(
        t->Xt, t->perm, t->bnd, (int)t->n, t->s0, ws.bin_off, ws.items_q, ws.items_mask, ws.leafv, kp, qc, t->dm,
        ws.leaf_pos, ws.ksmp, ws.lflags, reinterpret_cast<unsigned long long*>(&ws.stats->n_evals),
        reinterpret_cast<unsigned long long*>(&ws.stats->n_items));
    return cudaGetLastError();
}

// Leaf finish for bins of 65..128 points (seven halvings below the bin,
// d <= 16): chunks of 128 items, one item per thread.
//  * Node sums: warp w owns the bin's quarter w (the depth-2 node w below the
//    bin) and evaluates only its real points, for two items per lane packed
//    into the two FP32x2 lanes (both use the same point coordinates), in
//    groups of the 2..4 points of a depth-5 node.  It keeps the sums of
//    depths 2..4 (nodes 4..31 in heap order).
//  * Descent: each thread forms its item's nodes 2 and 3 and descends the
//    item's samples through depths 0..3 on the kept sums.  Below the depth-4
//    node reached (4..8 points) it evaluates that node's points again with the
//    same arithmetic (scalar FP32, the same rounding as one packed lane) and
//    takes the remaining decisions on partial sums of those values.
// Two barriers per chunk of 128 items.
constexpr int kLC = 128;  // items per chunk = threads per CTA
constexpr int kLV = 31;   // kept node sums per item (node h at h - 1), odd row stride
constexpr int kL128List = 1024;  // (item, sample) pairs descended per window

// Kernel values of the point at Pr for two queries (packed lanes), the point
// dropped for a query whose own local index it is.  F: the kernel family.
template <int D, int F, bool SELF>
__device__ __forceinline__ uint64_t leaf_kv2(const uint64_t (&qd)[D], const float4* __restrict__ Pr, uint64_t nc2,
                                             int r, int sa, int sb) {
    constexpr int DH = (D + 1) / 2;
    uint64_t s2 = 0ull, s3 = 0ull;
#pragma unroll
    for (int u = 0; u < DH; ++u) {
        const float4 c4 = Pr[u];
        uint64_t dd = f2_sub(qd[2 * u], f2_pack(c4.x, c4.y));
        s2 = u == 0 ? fam_first2<F>(dd) : fam_acc2<F>(dd, s2);
        if (2 * u + 1 < D) {
            dd = f2_sub(qd[2 * u + 1], f2_pack(c4.z, c4.w));
            s3 = u == 0 ? fam_first2<F>(dd) : fam_acc2<F>(dd, s3);
        }
    }
    if (D > 1) s2 = f2_add(s2, s3);
    const float2 sv = f2_unpack(f2_mul(fam_fin2<F>(s2), nc2));
    float ka = ex2_approx(sv.x), kb = ex2_approx(sv.y);
    if (SELF) {
        if (r == sa) ka = 0.f;
        if (r == sb) kb = 0.f;
    }
    return f2_pack(ka, kb);
}

// One lane of leaf_kv2, operation for operation.
template <int D, int F>
__device__ __forceinline__ float leaf_kv1(const float (&x)[D], const float4* __restrict__ Pr, float neg_c) {
    constexpr int DH = (D + 1) / 2;
    float s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int u = 0; u < DH; ++u) {
        const float4 c4 = Pr[u];
        float dd = __fsub_rn(x[2 * u], c4.x);
        s2 = u == 0 ? fam_first1<F>(dd) : fam_acc1<F>(dd, s2);
        if (2 * u + 1 < D) {
            dd = __fsub_rn(x[2 * u + 1], c4.z);
            s3 = u == 0 ? fam_first1<F>(dd) : fam_acc1<F>(dd, s3);
        }
    }
    if (D > 1) s2 = __fadd_rn(s2, s3);
    return ex2_approx(__fmul_rn(fam_fin1<F>(s2), neg_c));
}

// Sums of the eight depth-5 nodes of quarter w for the lane's two items.
template <int D, int F, bool SELF>
__device__ __forceinline__ void leaf_quarter(const uint64_t (&qd)[D], const float4* __restrict__ P2,
                                             const int32_t* __restrict__ r5, int w, uint64_t nc2, int sa, int sb,
                                             uint64_t (&n5)[8]) {
    constexpr int DH = (D + 1) / 2;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int r0 = r5[8 * w + j], c = r5[8 * w + j + 1] - r0;  // 2..4 points
        uint64_t v = f2_add(leaf_kv2<D, F, SELF>(qd, P2 + (size_t)r0 * DH, nc2, r0, sa, sb),
                            leaf_kv2<D, F, SELF>(qd, P2 + (size_t)(r0 + 1) * DH, nc2, r0 + 1, sa, sb));
        if (c > 2) {
            uint64_t v2 = leaf_kv2<D, F, SELF>(qd, P2 + (size_t)(r0 + 2) * DH, nc2, r0 + 2, sa, sb);
            if (c > 3) v2 = f2_add(v2, leaf_kv2<D, F, SELF>(qd, P2 + (size_t)(r0 + 3) * DH, nc2, r0 + 3, sa, sb));
            v = f2_add(v, v2);
        }
        n5[j] = v;
    }
}

template <int D>
struct Leaf128Layout {
    static constexpr int DP = (D + 3) & ~3;
    static constexpr int DH = (D + 1) / 2;
    static constexpr int QS = D | 1;  // odd row stride of the item coordinates
    static constexpr size_t P2 = 0;                                    // float4 [128][DH]: (c, c, c', c')
    static constexpr size_t R5 = P2 + (size_t)128 * DH * 16;           // int [33] depth-5 node starts
    static constexpr size_t QMASK = R5 + 48 * 4;                       // uint64 [128]
    static constexpr size_t QPOS = QMASK + (size_t)kLC * 8;            // int [128]
    static constexpr size_t QIDX = QPOS + (size_t)kLC * 4;             // int [128]
    static constexpr size_t QCO = QIDX + (size_t)kLC * 4;              // float [128][QS]
    static constexpr size_t V = QCO + (((size_t)kLC * QS * 4 + 15) & ~size_t(15));  // float [128][31]
    static constexpr size_t LIST = V + (size_t)kLC * kLV * 4;                  // uint16 [kL128List] (item, sample)
    static constexpr size_t WSUM = LIST + (size_t)kL128List * 2;               // int [4] samples per warp
    static constexpr size_t total = WSUM + 16;
};

template <int D, int F>
__global__ void __launch_bounds__(kLC)
leaf128_kernel(const float* __restrict__ Xt, const int32_t* __restrict__ perm, const int32_t* __restrict__ bnd,
               int s0, const int32_t* __restrict__ bin_off, const int32_t* __restrict__ items_q,
               const uint64_t* __restrict__ items_mask, KernelParams kp, int32_t* __restrict__ leaf_pos,
               float* __restrict__ ksmp, uint8_t* __restrict__ lflags, unsigned long long* __restrict__ n_evals,
               unsigned long long* __restrict__ n_items, long long nl) {
    using LY = Leaf128Layout<D>;
    constexpr int DP = LY::DP, DH = LY::DH, QS = LY::QS;
    extern __shared__ __align__(16) unsigned char smem128[];
    float4* P2 = reinterpret_cast<float4*>(smem128 + LY::P2);
    int32_t* r5 = reinterpret_cast<int32_t*>(smem128 + LY::R5);
    uint64_t* qmask = reinterpret_cast<uint64_t*>(smem128 + LY::QMASK);
    int32_t* qpos = reinterpret_cast<int32_t*>(smem128 + LY::QPOS);
    int32_t* qidx = reinterpret_cast<int32_t*>(smem128 + LY::QIDX);
    float* qco = reinterpret_cast<float*>(smem128 + LY::QCO);
    float* V = reinterpret_cast<float*>(smem128 + LY::V);
    uint16_t* plist = reinterpret_cast<uint16_t*>(smem128 + LY::LIST);
    int32_t* wsum = reinterpret_cast<int32_t*>(smem128 + LY::WSUM);
    const int b = blockIdx.x;
    const int base = bin_off[b * kBinSlots];
    const int cnt = bin_off[(b + 1) * kBinSlots] - base;
    const int nchunks = (cnt + kLC - 1) / kLC;
    if ((int)blockIdx.y >= nchunks) return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int p_lo = bnd[b], m = bnd[b + 1] - p_lo;  // 65 <= m <= 128
    if (tid < m) {
#pragma unroll
        for (int u = 0; u < DH; ++u) {
            const float c0 = Xt[(size_t)(p_lo + tid) * DP + 2 * u];
            const float c1 = (2 * u + 1 < D) ? Xt[(size_t)(p_lo + tid) * DP + 2 * u + 1] : 0.f;
            P2[(size_t)tid * DH + u] = make_float4(c0, c0, c1, c1);
        }
    }
    if (tid <= 32) {  // start of depth-5 node tid of the bin (tid = 32: the end)
        int a = 0, c = m;
        if (tid < 32) {
            for (int t = 4; t >= 0; --t) {
                const int mid = a + (c - a) / 2;
                if ((tid >> t) & 1) a = mid; else c = mid;
            }
        } else {
            a = m;
        }
        r5[tid] = a;
    }
    const uint64_t nc2 = f2_pack(kp.neg_c, kp.neg_c);
    const int L = kp.L;
    const size_t ibase = (size_t)base;
    unsigned long long ev_acc = 0, it_acc = 0;
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int it0 = chunk * kLC;
        const int qcnt = min(kLC, cnt - it0);
        if (tid < qcnt) {
            const int q = items_q[ibase + it0 + tid];
            qpos[tid] = q;
            qidx[tid] = perm[q];
            qmask[tid] = items_mask[ibase + it0 + tid];
#pragma unroll
            for (int t = 0; t < D; ++t) qco[tid * QS + t] = Xt[(size_t)q * DP + t];
        } else {
            qpos[tid] = -1;
            qmask[tid] = 0ull;
#pragma unroll
            for (int t = 0; t < D; ++t) qco[tid * QS + t] = 1e19f;  // far away: every value is 0
        }
        __syncthreads();
        // node sums of depths 2..4 over quarter w, two items per lane
        for (int pass = 0; pass < kLC / 64; ++pass) {
            if (64 * pass >= qcnt) break;  // warp-uniform
            const int ia = 64 * pass + lane, ib = ia + 32;
            uint64_t qd[D];
#pragma unroll
            for (int t = 0; t < D; ++t) qd[t] = f2_pack(qco[ia * QS + t], qco[ib * QS + t]);
            const int sa = qpos[ia] - p_lo, sb = qpos[ib] - p_lo;  // local index of the query itself
            const int lo = r5[8 * w], hi = r5[8 * w + 8];
            const bool self_here = kp.self_exclude &&
                                   __any_sync(0xffffffffu, (sa >= lo && sa < hi) || (sb >= lo && sb < hi));
            uint64_t n5[8];
            if (self_here) leaf_quarter<D, F, true>(qd, P2, r5, w, nc2, sa, sb, n5);
            else leaf_quarter<D, F, false>(qd, P2, r5, w, nc2, sa, sb, n5);
            uint64_t n4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) n4[i] = f2_add(n5[2 * i], n5[2 * i + 1]);
            const uint64_t n3a = f2_add(n4[0], n4[1]), n3b = f2_add(n4[2], n4[3]);
            const uint64_t n2 = f2_add(n3a, n3b);
            float* Va = V + (size_t)ia * kLV;
            float* Vb = V + (size_t)ib * kLV;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 v = f2_unpack(n4[i]);
                Va[15 + 4 * w + i] = v.x;
                Vb[15 + 4 * w + i] = v.y;
            }
            const float2 v3a = f2_unpack(n3a), v3b = f2_unpack(n3b), v2 = f2_unpack(n2);
            Va[7 + 2 * w] = v3a.x;
            Vb[7 + 2 * w] = v3a.y;
            Va[8 + 2 * w] = v3b.x;
            Vb[8 + 2 * w] = v3b.y;
            Va[3 + w] = v2.x;
            Vb[3 + w] = v2.y;
        }
        __syncthreads();
        // descents: the chunk's (item, sample) pairs spread over all threads
        // (an item holds 1..64 samples, so one thread per item would leave
        // most lanes idle behind the few items with many); exclusive offsets
        // of the items' sample counts, then windows of kL128List pairs.
        const int ns = tid < qcnt ? __popcll(qmask[tid]) : 0;
        int incl = ns;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        if (tid < qcnt) {
            float* row = V + (size_t)tid * kLV;
            row[1] = row[3] + row[4];  // node 2
            row[2] = row[5] + row[6];  // node 3
        }
        __syncthreads();
        int wbase = 0;
#pragma unroll
        for (int k = 0; k < kLC / 32; ++k) wbase += k < w ? wsum[k] : 0;
        const int total = wsum[0] + wsum[1] + wsum[2] + wsum[3];
        const int my_off = wbase + incl - ns;
        for (int r0 = 0; r0 < total; r0 += kL128List) {
            if (r0 > 0) __syncthreads();  // the previous window's pairs are taken
            if (ns > 0 && my_off < r0 + kL128List && my_off + ns > r0) {
                int o = my_off;
                for (uint64_t mk = qmask[tid]; mk; mk &= mk - 1ull, ++o)
                    if (o >= r0 && o < r0 + kL128List)
                        plist[o - r0] = (uint16_t)((tid << 6) | (__ffsll((long long)mk) - 1));
            }
            __syncthreads();
            const int cnt_w = min(kL128List, total - r0);
            for (int e = tid; e < cnt_w; e += kLC) {
                const int it = plist[e] >> 6, l = plist[e] & 63;
                const float* row = V + (size_t)it * kLV;
                const int my_pos = qpos[it];
                const int s_self = kp.self_exclude ? my_pos - p_lo : -1;
                const uint32_t qi = (uint32_t)qidx[it];
                float x[D];
#pragma unroll
                for (int t = 0; t < D; ++t) x[t] = qco[it * QS + t];
                int a = 0, c = m, h = 1;
                uint8_t f = 0;
                uint4 blk = make_uint4(0, 0, 0, 0);
                int blk_id = -1;
                for (int t = 0; t < 4; ++t) {  // nodes of >= 8 points
                    const uint32_t lev = (uint32_t)(s0 + t);
                    if ((int)(lev >> 2) != blk_id) {
                        blk_id = (int)(lev >> 2);
                        blk = draw_block(kp.seed, qi, (uint32_t)l, lev);
                    }
                    const int right = descend_decide(row[2 * h - 1], row[2 * h], block_word(blk, lev), kp.flag_eps, f);
                    const int mid = a + (c - a) / 2;
                    if (right) a = mid; else c = mid;
                    h = 2 * h + right;
                }
                // the depth-4 node [a, c) of 4..8 points, evaluated again
                const int a0 = a, cnt4 = c - a;
                float lf[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    lf[k] = 0.f;
                    if (k < cnt4 && a0 + k != s_self) lf[k] = leaf_kv1<D, F>(x, P2 + (size_t)(a0 + k) * DH, kp.neg_c);
                }
                for (int t = 4; t < 7; ++t) {
                    if (c - a < 2) break;
                    const int mid = a + (c - a) / 2;
                    float gl = 0.f, gr = 0.f;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int r = a0 + k;
                        if (r >= a && r < mid) gl += lf[k];
                        if (r >= mid && r < c) gr += lf[k];
                    }
                    const uint32_t lev = (uint32_t)(s0 + t);
                    if ((int)(lev >> 2) != blk_id) {
                        blk_id = (int)(lev >> 2);
                        blk = draw_block(kp.seed, qi, (uint32_t)l, lev);
                    }
                    const int right = descend_decide(gl, gr, block_word(blk, lev), kp.flag_eps, f);
                    if (right) a = mid; else c = mid;
                }
                float kval = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (a0 + k == a) kval = lf[k];
                const size_t o = (size_t)my_pos * L + l;
                if (FSG_INB(o, nl, kSiteLeaf128)) {
                    leaf_pos[o] = p_lo + a;
                    ksmp[o] = kval;
                    lflags[o] = f;
                }
            }
        }
        ev_acc += (unsigned long long)qcnt * (unsigned long long)m;
        it_acc += (unsigned long long)qcnt;
        __syncthreads();
    }
    if (tid == 0) {
        atomicAdd(n_evals, ev_acc);
        atomicAdd(n_items, it_acc);
    }
}


template <int D, int F>
cudaError_t launch_leaf128_d(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    int64_t S = leaf_default_splits(t, kp.L);
    if (t->tune.leaf_splits > 0) S = t->tune.leaf_splits;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    dim3 grid(t->nb, (unsigned)S);
    const auto& ws = t->ws;
    constexpr size_t smem = Leaf128Layout<D>::total;
    {
        const cudaError_t e = set_smem_limit(leaf128_kernel<D, F>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    leaf128_kernel<D, F><<<grid, kLC, smem, s>>>(t->Xt, t->perm, t->bnd, t->s0, ws.bin_off, ws.items_q, ws.items_mask,
                                              kp, ws.leaf_pos, ws.ksmp, ws.lflags,
                                              reinterpret_cast<unsigned long long*>(&ws.stats->n_evals),
                                              reinterpret_cast<unsigned long long*>(&ws.stats->n_items),
                                              t->n * (long long)kp.L);
    return cudaGetLastError();
}

}  // namespace

bool use_leaf128(const fsg_tree* t) {
    return t->dm == 7 && t->d <= kMaxFmaDim && t->n / t->nb >= 65;  // every bin holds 65..128 points
}

// CTAs per bin of the d <= 16 leaf kernels: a few waves over the expected
// items (one per (query, bin) reached, at most min(L, nb) per query).
int64_t leaf_default_splits(const fsg_tree* t, int L) {
    const int64_t items_est = t->n * (int64_t)(L < t->nb ? L : t->nb);
    const bool c128 = use_leaf128(t);
    const int qc = c128 ? 128 : leaf_queries_per_tile(t);
    const int64_t chunks_per_bin = (items_est / t->nb + qc - 1) / qc + 1;
    int64_t S = ((c128 ? 152 * 6 * 4 : 152 * 4 * 8) + t->nb - 1) / t->nb;
    if (S > chunks_per_bin) S = chunks_per_bin;
    return S < 1 ? 1 : S;
}

int leaf_queries_per_tile(const fsg_tree* t) {
    int qc = 8192 / (2 << t->dm);  // <= 32 KB of per-query trees, one query per lane
    if (qc > 32) qc = 32;
    if (qc < 1) qc = 1;
    return qc;
}

cudaError_t launch_descend_top(const fsg_tree* t, const KernelParams& kp, double* d_deg, int with_samples,
                               cudaStream_t s, int64_t q_lo, int64_t q_hi) {
    if (q_hi < 0) q_hi = t->n;
    int warps = 8;
    while (warps > 1 && (size_t)warps * 8 * t->nb > 96 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * 8 * t->nb;  // per warp: 2 nb tree nodes (later nb bin masks)
    {
        const cudaError_t e = set_smem_limit(descend_top_kernel, smem < 48 * 1024 ? 48 * 1024 : smem);
        if (e != cudaSuccess) return e;
    }
    int64_t blocks = (q_hi - q_lo + warps - 1) / warps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) return cudaSuccess;
    const auto& ws = t->ws;
    descend_top_kernel<<<(int)blocks, warps * 32, smem, s>>>(ws.binsum, (int)t->n, (int)q_lo, (int)q_hi, t->nb,
                                                            t->s0, t->perm, kp,
                                                            with_samples, d_deg, ws.degf, ws.flags, ws.leaf_pos,
                                                            ws.ksmp, ws.bin_count, ws.qitem_bin, ws.qitem_mask,
                                                            ws.qitem_cnt,
                                                            kp.resolve && with_samples ? t->rs.flev : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_bucket(const fsg_tree* t, const KernelParams& kp, cudaStream_t s, int64_t q_lo, int64_t q_hi) {
    if (q_hi < 0) q_hi = t->n;
    const auto& ws = t->ws;
    scan_bins_kernel<<<1, 1024, 0, s>>>(ws.bin_count, t->nb * kBinSlots, ws.bin_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t blocks = (q_hi - q_lo + 3) / 4;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) return cudaSuccess;
    const long long max_items = t->n * (long long)(ws.cap_L < t->nb ? ws.cap_L : t->nb);
    scatter_items_kernel<<<(int)blocks, 128, 0, s>>>(ws.qitem_bin, ws.qitem_mask, ws.qitem_cnt, (int)q_lo,
                                                     (int)q_hi, kp.L, ws.bin_off, ws.bin_cursor, ws.items_q,
                                                     ws.items_mask, max_items);
    return cudaGetLastError();
}

template <int F>
cudaError_t launch_leaf128_family(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    switch (t->d) {
        case 1: return launch_leaf128_d<1, F>(t, kp, s);
        case 2: return launch_leaf128_d<2, F>(t, kp, s);
        case 3: return launch_leaf128_d<3, F>(t, kp, s);
        case 4: return launch_leaf128_d<4, F>(t, kp, s);
        case 5: return launch_leaf128_d<5, F>(t, kp, s);
        case 6: return launch_leaf128_d<6, F>(t, kp, s);
        case 7: return launch_leaf128_d<7, F>(t, kp, s);
        case 8: return launch_leaf128_d<8, F>(t, kp, s);
        case 9: return launch_leaf128_d<9, F>(t, kp, s);
        case 10: return launch_leaf128_d<10, F>(t, kp, s);
        case 11: return launch_leaf128_d<11, F>(t, kp, s);
        case 12: return launch_leaf128_d<12, F>(t, kp, s);
        case 13: return launch_leaf128_d<13, F>(t, kp, s);
        case 14: return launch_leaf128_d<14, F>(t, kp, s);
        case 15: return launch_leaf128_d<15, F>(t, kp, s);
        default: return launch_leaf128_d<16, F>(t, kp, s);
    }
}

cudaError_t launch_leaf_finish(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    if (use_leaf128(t)) {
        switch (kp.family) {
            case kFamLaplace: return launch_leaf128_family<kFamLaplace>(t, kp, s);
            case kFamExp: return launch_leaf128_family<kFamExp>(t, kp, s);
            default: return launch_leaf128_family<kFamGauss>(t, kp, s);
        }
    }
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
        default: return launch_leaf_d<1, true>(t, kp, qt, s);  // d > 16: values from leaf_values_generic
    }
}

}  // namespace fsg
