// Re-decision of flagged descents in high precision (fsg_params.resolve).
//
// A descent decision of Algorithm 1 compares the draw u with the ratio
// g_left / (g_left + g_right).  The fused schedule takes it on FP32 sums and
// flags it when |u - ratio| falls inside the sums' error bound, so a flagged
// sample may differ from the exact method's.  This pass decides every flagged
// decision again on high-precision sums of both halves (double-single squared
// distances, values within relative error 2^-20, FP64 accumulation), compared
// in FP64 with the full 32-bit draw, u = word 2^-32.  A decision whose
// high-precision margin |u S - g_left| is still within the high-precision
// bound stays flagged; every other one equals the exact method's.
//
// Levels above the bins (their flagged levels recorded by descend_top):
//   1. compact   : the flagged samples;
//   2. jobs      : one job per flagged level of a sample, at the node its FP32
//                  path visited there (heap index from the bin it reached),
//                  counted per node;
//   3. scan      : job and CTA offsets per node;
//   4. scatter   : jobs grouped by node;
//   5. node sums : work item = one node, up to 32 of its jobs and a chunk of
//                  4,096 of its points: the chunk streams through shared
//                  memory once for all 32 queries (lane = job, warps over the
//                  points, the warps' FP64 partial sums added in warp order)
//                  instead of once per job, and large nodes spread over many
//                  CTAs; one partial sum per (job, chunk);
//   6. decide    : per sample, its flagged levels in order, each on the sum
//                  of its partials in chunk order; where the
//                  high-precision decision differs from the FP32 path, or a
//                  level inside the bin was flagged, the sample goes to the
//                  walker;
//   7. walker    : CTA per remaining sample: from the root where a decision
//                  changed (the FP32 node sums rebuilt from the query's bin
//                  sums in descend_top's order, bit-identical, high precision
//                  where they are flagged), else from its bin; then every level
//                  inside the bin on high-precision values of the bin's
//                  points, summed pairwise in FP64 over the halving tree.
// The sample's neighbour, its kernel value and its flags are overwritten in
// place, before the edge list is formed.  More flagged samples or jobs than
// the batched path's scratch holds, or padded d > 64, go to the walker from
// the root.
#include "fsg_internal.cuh"

FSG_BOUNDS_TU(resolve)

namespace fsg {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsJobs = 32;     // jobs (queries) of one node-sum CTA
constexpr int kRsTile = 256;    // points per shared-memory tile of a node-sum CTA
constexpr int kRsMaxDp = 64;    // batched node sums for padded d <= 64 (walker beyond)
constexpr int kRsChunk = 4096;  // points of a node per work item of the batched node sums
constexpr int kModeBin = 1, kModeFull = 2;

__device__ __forceinline__ int bin_of_pos(const int32_t* __restrict__ bnd, int nb, int pos) {
    int lo = 0, hi = nb;  // bnd[lo] <= pos < bnd[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bnd[mid] <= pos) lo = mid; else hi = mid;
    }
    return lo;
}

// Position range [a, c) of heap node h of the halving tree over [0, n).
__device__ __forceinline__ void node_range(int h, int n, int& a, int& c) {
    const int lev = 31 - __clz(h);
    a = 0;
    c = n;
    for (int t = lev - 1; t >= 0; --t) {
        const int mid = a + (c - a) / 2;
        if ((h >> t) & 1) a = mid; else c = mid;
    }
}

// Samples e in [e_lo, e_hi) (positions q_lo..q_hi - 1 times L) that are flagged.
__global__ void rs_compact_kernel(const uint8_t* __restrict__ flags, const uint8_t* __restrict__ lflags,
                                  const int32_t* __restrict__ leaf_pos, int64_t e_lo, int64_t e_hi, int64_t total,
                                  int32_t* __restrict__ list, int32_t* __restrict__ cnt) {
    for (int64_t e = e_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e_hi;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pos = leaf_pos[e];
        if (pos >= 0 && ((flags[e] | lflags[e]) & 1)) {
            const int slot = atomicAdd(&cnt[0], 1);
            if (FSG_INB(slot, total, kSiteResolveList)) list[slot] = (int32_t)e;
        }
    }
}

// cnt[0] flagged samples, cnt[1] jobs, cnt[2] walker entries, cnt[3] = 1
// when the batched path does not apply (every sample then goes to the walker
// from the root).
__global__ void rs_jobs_kernel(const int32_t* __restrict__ list, const int32_t* __restrict__ leaf_pos,
                               const uint16_t* __restrict__ flev, const int32_t* __restrict__ bnd, int nb, int s0,
                               int fcap, int dp, int32_t* __restrict__ sbin, int32_t* __restrict__ node_cnt,
                               int32_t* __restrict__ cnt) {
    const int F = cnt[0];
    if (F > fcap || dp > kRsMaxDp) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt[3] = 1;
        return;
    }
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < F; s += gridDim.x * blockDim.x) {
        const int e = list[s];
        const int b = bin_of_pos(bnd, nb, leaf_pos[e]);
        sbin[s] = b;
        for (uint32_t mm = flev[e]; mm; mm &= mm - 1u) {
            const int t = __ffs(mm) - 1;
            atomicAdd(&node_cnt[(1 << t) | (b >> (s0 - t))], 1);
        }
    }
}

// Point chunks of node h (kRsChunk positions each).
__device__ __forceinline__ int node_chunks(int h, int n) {
    int a, c;
    node_range(h, n, a, c);
    return (c - a + kRsChunk - 1) / kRsChunk;
}

// Exclusive scans (one CTA) per node of its jobs, of its work items (32 jobs
// x one chunk of points) and of its partial sums (jobs x chunks).
__global__ void __launch_bounds__(1024) rs_scan_kernel(const int32_t* __restrict__ node_cnt, int nb, int n,
                                                       int32_t* __restrict__ node_off, int32_t* __restrict__ cta_off,
                                                       int32_t* __restrict__ part_off, int jcap, int pcap,
                                                       int32_t* __restrict__ cnt) {
    __shared__ int32_t sj[1024], sc[1024], sp[1024];
    const int tid = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    int cj = 0, cc = 0, cp = 0;
    for (int u = 0; u < per; ++u) {
        const int h = tid * per + u;
        if (h >= 1 && h < nb && node_cnt[h] > 0) {
            const int pc = node_chunks(h, n);
            cj += node_cnt[h];
            cc += (node_cnt[h] + kRsJobs - 1) / kRsJobs * pc;
            cp += node_cnt[h] * pc;
        }
    }
    sj[tid] = cj;
    sc[tid] = cc;
    sp[tid] = cp;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int a = tid >= off ? sj[tid - off] : 0, b = tid >= off ? sc[tid - off] : 0;
        const int c = tid >= off ? sp[tid - off] : 0;
        __syncthreads();
        sj[tid] += a;
        sc[tid] += b;
        sp[tid] += c;
        __syncthreads();
    }
    int rj = sj[tid] - cj, rc = sc[tid] - cc, rp = sp[tid] - cp;
    for (int u = 0; u < per; ++u) {
        const int h = tid * per + u;
        if (h < nb) {
            node_off[h] = rj;
            cta_off[h] = rc;
            part_off[h] = rp;
            if (h >= 1 && node_cnt[h] > 0) {
                const int pc = node_chunks(h, n);
                rj += node_cnt[h];
                rc += (node_cnt[h] + kRsJobs - 1) / kRsJobs * pc;
                rp += node_cnt[h] * pc;
            }
        }
    }
    if (tid == 1023) {
        node_off[nb] = sj[1023];
        cta_off[nb] = sc[1023];
        part_off[nb] = sp[1023];
        cnt[1] = sj[1023];
        if (sj[1023] > jcap || sp[1023] > pcap) cnt[3] = 1;
    }
}

__global__ void rs_scatter_kernel(const int32_t* __restrict__ list, const uint16_t* __restrict__ flev,
                                  const int32_t* __restrict__ sbin, int s0, const int32_t* __restrict__ node_off,
                                  int32_t* __restrict__ node_cur, int32_t* __restrict__ job_s,
                                  int32_t* __restrict__ job_t, int32_t* __restrict__ slot_of,
                                  const int32_t* __restrict__ cnt) {
    if (cnt[3]) return;
    const int F = cnt[0];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < F; s += gridDim.x * blockDim.x) {
        const int b = sbin[s];
        for (uint32_t mm = flev[list[s]]; mm; mm &= mm - 1u) {
            const int t = __ffs(mm) - 1;
            const int h = (1 << t) | (b >> (s0 - t));
            const int slot = node_off[h] + atomicAdd(&node_cur[h], 1);
            job_s[slot] = s;
            job_t[slot] = t;
            slot_of[s * kRsMaxLevels + t] = slot;
        }
    }
}

// FP32 test of one point against the lane's query: false where the
// high-precision value would be flushed to zero (as hp_gauss_far0).  DP:
// padded dimension (0: runtime dp, query in shared memory).
template <int DP>
__device__ __forceinline__ bool rs_near(const float (&xr)[DP > 0 ? DP : 1], const float* __restrict__ xs,
                                        const float* __restrict__ y, int dp, float ch) {
    float s = 0.f;
    if (DP > 0) {
#pragma unroll
        for (int t = 0; t < DP; t += 4) {
            const float4 c = *reinterpret_cast<const float4*>(y + t);
            float dd = xr[t] - c.x; s = fmaf(dd, dd, s);
            dd = xr[t + 1] - c.y; s = fmaf(dd, dd, s);
            dd = xr[t + 2] - c.z; s = fmaf(dd, dd, s);
            dd = xr[t + 3] - c.w; s = fmaf(dd, dd, s);
        }
    } else {
        for (int t = 0; t < dp; ++t) {
            const float dd = xs[t] - y[t];
            s = fmaf(dd, dd, s);
        }
    }
    return !(s * ch > 127.f);
}

// The high-precision value of one point against the lane's query.
template <int DP>
__device__ __forceinline__ float rs_value(const float (&xr)[DP > 0 ? DP : 1], const float* __restrict__ xs,
                                          const float* __restrict__ y, int dp, float ch, float cl) {
    float sh = 0.f, sl = 0.f;
    if (DP > 0) {
#pragma unroll
        for (int t = 0; t < DP; ++t) hp_acc_sq(xr[t], y[t], sh, sl);
    } else {
        for (int t = 0; t < dp; ++t) hp_acc_sq(xs[t], y[t], sh, sl);
    }
    return hp_finish(sh, sl, ch, cl);
}

// High-precision sums of both children of a node, over one chunk of its
// points, for up to 32 of its jobs (lane = job, the CTA's warps over the
// chunk's points; the warps' FP64 partial sums are added in warp order).
template <int DP>
__global__ void __launch_bounds__(kRsThreads)
rs_node_sums_kernel(const float* __restrict__ Xt, int dp, int n, int L, int nb, const int32_t* __restrict__ list,
                    const int32_t* __restrict__ node_off, const int32_t* __restrict__ cta_off,
                    const int32_t* __restrict__ part_off, const int32_t* __restrict__ job_s, int self_exclude,
                    float ch, float cl, double* __restrict__ part, const int32_t* __restrict__ cnt) {
    extern __shared__ __align__(16) unsigned char smem_ns[];
    double* red = reinterpret_cast<double*>(smem_ns);                 // [warps][kRsJobs][2]
    float* pts = reinterpret_cast<float*>(red + kRsThreads / 32 * kRsJobs * 2);  // [tile][dp]
    float* qs = pts + kRsTile * dp;                                     // [job][dp + 1]
    int* qpos = reinterpret_cast<int*>(qs + kRsJobs * (dp + 1));        // [kRsJobs]
    if (cnt[3]) return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int total = cta_off[nb];
    const int qstride = dp + 1;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int lo = 0, hi = nb;  // node h: cta_off[h] <= item < cta_off[h + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cta_off[mid] <= item) lo = mid; else hi = mid;
        }
        const int h = lo;
        int a, c;
        node_range(h, n, a, c);
        const int mid = a + (c - a) / 2;
        const int pc = (c - a + kRsChunk - 1) / kRsChunk;
        const int local = item - cta_off[h];
        const int jc = local / pc, pk = local - jc * pc;
        const int j0 = node_off[h] + jc * kRsJobs;
        const int nj = min(kRsJobs, node_off[h + 1] - j0);
        const int pa = a + pk * kRsChunk, pe = min(c, pa + kRsChunk);
        __syncthreads();  // the previous item's shared data are no longer read
        if (tid < kRsJobs) qpos[tid] = tid < nj ? list[job_s[j0 + tid]] / L : -1;
        __syncthreads();
        for (int e = tid; e < kRsJobs * dp; e += kRsThreads) {
            const int jj = e / dp, t = e - jj * dp;
            qs[jj * qstride + t] = qpos[jj] >= 0 ? Xt[(size_t)qpos[jj] * dp + t] : 0.f;
        }
        __syncthreads();
        const int my_q = qpos[lane];
        const float* xs = qs + lane * qstride;
        float xr[DP > 0 ? DP : 1];
#pragma unroll
        for (int t = 0; t < (DP > 0 ? DP : 1); ++t) xr[t] = DP > 0 ? xs[t] : 0.f;
        double gl = 0.0, gr = 0.0;
        for (int p0 = pa; p0 < pe; p0 += kRsTile) {
            const int np = min(kRsTile, pe - p0);
            __syncthreads();  // the previous tile is no longer read
            const float4* src = reinterpret_cast<const float4*>(Xt + (size_t)p0 * dp);
            float4* dst = reinterpret_cast<float4*>(pts);
            for (int e = tid; e < np * dp / 4; e += kRsThreads) dst[e] = src[e];
            __syncthreads();
            if (my_q >= 0) {
                // warp w takes tile points w + 8 i (i < 32): the FP32 test of
                // all of them first, then the high-precision values of the
                // lane's near ones (per lane, in point order), so a lane does
                // the long evaluation only where its own query needs it
                uint32_t near = 0;
#pragma unroll 4
                for (int i = 0; i < 32; ++i) {
                    const int k = w + (kRsThreads / 32) * i;
                    if (k < np && rs_near<DP>(xr, xs, pts + k * dp, dp, ch)) near |= 1u << i;
                }
                for (uint32_t mm = near; mm; mm &= mm - 1u) {
                    const int k = w + (kRsThreads / 32) * (__ffs(mm) - 1);
                    const int p = p0 + k;
                    const float v = rs_value<DP>(xr, xs, pts + k * dp, dp, ch, cl);
                    if (!(self_exclude && p == my_q)) {
                        if (p < mid) gl += (double)v; else gr += (double)v;
                    }
                }
            }
        }
        red[(w * kRsJobs + lane) * 2] = gl;
        red[(w * kRsJobs + lane) * 2 + 1] = gr;
        __syncthreads();
        if (tid < nj) {
            double sl = 0.0, sr = 0.0;
#pragma unroll
            for (int k = 0; k < kRsThreads / 32; ++k) {
                sl += red[(k * kRsJobs + tid) * 2];
                sr += red[(k * kRsJobs + tid) * 2 + 1];
            }
            const int j = j0 + tid - node_off[h];  // the job's index within its node
            const size_t pi = (size_t)part_off[h] + (size_t)j * pc + pk;
            if (FSG_INB(pi, part_off[nb], kSiteResolvePart)) {
                part[pi * 2] = sl;
                part[pi * 2 + 1] = sr;
            }
        }
    }
}

// FP64 decision on high-precision sums: 1 = right.  hp_flag: the margin is
// within the sums' error bound (relative kHpEta each, plus the FP64 rounding
// of the accumulation and of u S - g_left, plus the values below 2^-126 that
// were flushed to zero: at most `tiny` in all).
__device__ __forceinline__ int hp_decide(double gl, double gr, uint32_t word, double tiny, uint8_t& f) {
    const double S = gl + gr;
    if (!(S > 0.0)) { f |= 2; return 1; }
    const double u = (double)word * 0x1p-32;
    const double dlt = u * S - gl;
    if (fabs(dlt) <= (kHpEta + 0x1p-40) * S + tiny) f |= 1;
    return dlt < 0.0 ? 0 : 1;
}

// Per flagged sample: its flagged levels above the bins, in order, on the
// high-precision sums.  Confirmed path and no flagged level inside the bin:
// done here; otherwise the sample goes to the walker (from its bin, or from
// the root where a decision changed).
__global__ void rs_decide_kernel(const int32_t* __restrict__ list, const int32_t* __restrict__ sbin,
                                 const uint16_t* __restrict__ flev, const int32_t* __restrict__ slot_of,
                                 const int32_t* __restrict__ node_off, const int32_t* __restrict__ part_off,
                                 const double* __restrict__ part, const int32_t* __restrict__ perm, int n, int s0,
                                 int L, uint64_t seed,
                                 uint8_t* __restrict__ flags, const uint8_t* __restrict__ lflags,
                                 int32_t* __restrict__ wlist, int32_t* __restrict__ cnt) {
    const int F = cnt[0];
    const bool batched = cnt[3] == 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < F; s += gridDim.x * blockDim.x) {
        if (!batched) {
            wlist[atomicAdd(&cnt[2], 1)] = s | (kModeFull << 30);
            continue;
        }
        const int e = list[s];
        const int q = e / L, l = e - q * L;
        const int b = sbin[s];
        const uint32_t i = (uint32_t)perm[q];
        uint8_t f = flags[e] & 2;  // a zero-mass node on the path stays recorded
        bool changed = false;
        uint4 blk = make_uint4(0, 0, 0, 0);
        int blk_id = -1;
        for (uint32_t mm = flev[e]; mm; mm &= mm - 1u) {
            const int t = __ffs(mm) - 1;
            if ((t >> 2) != blk_id) {
                blk_id = t >> 2;
                blk = draw_block(seed, i, (uint32_t)l, (uint32_t)t);
            }
            const int h = (1 << t) | (b >> (s0 - t));
            int a, c;
            node_range(h, n, a, c);
            // the job's partial sums over the node's point chunks, in chunk order
            const int pc = (c - a + kRsChunk - 1) / kRsChunk;
            const int j = slot_of[s * kRsMaxLevels + t] - node_off[h];
            const double* r = part + ((size_t)part_off[h] + (size_t)j * pc) * 2;
            double gl = 0.0, gr = 0.0;
            for (int k = 0; k < pc; ++k) {
                gl += r[2 * k];
                gr += r[2 * k + 1];
            }
            const int right = hp_decide(gl, gr, block_word(blk, (uint32_t)t), (double)(c - a) * 0x1p-126, f);
            if (right != (int)((b >> (s0 - t - 1)) & 1)) {
                changed = true;
                break;
            }
        }
        if (changed) {
            wlist[atomicAdd(&cnt[2], 1)] = s | (kModeFull << 30);
        } else {
            flags[e] = f;  // the levels above the bin, decided; the walker continues from the bin
            if (lflags[e] & 1) wlist[atomicAdd(&cnt[2], 1)] = s | (kModeBin << 30);
        }
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
__device__ __forceinline__ double hp_range(const float* __restrict__ Xt, int dp, const float* __restrict__ xq,
                                           int a, int c, int qpos, int self_exclude, float ch, float cl,
                                           double* red) {
    double s = 0.0;
#pragma unroll 2
    for (int p = a + (int)threadIdx.x; p < c; p += kRsThreads) {
        const float v = hp_gauss_far0(xq, Xt + (size_t)p * dp, dp, ch, cl);
        if (!(self_exclude && p == qpos)) s += (double)v;
    }
    return block_sum(s, red);
}

// The walker: CTA per sample of wlist (mode in the top two bits).
__global__ void __launch_bounds__(kRsThreads)
rs_walk_kernel(const float* __restrict__ Xt, int dp, const int32_t* __restrict__ perm,
               const int32_t* __restrict__ bnd, int nb, int s0, const float* __restrict__ binsum,
               const int32_t* __restrict__ list, const int32_t* __restrict__ sbin, const int32_t* __restrict__ wlist,
               const int32_t* __restrict__ cnt, KernelParams kp, int32_t* __restrict__ leaf_pos,
               float* __restrict__ ksmp, uint8_t* __restrict__ flags, uint8_t* __restrict__ lflags, int leafmax,
               long long nl) {
    extern __shared__ __align__(16) unsigned char smem_r[];
    float* tree = reinterpret_cast<float*>(smem_r);                       // [2 nb]
    double* V = reinterpret_cast<double*>(tree + 2 * nb + 2);             // [2 leafmax] halving-tree sums
    int32_t* spos = reinterpret_cast<int32_t*>(V + 2 * leafmax);          // [leafmax] slot -> position
    float* xq = reinterpret_cast<float*>(spos + leafmax);                 // [dp] query coordinates
    __shared__ double red[kRsThreads / 32];
    const int tid = threadIdx.x;
    const int L = kp.L;
    const int nw = cnt[2];
    for (int it = blockIdx.x; it < nw; it += gridDim.x) {
        const int wv = wlist[it];
        const int s = wv & 0x3fffffff, mode = (int)((uint32_t)wv >> 30);
        const int e = list[s];
        const int q = e / L, l = e - q * L;
        const uint32_t i = (uint32_t)perm[q];
        __syncthreads();  // the previous sample's shared data are no longer read
        for (int t = tid; t < dp; t += kRsThreads) xq[t] = Xt[(size_t)q * dp + t];
        uint8_t f = 0;
        int h = 1, a = 0, c = bnd[nb];
        uint4 blk = make_uint4(0, 0, 0, 0);
        int blk_id = -1;
        if (mode == kModeBin) {  // the path above the bin is decided
            const int b = sbin[s];
            a = bnd[b];
            c = bnd[b + 1];
            f = flags[e];
        } else {
            for (int b = tid; b < nb; b += kRsThreads) tree[nb + b] = binsum[(size_t)q * nb + b];
            __syncthreads();
            // node sums of levels s0-1 .. 0, pairwise, as descend_top formed them
            for (int lev = s0 - 1; lev >= 0; --lev) {
                for (int x = (1 << lev) + tid; x < (2 << lev); x += kRsThreads) tree[x] = tree[2 * x] + tree[2 * x + 1];
                __syncthreads();
            }
            const float root = tree[1];
            const float abs_tol = kp.kde_eps > 0.f ? kp.kde_eps * root / (1.f - kp.kde_eps) : 0.f;
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
                    const double gl = hp_range(Xt, dp, xq, a, mid, q, kp.self_exclude, kp.hp_ch, kp.hp_cl, red);
                    const double gr = hp_range(Xt, dp, xq, mid, c, q, kp.self_exclude, kp.hp_ch, kp.hp_cl, red);
                    right = hp_decide(gl, gr, word, (double)(c - a) * 0x1p-126, f);
                } else {
                    f |= f32;
                }
                if (right) a = mid; else c = mid;
                h = 2 * h + right;
            }
        }
        __syncthreads();  // xq complete
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
                v = (double)hp_gauss_far0(xq, Xt + (size_t)pos * dp, dp, kp.hp_ch, kp.hp_cl);
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
                    right = hp_decide(V[2 * hh], V[2 * hh + 1], block_word(blk, lev), (double)(hi - lo) * 0x1p-126,
                                      f);
                    const int md = lo + (hi - lo) / 2;
                    if (right) lo = md; else hi = md;
                }
                hh = 2 * hh + right;
            }
            if (FSG_INB(e, nl, kSiteResolveWalk)) {
                leaf_pos[e] = spos[hh - leaf0];
                ksmp[e] = (float)V[hh];
                flags[e] = f;
                lflags[e] = 0;
            }
        }
    }
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

size_t walk_smem(const fsg_tree* t) {
    const int leafmax = 1 << t->dm;
    return (size_t)(2 * t->nb + 2) * 4 + (size_t)2 * leafmax * 8 + (size_t)leafmax * 4 + (size_t)t->dp * 4 + 16;
}

}  // namespace

bool resolve_supported(const fsg_tree* t) { return t->d <= 4096 && t->nb <= 4096 && (1 << t->dm) <= 1024; }

// Lays out (and allocates on first use, or when n L grows) the re-decision's
// scratch: room for n L flagged samples in the walker's list, and for
// max(65,536, n L / 64) of them (twice as many jobs) in the batched path.
int ensure_resolve(fsg_tree* t, int L, cudaStream_t s) {
    ResolveWs& rs = t->rs;
    const int64_t nl = t->n * (int64_t)L;
    if (rs.base && rs.cap_nl >= nl) return FSG_OK;
    const int64_t fcap64 = nl / 64 > 65536 ? nl / 64 : (nl < 65536 ? nl : 65536);
    const int32_t fcap = (int32_t)fcap64, jcap = (int32_t)(2 * fcap64);
    // partial sums: a job at a node of size m holds ceil(m / kRsChunk) of them
    const int64_t pcap64 = 4 * (int64_t)jcap + 64 * ((t->n + kRsChunk - 1) / kRsChunk);
    const int32_t pcap = (int32_t)(pcap64 < 0x7fffffff ? pcap64 : 0x7fffffff);
    const size_t o_flev = 0;
    const size_t o_list = up256(o_flev + sizeof(uint16_t) * (size_t)nl);
    const size_t o_sbin = up256(o_list + sizeof(int32_t) * (size_t)nl);
    const size_t o_ncnt = up256(o_sbin + sizeof(int32_t) * (size_t)fcap);
    const size_t o_ncur = up256(o_ncnt + sizeof(int32_t) * (size_t)t->nb);
    const size_t o_noff = up256(o_ncur + sizeof(int32_t) * (size_t)t->nb);
    const size_t o_coff = up256(o_noff + sizeof(int32_t) * (size_t)(t->nb + 1));
    const size_t o_poff = up256(o_coff + sizeof(int32_t) * (size_t)(t->nb + 1));
    const size_t o_js = up256(o_poff + sizeof(int32_t) * (size_t)(t->nb + 1));
    const size_t o_jt = up256(o_js + sizeof(int32_t) * (size_t)jcap);
    const size_t o_slot = up256(o_jt + sizeof(int32_t) * (size_t)jcap);
    const size_t o_part = up256(o_slot + sizeof(int32_t) * kRsMaxLevels * (size_t)fcap);
    const size_t o_wl = up256(o_part + sizeof(double) * 2 * (size_t)pcap);
    const size_t o_cnt = up256(o_wl + sizeof(int32_t) * (size_t)nl);
    const size_t total = up256(o_cnt + sizeof(int32_t) * 8);
    if (rs.base) {
        if (t->pool) {
            cudaFreeAsync(rs.base, t->alloc_stream);
        } else {
            cudaStreamSynchronize(s);
            cudaFree(rs.base);
        }
        rs.base = nullptr;
        rs.cap_nl = 0;
    }
    const cudaError_t e = t->pool ? cudaMallocFromPoolAsync(&rs.base, total, t->pool, t->alloc_stream)
                                  : cudaMalloc(&rs.base, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rs.base = nullptr;
        return e == cudaErrorMemoryAllocation ? FSG_ERR_OOM : FSG_ERR_CUDA;
    }
    char* b = static_cast<char*>(rs.base);
    rs.bytes = total;
    rs.cap_nl = nl;
    rs.fcap = fcap;
    rs.jcap = jcap;
    rs.flev = reinterpret_cast<uint16_t*>(b + o_flev);
    rs.list = reinterpret_cast<int32_t*>(b + o_list);
    rs.sbin = reinterpret_cast<int32_t*>(b + o_sbin);
    rs.node_cnt = reinterpret_cast<int32_t*>(b + o_ncnt);
    rs.node_cur = reinterpret_cast<int32_t*>(b + o_ncur);
    rs.node_off = reinterpret_cast<int32_t*>(b + o_noff);
    rs.cta_off = reinterpret_cast<int32_t*>(b + o_coff);
    rs.part_off = reinterpret_cast<int32_t*>(b + o_poff);
    rs.job_s = reinterpret_cast<int32_t*>(b + o_js);
    rs.job_t = reinterpret_cast<int32_t*>(b + o_jt);
    rs.slot_of = reinterpret_cast<int32_t*>(b + o_slot);
    rs.part = reinterpret_cast<double*>(b + o_part);
    rs.pcap = pcap;
    rs.wlist = reinterpret_cast<int32_t*>(b + o_wl);
    rs.cnt = reinterpret_cast<int32_t*>(b + o_cnt);
    return FSG_OK;
}

cudaError_t launch_resolve(const fsg_tree* t, const KernelParams& kp, cudaStream_t s, int64_t q_lo,
                           int64_t q_hi) {
    const auto& ws = t->ws;
    const ResolveWs& rs = t->rs;
    const int64_t total = t->n * (int64_t)kp.L;
    if (q_hi < 0) q_hi = t->n;
    const int64_t e_lo = q_lo * kp.L, e_hi = q_hi * kp.L;
    cudaError_t e = cudaMemsetAsync(rs.cnt, 0, sizeof(int32_t) * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rs.node_cnt, 0, sizeof(int32_t) * (size_t)t->nb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rs.node_cur, 0, sizeof(int32_t) * (size_t)t->nb, s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (e_hi - e_lo + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    rs_compact_kernel<<<(int)blocks, 256, 0, s>>>(ws.flags, ws.lflags, ws.leaf_pos, e_lo, e_hi, total, rs.list,
                                                  rs.cnt);
    const int fb = (rs.fcap + 255) / 256 < 152 * 8 ? (rs.fcap + 255) / 256 : 152 * 8;
    rs_jobs_kernel<<<fb, 256, 0, s>>>(rs.list, ws.leaf_pos, rs.flev, t->bnd, t->nb, t->s0, rs.fcap, t->dp, rs.sbin,
                                      rs.node_cnt, rs.cnt);
    rs_scan_kernel<<<1, 1024, 0, s>>>(rs.node_cnt, t->nb, (int)t->n, rs.node_off, rs.cta_off, rs.part_off, rs.jcap,
                                      rs.pcap, rs.cnt);
    rs_scatter_kernel<<<fb, 256, 0, s>>>(rs.list, rs.flev, rs.sbin, t->s0, rs.node_off, rs.node_cur, rs.job_s,
                                         rs.job_t, rs.slot_of, rs.cnt);
    if (t->dp <= kRsMaxDp) {
        const size_t ns_smem = (size_t)kRsThreads / 32 * kRsJobs * 2 * 8 +
                               (size_t)(kRsTile * t->dp + kRsJobs * (t->dp + 1) + kRsJobs) * 4;
        auto ns = t->dp == 4 ? rs_node_sums_kernel<4> : t->dp == 8 ? rs_node_sums_kernel<8>
                : t->dp == 12 ? rs_node_sums_kernel<12> : t->dp == 16 ? rs_node_sums_kernel<16>
                : rs_node_sums_kernel<0>;
        e = set_smem_limit(ns, ns_smem);
        if (e != cudaSuccess) return e;
        ns<<<152 * 4, kRsThreads, ns_smem, s>>>(t->Xt, t->dp, (int)t->n, kp.L, t->nb, rs.list, rs.node_off,
                                                 rs.cta_off, rs.part_off, rs.job_s, kp.self_exclude, kp.hp_ch,
                                                 kp.hp_cl, rs.part, rs.cnt);
    }
    const int nlb = (int)((total + 255) / 256 < 152 * 8 ? (total + 255) / 256 : 152 * 8);
    rs_decide_kernel<<<nlb, 256, 0, s>>>(rs.list, rs.sbin, rs.flev, rs.slot_of, rs.node_off, rs.part_off, rs.part,
                                         t->perm, (int)t->n, t->s0, kp.L, kp.seed, ws.flags, ws.lflags, rs.wlist,
                                         rs.cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = walk_smem(t);
    e = set_smem_limit(rs_walk_kernel, smem);
    if (e != cudaSuccess) return e;
    rs_walk_kernel<<<152 * 4, kRsThreads, smem, s>>>(t->Xt, t->dp, t->perm, t->bnd, t->nb, t->s0, ws.binsum, rs.list,
                                                    rs.sbin, rs.wlist, rs.cnt, kp, ws.leaf_pos, ws.ksmp, ws.flags,
                                                    ws.lflags, 1 << t->dm, total);
    return cudaGetLastError();
}

}  // namespace fsg
