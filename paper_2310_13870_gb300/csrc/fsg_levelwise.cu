// The plain FP32 exact path (schedule FSG_SCHED_LEVELWISE): Algorithm 1 taken
// literally on the GPU, one launch per level of the halving tree.  At level
// lev every distinct node reached by a query's samples gets both halves'
// KDEs (Eq. 1) computed afresh with FP32 direct differences, one warp per
// query (lanes striding over the node's points for d <= 16, over each point's
// coordinates for larger d), butterfly sums; then each
// sample at that node takes its decision.  There is no bin pass and no reuse
// of sums across levels: this is the comparison point for the fused
// schedule, and gives the same samples up to flagged decisions.
// The carried-denominator variant (FSG_SCHED_CARRIED) sums only the left
// child at levels >= 1 and carries each sample's node sum down, taking g_R as
// g_node - g_L: half the evaluations per level, paid for in precision (the
// carried error bound widens the flag tolerance as the descent goes right).
#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr unsigned kFullLw = 0xffffffffu;

// Query coordinates held in registers for DP <= 16 (DP = padded dimension,
// padding coordinates are zero on both sides); DP == 0 reads them from memory.
template <int DP>
struct Query {
    float4 v[DP / 4];
    __device__ __forceinline__ const float* row() const { return nullptr; }
    __device__ __forceinline__ void load(const float* __restrict__ xq, int) {
#pragma unroll
        for (int c = 0; c < DP / 4; ++c) v[c] = reinterpret_cast<const float4*>(xq)[c];
    }
    __device__ __forceinline__ float dist2(const float* __restrict__ xp, int) const {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < DP / 4; ++c) {
            const float4 p = reinterpret_cast<const float4*>(xp)[c];
            float dd = v[c].x - p.x; s = fmaf(dd, dd, s);
            dd = v[c].y - p.y; s = fmaf(dd, dd, s);
            dd = v[c].z - p.z; s = fmaf(dd, dd, s);
            dd = v[c].w - p.w; s = fmaf(dd, dd, s);
        }
        return s;
    }
};
template <>
struct Query<0> {
    const float* x;
    __device__ __forceinline__ void load(const float* __restrict__ xq, int) { x = xq; }
    __device__ __forceinline__ const float* row() const { return x; }
    __device__ __forceinline__ float dist2(const float* __restrict__ xp, int dp) const {
        float s = 0.f;
        for (int c = 0; c < dp; c += 4) {
            const float4 a = *reinterpret_cast<const float4*>(x + c);
            const float4 p = *reinterpret_cast<const float4*>(xp + c);
            float dd = a.x - p.x; s = fmaf(dd, dd, s);
            dd = a.y - p.y; s = fmaf(dd, dd, s);
            dd = a.z - p.z; s = fmaf(dd, dd, s);
            dd = a.w - p.w; s = fmaf(dd, dd, s);
        }
        return s;
    }
};

// Sums of k(x_q, x_p) over [nlo, mid) and [mid, nhi), reduced over the warp.
// d <= 16: lanes stride over the node's points; larger d: the warp takes one
// point at a time with lanes striding over its coordinates (coalesced rows).
template <int DP>
__device__ __forceinline__ void node_sums(const Query<DP>& xq, const float* __restrict__ Xt, int dp, int q,
                                          int nlo, int mid, int nhi, const KernelParams& kp, int lane, float& gl,
                                          float& gr) {
    // (the carried-denominator schedule passes nhi = mid: the left half only)
    gl = 0.f;
    gr = 0.f;
    if constexpr (DP == 0) {
        const float* xqr = xq.row();
        for (int p = nlo; p < nhi; ++p) {
            const float* xp = Xt + (size_t)p * dp;
            float s = 0.f;
            for (int t = lane; t < dp; t += 32) {
                const float dd = xqr[t] - xp[t];
                s = fmaf(dd, dd, s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFullLw, s, o);
            float k = ex2_approx(s * kp.neg_c);
            if (kp.self_exclude && p == q) k = 0.f;
            if (p < mid) gl += k; else gr += k;
        }
    } else {
        for (int p = nlo + lane; p < nhi; p += 32) {
            float k = ex2_approx(xq.dist2(Xt + (size_t)p * dp, dp) * kp.neg_c);
            if (kp.self_exclude && p == q) k = 0.f;
            if (p < mid) gl += k; else gr += k;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gl += __shfl_xor_sync(kFullLw, gl, o);
            gr += __shfl_xor_sync(kFullLw, gr, o);
        }
    }
}

// Carried-denominator decision (the variant of Algorithm 1 that sums only the
// left child and takes g_R = g_node - g_L from the parent's sum): go right iff
// u g_node >= g_L.  eg bounds the absolute error of the carried g_node, eps the
// relative error of a fresh FP32 sum; the decision is flagged when
// |u g_node - g_L| < eg + 2 eps g_L + 2^-22 g_node, which covers both.  The
// chosen child's sum and its error bound replace (g, eg): g_L (fresh), or
// g - g_L, whose bound adds the parent's, g_L's and the subtraction's rounding.
__device__ __forceinline__ int carried_decide(float gl, float& g, float& eg, uint32_t word, float eps, uint8_t& f) {
    if (!(g > 0.f)) {
        f |= 2;
        return 1;
    }
    const float u = __uint2float_rz(word >> 8) * 0x1p-24f;
    const float dlt = fmaf(u, g, -gl);
    if (fabsf(dlt) < eg + 2.f * eps * gl + 0x1p-22f * g) f |= 1;
    if (dlt < 0.f) {
        g = gl;
        eg = eps * gl;
        return 0;
    }
    const float gr = g - gl;
    eg = eg + eps * gl + 0x1p-24f * fabsf(gr);
    g = gr;
    return 1;
}

// Level 0: the root [0, n) of every query, i.e. its degree, and (with
// samples) the first decision of each of its L samples.
template <int DP>
__global__ void __launch_bounds__(128)
levelwise_root_kernel(const float* __restrict__ Xt, int n, int dp, const int32_t* __restrict__ perm,
                      KernelParams kp, int with_samples, int32_t* __restrict__ lo_s, int32_t* __restrict__ hi_s,
                      uint8_t* __restrict__ flags, double* __restrict__ d_deg, float* __restrict__ degf,
                      unsigned long long* __restrict__ n_evals, float* __restrict__ g_s, float* __restrict__ eg_s) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (q >= n) return;
    Query<DP> xq;
    xq.load(Xt + (size_t)q * dp, dp);
    const int mid = n / 2;
    float gl, gr;
    node_sums<DP>(xq, Xt, dp, q, 0, mid, n, kp, lane, gl, gr);
    const uint32_t i = (uint32_t)perm[q];
    if (lane == 0) {
        degf[q] = gl + gr;
        if (d_deg) d_deg[i] = (double)(gl + gr);
        atomicAdd(n_evals, (unsigned long long)n);
    }
    if (!with_samples) return;
    for (int l = lane; l < kp.L; l += 32) {
        uint8_t f = 0;
        int lo = 0, hi = n;
        float g = gl + gr, eg = kp.flag_eps * g;  // carried state (the carried schedule)
        if (n >= 2) {
            const uint4 blk = draw_block(kp.seed, i, (uint32_t)l, 0u);
            const int right = g_s ? carried_decide(gl, g, eg, blk.x, kp.flag_eps, f)
                                  : descend_decide(gl, gr, blk.x, kp.flag_eps, f);
            if (right) lo = mid; else hi = mid;
        }
        lo_s[(size_t)q * kp.L + l] = lo;
        hi_s[(size_t)q * kp.L + l] = hi;
        flags[(size_t)q * kp.L + l] = f;
        if (g_s) {
            g_s[(size_t)q * kp.L + l] = g;
            eg_s[(size_t)q * kp.L + l] = eg;
        }
    }
}

// Level lev >= 1: samples are grouped by their current node (nodes of one
// level are identified by their first position); each distinct node is summed
// once, then every sample at it decides.  lo_s/hi_s: [n][L] node of each
// sample; flags: [n][L], accumulated over the levels.
template <int DP>
__global__ void __launch_bounds__(128)
levelwise_step_kernel(const float* __restrict__ Xt, int n, int dp, const int32_t* __restrict__ perm,
                      KernelParams kp, int lev, int32_t* __restrict__ lo_s, int32_t* __restrict__ hi_s,
                      uint8_t* __restrict__ flags, const float* __restrict__ degf,
                      unsigned long long* __restrict__ n_evals, float* __restrict__ g_s, float* __restrict__ eg_s) {
    __shared__ int32_t sk[4][kMaxL];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * 4 + w;
    if (q >= n || !(degf[q] > 0.f)) return;  // zero-degree queries draw no sample
    const int L = kp.L;
    const uint32_t i = (uint32_t)perm[q];
    int lo[2], hi[2];
    uint8_t f[2];
    bool act[2];
    float g[2] = {0.f, 0.f}, eg[2] = {0.f, 0.f};  // carried node sums (the carried schedule)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int l = lane + 32 * r;
        act[r] = false;
        lo[r] = hi[r] = 0;
        f[r] = 0;
        if (l < L) {
            lo[r] = lo_s[(size_t)q * L + l];
            hi[r] = hi_s[(size_t)q * L + l];
            f[r] = flags[(size_t)q * L + l];
            act[r] = hi[r] - lo[r] >= 2;
            if (g_s) {
                g[r] = g_s[(size_t)q * L + l];
                eg[r] = eg_s[(size_t)q * L + l];
            }
        }
        sk[w][l] = act[r] ? lo[r] : -1;
    }
    __syncwarp();
    uint64_t M[2] = {0ull, 0ull};
    for (int e = 0; e < kMaxL; ++e) {
        const int v = sk[w][e];
#pragma unroll
        for (int r = 0; r < 2; ++r) M[r] |= (uint64_t)(act[r] && v == lo[r]) << e;
    }
    uint32_t b0, b1;
    {
        const bool l0 = act[0] && (M[0] & ((1ull << lane) - 1ull)) == 0ull;
        const bool l1 = act[1] && (M[1] & ((1ull << (lane + 32)) - 1ull)) == 0ull;
        b0 = __ballot_sync(kFullLw, l0);
        b1 = __ballot_sync(kFullLw, l1);
    }
    if (!(b0 | b1)) return;
    Query<DP> xq;
    xq.load(Xt + (size_t)q * dp, dp);
    unsigned long long evals = 0;
    while (b0 | b1) {  // each distinct node in turn (warp-uniform)
        int src_r, src_lane;
        if (b0) { src_r = 0; src_lane = __ffs(b0) - 1; b0 &= b0 - 1; }
        else { src_r = 1; src_lane = __ffs(b1) - 1; b1 &= b1 - 1; }
        const int nlo = __shfl_sync(kFullLw, src_r ? lo[1] : lo[0], src_lane);
        const int nhi = __shfl_sync(kFullLw, src_r ? hi[1] : hi[0], src_lane);
        const int mid = nlo + (nhi - nlo) / 2;
        float gl, gr;
        node_sums<DP>(xq, Xt, dp, q, nlo, mid, g_s ? mid : nhi, kp, lane, gl, gr);
        evals += (unsigned long long)((g_s ? mid : nhi) - nlo);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (act[r] && lo[r] == nlo) {
                const uint32_t l = (uint32_t)(lane + 32 * r);
                const uint4 blk = draw_block(kp.seed, i, l, (uint32_t)lev);
                const uint32_t word = block_word(blk, (uint32_t)lev);
                const int right = g_s ? carried_decide(gl, g[r], eg[r], word, kp.flag_eps, f[r])
                                      : descend_decide(gl, gr, word, kp.flag_eps, f[r]);
                if (right) lo[r] = mid; else hi[r] = mid;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int l = lane + 32 * r;
        if (act[r]) {
            lo_s[(size_t)q * L + l] = lo[r];
            hi_s[(size_t)q * L + l] = hi[r];
            flags[(size_t)q * L + l] = f[r];
            if (g_s) {
                g_s[(size_t)q * L + l] = g[r];
                eg_s[(size_t)q * L + l] = eg[r];
            }
        }
    }
    if (lane == 0) atomicAdd(n_evals, evals);
}

// Leaves: sampled position and its kernel value (for the weights of
// Algorithm 2); zero-degree queries get no sample.
__global__ void levelwise_finish_kernel(const float* __restrict__ Xt, int n, int d, int dp, KernelParams kp,
                                        const int32_t* __restrict__ lo_s, const float* __restrict__ degf,
                                        uint8_t* __restrict__ flags, int32_t* __restrict__ leaf_pos,
                                        float* __restrict__ ksmp, uint8_t* __restrict__ lflags) {
    const int L = kp.L;
    const int64_t total = (int64_t)n * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / L);
        lflags[e] = 0;
        if (!(degf[q] > 0.f)) {
            leaf_pos[e] = -1;
            ksmp[e] = 0.f;
            flags[e] = (n > 1 || !kp.self_exclude) ? 2 : 0;
            continue;
        }
        const int p = lo_s[e];
        leaf_pos[e] = p;
        const float* a = Xt + (size_t)q * dp;
        const float* b = Xt + (size_t)p * dp;
        float s = 0.f;
        for (int t = 0; t < d; ++t) {
            const float dd = a[t] - b[t];
            s = fmaf(dd, dd, s);
        }
        ksmp[e] = (kp.self_exclude && p == q) ? 0.f : ex2_approx(s * kp.neg_c);
    }
}

template <int DP>
cudaError_t launch_levels(const fsg_tree* t, const KernelParams& kp, double* d_deg, int with_samples, int carried,
                          cudaStream_t s, int64_t* launches) {
    const auto& ws = t->ws;
    const int n = (int)t->n;
    // the per-sample node ranges live in the item arrays, unused by this
    // schedule; the carried sums and their error bounds in the leaf outputs,
    // which the finish kernel writes only after the last level
    int32_t* lo_s = ws.qitem_bin;
    int32_t* hi_s = reinterpret_cast<int32_t*>(ws.qitem_mask);
    float* g_s = carried ? ws.ksmp : nullptr;
    float* eg_s = carried ? reinterpret_cast<float*>(ws.leaf_pos) : nullptr;
    unsigned long long* ev = reinterpret_cast<unsigned long long*>(&ws.stats->n_evals);
    const int grid = (n + 3) / 4;
    levelwise_root_kernel<DP><<<grid, 128, 0, s>>>(t->Xt, n, t->dp, t->perm, kp, with_samples, lo_s, hi_s,
                                                   ws.flags, d_deg, ws.degf, ev, g_s, eg_s);
    cudaError_t e = cudaGetLastError();
    *launches += 1;
    if (!with_samples) return e;
    for (int lev = 1; lev < t->depth && e == cudaSuccess; ++lev) {
        levelwise_step_kernel<DP><<<grid, 128, 0, s>>>(t->Xt, n, t->dp, t->perm, kp, lev, lo_s, hi_s, ws.flags,
                                                       ws.degf, ev, g_s, eg_s);
        e = cudaGetLastError();
        *launches += 1;
    }
    if (e != cudaSuccess) return e;
    int64_t g = ((int64_t)n * kp.L + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    levelwise_finish_kernel<<<(int)g, 256, 0, s>>>(t->Xt, n, t->d, t->dp, kp, lo_s, ws.degf, ws.flags, ws.leaf_pos,
                                                    ws.ksmp, ws.lflags);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace

// The whole descent (or, without samples, the degrees alone) by the levelwise
// schedule.  Statistics: n_evals counts every kernel evaluation executed.
cudaError_t launch_levelwise(const fsg_tree* t, const KernelParams& kp, double* d_deg, int with_samples,
                             int carried, cudaStream_t s, int64_t* launches) {
    switch (t->dp) {
        case 4: return launch_levels<4>(t, kp, d_deg, with_samples, carried, s, launches);
        case 8: return launch_levels<8>(t, kp, d_deg, with_samples, carried, s, launches);
        case 12: return launch_levels<12>(t, kp, d_deg, with_samples, carried, s, launches);
        case 16: return launch_levels<16>(t, kp, d_deg, with_samples, carried, s, launches);
        default: return launch_levels<0>(t, kp, d_deg, with_samples, carried, s, launches);
    }
}

}  // namespace fsg
