// KDE tiles for any dimension d (used for d > 16): the squared distances of a
// tile of 128 queries x 64 points are accumulated over the coordinates in
// chunks of 32 (FP32 direct differences, (x_t - y_t)^2, so there is no
// cancellation whatever the norms), then exponentiated with ex2.  Thread
// (tq, tp) of 256 holds queries 8 tq .. 8 tq + 7 and points 4 tp .. 4 tp + 3.
//
//   kde_bins_generic_kernel   : bin sums (the bin pass of Eq. 1) for every
//                               query, per chunk of bins, like the d <= 16 pass;
//   leaf_values_generic_kernel: for the items (queries) of one bin, the kernel
//                               value at every leaf slot of the bin's tree,
//                               written to a global [item][slot] buffer that the
//                               leaf finish reads.
#include <climits>

#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr int kGT = 256;     // threads
constexpr int kGQ = 128;     // queries per tile
constexpr int kGP = 64;      // points per tile
constexpr int kGK = 32;      // coordinates per chunk

// Loads the coordinate chunk [k0, k0 + 32) of `rows` (positions, -1 = none)
// transposed into S[k][r] (r < nrows).  Rows are Xt rows of stride dp.
__device__ __forceinline__ void load_chunk(float* __restrict__ S, int nrows, const int* __restrict__ rows,
                                           const float* __restrict__ Xt, int dp, int k0) {
    for (int e = threadIdx.x; e < nrows * (kGK / 4); e += kGT) {
        const int r = e % nrows, v = e / nrows;
        const int k = k0 + 4 * v;
        const int pos = rows[r];
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pos >= 0 && k < dp) x = *reinterpret_cast<const float4*>(Xt + (size_t)pos * dp + k);
        S[(4 * v + 0) * nrows + r] = x.x;
        S[(4 * v + 1) * nrows + r] = x.y;
        S[(4 * v + 2) * nrows + r] = x.z;
        S[(4 * v + 3) * nrows + r] = x.w;
    }
}

// acc[i][j] += sum over the chunk of (q_i - p_j)^2.
__device__ __forceinline__ void accumulate_chunk(const float* __restrict__ Qs, const float* __restrict__ Ps, int tq,
                                                 int tp, float (&acc)[8][4]) {
#pragma unroll 4
    for (int k = 0; k < kGK; ++k) {
        const float4 qa = *reinterpret_cast<const float4*>(Qs + k * kGQ + 8 * tq);
        const float4 qb = *reinterpret_cast<const float4*>(Qs + k * kGQ + 8 * tq + 4);
        const float4 pv = *reinterpret_cast<const float4*>(Ps + k * kGP + 4 * tp);
        const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        const float pp[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float dd = qv[i] - pp[j];
                acc[i][j] = fmaf(dd, dd, acc[i][j]);
            }
        }
    }
}

__global__ void __launch_bounds__(kGT, 2)
kde_bins_generic_kernel(const float* __restrict__ Xt, int n, int d, int dp, const int32_t* __restrict__ bnd, int nb,
                        int bpc, float neg_c, int self_exclude, float* __restrict__ binsum) {
    __shared__ __align__(16) float Qs[kGK * kGQ];
    __shared__ __align__(16) float Ps[kGK * kGP];
    __shared__ float part[16][kGQ][2];
    __shared__ int qrow[kGQ], prow[kGP];
    __shared__ int bnd_s[9];
    extern __shared__ float outs[];  // [kGQ][bpc]
    const int tid = threadIdx.x, tq = tid & 15, tp = tid >> 4;
    const int qbase = blockIdx.x * kGQ;
    const int b0 = blockIdx.y * bpc;
    const int nbc = min(nb, b0 + bpc) - b0;
    if (tid <= nbc) bnd_s[tid] = bnd[b0 + tid];
    if (tid < kGQ) qrow[tid] = qbase + tid < n ? qbase + tid : -1;
    for (int e = tid; e < kGQ * bpc; e += kGT) outs[e] = 0.f;
    __syncthreads();
    const int pa = bnd_s[0], pe = bnd_s[nbc];
    for (int t0 = pa; t0 < pe; t0 += kGP) {
        const int np = min(kGP, pe - t0);
        if (tid < kGP) prow[tid] = tid < np ? t0 + tid : -1;
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < dp; k0 += kGK) {
            __syncthreads();
            load_chunk(Qs, kGQ, qrow, Xt, dp, k0);
            load_chunk(Ps, kGP, prow, Xt, dp, k0);
            __syncthreads();
            accumulate_chunk(Qs, Ps, tq, tp, acc);
        }
        // Bin of the tile's first point; the tile spans at most two bins.
        int bt = 0;
        while (bt + 1 < nbc && bnd_s[bt + 1] <= t0) ++bt;
        const int split = bt + 1 < nbc ? bnd_s[bt + 1] : INT_MAX;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = qbase + 8 * tq + i;
            float s0v = 0.f, s1v = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = t0 + 4 * tp + j;
                if (4 * tp + j < np) {
                    float k = ex2_approx(acc[i][j] * neg_c);
                    if (self_exclude && p == q) k = 0.f;
                    if (p < split) s0v += k; else s1v += k;
                }
            }
            part[tp][8 * tq + i][0] = s0v;
            part[tp][8 * tq + i][1] = s1v;
        }
        __syncthreads();
        {
            const int q = tid & (kGQ - 1), sl = tid >> 7;
            float s = 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) s += part[u][q][sl];
            const int bb = bt + sl;
            if (bb < nbc) outs[q * bpc + bb] += s;
        }
    }
    __syncthreads();
    const int nq = min(kGQ, n - qbase);
    for (int e = tid; e < nq * nbc; e += kGT) {
        const int ql = e / nbc, b = e - ql * nbc;
        binsum[(size_t)(qbase + ql) * nb + b0 + b] = outs[ql * bpc + b];
    }
}

// Leaf values: CTA (b, y) handles item chunks y, y + gridDim.y, ... of bin
// b's segment; slots of the bin's perfect tree whose node is empty get 0.
__global__ void __launch_bounds__(kGT, 2)
leaf_values_generic_kernel(const float* __restrict__ Xt, int dp, const int32_t* __restrict__ bnd,
                           const int32_t* __restrict__ bin_off, const int32_t* __restrict__ items_q, float neg_c,
                           int self_exclude, int leafmax, float* __restrict__ Vg) {
    __shared__ __align__(16) float Qs[kGK * kGQ];
    __shared__ __align__(16) float Ps[kGK * kGP];
    __shared__ int qrow[kGQ], prow[kGP];
    const int tid = threadIdx.x, tq = tid & 15, tp = tid >> 4;
    const int b = blockIdx.x;
    const int seg = bin_off[b * kBinSlots];
    const int cnt = bin_off[(b + 1) * kBinSlots] - seg;
    const int nchunks = (cnt + kGQ - 1) / kGQ;
    if ((int)blockIdx.y >= nchunks) return;
    const int p_lo = bnd[b], m = bnd[b + 1] - p_lo;
    const int dm = ceil_log2_dev(m), leaf0 = 1 << dm;
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int it0 = chunk * kGQ;
        const int qcnt = min(kGQ, cnt - it0);
        for (int s0 = 0; s0 < leaf0; s0 += kGP) {
            __syncthreads();
            if (tid < kGQ) qrow[tid] = tid < qcnt ? items_q[seg + it0 + tid] : -1;
            if (tid < kGP) {
                const int sl = s0 + tid;
                int pos = -1;
                if (sl < leaf0) {
                    int a = 0, c = m;
                    for (int t = dm - 1; t >= 0; --t) {
                        const int mid = a + (c - a) / 2;
                        if ((sl >> t) & 1) a = mid; else c = mid;
                    }
                    if (c - a == 1) pos = p_lo + a;
                }
                prow[tid] = pos;
            }
            float acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
            for (int k0 = 0; k0 < dp; k0 += kGK) {
                __syncthreads();
                load_chunk(Qs, kGQ, qrow, Xt, dp, k0);
                load_chunk(Ps, kGP, prow, Xt, dp, k0);
                __syncthreads();
                accumulate_chunk(Qs, Ps, tq, tp, acc);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int qq = 8 * tq + i;
                if (qq >= qcnt) continue;
                const int qp = qrow[qq];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int sl = s0 + 4 * tp + j;
                    if (sl < leaf0) {
                        const int pp = prow[4 * tp + j];
                        float k = pp >= 0 ? ex2_approx(acc[i][j] * neg_c) : 0.f;
                        if (self_exclude && pp == qp) k = 0.f;
                        Vg[(size_t)(seg + it0 + qq) * leafmax + sl] = k;
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_kde_bins_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const int qblocks = (int)((t->n + kGQ - 1) / kGQ);
    int chunks = (2048 + qblocks - 1) / qblocks;
    if (chunks < 1) chunks = 1;
    if (chunks > t->nb) chunks = t->nb;
    int bpc = (t->nb + chunks - 1) / chunks;
    if (bpc > 8) bpc = 8;
    chunks = (t->nb + bpc - 1) / bpc;
    dim3 grid(qblocks, chunks);
    kde_bins_generic_kernel<<<grid, kGT, (size_t)kGQ * bpc * 4, s>>>(t->Xt, (int)t->n, t->d, t->dp, t->bnd, t->nb,
                                                                    bpc, kp.neg_c, kp.self_exclude, t->ws.binsum);
    return cudaGetLastError();
}

cudaError_t launch_leaf_values_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const int64_t items_est = t->n * (int64_t)(kp.L < t->nb ? kp.L : t->nb);
    const int64_t chunks_per_bin = (items_est / t->nb + kGQ - 1) / kGQ + 1;
    int64_t S = (152 * 2 * 8 + t->nb - 1) / t->nb;
    if (S > chunks_per_bin) S = chunks_per_bin;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    dim3 grid(t->nb, (unsigned)S);
    leaf_values_generic_kernel<<<grid, kGT, 0, s>>>(t->Xt, t->dp, t->bnd, t->ws.bin_off, t->ws.items_q, kp.neg_c,
                                                    kp.self_exclude, 1 << t->dm, t->ws.leafv);
    return cudaGetLastError();
}

}  // namespace fsg
