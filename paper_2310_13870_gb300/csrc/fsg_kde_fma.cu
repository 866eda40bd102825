// Bin pass of the KDE (Eq. 1) for d <= 16: for every query point and every
// node of level s0 of the halving tree (a "bin", a contiguous range of tree
// positions) the exact sum of k(x_q, x_p) over the bin's points.  Summing
// bins gives every node sum of the top s0 levels, including the degree
// g_[1,n] (Algorithm 2) and both halves at each of those levels of Algorithm 1.
//
// Arithmetic: FP32 direct differences (no ||x||^2 + ||y||^2 - 2xy expansion,
// hence no cancellation), packed FP32x2 on pairs of queries, one ex2 per pair
// element; per-bin sums accumulate in runs of <= 64 points before being added
// to the running bin total.
//
// Layout: CTA = 128 threads x (2*QP) queries per thread; blockIdx.y selects a
// chunk of `bpc` consecutive bins.  Point tiles (128 points, each coordinate
// stored twice so that one 64-bit shared load yields an FP32x2 operand) are
// staged into shared memory by cp.async.bulk on a 3-stage mbarrier ring.
// Bin totals are staged in shared memory and written out as [query][bin] rows.
#include <climits>

#include "fsg_internal.cuh"

namespace fsg {
namespace {

constexpr int kThreadsA = 128;
constexpr int kTileA = 128;
constexpr int kStagesA = 3;
constexpr int kRunA = 64;

template <int D>
struct QueriesPerThread {
    static constexpr int QP = D <= 4 ? 4 : 2;  // pairs of queries per thread
};

template <int D, int QP, bool MASK>
__device__ __forceinline__ void point_body(const float* __restrict__ tp, int p, int gpos, const uint64_t (&q)[QP][D],
                                           const int32_t (&qpos)[QP][2], uint64_t nc2, uint64_t (&acc)[QP]) {
    constexpr int DP = (D + 3) & ~3;
    const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(tp + (size_t)p * DP * 2);
    uint64_t c[D];
#pragma unroll
    for (int v = 0; v < (D + 1) / 2; ++v) {
        const ulonglong2 u = cp[v];
        c[2 * v] = u.x;
        if (2 * v + 1 < D) c[2 * v + 1] = u.y;
    }
#pragma unroll
    for (int k = 0; k < QP; ++k) {
        uint64_t dd = f2_sub(q[k][0], c[0]);
        uint64_t s = f2_mul(dd, dd);
#pragma unroll
        for (int t = 1; t < D; ++t) {
            dd = f2_sub(q[k][t], c[t]);
            s = f2_fma(dd, dd, s);
        }
        s = f2_mul(s, nc2);
        const float2 sv = f2_unpack(s);
        float e0 = ex2_approx(sv.x);
        float e1 = ex2_approx(sv.y);
        if (MASK) {
            if (gpos == qpos[k][0]) e0 = 0.f;
            if (gpos == qpos[k][1]) e1 = 0.f;
        }
        acc[k] = f2_add(acc[k], f2_pack(e0, e1));
    }
}

template <int D>
__global__ void __launch_bounds__(kThreadsA, 3)
kde_bins_kernel(const float* __restrict__ Xdup, const float* __restrict__ Xt, int n,
                const int32_t* __restrict__ bnd, int nb, int bpc, float neg_c, int self_exclude,
                float* __restrict__ binsum, int32_t* __restrict__ status) {
    constexpr int DP = (D + 3) & ~3;
    constexpr int QP = QueriesPerThread<D>::QP;
    constexpr int QCTA = kThreadsA * 2 * QP;
    constexpr int STAGE_FLOATS = kTileA * DP * 2;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* pts = reinterpret_cast<float*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(pts + kStagesA * STAGE_FLOATS);
    int32_t* bnd_s = reinterpret_cast<int32_t*>(bars + kStagesA);
    float* outs = reinterpret_cast<float*>(bnd_s + ((bpc + 1 + 3) & ~3));

    const int tid = threadIdx.x;
    const int qbase = blockIdx.x * QCTA;
    const int b0 = blockIdx.y * bpc;
    const int nbc = min(nb, b0 + bpc) - b0;
    for (int b = tid; b <= nbc; b += kThreadsA) bnd_s[b] = bnd[b0 + b];
    if (tid == 0) {
        for (int s = 0; s < kStagesA; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int pa = bnd_s[0], pe = bnd_s[nbc];
    const int ntiles = (pe - pa + kTileA - 1) / kTileA;
    if (tid == 0) {
        for (int s = 0; s < kStagesA && s < ntiles; ++s) {
            const int p0 = pa + s * kTileA;
            const uint32_t bytes = (uint32_t)min(kTileA, pe - p0) * DP * 2 * 4;
            mbar_arrive_expect_tx(&bars[s], bytes);
            bulk_g2s(pts + s * STAGE_FLOATS, Xdup + (size_t)p0 * DP * 2, bytes, &bars[s]);
        }
    }

    // This thread's queries: pair k holds local queries 2*(k*128 + tid) + {0,1}.
    uint64_t q[QP][D];
    int32_t qpos[QP][2];
#pragma unroll
    for (int k = 0; k < QP; ++k) {
        const int ql = 2 * (k * kThreadsA + tid);
        const int g0 = qbase + ql, g1 = g0 + 1;
        qpos[k][0] = g0 < n ? g0 : -1;
        qpos[k][1] = g1 < n ? g1 : -1;
#pragma unroll
        for (int t = 0; t < D; ++t) {
            const float x0 = g0 < n ? Xt[(size_t)g0 * DP + t] : 0.f;
            const float x1 = g1 < n ? Xt[(size_t)g1 * DP + t] : 0.f;
            q[k][t] = f2_pack(x0, x1);
        }
    }
    const uint64_t nc2 = f2_pack(neg_c, neg_c);
    uint64_t binacc[QP];
#pragma unroll
    for (int k = 0; k < QP; ++k) binacc[k] = 0ull;
    int bin = 0;
    int next_b = nbc > 0 ? bnd_s[1] : INT_MAX;
    const int qlo = qbase, qhi = min(n, qbase + QCTA);

    for (int tile = 0; tile < ntiles; ++tile) {
        const int s = tile % kStagesA;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)(tile / kStagesA) & 1u, status);
        if (__syncthreads_or(!ok)) {
            // A copy never completed: wait (bounded) for the others in flight, then leave.
            for (int t2 = tile + 1; t2 < min(ntiles, tile + kStagesA); ++t2)
                mbar_wait_bounded(&bars[t2 % kStagesA], (uint32_t)(t2 / kStagesA) & 1u, status);
            return;
        }
        const float* tp = pts + s * STAGE_FLOATS;
        const int t0 = pa + tile * kTileA;
        const int cnt = min(kTileA, pe - t0);
        int p = 0;
        while (p < cnt) {
            int run_end = min(cnt, next_b - t0);
            run_end = min(run_end, p + kRunA);
            uint64_t acc[QP];
#pragma unroll
            for (int k = 0; k < QP; ++k) acc[k] = 0ull;
            const bool diag = self_exclude && (t0 + p < qhi) && (t0 + run_end > qlo);
            if (!diag) {
#pragma unroll 2
                for (; p < run_end; ++p) point_body<D, QP, false>(tp, p, t0 + p, q, qpos, nc2, acc);
            } else {
                for (; p < run_end; ++p) point_body<D, QP, true>(tp, p, t0 + p, q, qpos, nc2, acc);
            }
#pragma unroll
            for (int k = 0; k < QP; ++k) binacc[k] = f2_add(binacc[k], acc[k]);
            while (t0 + p == next_b && bin < nbc) {
#pragma unroll
                for (int k = 0; k < QP; ++k) {
                    const int ql = 2 * (k * kThreadsA + tid);
                    const float2 v = f2_unpack(binacc[k]);
                    outs[ql * bpc + bin] = v.x;
                    outs[(ql + 1) * bpc + bin] = v.y;
                    binacc[k] = 0ull;
                }
                ++bin;
                next_b = bin < nbc ? bnd_s[bin + 1] : INT_MAX;
            }
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0 && tile + kStagesA < ntiles) {
            const int p0 = pa + (tile + kStagesA) * kTileA;
            const uint32_t bytes = (uint32_t)min(kTileA, pe - p0) * DP * 2 * 4;
            mbar_arrive_expect_tx(&bars[s], bytes);
            bulk_g2s(pts + s * STAGE_FLOATS, Xdup + (size_t)p0 * DP * 2, bytes, &bars[s]);
        }
    }
    __syncthreads();
    const int nq = min(QCTA, n - qbase);
    for (int e = tid; e < nq * nbc; e += kThreadsA) {
        const int ql = e / nbc, b = e - ql * nbc;
        binsum[(size_t)(qbase + ql) * nb + b0 + b] = outs[ql * bpc + b];
    }
}

template <int D>
cudaError_t launch_d(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    constexpr int DP = (D + 3) & ~3;
    constexpr int QCTA = kThreadsA * 2 * QueriesPerThread<D>::QP;
    const int qblocks = (int)((t->n + QCTA - 1) / QCTA);
    // Enough CTAs for several waves on 152 SMs; at most 8 bins per CTA.
    int chunks = (2048 + qblocks - 1) / qblocks;
    if (chunks < 1) chunks = 1;
    if (chunks > t->nb) chunks = t->nb;
    int bpc = (t->nb + chunks - 1) / chunks;
    if (bpc > 8) bpc = 8;
    chunks = (t->nb + bpc - 1) / bpc;
    const size_t smem = (size_t)kStagesA * kTileA * DP * 2 * 4 + kStagesA * 8 + ((bpc + 1 + 3) & ~3) * 4 +
                        (size_t)QCTA * bpc * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kde_bins_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             96 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid(qblocks, chunks);
    kde_bins_kernel<D><<<grid, kThreadsA, smem, s>>>(t->Xdup, t->Xt, (int)t->n, t->bnd, t->nb, bpc, kp.neg_c,
                                                     kp.self_exclude, t->ws.binsum, t->status);
    return cudaGetLastError();
}

}  // namespace

bool kde_bins_supported(const fsg_tree* t) { return t->d >= 1 && t->d <= kMaxFmaDim && t->Xdup != nullptr; }

cudaError_t launch_kde_bins(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    switch (t->d) {
        case 1: return launch_d<1>(t, kp, s);
        case 2: return launch_d<2>(t, kp, s);
        case 3: return launch_d<3>(t, kp, s);
        case 4: return launch_d<4>(t, kp, s);
        case 5: return launch_d<5>(t, kp, s);
        case 6: return launch_d<6>(t, kp, s);
        case 7: return launch_d<7>(t, kp, s);
        case 8: return launch_d<8>(t, kp, s);
        case 9: return launch_d<9>(t, kp, s);
        case 10: return launch_d<10>(t, kp, s);
        case 11: return launch_d<11>(t, kp, s);
        case 12: return launch_d<12>(t, kp, s);
        case 13: return launch_d<13>(t, kp, s);
        case 14: return launch_d<14>(t, kp, s);
        case 15: return launch_d<15>(t, kp, s);
        case 16: return launch_d<16>(t, kp, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsg

// ---------------------------------------------------------------------------
// Symmetric bin pass.  k(x_q, x_p) = k(x_p, x_q), so each unordered pair is
// evaluated once: CTA (k1, k2), k2 >= k1, takes the 8 bins of block k1 as
// queries (warp w <-> bin 8 k1 + w, lane <-> 4 consecutive queries of that
// bin, as two FP32x2 pairs) and the points of block k2.  The value is added
// to the query's row (register accumulators per bin, as in the plain pass)
// and, for k2 > k1, to the point's row at the query's bin: the warp's 4 x 32
// values per point are summed by a 16-point reduce-scatter across lanes, so
// each lane ends up holding the bin sum of one point.  Diagonal blocks
// (k2 == k1) are evaluated in both orders and not mirrored.  Every (row, bin)
// entry has exactly one writer; rows are staged in shared memory and written
// as 32-byte pieces.  Requires bins of at most 128 points.
// ---------------------------------------------------------------------------
namespace fsg {
namespace {

constexpr int kSymWarps = 8;        // bins per block
constexpr int kSymThreads = kSymWarps * 32;
constexpr int kSymTile = 128;       // points per shared-memory stage
constexpr int kSymStages = 3;
constexpr int kSymBatch = 16;       // points per mirror reduce-scatter

template <int D, bool MASK>
__device__ __forceinline__ float sym_point(const float* __restrict__ tp, int p, int gpos, const uint64_t (&q)[2][D],
                                           const int32_t (&qmask)[4], uint64_t nc2, uint64_t (&acc)[2]) {
    constexpr int DP = (D + 3) & ~3;
    const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(tp + (size_t)p * DP * 2);
    uint64_t c[D];
#pragma unroll
    for (int v = 0; v < (D + 1) / 2; ++v) {
        const ulonglong2 u = cp[v];
        c[2 * v] = u.x;
        if (2 * v + 1 < D) c[2 * v + 1] = u.y;
    }
    uint64_t e2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        // two interleaved accumulation chains (even / odd coordinates)
        uint64_t dd = f2_sub(q[k][0], c[0]);
        uint64_t s = f2_mul(dd, dd);
        uint64_t s1 = 0ull;
        if (D > 1) {
            dd = f2_sub(q[k][1], c[1]);
            s1 = f2_mul(dd, dd);
        }
#pragma unroll
        for (int t = 2; t < D; ++t) {
            dd = f2_sub(q[k][t], c[t]);
            if (t & 1) s1 = f2_fma(dd, dd, s1); else s = f2_fma(dd, dd, s);
        }
        if (D > 1) s = f2_add(s, s1);
        s = f2_mul(s, nc2);
        const float2 sv = f2_unpack(s);
        float e0 = ex2_approx(sv.x);
        float e1 = ex2_approx(sv.y);
        if (MASK) {
            if (gpos == qmask[2 * k]) e0 = 0.f;
            if (gpos == qmask[2 * k + 1]) e1 = 0.f;
        }
        e2[k] = f2_pack(e0, e1);
        acc[k] = f2_add(acc[k], e2[k]);
    }
    const float2 t = f2_unpack(f2_add(e2[0], e2[1]));
    return t.x + t.y;
}

// Sum over the 32 lanes of v[j] (j < 16) for 16 points; lane l returns the
// total of point (l & 15).
__device__ __forceinline__ float reduce_scatter16(float (&v)[kSymBatch], int lane) {
#pragma unroll
    for (int half = 8; half >= 1; half >>= 1) {
        const bool up = (lane & half) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = up ? v[j] : v[j + half];
            const float keep = up ? v[j + half] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// The point loop of one symmetric tile; MIRROR = off-diagonal block.
// Returns false if a bounded wait ran out.
template <int D, bool MIRROR>
__device__ __forceinline__ bool sym_tiles(float* pts, uint64_t* bars, const float* __restrict__ Xdup, int pa, int pe,
                                          int ntiles, const int32_t* pbnd, int npb, const uint64_t (&q)[2][D],
                                          const int32_t (&qmask)[4], uint64_t nc2, float* outs, float* mir, int w,
                                          int lane, int tid, bool wvalid, int32_t* status) {
    constexpr int DP = (D + 3) & ~3;
    constexpr int STAGE_FLOATS = kSymTile * DP * 2;
    uint64_t binacc[2] = {0ull, 0ull};
    int bin = 0;
    int next_b = pbnd[1];

    for (int tile = 0; tile < ntiles; ++tile) {
        const int s = tile % kSymStages;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)(tile / kSymStages) & 1u, status);
        if (__syncthreads_or(!ok)) {
            for (int t2 = tile + 1; t2 < min(ntiles, tile + kSymStages); ++t2)
                mbar_wait_bounded(&bars[t2 % kSymStages], (uint32_t)(t2 / kSymStages) & 1u, status);
            return false;
        }
        const float* tp = pts + s * STAGE_FLOATS;
        const int t0 = pa + tile * kSymTile;
        const int cnt = min(kSymTile, pe - t0);
        for (int pb = 0; pb < cnt; pb += kSymBatch) {
            const int nbat = min(kSymBatch, cnt - pb);
            float colv[kSymBatch];
#pragma unroll
            for (int j = 0; j < kSymBatch; ++j) {
                colv[j] = 0.f;
                if (j < nbat) {
                    const int gp = t0 + pb + j;
                    colv[j] = sym_point<D, !MIRROR>(tp, pb + j, gp, q, qmask, nc2, binacc);
                    if (gp + 1 == next_b) {  // end of a point bin: store this lane's 4 row sums
                        const float2 v0 = f2_unpack(binacc[0]), v1 = f2_unpack(binacc[1]);
                        const int qb = (w * 32 + lane) * 4;
                        outs[(qb + 0) * kSymWarps + bin] = v0.x;
                        outs[(qb + 1) * kSymWarps + bin] = v0.y;
                        outs[(qb + 2) * kSymWarps + bin] = v1.x;
                        outs[(qb + 3) * kSymWarps + bin] = v1.y;
                        binacc[0] = binacc[1] = 0ull;
                        ++bin;
                        next_b = bin < npb ? pbnd[bin + 1] : -1;
                    }
                }
            }
            if (MIRROR) {
                const float tot = reduce_scatter16(colv, lane);
                const int pl = lane & 15;
                if (lane < 16 && pl < nbat && wvalid) mir[(t0 + pb - pa + pl) * kSymWarps + w] = tot;
            }
        }
        __syncthreads();
        if (tid == 0 && tile + kSymStages < ntiles) {
            const int p0 = pa + (tile + kSymStages) * kSymTile;
            const uint32_t bytes = (uint32_t)min(kSymTile, pe - p0) * DP * 2 * 4;
            mbar_arrive_expect_tx(&bars[s], bytes);
            bulk_g2s(pts + s * STAGE_FLOATS, Xdup + (size_t)p0 * DP * 2, bytes, &bars[s]);
        }
    }
    return true;
}

template <int D>
__global__ void __launch_bounds__(kSymThreads, 2)
kde_bins_sym_kernel(const float* __restrict__ Xdup, const float* __restrict__ Xt, int n,
                    const int32_t* __restrict__ bnd, int nb, float neg_c, int self_exclude,
                    float* __restrict__ binsum, int32_t* __restrict__ status) {
    constexpr int DP = (D + 3) & ~3;
    constexpr int STAGE_FLOATS = kSymTile * DP * 2;
    constexpr int QMAX = kSymWarps * 128;  // query slots per block
    const int k2 = blockIdx.x, k1 = blockIdx.y;
    if (k2 < k1) return;
    const bool mirror = k2 > k1;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* pts = reinterpret_cast<float*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(pts + kSymStages * STAGE_FLOATS);
    int32_t* bnd_s = reinterpret_cast<int32_t*>(bars + kSymStages);   // 2 x (kSymWarps + 1)
    float* outs = reinterpret_cast<float*>(bnd_s + 2 * (kSymWarps + 1) + 2);  // [QMAX][8]
    float* mir = outs + QMAX * kSymWarps;                                     // [8 * 128][8]

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int qb0 = k1 * kSymWarps, pb0 = k2 * kSymWarps;
    const int nqb = min(kSymWarps, nb - qb0), npb = min(kSymWarps, nb - pb0);
    if (tid <= nqb) bnd_s[tid] = bnd[qb0 + tid];
    if (tid <= npb) bnd_s[kSymWarps + 1 + tid] = bnd[pb0 + tid];
    if (tid == 0) {
        for (int s = 0; s < kSymStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int32_t* pbnd = bnd_s + kSymWarps + 1;
    const int pa = pbnd[0], pe = pbnd[npb];
    const int ntiles = (pe - pa + kSymTile - 1) / kSymTile;
    if (tid == 0) {
        for (int s = 0; s < kSymStages && s < ntiles; ++s) {
            const int p0 = pa + s * kSymTile;
            const uint32_t bytes = (uint32_t)min(kSymTile, pe - p0) * DP * 2 * 4;
            mbar_arrive_expect_tx(&bars[s], bytes);
            bulk_g2s(pts + s * STAGE_FLOATS, Xdup + (size_t)p0 * DP * 2, bytes, &bars[s]);
        }
    }
    // This warp's bin and this lane's four queries (two FP32x2 pairs).
    const bool wvalid = w < nqb;
    const int qlo = wvalid ? bnd_s[w] : 0, qhi = wvalid ? bnd_s[w + 1] : 0;
    uint64_t q[2][D];
    int32_t qpos[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int g = qlo + 4 * lane + h;
        qpos[h] = g < qhi ? g : -1;
    }
    // Empty query slots sit at coordinate 1e19: every difference squared
    // overflows to +inf, so their kernel values (and mirror share) are 0.
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
        for (int t = 0; t < D; ++t) {
            const float x0 = qpos[2 * k] >= 0 ? Xt[(size_t)qpos[2 * k] * DP + t] : 1e19f;
            const float x1 = qpos[2 * k + 1] >= 0 ? Xt[(size_t)qpos[2 * k + 1] * DP + t] : 1e19f;
            q[k][t] = f2_pack(x0, x1);
        }
    }
    const uint64_t nc2 = f2_pack(neg_c, neg_c);
    // self term: only the diagonal block can meet a query's own position
    int32_t qmask[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) qmask[h] = (!mirror && self_exclude) ? qpos[h] : -1;
    const bool done = mirror
        ? sym_tiles<D, true>(pts, bars, Xdup, pa, pe, ntiles, pbnd, npb, q, qmask, nc2, outs, mir, w, lane, tid,
                             wvalid, status)
        : sym_tiles<D, false>(pts, bars, Xdup, pa, pe, ntiles, pbnd, npb, q, qmask, nc2, outs, mir, w, lane, tid,
                              wvalid, status);
    if (!done) return;
    __syncthreads();
    // Query rows: bins pb0 .. pb0+npb-1 of every query of this block.
    const int qa = bnd_s[0], qe = bnd_s[nqb];
    for (int e = tid; e < (qe - qa) * npb; e += kSymThreads) {
        const int r = e / npb, b = e - r * npb;
        const int g = qa + r;
        int wq = 0;
        while (wq + 1 < nqb && g >= bnd_s[wq + 1]) ++wq;
        const int slot = wq * 128 + (g - bnd_s[wq]);
        binsum[(size_t)g * nb + pb0 + b] = outs[slot * kSymWarps + b];
    }
    // Point rows (mirror): bins qb0 .. qb0+nqb-1 of every point of block k2.
    if (mirror) {
        for (int e = tid; e < (pe - pa) * nqb; e += kSymThreads) {
            const int r = e / nqb, b = e - r * nqb;
            binsum[(size_t)(pa + r) * nb + qb0 + b] = mir[r * kSymWarps + b];
        }
    }
}

template <int D>
cudaError_t launch_sym_d(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    constexpr int DP = (D + 3) & ~3;
    const int nblk = (t->nb + kSymWarps - 1) / kSymWarps;
    const size_t smem = (size_t)kSymStages * kSymTile * DP * 2 * 4 + kSymStages * 8 +
                        (2 * (kSymWarps + 1) + 2) * 4 + (size_t)kSymWarps * 128 * kSymWarps * 4 * 2;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kde_bins_sym_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid(nblk, nblk);
    kde_bins_sym_kernel<D><<<grid, kSymThreads, smem, s>>>(t->Xdup, t->Xt, (int)t->n, t->bnd, t->nb, kp.neg_c,
                                                          kp.self_exclude, t->ws.binsum, t->status);
    return cudaGetLastError();
}

}  // namespace

bool kde_bins_sym_supported(const fsg_tree* t) {
    return kde_bins_supported(t) && t->mmax <= 128;
}

cudaError_t launch_kde_bins_sym(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    switch (t->d) {
        case 1: return launch_sym_d<1>(t, kp, s);
        case 2: return launch_sym_d<2>(t, kp, s);
        case 3: return launch_sym_d<3>(t, kp, s);
        case 4: return launch_sym_d<4>(t, kp, s);
        case 5: return launch_sym_d<5>(t, kp, s);
        case 6: return launch_sym_d<6>(t, kp, s);
        case 7: return launch_sym_d<7>(t, kp, s);
        case 8: return launch_sym_d<8>(t, kp, s);
        case 9: return launch_sym_d<9>(t, kp, s);
        case 10: return launch_sym_d<10>(t, kp, s);
        case 11: return launch_sym_d<11>(t, kp, s);
        case 12: return launch_sym_d<12>(t, kp, s);
        case 13: return launch_sym_d<13>(t, kp, s);
        case 14: return launch_sym_d<14>(t, kp, s);
        case 15: return launch_sym_d<15>(t, kp, s);
        case 16: return launch_sym_d<16>(t, kp, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fsg
