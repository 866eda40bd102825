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
#include <vector>

#include "fsg_internal.cuh"

FSG_BOUNDS_TU(fma)

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
        const size_t o = (size_t)(qbase + ql) * nb + b0 + b;
        if (FSG_INB(o, (long long)n * nb, kSitePlainRow)) binsum[o] = outs[ql * bpc + b];
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
    {
        const cudaError_t e = set_smem_limit(kde_bins_kernel<D>, 96 * 1024);
        if (e != cudaSuccess) return e;
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
// evaluated once.  Bins are grouped into blocks of G consecutive bins; CTA
// (k1, k2), k2 >= k1, takes the queries of block k1 and the points of block k2.
//
// Query side: the block's queries are laid out over the CTA's 256 lanes, each
// bin on its own run of ceil(m/4) lanes (4 consecutive queries per lane, as
// two FP32x2 pairs), so no lane mixes two bins and few lane slots are empty
// whatever the bin size m.  A warp's 32 lanes then meet at most three bins
// (every bin spans >= 16 lanes): "first" bin on the low lanes, "middle" bin,
// "last" bin on the high lanes.
//
// Point side: one shared-memory stage per point bin (cp.async.bulk on an
// mbarrier ring), so a bin's row sums are complete when its stage is done.
//
// Each value goes to the query's row (register accumulators, written when the
// point bin ends) and, for k2 > k1, to the point's row at the query's bin:
// per batch of 16 points the warp reduce-scatters the lane sums of its
// first/last bins (half-warp sums: first bin on lanes 0-15, last bin on lanes
// 16-31, or their total when there is no last bin) and of its middle bin,
// and adds them to a shared-memory row per point.  A bin spans at most two
// warps, so each (point, bin) entry receives at most two additions onto zero,
// whose result does not depend on their order.  Diagonal blocks (k2 == k1)
// are evaluated in both orders and not mirrored.
// Requires bins of 61..128 points (at most 16 per block).
// ---------------------------------------------------------------------------
namespace fsg {
namespace {

constexpr int kSymWarps = 8;
constexpr int kSymThreads = kSymWarps * 32;
constexpr int kSymMaxBin = 128;     // points per bin (one shared-memory stage)
constexpr int kSymMinBin = 61;      // a bin covers >= 16 lanes
constexpr int kSymNodes = 16;       // bins per block at most
constexpr int kSymMRow = kSymNodes + 1;  // mirror row stride: odd, so the B lanes that add to
                                         // B consecutive rows hit B distinct banks
constexpr int kSymStages = 3;
// points per mirror reduce-scatter (fewer for large d, to stay within 128 registers)
template <int D>
struct SymBatch {
    static constexpr int B = D <= 9 ? 16 : 8;
};
// CTAs per SM the register budget is cut for: three (80 registers) where that
// costs at most a few spilled words, two (128 registers) elsewhere.
template <int D>
struct SymOccupancy {
    static constexpr int value = (D <= 8 || D == 10) ? 3 : 2;
};

// Kernel values of one point against the lane's four queries; adds them to
// the row accumulators and returns their sum.  F: the kernel family.
template <int D, int F, bool MASK>
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
        // one accumulation chain per query pair: the two pairs and the
        // batch's points give the independent work (a second chain per pair,
        // even / odd coordinates, cost an extra add and measured 2% slower)
        uint64_t dd = f2_sub(q[k][0], c[0]);
        uint64_t s = fam_first2<F>(dd);
#pragma unroll
        for (int t = 1; t < D; ++t) {
            dd = f2_sub(q[k][t], c[t]);
            s = fam_acc2<F>(dd, s);
        }
        s = f2_mul(fam_fin2<F>(s), nc2);
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

// Reduce-scatter of v[j] (j < B) over lanes: lane l returns the sum over its
// half-warp (lanes 0-15 or 16-31) of point l % B.
template <int B>
__device__ __forceinline__ float reduce_scatter_half(float (&v)[B], int lane) {
#pragma unroll
    for (int half = B / 2; half >= 1; half >>= 1) {
        const bool up = (lane & half) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = up ? v[j] : v[j + half];
            const float keep = up ? v[j + half] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    float r = v[0];
    if (B < 16) r += __shfl_xor_sync(0xffffffffu, r, 8);  // B == 8: lanes l and l ^ 8 hold halves
    return r;
}

// Per-warp description of the query bins its lanes meet.
struct SymWarp {
    int nseg;   // bins met (0..3)
    int rf;     // block-local index of the first one
    bool mid;   // this lane's queries are in the middle bin
};

// One batch of points (FULL: a whole batch, no bounds tests).
template <int D, int F, bool MIRROR, bool FULL>
__device__ __forceinline__ void sym_batch(const float* __restrict__ tp, int pb, int nbat, int gp0,
                                          const uint64_t (&q)[2][D], const int32_t (&qmask)[4], uint64_t nc2,
                                          uint64_t (&acc)[2], const SymWarp& sw, float* mrow, int lane) {
    constexpr int B = SymBatch<D>::B;
    float colE[B], colM[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        float tot = 0.f;
        if (FULL || j < nbat) tot = sym_point<D, F, !MIRROR>(tp, pb + j, gp0 + j, q, qmask, nc2, acc);
        colE[j] = sw.mid ? 0.f : tot;
        colM[j] = sw.mid ? tot : 0.f;
    }
    if (MIRROR && sw.nseg > 0) {  // warp-uniform
        const int pl = lane & (B - 1);
        float eh = reduce_scatter_half<B>(colE, lane);
        if (sw.nseg < 3) eh += __shfl_xor_sync(0xffffffffu, eh, 16);
        if (FULL || pl < nbat) {
            if (lane < B) atomicAdd(&mrow[(pb + pl) * kSymMRow + sw.rf], eh);
            else if (sw.nseg == 3 && lane >= 16 && lane < 16 + B)
                atomicAdd(&mrow[(pb + pl) * kSymMRow + sw.rf + 2], eh);
        }
        if (sw.nseg > 1) {
            float mh = reduce_scatter_half<B>(colM, lane);
            mh += __shfl_xor_sync(0xffffffffu, mh, 16);
            if ((FULL || pl < nbat) && lane < B) atomicAdd(&mrow[(pb + pl) * kSymMRow + sw.rf + 1], mh);
        }
    }
}

// The point-bin loop of one CTA.  Returns false if a bounded wait ran out.
template <int D, int F, bool MIRROR>
__device__ __forceinline__ bool sym_bins(float* pts, float* mir, uint64_t* bars, const float* __restrict__ Xdup,
                                         const int32_t* pbn, int np, const uint64_t (&q)[2][D],
                                         const int32_t (&qmask)[4], const int32_t (&qpos)[4], uint64_t nc2,
                                         const SymWarp& sw, int lane, int tid, int32_t* status,
                                         float* __restrict__ binsum, int nb, int pn0, int qn0, int nq,
                                         long long bins_lim) {
    constexpr int DP = (D + 3) & ~3;
    constexpr int STAGE_FLOATS = kSymMaxBin * DP * 2;
    for (int b = 0; b < np; ++b) {
        const int s = b % kSymStages;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)(b / kSymStages) & 1u, status);
        if (__syncthreads_or(!ok)) {
            for (int b2 = b + 1; b2 < min(np, b + kSymStages); ++b2)
                mbar_wait_bounded(&bars[b2 % kSymStages], (uint32_t)(b2 / kSymStages) & 1u, status);
            return false;
        }
        const float* tp = pts + s * STAGE_FLOATS;
        float* mrow = mir + (b & 1) * kSymMaxBin * kSymMRow;
        const int t0 = pbn[b], cnt = pbn[b + 1] - t0;
        uint64_t acc[2] = {0ull, 0ull};
        constexpr int B = SymBatch<D>::B;
        int pb = 0;
        for (; pb + B <= cnt; pb += B)
            sym_batch<D, F, MIRROR, true>(tp, pb, B, t0 + pb, q, qmask, nc2, acc, sw, mrow, lane);
        if (pb < cnt) sym_batch<D, F, MIRROR, false>(tp, pb, cnt - pb, t0 + pb, q, qmask, nc2, acc, sw, mrow, lane);
        {   // this point bin's row sums of the lane's queries
            const float2 v0 = f2_unpack(acc[0]), v1 = f2_unpack(acc[1]);
            const float vv[4] = {v0.x, v0.y, v1.x, v1.y};
#pragma unroll
            for (int h = 0; h < 4; ++h)
                if (qpos[h] >= 0 && FSG_INB((size_t)qpos[h] * nb + pn0 + b, bins_lim, kSiteSymRow))
                    binsum[(size_t)qpos[h] * nb + pn0 + b] = vv[h];
        }
        __syncthreads();
        if (tid == 0 && b + kSymStages < np) {
            const int p0 = pbn[b + kSymStages];
            const uint32_t bytes = (uint32_t)(pbn[b + kSymStages + 1] - p0) * DP * 2 * 4;
            mbar_arrive_expect_tx(&bars[s], bytes);
            bulk_g2s(pts + s * STAGE_FLOATS, Xdup + (size_t)p0 * DP * 2, bytes, &bars[s]);
        }
        if (MIRROR) {  // mirror rows of this bin's points: query bins qn0 .. qn0+nq-1
            for (int e = tid; e < cnt * nq; e += kSymThreads) {
                const int r = e / nq, c = e - r * nq;
                if (FSG_INB((size_t)(t0 + r) * nb + qn0 + c, bins_lim, kSiteSymMirror))
                    binsum[(size_t)(t0 + r) * nb + qn0 + c] = mrow[r * kSymMRow + c];
                mrow[r * kSymMRow + c] = 0.f;
            }
        }
    }
    return true;
}

// One block pair (k1, k2 >= k1) of one tree: the body of the symmetric pass.
template <int D, int F>
__device__ __forceinline__ void sym_block_pair(const float* __restrict__ Xdup, const float* __restrict__ Xt,
                                               const int32_t* __restrict__ bnd, int nb, int G, float neg_c,
                                               int self_exclude, float* __restrict__ binsum,
                                               int32_t* __restrict__ status, int k1, int k2,
                                               unsigned char* smem_raw) {
    constexpr int DP = (D + 3) & ~3;
    constexpr int STAGE_FLOATS = kSymMaxBin * DP * 2;
    const bool mirror = k2 > k1;
#ifdef FSG_BOUNDS_CHECK
    const long long bins_lim = (long long)bnd[nb] * nb;  // n x nb bin sums
#else
    const long long bins_lim = 0;
#endif
    float* pts = reinterpret_cast<float*>(smem_raw);                       // [stages][128][DP][2]
    float* mir = pts + kSymStages * STAGE_FLOATS;                          // [2][128][kSymMRow]
    uint64_t* bars = reinterpret_cast<uint64_t*>(mir + 2 * kSymMaxBin * kSymMRow);
    int32_t* qb = reinterpret_cast<int32_t*>(bars + kSymStages);           // query bin bounds [G+1]
    int32_t* pbn = qb + kSymNodes + 1;                                     // point bin bounds [G+1]
    int32_t* lb = pbn + kSymNodes + 1;                                     // first lane of each query bin

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int qn0 = k1 * G, pn0 = k2 * G;
    const int nq = min(G, nb - qn0), np = min(G, nb - pn0);
    if (tid <= nq) qb[tid] = bnd[qn0 + tid];
    if (tid <= np) pbn[tid] = bnd[pn0 + tid];
    for (int i = tid; i < 2 * kSymMaxBin * kSymMRow; i += kSymThreads) mir[i] = 0.f;
    if (tid == 0) {
        for (int s = 0; s < kSymStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        lb[0] = 0;
        for (int r = 0; r < nq; ++r) lb[r + 1] = lb[r] + (qb[r + 1] - qb[r] + 3) / 4;
        for (int s = 0; s < kSymStages && s < np; ++s) {
            const uint32_t bytes = (uint32_t)(pbn[s + 1] - pbn[s]) * DP * 2 * 4;
            mbar_arrive_expect_tx(&bars[s], bytes);
            bulk_g2s(pts + s * STAGE_FLOATS, Xdup + (size_t)pbn[s] * DP * 2, bytes, &bars[s]);
        }
    }
    __syncthreads();
    // This lane's query bin and four queries; the bins this warp meets.
    const int nl = lb[nq];
    auto bin_of_lane = [&](int x) {
        int r = 0;
        while (r + 1 < nq && x >= lb[r + 1]) ++r;
        return r;
    };
    const int ru = tid < nl ? bin_of_lane(tid) : -1;
    SymWarp sw;
    sw.rf = w * 32 < nl ? bin_of_lane(w * 32) : 0;
    sw.nseg = w * 32 < nl ? bin_of_lane(min(w * 32 + 31, nl - 1)) - sw.rf + 1 : 0;
    sw.mid = ru >= 0 && ru == sw.rf + 1;
    int32_t qpos[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int g = ru >= 0 ? qb[ru] + 4 * (tid - lb[ru]) + h : 0;
        qpos[h] = (ru >= 0 && g < qb[ru + 1]) ? g : -1;
    }
    // Empty query slots sit at coordinate 1e19: every difference squared
    // overflows to +inf, so their kernel values (and mirror share) are 0.
    uint64_t q[2][D];
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
    if (mirror)
        sym_bins<D, F, true>(pts, mir, bars, Xdup, pbn, np, q, qmask, qpos, nc2, sw, lane, tid, status, binsum, nb,
                          pn0, qn0, nq, bins_lim);
    else
        sym_bins<D, F, false>(pts, mir, bars, Xdup, pbn, np, q, qmask, qpos, nc2, sw, lane, tid, status, binsum, nb,
                           pn0, qn0, nq, bins_lim);
}

template <int D, int F>
__global__ void __launch_bounds__(kSymThreads, SymOccupancy<D>::value)
kde_bins_sym_kernel(const float* __restrict__ Xdup, const float* __restrict__ Xt, const int32_t* __restrict__ bnd,
                    int nb, int G, float neg_c, int self_exclude, float* __restrict__ binsum,
                    int32_t* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int k2 = blockIdx.x, k1 = blockIdx.y;
    if (k2 < k1) return;
    sym_block_pair<D, F>(Xdup, Xt, bnd, nb, G, neg_c, self_exclude, binsum, status, k1, k2, smem_raw);
}

// The symmetric pass of many trees in one launch (batches of point sets):
// CTA i takes the i-th block pair over all trees' triangles (k2 >= k1),
// trees in table order.
template <int D, int F>
__device__ __forceinline__ void sym_packed_item(const SymPackDesc* __restrict__ descs, int count, int item,
                                                unsigned char* smem_raw) {
    int lo = 0, hi = count;  // tree: descs[lo].pair_off <= item < descs[lo + 1].pair_off
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (descs[mid].pair_off <= item) lo = mid; else hi = mid;
    }
    const SymPackDesc& dsc = descs[lo];
    int k1 = 0, rem = item - dsc.pair_off;
    while (rem >= dsc.nblk - k1) { rem -= dsc.nblk - k1; ++k1; }
    sym_block_pair<D, F>(dsc.Xdup, dsc.Xt, dsc.bnd, dsc.nb, dsc.G, dsc.neg_c, dsc.self_exclude, dsc.binsum,
                         dsc.status, k1, k1 + rem, smem_raw);
}

template <int D, int F>
__global__ void __launch_bounds__(kSymThreads, SymOccupancy<D>::value)
kde_bins_sym_packed_kernel(const SymPackDesc* __restrict__ descs, int count) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    sym_packed_item<D, F>(descs, count, blockIdx.x, smem_raw);
}

// The same with the descriptors as a kernel parameter (up to kSymPackMax trees).
template <int D, int F>
__global__ void __launch_bounds__(kSymThreads, SymOccupancy<D>::value)
kde_bins_sym_packed_param_kernel(const __grid_constant__ SymPackTable tab) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    sym_packed_item<D, F>(tab.d, tab.count, blockIdx.x, smem_raw);
}

// Bins per block: as many as fit the CTA's 256 lanes (fewer if tuned so).
int sym_block_bins(const fsg_tree* t) {
    int g = kSymThreads / ((t->mmax + 3) / 4);
    if (g > kSymNodes) g = kSymNodes;
    if (t->tune.sym_bins > 0 && t->tune.sym_bins < g) g = t->tune.sym_bins;
    return g;
}

template <int D, int F>
cudaError_t launch_sym_d(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    constexpr int DP = (D + 3) & ~3;
    const int G = sym_block_bins(t);
    const int nblk = (t->nb + G - 1) / G;
    const size_t smem = (size_t)kSymStages * kSymMaxBin * DP * 2 * 4 + (size_t)2 * kSymMaxBin * kSymMRow * 4 +
                        kSymStages * 8 + 3 * (kSymNodes + 1) * 4;
    {
        const cudaError_t e = set_smem_limit(kde_bins_sym_kernel<D, F>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(nblk, nblk);
    kde_bins_sym_kernel<D, F><<<grid, kSymThreads, smem, s>>>(t->Xdup, t->Xt, t->bnd, t->nb, G, kp.neg_c,
                                                          kp.self_exclude, t->ws.binsum, t->status);
    return cudaGetLastError();
}

}  // namespace

bool kde_bins_sym_supported(const fsg_tree* t) {
    return kde_bins_supported(t) && t->mmax <= kSymMaxBin && t->n / t->nb >= kSymMinBin;
}

// Kernel evaluations the symmetric pass executes: every ordered pair inside a
// diagonal block, every unordered pair across blocks.
int64_t kde_bins_sym_evals(const fsg_tree* t) {
    const int G = sym_block_bins(t);
    // node sizes follow from the halving rule: floor or ceil of n / nb
    std::vector<int64_t> size(t->nb);
    for (int b = 0; b < t->nb; ++b) {
        int64_t lo = 0, hi = t->n;
        for (int l = t->s0 - 1; l >= 0; --l) {
            const int64_t mid = lo + (hi - lo) / 2;
            if ((b >> l) & 1) lo = mid; else hi = mid;
        }
        size[b] = hi - lo;
    }
    int64_t sq = 0;
    for (int b0 = 0; b0 < t->nb; b0 += G) {
        int64_t sb = 0;
        for (int b = b0; b < b0 + G && b < t->nb; ++b) sb += size[b];
        sq += sb * sb;
    }
    return (t->n * t->n + sq) / 2;
}

namespace {
template <int F>
cudaError_t launch_sym_family(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    switch (t->d) {
        case 1: return launch_sym_d<1, F>(t, kp, s);
        case 2: return launch_sym_d<2, F>(t, kp, s);
        case 3: return launch_sym_d<3, F>(t, kp, s);
        case 4: return launch_sym_d<4, F>(t, kp, s);
        case 5: return launch_sym_d<5, F>(t, kp, s);
        case 6: return launch_sym_d<6, F>(t, kp, s);
        case 7: return launch_sym_d<7, F>(t, kp, s);
        case 8: return launch_sym_d<8, F>(t, kp, s);
        case 9: return launch_sym_d<9, F>(t, kp, s);
        case 10: return launch_sym_d<10, F>(t, kp, s);
        case 11: return launch_sym_d<11, F>(t, kp, s);
        case 12: return launch_sym_d<12, F>(t, kp, s);
        case 13: return launch_sym_d<13, F>(t, kp, s);
        case 14: return launch_sym_d<14, F>(t, kp, s);
        case 15: return launch_sym_d<15, F>(t, kp, s);
        case 16: return launch_sym_d<16, F>(t, kp, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

namespace {
// tab != nullptr: descriptors by value (kernel parameter), else d_descs.
template <int D, int F>
cudaError_t launch_sym_packed_d(const SymPackDesc* d_descs, const SymPackTable* tab, int count, int total,
                                cudaStream_t s) {
    constexpr int DP = (D + 3) & ~3;
    const size_t smem = (size_t)kSymStages * kSymMaxBin * DP * 2 * 4 + (size_t)2 * kSymMaxBin * kSymMRow * 4 +
                        kSymStages * 8 + 3 * (kSymNodes + 1) * 4;
    if (tab) {
        const cudaError_t e = set_smem_limit(kde_bins_sym_packed_param_kernel<D, F>, (int)smem);
        if (e != cudaSuccess) return e;
        kde_bins_sym_packed_param_kernel<D, F><<<total, kSymThreads, smem, s>>>(*tab);
    } else {
        const cudaError_t e = set_smem_limit(kde_bins_sym_packed_kernel<D, F>, (int)smem);
        if (e != cudaSuccess) return e;
        kde_bins_sym_packed_kernel<D, F><<<total, kSymThreads, smem, s>>>(d_descs, count);
    }
    return cudaGetLastError();
}
template <int F>
cudaError_t launch_sym_packed_family(int d, const SymPackDesc* d_descs, const SymPackTable* tab, int count,
                                     int total, cudaStream_t s) {
    switch (d) {
        case 1: return launch_sym_packed_d<1, F>(d_descs, tab, count, total, s);
        case 2: return launch_sym_packed_d<2, F>(d_descs, tab, count, total, s);
        case 3: return launch_sym_packed_d<3, F>(d_descs, tab, count, total, s);
        case 4: return launch_sym_packed_d<4, F>(d_descs, tab, count, total, s);
        case 5: return launch_sym_packed_d<5, F>(d_descs, tab, count, total, s);
        case 6: return launch_sym_packed_d<6, F>(d_descs, tab, count, total, s);
        case 7: return launch_sym_packed_d<7, F>(d_descs, tab, count, total, s);
        case 8: return launch_sym_packed_d<8, F>(d_descs, tab, count, total, s);
        case 9: return launch_sym_packed_d<9, F>(d_descs, tab, count, total, s);
        case 10: return launch_sym_packed_d<10, F>(d_descs, tab, count, total, s);
        case 11: return launch_sym_packed_d<11, F>(d_descs, tab, count, total, s);
        case 12: return launch_sym_packed_d<12, F>(d_descs, tab, count, total, s);
        case 13: return launch_sym_packed_d<13, F>(d_descs, tab, count, total, s);
        case 14: return launch_sym_packed_d<14, F>(d_descs, tab, count, total, s);
        case 15: return launch_sym_packed_d<15, F>(d_descs, tab, count, total, s);
        case 16: return launch_sym_packed_d<16, F>(d_descs, tab, count, total, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

int sym_pack_fill(const fsg_tree* t, const KernelParams& kp, int pair_off, SymPackDesc* out) {
    const int G = sym_block_bins(t);
    const int nblk = (t->nb + G - 1) / G;
    out->Xdup = t->Xdup;
    out->Xt = t->Xt;
    out->bnd = t->bnd;
    out->binsum = t->ws.binsum;
    out->status = t->status;
    out->nb = t->nb;
    out->G = G;
    out->nblk = nblk;
    out->pair_off = pair_off;
    out->neg_c = kp.neg_c;
    out->self_exclude = kp.self_exclude;
    return nblk * (nblk + 1) / 2;
}

cudaError_t launch_kde_bins_sym_packed(const SymPackDesc* d_descs, int count, int total, int d, int family,
                                       cudaStream_t s) {
    if (count < 1 || total < 1) return cudaSuccess;
    switch (family) {
        case kFamLaplace: return launch_sym_packed_family<kFamLaplace>(d, d_descs, nullptr, count, total, s);
        case kFamExp: return launch_sym_packed_family<kFamExp>(d, d_descs, nullptr, count, total, s);
        default: return launch_sym_packed_family<kFamGauss>(d, d_descs, nullptr, count, total, s);
    }
}

cudaError_t launch_kde_bins_sym_packed(const SymPackTable& tab, int total, int d, int family, cudaStream_t s) {
    if (tab.count < 1 || total < 1) return cudaSuccess;
    switch (family) {
        case kFamLaplace: return launch_sym_packed_family<kFamLaplace>(d, nullptr, &tab, tab.count, total, s);
        case kFamExp: return launch_sym_packed_family<kFamExp>(d, nullptr, &tab, tab.count, total, s);
        default: return launch_sym_packed_family<kFamGauss>(d, nullptr, &tab, tab.count, total, s);
    }
}

cudaError_t launch_kde_bins_sym(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    switch (kp.family) {
        case kFamLaplace: return launch_sym_family<kFamLaplace>(t, kp, s);
        case kFamExp: return launch_sym_family<kFamExp>(t, kp, s);
        default: return launch_sym_family<kFamGauss>(t, kp, s);
    }
}

}  // namespace fsg
