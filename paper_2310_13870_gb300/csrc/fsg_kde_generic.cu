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
//                               leaf finish reads;
//   kde_bins_generic_sym_kernel: the bin pass evaluating each unordered pair
//                               once (bins of <= 128 points), see below.
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

// acc[i][j] += sum over the chunk of (q_i - p_j)^2 (F: the kernel family's
// distance term, fam_acc1).
template <int F>
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
                acc[i][j] = fam_acc1<F>(dd, acc[i][j]);
            }
        }
    }
}

template <int F>
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
            accumulate_chunk<F>(Qs, Ps, tq, tp, acc);
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
                    float k = ex2_approx(fam_fin1<F>(acc[i][j]) * neg_c);
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

// ---------------------------------------------------------------------------
// Symmetric bin pass for d > 16.  The positions are cut into tiles of 128;
// CTA (i, j >= i) (a linear index over the triangle) evaluates the 128 x 128
// block of tile i (queries) against tile j (points) once, with FP32x2 pairs of
// queries against duplicated point coordinates.  Its row sums go to (query,
// point bin) and, for j > i, its column sums to (point, query bin).  The
// partial sums are reduced in shared memory in a fixed order, then added with
// one atomic addition per (row, bin) and CTA into bin sums zeroed beforehand.
// A bin of <= 128 points meets at most two tiles, so every bin sum receives
// at most two additions onto zero and does not depend on their order.
// ---------------------------------------------------------------------------
constexpr int kST = 128;             // tile side (queries and points)
constexpr int kSK = 32;              // coordinates per chunk
constexpr int kSQS = kST + 4;        // transposed query row stride (floats)
constexpr int kSPS = kST + 2;        // transposed point row stride (float pairs)
constexpr size_t kSymGenSmem = (size_t)kSK * kSQS * 4 + (size_t)kSK * kSPS * 8;  // one stage

// Packed 128 x 128 tiles.  Thread (tq, tp) of 256 holds the rows 4 tq .. 4 tq + 3
// and 64 + 4 tq .. 64 + 4 tq + 3 (four FP32x2 pairs) and the columns 4 tp ..
// 4 tp + 3 and 64 + 4 tp .. 64 + 4 tp + 3 (NPG = 1: the first group only).
__device__ __forceinline__ int tile_row(int tq, int i) { return i < 4 ? 4 * tq + i : 64 + 4 * tq + i - 4; }

// Chunk [k0, k0 + 32) of 128 rows, transposed: rows into Qs[k][r] (absent rows
// get `fill` on real coordinates), columns into Ps[k][r] twice (absent: 0).
// Warp w stores coordinate group v = w of 32 consecutive rows per step, so the
// transposed stores of a warp hit 32 different banks.
template <typename RowQ, typename RowP>
__device__ __forceinline__ void load_tiles(float* __restrict__ Qs, float* __restrict__ Ps, RowQ rowq, RowP rowp,
                                           const float* __restrict__ Xt, int dp, int k0, float fill) {
    const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;
    const int k = k0 + 4 * v;
    float2* pd = reinterpret_cast<float2*>(Ps);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const int r = 32 * it + lane;
        const int qpos = rowq(r), ppos = rowp(r);
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < dp) {
            x = qpos >= 0 ? *reinterpret_cast<const float4*>(Xt + (size_t)qpos * dp + k)
                          : make_float4(fill, fill, fill, fill);
        }
        Qs[(4 * v + 0) * kSQS + r] = x.x;
        Qs[(4 * v + 1) * kSQS + r] = x.y;
        Qs[(4 * v + 2) * kSQS + r] = x.z;
        Qs[(4 * v + 3) * kSQS + r] = x.w;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ppos >= 0 && k < dp) y = *reinterpret_cast<const float4*>(Xt + (size_t)ppos * dp + k);
        pd[(4 * v + 0) * kSPS + r] = make_float2(y.x, y.x);
        pd[(4 * v + 1) * kSPS + r] = make_float2(y.y, y.y);
        pd[(4 * v + 2) * kSPS + r] = make_float2(y.z, y.z);
        pd[(4 * v + 3) * kSPS + r] = make_float2(y.w, y.w);
    }
}

// acc[a][b] += (row pair a - column b)^2 over the 32 coordinates of the chunk.
template <int NPG, int F>
__device__ __forceinline__ void accumulate_pairs(const float* __restrict__ Qs, const float* __restrict__ Ps, int tq,
                                                 int tp, uint64_t (&acc)[4][4 * NPG]) {
#pragma unroll 2
    for (int k = 0; k < kSK; ++k) {
        const ulonglong2 qa = *reinterpret_cast<const ulonglong2*>(Qs + k * kSQS + 4 * tq);
        const ulonglong2 qb = *reinterpret_cast<const ulonglong2*>(Qs + k * kSQS + 64 + 4 * tq);
        const uint64_t qv[4] = {qa.x, qa.y, qb.x, qb.y};
        const ulonglong2* pr = reinterpret_cast<const ulonglong2*>(Ps + 2 * (k * kSPS));
        uint64_t pv[4 * NPG];
#pragma unroll
        for (int g = 0; g < NPG; ++g) {
            const ulonglong2 p0 = pr[32 * g + 2 * tp], p1 = pr[32 * g + 2 * tp + 1];
            pv[4 * g + 0] = p0.x;
            pv[4 * g + 1] = p0.y;
            pv[4 * g + 2] = p1.x;
            pv[4 * g + 3] = p1.y;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = 0; b < 4 * NPG; ++b) {
                const uint64_t dd = f2_sub(qv[a], pv[b]);
                acc[a][b] = fam_acc2<F>(dd, acc[a][b]);
            }
        }
    }
}

// Tile pair (i, j >= i) of the linear index L over the upper triangle of T
// tiles: an FP32 estimate of the row, corrected exactly in integers.
__device__ __forceinline__ void tri_index(long long L, int T, int& i, int& j) {
    const float b = 2.f * (float)T + 1.f;
    long long ii = (long long)((b - sqrtf(fmaxf(b * b - 8.f * (float)L, 0.f))) * 0.5f);
    auto start = [&](long long r) { return r * T - r * (r - 1) / 2; };
    if (ii < 0) ii = 0;
    if (ii > T - 1) ii = T - 1;
    while (ii > 0 && start(ii) > L) --ii;
    while (ii + 1 < T && start(ii + 1) <= L) ++ii;
    i = (int)ii;
    j = (int)(ii + (L - start(ii)));
}

// Bin of position x: s0 halving steps from the root (left half = floor(size/2)).
__device__ __forceinline__ int bin_of(int n, int s0, int x) {
    int b = 0, lo = 0, hi = n;
    for (int t = 0; t < s0; ++t) {
        const int mid = lo + (hi - lo) / 2;
        b <<= 1;
        if (x >= mid) {
            b |= 1;
            lo = mid;
        } else {
            hi = mid;
        }
    }
    return b;
}

// Adds v to the slot lb (0..2) of a 3-slot accumulator without indexing.
__device__ __forceinline__ void add3(float (&r)[3], int lb, float v) {
    r[0] += lb == 0 ? v : 0.f;
    r[1] += lb == 1 ? v : 0.f;
    r[2] += lb == 2 ? v : 0.f;
}

// Transposed tiles: tile i holds, for k < dpc (d padded to a multiple of 32),
// the query layout Q[k][132] (absent rows at 1e19 on real coordinates) and
// then the duplicated point layout P[k][130][2] (absent rows 0).  Built per
// (tile, 32-coordinate chunk) through a shared-memory transpose.
__global__ void __launch_bounds__(kGT)
generic_tiles_kernel(const float* __restrict__ Xt, int n, int d, int dp, int dpc, float* __restrict__ Xtt) {
    __shared__ float sm[kST][kSK + 1];
    const int i = blockIdx.x, c = blockIdx.y;
    const int k0 = c * kSK;
    for (int e = threadIdx.x; e < kST * kSK; e += kGT) {
        const int r = e / kSK, k = e - r * kSK;
        const int pos = i * kST + r;
        sm[r][k] = (pos < n && k0 + k < d) ? Xt[(size_t)pos * dp + k0 + k] : 0.f;
    }
    __syncthreads();
    float* tileQ = Xtt + (size_t)i * dpc * (kSQS + 2 * kSPS);
    float* tileP = tileQ + (size_t)dpc * kSQS;
    for (int e = threadIdx.x; e < kSK * kSQS; e += kGT) {
        const int k = e / kSQS, r = e - k * kSQS;
        const int pos = i * kST + r;
        float v = 0.f;
        if (r < kST) v = pos < n ? sm[r][k] : (k0 + k < d ? 1e19f : 0.f);
        tileQ[(size_t)(k0 + k) * kSQS + r] = v;
    }
    for (int e = threadIdx.x; e < kSK * kSPS; e += kGT) {
        const int k = e / kSPS, r = e - k * kSPS;
        const float v = r < kST ? sm[r][k] : 0.f;
        reinterpret_cast<float2*>(tileP)[(size_t)(k0 + k) * kSPS + r] = make_float2(v, v);
    }
}

template <int F>
__global__ void __launch_bounds__(kGT, 2)
kde_bins_generic_sym_kernel(const float* __restrict__ Xtt, int n, int dpc, const int32_t* __restrict__ bnd, int nb,
                            int s0, int T, float neg_c, int self_exclude, float* __restrict__ binsum,
                            int32_t* __restrict__ status) {
    extern __shared__ __align__(16) float gsm[];
    constexpr int kStageFloats = kSK * kSQS + kSK * kSPS * 2;
    uint64_t* bars = reinterpret_cast<uint64_t*>(gsm + 2 * kStageFloats);
    __shared__ int qb_s[4], pb_s[4];                   // bin bounds met by the two tiles
    __shared__ int qbin0, pbin0, nqbin, npbin;
    int ti, tj;
    tri_index((long long)blockIdx.x, T, ti, tj);
    const bool mirror = tj > ti;
    const int tid = threadIdx.x, tq = tid & 15, tp = tid >> 4;
    const int Q0 = ti * kST, P0 = tj * kST;
    const int nchunks = dpc / kSK;
    const size_t tile_floats = (size_t)dpc * (kSQS + 2 * kSPS);
    const float* tQ = Xtt + (size_t)ti * tile_floats;
    const float* tP = Xtt + (size_t)tj * tile_floats + (size_t)dpc * kSQS;
    constexpr uint32_t kQBytes = kSK * kSQS * 4, kPBytes = kSK * kSPS * 8;
    auto issue = [&](int c, int st) {
        float* dst = gsm + st * kStageFloats;
        mbar_arrive_expect_tx(&bars[st], kQBytes + kPBytes);
        bulk_g2s(dst, tQ + (size_t)c * kSK * kSQS, kQBytes, &bars[st]);
        bulk_g2s(dst + kSK * kSQS, tP + (size_t)c * kSK * kSPS * 2, kPBytes, &bars[st]);
    };
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        issue(0, 0);
        if (nchunks > 1) issue(1, 1);
    }
    if (tid < 4) {  // the bins met by the two tiles (no memory access)
        const int x = tid == 0 ? Q0 : tid == 1 ? P0 : tid == 2 ? min(Q0 + kST, n) - 1 : min(P0 + kST, n) - 1;
        const int b = bin_of(n, s0, x);
        if (tid == 0) qbin0 = b;
        if (tid == 1) pbin0 = b;
        __syncwarp(0xfu);
        if (tid == 2) nqbin = b - qbin0 + 1;
        if (tid == 3) npbin = b - pbin0 + 1;
    }
    __syncthreads();
    if (tid < 4) {
        qb_s[tid] = bnd[min(qbin0 + tid, nb)];
        pb_s[tid] = bnd[min(pbin0 + tid, nb)];
    }
    uint64_t acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0ull;
    for (int c = 0; c < nchunks; ++c) {
        const int st = c & 1;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)(c >> 1) & 1u, status);
        if (__syncthreads_or(!ok)) {  // a copy did not land in time: drain (bounded) and stop
            if (tid == 0) {
                mbar_wait_bounded(&bars[st], (uint32_t)(c >> 1) & 1u, status);
                if (c + 1 < nchunks) mbar_wait_bounded(&bars[st ^ 1], (uint32_t)((c + 1) >> 1) & 1u, status);
            }
            __syncthreads();
            return;
        }
        const float* Qs = gsm + st * kStageFloats;
        accumulate_pairs<2, F>(Qs, Qs + kSK * kSQS, tq, tp, acc);
        __syncthreads();  // stage st is free again
        if (tid == 0 && c + 2 < nchunks) issue(c + 2, st);
    }
    // kernel values of the thread's 8 queries x 8 points
    float kv[8][8];
    const uint64_t nc2 = f2_pack(neg_c, neg_c);
    const bool last = P0 + kST > n;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float2 sv = f2_unpack(f2_mul(fam_fin2<F>(acc[a][b]), nc2));
            const int p = P0 + tile_row(tp, b);
            const int q0 = Q0 + tile_row(tq, 2 * a);
            float k0 = ex2_approx(sv.x), k1 = ex2_approx(sv.y);
            if (last && p >= n) k0 = k1 = 0.f;
            if (self_exclude && !mirror) {
                if (p == q0) k0 = 0.f;
                if (p == q0 + 1) k1 = 0.f;
            }
            kv[2 * a][b] = k0;
            kv[2 * a + 1][b] = k1;
        }
    }
    // the stages are free: they become the partial-sum buffers
    float* rowpart = gsm;                   // [16 tp][128 q][3 point bins]
    float* colpart = gsm + 16 * kST * 3;    // [16 tq][128 p][3 query bins]
    {
        // row partials: a group of 4 consecutive points usually lies in one bin
        int lbp[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int p = P0 + tile_row(tp, b);
            lbp[b] = (p >= pb_s[1]) + (p >= pb_s[2]);
        }
        const bool g0 = lbp[0] == lbp[3], g1 = lbp[4] == lbp[7];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float r3[3] = {0.f, 0.f, 0.f};
            if (g0) {
                add3(r3, lbp[0], (kv[i][0] + kv[i][1]) + (kv[i][2] + kv[i][3]));
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b) add3(r3, lbp[b], kv[i][b]);
            }
            if (g1) {
                add3(r3, lbp[4], (kv[i][4] + kv[i][5]) + (kv[i][6] + kv[i][7]));
            } else {
#pragma unroll
                for (int b = 4; b < 8; ++b) add3(r3, lbp[b], kv[i][b]);
            }
            float* dst = rowpart + (tp * kST + tile_row(tq, i)) * 3;
            dst[0] = r3[0];
            dst[1] = r3[1];
            dst[2] = r3[2];
        }
        if (mirror) {
            // column partials: a group of 4 consecutive queries usually lies in one bin
            int lbq[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = Q0 + tile_row(tq, i);
                lbq[i] = (q >= qb_s[1]) + (q >= qb_s[2]);
            }
            const bool q0u = lbq[0] == lbq[3], q1u = lbq[4] == lbq[7];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                float c3[3] = {0.f, 0.f, 0.f};
                if (q0u) {
                    add3(c3, lbq[0], (kv[0][b] + kv[1][b]) + (kv[2][b] + kv[3][b]));
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) add3(c3, lbq[i], kv[i][b]);
                }
                if (q1u) {
                    add3(c3, lbq[4], (kv[4][b] + kv[5][b]) + (kv[6][b] + kv[7][b]));
                } else {
#pragma unroll
                    for (int i = 4; i < 8; ++i) add3(c3, lbq[i], kv[i][b]);
                }
                float* dst = colpart + (tq * kST + tile_row(tp, b)) * 3;
                dst[0] = c3[0];
                dst[1] = c3[1];
                dst[2] = c3[2];
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kST * 3; e += kGT) {
        const int r = e / 3, b = e - 3 * r;
        if (b < npbin && Q0 + r < n) {
            float s = 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) s += rowpart[(u * kST + r) * 3 + b];
            atomicAdd(&binsum[(size_t)(Q0 + r) * nb + pbin0 + b], s);
        }
        if (mirror && b < nqbin && P0 + r < n) {
            float s = 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) s += colpart[(u * kST + r) * 3 + b];
            atomicAdd(&binsum[(size_t)(P0 + r) * nb + qbin0 + b], s);
        }
    }
}

// Leaf values (d > 16): CTA (b, y) takes item chunks y, y + gridDim.y, ... of
// bin b's segment: 128 items (rows) against the leaf slots of the bin's
// perfect tree (columns, 64 NPG per tile; slots whose node is empty get 0),
// packed as in the symmetric pass; rows of leafv[item][slot] written as float4.
template <int NPG, int F>
__global__ void __launch_bounds__(kGT, 2)
leaf_values_generic_kernel(const float* __restrict__ Xt, int dp, const int32_t* __restrict__ bnd,
                           const int32_t* __restrict__ bin_off, const int32_t* __restrict__ items_q, float neg_c,
                           int self_exclude, int leafmax, float* __restrict__ Vg) {
    extern __shared__ __align__(16) float gsm[];
    float* Qs = gsm;
    float* Ps = gsm + kSK * kSQS;
    __shared__ int qrow[kST], prow[kST];
    const int tid = threadIdx.x, tq = tid & 15, tp = tid >> 4;
    const int b = blockIdx.x;
    const int seg = bin_off[b * kBinSlots];
    const int cnt = bin_off[(b + 1) * kBinSlots] - seg;
    const int nchunks = (cnt + kST - 1) / kST;
    if ((int)blockIdx.y >= nchunks) return;
    const int p_lo = bnd[b], m = bnd[b + 1] - p_lo;
    const int dm = ceil_log2_dev(m), leaf0 = 1 << dm;
    const uint64_t nc2 = f2_pack(neg_c, neg_c);
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int it0 = chunk * kST;
        const int qcnt = min(kST, cnt - it0);
        for (int s0 = 0; s0 < leaf0; s0 += 64 * NPG) {
            __syncthreads();
            if (tid < kST) {
                qrow[tid] = tid < qcnt ? items_q[seg + it0 + tid] : -1;
                const int sl = s0 + tid;
                int pos = -1;
                if (tid < 64 * NPG && sl < leaf0) {
                    int a = 0, c = m;
                    for (int t = dm - 1; t >= 0; --t) {
                        const int mid = a + (c - a) / 2;
                        if ((sl >> t) & 1) a = mid; else c = mid;
                    }
                    if (c - a == 1) pos = p_lo + a;
                }
                prow[tid] = pos;
            }
            uint64_t acc[4][4 * NPG];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4 * NPG; ++c) acc[a][c] = 0ull;
            for (int k0 = 0; k0 < dp; k0 += kSK) {
                __syncthreads();
                load_tiles(Qs, Ps, [&](int r) { return qrow[r]; }, [&](int r) { return prow[r]; }, Xt, dp, k0, 0.f);
                __syncthreads();
                accumulate_pairs<NPG, F>(Qs, Ps, tq, tp, acc);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float o[2][4 * NPG];
#pragma unroll
                for (int c = 0; c < 4 * NPG; ++c) {
                    const float2 sv = f2_unpack(f2_mul(fam_fin2<F>(acc[a][c]), nc2));
                    const int pp = prow[tile_row(tp, c)];
                    float k0 = pp >= 0 ? ex2_approx(sv.x) : 0.f, k1 = pp >= 0 ? ex2_approx(sv.y) : 0.f;
                    if (self_exclude) {
                        if (pp == qrow[tile_row(tq, 2 * a)]) k0 = 0.f;
                        if (pp == qrow[tile_row(tq, 2 * a) + 1]) k1 = 0.f;
                    }
                    o[0][c] = k0;
                    o[1][c] = k1;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int rr = tile_row(tq, 2 * a) + h;
                    if (rr >= qcnt) continue;
                    float* dst = Vg + (size_t)(seg + it0 + rr) * leafmax + s0;
#pragma unroll
                    for (int g = 0; g < NPG; ++g) {
                        const int sl = 64 * g + 4 * tp;
                        if (leaf0 >= 4) {
                            if (s0 + sl < leaf0)
                                *reinterpret_cast<float4*>(dst + sl) =
                                    make_float4(o[h][4 * g], o[h][4 * g + 1], o[h][4 * g + 2], o[h][4 * g + 3]);
                        } else {  // rows of 1 or 2 slots
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if (s0 + sl + c < leaf0) dst[sl + c] = o[h][4 * g + c];
                        }
                    }
                }
            }
        }
    }
}

}  // namespace

bool kde_bins_generic_sym_supported(const fsg_tree* t) {
    return t->d > kMaxFmaDim && t->mmax <= kST && t->Xtt != nullptr;
}

// Bytes of the transposed tiles of a tree of n points of dimension d.
size_t generic_tile_bytes(int64_t n, int32_t d) {
    const int64_t T = (n + kST - 1) / kST;
    const int64_t dpc = ((d + 3) / 4 * 4 + kSK - 1) / kSK * kSK;
    return sizeof(float) * (size_t)T * (size_t)dpc * (kSQS + 2 * kSPS);
}

// Evaluations executed by the symmetric generic pass: the triangle of tiles.
int64_t kde_bins_generic_sym_evals(const fsg_tree* t) {
    const int64_t T = (t->n + kST - 1) / kST;
    return T * (T + 1) / 2 * kST * kST;
}

namespace {
template <int F>
cudaError_t launch_generic_f(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    if (kde_bins_generic_sym_supported(t)) {
        const size_t smem = 2 * kSymGenSmem + 2 * sizeof(uint64_t);  // two stages and their mbarriers
        {
            const cudaError_t e = set_smem_limit(kde_bins_generic_sym_kernel<F>, (int)smem);
            if (e != cudaSuccess) return e;
        }
        const int64_t T = (t->n + kST - 1) / kST;
        const int dpc = (t->dp + kSK - 1) / kSK * kSK;
        dim3 pg((unsigned)T, (unsigned)(dpc / kSK));
        generic_tiles_kernel<<<pg, kGT, 0, s>>>(t->Xt, (int)t->n, t->d, t->dp, dpc, t->Xtt);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemsetAsync(t->ws.binsum, 0, sizeof(float) * (size_t)t->n * t->nb, s);
        if (e != cudaSuccess) return e;
        const int64_t ctas = T * (T + 1) / 2;
        if (ctas > INT_MAX) return cudaErrorInvalidValue;
        kde_bins_generic_sym_kernel<F><<<(unsigned)ctas, kGT, smem, s>>>(t->Xtt, (int)t->n, dpc, t->bnd, t->nb,
                                                                       t->s0, (int)T, kp.neg_c, kp.self_exclude,
                                                                       t->ws.binsum, t->status);
        return cudaGetLastError();
    }
    const int qblocks = (int)((t->n + kGQ - 1) / kGQ);
    int chunks = (2048 + qblocks - 1) / qblocks;
    if (chunks < 1) chunks = 1;
    if (chunks > t->nb) chunks = t->nb;
    int bpc = (t->nb + chunks - 1) / chunks;
    if (bpc > 8) bpc = 8;
    chunks = (t->nb + bpc - 1) / bpc;
    dim3 grid(qblocks, chunks);
    kde_bins_generic_kernel<F><<<grid, kGT, (size_t)kGQ * bpc * 4, s>>>(t->Xt, (int)t->n, t->d, t->dp, t->bnd, t->nb,
                                                                       bpc, kp.neg_c, kp.self_exclude,
                                                                       t->ws.binsum);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_kde_bins_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    switch (kp.family) {
        case kFamLaplace: return launch_generic_f<kFamLaplace>(t, kp, s);
        case kFamExp: return launch_generic_f<kFamExp>(t, kp, s);
        default: return launch_generic_f<kFamGauss>(t, kp, s);
    }
}

namespace {

// Fused leaf phase for d > 16 and bins of at most 128 points: per chunk of
// 128 items of a bin, the kernel values against the bin's m points (compact:
// column j = point p_lo + j) in the packed 128 x 128 tile of the bin pass,
// kept in shared memory (over the coordinate tiles, which are idle by then);
// then the 16 depth-4 node sums of every item (two threads per item) and
// their tree; then every sample of the chunk's items, spread over all threads,
// descends through the bin (descend_bin_row).  No value goes to HBM.
constexpr int kLfVS = kST + 1;  // value row stride (odd)
constexpr size_t kLfU = (size_t)kST * kLfVS * 4 > kSymGenSmem ? (size_t)kST * kLfVS * 4 : kSymGenSmem;
constexpr size_t kLfBT = kLfU;                          // [128][33] depth-4 node sums and their tree
constexpr size_t kLfMask = kLfBT + (size_t)kST * 33 * 4;  // [128] sample masks
constexpr size_t kLfPre = kLfMask + (size_t)kST * 8;      // [129] samples before item r
constexpr size_t kLfB4 = kLfPre + 132 * 4;                // [17] depth-4 node starts
constexpr size_t kLfSmem = kLfB4 + 20 * 4;

template <int F>
__global__ void __launch_bounds__(kGT, 2)
leaf_fused_generic_kernel(const float* __restrict__ Xt, int dp, const int32_t* __restrict__ bnd, int s0,
                          const int32_t* __restrict__ bin_off, const int32_t* __restrict__ items_q,
                          const uint64_t* __restrict__ items_mask, const int32_t* __restrict__ perm, KernelParams kp,
                          int32_t* __restrict__ leaf_pos, float* __restrict__ ksmp, uint8_t* __restrict__ lflags,
                          unsigned long long* __restrict__ n_evals, unsigned long long* __restrict__ n_items) {
    extern __shared__ __align__(16) float gsm[];
    float* Qs = gsm;
    float* Ps = gsm + kSK * kSQS;
    float* V = gsm;  // after the coordinate loop
    unsigned char* sb = reinterpret_cast<unsigned char*>(gsm);
    float* bt_all = reinterpret_cast<float*>(sb + kLfBT);
    uint64_t* qmask = reinterpret_cast<uint64_t*>(sb + kLfMask);
    int32_t* prefix = reinterpret_cast<int32_t*>(sb + kLfPre);
    int32_t* bnd4 = reinterpret_cast<int32_t*>(sb + kLfB4);
    __shared__ int qrow[kST], prow[kST];
    const int tid = threadIdx.x, tq = tid & 15, tp = tid >> 4;
    const int b = blockIdx.x;
    const int seg = bin_off[b * kBinSlots];
    const int cnt = bin_off[(b + 1) * kBinSlots] - seg;
    const int nchunks = (cnt + kST - 1) / kST;
    if ((int)blockIdx.y >= nchunks) return;
    const int p_lo = bnd[b], m = bnd[b + 1] - p_lo;  // m <= 128
    const int dm = ceil_log2_dev(m);
    const uint64_t nc2 = f2_pack(kp.neg_c, kp.neg_c);
    if (tid < kST) prow[tid] = tid < m ? p_lo + tid : -1;
    if (tid <= 16) bnd4[tid] = depth4_start(tid, m);
    unsigned long long ev_acc = 0, it_acc = 0;
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int it0 = chunk * kST;
        const int qcnt = min(kST, cnt - it0);
        __syncthreads();  // the previous chunk's descents are done with V, qmask and prefix
        if (tid < kST) {
            qrow[tid] = tid < qcnt ? items_q[seg + it0 + tid] : -1;
            qmask[tid] = tid < qcnt ? items_mask[seg + it0 + tid] : 0ull;
        }
        uint64_t acc[4][8];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[a][c] = 0ull;
        for (int k0 = 0; k0 < dp; k0 += kSK) {
            __syncthreads();
            load_tiles(Qs, Ps, [&](int r) { return qrow[r]; }, [&](int r) { return prow[r]; }, Xt, dp, k0, 0.f);
            __syncthreads();
            accumulate_pairs<2, F>(Qs, Ps, tq, tp, acc);
        }
        __syncthreads();  // every thread is done with Qs and Ps: V takes their place
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int col = tile_row(tp, c);
                const int pp = prow[col];
                const float2 sv = f2_unpack(f2_mul(fam_fin2<F>(acc[a][c]), nc2));
                const int r0 = tile_row(tq, 2 * a);
                float k0v = pp >= 0 ? ex2_approx(sv.x) : 0.f, k1v = pp >= 0 ? ex2_approx(sv.y) : 0.f;
                if (kp.self_exclude) {
                    if (pp == qrow[r0]) k0v = 0.f;
                    if (pp == qrow[r0 + 1]) k1v = 0.f;
                }
                V[r0 * kLfVS + col] = k0v;
                V[(r0 + 1) * kLfVS + col] = k1v;
            }
        }
        // samples of the chunk's items: prefix[r] = samples of items < r
        if (tid < kST) {
            int x = __popcll(qmask[tid]);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if ((tid & 31) >= o) x += y;
            }
            prefix[tid + 1] = x;  // inclusive within the warp
        }
        __syncthreads();
        // depth-4 node sums: item r = tid % 128, nodes 8 hh .. 8 hh + 7
        {
            const int r = tid & (kST - 1), hh = tid >> 7;
            const float* vr = V + r * kLfVS;
            float* bt = bt_all + r * 33;
            for (int k = 8 * hh; k < 8 * hh + 8; ++k) {
                float sacc = 0.f;
                for (int j = bnd4[k]; j < bnd4[k + 1]; ++j) sacc += vr[j];
                bt[16 + k] = sacc;
            }
        }
        if (tid == 0) {  // warp totals into the prefix
            prefix[0] = 0;
            for (int w2 = 1; w2 < 4; ++w2) {
                const int add = prefix[32 * w2];
                for (int i = 32 * w2 + 1; i <= 32 * w2 + 32; ++i) prefix[i] += add;
            }
        }
        __syncthreads();
        if (tid < kST) {
            float* bt = bt_all + tid * 33;
#pragma unroll
            for (int h = 15; h >= 1; --h) bt[h] = bt[2 * h] + bt[2 * h + 1];
        }
        __syncthreads();
        const int total = prefix[kST];
        for (int gsm_i = tid; gsm_i < total; gsm_i += kGT) {
            int lo = 0, hi = kST;  // item: prefix[lo] <= gsm_i < prefix[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (prefix[mid] <= gsm_i) lo = mid; else hi = mid;
            }
            uint64_t mk = qmask[lo];
            for (int k = gsm_i - prefix[lo]; k > 0; --k) mk &= mk - 1ull;
            const int l = __ffsll((long long)mk) - 1;
            const int ip = qrow[lo];
            const float* vi = V + lo * kLfVS;
            uint8_t f = 0;
            const int a = descend_bin_row(vi, bt_all + lo * 33, m, dm, s0, kp.seed, (uint32_t)perm[ip], (uint32_t)l,
                                          kp.flag_eps, f);
            const size_t o = (size_t)ip * kp.L + l;
            leaf_pos[o] = p_lo + a;
            ksmp[o] = vi[a];
            lflags[o] = f;
        }
        ev_acc += (unsigned long long)qcnt * (unsigned long long)m;
        it_acc += (unsigned long long)qcnt;
    }
    if (tid == 0) {
        atomicAdd(n_evals, ev_acc);
        atomicAdd(n_items, it_acc);
    }
}

}  // namespace

bool leaf_fused_generic_supported(const fsg_tree* t) { return t->d > kMaxFmaDim && t->mmax <= kST; }

cudaError_t launch_leaf_fused_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const int64_t items_est = t->n * (int64_t)(kp.L < t->nb ? kp.L : t->nb);
    const int64_t chunks_per_bin = (items_est / t->nb + kST - 1) / kST + 1;
    int64_t S = (152 * 2 * 8 + t->nb - 1) / t->nb;
    if (S > chunks_per_bin) S = chunks_per_bin;
    if (t->tune.leaf_splits > 0) S = t->tune.leaf_splits;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    auto kern = kp.family == kFamLaplace ? leaf_fused_generic_kernel<kFamLaplace>
                : kp.family == kFamExp     ? leaf_fused_generic_kernel<kFamExp>
                                           : leaf_fused_generic_kernel<kFamGauss>;
    {
        const cudaError_t e = set_smem_limit(kern, (int)kLfSmem);
        if (e != cudaSuccess) return e;
    }
    const auto& ws = t->ws;
    kern<<<dim3(t->nb, (unsigned)S), kGT, kLfSmem, s>>>(
        t->Xt, t->dp, t->bnd, t->s0, ws.bin_off, ws.items_q, ws.items_mask, t->perm, kp, ws.leaf_pos, ws.ksmp,
        ws.lflags, reinterpret_cast<unsigned long long*>(&ws.stats->n_evals),
        reinterpret_cast<unsigned long long*>(&ws.stats->n_items));
    return cudaGetLastError();
}

cudaError_t launch_leaf_values_generic(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const int64_t items_est = t->n * (int64_t)(kp.L < t->nb ? kp.L : t->nb);
    const int64_t chunks_per_bin = (items_est / t->nb + kST - 1) / kST + 1;
    int64_t S = (152 * 2 * 8 + t->nb - 1) / t->nb;
    if (S > chunks_per_bin) S = chunks_per_bin;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    dim3 grid(t->nb, (unsigned)S);
    const bool wide = (1 << t->dm) > 64;
    using K = void (*)(const float*, int, const int32_t*, const int32_t*, const int32_t*, float, int, int, float*);
    const K kern = kp.family == kFamLaplace ? (wide ? (K)leaf_values_generic_kernel<2, kFamLaplace>
                                                    : (K)leaf_values_generic_kernel<1, kFamLaplace>)
                   : kp.family == kFamExp   ? (wide ? (K)leaf_values_generic_kernel<2, kFamExp>
                                                    : (K)leaf_values_generic_kernel<1, kFamExp>)
                                            : (wide ? (K)leaf_values_generic_kernel<2, kFamGauss>
                                                    : (K)leaf_values_generic_kernel<1, kFamGauss>);
    {
        const cudaError_t e = set_smem_limit(kern, kSymGenSmem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kGT, kSymGenSmem, s>>>(t->Xt, t->dp, t->bnd, t->ws.bin_off, t->ws.items_q, kp.neg_c,
                                        kp.self_exclude, 1 << t->dm, t->ws.leafv);
    return cudaGetLastError();
}

}  // namespace fsg
