// Split-precision tensor-core bin pass (FSG_PREC_SPLIT_BF16) for FP32 data,
// d <= 64: the bin sums of Eq. 1 for every query, like the other bin passes,
// with the dot products on the tensor cores.
//
// CTA = one tile of 128 queries (128 consecutive tree positions) x one chunk
// of bins.  Both operands are centred at the query tile's centre c (the mean
// of its points): a = x - c, b = y - c.  Under a spatial tree order
// (fsg_spatial_order) a tile is a compact group, the centred norms are small
// next to the data's spread, and ||x - y||^2 = ||a||^2 + ||b||^2 - 2 a.b loses
// little to cancellation.  Each centred FP32 coordinate is split into three
// BF16 parts, v = hi + mid + lo, each part the BF16 rounding of what the
// previous ones leave (the residuals are exact in FP32; the three parts hold
// 24 significand bits), and a.b is accumulated in FP32 in TMEM as six
// products per coordinate,
//   lo.hi + hi.lo + mid.mid + mid.hi + hi.mid + hi.hi
// (small terms first; mid.lo, lo.mid and lo.lo lie below 2^-24 relative).
// Every BF16 x BF16 product is exact in FP32.
//
// The query side does not depend on the bin chunk: split_prep_kernel writes
// each query tile's parts, centred norms and centre once per launch, and
// every CTA of that tile bulk-copies the image (49,920 bytes).
//
// Warp roles (13 warps):
//   warps 0-3 : producers: per tile of 128 points the centred, split point
//               parts and their norms, two stages (shared-memory stores, a
//               proxy fence, an mbarrier arrive per thread);
//   warp 4    : TMEM allocation; one thread issues the 6 x ceil(d / 16)
//               tcgen05.mma (K = 16; 24 at d > 48)
//               of a tile into one of two 128-column accumulators;
//   warps 5-12: epilogue, two per TMEM lane quadrant (one per half of the 128
//               columns): kernel values and bin sums, as in the 8-bit pass.
// Every mbarrier wait is bounded; on a timeout the CTA records
// FSG_ERR_TIMEOUT, stops, waits (bounded) for its own MMAs and frees TMEM.
#include <cuda_bf16.h>

#include <cmath>

#include "fsg_tc.cuh"

namespace fsg {
namespace {

constexpr int kSpM = 128;             // queries per tile
constexpr int kSpN = 128;             // points per tile
constexpr int kSpDim = 64;            // coordinates (d <= 64, zero-padded)
constexpr int kSpStages = 2;
constexpr int kSpParts = 3;           // hi, mid, lo
constexpr int kSpEpiWarps = 8;
constexpr int kSpThreads = 32 * (5 + kSpEpiWarps);
constexpr int kSpMaxBins = 48;        // bins per chunk
constexpr uint32_t kPart = 128u * 128u;  // one part of 128 rows x 64 BF16 (128-byte swizzled rows)
constexpr uint32_t kTmemCols = 256;   // two 128-column accumulators
constexpr int kSpMaxTiles = 252;      // point tiles per CTA (kept list)
// A query tile's image, written once per launch by split_prep_kernel and
// bulk-copied by every CTA of that tile: its three swizzled parts, then the
// centred norms of its 128 rows, then its centre.
constexpr uint32_t kQImg = kSpParts * kPart + kSpM * 4 + kSpDim * 4;
// log2 of "no lower bound" / "no approximation budget": far below any
// log2(count) + neg_c * gap^2 that is not already an exact zero (> -128 - 8)
constexpr float kNoBound = -1.0e30f;

// The split form's per-tree workspace: bin boxes [nb][128], query-tile boxes
// [qblocks][128], the query tiles' degree lower bounds (log2) [qblocks, padded
// to 128], the query tiles' images, then the bins' images.  Every array starts
// 16-byte aligned (the float arrays are multiples of 512 bytes, an image
// 49,920 bytes).
struct SplitWs {
    float* bin_boxes;
    float* tile_boxes;
    float* tile_lb;
    unsigned char* tile_img;
    unsigned char* bin_img;
    int64_t qblocks;
    __host__ SplitWs(const fsg_tree* t) {
        qblocks = (t->n + kSpM - 1) / kSpM;
        bin_boxes = t->sboxes;
        tile_boxes = bin_boxes + (size_t)t->nb * 128;
        tile_lb = tile_boxes + (size_t)qblocks * 128;
        tile_img = reinterpret_cast<unsigned char*>(tile_lb + (size_t)(qblocks + 127) / 128 * 128);
        bin_img = tile_img + (size_t)qblocks * kQImg;
    }
};

struct SpLayout {
    static constexpr uint32_t A = 0;                                      // [3][128 rows]
    static constexpr uint32_t B = A + kSpParts * kPart;                   // [stages][3][128 rows]
    static constexpr uint32_t CN = B + kSpStages * kSpParts * kPart;      // [stages][128] point norms
    static constexpr uint32_t AN = CN + kSpStages * kSpN * 4;             // [128] query norms
    static constexpr uint32_t CEN = AN + kSpM * 4;                        // [64] centre
    static constexpr uint32_t BARS = CEN + kSpDim * 4;                    // full[2] empty[2] tfull[2] tempty[2] fin qbar
    static constexpr uint32_t SLOT = BARS + (2 * kSpStages + 6) * 8;      // TMEM slot, abort flag
    static constexpr uint32_t BND = SLOT + 16;                            // [kSpMaxBins + 1]
    static constexpr uint32_t QLO = (BND + (kSpMaxBins + 1) * 4 + 15) & ~15u;  // [64] query tile's box: low corner
    static constexpr uint32_t QHI = QLO + kSpDim * 4;                     // [64] high corner
    static constexpr uint32_t TL = QHI + kSpDim * 4;                      // [kSpMaxTiles] kept point tiles, count
    static constexpr uint32_t PN = TL + (kSpMaxTiles + 4) * 4;            // [8 warps][64] norms of a warp's columns
    static constexpr uint32_t OUTS = PN + kSpEpiWarps * 64 * 4;           // [2 halves][128][bpc]
    static constexpr uint32_t total(int bpc) { return OUTS + 2u * kSpM * (uint32_t)bpc * 4u; }
};
static_assert(SpLayout::BARS % 8 == 0 && SpLayout::PN % 16 == 0 && SpLayout::B % 1024 == 0, "layout");
static_assert(1024 + SpLayout::total(kSpMaxBins) <= 227 * 1024, "shared memory of a full chunk");
static_assert(SpLayout::AN == SpLayout::CN + kSpStages * kSpN * 4 && SpLayout::CEN == SpLayout::AN + kSpM * 4 &&
                  SpLayout::AN % 16 == 0 && kQImg % 16 == 0,
              "the query image's norms and centre land in AN and CEN by 16-byte bulk copies");

// Three BF16 parts of two values, packed (low half = a, high half = b): each
// part the BF16 rounding of what the previous parts leave (exact residuals).
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    const float ra = __fsub_rn(a, __uint_as_float(hi << 16)), rb = __fsub_rn(b, __uint_as_float(hi & 0xffff0000u));
    const __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
    mid = *reinterpret_cast<const uint32_t*>(&m);
    const float sa = __fsub_rn(ra, __uint_as_float(mid << 16)), sb = __fsub_rn(rb, __uint_as_float(mid & 0xffff0000u));
    const __nv_bfloat162 l = __floats2bfloat162_rn(sa, sb);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// One operand row's coordinates (tree position p, zeros for p < 0).
__device__ __forceinline__ void load_row(const float* __restrict__ Xt, int dp, int p, float4 (&x)[kSpDim / 4]) {
#pragma unroll
    for (int u = 0; u < kSpDim / 4; ++u)
        x[u] = (p >= 0 && 4 * u < dp) ? *reinterpret_cast<const float4*>(Xt + (size_t)p * dp + 4 * u)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The row centred, split and stored as three 128-byte swizzled rows at
// parts + part * kPart; returns its squared norm.  A point's coordinates past
// d are zero, as are the centre's, so they stay zero; `valid` = false (no
// point) stores zero rows.  Only the first nch 16-byte chunks (coordinates
// 0 .. 8 nch - 1) are written: the caller keeps the others zero.
__device__ __forceinline__ float split_row(const float4 (&x)[kSpDim / 4], bool valid, const float* __restrict__ cen,
                                           unsigned char* parts, int row, int nch = 8) {
    float norm = 0.f;
    if (!valid) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k >= nch) break;
            const uint32_t off = (uint32_t)row * 128u + (uint32_t)((k ^ (row & 7)) << 4);
            *reinterpret_cast<uint4*>(parts + off) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(parts + kPart + off) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(parts + 2 * kPart + off) = make_uint4(0u, 0u, 0u, 0u);
        }
        return 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {  // 16-byte chunk k = coordinates 8k .. 8k + 7
        if (k >= nch) break;
        const float v[8] = {x[2 * k].x, x[2 * k].y, x[2 * k].z, x[2 * k].w,
                            x[2 * k + 1].x, x[2 * k + 1].y, x[2 * k + 1].z, x[2 * k + 1].w};
        float a[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            a[i] = __fsub_rn(v[i], cen[8 * k + i]);
            norm = __fmaf_rn(a[i], a[i], norm);
        }
        uint4 hi, mid, lo;
        split2(a[0], a[1], hi.x, mid.x, lo.x);
        split2(a[2], a[3], hi.y, mid.y, lo.y);
        split2(a[4], a[5], hi.z, mid.z, lo.z);
        split2(a[6], a[7], hi.w, mid.w, lo.w);
        const uint32_t off = (uint32_t)row * 128u + (uint32_t)((k ^ (row & 7)) << 4);
        *reinterpret_cast<uint4*>(parts + off) = hi;
        *reinterpret_cast<uint4*>(parts + kPart + off) = mid;
        *reinterpret_cast<uint4*>(parts + 2 * kPart + off) = lo;
    }
    return norm;
}

__global__ void __launch_bounds__(kSpThreads, 1)
kde_bins_split_kernel(const float* __restrict__ Xt, int dp, int d, int n, const int32_t* __restrict__ bnd, int nb,
                      int bpc, float neg_c, int self_exclude, const float* __restrict__ boxes,
                      const float* __restrict__ qboxes, const unsigned char* __restrict__ qimg,
                      const float* __restrict__ tile_lb, float log2_budget,
                      float* __restrict__ binsum, unsigned long long* __restrict__ n_evals,
                      unsigned long long* __restrict__ n_bin_evals, int32_t* __restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_align1024(smem_raw);
    unsigned char* sA = base + SpLayout::A;
    unsigned char* sB = base + SpLayout::B;
    float* cn = reinterpret_cast<float*>(base + SpLayout::CN);
    float* an = reinterpret_cast<float*>(base + SpLayout::AN);
    float* cen = reinterpret_cast<float*>(base + SpLayout::CEN);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + SpLayout::BARS);
    uint64_t* empty = full + kSpStages;
    uint64_t* tfull = empty + kSpStages;
    uint64_t* tempty = tfull + 2;
    uint64_t* fin = tempty + 2;
    uint64_t* qbar = fin + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + SpLayout::SLOT);
    volatile int32_t* abort_flag = reinterpret_cast<int32_t*>(base + SpLayout::SLOT + 4);
    int32_t* bnd_s = reinterpret_cast<int32_t*>(base + SpLayout::BND);
    float* pn_all = reinterpret_cast<float*>(base + SpLayout::PN);
    float* qlo = reinterpret_cast<float*>(base + SpLayout::QLO);
    float* qhi = reinterpret_cast<float*>(base + SpLayout::QHI);
    int32_t* tl = reinterpret_cast<int32_t*>(base + SpLayout::TL);  // kept tiles; tl[kSpMaxTiles] = their count
    float* outs = reinterpret_cast<float*>(base + SpLayout::OUTS);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * kSpM;
    const int b0 = blockIdx.y * bpc;
    const int nbc = min(nb, b0 + bpc) - b0;
    const int nqv = min(kSpM, n - q0);  // queries of this tile
    if (tid <= nbc) bnd_s[tid] = bnd[b0 + tid];
    if (tid < kSpDim) {  // the query tile's bounding box
        qlo[tid] = qboxes[(size_t)blockIdx.x * 128 + tid];
        qhi[tid] = qboxes[(size_t)blockIdx.x * 128 + 64 + tid];
    }
    __syncthreads();
    const int pa = bnd_s[0], pe = bnd_s[nbc];
    const int ntall = (pe - pa + kSpN - 1) / kSpN;
    // approximate bin pass: a tile whose bound count * 2^(neg_c gap^2) is at
    // most 2^thr (= kde_eps / T of the query tile's degree lower bound) is
    // skipped; exact pass (log2_budget = kNoBound): thr is about kNoBound
    const float thr = log2_budget + tile_lb[blockIdx.x];
    // Point tiles whose every kernel value is exactly zero in FP32 are skipped:
    // when the gap between the query tile's box and the union of the boxes of
    // the tile's bins puts neg_c * d^2 below -128, every ex2 is below 2^-126
    // and flushes to +0 (two units of margin over the rounding of d^2), so the
    // bin sums are the same bit for bit.  With kde_eps > 0 so are the tiles
    // whose whole contribution is bounded by the approximation's budget.
    // The chunk's bin boxes are staged in
    // the (not yet used) output buffer; warp w tests tiles w, w + 13, ... with
    // its lanes over the coordinates; warp 0 lists the kept tiles in order.
    float* bx = outs;  // [nbc][128]: low corner, high corner
    for (int e = tid; e < nbc * 128; e += kSpThreads) bx[e] = boxes[(size_t)b0 * 128 + e];
    __syncthreads();
    for (int t = warp; t < ntall; t += kSpThreads / 32) {
        const int ps = pa + t * kSpN, pq = min(pe, ps + kSpN);
        int bf = 0;  // the tile's bins are bf .. bl (consecutive)
        while (bf + 1 < nbc && bnd_s[bf + 1] <= ps) ++bf;
        int bl = bf;
        while (bl + 1 < nbc && bnd_s[bl + 1] < pq) ++bl;
        float d2 = 0.f;
        for (int c = lane; c < d; c += 32) {
            float lo = bx[bf * 128 + c], hi = bx[bf * 128 + 64 + c];
            for (int b = bf + 1; b <= bl; ++b) {
                lo = fminf(lo, bx[b * 128 + c]);
                hi = fmaxf(hi, bx[b * 128 + 64 + c]);
            }
            const float gap = fmaxf(0.f, fmaxf(lo - qhi[c], qlo[c] - hi));
            d2 = fmaf(gap, gap, d2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        const float lg = neg_c * d2;
        if (lane == 0 && t < kSpMaxTiles)  // keep flag, compacted below
            tl[t] = !(lg < -128.f || lg + __log2f((float)(pq - ps)) <= thr);
    }
    __syncthreads();
    if (warp == 0) {
        int kept = 0;
        for (int t0 = 0; t0 < ntall; t0 += 32) {
            const int t = t0 + lane;
            const bool keep = t < ntall && tl[t] != 0;
            const uint32_t bal = __ballot_sync(0xffffffffu, keep);
            __syncwarp();  // every lane has read its flag before any is overwritten
            if (keep) tl[kept + __popc(bal & ((1u << lane) - 1u))] = t;
            kept += __popc(bal);
            __syncwarp();
        }
        if (lane == 0) tl[kSpMaxTiles] = kept;
    }
    __syncthreads();
    const int ntile = tl[kSpMaxTiles];  // tiles processed (the list's order is the tiles' order)
    if (ntile == 0) {  // every value of this CTA is zero: its bin sums are 0, nothing else to do
        for (int e = tid; e < nqv * nbc; e += kSpThreads) {
            const int ql = e / nbc, b = e - ql * nbc;
            binsum[(size_t)(q0 + ql) * nb + b0 + b] = 0.f;
        }
        return;
    }
    for (int e = tid; e < 2 * kSpM * bpc; e += kSpThreads) outs[e] = 0.f;
    // Coordinates past d are zero in every part: the producers write the first
    // nch 16-byte chunks of a row, the rest of the point stages is cleared
    // once here, and the MMAs run only the kk K-steps of 16 that hold data.
    const int nch = (d + 7) / 8, kk = (d + 15) / 16;
    if (nch < 8) {
        for (int e = tid; e < (int)(kSpStages * kSpParts * kPart / 16); e += kSpThreads)
            reinterpret_cast<uint4*>(sB)[e] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kSpStages; ++s) {
            mbar_init(&full[s], 128);                // the producers' arrivals
            mbar_init(&empty[s], 1 + kSpEpiWarps);   // MMA commit + the epilogue warps (point norms read)
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 32 * kSpEpiWarps);
        }
        mbar_init(fin, 1);
        mbar_init(qbar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the query tile's parts, norms and centre: one image, bulk-copied
    if (tid == 0) {
        const unsigned char* src = qimg + (size_t)blockIdx.x * kQImg;
        mbar_arrive_expect_tx(qbar, kQImg);
        bulk_g2s(sA, src, kSpParts * kPart, qbar);
        bulk_g2s(an, src + kSpParts * kPart, kSpM * 4, qbar);
        bulk_g2s(cen, src + kSpParts * kPart + kSpM * 4, kSpDim * 4, qbar);
    }
    const bool qready = mbar_wait_bounded(qbar, 0u, status);
    if (!qready) *abort_flag = 1;
    __syncthreads();
    int mma_issued = 0;

    if (warp < 4) {
        // ---- producers: point tile t into stage t % 2; the next tile's row is
        // loaded while this thread waits for its stage to be free
        float4 x[kSpDim / 4];
        int p = ntile > 0 ? pa + tl[0] * kSpN + tid : pe;
        load_row(Xt, dp, p < pe ? p : -1, x);
        for (int t = 0; t < ntile && !*abort_flag; ++t) {
            const int s = t % kSpStages;
            if (!mbar_wait_bounded(&empty[s], ((uint32_t)(t / kSpStages) & 1u) ^ 1u, status)) {
                *abort_flag = 1;
                break;
            }
            cn[s * kSpN + tid] = split_row(x, p < pe, cen, sB + (uint32_t)s * kSpParts * kPart, tid, nch);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
            if (t + 1 < ntile) {
                p = pa + tl[t + 1] * kSpN + tid;
                load_row(Xt, dp, p < pe ? p : -1, x);
            }
        }
    } else if (warp == 4) {
        if (lane == 0) {
            // ---- MMA issuer: six products per coordinate, small terms first
            const int pi[6] = {2, 0, 1, 1, 0, 0};  // A part (0 hi, 1 mid, 2 lo)
            const int pj[6] = {0, 2, 1, 0, 1, 0};  // B part
            const uint32_t idesc = idesc_bf16(kSpM, kSpN);
            for (int t = 0; t < ntile && !*abort_flag; ++t) {
                const int a = t & 1, s = t % kSpStages;
                if (!mbar_wait_bounded(&tempty[a], ((uint32_t)(t >> 1) & 1u) ^ 1u, status) ||
                    !mbar_wait_bounded(&full[s], (uint32_t)(t / kSpStages) & 1u, status)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(a * kSpN);
#pragma unroll
                for (int u = 0; u < 6; ++u) {
                    const uint64_t da = sdesc(smem_u32(sA + pi[u] * kPart));
                    const uint64_t db = sdesc(smem_u32(sB + (uint32_t)s * kSpParts * kPart + pj[u] * kPart));
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // 32 bytes of K per MMA inside the swizzled row
                        if (k >= kk) break;
                        umma_bf16(dt, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (u | k) != 0 ? 1u : 0u);
                    }
                }
                mma_issued = 1;
                umma_commit(&empty[s]);
                umma_commit(&tfull[a]);
            }
        }
    } else {
        // ---- epilogue: TMEM lane quadrant (warp % 4), row = query; column half (warp - 5) / 4
        constexpr int kCols = kSpN / 2;
        const int ew = warp - 5;
        const int quad = warp & 3;
        const int half = ew >> 2;
        const int r = 32 * quad + lane;
        const int q = q0 + r;
        const float nq = an[r];
        float* pn = pn_all + ew * kCols;
        float* orow = outs + (half * kSpM + r) * bpc;  // partial sums of this column half
        int bin = 0;
        int next_b = nbc > 0 ? bnd_s[1] : INT_MAX;
        for (int t = 0; t < ntile; ++t) {
            const int a = t & 1, s = t % kSpStages;
            if (*abort_flag || !mbar_wait_bounded(&tfull[a], (uint32_t)(t >> 1) & 1u, status) ||
                !mbar_wait_bounded(&full[s], (uint32_t)(t / kSpStages) & 1u, status)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int c0 = pa + tl[t] * kSpN + half * kCols;  // first point of this warp's columns
            __syncwarp();
            pn[lane] = cn[s * kSpN + half * kCols + lane];
            pn[lane + 32] = cn[s * kSpN + half * kCols + lane + 32];
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // this stage's point norms are read
            while (next_b <= c0) {  // bins that ended in the other half
                ++bin;
                next_b = bin < nbc ? bnd_s[bin + 1] : INT_MAX;
            }
            const bool check = c0 + kCols > pe || (self_exclude && c0 < q0 + kSpM && q0 < c0 + kCols);
            float acc = 0.f;
            const uint32_t tcol = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(a * kSpN + half * kCols);
            uint32_t rb[2][32];
            tmem_issue32(tcol, rb[0]);
#pragma unroll
            for (int cc = 0; cc < kCols; cc += 32) {
                const int cur = (cc >> 5) & 1;
                tmem_wait32(rb[cur]);  // the only load in flight
                if (cc + 32 < kCols) tmem_issue32(tcol + (uint32_t)(cc + 32), rb[cur ^ 1]);
                if (check)
                    tc_row_chunk<true>(rb[cur], pn + cc, c0 + cc, nq, neg_c, q, pe, self_exclude, acc, bin, next_b,
                                       bnd_s, nbc, orow);
                else
                    tc_row_chunk<false>(rb[cur], pn + cc, c0 + cc, nq, neg_c, q, pe, self_exclude, acc, bin, next_b,
                                        bnd_s, nbc, orow);
            }
            if (bin < nbc) orow[bin] += acc;  // the bin that continues past this half
            tc_fence_before();
            mbar_arrive(&tempty[a]);
        }
    }
    __syncthreads();
    if (!*abort_flag) {
        const int nq = min(kSpM, n - q0);
        if (tid == 0) {  // evaluations executed: the kept tiles' points against the tile's queries
            unsigned long long pts = 0;
            for (int j = 0; j < ntile; ++j) pts += (unsigned long long)(min(pe, pa + (tl[j] + 1) * kSpN) - (pa + tl[j] * kSpN));
            atomicAdd(n_evals, pts * (unsigned long long)nq);
            atomicAdd(n_bin_evals, pts * (unsigned long long)nq);
        }
        for (int e = tid; e < nq * nbc; e += kSpThreads) {
            const int ql = e / nbc, b = e - ql * nbc;
            binsum[(size_t)(q0 + ql) * nb + b0 + b] = outs[ql * bpc + b] + outs[(kSpM + ql) * bpc + b];
        }
    }
    if (tid == 0 && !qready) mbar_wait_bounded(qbar, 0u, status);  // the query image copy still in flight
    if (warp == 4) {
        if (lane == 0 && mma_issued) {
            // all MMAs of this CTA must be complete before TMEM is freed
            umma_commit(fin);
            mbar_wait_bounded(fin, 0u, status);
        }
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Per bin, the bounding box of its points (coordinates past d are 0): block
// b, thread = coordinate.
__global__ void bin_boxes_kernel(const float* __restrict__ Xt, int dp, int d, const int32_t* __restrict__ bnd,
                                 float* __restrict__ boxes) {
    const int b = blockIdx.x, c = threadIdx.x;
    float lo = 0.f, hi = 0.f;
    if (c < d) {
        const int p0 = bnd[b], p1 = bnd[b + 1];
        lo = hi = Xt[(size_t)p0 * dp + c];
        for (int p = p0 + 1; p < p1; ++p) {
            const float x = Xt[(size_t)p * dp + c];
            lo = fminf(lo, x);
            hi = fmaxf(hi, x);
        }
    }
    boxes[(size_t)b * 128 + c] = lo;
    boxes[(size_t)b * 128 + 64 + c] = hi;
}

// The image of nv <= 128 consecutive tree positions p0 .. p0 + nv - 1 (128
// threads, thread = row): centre c (the mean of the points; any centre is
// exact, a near one is accurate), each row centred and split into three
// swizzled BF16 parts, the rows' centred squared norms, c; rows past nv are
// zero.  With box != nullptr also the points' bounding box (low, high corner).
// xs [128][kImgStride] (16-byte aligned) and cen [64] are the block's shared
// staging; xs keeps the rows (zeros past nv) on return.
constexpr int kImgStride = kSpDim + 4;  // row stride in floats: conflict-free 16-byte stores and column reads
__device__ __forceinline__ void write_image(const float* __restrict__ Xt, int dp, int d, int p0, int nv,
                                            unsigned char* __restrict__ img, float* __restrict__ box, float* xs,
                                            float* cen) {
    constexpr int kStride = kImgStride;
    const int r = threadIdx.x;
    float4 x[kSpDim / 4];
    load_row(Xt, dp, r < nv ? p0 + r : -1, x);
#pragma unroll
    for (int u = 0; u < kSpDim / 4; ++u) *reinterpret_cast<float4*>(xs + r * kStride + 4 * u) = x[u];
    __syncthreads();
    if (r < kSpDim) {
        float lo = 0.f, hi = 0.f, c = 0.f;
        if (r < d) {
            lo = hi = xs[r];
            for (int q = 0; q < nv; ++q) {
                const float v = xs[q * kStride + r];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
                c += v;
            }
            c /= (float)nv;
        }
        if (box) {
            box[r] = lo;
            box[64 + r] = hi;
        }
        cen[r] = c;
    }
    __syncthreads();
    const float norm = split_row(x, r < nv, cen, img, r);
    reinterpret_cast<float*>(img + kSpParts * kPart)[r] = norm;
    if (r < kSpDim) reinterpret_cast<float*>(img + kSpParts * kPart + kSpM * 4)[r] = cen[r];
}

// Per tile of 128 consecutive tree positions (block tb): its bounding box and
// its image, the query operand of the bin pass.  With lb != nullptr also a
// lower bound of its queries' degrees for the approximate pass: the smallest
// over its queries of the exact sum over the tile's own points (FP32 direct
// differences; the self term under INCLUDE, not under EXCLUDE), less 2^-16 of
// it for rounding, stored as log2 (kNoBound when it is 0).
__global__ void __launch_bounds__(kSpM) split_prep_kernel(const float* __restrict__ Xt, int dp, int d, int n,
                                                          float* __restrict__ boxes, unsigned char* __restrict__ qimg,
                                                          float* __restrict__ lb, float neg_c, int self_exclude) {
    __shared__ __align__(16) float xs[kSpM * kImgStride];
    __shared__ float cen[kSpDim];
    __shared__ float wmin[kSpM / 32];
    const int tb = blockIdx.x, p0 = tb * kSpM, nv = min(kSpM, n - p0);
    write_image(Xt, dp, d, p0, nv, qimg + (size_t)tb * kQImg, boxes + (size_t)tb * 128, xs, cen);
    if (!lb) return;
    const int r = threadIdx.x;
    constexpr int kStride = kImgStride;
    const float* rows = xs;  // the tile's rows, staged by write_image
    float4 x[kSpDim / 4];
#pragma unroll
    for (int u = 0; u < kSpDim / 4; ++u) x[u] = *reinterpret_cast<const float4*>(rows + r * kStride + 4 * u);
    float sum = 3.0e38f;  // rows past nv take no part in the minimum
    if (r < nv) {
        sum = 0.f;
        for (int j = 0; j < nv; ++j) {
            if (j == r && self_exclude) continue;
            float d2 = 0.f;
#pragma unroll
            for (int u = 0; u < kSpDim / 4; ++u) {
                if (4 * u >= dp) break;
                const float4 y = *reinterpret_cast<const float4*>(rows + j * kStride + 4 * u);
                const float a = x[u].x - y.x, b = x[u].y - y.y, c = x[u].z - y.z, e = x[u].w - y.w;
                d2 = fmaf(a, a, d2);
                d2 = fmaf(b, b, d2);
                d2 = fmaf(c, c, d2);
                d2 = fmaf(e, e, d2);
            }
            sum += ex2_approx(neg_c * d2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum = fminf(sum, __shfl_xor_sync(0xffffffffu, sum, o));
    if ((r & 31) == 0) wmin[r >> 5] = sum;
    __syncthreads();
    if (r == 0) {
        float m = wmin[0];
        for (int w = 1; w < kSpM / 32; ++w) m = fminf(m, wmin[w]);
        m *= 1.f - 0x1p-16f;
        lb[tb] = m > 0.f ? __log2f(m) : kNoBound;
    }
}

// Per bin of at most 128 points (block b): its image, the point operand of
// the split-precision leaf phase.
__global__ void __launch_bounds__(kSpM) bin_images_kernel(const float* __restrict__ Xt, int dp, int d,
                                                          const int32_t* __restrict__ bnd,
                                                          unsigned char* __restrict__ bimg) {
    __shared__ __align__(16) float xs[kSpM * kImgStride];
    __shared__ float cen[kSpDim];
    const int b = blockIdx.x, p0 = bnd[b];
    write_image(Xt, dp, d, p0, bnd[b + 1] - p0, bimg + (size_t)b * kQImg, nullptr, xs, cen);
}

// ---------------------------------------------------------------------------
// Split-precision leaf phase (d in 17..64, bins of at most 128 points): per
// chunk of 128 items of a bin, the kernel values of each item's query against
// the bin's m points, k = ex2(neg_c ||a - b||^2) with a, b centred at the
// bin's centre and a.b from the six BF16 products on the tensor cores (the
// bin pass's arithmetic, so the mode's bound covers both phases); the values
// stay in shared memory for the descents through the bin (the depth-4 node
// sums, then descend_bin_row), as in the FP32 fused leaf kernel.
//
// Per CTA (one bin, chunks blockIdx.y, + gridDim.y, ...; 256 threads, two
// CTAs per SM): the bin's norms and centre are bulk-copied once; per chunk
// thread 0 bulk-copies the bin's three parts (B), all threads gather, centre
// and split the items' query rows (A: thread pair per row, half the
// coordinates each), thread 0 issues the 6 x ceil(d / 16) MMAs of N = m
// rounded up to 16 into a 128-column accumulator, and thread = (row, column
// half) turns its TMEM lane into values.  The value rows and the depth-4
// trees take the place of A and B, which are idle by then; the next chunk's
// copy starts after the descents.  Every wait is bounded; on a timeout the
// CTA records FSG_ERR_TIMEOUT, waits (bounded) for its own copies and MMAs,
// frees TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int kLsThreads = 256;
constexpr int kLsVS = kSpN + 1;  // value row stride (odd)

struct LsLayout {
    static constexpr uint32_t A = 0;                                   // [3][128 rows] query parts
    static constexpr uint32_t B = A + kSpParts * kPart;                // [3][128 rows] the bin's parts
    static constexpr uint32_t V = 0;                                   // [128][kLsVS] values (over A and B)
    static constexpr uint32_t BT = V + kSpM * kLsVS * 4;               // [128][33] depth-4 node sums and tree
    static constexpr uint32_t BN = B + kSpParts * kPart;               // [128] the bin's centred norms
    static constexpr uint32_t BCEN = BN + kSpN * 4;                    // [64] the bin's centre
    static constexpr uint32_t AN = BCEN + kSpDim * 4;                  // [2][128] query norm halves
    static constexpr uint32_t ROWPOS = AN + 2 * kSpM * 4;              // [128] item query positions
    static constexpr uint32_t QMASK = ROWPOS + kSpM * 4;               // [128] item sample masks
    static constexpr uint32_t PREFIX = QMASK + kSpM * 8;               // [129] samples before item r (+ 3)
    static constexpr uint32_t BND4 = PREFIX + 132 * 4;                 // [17] depth-4 node starts (+ 3)
    static constexpr uint32_t BARS = BND4 + 20 * 4;                    // nbar, bbar, accf, fin
    static constexpr uint32_t SLOT = BARS + 4 * 8;                     // TMEM slot
    static constexpr uint32_t total = SLOT + 16;
};
static_assert(LsLayout::BT + kSpM * 33 * 4 <= LsLayout::BN, "values and trees fit over the operands");
static_assert(LsLayout::BCEN == LsLayout::BN + kSpN * 4 && LsLayout::BN % 16 == 0 && LsLayout::QMASK % 8 == 0 &&
                  LsLayout::BARS % 8 == 0,
              "layout");
static_assert(2 * (1024 + LsLayout::total + 1024) <= 228 * 1024, "two CTAs per SM");

// Coordinates 32 h .. 32 h + 31 of tree position p (zeros past dp, or for p < 0).
__device__ __forceinline__ void load_half_row(const float* __restrict__ Xt, int dp, int p, int h, float4 (&x)[8]) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int c = 32 * h + 4 * u;
        x[u] = (p >= 0 && c < dp) ? *reinterpret_cast<const float4*>(Xt + (size_t)p * dp + c)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Chunks 4 h .. 4 h + 3 of a row (those below nchw), centred at cen, split
// and stored like split_row; returns their part of the squared norm.
__device__ __forceinline__ float split_half_row(const float4 (&x)[8], bool valid, const float* __restrict__ cen,
                                                unsigned char* parts, int row, int h, int nchw) {
    float norm = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = 4 * h + i;
        if (k >= nchw) break;
        const uint32_t off = (uint32_t)row * 128u + (uint32_t)((k ^ (row & 7)) << 4);
        if (!valid) {
            *reinterpret_cast<uint4*>(parts + off) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(parts + kPart + off) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(parts + 2 * kPart + off) = make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        const float v[8] = {x[2 * i].x, x[2 * i].y, x[2 * i].z, x[2 * i].w,
                            x[2 * i + 1].x, x[2 * i + 1].y, x[2 * i + 1].z, x[2 * i + 1].w};
        float a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            a[j] = __fsub_rn(v[j], cen[8 * k + j]);
            norm = __fmaf_rn(a[j], a[j], norm);
        }
        uint4 hi, mid, lo;
        split2(a[0], a[1], hi.x, mid.x, lo.x);
        split2(a[2], a[3], hi.y, mid.y, lo.y);
        split2(a[4], a[5], hi.z, mid.z, lo.z);
        split2(a[6], a[7], hi.w, mid.w, lo.w);
        *reinterpret_cast<uint4*>(parts + off) = hi;
        *reinterpret_cast<uint4*>(parts + kPart + off) = mid;
        *reinterpret_cast<uint4*>(parts + 2 * kPart + off) = lo;
    }
    return norm;
}

__global__ void __launch_bounds__(kLsThreads, 2)
leaf_split_tc_kernel(const float* __restrict__ Xt, int dp, int d, const unsigned char* __restrict__ bimg,
                     const int32_t* __restrict__ bnd, const int32_t* __restrict__ bin_off,
                     const int32_t* __restrict__ items_q, const uint64_t* __restrict__ items_mask,
                     const int32_t* __restrict__ perm, KernelParams kp, int s0, int32_t* __restrict__ leaf_pos,
                     float* __restrict__ ksmp, uint8_t* __restrict__ lflags, unsigned long long* __restrict__ n_evals,
                     unsigned long long* __restrict__ n_items, int32_t* __restrict__ status) {
    const int b = blockIdx.x;
    const int seg = bin_off[b * kBinSlots];
    const int cnt = bin_off[(b + 1) * kBinSlots] - seg;
    const int nchunks = (cnt + kSpM - 1) / kSpM;
    if ((int)blockIdx.y >= nchunks) return;
    const int p_lo = bnd[b], m = bnd[b + 1] - p_lo;  // m <= 128
    const int N = (m + 15) & ~15;                     // MMA columns
    const int dm = ceil_log2_dev(m);
    const uint32_t idesc = idesc_bf16(kSpM, N);
    const int kk = (d + 15) / 16, nchw = 2 * kk;  // K-steps; 16-byte chunks the MMAs read

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_align1024(smem_raw);
    unsigned char* sA = base + LsLayout::A;
    unsigned char* sB = base + LsLayout::B;
    float* vrows = reinterpret_cast<float*>(base + LsLayout::V);
    float* btree = reinterpret_cast<float*>(base + LsLayout::BT);
    float* bn = reinterpret_cast<float*>(base + LsLayout::BN);
    float* bcen = reinterpret_cast<float*>(base + LsLayout::BCEN);
    float* anp = reinterpret_cast<float*>(base + LsLayout::AN);
    int32_t* rowpos = reinterpret_cast<int32_t*>(base + LsLayout::ROWPOS);
    uint64_t* qmask = reinterpret_cast<uint64_t*>(base + LsLayout::QMASK);
    int32_t* prefix = reinterpret_cast<int32_t*>(base + LsLayout::PREFIX);
    int32_t* bnd4 = reinterpret_cast<int32_t*>(base + LsLayout::BND4);
    uint64_t* nbar = reinterpret_cast<uint64_t*>(base + LsLayout::BARS);  // the bin's norms and centre landed
    uint64_t* bbar = nbar + 1;                                            // the bin's parts landed (per chunk)
    uint64_t* accf = nbar + 2;                                            // the chunk's MMAs complete
    uint64_t* fin = nbar + 3;                                             // teardown
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + LsLayout::SLOT);

    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(nbar, 1);
        mbar_init(bbar, 1);
        mbar_init(accf, 1);
        mbar_init(fin, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid <= 16) bnd4[tid] = depth4_start(tid, m);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const unsigned char* img = bimg + (size_t)b * kQImg;
    if (tid == 0) {
        mbar_arrive_expect_tx(nbar, kSpN * 4 + kSpDim * 4);
        bulk_g2s(bn, img + kSpParts * kPart, kSpN * 4 + kSpDim * 4, nbar);
    }
    bool ok = mbar_wait_bounded(nbar, 0u, status);
    bool mma_issued = false;
    int nfill = 0, ncons = 0;  // thread 0: bin-part copies issued / seen complete
    int tiles = 0;             // chunks whose accumulator completed
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        if (__syncthreads_or(!ok)) { ok = false; break; }
        const int it0 = chunk * kSpM;
        const int qcnt = min(kSpM, cnt - it0);
        if (tid == 0) {  // B: the previous chunk's values and trees over it are no longer read
            mbar_arrive_expect_tx(bbar, kSpParts * kPart);
            bulk_g2s(sB, img, kSpParts * kPart, bbar);
            ++nfill;
        }
        if (tid < kSpM) {
            rowpos[tid] = tid < qcnt ? items_q[seg + it0 + tid] : -1;
            qmask[tid] = tid < qcnt ? items_mask[seg + it0 + tid] : 0ull;
        }
        __syncthreads();
        {  // A: the items' query rows, centred at the bin's centre and split
            const int r = tid & (kSpM - 1), h = tid >> 7;
            const int pos = rowpos[r];
            float4 x[8];
            load_half_row(Xt, dp, pos, h, x);
            anp[h * kSpM + r] = split_half_row(x, pos >= 0, bcen, sA, r, h, nchw);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            ok = mbar_wait_bounded(bbar, (uint32_t)tiles & 1u, status);
            if (ok) {
                ++ncons;
                tc_fence_after();
                const int pi[6] = {2, 0, 1, 1, 0, 0};  // A part (0 hi, 1 mid, 2 lo)
                const int pj[6] = {0, 2, 1, 0, 1, 0};  // B part
#pragma unroll
                for (int u = 0; u < 6; ++u) {
                    const uint64_t da = sdesc(smem_u32(sA + pi[u] * kPart));
                    const uint64_t db = sdesc(smem_u32(sB + pj[u] * kPart));
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k >= kk) break;
                        umma_bf16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (u | k) != 0 ? 1u : 0u);
                    }
                }
                mma_issued = true;
                umma_commit(accf);
            }
        }
        if (__syncthreads_or(!ok)) { ok = false; break; }
        ok = mbar_wait_bounded(accf, (uint32_t)tiles & 1u, status);
        ++tiles;
        if (__syncthreads_or(!ok)) { ok = false; break; }
        tc_fence_after();
        // values: row r = TMEM lane (warps w and w + 4 read lanes 32 (w % 4) ..
        // + 31), half hh takes the 32-column steps hh, hh + 2, ...; the MMAs
        // are complete, so the rows may overwrite A and B
        const int r = tid & (kSpM - 1), hh = tid >> 7;
        const int qp = rowpos[r];
        const float nq = anp[r] + anp[kSpM + r];
        float* vr = vrows + (size_t)r * kLsVS;
        const int sc = (kp.self_exclude && qp >= p_lo && qp < p_lo + m) ? qp - p_lo : -1;  // the query itself
        const float neg_c = kp.neg_c;
#pragma unroll 1
        for (int c0 = 32 * hh; c0 < N; c0 += 64) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
            if (c0 + 32 <= N) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float arg = fmaf(-2.f, v[j], nq + bn[c0 + j]);
                    vr[c0 + j] = ex2_approx(fmaxf(arg, 0.f) * neg_c);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {  // N - c0 = 16
                    const float arg = fmaf(-2.f, v[j], nq + bn[c0 + j]);
                    vr[c0 + j] = ex2_approx(fmaxf(arg, 0.f) * neg_c);
                }
            }
            if (sc >= c0 && sc < c0 + 32) vr[sc] = 0.f;
        }
        // samples of the chunk's items: prefix[r] = samples of items < r
        if (tid < kSpM) {
            int x = __popcll(qmask[tid]);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if ((tid & 31) >= o) x += y;
            }
            prefix[tid + 1] = x;  // inclusive within the warp
        }
        __syncthreads();
        // the 16 depth-4 node sums of row r: half hh sums nodes 8 hh .. 8 hh + 7
        float* bt = btree + (size_t)r * 33;  // odd stride: the lanes' rows hit distinct banks
        for (int k = 8 * hh; k < 8 * hh + 8; ++k) {
            float acc = 0.f;
            for (int j = bnd4[k]; j < bnd4[k + 1]; ++j) acc += vr[j];
            bt[16 + k] = acc;
        }
        if (tid == 0) {  // warp totals into the prefix
            prefix[0] = 0;
            for (int w2 = 1; w2 < 4; ++w2) {
                const int add = prefix[32 * w2];
                for (int i = 32 * w2 + 1; i <= 32 * w2 + 32; ++i) prefix[i] += add;
            }
        }
        __syncthreads();
        if (hh == 0) {
#pragma unroll
            for (int h = 15; h >= 1; --h) bt[h] = bt[2 * h] + bt[2 * h + 1];
        }
        __syncthreads();
        // descents: the chunk's samples spread over all threads
        const int total = prefix[kSpM];
        for (int gs = tid; gs < total; gs += kLsThreads) {
            int lo = 0, hi = kSpM;  // item: prefix[lo] <= gs < prefix[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (prefix[mid] <= gs) lo = mid; else hi = mid;
            }
            uint64_t mk = qmask[lo];
            for (int k = gs - prefix[lo]; k > 0; --k) mk &= mk - 1ull;
            const int l = __ffsll((long long)mk) - 1;
            const int ip = rowpos[lo];
            const float* vi = vrows + (size_t)lo * kLsVS;
            uint8_t f = 0;
            const int a = descend_bin_row(vi, btree + (size_t)lo * 33, m, dm, s0, kp.seed, (uint32_t)perm[ip],
                                          (uint32_t)l, kp.flag_eps, f);
            const size_t o = (size_t)ip * kp.L + l;
            leaf_pos[o] = p_lo + a;
            ksmp[o] = vi[a];
            lflags[o] = f;
        }
        // the next chunk's copy and MMAs (async proxy) follow these accesses
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    if (tid == 0 && ok) {
        unsigned long long its = 0;
        for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) its += (unsigned long long)min(kSpM, cnt - chunk * kSpM);
        atomicAdd(n_items, its);
        atomicAdd(n_evals, its * (unsigned long long)m);
    }
    // teardown: own copies landed, own MMAs complete, then free TMEM
    if (tid == 0) {
        if (!ok) mbar_wait_bounded(nbar, 0u, status);
        for (int g = ncons; g < nfill; ++g) mbar_wait_bounded(bbar, (uint32_t)g & 1u, status);
        if (mma_issued) {
            umma_commit(fin);
            mbar_wait_bounded(fin, 0u, status);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
    }
}

}  // namespace

// d <= 64 (coordinates zero-padded to 64); every bin of at least 32 points, so
// at most one bin ends in the 32 columns of an epilogue step.
bool kde_bins_split_supported(const fsg_tree* t) { return t->d <= kSpDim && t->n / t->nb >= 32; }

// Bin boxes, tile boxes, the tiles' images, then (for the split leaf phase)
// the bins' images; every array starts 16-byte aligned (the boxes are
// multiples of 512 bytes, an image 49,920 bytes).
size_t split_workspace_bytes(int64_t n, int64_t nb, bool bin_images) {
    const int64_t qblocks = (n + kSpM - 1) / kSpM;
    return sizeof(float) * (size_t)(nb + qblocks + (qblocks + 127) / 128) * 128 +
           (size_t)(qblocks + (bin_images ? nb : 0)) * kQImg;
}

bool leaf_split_tc_supported(const fsg_tree* t) {
    return t->d > kMaxFmaDim && t->d <= kSpDim && t->mmax <= kSpN && kde_bins_split_supported(t);
}

cudaError_t launch_leaf_split_tc(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    if (!t->sboxes || !leaf_split_tc_supported(t)) return cudaErrorInvalidValue;
    unsigned char* bimg = SplitWs(t).bin_img;
    const size_t smem = 1024 + LsLayout::total;
    {
        const cudaError_t e = set_smem_limit(leaf_split_tc_kernel, (int)smem);
        if (e != cudaSuccess) return e;
    }
    bin_images_kernel<<<t->nb, kSpM, 0, s>>>(t->Xt, t->dp, t->d, t->bnd, bimg);
    const int64_t items_est = t->n * (int64_t)(kp.L < t->nb ? kp.L : t->nb);
    const int64_t chunks_per_bin = (items_est / t->nb + kSpM - 1) / kSpM + 1;
    int64_t S = (152 * 2 * 8 + t->nb - 1) / t->nb;
    if (S > chunks_per_bin) S = chunks_per_bin;
    if (t->tune.leaf_splits > 0) S = t->tune.leaf_splits;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    const auto& ws = t->ws;
    leaf_split_tc_kernel<<<dim3(t->nb, (unsigned)S), kLsThreads, smem, s>>>(
        t->Xt, t->dp, t->d, bimg, t->bnd, ws.bin_off, ws.items_q, ws.items_mask, t->perm, kp, t->s0, ws.leaf_pos,
        ws.ksmp, ws.lflags, reinterpret_cast<unsigned long long*>(&ws.stats->n_evals),
        reinterpret_cast<unsigned long long*>(&ws.stats->n_items), t->status);
    return cudaGetLastError();
}

cudaError_t launch_kde_bins_split(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const int qblocks = (int)((t->n + kSpM - 1) / kSpM);
    int chunks = (4 * 152 + qblocks - 1) / qblocks;
    if (chunks < 1) chunks = 1;
    if (chunks > t->nb) chunks = t->nb;
    int bpc = (t->nb + chunks - 1) / chunks;
    if (bpc > kSpMaxBins) bpc = kSpMaxBins;
    while (bpc > 1 && ((int64_t)bpc * t->mmax + kSpN - 1) / kSpN > kSpMaxTiles) --bpc;  // the kept-tile list
    if (((int64_t)bpc * t->mmax + kSpN - 1) / kSpN > kSpMaxTiles) return cudaErrorInvalidValue;
    chunks = (t->nb + bpc - 1) / bpc;
    const size_t smem = 1024 + SpLayout::total(bpc);
    {
        const cudaError_t e = set_smem_limit(kde_bins_split_kernel, 227 * 1024);
        if (e != cudaSuccess) return e;
    }
    if (!t->sboxes) return cudaErrorInvalidValue;
    const SplitWs ws(t);
    const bool approx = kp.kde_eps > 0.f;
    // error budget: a query meets at most `sweep` point tiles over all chunks
    const double sweep = (double)((t->n + kSpN - 1) / kSpN + chunks);
    const float log2_budget = approx ? (float)(std::log2((double)kp.kde_eps) - std::log2(sweep)) : kNoBound;
    bin_boxes_kernel<<<t->nb, kSpDim, 0, s>>>(t->Xt, t->dp, t->d, t->bnd, ws.bin_boxes);
    split_prep_kernel<<<qblocks, kSpM, 0, s>>>(t->Xt, t->dp, t->d, (int)t->n, ws.tile_boxes, ws.tile_img,
                                               approx ? ws.tile_lb : nullptr, kp.neg_c, kp.self_exclude);
    if (!approx) {  // the kernel reads tile_lb[q] + kNoBound: any small finite value
        cudaError_t e = cudaMemsetAsync(ws.tile_lb, 0, sizeof(float) * (size_t)qblocks, s);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(qblocks, chunks);
    kde_bins_split_kernel<<<grid, kSpThreads, smem, s>>>(
        t->Xt, t->dp, t->d, (int)t->n, t->bnd, t->nb, bpc, kp.neg_c, kp.self_exclude, ws.bin_boxes, ws.tile_boxes, ws.tile_img,
        ws.tile_lb, log2_budget, t->ws.binsum,
        reinterpret_cast<unsigned long long*>(&t->ws.stats->n_evals),
        reinterpret_cast<unsigned long long*>(&t->ws.stats->n_bin_evals), t->status);
    return cudaGetLastError();
}

}  // namespace fsg
