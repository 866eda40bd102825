// Tensor-core bin pass (tcgen05 + TMEM + TMA) for d >= 64 on data that are
// exact multiples of 1/255 in [0,1] (8-bit images).  Scaled by 255 the
// coordinates are integers 0..255, exact in BF16, so every product of the
// dot-product GEMM is exact and only its FP32 accumulation rounds:
//   ||x - y||^2 = ||x||^2 + ||y||^2 - 2 x.y   (integer units, exact norms),
//   k = ex2(neg_c / 255^2 * ||x - y||^2),
// or for the exponential kernel k = ex2(neg_c / 255 * sqrt(||255 x - 255 y||^2)).
//
// CTA = one block of 128 queries x one chunk of bins (their points), 10 warps:
//   warp 0 (one thread): TMA producer, 4-stage ring of {A: 128 query rows,
//                        B: 256 point rows} x 64 coordinates (128-byte swizzle);
//   warp 1 (one thread): MMA issuer, tcgen05.mma kind::f16 M=128 N=256 K=16,
//                        FP32 accumulators in TMEM, two 256-column buffers;
//                        warp 1 also allocates / frees the 512 TMEM columns;
//   warps 2..9         : epilogue, two per TMEM lane quadrant (one per half of
//                        the 256 columns): tcgen05.ld of 64 dot products per
//                        wait, kernel values, per-bin partial sums kept per
//                        column half (each row has one owner thread per half)
//                        and added half 0 + half 1 at the end.
// Every mbarrier wait is bounded; on a timeout the CTA records
// FSG_ERR_TIMEOUT, stops, waits (bounded) for its MMAs and frees TMEM.
//
// The same kernels serve the split precision (FSG_PREC_SPLIT_BF16) for FP32
// data at d > 64.  Each coordinate is held as three BF16 parts, x = hi + mid
// + lo exactly for |x| >= 2^-100 (each part the BF16 rounding of what the
// previous ones leave; smaller values add nothing at FP32 precision),
// in one row of 3 dpad values; x.y is accumulated in FP32 in TMEM from six of
// the nine part products, the small ones first (lo.hi, hi.lo, mid.mid,
// mid.hi, hi.mid, hi.hi: the three left out lie below 2^-24 of |x||y|), each
// an exact BF16 product.  The K loop simply runs over 6 dpad / 64 chunks, the
// chunk's A and B columns taken from the parts of the product it belongs
// to; the epilogue is the 8-bit path's with data-unit norms.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <climits>
#include <cmath>

#include "fsg_tc.cuh"

FSG_BOUNDS_TU(tc)

namespace fsg {
namespace {

constexpr int kTcM = 128;
constexpr int kTcN = 256;
constexpr int kTcK = 64;   // BF16 coordinates per 128-byte swizzled row
constexpr int kTcStages = 4;
constexpr int kTcEpiWarps = 8;  // epilogue warps (2 or 4 per TMEM lane quadrant)
constexpr uint32_t kABytes = kTcM * 128;
constexpr uint32_t kBBytes = kTcN * 128;
constexpr uint32_t kStageBytes = kABytes + kBBytes;
constexpr uint32_t kTmemCols = 512;

constexpr uint32_t kIdesc = idesc_bf16(kTcM, kTcN);

// Split form: the parts (0 hi, 1 mid, 2 lo) of A and of B in product j of a
// K chunk's six, one nibble per product, small products first.
constexpr uint32_t kSplitPartA = 0x001102u;  // lo, hi, mid, mid, hi, hi
constexpr uint32_t kSplitPartB = 0x010120u;  // hi, lo, mid, hi, mid, hi
// Column of virtual K chunk v (of kv = 6 kchunks in the split form, else v
// itself) in the A and B rows.
__device__ __forceinline__ void split_cols(int v, int kchunks, bool split, int& xa, int& xb) {
    if (!split) {
        xa = xb = v * kTcK;
        return;
    }
    const int j = v / kchunks, k = v - j * kchunks;
    const int dpad = kchunks * kTcK;
    xa = (int)((kSplitPartA >> (4 * j)) & 0xFu) * dpad + k * kTcK;
    xb = (int)((kSplitPartB >> (4 * j)) & 0xFu) * dpad + k * kTcK;
}

// SYM = false: CTA (x, y) = queries 128 x .. 128 x + 127 against the points
// of bins y bpc .. y bpc + bpc - 1 (every pair evaluated, both orders).
// SYM = true (the kernel is symmetric): bins are grouped in chunks of bpc; CTA
// (t, pair) takes row tile t (128 positions) of chunk k1 against the points
// of chunk k2 >= k1, pair = the index of (k1, k2) in the triangle.  Off the
// diagonal each value also goes to the column point's sum at the row's bin:
// per 32 columns a warp writes its 32 x 32 values to a transposed tile in
// shared memory and each lane adds its column's 32 rows in order, apart by
// bin (at most two bins: bins hold more than 32 points); the four lane
// quadrants' partials are added in a fixed order, and one atomic addition
// per (point, bin) and CTA goes into bin sums zeroed beforehand.  A bin meets at most two row
// tiles, so every such sum receives at most two additions onto zero, whose
// result does not depend on their order.
template <int EW, int ST, bool SYM, bool EXPD, bool SPLIT>
__global__ void __launch_bounds__(64 + 32 * EW, 1)
kde_bins_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const float* __restrict__ norms, int n, int kchunks, const int32_t* __restrict__ bnd, int nb,
                   int bpc, int nchunk, float neg_c, int self_exclude, float* __restrict__ binsum,
                   int32_t* __restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    constexpr uint32_t kStage = kABytes + kBBytes;
    constexpr int kCols = kTcN / (EW / 4);  // columns of each epilogue warp per tile
    unsigned char* base = smem_align1024(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + ST * kStage);
    uint64_t* empty = full + ST;
    uint64_t* tfull = empty + ST;
    uint64_t* tempty = tfull + 2;
    uint64_t* fin = tempty + 2;
    uint64_t* colbar = fin + 1;                                   // [EW / 4] column-part barriers
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(colbar + 2);
    int32_t* flags = reinterpret_cast<int32_t*>(tmem_slot + 1);  // [0] abort, [1] stages consumed by MMA
    int32_t* winfo = flags + 2;                                   // [4] warp's first bin, [4] rows in it
    int32_t* bnd_s = winfo + 8;                                   // bpc + 1 (column bins)
    int32_t* rbnd_s = bnd_s + ((bpc + 1 + 3) & ~3);                // bpc + 1 (row bins, SYM)
    // [epilogue warp][kCols], 16-byte aligned (float4 broadcast reads)
    float* pnorm = reinterpret_cast<float*>(rbnd_s + ((bpc + 1 + 3) & ~3));
    pnorm += ((16u - (smem_u32(pnorm) & 15u)) & 15u) / 4u;
    float* outs = pnorm + EW * kCols;                              // [EW/4 parts][128][bpc]
    float* colpart = outs + (EW / 4) * kTcM * bpc;                 // SYM: [2][EW/4][4][kCols][2]
    // SYM: [EW][32][36] transposed tiles, 16-byte aligned (float4 stores)
    float* ctile = colpart + 2 * (EW / 4) * 4 * kCols * 2;
    ctile += ((16u - (smem_u32(ctile) & 15u)) & 15u) / 4u;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int q0, b0, rb0 = 0, row_end = n;
    bool mirror = false;
    if (SYM) {
        int k1 = 0, rem = blockIdx.y;
        while (rem >= nchunk - k1) { rem -= nchunk - k1; ++k1; }
        const int k2 = k1 + rem;
        rb0 = k1 * bpc;
        const int rb1 = min(nb, rb0 + bpc);
        q0 = bnd[rb0] + (int)blockIdx.x * kTcM;
        row_end = bnd[rb1];
        if (q0 >= row_end) return;  // chunk k1 has fewer row tiles
        b0 = k2 * bpc;
        mirror = k2 > k1;
        if (tid <= rb1 - rb0) rbnd_s[tid] = bnd[rb0 + tid];
    } else {
        q0 = blockIdx.x * kTcM;
        b0 = blockIdx.y * bpc;
    }
    const int nbc = min(nb, b0 + bpc) - b0;
    const int nrows = min(kTcM, row_end - q0);
    if (tid <= nbc) bnd_s[tid] = bnd[b0 + tid];
    for (int e = tid; e < (EW / 4) * kTcM * bpc; e += (64 + 32 * EW)) outs[e] = 0.f;
    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 32 * EW);
        }
        mbar_init(fin, 1);
        for (int h = 0; h < EW / 4; ++h) mbar_init(&colbar[h], 4);
        flags[0] = 0;
        flags[1] = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (SYM && tid < 4) {  // lane quadrant tid: the bin of its first row and how many of its rows it holds
        const int r0 = q0 + 32 * tid;
        int wb = -1, cnt = 0;
        if (r0 < row_end) {
            wb = 0;
            while (rbnd_s[wb + 1] <= r0) ++wb;
            cnt = min(32, rbnd_s[wb + 1] - r0);
        }
        winfo[tid] = wb;
        winfo[4 + tid] = cnt;
    }
    __syncthreads();
    const uint32_t tmem = *tmem_slot;
    const int pa = bnd_s[0], pe = bnd_s[nbc];
    const int ntile = (pe - pa + kTcN - 1) / kTcN;
    const int kv = SPLIT ? 6 * kchunks : kchunks;  // K chunks of one tile
    const int total = ntile * kv;
    volatile int32_t* abort_flag = flags;
    volatile int32_t* consumed = flags + 1;
    int mma_issued = 0;
    int issued = 0;  // TMA stages issued (producer thread)

    // The 8-bit form needs exact 8-bit values (checked when the tree is built
    // or updated); the split form takes any FP32 data.
    const bool inexact = !SPLIT && status[1] != 0;

    if (!inexact && warp == 0 && lane == 0) {
        // ---- TMA producer
        for (int it = 0; it < total && !*abort_flag; ++it) {
            const int s = it % ST;
            if (!mbar_wait_bounded(&empty[s], ((uint32_t)(it / ST) & 1u) ^ 1u, status)) {
                *abort_flag = 1;
                break;
            }
            const int tile = it / kv, kc = it - tile * kv;
            int xa, xb;
            split_cols(kc, kchunks, SPLIT, xa, xb);
            unsigned char* st = base + s * kStage;
            mbar_arrive_expect_tx(&full[s], kStage);
            tma_load_2d(st, &tmA, xa, q0, &full[s]);
            tma_load_2d(st + kABytes, &tmB, xb, pa + tile * kTcN, &full[s]);
            issued = it + 1;
        }
    } else if (!inexact && warp == 1 && lane == 0) {
        // ---- MMA issuer
        for (int tile = 0; tile < ntile && !*abort_flag; ++tile) {
            const int a = tile & 1;
            if (!mbar_wait_bounded(&tempty[a], ((uint32_t)(tile >> 1) & 1u) ^ 1u, status)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t dt = tmem + (uint32_t)(a * kTcN);
            bool ok = true;
            for (int kc = 0; kc < kv; ++kc) {
                const int it = tile * kv + kc;
                const int s = it % ST;
                if (!mbar_wait_bounded(&full[s], (uint32_t)(it / ST) & 1u, status)) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(base + s * kStage);
                const uint64_t da = sdesc(sa), db = sdesc(sa + kABytes);
#pragma unroll
                for (int k = 0; k < kTcK / 16; ++k)  // 32 bytes of K per MMA inside the swizzled row
                    umma_bf16(dt, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kIdesc, (kc | k) != 0 ? 1u : 0u);
                mma_issued = 1;
                umma_commit(&empty[s]);
                *consumed = it + 1;
            }
            if (!ok) break;
            umma_commit(&tfull[a]);
        }
    } else if (!inexact && warp >= 2) {
        // ---- epilogue: TMEM lane quadrant (warp % 4), row = query; column part (warp - 2) / 4
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        const int r = 32 * quad + lane;
        const int q = q0 + r;
        const bool rvalid = r < nrows;
        const float nq = rvalid ? norms[q] : 0.f;
        float* pn = pnorm + (warp - 2) * kCols;
        float* orow = outs + (half * kTcM + r) * bpc;  // partial sums of this column part
        // SYM: rows of this warp in its first bin (the rest, if any, in the next)
        const int w_split = SYM ? winfo[4 + quad] : 32;
        int bin = 0;
        int next_b = nbc > 0 ? bnd_s[1] : INT_MAX;
        // point norms of this warp's columns, one tile ahead
        float nn[kCols / 32];
        auto load_norms = [&](int tile) {
            const int c = pa + tile * kTcN + half * kCols;
#pragma unroll
            for (int i = 0; i < kCols / 32; ++i) {
                const int p = c + 32 * i + lane;
                nn[i] = p < pe ? norms[p] : 0.f;
            }
        };
        load_norms(0);
        for (int tile = 0; tile < ntile; ++tile) {
            const int a = tile & 1;
            if (*abort_flag || !mbar_wait_bounded(&tfull[a], (uint32_t)(tile >> 1) & 1u, status)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int c0 = pa + tile * kTcN + half * kCols;  // first point of this warp's columns
            __syncwarp();
#pragma unroll
            for (int i = 0; i < kCols / 32; ++i) pn[32 * i + lane] = nn[i];
            __syncwarp();
            if (tile + 1 < ntile) load_norms(tile + 1);
            while (next_b <= c0) {  // bins that ended in the other half
                ++bin;
                next_b = bin < nbc ? bnd_s[bin + 1] : INT_MAX;
            }
            const bool check = c0 + kCols > pe || (self_exclude && c0 < q0 + kTcM && q0 < c0 + kCols);
            float acc = 0.f;
            float* cp = colpart + (((size_t)(tile & 1) * (EW / 4) + half) * 4 + quad) * kCols * 2;
            const uint32_t tcol = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(a * kTcN + half * kCols);
            // 32 columns per step, the next step's TMEM load in flight
            uint32_t rb[2][32];
            tmem_issue32(tcol, rb[0]);
#pragma unroll
            for (int cc = 0; cc < kCols; cc += 32) {
                const int cur = (cc >> 5) & 1;
                tmem_wait32(rb[cur]);  // the only load in flight
                if (cc + 32 < kCols) tmem_issue32(tcol + (uint32_t)(cc + 32), rb[cur ^ 1]);
                float v[32];
                if (check)
                    tc_values32<true, EXPD, SPLIT>(rb[cur], pn + cc, c0 + cc, nq, neg_c, q, pe, self_exclude, v);
                else
                    tc_values32<false, EXPD, SPLIT>(rb[cur], pn + cc, c0 + cc, nq, neg_c, q, pe, self_exclude, v);
                if (SYM && !rvalid) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                }
                if (SYM && mirror) {  // warp-uniform
                    // column sums through a transposed 32 x 32 tile: row = lane
                    // written as 16-byte pieces (row stride 36 floats: no bank
                    // conflict either way); then lanes l and l + 16 take the
                    // column pair 2 (l % 16), 2 (l % 16) + 1 as FP32x2 values,
                    // rows 0..15 and 16..31 in order, those of the warp's first
                    // bin and the rest apart, and the two halves are added
                    float* tw = ctile + (warp - 2) * 32 * 36;
                    __syncwarp();  // the previous chunk's reads are done
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4*>(tw + lane * 36 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    __syncwarp();
                    const int hrow = (lane >> 4) * 16, c2 = 2 * (lane & 15);
                    uint64_t sa = f2_pack(0.f, 0.f), sb = sa;
#pragma unroll
                    for (int rr = 0; rr < 16; ++rr) {
                        const uint64_t x = *reinterpret_cast<const uint64_t*>(tw + (hrow + rr) * 36 + c2);
                        if (hrow + rr < w_split) sa = f2_add(sa, x); else sb = f2_add(sb, x);
                    }
                    sa = f2_add(sa, __shfl_xor_sync(0xffffffffu, sa, 16));
                    sb = f2_add(sb, __shfl_xor_sync(0xffffffffu, sb, 16));
                    if (lane < 16) {  // rows 0..15 + rows 16..31; colpart is 4-byte aligned: scalar stores
                        const float2 a = f2_unpack(sa), b = f2_unpack(sb);
                        float* o = cp + 2 * (cc + c2);
                        o[0] = a.x;
                        o[1] = b.x;
                        o[2] = a.y;
                        o[3] = b.y;
                    }
                }
                tc_row_bins(v, c0 + cc, acc, bin, next_b, bnd_s, nbc, orow);
            }
            if (bin < nbc) orow[bin] += acc;  // the bin that continues past this half
            tc_fence_before();
            mbar_arrive(&tempty[a]);
            if (SYM && mirror) {
                // the four quadrants' partials of this column part, added in
                // quadrant order per row bin of the tile, into the points' sums
                __syncwarp();
                if (lane == 0) mbar_arrive(&colbar[half]);
                if (!mbar_wait_bounded(&colbar[half], (uint32_t)tile & 1u, status)) {
                    *abort_flag = 1;
                    break;
                }
                const int j = 32 * ((warp - 2) & 3) + lane;  // this thread's column of the part
                const int p = c0 + j;
                const float* cpb = colpart + ((size_t)(tile & 1) * (EW / 4) + half) * 4 * kCols * 2;
                const int lq = (nrows - 1) >> 5;  // the quadrant of the last row
                const int tb_lo = winfo[0], tb_hi = winfo[lq] + (((nrows - 1) & 31) >= winfo[4 + lq] ? 1 : 0);
                if (p < pe) {
                    for (int tb = tb_lo; tb <= tb_hi; ++tb) {
                        float sum = 0.f;
#pragma unroll
                        for (int qd = 0; qd < 4; ++qd) {
                            const int wb = winfo[qd];
                            if (wb < 0) continue;
                            if (wb == tb) sum += cpb[(qd * kCols + j) * 2];
                            else if (wb + 1 == tb) sum += cpb[(qd * kCols + j) * 2 + 1];
                        }
                        if (FSG_INB((size_t)p * nb + rb0 + tb, (long long)n * nb, kSiteTcCol))
                            atomicAdd(&binsum[(size_t)p * nb + rb0 + tb], sum);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (!inexact && !*abort_flag) {
        for (int e = tid; e < nrows * nbc; e += (64 + 32 * EW)) {
            const int ql = e / nbc, b = e - ql * nbc;
            float v = outs[ql * bpc + b];
#pragma unroll
            for (int h = 1; h < EW / 4; ++h) v += outs[(h * kTcM + ql) * bpc + b];
            if (FSG_INB((size_t)(q0 + ql) * nb + b0 + b, (long long)n * nb, kSiteTcRow))
                binsum[(size_t)(q0 + ql) * nb + b0 + b] = v;
        }
    }
    if (inexact && tid == 0) atomicExch(status, FSG_ERR_UNSUPPORTED);
    if (tid == 0) {
        // after an abort: wait (bounded) for this CTA's own copies still in flight
        for (int it = *consumed; it < issued; ++it)
            mbar_wait_bounded(&full[it % ST], (uint32_t)(it / ST) & 1u, status);
    }
    if (warp == 1) {
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

// BF16 copy of 255 * x (integers 0..255) padded to a multiple of 64
// coordinates, and exact integer squared norms.
__global__ void tc_prep_kernel(const float* __restrict__ Xt, int64_t n, int d, int dp, int dpad,
                               __nv_bfloat16* __restrict__ Xb, float* __restrict__ norms) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; p < n; p += (int64_t)gridDim.x * blockDim.y) {
        int64_t sq = 0;
        for (int t = threadIdx.x; t < dpad; t += 32) {
            const float v = t < d ? rintf(Xt[p * dp + t] * 255.f) : 0.f;
            Xb[p * dpad + t] = __float2bfloat16_rn(v);
            const int iv = (int)v;
            sq += (int64_t)iv * iv;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (threadIdx.x == 0) norms[p] = (float)sq;
    }
}

// Split form: the three BF16 parts of every coordinate (x = hi + mid + lo:
// each residual is exact in FP32, and the last one fits in eight bits) in
// rows of 3 dpad values, and the squared norms summed in FP64 and rounded
// once.  One warp per point.
__global__ void splitk_prep_kernel(const float* __restrict__ Xt, int64_t n, int d, int dp, int dpad,
                                   __nv_bfloat16* __restrict__ Xs, float* __restrict__ norms) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; p < n; p += (int64_t)gridDim.x * blockDim.y) {
        double sq = 0.0;
        __nv_bfloat16* row = Xs + (size_t)p * 3 * dpad;
        for (int t = threadIdx.x; t < dpad; t += 32) {
            const float x = t < d ? Xt[p * dp + t] : 0.f;
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            const float r1 = __fsub_rn(x, __bfloat162float(hi));
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const float r2 = __fsub_rn(r1, __bfloat162float(mid));
            row[t] = hi;
            row[dpad + t] = mid;
            row[2 * dpad + t] = __float2bfloat16_rn(r2);
            sq = fma((double)x, (double)x, sq);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (threadIdx.x == 0) norms[p] = (float)sq;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

// Allocates and fills the BF16 copy, the norms and the two tensor maps.
int tc_prepare(fsg_tree* t, cudaStream_t s) {
    const int dpad = (t->d + kTcK - 1) / kTcK * kTcK;
    if (!t->Xb) {
        cudaError_t e = cudaMalloc((void**)&t->Xb, sizeof(__nv_bfloat16) * (size_t)t->n_pad * dpad);
        if (e == cudaSuccess) e = cudaMalloc((void**)&t->norms, sizeof(float) * (size_t)t->n_pad);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return FSG_ERR_OOM;
        }
        cudaMemsetAsync(t->Xb, 0, sizeof(__nv_bfloat16) * (size_t)t->n_pad * dpad, s);
        PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
        if (!enc) return FSG_ERR_UNSUPPORTED;
        const cuuint64_t gdim[2] = {(cuuint64_t)dpad, (cuuint64_t)t->n};
        const cuuint64_t gstride[1] = {(cuuint64_t)dpad * 2};
        const cuuint32_t estride[2] = {1, 1};
        const cuuint32_t boxA[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
        const cuuint32_t boxB[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcN};
        CUresult r1 = enc(reinterpret_cast<CUtensorMap*>(t->tmap_a), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t->Xb, gdim,
                          gstride, boxA, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult r2 = enc(reinterpret_cast<CUtensorMap*>(t->tmap_b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t->Xb, gdim,
                          gstride, boxB, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        const cuuint32_t boxP[2] = {(cuuint32_t)kTcK, 16u};  // point rows of the leaf kernel
        CUresult r3 = enc(reinterpret_cast<CUtensorMap*>(t->tmap_p), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t->Xb, gdim,
                          gstride, boxP, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS || r3 != CUDA_SUCCESS)
            return FSG_ERR_UNSUPPORTED;
        t->dpad = dpad;
    }
    dim3 block(32, 8);
    int64_t g = (t->n + 7) / 8;
    if (g > 152 * 64) g = 152 * 64;
    tc_prep_kernel<<<(int)g, block, 0, s>>>(t->Xt, t->n, t->d, t->dp, dpad, reinterpret_cast<__nv_bfloat16*>(t->Xb),
                                            t->norms);
    return cudaGetLastError() == cudaSuccess ? FSG_OK : FSG_ERR_CUDA;
}

bool kde_bins_tc_supported(const fsg_tree* t) { return t->Xb != nullptr && t->d >= 64; }

// Bins of at least 33 points: at most one bin ends in the 32 columns of an
// epilogue step (or a single bin).
bool splitk_supported(const fsg_tree* t) { return t->d > 64 && (t->nb == 1 || t->n / t->nb >= 33); }

// Describes (every call: host-only) and fills the split form's image; Xs and
// snorms are allocated by the caller ([n_pad][3 dpad] BF16, [n_pad] floats,
// the padding rows zero).
int splitk_prepare(fsg_tree* t, cudaStream_t s) {
    const int dpad = (t->d + kTcK - 1) / kTcK * kTcK;
    if (!t->Xs || !t->snorms) return FSG_ERR_INVALID_ARG;
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return FSG_ERR_UNSUPPORTED;
    const cuuint64_t gdim[2] = {(cuuint64_t)(3 * dpad), (cuuint64_t)t->n};
    const cuuint64_t gstride[1] = {(cuuint64_t)(3 * dpad) * 2};
    const cuuint32_t estride[2] = {1, 1};
    const cuuint32_t boxA[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
    const cuuint32_t boxB[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcN};
    const cuuint32_t boxP[2] = {(cuuint32_t)kTcK, 16u};
    CUresult r1 = enc(reinterpret_cast<CUtensorMap*>(t->tmap_sa), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t->Xs, gdim,
                      gstride, boxA, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(reinterpret_cast<CUtensorMap*>(t->tmap_sb), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t->Xs, gdim,
                      gstride, boxB, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r3 = enc(reinterpret_cast<CUtensorMap*>(t->tmap_sp), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t->Xs, gdim,
                      gstride, boxP, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS || r3 != CUDA_SUCCESS) return FSG_ERR_UNSUPPORTED;
    t->dpad = dpad;
    dim3 block(32, 8);
    int64_t g = (t->n + 7) / 8;
    if (g > 152 * 64) g = 152 * 64;
    splitk_prep_kernel<<<(int)g, block, 0, s>>>(t->Xt, t->n, t->d, t->dp, dpad,
                                                reinterpret_cast<__nv_bfloat16*>(t->Xs), t->snorms);
    return cudaGetLastError() == cudaSuccess ? FSG_OK : FSG_ERR_CUDA;
}

namespace {
constexpr int kTcSymStages = 3;
constexpr int kTcSymMaxBins = 16;  // bins per chunk of the symmetric pass

size_t tc_bins_smem(int ew, int bpc, int st, bool sym) {
    const int kcols = kTcN / (ew / 4);
    return 1024 + (size_t)st * kStageBytes + 8 * (2 * st + 7) + 16 + 8 * 4 + 2 * (size_t)((bpc + 1 + 3) & ~3) * 4 +
           16 + (size_t)ew * kcols * 4 + (size_t)(ew / 4) * kTcM * bpc * 4 +
           (sym ? (size_t)2 * (ew / 4) * 4 * kcols * 2 * 4 + 16 + (size_t)ew * 32 * 36 * 4 : 0);
}

// Bins per chunk of the symmetric pass: the chunks' positions are cut into
// 128-row tiles, so pick the count (8..16) whose chunks fill their last tile
// best.  0: the symmetric pass does not apply (bins of fewer than 33 points
// could put three bins in one warp's 32 rows).
int tc_sym_bins(const fsg_tree* t) {
    if (t->n / t->nb < 33 || t->nb < 2) return 0;
    int best = 0;
    double best_fill = -1.0;
    for (int g = 8; g <= kTcSymMaxBins; ++g) {
        const double rows = (double)g * t->n / t->nb;
        const double tiles = std::ceil(rows / kTcM);
        const double fill = rows / (tiles * kTcM);
        if (fill > best_fill + 1e-9) { best_fill = fill; best = g; }
    }
    if (t->tune.tc_bins > 0 && t->tune.tc_bins <= kTcSymMaxBins) best = t->tune.tc_bins;
    return best;
}
}  // namespace

bool kde_bins_tc_sym(const fsg_tree* t) { return tc_sym_bins(t) > 0; }

// Pairs the tensor-core bin pass evaluates: n^2, or for the symmetric pass
// (n^2 + sum_k P_k^2) / 2, P_k the positions of chunk k (its diagonal blocks
// are evaluated in both orders).
int64_t kde_bins_tc_evals(const fsg_tree* t) {
    const int G = tc_sym_bins(t);
    if (G == 0) return t->n * t->n;
    int64_t sq = 0;
    for (int b0 = 0; b0 < t->nb; b0 += G) {
        auto start = [&](int b) {
            if (b >= t->nb) return t->n;
            int64_t lo = 0, hi = t->n;
            for (int l = t->s0 - 1; l >= 0; --l) {
                const int64_t mid = lo + (hi - lo) / 2;
                if ((b >> l) & 1) lo = mid; else hi = mid;
            }
            return lo;
        };
        const int64_t pk = start(b0 + G) - start(b0);
        sq += pk * pk;
    }
    return (t->n * t->n + sq) / 2;
}

// The scale of the exponent in integer units: ||255 x - 255 y||^2 = 255^2
// ||x - y||^2 for the Gaussian, its square root 255 ||x - y|| for the
// exponential kernel.
static float tc_neg_c(const KernelParams& kp) {
    if (kp.precision == FSG_PREC_SPLIT_BF16) return kp.neg_c;  // data units
    return kp.family == kFamExp ? kp.neg_c / 255.f : kp.neg_c / (255.f * 255.f);
}

template <bool EXPD, bool SPLIT>
cudaError_t launch_kde_bins_tc_f(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const float nc = tc_neg_c(kp);
    const bool split = SPLIT;
    if (split && !t->Xs) return cudaErrorInvalidValue;
    const CUtensorMap& ta = *reinterpret_cast<const CUtensorMap*>(split ? t->tmap_sa : t->tmap_a);
    const CUtensorMap& tb = *reinterpret_cast<const CUtensorMap*>(split ? t->tmap_sb : t->tmap_b);
    const float* norms = split ? t->snorms : t->norms;
    const int G = tc_sym_bins(t);
    if (G > 0) {
        const int nchunk = (t->nb + G - 1) / G;
        const int tmax = (int)((((int64_t)G * t->mmax) + kTcM - 1) / kTcM);
        const size_t smem = tc_bins_smem(kTcEpiWarps, G, kTcSymStages, true);
        auto kern = kde_bins_tc_kernel<kTcEpiWarps, kTcSymStages, true, EXPD, SPLIT>;
        cudaError_t e = set_smem_limit(kern, smem);
        if (e != cudaSuccess) return e;
        // the sums that the mirrored values reach are accumulated onto zero
        e = cudaMemsetAsync(t->ws.binsum, 0, sizeof(float) * (size_t)t->n * t->nb, s);
        if (e != cudaSuccess) return e;
        dim3 grid(tmax, nchunk * (nchunk + 1) / 2);
        kern<<<grid, 64 + 32 * kTcEpiWarps, smem, s>>>(ta, tb, norms, (int)t->n, t->dpad / kTcK, t->bnd, t->nb, G,
                                                       nchunk, nc, kp.self_exclude, t->ws.binsum, t->status);
        return cudaGetLastError();
    }
    const int qblocks = (int)((t->n + kTcM - 1) / kTcM);
    int chunks = (4 * 152 + qblocks - 1) / qblocks;
    if (chunks < 1) chunks = 1;
    if (chunks > t->nb) chunks = t->nb;
    int bpc = (t->nb + chunks - 1) / chunks;
    if (bpc > 24) bpc = 24;  // two [128][bpc] sum arrays beside the 4-stage ring
    if (t->tune.tc_bins > 0 && t->tune.tc_bins < bpc) bpc = t->tune.tc_bins;
    chunks = (t->nb + bpc - 1) / bpc;
    const size_t smem = tc_bins_smem(kTcEpiWarps, bpc, kTcStages, false);
    auto kern = kde_bins_tc_kernel<kTcEpiWarps, kTcStages, false, EXPD, SPLIT>;
    {
        const cudaError_t e = set_smem_limit(kern, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(qblocks, chunks);
    kern<<<grid, 64 + 32 * kTcEpiWarps, smem, s>>>(ta, tb, norms, (int)t->n, t->dpad / kTcK, t->bnd, t->nb, bpc,
                                                   chunks, nc, kp.self_exclude, t->ws.binsum, t->status);
    return cudaGetLastError();
}

cudaError_t launch_kde_bins_tc(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    // the split form is Gaussian only (the path checks refuse the others)
    if (kp.precision == FSG_PREC_SPLIT_BF16) return launch_kde_bins_tc_f<false, true>(t, kp, s);
    return kp.family == kFamExp ? launch_kde_bins_tc_f<true, false>(t, kp, s)
                                : launch_kde_bins_tc_f<false, false>(t, kp, s);
}

}  // namespace fsg

// ---------------------------------------------------------------------------
// Tensor-core leaf finish: for the items (queries) of one bin, the kernel
// value of every (item, point) pair of the bin, k = ex2(neg_c (||x||^2 +
// ||y||^2 - 2 x.y)) in the same integer units as the bin pass, then the
// remaining levels of the item's samples.  CTA (b, y) handles chunks of 128
// items of bin b (3-stage ring over K chunks of 64 coordinates, 128-byte
// swizzled K-major):
//   A = the 128 item rows, gathered with cp.async (16 bytes per copy);
//   B = the bin's m points, contiguous in tree order, by TMA in boxes of 16
//       rows (N = m rounded up to 16 columns; columns past m are ignored);
// one thread issues tcgen05.mma M=128 x N x K=16, and each of the four warps
// reads its TMEM lane quadrant: thread = item, its row of values kept in
// shared memory (the idle stages).  The thread then descends each of the
// item's samples through the bin's halving tree: the 16 nodes of depth 4 are
// summed once per item (and their tree above), deeper nodes are sums over
// their points' values, with the same Philox draws and decision rule as
// every other level; it writes the sampled position, kernel value and flags.
// Several CTAs share an SM (three with a 2-stage ring for bins of up to 80
// points, else two), so one CTA's epilogue and descents overlap the others'
// copies and MMAs.
// ---------------------------------------------------------------------------
namespace fsg {
namespace {

// Stages of the K ring (template parameter ST): 2 where the value rows fit
// two stages and three CTAs fit an SM (bins of up to 80 points: one CTA's
// epilogue and descents then overlap two others' copies and MMAs), else 3
// with two CTAs per SM.
constexpr int kLvThreads = 256;  // two threads per item row (TMEM lane): warps w and w + 4
constexpr int kLvBox = 16;  // point rows per TMA box

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// Shared-memory layout of the leaf kernel for point operands of up to nmax
// rows (nmax a multiple of 16); the same arithmetic on host and device.
struct LvLayout {
    uint32_t kB, stage, bars, rowpos, qmask, prefix, pnorm, bnd4, btree, total;
    bool tree_in_stages;
    bool rows_fit;  // the [128][nmax + 1] value rows fit the stages
    __host__ __device__ LvLayout(int nmax, int nst) {
        kB = (uint32_t)nmax * 128u;
        stage = 128u * 128u + kB;
        bars = (uint32_t)nst * stage;                    // done[nst], full[nst], accf, fin
        rowpos = bars + 8 * (2 * nst + 2) + 16;          // + TMEM slot
        qmask = rowpos + 128 * 4;                        // [128] sample masks of the chunk's items
        prefix = qmask + 128 * 8;                        // [129] samples before each item (+ 3 words)
        pnorm = prefix + 132 * 4;
        bnd4 = pnorm + (uint32_t)nmax * 4;
        const uint32_t after = bnd4 + 17 * 4 + 12;
        rows_fit = (size_t)128 * (nmax + 1) * 4 <= (size_t)nst * stage;
        tree_in_stages = (size_t)128 * (nmax + 1 + 33) * 4 <= (size_t)nst * stage;
        btree = tree_in_stages ? 128u * (uint32_t)(nmax + 1) * 4u : ((after + 15u) & ~15u);
        total = tree_in_stages ? after : btree + 128 * 33 * 4;
    }
};

template <int ST>
__global__ void __launch_bounds__(kLvThreads, ST == 2 ? 3 : 2)
leaf_values_tc_kernel(const __grid_constant__ CUtensorMap tmP, const __nv_bfloat16* __restrict__ Xb,
                      const float* __restrict__ norms, int dpad, int nmax, const int32_t* __restrict__ bnd,
                      const int32_t* __restrict__ bin_off, const int32_t* __restrict__ items_q,
                      const uint64_t* __restrict__ items_mask, const int32_t* __restrict__ perm, KernelParams kp,
                      float neg_c, int s0, int32_t* __restrict__ leaf_pos, float* __restrict__ ksmp,
                      uint8_t* __restrict__ lflags, unsigned long long* __restrict__ n_evals,
                      unsigned long long* __restrict__ n_items, int32_t* __restrict__ status, int split) {
    const int self_exclude = kp.self_exclude;
    const bool expd = kp.family == kFamExp;  // exponential kernel: the distance, not its square
    const int b = blockIdx.x;
    const int seg = bin_off[b * kBinSlots];
    const int cnt = bin_off[(b + 1) * kBinSlots] - seg;
    const int nchunks = (cnt + 127) / 128;
    if ((int)blockIdx.y >= nchunks) return;
    const int p_lo = bnd[b], m = bnd[b + 1] - p_lo;
    const int N = (m + 15) & ~15;  // MMA columns (<= nmax)
    const int dm = ceil_log2_dev(m);
    uint32_t tcols = 32;
    while ((int)tcols < N) tcols <<= 1;
    const uint32_t idesc = idesc_bf16(128, N);
    const LvLayout ly(nmax, ST);
    const uint32_t kA = 128u * 128u;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_align1024(smem_raw);
    uint64_t* done = reinterpret_cast<uint64_t*>(base + ly.bars);  // MMAs reading a stage are done
    uint64_t* full = done + ST;                              // a stage's point rows landed
    uint64_t* accf = full + ST;                              // accumulator complete
    uint64_t* fin = accf + 1;                                       // teardown
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    int32_t* rowpos = reinterpret_cast<int32_t*>(base + ly.rowpos);  // [128] item query positions
    uint64_t* qmask = reinterpret_cast<uint64_t*>(base + ly.qmask);  // [128] item sample masks
    int32_t* prefix = reinterpret_cast<int32_t*>(base + ly.prefix);  // [129] samples before item r
    float* pnorm = reinterpret_cast<float*>(base + ly.pnorm);        // [nmax] point norms
    int32_t* bnd4 = reinterpret_cast<int32_t*>(base + ly.bnd4);      // [17] depth-4 node starts
    // [128][nmax + 1] values per item: the stages are idle during the epilogue
    // (all copies landed, all MMAs of the chunk complete), so the rows live there
    float* vrows = reinterpret_cast<float*>(base);
    const int vstride = nmax + 1;
    float* btree = reinterpret_cast<float*>(base + ly.btree);  // [128][33] depth-4 node sums and their tree

    const int tid = threadIdx.x, warp = tid >> 5;
    const int kchunks = dpad / 64;
    const int kv = split ? 6 * kchunks : kchunks;    // K chunks of one accumulation
    const size_t rstride = split ? 3 * (size_t)dpad : (size_t)dpad;  // BF16 values per point row
    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&done[s], 1);
            mbar_init(&full[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(fin, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int j = tid; j < N; j += kLvThreads) pnorm[j] = j < m ? norms[p_lo + j] : 0.f;
    if (tid <= 16) bnd4[tid] = depth4_start(tid, m);  // depth-4 node starts of the bin (tid = 16: the end)
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    int g = 0;      // stage uses issued so far (stage g % ST, its use number g / ST)
    int tiles = 0;  // accumulator tiles completed
    bool mma_issued = false;
    bool ok = true;
    int nfill = 0, ncons = 0;  // thread 0: stage uses whose TMA was issued / whose arrival was seen
    // This thread's 16-byte pieces of the item rows: rows tid / 8 + 32 i
    // (i < 4), piece tid % 8 of each 128-byte row, at the 128-byte-swizzled
    // position (the row's phase within its 8-row group is the same for all i).
    const uint32_t gdst = (uint32_t)(tid >> 3) * 128u + (uint32_t)(((tid & 7) ^ ((tid >> 3) & 7)) << 4);
    const __nv_bfloat16* gsrc[4];
    uint32_t gbytes = 0;  // bit i: row i holds an item
    // K chunk kc (64 coordinates) into stage s: the 128 item rows by cp.async
    // (empty rows are 0), the point rows by TMA (one thread)
    auto fill = [&](int kc, int s) {
        unsigned char* st = base + s * ly.stage;
        int xa, xb;
        split_cols(kc, kchunks, split != 0, xa, xb);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            cp_async16(st + gdst + i * 4096, gsrc[i] + xa, ((gbytes >> i) & 1u) ? 16 : 0);
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (tid == 0) {
            mbar_arrive_expect_tx(&full[s], (uint32_t)N * 128u);
            for (int j = 0; j < N; j += kLvBox)
                tma_load_2d(st + kA + (uint32_t)j * 128u, &tmP, xb, p_lo + j, &full[s]);
            ++nfill;
        }
    };
    // waits until the MMAs of stage use g2 - ST are done
    auto stage_free = [&](int g2) -> bool {
        const int use = g2 / ST;
        if (use == 0) return true;
        return mbar_wait_bounded(&done[g2 % ST], (uint32_t)(use - 1) & 1u, status);
    };
    for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int it0 = chunk * 128;
        const int qcnt = min(128, cnt - it0);
        if (tid < 128) {
            rowpos[tid] = tid < qcnt ? items_q[seg + it0 + tid] : -1;
            qmask[tid] = tid < qcnt ? items_mask[seg + it0 + tid] : 0ull;
        }
        __syncthreads();
        gbytes = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int pos = rowpos[(tid >> 3) + 32 * i];
            gsrc[i] = Xb + (size_t)(pos >= 0 ? pos : 0) * rstride + (tid & 7) * 8;
            gbytes |= (pos >= 0 ? 1u : 0u) << i;
        }
        const int pre = min(ST - 1, kv);
        for (int kc = 0; kc < pre; ++kc) {
            if (ok) ok = stage_free(g + kc);
            if (ok) fill(kc, (g + kc) % ST);
        }
        for (int kc = 0; kc < kv; ++kc) {
            const int gs = g + kc, s = gs % ST;
            if (kc + pre < kv) {
                if (ok) ok = stage_free(g + kc + pre);
                if (ok) fill(kc + pre, (g + kc + pre) % ST);
                asm volatile("cp.async.wait_group %0;" ::"n"(ST - 1) : "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (__syncthreads_or(!ok)) { ok = false; break; }
            if (tid == 0) {
                ok = mbar_wait_bounded(&full[s], (uint32_t)(gs / ST) & 1u, status);
                if (ok) {
                    ++ncons;
                    tc_fence_after();
                    const uint32_t sa = smem_u32(base + s * ly.stage);
                    const uint64_t da = sdesc(sa), db = sdesc(sa + kA);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                            "l"(da + (uint64_t)(2 * k)), "l"(db + (uint64_t)(2 * k)), "r"(idesc),
                            "r"((kc | k) != 0 ? 1u : 0u)
                            : "memory");
                    }
                    mma_issued = true;
                    umma_commit(&done[s]);
                    if (kc == kv - 1) umma_commit(accf);
                }
            }
        }
        if (__syncthreads_or(!ok)) { ok = false; break; }
        g += kv;
        // epilogue: item row r = TMEM lane (warps w and w + 4 read lanes
        // 32 (w % 4) .. + 31), half hh of the thread pair takes the 32-column
        // steps hh, hh + 2, ...
        ok = mbar_wait_bounded(accf, (uint32_t)tiles & 1u, status);
        ++tiles;
        if (__syncthreads_or(!ok)) { ok = false; break; }
        tc_fence_after();
        const int r = tid & 127, hh = tid >> 7;
        const int qp = rowpos[r];
        const float nq = qp >= 0 ? norms[qp] : 0.f;
        float* vr = vrows + (size_t)r * vstride;
        const int sc = (self_exclude && qp >= p_lo && qp < p_lo + m) ? qp - p_lo : -1;  // the query itself
        // columns past m (up to N, zero or another bin's rows) land in the
        // row's padding (stride nmax + 1 >= N) and are never read
#pragma unroll 1
        for (int c0 = 32 * hh; c0 < N; c0 += 64) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
            if (c0 + 32 <= N) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float arg = fmaxf(fmaf(-2.f, v[j], nq + pnorm[c0 + j]), 0.f);
                    vr[c0 + j] = ex2_approx((expd ? sqrt_approx(arg) : arg) * neg_c);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {  // N - c0 = 16
                    const float arg = fmaxf(fmaf(-2.f, v[j], nq + pnorm[c0 + j]), 0.f);
                    vr[c0 + j] = ex2_approx((expd ? sqrt_approx(arg) : arg) * neg_c);
                }
            }
            if (sc >= c0 && sc < c0 + 32) vr[sc] = 0.f;
        }
        // samples of the chunk's items: prefix[r] = samples of items < r
        if (tid < 128) {
            const int c = __popcll(qmask[tid]);
            int x = c;
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
        const int total = prefix[128];
        for (int gsm = tid; gsm < total; gsm += kLvThreads) {
            int lo = 0, hi = 128;  // item: prefix[lo] <= gsm < prefix[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (prefix[mid] <= gsm) lo = mid; else hi = mid;
            }
            const int it = lo;
            uint64_t mk = qmask[it];
            for (int k = gsm - prefix[it]; k > 0; --k) mk &= mk - 1ull;
            const int l = __ffsll((long long)mk) - 1;
            const int ip = rowpos[it];
            const uint32_t qi = (uint32_t)perm[ip];
            const float* vi = vrows + (size_t)it * vstride;
            const float* bi = btree + (size_t)it * 33;
            uint8_t f = 0;
            const int a = descend_bin_row(vi, bi, m, dm, s0, kp.seed, qi, (uint32_t)l, kp.flag_eps, f);
            const size_t o = (size_t)ip * kp.L + l;
            leaf_pos[o] = p_lo + a;
            ksmp[o] = vi[a];
            lflags[o] = f;
        }
        tc_fence_before();
        __syncthreads();  // TMEM, the stages and rowpos are reused by the next chunk
    }
    if (tid == 0 && ok && (int)blockIdx.y < nchunks) {
        unsigned long long its = 0;
        for (int chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) its += (unsigned long long)min(128, cnt - chunk * 128);
        atomicAdd(n_items, its);
        atomicAdd(n_evals, its * (unsigned long long)m);
    }
    // teardown: own copies landed (cp.async and TMA), own MMAs complete, then free TMEM
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (tid == 0) {
        // point rows still in flight (an aborted chunk): let them land
        for (int gs = ncons; gs < nfill; ++gs)
            mbar_wait_bounded(&full[gs % ST], (uint32_t)(gs / ST) & 1u, status);
        if (mma_issued) {
            umma_commit(fin);
            mbar_wait_bounded(fin, 0u, status);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

}  // namespace

cudaError_t launch_leaf_values_tc(const fsg_tree* t, const KernelParams& kp, cudaStream_t s) {
    const int nmax = (t->mmax + 15) & ~15;  // point rows of the largest bin, rounded to the TMA box
    if (nmax > 256) return cudaErrorInvalidValue;
    // two stages when the value rows fit them and three CTAs fit the SM's
    // 228 KB (1 KB reserved per CTA); three stages always hold the rows
    const LvLayout l2(nmax, 2);
    const bool two = l2.rows_fit && 3 * (2048 + (size_t)l2.total) <= 228 * 1024;
    const size_t smem = 1024 + (size_t)(two ? l2.total : LvLayout(nmax, 3).total);
    auto kern = two ? leaf_values_tc_kernel<2> : leaf_values_tc_kernel<3>;
    {
        const cudaError_t e = set_smem_limit(kern, 227 * 1024);
        if (e != cudaSuccess) return e;
    }
    const int64_t items_est = t->n * (int64_t)(kp.L < t->nb ? kp.L : t->nb);
    const int64_t chunks_per_bin = (items_est / t->nb + 127) / 128 + 1;
    int64_t S = (152 * 2 * 8 + t->nb - 1) / t->nb;
    if (S > chunks_per_bin) S = chunks_per_bin;
    if (t->tune.leaf_splits > 0) S = t->tune.leaf_splits;
    if (S < 1) S = 1;
    if (S > 65535) S = 65535;
    dim3 grid(t->nb, (unsigned)S);
    const auto& ws = t->ws;
    const int split = kp.precision == FSG_PREC_SPLIT_BF16 ? 1 : 0;
    if (split && !t->Xs) return cudaErrorInvalidValue;
    kern<<<grid, kLvThreads, smem, s>>>(
        *reinterpret_cast<const CUtensorMap*>(split ? t->tmap_sp : t->tmap_p),
        reinterpret_cast<const __nv_bfloat16*>(split ? t->Xs : t->Xb), split ? t->snorms : t->norms, t->dpad, nmax,
        t->bnd, ws.bin_off, ws.items_q, ws.items_mask, t->perm, kp, tc_neg_c(kp), t->s0, ws.leaf_pos, ws.ksmp,
        ws.lflags, reinterpret_cast<unsigned long long*>(&ws.stats->n_evals),
        reinterpret_cast<unsigned long long*>(&ws.stats->n_items), t->status, split);
    return cudaGetLastError();
}

}  // namespace fsg
