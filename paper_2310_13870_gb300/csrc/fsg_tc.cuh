// tcgen05 / TMA / TMEM helpers shared by the tensor-core kernels (device
// code only): shared-memory matrix descriptors, MMA issue and commit, TMEM
// loads, and the epilogue step that turns 32 dot products of one row into
// kernel values and adds them to the row's bin sums.
#ifndef FSG_TC_CUH
#define FSG_TC_CUH

#include <cuda.h>

#include <climits>

#include "fsg_internal.cuh"

namespace fsg {

// Shared-memory matrix descriptor (tcgen05): K-major, 128-byte swizzle,
// 8-row groups of 1024 bytes.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;               // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// M x N (M = 128, N a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One tcgen05.mma kind::f16 (BF16 operands, FP32 accumulator in TMEM);
// accumulate = 0 overwrites the accumulator.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Issue a 32-column load of this warp's TMEM lanes (completed by tmem_wait).
__device__ __forceinline__ void tmem_issue32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// Wait for this thread's TMEM loads; the registers of the load being waited
// for are operands, so no use of them can move above the wait.
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Balanced pairwise sum of 32 values (fixed order: x[j] += x[j + w] for
// w = 16, 8, 4, 2, 1), the first four levels on FP32x2 pairs.
__device__ __forceinline__ float tree_sum32(float (&x)[32]) {
    uint64_t p[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) p[j] = f2_pack(x[2 * j], x[2 * j + 1]);
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
#pragma unroll
        for (int j = 0; j < w; ++j) p[j] = f2_add(p[j], p[j + w]);
    }
    const float2 t = f2_unpack(p[0]);
    return t.x + t.y;
}

// Kernel values v[0..31] of 32 columns of one row from its 32 dot products.
// pn: the 32 columns' norms, 16-byte aligned (read as float4 broadcasts).
// CHECK: test for the ragged end (p >= pe) and the query's own position.
// EXPD: the exponential kernel (Sec. 2.1), whose exponent scales the
// Euclidean distance, the square root of the exact integer squared distance.
// CLAMP: clamp the squared distance at zero (the split form, whose expansion
// can round below zero; on 8-bit data it is an exact non-negative integer
// while the norms stay below 2^24, and otherwise off by the norms' rounding
// on either side of zero).
template <bool CHECK, bool EXPD = false, bool CLAMP = true>
__device__ __forceinline__ void tc_values32(const uint32_t (&r)[32], const float* __restrict__ pn, int pc, float nq,
                                            float neg_c, int q, int pe, int self_exclude, float (&v)[32]) {
    const uint64_t nq2 = f2_pack(nq, nq), m2 = f2_pack(-2.f, -2.f), nc2 = f2_pack(neg_c, neg_c);
#pragma unroll
    for (int j4 = 0; j4 < 32; j4 += 4) {
        const float4 p4 = *reinterpret_cast<const float4*>(pn + j4);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j4 + 2 * h;
            // integer units: exact while the sums stay below 2^24
            const uint64_t arg = f2_fma(m2, f2_pack(__uint_as_float(r[j]), __uint_as_float(r[j + 1])),
                                        f2_add(nq2, h ? f2_pack(p4.z, p4.w) : f2_pack(p4.x, p4.y)));
            const float2 a = f2_unpack(arg);
            float x0 = CLAMP ? fmaxf(a.x, 0.f) : a.x, x1 = CLAMP ? fmaxf(a.y, 0.f) : a.y;
            if (EXPD) {
                x0 = sqrt_approx(x0);
                x1 = sqrt_approx(x1);
            }
            const float2 e = f2_unpack(f2_mul(f2_pack(x0, x1), nc2));
            float k0 = ex2_approx(e.x), k1 = ex2_approx(e.y);
            if (CHECK) {
                if (pc + j >= pe || (self_exclude && pc + j == q)) k0 = 0.f;
                if (pc + j + 1 >= pe || (self_exclude && pc + j + 1 == q)) k1 = 0.f;
            }
            v[j] = k0;
            v[j + 1] = k1;
        }
    }
}

// The 32 values of one row added to the row's bin sums.  Bins hold more than
// 32 points, so at most one bin ends inside the 32 columns (at a column that
// is the same for every row of the warp).  v is consumed.
__device__ __forceinline__ void tc_row_bins(float (&v)[32], int pc, float& acc, int& bin, int& next_b,
                                            const int32_t* __restrict__ bnd_s, int nbc, float* __restrict__ orow) {
    const int jb = next_b - 1 - pc;  // the current bin ends after column jb
    if (jb >= 0 && jb < 32) {
        float hi[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            hi[j] = j > jb ? v[j] : 0.f;
            v[j] = j > jb ? 0.f : v[j];
        }
        orow[bin] += acc + tree_sum32(v);
        acc = tree_sum32(hi);
        ++bin;
        next_b = bin < nbc ? bnd_s[bin + 1] : INT_MAX;
    } else {
        acc += tree_sum32(v);
    }
}

// Kernel values of 32 columns of one row, added to the row's bin sums.
template <bool CHECK>
__device__ __forceinline__ void tc_row_chunk(const uint32_t (&r)[32], const float* __restrict__ pn, int pc, float nq,
                                             float neg_c, int q, int pe, int self_exclude, float& acc, int& bin,
                                             int& next_b, const int32_t* __restrict__ bnd_s, int nbc,
                                             float* __restrict__ orow) {
    float v[32];
    tc_values32<CHECK>(r, pn, pc, nq, neg_c, q, pe, self_exclude, v);
    tc_row_bins(v, pc, acc, bin, next_b, bnd_s, nbc, orow);
}

}  // namespace fsg

#endif  // FSG_TC_CUH
