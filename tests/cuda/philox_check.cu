// Test-only: Philox4x32-10 blocks from cuRAND (an independent implementation)
// and from the library's device generator, for the same (key, counter).
// cuRAND's curand_init(seed, subsequence s, offset 4*(l*2^32 + k)) puts its
// counter at (k, l, s, 0) with key (seed low, seed high); the library's block
// for (point i, sample l, level lev) uses counter (i, l, lev/4, 0).
#include <curand_kernel.h>

#include "fsg_internal.cuh"

__global__ void philox_pair_kernel(unsigned long long seed, int nsub, int nk, int nl, uint4* cr, uint4* fs) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsub * nl) return;
    const int s = t / nl, l = t % nl;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, (unsigned long long)s, 4ull * (((unsigned long long)l << 32)), &st);
    for (int k = 0; k < nk; ++k) {
        cr[(size_t)t * nk + k] = curand4(&st);
        fs[(size_t)t * nk + k] = fsg::draw_block(seed, (uint32_t)k, (uint32_t)l, (uint32_t)(4 * s));
    }
}

extern "C" int philox_check(unsigned long long seed, int nsub, int nk, int nl, unsigned int* h_cr,
                            unsigned int* h_fs) {
    const size_t cnt = (size_t)nsub * nk * nl;
    uint4 *cr = nullptr, *fs = nullptr;
    if (cudaMalloc(&cr, cnt * sizeof(uint4)) != cudaSuccess) return 1;
    if (cudaMalloc(&fs, cnt * sizeof(uint4)) != cudaSuccess) return 1;
    const int threads = nsub * nl;
    philox_pair_kernel<<<(threads + 127) / 128, 128>>>(seed, nsub, nk, nl, cr, fs);
    int rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
    if (!rc) rc = cudaMemcpy(h_cr, cr, cnt * sizeof(uint4), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : 3;
    if (!rc) rc = cudaMemcpy(h_fs, fs, cnt * sizeof(uint4), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : 3;
    cudaFree(cr);
    cudaFree(fs);
    return rc;
}
