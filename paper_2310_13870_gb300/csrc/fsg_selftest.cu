// Self-test of the failure path of the bounded device waits: one warp
// initialises an mbarrier that nothing will complete and waits on it the way
// every pipeline of the library waits (try_wait with a suspend hint, a
// wall-clock limit checked every 32 polls).  When the limit runs out the
// kernel writes FSG_ERR_TIMEOUT to the status word and returns; nothing
// traps, no copy or MMA is in flight, and the context stays usable.
#include "fsg_internal.cuh"

namespace fsg {
namespace {

__global__ void wait_timeout_kernel(uint64_t limit_ns, int32_t* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none is made
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x != 0) return;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_sleep(&bar, 0u, 10000u)) return;  // never: the phase cannot complete
        if ((it & 31u) == 0u && global_ns() - t0 > limit_ns) {
            atomicExch(status, kStatusTimeout);
            return;
        }
    }
}

}  // namespace
}  // namespace fsg

extern "C" int fsg_selftest_wait_timeout(int64_t limit_ns, void* stream) {
    if (limit_ns < 1000 || limit_ns > 10000000000ll) return FSG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* d_status = nullptr;
    cudaError_t e = cudaMalloc(&d_status, sizeof(int32_t));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FSG_ERR_OOM : FSG_ERR_CUDA;
    int32_t st = -1;
    e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) {
        fsg::wait_timeout_kernel<<<1, 32, 0, s>>>((uint64_t)limit_ns, d_status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_status);
    if (e != cudaSuccess) return FSG_ERR_CUDA;
    return st;  // FSG_ERR_TIMEOUT when the wait ran out as designed
}
