// wave_selftest.cu -- failure detection of the bounded device-side waits.
//
// Every wait of the pass kernel (an mbarrier phase that a TMA copy completes)
// gives up after a time limit, records bit 0 in the plan's error word and
// lets the thread block return, so a copy that never lands is reported as
// WAVE_ERR_TIMEOUT instead of hanging the GPU.  This entry point exercises
// exactly that path: one block waits, with the same helper, on an mbarrier
// that nothing ever arrives on.
#include "wave_pass.cuh"

#include <string>

#include "wave_host.h"

namespace {

__global__ void selftest_wait_kernel(int* err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        wave::detail::mbar_init(wave::detail::smem_u32(&bar), 1);
        wave::detail::fence_mbar_init();
    }
    __syncthreads();
    // phase 0 never completes: no thread arrives and no copy is in flight
    if (!wave::detail::mbar_wait(wave::detail::smem_u32(&bar), 0, limit_ns)) atomicOr(err, 1);
}

}  // namespace

extern "C" wave_status wave_selftest_timeout(double limit_ms)
{
    if (!(limit_ms > 0.0) || limit_ms > 10000.0)
        return wave::fail(WAVE_ERR_ARG, "wave_selftest_timeout: limit_ms must be in (0, 10000]");
    int* err = nullptr;
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        selftest_wait_kernel<<<1, 32>>>(err, static_cast<unsigned long long>(limit_ms * 1e6));
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return wave::fail(WAVE_ERR_CUDA, std::string("wave_selftest_timeout: ") + cudaGetErrorString(e));
    if (h & 1) return wave::fail(WAVE_ERR_TIMEOUT, "bounded wait gave up as intended");
    return WAVE_OK;
}
