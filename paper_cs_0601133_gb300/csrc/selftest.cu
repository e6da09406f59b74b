// Self-test of the kernels' bounded waits: a wait on an mbarrier that nothing
// will ever complete must give up after its limit, record the failure in the
// device error word and return, leaving the context usable.
#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

__global__ void wait_timeout_kernel(int* err, long long limit_cycles) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);   // one arrival expected, none will come
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0u, &abort_flag, err, kDevTimeoutProducer, limit_cycles);
    __syncthreads();
}

}  // namespace

}  // namespace ffgpu

using namespace ffgpu;

extern "C" ffgpu_status ffgpu_selftest_wait_timeout(int64_t limit_cycles, void* stream) {
    if (limit_cycles < 1 || limit_cycles > (int64_t)kWaitLimitCycles) return FFGPU_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Pool* pool = nullptr;
    const ffgpu_status st = pool_get(s, 0, &pool);
    if (st != FFGPU_OK) return st;
    wait_timeout_kernel<<<1, 32, 0, s>>>(pool->err, (long long)limit_cycles);
    return cudaGetLastError() == cudaSuccess ? FFGPU_OK : FFGPU_ERR_CUDA;
}
