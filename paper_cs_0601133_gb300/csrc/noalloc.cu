// ffgpu_fgemm_noalloc: fgemm for callers that must not allocate device memory.
//
// The regular entry points take their scratch (channel planes and residue
// slots) from a pool grown with stream-ordered allocation.  Some callers cannot
// let a library allocate: a host framework that owns every byte of device
// memory and hands out only pre-sized buffers, a latency-critical path where an
// allocation's implicit synchronisation or failure is not acceptable, or a
// process that has already reserved the whole device.  For them this file
// keeps the scratch in a statically sized device array that the module owns
// from the moment it is loaded; the call itself allocates nothing.
#include <map>
#include <mutex>

#include "internal.h"

namespace ffgpu {

namespace {

// Fixed size of the static scratch.  Every GPU that loads the library keeps
// this much device memory until the process exits.
constexpr size_t kNoAllocScratchBytes = FFGPU_NOALLOC_SCRATCH_BYTES;  // 64 MiB
constexpr size_t kNoAllocErrBytes = 256;                      // error word at the front
constexpr int kNoAllocMaxGrid = 32;                           // persistent CTAs (residue slots)

// Device-side scratch.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
std::map<int, unsigned char*> g_noalloc_addr;  // device ordinal -> device address of the scratch

// Device address of the scratch on the current device, looked up once per
// device (the lookup may load the module on that device).
ffgpu_status scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return FFGPU_OK;
    }
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    g_noalloc_addr[dev] = static_cast<unsigned char*>(ptr);
    *out = static_cast<unsigned char*>(ptr);
    return FFGPU_OK;
}

}  // namespace

}  // namespace ffgpu

using namespace ffgpu;

extern "C" ffgpu_status ffgpu_fgemm_noalloc(int64_t m, int64_t n, int64_t k, uint32_t p,
                                            uint32_t alpha, const uint32_t* A, int64_t lda,
                                            const uint32_t* B, int64_t ldb, uint32_t beta,
                                            uint32_t* C, int64_t ldc, void* stream) {
    ffgpu_status st = check_args(m, n, k, p, A, lda, B, ldb, C, ldc);
    if (st != FFGPU_OK || m == 0 || n == 0) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    // A product on the CUDA-core route needs only its k-split partial sums,
    // sized with the SM count that route's launch uses; any other product
    // needs the tensor-core layout (planes, and the slots of at most
    // kNoAllocMaxGrid persistent CTAs).
    const size_t need = fgemm_small(m, n, k) ? small_ws_bytes(m, n, k, sm_count(dev))
                                             : fgemm_ws_bytes_min(m, n, k, p, kNoAllocMaxGrid);
    if (need > kNoAllocScratchBytes - kNoAllocErrBytes) return FFGPU_ERR_NOMEM;  // beyond the static maximum
    unsigned char* scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != FFGPU_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: the error word must start
    // at zero; the planes and slots are fully rewritten before they are read.
    int* err = reinterpret_cast<int*>(scratch);
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    return fgemm_run(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, scratch + kNoAllocErrBytes,
                     kNoAllocScratchBytes - kNoAllocErrBytes, err, s, kNoAllocMaxGrid, true);
}
