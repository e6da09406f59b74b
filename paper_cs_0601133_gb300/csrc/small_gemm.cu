// Exact fgemm on the CUDA cores for small contractions.
//
// The tensor-core path pays fixed costs per call (two conversion launches,
// one product per residue channel, the CRT epilogue) that dwarf the
// arithmetic of a small product such as the 64 x 64 x 64 multiplier blocks of
// LQUP.  Here every output is an exact dot product: 32-bit words multiplied
// into 64 bits and summed in a 96-bit accumulator (three 32-bit words with
// carry chains), which stays exact for any inputs and any k < 2^32, reduced
// mod p once, then alpha and beta applied (the delayed reduction of section
// 3.1 taken to its limit: one reduction per output).  64 x 64 output tiles,
// 256 threads with 4 x 4 outputs each, k staged through shared memory 32 at a
// time.
#include <algorithm>
#include <atomic>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kSmT = 64;   // output tile (rows and columns)
constexpr int kSmK = 32;   // k chunk
constexpr int kSmThreads = 256;

__device__ __forceinline__ void mac96(uint32_t& lo, uint32_t& mid, uint32_t& hi, uint32_t a, uint32_t b) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"(a), "r"(b));
}

__global__ void __launch_bounds__(kSmThreads) small_gemm_kernel(int m, int n, int k, const uint32_t* __restrict__ A,
                                                                long long lda, const uint32_t* __restrict__ B,
                                                                long long ldb, uint32_t* C, long long ldc, uint32_t p,
                                                                unsigned long long mu, uint32_t two64p,
                                                                uint32_t alpha, uint32_t beta) {
    __shared__ __align__(16) uint32_t As[kSmK][kSmT];  // As[kk][row]
    __shared__ __align__(16) uint32_t Bs[kSmK][kSmT];  // Bs[kk][col]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.y * kSmT, col0 = blockIdx.x * kSmT;
    uint32_t lo[4][4], mid[4][4], hi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) lo[i][j] = mid[i][j] = hi[i][j] = 0u;
    for (int k0 = 0; k0 < k; k0 += kSmK) {
        {
            const int r = tid >> 2, kk0 = (tid & 3) * 8, gi = row0 + r;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int gk = k0 + kk0 + e;
                As[kk0 + e][r] = (gi < m && gk < k) ? __ldg(A + (long long)gi * lda + gk) : 0u;
            }
        }
        {
            const int kk = tid >> 3, c0 = (tid & 7) * 8, gk = k0 + kk;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int gj = col0 + c0 + e;
                Bs[kk][c0 + e] = (gk < k && gj < n) ? __ldg(B + (long long)gk * ldb + gj) : 0u;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kSmK; ++kk) {
            const uint4 a = *reinterpret_cast<const uint4*>(&As[kk][ty * 4]);
            const uint4 b = *reinterpret_cast<const uint4*>(&Bs[kk][tx * 4]);
            const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mac96(lo[i][j], mid[i][j], hi[i][j], av[i], bv[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = row0 + ty * 4 + i;
        if (gi >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = col0 + tx * 4 + j;
            if (gj >= n) continue;
            // (hi 2^64 + mid 2^32 + lo) mod p
            const uint32_t th = mod_u64((unsigned long long)mod_u64(hi[i][j], p, mu) * two64p, p, mu);
            const uint32_t tl = mod_u64(((unsigned long long)mid[i][j] << 32) | lo[i][j], p, mu);
            const uint32_t v = th + tl >= p ? th + tl - p : th + tl;
            uint32_t* cp = C + (long long)gi * ldc + gj;
            const unsigned long long acc =
                (unsigned long long)alpha * v + (beta ? (unsigned long long)beta * (*cp) : 0ull);
            *cp = mod_u64(acc, p, mu);
        }
    }
}

}  // namespace

// Products with m n k at most this many multiply-adds go to the CUDA-core
// kernel by default (the measured crossover with the tensor-core path is near
// 10^8); 0 sends every product to the tensor cores.
static std::atomic<int64_t> g_small_macs{int64_t(1) << 27};

void set_small_threshold(int64_t macs) { g_small_macs.store(macs < 0 ? 0 : macs); }
int64_t small_threshold() { return g_small_macs.load(); }

bool fgemm_small(int64_t m, int64_t n, int64_t k) {
    if (g_tune_override.kernel >= 0) return false;
    const double macs = double(m) * double(n) * double(k);
    return k > 0 && macs <= double(g_small_macs.load()) && k < (int64_t(1) << 31) &&
           m <= int64_t(65535) * kSmT;
}

cudaError_t launch_small_gemm(int64_t m, int64_t n, int64_t k, const uint32_t* A, int64_t lda, const uint32_t* B,
                              int64_t ldb, uint32_t* C, int64_t ldc, uint32_t p, uint32_t alpha, uint32_t beta,
                              cudaStream_t s) {
    if (m == 0 || n == 0) return cudaSuccess;
    const unsigned long long mu = ~0ull / p;
    const uint32_t two64p = (uint32_t)(((unsigned __int128)1 << 64) % p);
    const dim3 grid((unsigned)((n + kSmT - 1) / kSmT), (unsigned)((m + kSmT - 1) / kSmT));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    small_gemm_kernel<<<grid, kSmThreads, 0, s>>>((int)m, (int)n, (int)k, A, lda, B, ldb, C, ldc, p, mu, two64p,
                                                  alpha % p, beta % p);
    return cudaGetLastError();
}

}  // namespace ffgpu
