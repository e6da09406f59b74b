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
// 256 threads with 4 x 4 outputs each, k staged 32 at a time through two
// shared-memory buffers (32 x 32 tiles with 64 threads for the batched
// launch's products with a dimension of at most 32).  When the tiles leave SMs idle, k is split (the
// rule and its measurements are at small_splits): each split writes its exact
// 96-bit partial sums to the workspace and a second kernel adds them, reduces
// mod p and applies alpha and beta (C is then written only after every read
// of A and B).
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

// (hi 2^64 + mid 2^32 + lo) mod p, then alpha v + beta c mod p
__device__ __forceinline__ uint32_t finish96(uint32_t lo, uint32_t mid, uint32_t hi, uint32_t c, uint32_t p,
                                             unsigned long long mu, uint32_t two64p, uint32_t alpha, uint32_t beta) {
    const uint32_t th = mod_u64((unsigned long long)mod_u64(hi, p, mu) * two64p, p, mu);
    const uint32_t tl = mod_u64(((unsigned long long)mid << 32) | lo, p, mu);
    const uint32_t v = th + tl >= p ? th + tl - p : th + tl;
    const unsigned long long acc = (unsigned long long)alpha * v + (unsigned long long)beta * c;
    return mod_u64(acc, p, mu);
}

// One T x T output tile (rows row0.., columns col0..) over the k-range
// [kbeg, kend), T * T / 16 threads with 4 x 4 outputs each: with part null
// it finishes the outputs itself, else it stores its partial sums at part
// (uint4 per output: lo, mid, hi, 0; m x n).  The k chunks are staged in two
// shared-memory buffers by asynchronous copies (words outside the matrices
// arrive as zeros), the next chunk's copies in flight while the current one
// is multiplied.
__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int T, bool kTrimK>
__device__ __forceinline__ void small_tile(int m, int n, int kbeg, int kend, int row0, int col0,
                                           const uint32_t* __restrict__ A, long long lda,
                                           const uint32_t* __restrict__ B, long long ldb, uint32_t* C, long long ldc,
                                           uint4* __restrict__ part, uint32_t p, unsigned long long mu,
                                           uint32_t two64p, uint32_t alpha, uint32_t beta) {
    constexpr int NT = T * T / 16;       // threads
    constexpr int PER = T * kSmK / NT;   // staged words per thread and operand (8 for T = 64, 16 for T = 32)
    __shared__ __align__(16) uint32_t As[2][kSmK][T];  // As[buf][kk][row]
    __shared__ __align__(16) uint32_t Bs[2][kSmK][T];  // Bs[buf][kk][col]
    const int tid = threadIdx.x, tx = tid % (T / 4), ty = tid / (T / 4);
    uint32_t lo[4][4], mid[4][4], hi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) lo[i][j] = mid[i][j] = hi[i][j] = 0u;
    // A: row r, k-run of PER words; B: k row kk, column run of PER words
    const int ar = tid / (kSmK / PER), akk0 = (tid % (kSmK / PER)) * PER, agi = row0 + ar;
    const int bkk = tid / (T / PER), bc0 = (tid % (T / PER)) * PER;
    auto stage = [&](int buf, int k0) {
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int gk = k0 + akk0 + e;
            const bool ok = agi < m && gk < kend;
            cp_async4(&As[buf][akk0 + e][ar], ok ? A + (long long)agi * lda + gk : A, ok);
        }
        const int gk = k0 + bkk;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int gj = col0 + bc0 + e;
            const bool ok = gk < kend && gj < n;
            cp_async4(&Bs[buf][bkk][bc0 + e], ok ? B + (long long)gk * ldb + gj : B, ok);
        }
        cp_async_commit();
    };
    if (kbeg < kend) stage(0, kbeg);
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += kSmK, buf ^= 1) {
        if (k0 + kSmK < kend) {
            stage(buf ^ 1, k0 + kSmK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        auto step = [&](int kk) {
            const uint4 a = *reinterpret_cast<const uint4*>(&As[buf][kk][ty * 4]);
            const uint4 b = *reinterpret_cast<const uint4*>(&Bs[buf][kk][tx * 4]);
            const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mac96(lo[i][j], mid[i][j], hi[i][j], av[i], bv[j]);
        };
        if (!kTrimK || kend - k0 >= kSmK) {
#pragma unroll 4
            for (int kk = 0; kk < kSmK; ++kk) step(kk);
        } else {
            // kTrimK: the last, partial chunk takes only its words (the rest
            // are zeros), which pays where most products have a ragged k
#pragma unroll 4
            for (int kk = 0; kk < kend - k0; ++kk) step(kk);
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
            if (part) {
                part[(long long)gi * n + gj] = make_uint4(lo[i][j], mid[i][j], hi[i][j], 0u);
            } else {
                uint32_t* cp = C + (long long)gi * ldc + gj;
                *cp = finish96(lo[i][j], mid[i][j], hi[i][j], beta ? *cp : 0u, p, mu, two64p, alpha, beta);
            }
        }
    }
}

// Split s = blockIdx.z sums k-range [s kps, (s + 1) kps); with part null it
// finishes the outputs itself, else it stores its partial sums there
// (split-major, m x n each).
__global__ void __launch_bounds__(kSmThreads) small_gemm_kernel(int m, int n, int k, int kps,
                                                                const uint32_t* __restrict__ A, long long lda,
                                                                const uint32_t* __restrict__ B, long long ldb,
                                                                uint32_t* C, long long ldc, uint4* __restrict__ part,
                                                                uint32_t p, unsigned long long mu, uint32_t two64p,
                                                                uint32_t alpha, uint32_t beta) {
    const int kbeg = blockIdx.z * kps, kend = min(k, kbeg + kps);
    small_tile<kSmT, false>(m, n, kbeg, kend, blockIdx.y * kSmT, blockIdx.x * kSmT, A, lda, B, ldb, C, ldc,
                     part ? part + (long long)blockIdx.z * m * n : nullptr, p, mu, two64p, alpha, beta);
}

// Many independent small products in one launch: CTA t computes tile
// t - jobs[j].tile0 of job j = tile_job[t] (row-major over the job's T x T
// tiles).
template <int T>
__global__ void __launch_bounds__(T * T / 16) small_grouped_kernel(const SmallJob* __restrict__ jobs,
                                                                   const int* __restrict__ tile_job) {
    const int t = blockIdx.x;
    const SmallJob& J = jobs[tile_job[t]];
    const int local = t - J.tile0;
    const int tr = local / J.tiles_n, tc = local - tr * J.tiles_n;
    small_tile<T, true>(J.m, J.n, 0, J.k, tr * T, tc * T, J.A, J.lda, J.B, J.ldb, J.C, J.ldc, nullptr, J.p, J.mu,
                  J.two64p, J.alpha, J.beta);
}

// Sum of the splits' partial sums (below k 2^64 < 2^96, so three words and
// their carries suffice), then the reduction and alpha, beta.
__global__ void __launch_bounds__(kSmThreads) small_reduce_kernel(int m, int n, int splits,
                                                                  const uint4* __restrict__ part, uint32_t* C,
                                                                  long long ldc, uint32_t p, unsigned long long mu,
                                                                  uint32_t two64p, uint32_t alpha, uint32_t beta) {
    const long long total = (long long)m * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        uint32_t lo = 0u, mid = 0u, hi = 0u;
        for (int z = 0; z < splits; ++z) {
            const uint4 q = __ldg(part + z * total + e);
            asm("add.cc.u32 %0, %0, %3;\n\t"
                "addc.cc.u32 %1, %1, %4;\n\t"
                "addc.u32 %2, %2, %5;"
                : "+r"(lo), "+r"(mid), "+r"(hi)
                : "r"(q.x), "r"(q.y), "r"(q.z));
        }
        const int gi = (int)(e / n), gj = (int)(e - (long long)gi * n);
        uint32_t* cp = C + (long long)gi * ldc + gj;
        *cp = finish96(lo, mid, hi, beta ? *cp : 0u, p, mu, two64p, alpha, beta);
    }
}

// Number of k-splits for a product (at most 16, each at least one 32-long
// chunk).  A split costs the partial sums' round trip and a second launch, so
// k is split only while the CTAs still fit one per SM, and past half the SMs
// only when every split keeps at least two chunks.  Measured per product on
// one GPU (us, 256 threads; s = splits): 64x4096x64 s1 14.4 / s2 16.4,
// 64x2048x64 16.4 / 14.3, 128x2048x128 s1 22.6 / s2 20.5, 128x4096x128
// 22.6 / 29.7, 128x8192x128 36.9 / 52.1, 256^3 s1 38.9 / s4 16.5 / s8 15.4,
// 512^3 s1 69.7 / s2 43.0 / s4 41.0, 64x64x2048 s1 253 / s16 26.7; the rule
// this replaced (split until two waves of CTAs) took the slower choice for
// every product of 64 to 256 tiles.
int small_splits(int64_t m, int64_t n, int64_t k, int sms) {
    const int64_t tiles = ((m + kSmT - 1) / kSmT) * ((n + kSmT - 1) / kSmT);
    const int64_t chunks = (k + kSmK - 1) / kSmK;
    int s = 1;
    while (s < 16 && 2 * s <= chunks && tiles * 2 * s <= sms && (tiles * 4 * s <= sms || 4 * s <= chunks)) s *= 2;
    return s;
}

}  // namespace

// Products with m n k at most this many multiply-adds go to the CUDA-core
// kernel by default (the measured crossover with the tensor-core path is near
// 10^8); 0 sends every product to the tensor cores.
static std::atomic<int64_t> g_small_macs{int64_t(1) << 27};

void set_small_threshold(int64_t macs) { g_small_macs.store(macs < 0 ? 0 : macs); }
int64_t small_threshold() { return g_small_macs.load(); }

bool fgemm_small(int64_t m, int64_t n, int64_t k) {
    const bool fits = k > 0 && k < (int64_t(1) << 31) && m <= int64_t(65535) * kSmT;
    if (g_tune_override.route >= 0) return fits && g_tune_override.route == 1;  // a tuned plan's route
    if (g_tune_override.kernel >= 0) return false;
    const double macs = double(m) * double(n) * double(k);
    return fits && macs <= double(g_small_macs.load());
}

void small_job(SmallJob& J, const ffgpu_fgemm_desc& d, int tile0, int tile) {
    J.A = d.A;
    J.B = d.B;
    J.C = d.C;
    J.lda = d.lda;
    J.ldb = d.ldb;
    J.ldc = d.ldc;
    J.mu = ~0ull / d.p;
    J.m = (int)d.m;
    J.n = (int)d.n;
    J.k = (int)d.k;
    J.tiles_n = (int)((d.n + tile - 1) / tile);
    J.tile0 = tile0;
    J.p = d.p;
    J.alpha = d.alpha % d.p;
    J.beta = d.beta % d.p;
    J.two64p = (uint32_t)(((unsigned __int128)1 << 64) % d.p);
}

int64_t small_tiles(int64_t m, int64_t n, int tile) { return ((m + tile - 1) / tile) * ((n + tile - 1) / tile); }

// tile 64 (256 threads) or 32 (64 threads)
cudaError_t launch_small_grouped(const SmallJob* jobs, const int* tile_job, int64_t tiles, int tile, cudaStream_t s) {
    if (tiles == 0) return cudaSuccess;
    if (tiles > INT32_MAX || (tile != 32 && tile != 64)) return cudaErrorInvalidConfiguration;
    if (tile == 64)
        small_grouped_kernel<64><<<(unsigned)tiles, 256, 0, s>>>(jobs, tile_job);
    else
        small_grouped_kernel<32><<<(unsigned)tiles, 64, 0, s>>>(jobs, tile_job);
    return cudaGetLastError();
}

size_t small_ws_bytes(int64_t m, int64_t n, int64_t k, int sms) {
    const int sp = small_splits(m, n, k, sms);
    return sp > 1 ? size_t(sp) * m * n * sizeof(uint4) : 0;
}

cudaError_t launch_small_gemm(int64_t m, int64_t n, int64_t k, const uint32_t* A, int64_t lda, const uint32_t* B,
                              int64_t ldb, uint32_t* C, int64_t ldc, uint32_t p, uint32_t alpha, uint32_t beta,
                              void* ws, size_t ws_bytes, int sms, cudaStream_t s) {
    if (m == 0 || n == 0) return cudaSuccess;
    const unsigned long long mu = ~0ull / p;
    const uint32_t two64p = (uint32_t)(((unsigned __int128)1 << 64) % p);
    int sp = small_splits(m, n, k, sms);
    if (sp > 1 && (!ws || size_t(sp) * m * n * sizeof(uint4) > ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 15)))
        sp = 1;
    const int64_t chunks = (k + kSmK - 1) / kSmK;
    const int kps = (int)(((chunks + sp - 1) / sp) * kSmK);
    const dim3 grid((unsigned)((n + kSmT - 1) / kSmT), (unsigned)((m + kSmT - 1) / kSmT), (unsigned)sp);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    uint4* part = sp > 1 ? static_cast<uint4*>(ws) : nullptr;
    small_gemm_kernel<<<grid, kSmThreads, 0, s>>>((int)m, (int)n, (int)k, kps, A, lda, B, ldb, C, ldc, part, p, mu,
                                                  two64p, alpha % p, beta % p);
    if (sp > 1) {
        const long long blocks = std::min<long long>((m * n + kSmThreads - 1) / kSmThreads, (long long)sms * 8);
        small_reduce_kernel<<<(unsigned)blocks, kSmThreads, 0, s>>>((int)m, (int)n, sp, part, C, ldc, p, mu, two64p,
                                                                    alpha % p, beta % p);
    }
    return cudaGetLastError();
}

}  // namespace ffgpu
