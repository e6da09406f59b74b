// Comparison paths for fgemm: the paper's own design carried on GB300's
// floating-point units, exact because the delayed-reduction bound holds.
//
//  * FP64 (DMMA, legacy warp-level mma.sync m8n8k4): residues carried as
//    doubles, the `Zpz-double` representation of section 2.1.2.  Balanced
//    residues |x| <= (p-1)/2 (eq. 2); the accumulator is reduced mod p after
//    every 16-long k-tile, so 16*((p-1)/2)^2 + 1.5p < 2^53: p < 2^25.
//  * FP32 (SIMT FFMA): residues of p <= 256 carried as floats; the accumulator
//    is reduced after R products with R*((p-1)/2)^2 + p < 2^24 (eq. 1-2 with
//    gamma = 24 for a sign-magnitude accumulator).
// Both reduce the final value exactly, then C = (alpha*X + beta*C) mod p.
#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

__device__ __forceinline__ int centred(uint32_t x, uint32_t p, unsigned long long mu, uint32_t half) {
    const uint32_t r = mod_u64(x, p, mu);
    return r > half ? (int)r - (int)p : (int)r;
}

// canonical residue of an exact integer held in a double, |v| < 2^53
__device__ __forceinline__ uint32_t canon_f64(double v, double pd, double invp, uint32_t p) {
    const double q = rint(v * invp);
    long long r = (long long)fma(-q, pd, v);
    r %= (long long)p;
    if (r < 0) r += p;
    return (uint32_t)r;
}

__device__ __forceinline__ void epilogue_store(uint32_t* C, long long ldc, int row, int col, int m, int n,
                                               uint32_t x, uint32_t p, unsigned long long mu, uint32_t al,
                                               uint32_t be) {
    if (row >= m || col >= n) return;
    uint32_t* ptr = C + (long long)row * ldc + col;
    const unsigned long long old = be ? *ptr : 0u;
    *ptr = mod_u64((unsigned long long)al * x + (unsigned long long)be * old, p, mu);
}

// ---------------------------------------------------------------------------
// FP64 DMMA: block 64 x 64, 4 warps of 32 x 32 (4 x 4 fragments of 8 x 8), k-tile 16.
// mma.m8n8k4.f64 fragments: A one element (row = lane/4, col = lane%4), B one
// element (row = lane%4, col = lane/4), C two (row = lane/4, cols 2*(lane%4)+{0,1}).
constexpr int kDT = 64, kDK = 16;

__global__ void __launch_bounds__(128) dmma_fgemm_kernel(int m, int n, int k, const uint32_t* __restrict__ A,
                                                         long long lda, const uint32_t* __restrict__ B,
                                                         long long ldb, uint32_t* C, long long ldc, uint32_t p,
                                                         unsigned long long mu, uint32_t al, uint32_t be) {
    __shared__ double sA[kDT][kDK + 1];
    __shared__ double sB[kDK][kDT + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wr = (warp >> 1) * 32, wc = (warp & 1) * 32;
    const int g = lane >> 2, t4 = lane & 3;
    const int row0 = blockIdx.y * kDT, col0 = blockIdx.x * kDT;
    const uint32_t half = p / 2;
    const double pd = (double)p, invp = 1.0 / (double)p;
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    for (int k0 = 0; k0 < k; k0 += kDK) {
        for (int idx = threadIdx.x; idx < kDT * kDK; idx += 128) {
            const int r = idx / kDK, c = idx % kDK;
            const int gr = row0 + r, gc = k0 + c;
            sA[r][c] = (gr < m && gc < k) ? (double)centred(A[(long long)gr * lda + gc], p, mu, half) : 0.0;
        }
        for (int idx = threadIdx.x; idx < kDK * kDT; idx += 128) {
            const int r = idx / kDT, c = idx % kDT;
            const int gr = k0 + r, gc = col0 + c;
            sB[r][c] = (gr < k && gc < n) ? (double)centred(B[(long long)gr * ldb + gc], p, mu, half) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kDK; kk += 4) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[wr + i * 8 + g][kk + t4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk + t4][wc + j * 8 + g];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                        : "+d"(acc[i][j][0]), "+d"(acc[i][j][1])
                        : "d"(a[i]), "d"(b[j]));
        }
        // delayed reduction: keep |acc| <= 1.5 p before the next k-tile
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) acc[i][j][e] = fma(-rint(acc[i][j][e] * invp), pd, acc[i][j][e]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int row = row0 + wr + i * 8 + g;
                const int col = col0 + wc + j * 8 + 2 * t4 + e;
                epilogue_store(C, ldc, row, col, m, n, canon_f64(acc[i][j][e], pd, invp, p), p, mu, al, be);
            }
}

// ---------------------------------------------------------------------------
// FP32 SIMT: block 128 x 128, 256 threads of 8 x 8 outputs, k-tile 8.
constexpr int kST = 128, kSK = 8;

__global__ void __launch_bounds__(256) sgemm_fgemm_kernel(int m, int n, int k, const uint32_t* __restrict__ A,
                                                          long long lda, const uint32_t* __restrict__ B,
                                                          long long ldb, uint32_t* C, long long ldc, uint32_t p,
                                                          unsigned long long mu, uint32_t al, uint32_t be,
                                                          int reduce_tiles) {
    __shared__ float sA[kSK][kST];
    __shared__ float sB[kSK][kST];
    const int tr = (threadIdx.x >> 4) * 8, tc = (threadIdx.x & 15) * 8;
    const int row0 = blockIdx.y * kST, col0 = blockIdx.x * kST;
    const uint32_t half = p / 2;
    const float pf = (float)p, invp = 1.0f / (float)p;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    int since = 0;
    for (int k0 = 0; k0 < k; k0 += kSK) {
        for (int idx = threadIdx.x; idx < kST * kSK; idx += 256) {
            const int r = idx / kSK, c = idx % kSK;
            const int gr = row0 + r, gc = k0 + c;
            sA[c][r] = (gr < m && gc < k) ? (float)centred(A[(long long)gr * lda + gc], p, mu, half) : 0.f;
            const int br = k0 + (idx / kST), bc = col0 + (idx % kST);
            sB[idx / kST][idx % kST] =
                (br < k && bc < n) ? (float)centred(B[(long long)br * ldb + bc], p, mu, half) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kSK; ++kk) {
            float a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = sA[kk][tr + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = sB[kk][tc + j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
        if (++since == reduce_tiles) {  // delayed reduction (eq. 1 with gamma = 24)
            since = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(-rintf(acc[i][j] * invp), pf, acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float q = rintf(acc[i][j] * invp);
            int r = (int)fmaf(-q, pf, acc[i][j]);
            r %= (int)p;
            if (r < 0) r += (int)p;
            epilogue_store(C, ldc, row0 + tr + i, col0 + tc + j, m, n, (uint32_t)r, p, mu, al, be);
        }
}

}  // namespace

// Largest p each comparison path computes exactly (see the bounds above).
uint32_t dmma_max_p() { return (1u << 25) - 1; }
uint32_t sgemm_max_p() { return 256u; }

// Number of k-tiles (of 8) the FP32 path may sum before a reduction.
int sgemm_reduce_tiles(uint32_t p) {
    const long long h = p / 2;
    long long R = ((1ll << 24) - 2 * (long long)p) / (h * h > 0 ? h * h : 1);
    if (R > (1ll << 20)) R = 1ll << 20;
    const int tiles = (int)(R / kSK);
    return tiles < 1 ? 1 : tiles;
}

cudaError_t launch_dmma_fgemm(int m, int n, int k, const uint32_t* A, long long lda, const uint32_t* B,
                              long long ldb, uint32_t* C, long long ldc, uint32_t p, uint32_t al, uint32_t be,
                              cudaStream_t s) {
    dim3 grid((n + kDT - 1) / kDT, (m + kDT - 1) / kDT);
    dmma_fgemm_kernel<<<grid, 128, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, p, ~0ull / p, al, be);
    return cudaGetLastError();
}

cudaError_t launch_sgemm_fgemm(int m, int n, int k, const uint32_t* A, long long lda, const uint32_t* B,
                               long long ldb, uint32_t* C, long long ldc, uint32_t p, uint32_t al, uint32_t be,
                               cudaStream_t s) {
    dim3 grid((n + kST - 1) / kST, (m + kST - 1) / kST);
    sgemm_fgemm_kernel<<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, p, ~0ull / p, al, be,
                                             sgemm_reduce_tiles(p));
    return cudaGetLastError();
}

}  // namespace ffgpu
