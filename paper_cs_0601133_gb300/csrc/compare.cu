// Comparison paths for fgemm: the paper's own design carried on GB300's
// floating-point units, exact because the delayed-reduction bound holds.
//
//  * FP64 (DMMA, legacy warp-level mma.sync m8n8k4): residues carried as
//    doubles, the `Zpz-double` representation of section 2.1.2.  Balanced
//    residues |x| <= (p-1)/2 (eq. 2); the accumulator is reduced mod p after
//    every 16-long k-tile, so 16*((p-1)/2)^2 + 1.5p < 2^53: p < 2^25.
//  * FP32 (SIMT FFMA): residues of p <= 256 carried as floats (written once as
//    centred floats); the accumulator is reduced after R products with
//    R*((p-1)/2)^2 + 2p <= 2^24 (eq. 1-2 with gamma = 24 for a sign-magnitude
//    accumulator).
// Both reduce the final value exactly, then C = (alpha*X + beta*C) mod p.
#include <algorithm>

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
// FP32 SIMT.  The operands are first written once as centred residues in
// float (|x| <= (p-1)/2 <= 127, exact), zero-padded to whole tiles: A as
// [mp][kp], B as [kp][np].  The product kernel: block 128 x 128, 256 threads
// of 8 x 8 outputs (rows r4 + {0..3} and 64 + r4 + {0..3}, likewise columns,
// so that the 16-byte shared-memory reads of a warp are conflict-free),
// k-tiles of 16 double-buffered through registers (one barrier per tile),
// the accumulator reduced mod p after every R products (eq. 1-2 with
// gamma = 24, R a multiple of 16).
constexpr int kST = 128, kSK = 16;

__global__ void __launch_bounds__(256) centred_f32_kernel(const uint32_t* __restrict__ X, long long ldx, int rows,
                                                          int cols, int rows_pad, int cols_pad, uint32_t p,
                                                          unsigned long long mu, float* __restrict__ Y) {
    const uint32_t half = p / 2;
    const long long total = (long long)rows_pad * cols_pad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols_pad), c = (int)(e - (long long)r * cols_pad);
        Y[e] = (r < rows && c < cols) ? (float)centred(__ldg(X + (long long)r * ldx + c), p, mu, half) : 0.f;
    }
}

__global__ void __launch_bounds__(256) sgemm_fgemm_kernel(int m, int n, int kp, int np, const float* __restrict__ A,
                                                          const float* __restrict__ B, uint32_t* C, long long ldc,
                                                          uint32_t p, unsigned long long mu, uint32_t al, uint32_t be,
                                                          int reduce_tiles) {
    __shared__ __align__(16) float sA[2][kSK][kST];  // A tile transposed: [k][row]
    __shared__ __align__(16) float sB[2][kSK][kST];  // B tile: [k][col]
    const int tid = threadIdx.x;
    const int r4 = (tid >> 4) * 4, c4 = (tid & 15) * 4;
    const int row0 = blockIdx.y * kST, col0 = blockIdx.x * kST;
    const float pf = (float)p, invp = 1.0f / (float)p;
    // loads of one k-tile: A 128 rows x 16 = 512 float4, B 16 x 128 = 512 float4, two of each per thread
    const int la_r = tid >> 2, la_k = (tid & 3) * 4;        // A: rows la_r and la_r + 64, k la_k..+3
    const int lb_k = tid >> 5, lb_c = (tid & 31) * 4;       // B: k rows lb_k and lb_k + 8, cols lb_c..+3
    const float* pa = A + (long long)(row0 + la_r) * kp + la_k;
    const float* pb = B + (long long)lb_k * np + col0 + lb_c;
    float4 ra0, ra1, rb0, rb1;
    auto load = [&](int k0) {
        ra0 = *reinterpret_cast<const float4*>(pa + k0);
        ra1 = *reinterpret_cast<const float4*>(pa + 64ll * kp + k0);
        rb0 = *reinterpret_cast<const float4*>(pb + (long long)k0 * np);
        rb1 = *reinterpret_cast<const float4*>(pb + (long long)(k0 + 8) * np);
    };
    auto store = [&](int buf) {
        sA[buf][la_k + 0][la_r] = ra0.x;
        sA[buf][la_k + 1][la_r] = ra0.y;
        sA[buf][la_k + 2][la_r] = ra0.z;
        sA[buf][la_k + 3][la_r] = ra0.w;
        sA[buf][la_k + 0][la_r + 64] = ra1.x;
        sA[buf][la_k + 1][la_r + 64] = ra1.y;
        sA[buf][la_k + 2][la_r + 64] = ra1.z;
        sA[buf][la_k + 3][la_r + 64] = ra1.w;
        *reinterpret_cast<float4*>(&sB[buf][lb_k][lb_c]) = rb0;
        *reinterpret_cast<float4*>(&sB[buf][lb_k + 8][lb_c]) = rb1;
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int tiles = kp / kSK;
    load(0);
    store(0);
    __syncthreads();
    int since = 0;
    for (int t = 0; t < tiles; ++t) {
        const int buf = t & 1;
        if (t + 1 < tiles) load((t + 1) * kSK);
#pragma unroll
        for (int kk = 0; kk < kSK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sA[buf][kk][r4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sA[buf][kk][64 + r4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sB[buf][kk][c4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sB[buf][kk][64 + c4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (++since == reduce_tiles) {  // delayed reduction (eq. 1-2 with gamma = 24)
            since = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(-rintf(acc[i][j] * invp), pf, acc[i][j]);
        }
        if (t + 1 < tiles) store(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = row0 + (i < 4 ? r4 + i : 64 + r4 + i - 4);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = col0 + (j < 4 ? c4 + j : 64 + c4 + j - 4);
            const float q = rintf(acc[i][j] * invp);
            int r = (int)fmaf(-q, pf, acc[i][j]);
            r %= (int)p;
            if (r < 0) r += (int)p;
            epilogue_store(C, ldc, row, col, m, n, (uint32_t)r, p, mu, al, be);
        }
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

// Workspace of the FP32 path: the float operands, zero-padded to whole tiles.
size_t sgemm_ws_bytes(int64_t m, int64_t n, int64_t k) {
    const int64_t mp = (m + kST - 1) / kST * kST, np = (n + kST - 1) / kST * kST, kp = (k + kSK - 1) / kSK * kSK;
    return ((size_t(mp) * kp * 4 + 255) & ~size_t(255)) + size_t(kp) * np * 4;
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
                               void* ws, cudaStream_t s) {
    const int mp = (m + kST - 1) / kST * kST, np = (n + kST - 1) / kST * kST, kp = (k + kSK - 1) / kSK * kSK;
    float* Af = static_cast<float*>(ws);
    float* Bf = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) +
                                         ((size_t(mp) * kp * 4 + 255) & ~size_t(255)));
    const unsigned long long mu = ~0ull / p;
    auto blocks = [](long long work) { return (int)std::min<long long>((work + 255) / 256, 152ll * 16); };
    centred_f32_kernel<<<blocks((long long)mp * kp), 256, 0, s>>>(A, lda, m, k, mp, kp, p, mu, Af);
    centred_f32_kernel<<<blocks((long long)kp * np), 256, 0, s>>>(B, ldb, k, n, kp, np, p, mu, Bf);
    dim3 grid(np / kST, mp / kST);
    sgemm_fgemm_kernel<<<grid, 256, 0, s>>>(m, n, kp, np, Af, Bf, C, ldc, p, mu, al, be, sgemm_reduce_tiles(p));
    return cudaGetLastError();
}

}  // namespace ffgpu
