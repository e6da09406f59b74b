// Conversion of uint32 words into bf16 channel planes, and small elementwise
// kernels mod p.  All of them are HBM-bound.
//
// The conversion is the "few conversions" step the paper keeps out of the
// product (section 1 and section 2.1.2: a residue is embedded in Z, here as a
// centred representative, eq. 2): x -> x mod p -> centred x~ in
// [-(p-1)/2, p/2] -> for each odd modulus m_c the balanced residue of
// x~ mod m_c in [-(m_c-1)/2, (m_c-1)/2], written as an exact bf16.  With a
// single modulus (p <= 255) the plane holds x~ itself.  Rows are padded with zeros to a multiple of 64
// columns so every tensor-core tile sees whole 128-byte rows.
#include <cuda_bf16.h>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

// Residues of 8 words in every channel, packed 8 x bf16 per channel and
// stored at dst[c * stride16].
//   x mod p: 32-bit Barrett (quotient estimate umulhi(x, floor((2^32-1)/p)) is
//            at most one below, one correction);
//   centring: x~ = x mod p if <= floor(p/2), else -(p - x mod p); kept as a
//            magnitude y and a sign;
//   balanced residue of y mod m: q = floor((y + (m-1)/2) / m) by a 32-bit
//            magic multiply (magic = ceil(2^39/m), exact for y < 2^31 and
//            m <= 255), r = y - q m in [-(m-1)/2, (m-1)/2]; the sign of x~ is
//            applied to the bf16 pattern (negation flips its sign bit).
__device__ __forceinline__ void residues8(const ConvertParams& cp, const uint32_t (&x)[8],
                                          uint4* __restrict__ dst, size_t stride16) {
    uint32_t y[8];
    uint32_t sign[4];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        bool neg;
        if (cp.signed_input) {  // integer mode: the signed word itself, as magnitude and sign
            const int32_t v = (int32_t)x[e];
            neg = v < 0;
            y[e] = neg ? 0u - x[e] : x[e];
        } else {
            const uint32_t q = __umulhi(x[e], cp.mu32);
            uint32_t r = x[e] - q * cp.p;
            if (r >= cp.p) r -= cp.p;
            neg = r > cp.half_p;
            y[e] = neg ? cp.p - r : r;
        }
        if ((e & 1) == 0) sign[e >> 1] = neg ? 0x8000u : 0u;
        else sign[e >> 1] |= neg ? 0x80000000u : 0u;
    }
    if (cp.direct) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 b = __floats2bfloat162_rn((float)y[2 * i], (float)y[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t*>(&b) ^ sign[i];
        }
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        return;
    }
#pragma unroll 1
    for (int c = 0; c < cp.nch; ++c) {
        const uint32_t m = cp.mod[c], mg = cp.magic32[c], h = (m - 1) >> 1;
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float f[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const uint32_t v = y[2 * i + t];
                const uint32_t q = __umulhi(v + h, mg) >> 7;
                f[t] = (float)(int)(v - q * m);
            }
            const __nv_bfloat162 b = __floats2bfloat162_rn(f[0], f[1]);
            w[i] = *reinterpret_cast<const uint32_t*>(&b) ^ sign[i];
        }
        dst[(size_t)c * stride16] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Rows [r_begin, r_end) of X (rows x cols, ldx) -> planes[c][r][colsp]; rows
// at or past `rows` (padding up to a tile multiple) are written as zeros.
__device__ __forceinline__ void convert_rows_range(const uint32_t* __restrict__ X, long long ldx, int rows,
                                                   int cols, int colsp, int r_begin, int r_end,
                                                   const ConvertParams& cp, uint4* __restrict__ planes,
                                                   size_t plane16, int vec_ok, long long tid,
                                                   long long nthreads) {
    const long long gpr = colsp / 8;
    const long long total = (long long)(r_end - r_begin) * gpr;
    for (long long g = tid; g < total; g += nthreads) {
        const int r = r_begin + (int)(g / gpr);
        const int c0 = (int)(g % gpr) * 8;
        uint32_t x[8];
        if (r >= rows) {
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = 0u;
        } else {
            const uint32_t* src = X + (long long)r * ldx + c0;
            if (vec_ok && c0 + 8 <= cols) {
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(src));
                const uint4 b = __ldg(reinterpret_cast<const uint4*>(src) + 1);
                x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
                x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] = (c0 + e < cols) ? __ldg(src + e) : 0u;
            }
        }
        residues8(cp, x, planes + ((size_t)r * colsp + c0) / 8, plane16);
    }
}

// X: rows x cols (ldx) -> planes[c][rows][colsp], colsp a multiple of 64.
__global__ void __launch_bounds__(256) convert_rows_kernel(const uint32_t* __restrict__ X, long long ldx,
                                                           int rows, int cols, int colsp,
                                                           const __grid_constant__ ConvertParams cp,
                                                           uint4* __restrict__ planes, int vec_ok) {
    const size_t plane16 = (size_t)rows * colsp / 8;  // plane size in 16-byte units
    convert_rows_range(X, ldx, rows, cols, colsp, 0, rows, cp, planes, plane16, vec_ok,
                       blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// One 64 x 64 tile (rows [r0, r0+64) = inner dimension, columns [c0, c0+64))
// of X (rows x cols, ldx) -> planes[c][col][rowsp] (transposed so that the
// inner dimension is contiguous).  Columns at or past `cols` up to cols_pad are
// written as zeros.
__device__ __forceinline__ void convert_transpose_tile(const uint32_t* __restrict__ X, long long ldx, int rows,
                                                       int cols, int cols_pad, int rowsp, int r0, int c0,
                                                       const ConvertParams& cp, uint4* __restrict__ planes,
                                                       size_t plane16, uint32_t (*tile)[65]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int idx = threadIdx.x + 256 * i;
        const int rr = idx >> 6, cc = idx & 63;
        const int gr = r0 + rr, gc = c0 + cc;
        tile[rr][cc] = (gr < rows && gc < cols) ? __ldg(X + (long long)gr * ldx + gc) : 0u;
    }
    __syncthreads();
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
        const int w = threadIdx.x + 256 * it;
        const int cl = w >> 3, g = w & 7;
        const int gc = c0 + cl;
        if (gc >= cols_pad) continue;
        uint32_t x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = tile[g * 8 + e][cl];
        residues8(cp, x, planes + ((size_t)gc * rowsp + r0 + g * 8) / 8, plane16);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) convert_transpose_kernel(const uint32_t* __restrict__ X,
                                                                long long ldx, int rows, int cols,
                                                                int rowsp,
                                                                const __grid_constant__ ConvertParams cp,
                                                                uint4* __restrict__ planes) {
    __shared__ uint32_t tile[64][65];
    convert_transpose_tile(X, ldx, rows, cols, cols, rowsp, blockIdx.y * 64, blockIdx.x * 64, cp, planes,
                           (size_t)cols * rowsp / 8, tile);
}

// Grouped conversions: block b serves the instance i with
// block_begin[i] <= b < block_begin[i+1] (binary search).
__device__ __forceinline__ int find_job(const long long* __restrict__ block_begin, int njobs, long long b) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (block_begin[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kRowsPerGroupedBlock = 16;

__global__ void __launch_bounds__(256) convert_rows_grouped_kernel(const ConvJob* __restrict__ jobs,
                                                                   const long long* __restrict__ block_begin,
                                                                   int njobs) {
    const int i = find_job(block_begin, njobs, blockIdx.x);
    const ConvJob& J = jobs[i];
    const int lb = (int)(blockIdx.x - block_begin[i]);
    const int r_begin = lb * kRowsPerGroupedBlock;
    const int r_end = min(J.rows_pad, r_begin + kRowsPerGroupedBlock);
    convert_rows_range(J.X, J.ldx, J.rows, J.cols, J.kp, r_begin, r_end, J.cp, J.dst, J.plane16, J.vec_ok,
                       threadIdx.x, blockDim.x);
}

__global__ void __launch_bounds__(256) convert_transpose_grouped_kernel(const ConvJob* __restrict__ jobs,
                                                                        const long long* __restrict__ block_begin,
                                                                        int njobs) {
    __shared__ uint32_t tile[64][65];
    const int i = find_job(block_begin, njobs, blockIdx.x);
    const ConvJob& J = jobs[i];
    const int lb = (int)(blockIdx.x - block_begin[i]);
    const int tiles_c = (J.rows_pad + 63) / 64;   // output rows (columns of B), padded
    const int tc = lb % tiles_c, tk = lb / tiles_c;
    // B: rows = k (inner dimension), cols = n, rows_pad = n padded, kp = k padded
    convert_transpose_tile(J.X, J.ldx, J.rows, J.cols, J.rows_pad, J.kp, tk * 64, tc * 64, J.cp, J.dst,
                           J.plane16, tile);
}

__global__ void __launch_bounds__(256) scale_kernel(uint32_t* C, long long ldc, int m, int n, uint32_t p,
                                                    uint32_t beta, unsigned long long mu) {
    const long long total = (long long)m * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / n), c = (int)(i - (long long)r * n);
        uint32_t* ptr = C + (long long)r * ldc + c;
        *ptr = mod_u64((unsigned long long)beta * (*ptr), p, mu);
    }
}

// The word at (r, c) of a signed sum of blocks, reduced mod p: each term's
// word reduced by the 32-bit Barrett step of residues8, added (or its
// negative added) modulo p; the result is a canonical residue.
__device__ __forceinline__ uint32_t sum_at(const SumSrc& S, long long r, int c, uint32_t p, uint32_t mu32) {
    uint32_t acc = 0u;
    for (int t = 0; t < S.n; ++t) {
        const uint32_t x = __ldg(S.X[t] + r * S.ld[t] + c);
        const uint32_t q = __umulhi(x, mu32);
        uint32_t v = x - q * p;
        if (v >= p) v -= p;
        if (S.neg[t] && v != 0u) v = p - v;
        acc += v;  // both below p < 2^31: no wrap
        if (acc >= p) acc -= p;
    }
    return acc;
}

__global__ void __launch_bounds__(256) convert_rows_sum_kernel(const __grid_constant__ SumSrc S, int rows, int cols,
                                                               int colsp, const __grid_constant__ ConvertParams cp,
                                                               uint4* __restrict__ planes) {
    const size_t plane16 = (size_t)rows * colsp / 8;
    const long long gpr = colsp / 8;
    const long long total = (long long)rows * gpr;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(g / gpr);
        const int c0 = (int)(g % gpr) * 8;
        uint32_t x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = (c0 + e < cols) ? sum_at(S, r, c0 + e, cp.p, cp.mu32) : 0u;
        residues8(cp, x, planes + ((size_t)r * colsp + c0) / 8, plane16);
    }
}

__global__ void __launch_bounds__(256) convert_transpose_sum_kernel(const __grid_constant__ SumSrc S, int rows,
                                                                    int cols, int rowsp,
                                                                    const __grid_constant__ ConvertParams cp,
                                                                    uint4* __restrict__ planes) {
    __shared__ uint32_t tile[64][65];
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
#pragma unroll 1
    for (int i = 0; i < 16; ++i) {
        const int idx = threadIdx.x + 256 * i;
        const int rr = idx >> 6, cc = idx & 63;
        const int gr = r0 + rr, gc = c0 + cc;
        tile[rr][cc] = (gr < rows && gc < cols) ? sum_at(S, gr, gc, cp.p, cp.mu32) : 0u;
    }
    __syncthreads();
    const size_t plane16 = (size_t)cols * rowsp / 8;
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
        const int w = threadIdx.x + 256 * it;
        const int cl = w >> 3, g = w & 7;
        const int gc = c0 + cl;
        if (gc >= cols) continue;
        uint32_t x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = tile[g * 8 + e][cl];
        residues8(cp, x, planes + ((size_t)gc * rowsp + r0 + g * 8) / 8, plane16);
    }
}

__global__ void __launch_bounds__(256) sum_mod_kernel(const __grid_constant__ SumSrc S, int rows, int cols,
                                                      uint32_t p, uint32_t mu32, uint32_t* __restrict__ Z,
                                                      long long ldz) {
    const long long total = (long long)rows * cols;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(g / cols), c = (int)(g - (long long)r * cols);
        Z[(long long)r * ldz + c] = sum_at(S, r, c, p, mu32);
    }
}

int grid_for(long long work, int per_block) {
    long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

cudaError_t launch_convert_rows(const uint32_t* X, long long ldx, int rows, int cols, int colsp,
                                const ConvertParams& cp, void* planes, cudaStream_t s) {
    if (rows == 0 || colsp == 0) return cudaSuccess;
    const int vec_ok = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 4 == 0);
    const long long work = (long long)rows * (colsp / 8);
    convert_rows_kernel<<<grid_for(work, 256), 256, 0, s>>>(X, ldx, rows, cols, colsp, cp,
                                                             static_cast<uint4*>(planes), vec_ok);
    return cudaGetLastError();
}

cudaError_t launch_convert_transpose(const uint32_t* X, long long ldx, int rows, int cols, int rowsp,
                                     const ConvertParams& cp, void* planes, cudaStream_t s) {
    if (cols == 0 || rowsp == 0) return cudaSuccess;
    dim3 grid((cols + 63) / 64, rowsp / 64);
    convert_transpose_kernel<<<grid, 256, 0, s>>>(X, ldx, rows, cols, rowsp, cp,
                                                   static_cast<uint4*>(planes));
    return cudaGetLastError();
}

cudaError_t launch_convert_rows_sum(const SumSrc& X, int rows, int cols, int colsp, const ConvertParams& cp,
                                    void* planes, cudaStream_t s) {
    if (rows == 0 || colsp == 0) return cudaSuccess;
    const long long work = (long long)rows * (colsp / 8);
    convert_rows_sum_kernel<<<grid_for(work, 256), 256, 0, s>>>(X, rows, cols, colsp, cp, static_cast<uint4*>(planes));
    return cudaGetLastError();
}

cudaError_t launch_convert_transpose_sum(const SumSrc& X, int rows, int cols, int rowsp, const ConvertParams& cp,
                                         void* planes, cudaStream_t s) {
    if (cols == 0 || rowsp == 0) return cudaSuccess;
    dim3 grid((cols + 63) / 64, rowsp / 64);
    convert_transpose_sum_kernel<<<grid, 256, 0, s>>>(X, rows, cols, rowsp, cp, static_cast<uint4*>(planes));
    return cudaGetLastError();
}

cudaError_t launch_sum_mod(const SumSrc& X, int rows, int cols, uint32_t p, uint32_t* Z, long long ldz,
                           cudaStream_t s) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    sum_mod_kernel<<<grid_for((long long)rows * cols, 256), 256, 0, s>>>(X, rows, cols, p, 0xFFFFFFFFu / p, Z, ldz);
    return cudaGetLastError();
}

long long convert_rows_grouped_blocks(int rows_pad) {
    return (rows_pad + kRowsPerGroupedBlock - 1) / kRowsPerGroupedBlock;
}
long long convert_transpose_grouped_blocks(int cols_pad, int kp) { return (long long)((cols_pad + 63) / 64) * (kp / 64); }

cudaError_t launch_convert_rows_grouped(const ConvJob* jobs, const long long* block_begin, int njobs,
                                        long long nblocks, cudaStream_t s) {
    if (njobs == 0 || nblocks == 0) return cudaSuccess;
    convert_rows_grouped_kernel<<<(unsigned)nblocks, 256, 0, s>>>(jobs, block_begin, njobs);
    return cudaGetLastError();
}

cudaError_t launch_convert_transpose_grouped(const ConvJob* jobs, const long long* block_begin, int njobs,
                                             long long nblocks, cudaStream_t s) {
    if (njobs == 0 || nblocks == 0) return cudaSuccess;
    convert_transpose_grouped_kernel<<<(unsigned)nblocks, 256, 0, s>>>(jobs, block_begin, njobs);
    return cudaGetLastError();
}

cudaError_t launch_scale(uint32_t* C, long long ldc, int m, int n, uint32_t p, uint32_t beta,
                         unsigned long long mu, cudaStream_t s) {
    if (m == 0 || n == 0) return cudaSuccess;
    scale_kernel<<<grid_for((long long)m * n, 256), 256, 0, s>>>(C, ldc, m, n, p, beta, mu);
    return cudaGetLastError();
}

}  // namespace ffgpu
