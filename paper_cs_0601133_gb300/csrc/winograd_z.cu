// Winograd's algorithm without modular reduction (section 3.2): l recursive
// levels of the Table 2 schedule computed over Z, one reduction mod p at the
// very end, admitted only when Theorem 3.1 shows that no intermediate value
// leaves the exact range of the integer carrier.
//
// The paper's carrier is a double (exact integers below 2^53); here it is
// int64: the operands are balanced residues (|x| <= (p-1)/2, Corollary 3.3)
// in int32, the pre-additions stay in int32 (one level's operand is a sum of
// at most four entries -- S4 = A11 + A12 - A21 - A22 -- so after l levels it is
// at most 4^l (p-1)/2 in magnitude), the products are exact int64 dot
// products and the post-additions int64 sums.  Theorem 3.1
// bounds every intermediate value -- partial dot products included -- by
// (3^l (p-1)/2)^2 floor(k / 2^l) for balanced inputs; the routine requires
// that bound below 2^62 (Corollary 3.4 with gamma = 62) and 4^l (p-1)/2
// below 2^31.  Odd dimensions are peeled as in the appendix (the even block
// by Winograd, then a rank-1 update, a matrix-vector and a vector-matrix
// product).  alpha and beta are applied with the final reduction:
// C = (alpha (A B mod p) + beta C) mod p.
//
// Leaves of at least 2^24 multiply-adds run on the tensor cores as exact
// integer products (the integer mode of the residue-number-system kernel,
// channels sized for operands below 2^bits, bits from the 4^l growth of the
// operands), the smaller ones on the CUDA cores in int64.
//
// This is the variant the paper analyses, kept for fidelity: on this GPU the
// reductions it saves are free inside the memory-bound addition kernels, so
// the default route reduces mod p at every level (winograd.cu).
#include <algorithm>
#include <vector>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kZT = 64;   // product tile
constexpr int kZK = 32;   // k chunk

// C = A B + b C over Z (b in {-1, 0, 1}); int32 operands, int64 sums.
__global__ void __launch_bounds__(256) zgemm_kernel(int m, int n, int k, const int32_t* __restrict__ A, long long lda,
                                                    const int32_t* __restrict__ B, long long ldb, long long* C,
                                                    long long ldc, int b) {
    __shared__ int32_t As[kZK][kZT];
    __shared__ int32_t Bs[kZK][kZT];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.y * kZT, col0 = blockIdx.x * kZT;
    long long acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int k0 = 0; k0 < k; k0 += kZK) {
        {
            const int r = tid >> 2, kk0 = (tid & 3) * 8, gi = row0 + r;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int gk = k0 + kk0 + e;
                As[kk0 + e][r] = (gi < m && gk < k) ? A[(long long)gi * lda + gk] : 0;
            }
        }
        {
            const int kk = tid >> 3, c0 = (tid & 7) * 8, gk = k0 + kk;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int gj = col0 + c0 + e;
                Bs[kk][c0 + e] = (gk < k && gj < n) ? B[(long long)gk * ldb + gj] : 0;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kZK; ++kk) {
            int32_t a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                bb[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += (long long)a[i] * bb[j];
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
            long long* cp = C + (long long)gi * ldc + gj;
            *cp = acc[i][j] + (b ? (long long)b * *cp : 0);
        }
    }
}

// Z = X + s Y (int32, s = +-1).
__global__ void zadd32_kernel(int rows, int cols, const int32_t* X, long long ldx, const int32_t* Y, long long ldy,
                              int32_t* Z, long long ldz, int s) {
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
        Z[r * ldz + c] = X[r * ldx + c] + s * Y[r * ldy + c];
    }
}

// Z = X + s Y (int64, s in {-1, 0, 1}; Y may be null when s = 0).
__global__ void zadd64_kernel(int rows, int cols, const long long* X, long long ldx, const long long* Y, long long ldy,
                              long long* Z, long long ldz, int s) {
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
        Z[r * ldz + c] = X[r * ldx + c] + (s ? s * Y[r * ldy + c] : 0);
    }
}

// Balanced residue: x mod p, minus p above (p - 1) / 2.
__global__ void zcenter_kernel(int rows, int cols, const uint32_t* X, long long ldx, uint32_t p, unsigned long long mu,
                               int32_t* Y, long long ldy) {
    const long long total = (long long)rows * cols;
    const uint32_t half = (p - 1) / 2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
        const uint32_t x = mod_u64(X[r * ldx + c], p, mu);
        Y[r * ldy + c] = x > half ? (int32_t)((long long)x - p) : (int32_t)x;
    }
}

// C = (alpha (X mod p) + beta C) mod p.
__global__ void zfinish_kernel(int m, int n, const long long* X, long long ldx, uint32_t* C, long long ldc, uint32_t p,
                               unsigned long long mu, uint32_t alpha, uint32_t beta) {
    const long long total = (long long)m * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), c = (int)(e - (long long)r * n);
        const long long x = X[r * ldx + c];
        // |x| < 2^62: reduce the magnitude, then fix the sign
        const uint32_t mag = mod_u64((unsigned long long)(x < 0 ? -x : x), p, mu);
        const uint32_t v = x < 0 && mag ? p - mag : mag;
        uint32_t* cp = C + r * ldc + c;
        const unsigned long long acc = (unsigned long long)alpha * v + (beta ? (unsigned long long)beta * *cp : 0ull);
        *cp = mod_u64(acc, p, mu);
    }
}

int blocks_for(long long work) { return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, 152 * 16)); }

struct ZCtx {
    cudaStream_t s;
    unsigned char* base;   // bump allocator over the workspace
    size_t used, cap;
    bool dry;              // size the workspace only
    size_t peak;
    int bits;              // the leaves' operands are below 2^bits in magnitude (31: CUDA cores only)
    int sms;
    int* err;
};

template <class T>
T* zalloc(ZCtx& c, int64_t count) {
    const size_t bytes = (size_t(count) * sizeof(T) + 255) & ~size_t(255);
    T* p = c.dry ? nullptr : reinterpret_cast<T*>(c.base + c.used);
    c.used += bytes;
    c.peak = std::max(c.peak, c.used);
    return p;
}

// C = -C (int64).
__global__ void zneg64_kernel(int rows, int cols, long long* C, long long ldc) {
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), q = (int)(e - (long long)r * cols);
        C[r * ldc + q] = -C[r * ldc + q];
    }
}

// Leaves at least this large (multiply-adds) go to the tensor cores as exact
// integer products (the integer mode of the residue-number-system kernel).
constexpr double kZTensorMacs = double(int64_t(1) << 24);

ffgpu_status zgemm(ZCtx& c, int64_t m, int64_t n, int64_t k, const int32_t* A, int64_t lda, const int32_t* B,
                   int64_t ldb, long long* C, int64_t ldc, int b) {
    if (m == 0 || n == 0) return FFGPU_OK;  // k = 0 leaves C = b C
    if (k > 0 && c.bits <= 30 && double(m) * double(n) * double(k) >= kZTensorMacs) {
        // the exact product X = A B on the tensor cores, written (b = 0) or
        // added (b = 1) to C; b = -1 negates C first.  Exact: every value is
        // within Theorem 3.1's bound, below 2^62.
        const size_t mark = c.used;
        const size_t wsb = int_gemm_ws_bytes(m, n, k, c.bits, c.sms);
        unsigned char* ws = zalloc<unsigned char>(c, (int64_t)wsb);
        ffgpu_status st = FFGPU_OK;
        if (!c.dry) {
            if (b == -1 && timed_launch("winograd_z_add", c.s, [&] {
                    zneg64_kernel<<<blocks_for(m * n), 256, 0, c.s>>>((int)m, (int)n, C, ldc);
                    return cudaGetLastError();
                }) != cudaSuccess)
                st = FFGPU_ERR_CUDA;
            if (st == FFGPU_OK)
                st = int_gemm_run(m, n, k, c.bits, A, lda, B, ldb, C, ldc, b != 0, ws, wsb, c.err, c.s);
        }
        c.used = mark;
        return st;
    }
    if (c.dry) return FFGPU_OK;
    const dim3 grid((unsigned)((n + kZT - 1) / kZT), (unsigned)((m + kZT - 1) / kZT));
    if (grid.y > 65535u) return FFGPU_ERR_INVALID;
    return timed_launch("winograd_z_gemm", c.s, [&] {
               zgemm_kernel<<<grid, 256, 0, c.s>>>((int)m, (int)n, (int)k, A, lda, B, ldb, C, ldc, b);
               return cudaGetLastError();
           }) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

ffgpu_status add32(ZCtx& c, int64_t rows, int64_t cols, const int32_t* X, int64_t ldx, const int32_t* Y, int64_t ldy,
                   int32_t* Z, int64_t ldz, int s) {
    if (c.dry || rows == 0 || cols == 0) return FFGPU_OK;
    return timed_launch("winograd_z_add", c.s, [&] {
               zadd32_kernel<<<blocks_for(rows * cols), 256, 0, c.s>>>((int)rows, (int)cols, X, ldx, Y, ldy, Z, ldz,
                                                                       s);
               return cudaGetLastError();
           }) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

ffgpu_status add64(ZCtx& c, int64_t rows, int64_t cols, const long long* X, int64_t ldx, const long long* Y,
                   int64_t ldy, long long* Z, int64_t ldz, int s) {
    if (c.dry || rows == 0 || cols == 0) return FFGPU_OK;
    return timed_launch("winograd_z_add", c.s, [&] {
               zadd64_kernel<<<blocks_for(rows * cols), 256, 0, c.s>>>((int)rows, (int)cols, X, ldx, Y, ldy, Z, ldz,
                                                                       s);
               return cudaGetLastError();
           }) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

#define ZTRY(x)                           \
    do {                                  \
        const ffgpu_status st_ = (x);     \
        if (st_ != FFGPU_OK) return st_;  \
    } while (0)

// C = A B + b C over Z with `levels` Winograd levels (Table 2 with beta = b).
ffgpu_status wz(ZCtx& c, int levels, int64_t m, int64_t n, int64_t k, const int32_t* A, int64_t lda,
                const int32_t* B, int64_t ldb, long long* C, int64_t ldc, int b) {
    if (levels == 0 || std::min(std::min(m, n), k) < 2) return zgemm(c, m, n, k, A, lda, B, ldb, C, ldc, b);
    const int64_t m2 = m & ~int64_t(1), n2 = n & ~int64_t(1), k2 = k & ~int64_t(1);
    if (m2 != m || n2 != n || k2 != k) {
        // dynamic peeling: the even block by Winograd, then the odd parts classically
        ZTRY(wz(c, levels, m2, n2, k2, A, lda, B, ldb, C, ldc, b));
        if (k2 < k) ZTRY(zgemm(c, m2, n2, 1, A + k2, lda, B + k2 * ldb, ldb, C, ldc, 1));
        if (n2 < n) ZTRY(zgemm(c, m2, n - n2, k, A, lda, B + n2, ldb, C + n2, ldc, b));
        if (m2 < m) ZTRY(zgemm(c, m - m2, n, k, A + m2 * lda, lda, B, ldb, C + m2 * ldc, ldc, b));
        return FFGPU_OK;
    }
    const int64_t h = m / 2, kh = k / 2, w = n / 2;
    const int32_t *A11 = A, *A12 = A + kh, *A21 = A + h * lda, *A22 = A + h * lda + kh;
    const int32_t *B11 = B, *B12 = B + w, *B21 = B + kh * ldb, *B22 = B + kh * ldb + w;
    long long *C11 = C, *C12 = C + w, *C21 = C + h * ldc, *C22 = C + h * ldc + w;
    const size_t mark = c.used;
    int32_t* X1 = zalloc<int32_t>(c, h * kh);
    int32_t* X2 = zalloc<int32_t>(c, kh * w);
    long long* X3 = zalloc<long long>(c, h * w);
    const int L = levels - 1;
    ZTRY(add32(c, h, kh, A21, lda, A22, lda, X1, kh, 1));                // 1  S1 = A21 + A22
    ZTRY(add32(c, kh, w, B12, ldb, B11, ldb, X2, w, -1));                // 2  T1 = B12 - B11
    ZTRY(wz(c, L, h, w, kh, X1, kh, X2, w, X3, w, 0));                   // 3  P5 = S1 T1
    ZTRY(add64(c, h, w, X3, w, C22, ldc, C22, ldc, b));                  // 4  C22 = P5 + b C22
    ZTRY(add64(c, h, w, X3, w, C12, ldc, C12, ldc, b));                  // 5  C12 = P5 + b C12
    ZTRY(add32(c, h, kh, X1, kh, A11, lda, X1, kh, -1));                 // 6  S2 = S1 - A11
    ZTRY(add32(c, kh, w, B22, ldb, X2, w, X2, w, -1));                   // 7  T2 = B22 - T1
    ZTRY(wz(c, L, h, w, kh, A11, lda, B11, ldb, X3, w, 0));              // 8  P1 = A11 B11
    ZTRY(add64(c, h, w, X3, w, C11, ldc, C11, ldc, b));                  // 9  C11 = P1 + b C11
    ZTRY(wz(c, L, h, w, kh, X1, kh, X2, w, X3, w, 1));                   // 10 U2 = S2 T2 + P1
    ZTRY(wz(c, L, h, w, kh, A12, lda, B21, ldb, C11, ldc, 1));           // 11 U1 = A12 B21 + C11
    ZTRY(add32(c, h, kh, A12, lda, X1, kh, X1, kh, -1));                 // 12 S4 = A12 - S2
    ZTRY(add32(c, kh, w, X2, w, B21, ldb, X2, w, -1));                   // 13 T4 = T2 - B21
    ZTRY(wz(c, L, h, w, kh, X1, kh, B22, ldb, C12, ldc, 1));             // 14 C12 = S4 B22 + C12
    ZTRY(add64(c, h, w, X3, w, C12, ldc, C12, ldc, 1));                  // 15 U5 = U2 + C12
    ZTRY(wz(c, L, h, w, kh, A22, lda, X2, w, C21, ldc, -b));             // 16 P4 = A22 T4 - b C21
    ZTRY(add32(c, h, kh, A11, lda, A21, lda, X1, kh, -1));               // 17 S3 = A11 - A21
    ZTRY(add32(c, kh, w, B22, ldb, B12, ldb, X2, w, -1));                // 18 T3 = B22 - B12
    ZTRY(wz(c, L, h, w, kh, X1, kh, X2, w, X3, w, 1));                   // 19 U3 = S3 T3 + U2
    ZTRY(add64(c, h, w, X3, w, C22, ldc, C22, ldc, 1));                  // 20 U7 = U3 + C22
    ZTRY(add64(c, h, w, X3, w, C21, ldc, C21, ldc, -1));                 // 21 U6 = U3 - C21
    c.used = mark;
    return FFGPU_OK;
}

}  // namespace

// Largest k for which l levels run without reduction: every operand within
// int32 (4^l (p-1)/2 < 2^31) and Theorem 3.1's bound for balanced inputs,
// (3^l (p-1)/2)^2 floor(k / 2^l), below 2^62.  0 if no k qualifies.
int64_t winograd_z_kmax(uint32_t p, int levels) {
    if (p < 2 || levels < 1 || levels > 8) return 0;
    // largest magnitude of a balanced residue: (p - 1) / 2, and 1 for p = 2
    // (its residues are 0 and -1)
    const unsigned __int128 half = p == 2 ? 1 : (p - 1) / 2;
    unsigned __int128 t = half, ops = half;
    for (int i = 0; i < levels; ++i) {
        t *= 3;
        ops *= 4;
    }
    if (ops >= ((unsigned __int128)1 << 31)) return 0;
    const unsigned __int128 per = t * t;
    if (per == 0) return INT64_MAX;
    const unsigned __int128 lim = (unsigned __int128)1 << 62;
    // largest d = floor(k / 2^l) with per d < 2^62, then the largest k with that floor
    unsigned __int128 d = (lim - 1) / per;
    const unsigned __int128 k = (d + 1) * ((unsigned __int128)1 << levels) - 1;
    return k > (unsigned __int128)INT64_MAX ? INT64_MAX : (int64_t)k;
}

ffgpu_status winograd_z_run(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const uint32_t* A,
                            int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta, uint32_t* C, int64_t ldc,
                            int levels, cudaStream_t s) {
    if (levels < 1 || levels > 8) return FFGPU_ERR_INVALID;
    if (k > winograd_z_kmax(p, levels)) return FFGPU_ERR_UNSUPPORTED_P;
    if (m > int64_t(65535) * kZT) return FFGPU_ERR_INVALID;
    const unsigned long long mu = ~0ull / p;
    ZCtx c;
    c.s = s;
    c.base = nullptr;
    c.used = 0;
    c.cap = 0;
    c.dry = true;
    c.peak = 0;
    c.err = nullptr;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        c.sms = sm_count(dev);
        // the leaves' operands: sums of up to 4^levels balanced residues
        unsigned long long bound = p == 2 ? 1ull : (p - 1) / 2;
        for (int i = 0; i < levels; ++i) bound *= 4;
        int b = 0;
        while (b < 31 && (1ull << b) < bound) ++b;
        c.bits = std::max(b, 1);
    }
    // workspace: balanced A and B, the int64 product, the levels' temporaries
    auto plan = [&](ZCtx& z, int32_t** Ac, int32_t** Bc, long long** X) {
        *Ac = zalloc<int32_t>(z, m * k);
        *Bc = zalloc<int32_t>(z, k * n);
        *X = zalloc<long long>(z, m * n);
    };
    int32_t *Ac = nullptr, *Bc = nullptr;
    long long* X = nullptr;
    plan(c, &Ac, &Bc, &X);
    ZTRY(wz(c, levels, m, n, k, Ac, k, Bc, n, X, n, 0));
    Pool* pool = nullptr;
    ZTRY(pool_get(s, c.peak, &pool));
    c.dry = false;
    c.err = pool->err;
    c.base = static_cast<unsigned char*>(pool->ptr);
    c.cap = pool->bytes;
    c.used = 0;
    c.peak = 0;
    plan(c, &Ac, &Bc, &X);
    auto launch = [&](auto&& f) { return timed_launch("winograd_z_add", s, f) == cudaSuccess ? FFGPU_OK : FFGPU_ERR_CUDA; };
    ZTRY(launch([&] {
        zcenter_kernel<<<blocks_for(m * k), 256, 0, s>>>((int)m, (int)k, A, lda, p, mu, Ac, k);
        zcenter_kernel<<<blocks_for(k * n), 256, 0, s>>>((int)k, (int)n, B, ldb, p, mu, Bc, n);
        return cudaGetLastError();
    }));
    ZTRY(wz(c, levels, m, n, k, Ac, k, Bc, n, X, n, 0));
    return launch([&] {
        zfinish_kernel<<<blocks_for(m * n), 256, 0, s>>>((int)m, (int)n, X, n, C, ldc, p, mu, alpha % p, beta % p);
        return cudaGetLastError();
    });
}

}  // namespace ffgpu

extern "C" ffgpu_status ffgpu_winograd_unreduced_kmax(uint32_t p, int levels, int64_t* kmax) {
    if (!kmax || p < 2 || p > 0x7FFFFFFFu || levels < 1 || levels > 8) return FFGPU_ERR_INVALID;
    *kmax = ffgpu::winograd_z_kmax(p, levels);
    return FFGPU_OK;
}
