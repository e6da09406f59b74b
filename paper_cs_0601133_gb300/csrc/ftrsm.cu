// ftrsm: triangular solve with a matrix right-hand side over Z/pZ (section 4).
//
// Block recursive algorithm (Algorithm 1, section 4.1): split the triangle in
// two, solve the first half, update the other half of the right-hand side with
// one fgemm (B2 <- B2 - T21 X1, i.e. alpha = p - 1, beta = 1), solve the second
// half.  Recursion stops at triangles of at most kLeaf rows, which a
// substitution kernel solves directly mod p (one thread per independent
// right-hand-side column, or row for the right side).  Non-unit diagonals are
// inverted in the leaf kernel with the extended Euclidean algorithm (section
// 2.1.1, classical representation); a non-invertible diagonal entry is
// recorded in the device error word.  alpha is applied once up front.
#include <algorithm>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kLeaf = 64;         // largest triangle solved by substitution
constexpr int kLeafThreads = 64;   // right-hand sides per block

__device__ uint32_t inv_mod_dev(uint32_t a, uint32_t p) {
    long long r0 = p, r1 = a % p, s0 = 0, s1 = 1;
    while (r1 != 0) {
        const long long q = r0 / r1;
        long long t = r0 - q * r1;
        r0 = r1;
        r1 = t;
        t = s0 - q * s1;
        s0 = s1;
        s1 = t;
    }
    if (r0 != 1) return 0;
    if (s0 < 0) s0 += p;
    return (uint32_t)s0;
}

// Exact sum of products kept as a 128-bit value (hi, lo); reduced once.
struct Acc128 {
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(unsigned long long v) {
        lo += v;
        hi += (lo < v) ? 1ull : 0ull;
    }
    __device__ __forceinline__ uint32_t mod(uint32_t p, unsigned long long mu, uint32_t two64p) const {
        // (hi * 2^64 + lo) mod p with hi < 2^7: hi * (2^64 mod p) + lo mod p
        const unsigned long long a = (unsigned long long)mod_u64(hi, p, mu) * two64p;
        return mod_u64((unsigned long long)mod_u64(a, p, mu) + mod_u64(lo, p, mu), p, mu);
    }
};

// Left side: op(T) X = B with T t x t (t <= kLeaf); each thread owns one
// column of B.  upper: back substitution; otherwise forward substitution.
__global__ void __launch_bounds__(kLeafThreads) trsm_leaf_left(const uint32_t* __restrict__ T,
                                                               long long ldt, uint32_t* B, long long ldb,
                                                               int t, int ncols, int upper, int unit,
                                                               uint32_t p, unsigned long long mu,
                                                               uint32_t two64p, int* err) {
    __shared__ uint32_t sT[kLeaf][kLeaf + 1];
    __shared__ uint32_t sX[kLeaf][kLeafThreads];
    __shared__ uint32_t sD[kLeaf];
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
        const int i = idx / t, l = idx - i * t;
        sT[i][l] = mod_u64(__ldg(T + (long long)i * ldt + l), p, mu);
    }
    for (int i = threadIdx.x; i < t; i += blockDim.x) {
        if (unit) {
            sD[i] = 1u;
        } else {
            const uint32_t d = inv_mod_dev(mod_u64(__ldg(T + (long long)i * ldt + i), p, mu), p);
            if (d == 0) atomicCAS(err, 0, (int)kDevSingular);
            sD[i] = d;
        }
    }
    const int j = blockIdx.x * kLeafThreads + threadIdx.x;
    const bool active = j < ncols;
    if (active)
        for (int i = 0; i < t; ++i) sX[i][threadIdx.x] = mod_u64(B[(long long)i * ldb + j], p, mu);
    __syncthreads();
    if (!active) return;
    for (int s = 0; s < t; ++s) {
        const int i = upper ? t - 1 - s : s;
        Acc128 acc;
        const int lo = upper ? i + 1 : 0, hi = upper ? t : i;
        for (int l = lo; l < hi; ++l) acc.add((unsigned long long)sT[i][l] * sX[l][threadIdx.x]);
        const uint32_t sum = acc.mod(p, mu, two64p);
        const uint32_t b = sX[i][threadIdx.x];
        const uint32_t v = b >= sum ? b - sum : b + (p - sum);
        sX[i][threadIdx.x] = mod_u64((unsigned long long)v * sD[i], p, mu);
    }
    for (int i = 0; i < t; ++i) B[(long long)i * ldb + j] = sX[i][threadIdx.x];
}

// Right side: X op(T) = B with T t x t; each thread owns one row of B.
// upper: columns solved left to right; lower: right to left.
__global__ void __launch_bounds__(kLeafThreads) trsm_leaf_right(const uint32_t* __restrict__ T,
                                                                long long ldt, uint32_t* B, long long ldb,
                                                                int t, int nrows, int upper, int unit,
                                                                uint32_t p, unsigned long long mu,
                                                                uint32_t two64p, int* err) {
    __shared__ uint32_t sT[kLeaf][kLeaf + 1];
    __shared__ uint32_t sX[kLeaf][kLeafThreads];
    __shared__ uint32_t sD[kLeaf];
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
        const int l = idx / t, jj = idx - l * t;
        sT[l][jj] = mod_u64(__ldg(T + (long long)l * ldt + jj), p, mu);
    }
    for (int i = threadIdx.x; i < t; i += blockDim.x) {
        if (unit) {
            sD[i] = 1u;
        } else {
            const uint32_t d = inv_mod_dev(mod_u64(__ldg(T + (long long)i * ldt + i), p, mu), p);
            if (d == 0) atomicCAS(err, 0, (int)kDevSingular);
            sD[i] = d;
        }
    }
    const int r0 = blockIdx.x * kLeafThreads;
    // coalesced load of the block's rows: element (row rr, column jj)
    for (int idx = threadIdx.x; idx < kLeafThreads * t; idx += blockDim.x) {
        const int rr = idx / t, jj = idx - rr * t;
        if (r0 + rr < nrows) sX[jj][rr] = mod_u64(B[(long long)(r0 + rr) * ldb + jj], p, mu);
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r0 + r < nrows) {
        for (int s = 0; s < t; ++s) {
            const int jj = upper ? s : t - 1 - s;
            Acc128 acc;
            const int lo = upper ? 0 : jj + 1, hi = upper ? jj : t;
            for (int l = lo; l < hi; ++l) acc.add((unsigned long long)sX[l][r] * sT[l][jj]);
            const uint32_t sum = acc.mod(p, mu, two64p);
            const uint32_t b = sX[jj][r];
            const uint32_t v = b >= sum ? b - sum : b + (p - sum);
            sX[jj][r] = mod_u64((unsigned long long)v * sD[jj], p, mu);
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kLeafThreads * t; idx += blockDim.x) {
        const int rr = idx / t, jj = idx - rr * t;
        if (r0 + rr < nrows) B[(long long)(r0 + rr) * ldb + jj] = sX[jj][rr];
    }
}

struct TrsmCtx {
    int side, uplo, diag;
    uint32_t p;
    unsigned long long mu;
    uint32_t two64p;
    void* ws;
    size_t ws_bytes;
    int* err;
    cudaStream_t s;
};

ffgpu_status leaf(const TrsmCtx& c, int64_t t, int64_t nrhs, const uint32_t* T, int64_t ldt, uint32_t* B,
                  int64_t ldb) {
    if (t == 0 || nrhs == 0) return FFGPU_OK;
    const int blocks = (int)((nrhs + kLeafThreads - 1) / kLeafThreads);
    auto go = [&]() -> cudaError_t {
        if (c.side == 0)
            trsm_leaf_left<<<blocks, kLeafThreads, 0, c.s>>>(T, ldt, B, ldb, (int)t, (int)nrhs, c.uplo, c.diag, c.p,
                                                            c.mu, c.two64p, c.err);
        else
            trsm_leaf_right<<<blocks, kLeafThreads, 0, c.s>>>(T, ldt, B, ldb, (int)t, (int)nrhs, c.uplo, c.diag,
                                                             c.p, c.mu, c.two64p, c.err);
        return cudaGetLastError();
    };
    return timed_launch(c.side == 0 ? "trsm_leaf_left" : "trsm_leaf_right", c.s, go) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

// Update C <- C - X * Y (mod p) through the fgemm path.
ffgpu_status update(const TrsmCtx& c, int64_t m, int64_t n, int64_t k, const uint32_t* X, int64_t ldx,
                    const uint32_t* Y, int64_t ldy, uint32_t* C, int64_t ldc) {
    if (m == 0 || n == 0 || k == 0) return FFGPU_OK;
    return fgemm_run(m, n, k, c.p, c.p - 1, X, ldx, Y, ldy, 1, C, ldc, c.ws, c.ws_bytes, c.err, c.s, 0, false);
}

// Split point: half, rounded down to a multiple of the leaf size.
int64_t split(int64_t sz) {
    int64_t h = sz / 2;
    if (h > kLeaf) h = h / kLeaf * kLeaf;
    return std::max<int64_t>(1, h);
}

// side L: T is m x m, B is m x n.  side R: T is n x n, B is m x n.
ffgpu_status rec(const TrsmCtx& c, int64_t m, int64_t n, const uint32_t* T, int64_t ldt, uint32_t* B,
                 int64_t ldb) {
    const int64_t sz = c.side == 0 ? m : n;
    if (sz <= kLeaf) return leaf(c, sz, c.side == 0 ? n : m, T, ldt, B, ldb);
    const int64_t h = split(sz), r = sz - h;
    const uint32_t* T11 = T;
    const uint32_t* T12 = T + h;
    const uint32_t* T21 = T + h * ldt;
    const uint32_t* T22 = T + h * ldt + h;
    ffgpu_status st;
    if (c.side == 0) {
        uint32_t* B1 = B;
        uint32_t* B2 = B + h * ldb;
        if (c.uplo == 0) {  // lower: X1 = T11^-1 B1; B2 -= T21 X1; X2 = T22^-1 B2
            if ((st = rec(c, h, n, T11, ldt, B1, ldb)) != FFGPU_OK) return st;
            if ((st = update(c, r, n, h, T21, ldt, B1, ldb, B2, ldb)) != FFGPU_OK) return st;
            return rec(c, r, n, T22, ldt, B2, ldb);
        }
        // upper (Algorithm 1 as printed): X2 = T22^-1 B2; B1 -= T12 X2; X1 = T11^-1 B1
        if ((st = rec(c, r, n, T22, ldt, B2, ldb)) != FFGPU_OK) return st;
        if ((st = update(c, h, n, r, T12, ldt, B2, ldb, B1, ldb)) != FFGPU_OK) return st;
        return rec(c, h, n, T11, ldt, B1, ldb);
    }
    uint32_t* B1 = B;       // columns [0, h)
    uint32_t* B2 = B + h;   // columns [h, n)
    if (c.uplo == 1) {  // upper: X1 T11 = B1; B2 -= X1 T12; X2 T22 = B2
        if ((st = rec(c, m, h, T11, ldt, B1, ldb)) != FFGPU_OK) return st;
        if ((st = update(c, m, r, h, B1, ldb, T12, ldt, B2, ldb)) != FFGPU_OK) return st;
        return rec(c, m, r, T22, ldt, B2, ldb);
    }
    // lower: X2 T22 = B2; B1 -= X2 T21; X1 T11 = B1
    if ((st = rec(c, m, r, T22, ldt, B2, ldb)) != FFGPU_OK) return st;
    if ((st = update(c, m, h, r, B2, ldb, T21, ldt, B1, ldb)) != FFGPU_OK) return st;
    return rec(c, m, h, T11, ldt, B1, ldb);
}

}  // namespace

// Largest fgemm workspace any update of the recursion needs.
size_t ftrsm_ws_bytes(int side, int64_t m, int64_t n, uint32_t p, int sms) {
    const int64_t sz = side == 0 ? m : n;
    if (sz <= kLeaf) return 0;
    const int64_t h = split(sz), r = sz - h;
    // the top-level update is the largest: (r x h) x (h x rhs) or (rhs x h) x (h x r)
    if (side == 0) return std::max(fgemm_ws_bytes(r, n, h, p, sms), fgemm_ws_bytes(h, n, r, p, sms));
    return std::max(fgemm_ws_bytes(m, r, h, p, sms), fgemm_ws_bytes(m, h, r, p, sms));
}

ffgpu_status ftrsm_run(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                       const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, void* ws, size_t ws_bytes,
                       int* err, cudaStream_t s) {
    TrsmCtx c;
    c.side = side;
    c.uplo = uplo;
    c.diag = diag;
    c.p = p;
    c.mu = ~0ull / p;
    c.two64p = (uint32_t)(((unsigned __int128)1 << 64) % p);
    c.ws = ws;
    c.ws_bytes = ws_bytes;
    c.err = err;
    c.s = s;
    const uint32_t al = alpha % p;
    if (al != 1) {
        if (timed_launch("scale_mod_p", s, [&] { return launch_scale(B, ldb, (int)m, (int)n, p, al, c.mu, s); }) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
    }
    return rec(c, m, n, T, ldt, B, ldb);
}

}  // namespace ffgpu
