// ftrsm: triangular solve with a matrix right-hand side over Z/pZ (section 4).
//
// Block recursive algorithm (Algorithm 1, section 4.1): split the triangle in
// two on a block boundary, solve the first half, update the other half of the
// right-hand side with one fgemm (B2 <- B2 - T21 X1: alpha = p - 1, beta = 1),
// solve the second half.  The recursion stops at diagonal blocks of kBlk rows.
// All diagonal blocks are inverted up front by one kernel (one CTA per block,
// one thread per column of the inverse, substitution mod p; non-unit
// diagonals inverted by the extended Euclidean algorithm of section 2.1.1; a
// non-invertible diagonal entry is recorded in the device error word).  A leaf
// is then itself a tensor-core product: X_j = T_jj^{-1} B_j (left) or
// B_j T_jj^{-1} (right), written to a scratch panel and copied back.  alpha is
// applied once up front.
#include <algorithm>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kBlk = 128;   // diagonal block (leaf) size

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

// Exact sum of products as a 128-bit value (hi, lo); reduced once.
struct Acc128 {
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(unsigned long long v) {
        lo += v;
        hi += (lo < v) ? 1ull : 0ull;
    }
    __device__ __forceinline__ uint32_t mod(uint32_t p, unsigned long long mu, uint32_t two64p) const {
        const unsigned long long a = (unsigned long long)mod_u64(hi, p, mu) * two64p;
        return mod_u64((unsigned long long)mod_u64(a, p, mu) + mod_u64(lo, p, mu), p, mu);
    }
};

// Inverse of diagonal block b of T (rows/cols [b kBlk, b kBlk + tb)), written
// densely to Inv[b] (kBlk x kBlk, row-major, zeros outside the triangle).
// Thread j computes column j of the inverse: T x = e_j by forward (lower) or
// back (upper) substitution mod p; x lives in shared memory.
__global__ void __launch_bounds__(kBlk) trsm_invert_blocks(const uint32_t* __restrict__ T, long long ldt, int size,
                                                           int upper, int unit, uint32_t p, unsigned long long mu,
                                                           uint32_t two64p, uint32_t* __restrict__ Inv, int* err) {
    extern __shared__ uint32_t sm[];
    uint32_t* sX = sm;                 // [kBlk][kBlk]: x of thread j at sX[i*kBlk + j]
    uint32_t* sD = sm + kBlk * kBlk;   // [kBlk] inverse diagonal
    const int b = blockIdx.x;
    const int base = b * kBlk;
    const int tb = min(kBlk, size - base);
    const uint32_t* Tb = T + (long long)base * ldt + base;
    for (int i = threadIdx.x; i < tb; i += blockDim.x) {
        if (unit) {
            sD[i] = 1u;
        } else {
            const uint32_t d = inv_mod_dev(mod_u64(__ldg(Tb + (long long)i * ldt + i), p, mu), p);
            if (d == 0) atomicCAS(err, 0, (int)kDevSingular);
            sD[i] = d;
        }
    }
    __syncthreads();
    const int j = threadIdx.x;
    uint32_t* out = Inv + (size_t)b * kBlk * kBlk;
    if (j < tb) {
        for (int s = 0; s < tb; ++s) {
            const int i = upper ? tb - 1 - s : s;
            uint32_t v;
            if (upper ? i > j : i < j) {
                v = 0u;  // outside the triangle of column j
            } else {
                Acc128 acc;
                const int lo = upper ? i + 1 : j, hi = upper ? j + 1 : i;
                // any 32-bit word times a residue < 2^31 stays below 2^63; the
                // 128-bit sum of at most kBlk of them is reduced once
                for (int l = lo; l < hi; ++l)
                    acc.add((unsigned long long)__ldg(Tb + (long long)i * ldt + l) * sX[l * kBlk + j]);
                const uint32_t sum = acc.mod(p, mu, two64p);
                const uint32_t rhs = (i == j) ? 1u : 0u;
                const uint32_t t = rhs >= sum ? rhs - sum : rhs + (p - sum);
                v = mod_u64((unsigned long long)t * sD[i], p, mu);
            }
            sX[i * kBlk + j] = v;
        }
    }
    __syncthreads();
    // dense kBlk x kBlk block (zero padding beyond tb)
    for (int idx = threadIdx.x; idx < kBlk * kBlk; idx += blockDim.x) {
        const int r = idx / kBlk, c = idx % kBlk;
        out[idx] = (r < tb && c < tb) ? sX[r * kBlk + c] : 0u;
    }
}

struct TrsmCtx {
    int side, uplo, diag;
    uint32_t p;
    const uint32_t* inv;   // inverted diagonal blocks, kBlk x kBlk each
    uint32_t* panel;       // scratch for one leaf's result
    void* ws;
    size_t ws_bytes;
    int* err;
    cudaStream_t s;
};

ffgpu_status gemm(const TrsmCtx& c, int64_t m, int64_t n, int64_t k, uint32_t alpha, const uint32_t* X, int64_t ldx,
                  const uint32_t* Y, int64_t ldy, uint32_t beta, uint32_t* C, int64_t ldc) {
    if (m == 0 || n == 0 || k == 0) return FFGPU_OK;
    return fgemm_run(m, n, k, c.p, alpha, X, ldx, Y, ldy, beta, C, ldc, c.ws, c.ws_bytes, c.err, c.s, 0, false);
}

// Leaf: diagonal block starting at row/column `off` (global block index off / kBlk) of size tb.
ffgpu_status leaf(const TrsmCtx& c, int64_t off, int64_t tb, int64_t m, int64_t n, uint32_t* B, int64_t ldb) {
    const uint32_t* Inv = c.inv + size_t(off / kBlk) * kBlk * kBlk;
    ffgpu_status st;
    if (c.side == 0) {  // X = Inv (tb x tb) * B (tb x n)
        if ((st = gemm(c, tb, n, tb, 1, Inv, kBlk, B, ldb, 0, c.panel, n)) != FFGPU_OK) return st;
        return cudaMemcpy2DAsync(B, ldb * 4, c.panel, n * 4, n * 4, tb, cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
                   ? FFGPU_OK
                   : FFGPU_ERR_CUDA;
    }
    // X = B (m x tb) * Inv (tb x tb)
    if ((st = gemm(c, m, tb, tb, 1, B, ldb, Inv, kBlk, 0, c.panel, tb)) != FFGPU_OK) return st;
    return cudaMemcpy2DAsync(B, ldb * 4, c.panel, tb * 4, tb * 4, m, cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

// Split on a block boundary: the first half of the blocks.
int64_t split(int64_t sz) {
    const int64_t nb = (sz + kBlk - 1) / kBlk;
    return (nb / 2) * kBlk;
}

// Solve on the diagonal range [off, off + sz) of T.  side L: B is sz x n; side R: B is m x sz.
ffgpu_status rec(const TrsmCtx& c, int64_t off, int64_t sz, int64_t m, int64_t n, const uint32_t* T, int64_t ldt,
                 uint32_t* B, int64_t ldb) {
    if (sz <= kBlk) return leaf(c, off, sz, m, n, B, ldb);
    const int64_t h = split(sz), r = sz - h;
    const uint32_t* T12 = T + h;
    const uint32_t* T21 = T + h * ldt;
    const uint32_t* T22 = T + h * ldt + h;
    const uint32_t neg1 = c.p - 1;
    ffgpu_status st;
    if (c.side == 0) {
        uint32_t* B1 = B;
        uint32_t* B2 = B + h * ldb;
        if (c.uplo == 0) {  // lower: X1 = T11^-1 B1; B2 -= T21 X1; X2 = T22^-1 B2
            if ((st = rec(c, off, h, h, n, T, ldt, B1, ldb)) != FFGPU_OK) return st;
            if ((st = gemm(c, r, n, h, neg1, T21, ldt, B1, ldb, 1, B2, ldb)) != FFGPU_OK) return st;
            return rec(c, off + h, r, r, n, T22, ldt, B2, ldb);
        }
        // upper (Algorithm 1 as printed): X2 = T22^-1 B2; B1 -= T12 X2; X1 = T11^-1 B1
        if ((st = rec(c, off + h, r, r, n, T22, ldt, B2, ldb)) != FFGPU_OK) return st;
        if ((st = gemm(c, h, n, r, neg1, T12, ldt, B2, ldb, 1, B1, ldb)) != FFGPU_OK) return st;
        return rec(c, off, h, h, n, T, ldt, B1, ldb);
    }
    uint32_t* B1 = B;       // columns [0, h)
    uint32_t* B2 = B + h;   // columns [h, sz)
    if (c.uplo == 1) {  // upper: X1 T11 = B1; B2 -= X1 T12; X2 T22 = B2
        if ((st = rec(c, off, h, m, h, T, ldt, B1, ldb)) != FFGPU_OK) return st;
        if ((st = gemm(c, m, r, h, neg1, B1, ldb, T12, ldt, 1, B2, ldb)) != FFGPU_OK) return st;
        return rec(c, off + h, r, m, r, T22, ldt, B2, ldb);
    }
    // lower: X2 T22 = B2; B1 -= X2 T21; X1 T11 = B1
    if ((st = rec(c, off + h, r, m, r, T22, ldt, B2, ldb)) != FFGPU_OK) return st;
    if ((st = gemm(c, m, h, r, neg1, B2, ldb, T21, ldt, 1, B1, ldb)) != FFGPU_OK) return st;
    return rec(c, off, h, m, h, T, ldt, B1, ldb);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Workspace: inverted blocks | leaf panel | the largest fgemm's workspace.
size_t ftrsm_ws_bytes(int side, int64_t m, int64_t n, uint32_t p, int sms) {
    const int64_t sz = side == 0 ? m : n, rhs = side == 0 ? n : m;
    const int64_t nb = (sz + kBlk - 1) / kBlk;
    size_t fg = fgemm_ws_bytes(side == 0 ? kBlk : rhs, side == 0 ? rhs : kBlk, kBlk, p, sms);
    if (sz > kBlk) {
        const int64_t h = split(sz), r = sz - h;
        if (side == 0)
            fg = std::max(fg, std::max(fgemm_ws_bytes(r, n, h, p, sms), fgemm_ws_bytes(h, n, r, p, sms)));
        else
            fg = std::max(fg, std::max(fgemm_ws_bytes(m, r, h, p, sms), fgemm_ws_bytes(m, h, r, p, sms)));
    }
    return align256(size_t(nb) * kBlk * kBlk * 4) + align256(size_t(kBlk) * rhs * 4) + align256(fg);
}

ffgpu_status ftrsm_run(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                       const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, void* ws, size_t ws_bytes,
                       int* err, cudaStream_t s) {
    const int64_t sz = side == 0 ? m : n, rhs = side == 0 ? n : m;
    const int64_t nb = (sz + kBlk - 1) / kBlk;
    const size_t inv_bytes = align256(size_t(nb) * kBlk * kBlk * 4);
    const size_t panel_bytes = align256(size_t(kBlk) * rhs * 4);
    if (ws_bytes < inv_bytes + panel_bytes) return FFGPU_ERR_NOMEM;
    unsigned char* w = static_cast<unsigned char*>(ws);
    TrsmCtx c;
    c.side = side;
    c.uplo = uplo;
    c.diag = diag;
    c.p = p;
    c.inv = reinterpret_cast<uint32_t*>(w);
    c.panel = reinterpret_cast<uint32_t*>(w + inv_bytes);
    c.ws = w + inv_bytes + panel_bytes;
    c.ws_bytes = ws_bytes - inv_bytes - panel_bytes;
    c.err = err;
    c.s = s;
    const unsigned long long mu = ~0ull / p;
    const uint32_t two64p = (uint32_t)(((unsigned __int128)1 << 64) % p);
    const uint32_t al = alpha % p;
    if (al != 1) {
        if (timed_launch("scale_mod_p", s, [&] { return launch_scale(B, ldb, (int)m, (int)n, p, al, mu, s); }) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
    }
    const size_t smem = size_t(kBlk) * kBlk * 4 + kBlk * 4;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(trsm_invert_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
        attr_set = true;
    }
    if (timed_launch("trsm_invert_blocks", s, [&] {
            trsm_invert_blocks<<<(int)nb, kBlk, smem, s>>>(T, ldt, (int)sz, uplo, diag, p, mu, two64p,
                                                          const_cast<uint32_t*>(c.inv), err);
            return cudaGetLastError();
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    return rec(c, 0, sz, m, n, T, ldt, B, ldb);
}

}  // namespace ffgpu
