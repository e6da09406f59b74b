// ftrsm: triangular solve with a matrix right-hand side over Z/pZ (section 4).
//
// Block recursive algorithm (Algorithm 1, section 4.1): split the triangle in
// two on a block boundary, solve the first half, update the other half of the
// right-hand side with one fgemm (B2 <- B2 - T21 X1: alpha = p - 1, beta = 1),
// solve the second half.  The recursion stops at diagonal blocks of L rows,
// L between 128 and 1024 (two leaves up to 2048 rows, more beyond: the rule
// and its measurements are at leaf_size), whose inverses are computed up
// front: one kernel inverts every 128 x 128 diagonal block (one CTA per block
// in shared memory: 16 x 16 blocks by substitution mod p, then doubling on
// them, see trsm_invert_blocks; non-unit diagonals inverted by the extended
// Euclidean algorithm of section 2.1.1; a non-invertible diagonal entry is
// recorded in the device error word), then
// each doubling level s -> 2s forms the off-diagonal block of every pair
// [[A, 0], [C, D]] (lower; upper by symmetry) as -D^{-1} (C A^{-1}) with two
// batched products over all pairs at once (one grouped launch each).  A leaf
// is then itself a tensor-core product: X_j = T_jj^{-1} B_j (left) or
// B_j T_jj^{-1} (right), written to a scratch panel and copied back.  Fewer,
// larger leaves keep the number of launches low (each product has a fixed
// cost of tens of microseconds); the price is the leaf products, twice the
// work of solving the leaves.  alpha is applied once up front.
#include <algorithm>
#include <cstring>
#include <vector>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kBlk = 128;       // diagonal block inverted by substitution
constexpr int kMaxLeaf = 1024;  // largest leaf
constexpr int64_t kDoublingSmallMacs = int64_t(1) << 24;  // doubling products routed to the CUDA cores

// Leaf size for a triangle of size sz: the smallest power of two from 128
// rows that covers half of it, at most 1024 rows (two leaves up to
// sz = 2048, then more).  Each product costs tens of microseconds whatever
// its size, so fewer, larger leaves win although a leaf's product does twice
// its triangle's work: measured (ms, p = 65521, m = n, unit lower) with about
// eight / four / two leaves: n = 2048 0.976 / 0.817 / 0.775, n = 4096 1.595 /
// 1.331 / 1.333; n = 8192 takes eight leaves of 1024 rows either way.
int64_t leaf_size(int64_t sz) {
    int64_t L = kBlk;
    while (L < kMaxLeaf && L * 2 < sz) L *= 2;
    return L;
}

// Exact multiply-add into a 96-bit sum (lo, mid, hi): below 2^68 for the at
// most 64 products of residues < 2^31 that one entry of a block product sums.
__device__ __forceinline__ void inv_mac96(uint32_t& lo, uint32_t& mid, uint32_t& hi, uint32_t a, uint32_t b) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"(a), "r"(b));
}

// (hi 2^64 + mid 2^32 + lo) mod p.
__device__ __forceinline__ uint32_t inv_mod96(uint32_t lo, uint32_t mid, uint32_t hi, uint32_t p,
                                              unsigned long long mu, uint32_t two64p) {
    const uint32_t th = mod_u64((unsigned long long)mod_u64(hi, p, mu) * two64p, p, mu);
    const uint32_t tl = mod_u64(((unsigned long long)mid << 32) | lo, p, mu);
    return th + tl >= p ? th + tl - p : th + tl;
}

// Inverse of diagonal block b of T (rows/cols [b kBlk, b kBlk + tb)), written
// densely into the leaf-sized inverse that contains it (kBlk x kBlk, zeros
// outside the triangle and beyond tb).  One CTA per block, everything in
// shared memory: the block of T (reduced mod p; a ragged block padded with
// the identity, whose inverse it leaves unchanged), then the inverses of its
// eight 16 x 16 diagonal blocks by substitution (one warp per block, one lane
// per column, the column in registers: each entry is d_i (delta_ij - the dot
// product with the entries above it), d_i the inverse of the diagonal
// entry), then doubling on pairs of s-blocks, s = 16, 32, 64: the
// off-diagonal block of [[A, 0], [C, D]]^{-1} is -D^{-1} (C A^{-1}) (lower;
// -A^{-1} (C D^{-1}) for [[A, C], [0, D]]), two block products per level over
// all pairs at once, exact 96-bit sums reduced once per entry.  A
// non-invertible diagonal entry of a non-unit triangle is recorded in the
// device error word.
constexpr int kInvThreads = 1024;  // the kernel assumes blockDim.x == kInvThreads
constexpr int kInvSub = 16;          // diagonal blocks inverted by substitution
constexpr int kBS = kBlk + 1;        // padded row stride of the blocks in shared memory
constexpr size_t kInvSmemWords = size_t(2) * kBlk * kBS + size_t(kBlk) * kBlk / 4 + kBlk;

// One level's block products over all pairs: out_q = P_q Q_q (s x s, inner
// dimension s), negated when asked.  P_q and Q_q are s x s blocks of
// the shared arrays at the pair's offsets; out_q is written at its own.
struct InvBlk {
    const uint32_t* base;
    int stride;
    int r0, c0;    // the pair-0 block's corner
    int dr, dc;    // added per pair
};

__device__ __forceinline__ void inv_add96(uint32_t& lo, uint32_t& mid, uint32_t& hi, unsigned long long v) {
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"((uint32_t)v), "r"((uint32_t)(v >> 32)));
}

// A thread takes four entries of one row of out_q, columns cc + e s/4 (so that
// the lanes of a warp read consecutive words of Q_q), and sums their products
// four at a time in 64-bit words (4 (p - 1)^2 < 2^64), folded into 96 bits.
__device__ __forceinline__ void inv_level_product(int s, int npairs, InvBlk P, InvBlk Q, uint32_t* out,
                                                  int ostride, int or0, int oc0, int odr, int odc, bool negate,
                                                  uint32_t p, unsigned long long mu, uint32_t two64p) {
    const int sq = s / 4, per_pair = s * sq;
    for (int o = threadIdx.x; o < npairs * per_pair; o += blockDim.x) {
        const int q = o / per_pair, rem = o - q * per_pair, r = rem / sq, cc = rem - r * sq;
        const uint32_t* pr = P.base + (P.r0 + q * P.dr + r) * P.stride + P.c0 + q * P.dc;
        const uint32_t* qc = Q.base + (Q.r0 + q * Q.dr) * Q.stride + Q.c0 + q * Q.dc + cc;
        uint32_t lo[4] = {0u, 0u, 0u, 0u}, mid[4] = {0u, 0u, 0u, 0u}, hi[4] = {0u, 0u, 0u, 0u};
        for (int l0 = 0; l0 < s; l0 += 4) {
            unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
            for (int l = l0; l < l0 + 4; ++l) {
                const unsigned long long a = pr[l];
                const uint32_t* qr = qc + l * Q.stride;
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[e] += a * qr[e * sq];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) inv_add96(lo[e], mid[e], hi[e], acc[e]);
        }
        uint32_t* orow = out + (or0 + q * odr + r) * ostride + oc0 + q * odc + cc;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint32_t v = inv_mod96(lo[e], mid[e], hi[e], p, mu, two64p);
            if (negate && v != 0u) v = p - v;
            orow[e * sq] = v;
        }
    }
}

// Column j of the inverse of one kInvSub x kInvSub triangular block Tg (row
// stride kBS, inverse diagonal dg), by substitution: rows top to bottom
// (lower) or bottom to top (upper).  Entries outside the column's triangle
// stay zero, so every sum may run over all earlier (later) rows.
template <bool kUpper>
__device__ __forceinline__ void inv_sub_column(const uint32_t* Tg, const uint32_t* dg, int j, uint32_t (&x)[kInvSub],
                                               uint32_t p, unsigned long long mu, uint32_t two64p) {
#pragma unroll
    for (int i = 0; i < kInvSub; ++i) x[i] = 0u;
#pragma unroll
    for (int t = 0; t < kInvSub; ++t) {
        const int i = kUpper ? kInvSub - 1 - t : t;
        uint32_t lo = 0u, mid = 0u, hi = 0u;
#pragma unroll
        for (int l = kUpper ? i + 1 : 0; l < (kUpper ? kInvSub : i); ++l) inv_mac96(lo, mid, hi, Tg[i * kBS + l], x[l]);
        if (kUpper ? i <= j : i >= j) {
            const uint32_t a = inv_mod96(lo, mid, hi, p, mu, two64p);
            const uint32_t rhs = i == j ? 1u : 0u;
            const uint32_t v = rhs >= a ? rhs - a : rhs + (p - a);
            x[i] = mod_u64((unsigned long long)v * dg[i], p, mu);
        }
    }
}

__global__ void __launch_bounds__(kInvThreads) trsm_invert_blocks(const uint32_t* __restrict__ T, long long ldt,
                                                                  int size, int upper, int unit, uint32_t p,
                                                                  unsigned long long mu, uint32_t two64p,
                                                                  uint32_t* __restrict__ Inv, int leaf, int* err) {
    extern __shared__ uint32_t sm[];
    uint32_t* sT = sm;                      // [kBlk][kBS]: the block of T
    uint32_t* sX = sT + kBlk * kBS;         // [kBlk][kBS]: its inverse
    uint32_t* sTmp = sX + kBlk * kBS;       // a level's C A^{-1} (C D^{-1}) blocks, s x s each
    uint32_t* sD = sTmp + kBlk * kBlk / 4;  // [kBlk]: inverse diagonal
    const int b = blockIdx.x, base = b * kBlk, tb = min(kBlk, size - base);
    const uint32_t* Tb = T + (long long)base * ldt + base;
    // the block's words, sixteen loads in flight per thread at a time
    constexpr int kLd = kBlk * kBlk / kInvThreads, kBatch = 16;
    static_assert(kLd % kBatch == 0, "whole batches of loads");
#pragma unroll 1
    for (int u0 = 0; u0 < kLd; u0 += kBatch) {
        uint32_t v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = threadIdx.x + (u0 + u) * kInvThreads, r = idx / kBlk, c = idx - r * kBlk;
            v[u] = (r < tb && c < tb) ? __ldg(Tb + (long long)r * ldt + c) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = threadIdx.x + (u0 + u) * kInvThreads, r = idx / kBlk, c = idx - r * kBlk;
            sT[r * kBS + c] = (r < tb && c < tb) ? mod_u64(v[u], p, mu) : (r == c ? 1u : 0u);
            sX[r * kBS + c] = 0u;
        }
    }
    for (int i = threadIdx.x; i < kBlk; i += blockDim.x) {
        uint32_t d = 1u;
        if (!unit && i < tb) {
            d = inv_mod_dev(mod_u64(__ldg(Tb + (long long)i * ldt + i), p, mu), p);
            if (d == 0) atomicCAS(err, 0, (int)kDevSingular);
        }
        sD[i] = d;
    }
    __syncthreads();
    {
        // the kInvSub x kInvSub diagonal blocks: warp w takes block w, lane j its column j
        const int w = threadIdx.x >> 5, j = threadIdx.x & 31;
        if (w < kBlk / kInvSub && j < kInvSub) {
            const int g = w * kInvSub;
            const uint32_t* Tg = sT + g * kBS + g;
            uint32_t x[kInvSub];
            if (upper)
                inv_sub_column<true>(Tg, sD + g, j, x, p, mu, two64p);
            else
                inv_sub_column<false>(Tg, sD + g, j, x, p, mu, two64p);
#pragma unroll
            for (int i = 0; i < kInvSub; ++i) sX[(g + i) * kBS + g + j] = x[i];
        }
    }
    __syncthreads();
    for (int s = kInvSub; s < kBlk; s *= 2) {
        const int np = kBlk / (2 * s), s2 = 2 * s;
        if (!upper) {
            // tmp_q = C_q A_q^{-1}: C_q = T[b, a], A_q^{-1} = X[a, a]
            inv_level_product(s, np, InvBlk{sT, kBS, s, 0, s2, s2}, InvBlk{sX, kBS, 0, 0, s2, s2}, sTmp, s, 0, 0, s, 0,
                              false, p, mu, two64p);
            __syncthreads();
            // X[b, a] = -D_q^{-1} tmp_q, D_q^{-1} = X[b, b]
            inv_level_product(s, np, InvBlk{sX, kBS, s, s, s2, s2}, InvBlk{sTmp, s, 0, 0, s, 0}, sX, kBS, s, 0, s2, s2,
                              true, p, mu, two64p);
        } else {
            // tmp_q = C_q D_q^{-1}: C_q = T[a, b], D_q^{-1} = X[b, b]
            inv_level_product(s, np, InvBlk{sT, kBS, 0, s, s2, s2}, InvBlk{sX, kBS, s, s, s2, s2}, sTmp, s, 0, 0, s, 0,
                              false, p, mu, two64p);
            __syncthreads();
            // X[a, b] = -A_q^{-1} tmp_q, A_q^{-1} = X[a, a]
            inv_level_product(s, np, InvBlk{sX, kBS, 0, 0, s2, s2}, InvBlk{sTmp, s, 0, 0, s, 0}, sX, kBS, 0, s, s2, s2,
                              true, p, mu, two64p);
        }
        __syncthreads();
    }
    // the dense kBlk x kBlk block (zeros beyond tb) into its leaf's inverse
    const int per = leaf / kBlk;
    uint32_t* out = Inv + (size_t)(b / per) * leaf * leaf + (size_t)(b % per) * kBlk * (leaf + 1);
    for (int idx = threadIdx.x; idx < kBlk * kBlk; idx += blockDim.x) {
        const int r = idx / kBlk, c = idx - r * kBlk;
        out[(size_t)r * leaf + c] = (r < tb && c < tb) ? sX[r * kBS + c] : 0u;
    }
}

struct TrsmCtx {
    int side, uplo, diag;
    uint32_t p;
    int64_t L;             // leaf size
    const uint32_t* inv;   // inverted diagonal leaves, L x L each (leading dimension L)
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

// Leaf: diagonal block starting at row/column `off` (leaf index off / L) of size tb.
ffgpu_status leaf(const TrsmCtx& c, int64_t off, int64_t tb, int64_t m, int64_t n, uint32_t* B, int64_t ldb) {
    const uint32_t* Inv = c.inv + size_t(off / c.L) * c.L * c.L;
    ffgpu_status st;
    if (c.side == 0) {  // X = Inv (tb x tb) * B (tb x n)
        if ((st = gemm(c, tb, n, tb, 1, Inv, c.L, B, ldb, 0, c.panel, n)) != FFGPU_OK) return st;
        return cudaMemcpy2DAsync(B, ldb * 4, c.panel, n * 4, n * 4, tb, cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
                   ? FFGPU_OK
                   : FFGPU_ERR_CUDA;
    }
    // X = B (m x tb) * Inv (tb x tb)
    if ((st = gemm(c, m, tb, tb, 1, B, ldb, Inv, c.L, 0, c.panel, tb)) != FFGPU_OK) return st;
    return cudaMemcpy2DAsync(B, ldb * 4, c.panel, tb * 4, tb * 4, m, cudaMemcpyDeviceToDevice, c.s) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

// Split on a leaf boundary: the first half of the leaves.
int64_t split(int64_t sz, int64_t L) {
    const int64_t nb = (sz + L - 1) / L;
    return (nb / 2) * L;
}

// Solve on the diagonal range [off, off + sz) of T.  side L: B is sz x n; side R: B is m x sz.
ffgpu_status rec(const TrsmCtx& c, int64_t off, int64_t sz, int64_t m, int64_t n, const uint32_t* T, int64_t ldt,
                 uint32_t* B, int64_t ldb) {
    if (sz <= c.L) return leaf(c, off, sz, m, n, B, ldb);
    const int64_t h = split(sz, c.L), r = sz - h;
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

// The two batched products of doubling level s -> 2s (every pair of s-blocks
// inside a leaf): step 0 forms C A^{-1} (lower) or C D^{-1} (upper) into tmp,
// step 1 the off-diagonal block of the inverse, (p - 1) D^{-1} tmp (lower) or
// (p - 1) A^{-1} tmp (upper).  With null pointers it gives the shapes only.
void doubling_descs(int64_t sz, int64_t L, int64_t s, int uplo, uint32_t p, const uint32_t* T, int64_t ldt,
                    uint32_t* inv, uint32_t* tmp, int step, std::vector<ffgpu_fgemm_desc>& out) {
    const uint32_t* dummy = reinterpret_cast<const uint32_t*>(uintptr_t(256));  // shapes only: never dereferenced
    int64_t pair = 0;
    for (int64_t q0 = 0; q0 < sz; q0 += L) {
        const int64_t Lq = std::min(L, sz - q0);
        uint32_t* Iq = inv ? inv + size_t(q0 / L) * L * L : nullptr;
        for (int64_t ps = 0; ps + s < Lq; ps += 2 * s, ++pair) {
            const int64_t ds = std::min(s, Lq - ps - s);  // size of the second block
            const int64_t g = q0 + ps;
            uint32_t* tm = tmp ? tmp + size_t(pair) * s * s : nullptr;
            ffgpu_fgemm_desc d;
            std::memset(&d, 0, sizeof(d));
            d.p = p;
            d.beta = 0;
            if (uplo == 0) {  // [[A, 0], [C, D]]: inverse block (1,0) = -D^{-1} C A^{-1}
                if (step == 0) {
                    d.m = ds; d.n = s; d.k = s; d.alpha = 1;
                    d.A = T ? T + (g + s) * ldt + g : dummy; d.lda = ldt;
                    d.B = Iq ? Iq + ps * L + ps : dummy; d.ldb = L;
                    d.C = tm ? tm : const_cast<uint32_t*>(dummy); d.ldc = s;
                } else {
                    d.m = ds; d.n = s; d.k = ds; d.alpha = p - 1;
                    d.A = Iq ? Iq + (ps + s) * L + ps + s : dummy; d.lda = L;
                    d.B = tm ? tm : dummy; d.ldb = s;
                    d.C = Iq ? Iq + (ps + s) * L + ps : const_cast<uint32_t*>(dummy); d.ldc = L;
                }
            } else {  // [[A, C], [0, D]]: inverse block (0,1) = -A^{-1} C D^{-1}
                if (step == 0) {
                    d.m = s; d.n = ds; d.k = ds; d.alpha = 1;
                    d.A = T ? T + g * ldt + g + s : dummy; d.lda = ldt;
                    d.B = Iq ? Iq + (ps + s) * L + ps + s : dummy; d.ldb = L;
                    d.C = tm ? tm : const_cast<uint32_t*>(dummy); d.ldc = ds;
                } else {
                    d.m = s; d.n = ds; d.k = s; d.alpha = p - 1;
                    d.A = Iq ? Iq + ps * L + ps : dummy; d.lda = L;
                    d.B = tm ? tm : dummy; d.ldb = ds;
                    d.C = Iq ? Iq + ps * L + ps + s : const_cast<uint32_t*>(dummy); d.ldc = L;
                }
            }
            out.push_back(d);
        }
    }
}

// Delayed (left-looking) solve: leaf i in the order its dependences allow is
// X_i = Q_i * (the rows, or columns, of B that hold X_prev and B_i), one
// product whose inner dimension covers every earlier leaf at once -- each
// block of X is reduced mod p exactly once (the delayed reduction of
// Algorithms 2-3, section 4.2, restated: the residue system keeps the whole
// accumulation exact, so the bound never forces an intermediate reduction).
// Q_i holds Inv_i next to -W_i, W_i = Inv_i T_i,prev (side L) or
// T_prev,i Inv_i (side R), all W_i from one batched product.
struct LeafGeo {
    int64_t off, Li;   // leaf rows/columns [off, off + Li)
    int64_t pb, plen;  // the earlier leaves: [pb, pb + plen)
    int64_t ob, len;   // operand range [ob, ob + len) of B (rows for side L, columns for side R)
    size_t q;          // word offset of Q_i in the Q region
};

// Leaves in solve order with their geometry; returns the Q region's words.
size_t delayed_geometry(int side, int uplo, int64_t sz, int64_t L, std::vector<LeafGeo>& g) {
    const int64_t nl = (sz + L - 1) / L;
    // side L lower / side R upper: ascending; the other two: descending
    const bool asc = (side == 0) == (uplo == 0);
    size_t q = 0;
    for (int64_t t = 0; t < nl; ++t) {
        const int64_t i = asc ? t : nl - 1 - t;
        LeafGeo x;
        x.off = i * L;
        x.Li = std::min(L, sz - x.off);
        if (asc) {
            x.pb = 0;
            x.plen = x.off;
            x.ob = 0;
            x.len = x.off + x.Li;
        } else {
            x.pb = x.off + x.Li;
            x.plen = sz - x.pb;
            x.ob = x.off;
            x.len = sz - x.off;
        }
        x.q = q;
        q += size_t(x.Li) * x.len;
        g.push_back(x);
    }
    return q;
}

// The W_i products (Q's off-diagonal parts, negated); null pointers: shapes only.
void delayed_w_descs(int side, const std::vector<LeafGeo>& g, int64_t L, uint32_t p, const uint32_t* T,
                     int64_t ldt, const uint32_t* inv, uint32_t* Q, std::vector<ffgpu_fgemm_desc>& out) {
    const uint32_t* dummy = reinterpret_cast<const uint32_t*>(uintptr_t(256));  // shapes only: never dereferenced
    for (const LeafGeo& x : g) {
        if (x.plen == 0) continue;
        const uint32_t* Inv = inv ? inv + size_t(x.off / L) * L * L : dummy;
        uint32_t* Qi = Q ? Q + x.q : const_cast<uint32_t*>(dummy);
        const bool before = x.pb < x.off;  // the earlier leaves come first in the operand
        ffgpu_fgemm_desc d;
        std::memset(&d, 0, sizeof(d));
        d.p = p;
        d.alpha = p - 1;
        d.beta = 0;
        if (side == 0) {  // W = Inv_i (Li x Li) T[off.., pb..] (Li x plen), into Q_i (Li x len)
            d.m = x.Li; d.n = x.plen; d.k = x.Li;
            d.A = Inv; d.lda = L;
            d.B = T ? T + x.off * ldt + x.pb : dummy; d.ldb = ldt;
            d.C = Q ? Qi + (before ? 0 : x.Li) : Qi; d.ldc = x.len;
        } else {          // W = T[pb.., off..] (plen x Li) Inv_i (Li x Li), into Q_i (len x Li)
            d.m = x.plen; d.n = x.Li; d.k = x.Li;
            d.A = T ? T + x.pb * ldt + x.off : dummy; d.lda = ldt;
            d.B = Inv; d.ldb = L;
            d.C = Q ? Qi + (before ? 0 : size_t(x.Li) * x.Li) : Qi; d.ldc = x.Li;
        }
        out.push_back(d);
    }
}

struct TrsmLayout {
    int64_t L, nl;
    size_t inv, panel, tmp, qreg, rest;  // byte offsets; rest = start of the fgemm / batched workspace
    size_t fg;                           // bytes the products need
};

TrsmLayout trsm_layout(int side, int uplo, int algo, int64_t m, int64_t n, uint32_t p, int sms) {
    TrsmLayout Y;
    const int64_t sz = side == 0 ? m : n, rhs = side == 0 ? n : m;
    Y.L = leaf_size(sz);
    Y.nl = (sz + Y.L - 1) / Y.L;
    Y.inv = 0;
    Y.panel = align256(size_t(Y.nl) * Y.L * Y.L * 4);
    Y.tmp = Y.panel + align256(size_t(Y.L) * rhs * 4);
    Y.qreg = Y.tmp + align256(size_t(sz) * Y.L / 2 * 4 + 4);
    std::vector<LeafGeo> geo;
    size_t qwords = 0;
    if (algo == 1) qwords = delayed_geometry(side, uplo, sz, Y.L, geo);
    Y.rest = Y.qreg + align256(qwords * 4);
    size_t fg = fgemm_ws_bytes(side == 0 ? Y.L : rhs, side == 0 ? rhs : Y.L, Y.L, p, sms);
    if (sz > Y.L) {
        const int64_t h = split(sz, Y.L), r = sz - h;
        if (side == 0)
            fg = std::max(fg, std::max(fgemm_ws_bytes(r, n, h, p, sms), fgemm_ws_bytes(h, n, r, p, sms)));
        else
            fg = std::max(fg, std::max(fgemm_ws_bytes(m, r, h, p, sms), fgemm_ws_bytes(m, h, r, p, sms)));
    }
    {
        ScopedBatchSmall route(kDoublingSmallMacs);  // as the doubling levels run them (ftrsm_run)
        for (int64_t s = kBlk; s < Y.L; s *= 2)
            for (int step = 0; step < 2; ++step) {
                std::vector<ffgpu_fgemm_desc> d;
                doubling_descs(sz, Y.L, s, uplo, p, nullptr, sz, nullptr, nullptr, step, d);
                if (!d.empty()) fg = std::max(fg, batched_ws_bytes((int64_t)d.size(), d.data(), sms));
            }
    }
    if (algo == 1) {
        std::vector<ffgpu_fgemm_desc> d;
        delayed_w_descs(side, geo, Y.L, p, nullptr, sz, nullptr, nullptr, d);
        if (!d.empty()) fg = std::max(fg, batched_ws_bytes((int64_t)d.size(), d.data(), sms));
        for (const LeafGeo& x : geo)
            fg = std::max(fg, side == 0 ? fgemm_ws_bytes(x.Li, rhs, x.len, p, sms)
                                        : fgemm_ws_bytes(rhs, x.Li, x.len, p, sms));
    }
    Y.fg = fg;
    return Y;
}

ffgpu_status delayed_solve(const TrsmCtx& c, const TrsmLayout& Y, int64_t sz, int64_t m, int64_t n,
                           const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, uint32_t* Q) {
    std::vector<LeafGeo> geo;
    delayed_geometry(c.side, c.uplo, sz, Y.L, geo);
    // Q_i: the inverse part, then every W_i in one batched product
    for (const LeafGeo& x : geo) {
        const uint32_t* Inv = c.inv + size_t(x.off / Y.L) * Y.L * Y.L;
        const bool before = x.pb < x.off;
        uint32_t* dst;
        size_t dpitch;
        if (c.side == 0) {
            dst = Q + x.q + (before ? x.plen : 0);
            dpitch = size_t(x.len) * 4;
        } else {
            dst = Q + x.q + (before ? size_t(x.plen) * x.Li : 0);
            dpitch = size_t(x.Li) * 4;
        }
        if (cudaMemcpy2DAsync(dst, dpitch, Inv, size_t(Y.L) * 4, size_t(x.Li) * 4, x.Li, cudaMemcpyDeviceToDevice,
                              c.s) != cudaSuccess)
            return FFGPU_ERR_CUDA;
    }
    {
        std::vector<ffgpu_fgemm_desc> d;
        delayed_w_descs(c.side, geo, Y.L, c.p, T, ldt, c.inv, Q, d);
        if (!d.empty()) {
            const ffgpu_status st = batched_run_ws((int64_t)d.size(), d.data(), c.ws, c.ws_bytes, c.err, c.s);
            if (st != FFGPU_OK) return st;
        }
    }
    // one product per leaf, in dependence order
    for (const LeafGeo& x : geo) {
        ffgpu_status st;
        if (c.side == 0) {  // X_i = Q_i (Li x len) B[ob.., :] (len x n)
            if ((st = gemm(c, x.Li, n, x.len, 1, Q + x.q, x.len, B + x.ob * ldb, ldb, 0, c.panel, n)) != FFGPU_OK)
                return st;
            if (cudaMemcpy2DAsync(B + x.off * ldb, ldb * 4, c.panel, n * 4, n * 4, x.Li, cudaMemcpyDeviceToDevice,
                                  c.s) != cudaSuccess)
                return FFGPU_ERR_CUDA;
        } else {            // X_i = B[:, ob..] (m x len) Q_i (len x Li)
            if ((st = gemm(c, m, x.Li, x.len, 1, B + x.ob, ldb, Q + x.q, x.Li, 0, c.panel, x.Li)) != FFGPU_OK)
                return st;
            if (cudaMemcpy2DAsync(B + x.off, ldb * 4, c.panel, x.Li * 4, x.Li * 4, m, cudaMemcpyDeviceToDevice,
                                  c.s) != cudaSuccess)
                return FFGPU_ERR_CUDA;
        }
    }
    return FFGPU_OK;
}

}  // namespace

// The algorithm a call uses: FFGPU_TRSM_DEFAULT resolves to the recursive one,
// measured faster from n = 4096 on (the delayed variant's leaf products are
// skinny, L rows by n, and leave a partial wave of tiles).
int ftrsm_algo(int algo) { return algo == FFGPU_TRSM_DEFAULT ? FFGPU_TRSM_RECURSIVE : algo; }

// Workspace: leaf inverses | leaf panel | doubling temporaries | [Q] | the largest product's workspace.
size_t ftrsm_ws_bytes(int side, int uplo, int algo, int64_t m, int64_t n, uint32_t p, int sms) {
    if (ftrsm_algo(algo) == FFGPU_TRSM_CASCADE) return cascade_ws_bytes(side, m, n, p, sms);
    const TrsmLayout Y = trsm_layout(side, uplo, ftrsm_algo(algo), m, n, p, sms);
    return Y.rest + align256(Y.fg);
}

ffgpu_status ftrsm_run(int side, int uplo, int diag, int algo, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                       const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, void* ws, size_t ws_bytes,
                       int* err, cudaStream_t s) {
    const int64_t sz = side == 0 ? m : n;
    algo = ftrsm_algo(algo);
    if (algo == FFGPU_TRSM_CASCADE)
        return cascade_run(side, uplo, diag, m, n, p, alpha, T, ldt, B, ldb, ws, ws_bytes, err, s);
    int dev = 0;
    cudaGetDevice(&dev);
    const TrsmLayout Y = trsm_layout(side, uplo, algo, m, n, p, sm_count(dev));
    if (ws_bytes < Y.rest) return FFGPU_ERR_NOMEM;
    unsigned char* w = static_cast<unsigned char*>(ws);
    TrsmCtx c;
    c.side = side;
    c.uplo = uplo;
    c.diag = diag;
    c.p = p;
    c.L = Y.L;
    c.inv = reinterpret_cast<uint32_t*>(w + Y.inv);
    c.panel = reinterpret_cast<uint32_t*>(w + Y.panel);
    c.ws = w + Y.rest;
    c.ws_bytes = ws_bytes - Y.rest;
    c.err = err;
    c.s = s;
    uint32_t* inv = const_cast<uint32_t*>(c.inv);
    uint32_t* tmp = reinterpret_cast<uint32_t*>(w + Y.tmp);
    const unsigned long long mu = ~0ull / p;
    const uint32_t two64p = (uint32_t)(((unsigned __int128)1 << 64) % p);
    const uint32_t al = alpha % p;
    if (al != 1) {
        if (timed_launch("scale_mod_p", s, [&] { return launch_scale(B, ldb, (int)m, (int)n, p, al, mu, s); }) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
    }
    // leaf inverses: zero (the other triangle), 128-blocks by substitution, then doubling
    if (cudaMemsetAsync(inv, 0, size_t(Y.nl) * Y.L * Y.L * 4, s) != cudaSuccess) return FFGPU_ERR_CUDA;
    const size_t smem = kInvSmemWords * 4;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(trsm_invert_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
        attr_set = true;
    }
    const int nb = (int)((sz + kBlk - 1) / kBlk);  // one CTA per block
    if (timed_launch("trsm_invert_blocks", s, [&] {
            trsm_invert_blocks<<<nb, kInvThreads, smem, s>>>(T, ldt, (int)sz, uplo, diag, p, mu, two64p, inv, (int)Y.L,
                                                      err);
            return cudaGetLastError();
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    {
        // a doubling level is a batch of equal products: up to 256^3 (2^24
        // multiply-adds) each on the CUDA cores, larger ones on the tensor
        // cores (measured, n = 2048 / 4096 / 8192, p = 65521: 0.675 / 1.229 /
        // 4.348 ms; with the batch default 2^23: 0.719 / 1.280 / 4.432 ms;
        // with 2^27: 0.677 / 1.322 / 4.642 ms)
        ScopedBatchSmall route(kDoublingSmallMacs);
        for (int64_t lv = kBlk; lv < Y.L; lv *= 2) {
            for (int step = 0; step < 2; ++step) {
                std::vector<ffgpu_fgemm_desc> d;
                doubling_descs(sz, Y.L, lv, uplo, p, T, ldt, inv, tmp, step, d);
                if (d.empty()) continue;
                const ffgpu_status st = batched_run_ws((int64_t)d.size(), d.data(), c.ws, c.ws_bytes, err, s);
                if (st != FFGPU_OK) return st;
            }
        }
    }
    if (algo == FFGPU_TRSM_DELAYED)
        return delayed_solve(c, Y, sz, m, n, T, ldt, B, ldb, reinterpret_cast<uint32_t*>(w + Y.qreg));
    return rec(c, 0, sz, m, n, T, ldt, B, ldb);
}

}  // namespace ffgpu
