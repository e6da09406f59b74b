// ftrsm: triangular solve with a matrix right-hand side over Z/pZ (section 4).
//
// Block recursive algorithm (Algorithm 1, section 4.1): split the triangle in
// two on a block boundary, solve the first half, update the other half of the
// right-hand side with one fgemm (B2 <- B2 - T21 X1: alpha = p - 1, beta = 1),
// solve the second half.  The recursion stops at diagonal blocks of L rows,
// L between 128 and 1024 (two leaves up to 2048 rows, more beyond: the rule
// and its measurements are at leaf_size), whose inverses are computed up
// front: one kernel inverts every 128 x 128 diagonal block (one CTA per block,
// eight lanes per column of the inverse, substitution mod p; non-unit
// diagonals inverted by the extended Euclidean algorithm of section 2.1.1; a
// non-invertible diagonal entry is recorded in the device error word), then
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
// densely into the leaf-sized inverse that contains it (kBlk x kBlk, zeros
// outside the triangle).  Column j of the inverse solves T x = e_j by forward
// (lower) or back (upper) substitution mod p, independently of the other
// columns: a CTA takes kInvCols columns of one block (kBlk / kInvCols CTAs
// per block, so that the sequential chains of many columns run on many SMs),
// eight lanes per column; each step's dot product is split over the eight
// lanes (exact 128-bit partial sums, reduced once, combined by shuffles), so
// the chain is one short step per row, and it starts at the first row where
// one of the CTA's columns has a non-zero entry.
constexpr int kInvCols = 32;
constexpr int kInvThreads = 8 * kInvCols;
constexpr int kBX = kBlk + 1;  // padded column stride of the inverse in shared memory
__global__ void __launch_bounds__(kInvThreads) trsm_invert_blocks(const uint32_t* __restrict__ T, long long ldt,
                                                                  int size, int upper, int unit, uint32_t p,
                                                                  unsigned long long mu, uint32_t two64p,
                                                                  uint32_t* __restrict__ Inv, int leaf, int* err) {
    extern __shared__ uint32_t sm[];
    // this CTA's columns, column-major with a padded stride: entry (i, q kInvCols + jl) of the inverse at
    // sX[jl*kBX + i], so that the eight lanes of a column read consecutive words (distinct banks) in the
    // dot products below and the final copy, which walks the columns, spreads over the banks too
    uint32_t* sX = sm;
    uint32_t* sT = sm + kInvCols * kBX;          // [kBlk][kBlk]: the block of T
    uint32_t* sD = sT + kBlk * kBlk;             // [kBlk] inverse diagonal
    const int b = blockIdx.x / (kBlk / kInvCols), q = blockIdx.x % (kBlk / kInvCols);
    const int base = b * kBlk;
    const int tb = min(kBlk, size - base);
    const uint32_t* Tb = T + (long long)base * ldt + base;
    for (int idx = threadIdx.x; idx < tb * kBlk; idx += blockDim.x) {
        const int r = idx / kBlk, c = idx % kBlk;
        sT[idx] = c < tb ? __ldg(Tb + (long long)r * ldt + c) : 0u;
    }
    for (int i = threadIdx.x; i < tb; i += blockDim.x) {
        if (unit) {
            sD[i] = 1u;
        } else {
            const uint32_t d = inv_mod_dev(mod_u64(__ldg(Tb + (long long)i * ldt + i), p, mu), p);
            if (d == 0) atomicCAS(err, 0, (int)kDevSingular);
            sD[i] = d;
        }
    }
    for (int idx = threadIdx.x; idx < kInvCols * kBX; idx += blockDim.x) sX[idx] = 0u;
    __syncthreads();
    const int jl = threadIdx.x >> 3, gl = threadIdx.x & 7;
    const int j = q * kInvCols + jl;
    const bool col = j < tb;
    // rows above (lower) / below (upper) the CTA's first column are zero in all its columns
    const int s0 = upper ? max(0, tb - (q + 1) * kInvCols) : q * kInvCols;
    uint32_t* Xj = sX + jl * kBX;
    for (int s = s0; s < tb; ++s) {  // same trip count in every lane (shuffles below)
        const int i = upper ? tb - 1 - s : s;
        const bool act = col && (upper ? i <= j : i >= j);
        Acc128 acc;
        if (act) {
            // any 32-bit word times a residue < 2^31 stays below 2^63
            const uint32_t* Ti = sT + i * kBlk;
            const int lo = upper ? i + 1 : j, hi = upper ? j + 1 : i;
            for (int l = lo + gl; l < hi; l += 8) acc.add((unsigned long long)Ti[l] * Xj[l]);
        }
        uint32_t v = act ? acc.mod(p, mu, two64p) : 0u;
        for (int o = 4; o > 0; o >>= 1) {
            const uint32_t y = __shfl_xor_sync(0xffffffffu, v, o);
            v += y;
            v = v >= p ? v - p : v;
        }
        if (act && gl == 0) {
            const uint32_t rhs = (i == j) ? 1u : 0u;
            const uint32_t t = rhs >= v ? rhs - v : rhs + (p - v);
            Xj[i] = mod_u64((unsigned long long)t * sD[i], p, mu);
        }
        __syncwarp();
    }
    __syncthreads();
    // this CTA's columns of the dense kBlk x kBlk block (zero padding beyond tb)
    const int per = leaf / kBlk;
    uint32_t* out = Inv + (size_t)(b / per) * leaf * leaf + (size_t)(b % per) * kBlk * (leaf + 1);
    for (int idx = threadIdx.x; idx < kBlk * kInvCols; idx += blockDim.x) {
        const int r = idx / kInvCols, cl = idx % kInvCols, c = q * kInvCols + cl;
        out[(size_t)r * leaf + c] = (r < tb && c < tb) ? sX[cl * kBX + r] : 0u;
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
    const size_t smem = (size_t(kInvCols) * kBX + size_t(kBlk) * kBlk + kBlk) * 4;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(trsm_invert_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
        attr_set = true;
    }
    const int nb = (int)((sz + kBlk - 1) / kBlk) * (kBlk / kInvCols);  // CTAs: column groups of every block
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
