// LQUP over Z/pZ (section 5) and the rank, determinant and inverse derived
// from it (section 6).
//
// Factorization.  A (m x n, p prime) becomes A[rowperm][:, colperm] = L U,
// stored packed in place: L (m x r, unit lower trapezoidal, diagonal not
// stored) strictly below the diagonal of the first r columns, U (r x n, upper
// trapezoidal, non-zero diagonal) on and above it, zeros in rows >= r from
// column r on.  Pivot rule: rows are met top to bottom; a row whose Schur
// complement is non-zero becomes the next pivot row, its pivot column the
// first non-zero one in original column order; the pivot rows keep their
// order, so do the other rows and the other columns.  The paper leaves the
// pivot choice open; with this rule the factorization is unique, so the
// result equals the row-by-row elimination that defines it.
//
// Recursion (section 5, after Ibarra, Moran and Hui): split the rows in two,
// factor the top half (rank r1, its pivot columns moved to the front of the
// active columns), then for the bottom half [X Z]: G = X U11^{-1} (the
// triangular solve of the paper, done as one product with U11^{-1}),
// Z <- Z - G Y (fgemm with alpha = p - 1, beta = 1), factor Z, and rotate the
// top half's non-pivot rows below the bottom half's pivot rows.  Every
// subtree hands its parent the inverse of its pivot block: a leaf forms it in
// shared memory, an inner node assembles it from its halves with two
// products, so no node pays for a separate triangular inversion.  Columns are
// kept as one contiguous active range [c, n) in original order, so every
// product works on plain row-major blocks.
//
// Leaves (kLeafRows rows) are not split further when they need not be.  One
// CTA factors the leaf on a window of the first W active columns in shared
// memory (row by row: find the pivot with warp ballots, fraction-free
// elimination of the rows below, one batched inversion of the pivots at the
// end, the elimination matrix E formed).  A second, column-parallel kernel
// gives the rest of the leaf's rows as E times their original values and
// checks that every non-pivot row's residual there is zero.
// If it is, the window's decisions are exactly the definition's (a pivot in
// the window is the first non-zero of the whole row, since the window columns
// come first in original order) and the leaf is committed; if not, a pivot
// lies beyond the window, nothing has been written, and the leaf is split.  A
// single row whose window is zero takes its pivot from the first non-zero
// column the check found.  The host reads every leaf's outcome (rank, commit
// or split) before it issues the next step: the calls are host-synchronous.
//
// Look-ahead.  Where a node's update Z <- Z - G Y takes the tensor-core route
// and its bottom half has more than one leaf, the columns of the bottom
// half's first window are updated first on the caller's stream and the
// others on a side stream (its own workspace, all but two SMs), so that the
// first leaf's window kernel runs while the rest of the update does; every
// later launch makes the caller's stream wait for the side stream first.
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kLeafRows = 64;  // rows of a leaf
constexpr int kMaxWin = 256;   // widest column window of a leaf
constexpr int kRestCols = 64;  // columns per CTA in the rest-of-row kernel
constexpr int kThreads = 256;
constexpr int kWinThreads = 512;
constexpr int64_t kGWords = int64_t(1) << 21;  // scratch for a small G product (h2 r1 r1 <= 2^27, r1 > 64)

// A leaf's outcome, written by the window kernel (and the failure fields by
// the rest kernel); the first four ints are read back by the host.
struct LeafInfo {
    int rank;                 // pivots found in the window
    int fail;                 // some non-pivot row has a non-zero residual beyond the window
    int ident;                // the window's columns keep their order
    int firstnz;              // smallest column of such a residual (absolute index)
    int prow[kLeafRows];      // pivot rows (leaf-relative), in pivot order
    int newrow[kLeafRows];    // new leaf row i = old leaf row newrow[i]
    int newcol[kMaxWin];      // new window column q = old window column newcol[q]
};

// 128-bit sum of 64-bit products, reduced once: (hi 2^64 + lo) mod p with
// two64p = 2^64 mod p.
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

__device__ __forceinline__ uint32_t mulm(uint32_t a, uint32_t b, uint32_t p, unsigned long long mu) {
    return mod_u64((unsigned long long)a * b, p, mu);
}

// Window factorization of one leaf (one CTA of kWinThreads).  A points at
// (rb, c); the tile is h x WS (W real columns, zero padding up to WS, a
// multiple of 32).
//
// Fraction-free elimination, so that no row waits for a modular inverse: row
// t' below pivot k (row t, column j, scaled value P) becomes
// P row_t' - a row_t with a its scaled entry in column j, and its scale d_t'
// (the factor by which the stored row exceeds the true Schur complement) is
// multiplied by P (recovered afterwards from which steps touched the row).
// The pivot row is published with the Shoup quotients of its values, so a
// row's update needs no quotient of its own multiplier.  The rows live in registers (warp w holds rows w, w + 16,
// w + 32, w + 48; lane l columns l, l + 32, ...); per row one barrier: the
// pivot row and its pivot are published in shared memory, every warp updates
// its rows below it, and the warp that owns the next row updates that row
// first, finds its pivot (warp ballots) and publishes it.  Afterwards one
// batched inversion of the pivots (prefix and suffix products over a warp, one
// extended-Euclid inverse) gives the true multipliers
// l_t'k = a d_t / (P d_t') (prefix products of the inverse pivots per row) and
// the true U rows.  The leaf's elimination matrix E = (I + N)^{-1}
// (N[t'][t] = l_t'k, unit lower triangular) and the inverse of its pivot block
// U11 (r x r, upper triangular) are formed by doubling: [[A, 0], [C, D]]^{-1}
// has off-diagonal block -D^{-1} C A^{-1} (upper: -A^{-1} C D^{-1}), each level
// two small products over all pairs at once.
//
// Writes the leaf's new rows on the window (rows points at column c of the
// scratch rows), E (h x h, original row order), U11^{-1} (r x r, zeros below
// the diagonal, leading dimension ldu; skipped when Uig is null) and the
// LeafInfo.
constexpr int kRowsPerWarp = kLeafRows / (kWinThreads / 32);
// Doubling scratch per triangle: at level s the pairs' s x s products, at most
// kLeafRows^2 / 2 words for any h <= kLeafRows.
constexpr int kTmWords = kLeafRows * kLeafRows / 2;

template <int NC>
__device__ __forceinline__ uint32_t pick(const uint32_t (&v)[NC], int c) {
    uint32_t x = 0u;
#pragma unroll
    for (int i = 0; i < NC; ++i)
        if (i == c) x = v[i];
    return x;
}

// Publish row trow (held by this warp in vrow): its values, pivot column and
// pivot, in slot `slot`; the pivot becomes number kk.
template <int NC>
__device__ __forceinline__ void win_publish(const uint32_t (&vrow)[NC], int trow, int kk, int slot, uint32_t p,
                                            unsigned long long mu, uint32_t* s_row, uint32_t* s_rowq, int* s_j,
                                            uint32_t* s_Pv, uint32_t* s_Ps, int* s_prow, int* s_pcol, uint32_t* s_P,
                                            int* s_colpiv, int* s_rowpiv) {
    const int lane = threadIdx.x & 31;
    int j = -1;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const unsigned bal = __ballot_sync(0xffffffffu, vrow[c] != 0u);
        if (j < 0 && bal) j = 32 * c + __ffs(bal) - 1;
    }
    // the row's values and their Shoup quotients: every later row's update
    // multiplies them by its own entry a, so no quotient of a is needed
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        s_row[slot * kMaxWin + lane + 32 * c] = vrow[c];
        s_rowq[slot * kMaxWin + lane + 32 * c] = vrow[c] ? shoup_quot(vrow[c], p, mu) : 0u;
    }
    const uint32_t P = __shfl_sync(0xffffffffu, pick<NC>(vrow, j >> 5), j & 31);
    if (lane == 0) {
        s_j[slot] = j;
        if (j >= 0) {
            s_Pv[slot] = P;
            s_Ps[slot] = shoup_quot(P, p, mu);
            s_prow[kk] = trow;
            s_pcol[kk] = j;
            s_P[kk] = P;
            s_colpiv[j] = kk;
            s_rowpiv[trow] = kk;
        }
    }
}

// Row update: v <- P v - a u (mod p) with a = v[j].  Returns false if a = 0.
template <int NC>
__device__ __forceinline__ bool win_update(uint32_t (&v)[NC], const uint32_t (&u)[NC], const uint32_t (&uq)[NC],
                                           int jc, int jl, uint32_t P, uint32_t Ps, uint32_t p, uint32_t& a_out) {
    const uint32_t a = __shfl_sync(0xffffffffu, pick<NC>(v, jc), jl);
    a_out = a;
    if (a == 0u) return false;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const uint32_t x = shoup_mul(v[c], P, Ps, p), y = shoup_mul(a, u[c], uq[c], p);
        v[c] = x >= y ? x - y : x + (p - y);
    }
    return true;
}

template <int NC>
__device__ __forceinline__ int win_eliminate(uint32_t* T, int WS, int W, int h, uint32_t p, unsigned long long mu,
                                             uint32_t* Lsm, uint32_t* s_row, uint32_t* s_rowq, int* s_j,
                                             uint32_t* s_Pv, uint32_t* s_Ps, int* s_prow, int* s_pcol, uint32_t* s_P,
                                             int* s_colpiv, int* s_rowpiv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = kWinThreads / 32;
    uint32_t v[kRowsPerWarp][NC];
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp; ++rr) {
        const int tt = warp + nw * rr;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int q = lane + 32 * c;
            v[rr][c] = (tt < h && q < W) ? T[tt * WS + q] : 0u;
        }
    }
    int k = 0;
    if (warp == 0)
        win_publish<NC>(v[0], 0, 0, 0, p, mu, s_row, s_rowq, s_j, s_Pv, s_Ps, s_prow, s_pcol, s_P, s_colpiv,
                        s_rowpiv);
    __syncthreads();
    for (int t = 0; t < h; ++t) {
        const int b = t & 1;
        const int j = s_j[b];
        const int tn = t + 1;
        const bool owner = tn < h && (tn % nw) == warp;
        const int rn = tn / nw;
        if (j >= 0) {  // same value in every thread
            const uint32_t P = s_Pv[b], Ps = s_Ps[b];
            uint32_t u[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) u[c] = s_row[b * kMaxWin + lane + 32 * c];
            uint32_t uq[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) uq[c] = s_rowq[b * kMaxWin + lane + 32 * c];
            const int jc = j >> 5, jl = j & 31;
            // the next row first (its owner publishes it right after), then the others
#pragma unroll
            for (int rr = 0; rr < kRowsPerWarp; ++rr) {
                if (!(owner && rr == rn)) continue;
                uint32_t a;
                if (win_update<NC>(v[rr], u, uq, jc, jl, P, Ps, p, a) && lane == 0) Lsm[tn * h + k] = a;
                win_publish<NC>(v[rr], tn, k + 1, tn & 1, p, mu, s_row, s_rowq, s_j, s_Pv, s_Ps, s_prow, s_pcol,
                                s_P, s_colpiv, s_rowpiv);
            }
#pragma unroll
            for (int rr = 0; rr < kRowsPerWarp; ++rr) {
                const int tt = warp + nw * rr;
                if (tt <= tn || tt >= h) continue;  // warp-uniform
                uint32_t a;
                if (win_update<NC>(v[rr], u, uq, jc, jl, P, Ps, p, a) && lane == 0) Lsm[tt * h + k] = a;
            }
            ++k;
        } else if (owner) {
#pragma unroll
            for (int rr = 0; rr < kRowsPerWarp; ++rr)
                if (rr == rn)
                    win_publish<NC>(v[rr], tn, k, tn & 1, p, mu, s_row, s_rowq, s_j, s_Pv, s_Ps, s_prow, s_pcol,
                                    s_P, s_colpiv, s_rowpiv);
        }
        __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp; ++rr) {
        const int tt = warp + nw * rr;
        if (tt >= h) continue;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int q = lane + 32 * c;
            if (q < WS) T[tt * WS + q] = v[rr][c];
        }
    }
    return k;
}

__global__ void __launch_bounds__(kWinThreads, 1) lqup_window_kernel(const uint32_t* __restrict__ A, long long lda,
                                                                  int h, int W, int WS, uint32_t p,
                                                                  unsigned long long mu, uint32_t two64p,
                                                                  uint32_t* __restrict__ Eg, uint32_t* __restrict__ Uig,
                                                                  long long ldu, uint32_t* __restrict__ rows,
                                                                  long long ldr, LeafInfo* __restrict__ info) {
    extern __shared__ uint32_t sm[];
    uint32_t* T = sm;              // [h][WS]
    uint32_t* Lsm = T + h * WS;    // [h][h]: numerators a, then true multipliers (row t, pivot k)
    uint32_t* Es = Lsm + h * h;    // [h][h]: E
    uint32_t* Nd = Es + h * h;     // [h][h]: N by pivot row
    uint32_t* Ui = Nd + h * h;     // [h][h]: U11^{-1}
    uint32_t* TmE = Ui + h * h;          // [kTmWords]: doubling products (lower)
    uint32_t* TmU = TmE + kTmWords;      // [kTmWords]: doubling products (upper)
    __shared__ uint32_t s_row[2 * kMaxWin], s_rowq[2 * kMaxWin];
    __shared__ uint32_t s_d[kLeafRows], s_invd[kLeafRows];
    __shared__ uint32_t s_P[kLeafRows], s_invP[kLeafRows], s_c[kLeafRows];
    __shared__ int s_prow[kLeafRows], s_pcol[kLeafRows], s_pre[kLeafRows + 1];
    __shared__ int s_rowpiv[kLeafRows], s_colpiv[kMaxWin];
    __shared__ int s_newrow[kLeafRows], s_newcol[kMaxWin];
    __shared__ int s_j[2];
    __shared__ uint32_t s_Pv[2], s_Ps[2];
    __shared__ int s_cnt[kWinThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kWinThreads / 32;
    const uint32_t one = 1u % p;

    // eight independent loads in flight per thread before their stores
    for (int base = 0; base < h * WS; base += 8 * blockDim.x) {
        uint32_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = base + e * blockDim.x + tid;
            const int r = idx / WS, q = idx - r * WS;
            v[e] = (idx < h * WS && q < W) ? __ldg(A + (long long)r * lda + q) : 0u;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = base + e * blockDim.x + tid;
            if (idx < h * WS) T[idx] = v[e];
        }
    }
    for (int idx = tid; idx < h * h; idx += blockDim.x) {
        Lsm[idx] = 0u;
        Nd[idx] = 0u;
        Ui[idx] = 0u;
        const int r = idx / h;
        Es[idx] = (idx - r * h == r) ? one : 0u;
    }
    for (int x = tid; x < h; x += blockDim.x) s_rowpiv[x] = -1;
    for (int x = tid; x < kMaxWin; x += blockDim.x) s_colpiv[x] = -1;
    __syncthreads();

    const int r = WS <= 64   ? win_eliminate<2>(T, WS, W, h, p, mu, Lsm, s_row, s_rowq, s_j, s_Pv, s_Ps, s_prow,
                                                s_pcol, s_P, s_colpiv, s_rowpiv)
                  : WS <= 96 ? win_eliminate<3>(T, WS, W, h, p, mu, Lsm, s_row, s_rowq, s_j, s_Pv, s_Ps, s_prow,
                                                s_pcol, s_P, s_colpiv, s_rowpiv)
                             : win_eliminate<8>(T, WS, W, h, p, mu, Lsm, s_row, s_rowq, s_j, s_Pv, s_Ps, s_prow,
                                                s_pcol, s_P, s_colpiv, s_rowpiv);
    __syncthreads();

    // 1 / P_k for every pivot: prefix and suffix products over warp 0 (two per lane), one inverse
    if (warp == 0) {
        const uint32_t v0 = 2 * lane < r ? s_P[2 * lane] : one;
        const uint32_t v1 = 2 * lane + 1 < r ? s_P[2 * lane + 1] : one;
        const uint32_t loc = mulm(v0, v1, p, mu);
        uint32_t inc = loc, sinc = loc;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = mulm(inc, x, p, mu);
            const uint32_t y = __shfl_down_sync(0xffffffffu, sinc, o);
            if (lane + o < 32) sinc = mulm(sinc, y, p, mu);
        }
        uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
        uint32_t sexc = __shfl_down_sync(0xffffffffu, sinc, 1);
        if (lane == 0) exc = one;
        if (lane == 31) sexc = one;
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        uint32_t itot = lane == 0 ? inv_mod_dev(total, p) : 0u;
        itot = __shfl_sync(0xffffffffu, itot, 0);
        const uint32_t base = mulm(mulm(itot, exc, p, mu), sexc, p, mu);
        if (2 * lane < r) s_invP[2 * lane] = mulm(base, v1, p, mu);
        if (2 * lane + 1 < r) s_invP[2 * lane + 1] = mulm(base, v0, p, mu);
    }
    // number of pivot rows above each row
    for (int x = tid; x <= h; x += blockDim.x) {
        int cnt = 0;
        for (int q = 0; q < r; ++q) cnt += s_prow[q] < x;
        s_pre[x] = cnt;
    }
    __syncthreads();
    // scale of each row: the product of the pivots of the steps that touched it
    // (those whose numerator is non-zero), one warp per row
    for (int t = warp; t < h; t += nwarps) {
        const int pre = s_pre[t];
        const uint32_t g0 = lane < pre && Lsm[t * h + lane] ? s_P[lane] : one;
        const uint32_t g1 = lane + 32 < pre && Lsm[t * h + lane + 32] ? s_P[lane + 32] : one;
        uint32_t g = mulm(g0, g1, p, mu);
        for (int o = 16; o > 0; o >>= 1) g = mulm(g, __shfl_xor_sync(0xffffffffu, g, o), p, mu);
        if (lane == 0) s_d[t] = g;
    }
    __syncthreads();
    // c_k = d_{prow k} / P_k = 1 / (true pivot k)
    for (int x = tid; x < r; x += blockDim.x) {
        s_c[x] = mulm(s_d[s_prow[x]], s_invP[x], p, mu);
        Ui[x * h + x] = s_c[x];
    }
    __syncthreads();
    // true multipliers l_tk = a_tk c_k / (d_t before step k), one warp per row:
    // 1 / d_t before step k is the product of 1 / P_k' over the earlier steps
    // that touched row t (exclusive prefix products over the pivots)
    for (int t = warp; t < h; t += nwarps) {
        const int pre = s_pre[t];
        const uint32_t n0 = lane < pre ? Lsm[t * h + lane] : 0u;
        const uint32_t n1 = lane + 32 < pre ? Lsm[t * h + lane + 32] : 0u;
        const uint32_t f0 = n0 ? s_invP[lane] : one, f1 = n1 ? s_invP[lane + 32] : one;
        uint32_t i0 = f0, i1 = f1;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x0 = __shfl_up_sync(0xffffffffu, i0, o);
            const uint32_t x1 = __shfl_up_sync(0xffffffffu, i1, o);
            if (lane >= o) {
                i0 = mulm(i0, x0, p, mu);
                i1 = mulm(i1, x1, p, mu);
            }
        }
        const uint32_t tot0 = __shfl_sync(0xffffffffu, i0, 31), tot1 = __shfl_sync(0xffffffffu, i1, 31);
        uint32_t e0 = __shfl_up_sync(0xffffffffu, i0, 1), e1 = __shfl_up_sync(0xffffffffu, i1, 1);
        if (lane == 0) {
            e0 = one;
            e1 = one;
        }
        e1 = mulm(e1, tot0, p, mu);
        if (n0) {
            const uint32_t l = mulm(mulm(n0, s_c[lane], p, mu), e0, p, mu);
            Lsm[t * h + lane] = l;
            Nd[t * h + s_prow[lane]] = l;
        }
        if (n1) {
            const uint32_t l = mulm(mulm(n1, s_c[lane + 32], p, mu), e1, p, mu);
            Lsm[t * h + lane + 32] = l;
            Nd[t * h + s_prow[lane + 32]] = l;
        }
        if (lane == 0) s_invd[t] = mulm(tot0, tot1, p, mu);
    }
    __syncthreads();
    // true U rows (the other rows are zero on the window)
    for (int idx = tid; idx < h * WS; idx += blockDim.x) {
        const int t = idx / WS;
        if (s_rowpiv[t] >= 0 && T[idx]) T[idx] = mulm(T[idx], s_invd[t], p, mu);
    }
    __syncthreads();
    // doubling for E (h x h, unit lower) and U11^{-1} (r x r, upper); level s
    // pairs the blocks [b0, b0 + s) and [b0 + s, b0 + 2s), b0 = 2 s pr
    for (int ls = 0; (1 << ls) < h; ++ls) {
        const int s = 1 << ls;
        const int npE = (h - s + 2 * s - 1) / (2 * s);
        const int npU = r > s ? (r - s + 2 * s - 1) / (2 * s) : 0;
        // phase A: TmE = N21 E11 (ds x s per pair), TmU = U12 D^{-1} (s x du per pair)
        for (int idx = tid; idx < (npE + npU) << (2 * ls); idx += blockDim.x) {
            const bool lower = idx < (npE << (2 * ls));
            const int li = lower ? idx : idx - (npE << (2 * ls));
            const int pr = li >> (2 * ls), rem = li & ((s << ls) - 1);
            const int i = rem >> ls, jj = rem & (s - 1);
            const int b0 = 2 * s * pr;
            Acc128 acc;
            if (lower) {
                if (i >= min(s, h - b0 - s)) continue;
                const uint32_t* nrow = Nd + (b0 + s + i) * h + b0;
                for (int l = jj; l < s; ++l) acc.add((unsigned long long)nrow[l] * Es[(b0 + l) * h + b0 + jj]);
                TmE[li] = acc.mod(p, mu, two64p);
            } else {
                if (jj >= min(s, r - b0 - s)) continue;
                const uint32_t* urow = T + s_prow[b0 + i] * WS;
                for (int l = 0; l <= jj; ++l)
                    acc.add((unsigned long long)urow[s_pcol[b0 + s + l]] * Ui[(b0 + s + l) * h + b0 + s + jj]);
                TmU[li] = acc.mod(p, mu, two64p);
            }
        }
        __syncthreads();
        // phase B: E21 = -E22 TmE, (U11^{-1})12 = -A^{-1} TmU
        for (int idx = tid; idx < (npE + npU) << (2 * ls); idx += blockDim.x) {
            const bool lower = idx < (npE << (2 * ls));
            const int li = lower ? idx : idx - (npE << (2 * ls));
            const int pr = li >> (2 * ls), rem = li & ((s << ls) - 1);
            const int i = rem >> ls, jj = rem & (s - 1);
            const int b0 = 2 * s * pr;
            const int base = pr << (2 * ls);
            Acc128 acc;
            if (lower) {
                if (i >= min(s, h - b0 - s)) continue;
                const uint32_t* erow = Es + (b0 + s + i) * h + b0 + s;
                for (int l = 0; l <= i; ++l) acc.add((unsigned long long)erow[l] * TmE[base + (l << ls) + jj]);
                const uint32_t v = acc.mod(p, mu, two64p);
                Es[(b0 + s + i) * h + b0 + jj] = v ? p - v : 0u;
            } else {
                if (jj >= min(s, r - b0 - s)) continue;
                const uint32_t* arow = Ui + (b0 + i) * h + b0;
                for (int l = i; l < s; ++l) acc.add((unsigned long long)arow[l] * TmU[base + (l << ls) + jj]);
                const uint32_t v = acc.mod(p, mu, two64p);
                Ui[(b0 + i) * h + b0 + s + jj] = v ? p - v : 0u;
            }
        }
        __syncthreads();
    }

    // stable partitions: pivots first (in pivot order), then the rest ascending
    for (int x = tid; x < r; x += blockDim.x) {
        s_newrow[x] = s_prow[x];
        s_newcol[x] = s_pcol[x];
    }
    const unsigned lt = (1u << lane) - 1u;
    {
        const bool np = tid < W && s_colpiv[tid] < 0;
        const unsigned bal = __ballot_sync(0xffffffffu, np);
        if (lane == 0) s_cnt[warp] = __popc(bal);
        __syncthreads();
        int off = r;
        for (int w = 0; w < warp; ++w) off += s_cnt[w];
        if (np) s_newcol[off + __popc(bal & lt)] = tid;
        __syncthreads();
    }
    {
        const bool np = tid < h && s_rowpiv[tid] < 0;
        const unsigned bal = __ballot_sync(0xffffffffu, np);
        if (lane == 0) s_cnt[warp] = __popc(bal);
        __syncthreads();
        int off = r;
        for (int w = 0; w < warp; ++w) off += s_cnt[w];
        if (np) s_newrow[off + __popc(bal & lt)] = tid;
        __syncthreads();
    }

    if (tid == 0) {
        int ident = 1;
        for (int x = 0; x < r; ++x) ident &= (s_pcol[x] == x);
        info->rank = r;
        info->fail = 0;
        info->ident = ident;
        info->firstnz = INT_MAX;
    }
    for (int x = tid; x < h; x += blockDim.x) {
        info->newrow[x] = s_newrow[x];
        if (x < r) info->prow[x] = s_prow[x];
    }
    for (int x = tid; x < W; x += blockDim.x) info->newcol[x] = s_newcol[x];
    for (int idx = tid; idx < h * h; idx += blockDim.x) Eg[idx] = Es[idx];
    if (Uig)
        for (int idx = tid; idx < r * r; idx += blockDim.x) {
            const int i = idx / r, q = idx - i * r;
            Uig[(long long)i * ldu + q] = Ui[i * h + q];
        }
    // the leaf's new rows on the window: multipliers left of the diagonal of
    // the first r columns, the pivot rows' values on and right of it
    for (int idx = tid; idx < h * W; idx += blockDim.x) {
        const int i = idx / W, q = idx - i * W;
        const int t = s_newrow[i];
        uint32_t v;
        if (q < min(i, r))
            v = Lsm[t * h + q];
        else
            v = i < r ? T[t * WS + s_newcol[q]] : 0u;
        rows[(long long)i * ldr + q] = v;
    }
}

// The rest of the leaf's rows.  Blocks [0, nleft): columns [0, c), the rows
// only reordered.  Blocks from nleft on: kRestCols columns each from c + W
// on: new row i = E[newrow[i]] times the original columns (independent
// 128-bit dot products, no barrier between pivots); the non-pivot rows'
// residuals must be zero, else the leaf fails and the smallest such column is
// recorded.  A points at (rb, 0), rows at the scratch rows' column 0.
__global__ void __launch_bounds__(kThreads) lqup_rest_kernel(const uint32_t* __restrict__ A, long long lda, int h,
                                                             int c, int W, int n, int nleft, uint32_t p,
                                                             unsigned long long mu, uint32_t two64p,
                                                             const uint32_t* __restrict__ Eg,
                                                             uint32_t* __restrict__ rows, long long ldr,
                                                             LeafInfo* __restrict__ info) {
    extern __shared__ uint32_t sm[];
    __shared__ int s_newrow[kLeafRows];
    const int tid = threadIdx.x;
    const int r = info->rank;
    for (int x = tid; x < h; x += blockDim.x) s_newrow[x] = info->newrow[x];
    __syncthreads();
    if ((int)blockIdx.x < nleft) {
        const int col = blockIdx.x * blockDim.x + tid;
        if (col < c)
            for (int i0 = 0; i0 < h; i0 += 16) {  // sixteen loads in flight before their stores
                uint32_t v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    v[e] = i0 + e < h ? __ldg(A + (long long)s_newrow[i0 + e] * lda + col) : 0u;
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    if (i0 + e < h) rows[(long long)(i0 + e) * ldr + col] = v[e];
            }
        return;
    }
    const int q0 = c + W + (blockIdx.x - nleft) * kRestCols;
    const int nq = min(kRestCols, n - q0);
    uint32_t* R = sm;                   // [h][kRestCols]
    uint32_t* Es = R + h * kRestCols;   // [h][h]
    {
        // every load of the thread in flight before the stores (h <= 64: at
        // most 16 of R and 16 of E per thread)
        constexpr int kPer = kLeafRows * kRestCols / kThreads;
        uint32_t vr[kPer], ve[kPer];
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            const int idx = e * kThreads + tid;
            const int i = idx / kRestCols, q = idx % kRestCols;
            vr[e] = (i < h && q < nq) ? __ldg(A + (long long)i * lda + q0 + q) : 0u;
            ve[e] = idx < h * h ? __ldg(Eg + idx) : 0u;
        }
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            const int idx = e * kThreads + tid;
            if (idx < h * kRestCols) R[idx] = vr[e];
            if (idx < h * h) Es[idx] = ve[e];
        }
    }
    __syncthreads();
    const int q = tid % kRestCols;
    for (int i = tid / kRestCols; i < h; i += kThreads / kRestCols) {
        const int t = s_newrow[i];
        Acc128 acc;
        const uint32_t* Et = Es + t * h;
        for (int s = 0; s <= t; ++s) acc.add((unsigned long long)Et[s] * R[s * kRestCols + q]);
        const uint32_t v = acc.mod(p, mu, two64p);
        if (q < nq) {
            if (i >= r && v != 0u) {
                info->fail = 1;
                atomicMin(&info->firstnz, q0 + q);
            }
            rows[(long long)i * ldr + q0 + q] = i < r ? v : 0u;
        }
    }
}

// rowperm[rb + i] <- rowperm[rb + newrow[i]] (one CTA).
__global__ void lqup_rowperm_kernel(int32_t* rowperm, int h, const LeafInfo* __restrict__ info) {
    __shared__ int32_t s[kLeafRows];
    for (int x = threadIdx.x; x < h; x += blockDim.x) s[x] = rowperm[info->newrow[x]];
    __syncthreads();
    for (int x = threadIdx.x; x < h; x += blockDim.x) rowperm[x] = s[x];
}

// The window's column order applied to every row outside the leaf
// [skip_b, skip_e) and to colperm: A[row][c + q] <- A[row][c + newcol[q]].
__global__ void __launch_bounds__(kThreads) lqup_colperm_kernel(uint32_t* __restrict__ A, long long lda, int m,
                                                                int skip_b, int skip_e, int c, int W,
                                                                const LeafInfo* __restrict__ info,
                                                                int32_t* __restrict__ colperm) {
    __shared__ int s_nc[kMaxWin];
    const int tid = threadIdx.x;
    for (int x = tid; x < W; x += blockDim.x) s_nc[x] = info->newcol[x];
    __syncthreads();
    if (blockIdx.x == 0) {
        const int32_t v = tid < W ? colperm[c + s_nc[tid]] : 0;
        __syncthreads();
        if (tid < W) colperm[c + tid] = v;
        __syncthreads();
    }
    for (int row = blockIdx.x; row < m; row += gridDim.x) {
        if (row >= skip_b && row < skip_e) continue;  // same for the whole CTA
        uint32_t* a = A + (long long)row * lda + c;
        const uint32_t v = tid < W ? a[s_nc[tid]] : 0u;
        __syncthreads();
        if (tid < W) a[tid] = v;
        __syncthreads();
    }
}

// Column j moved to position c, columns [c, j) one to the right, in every row
// and in colperm (row index m).  One CTA per row; chunks right to left so that
// every value is read before it is overwritten.
__global__ void __launch_bounds__(kThreads) lqup_colrot_kernel(uint32_t* __restrict__ A, long long lda, int m, int c,
                                                               int j, int32_t* __restrict__ colperm) {
    const int tid = threadIdx.x;
    for (int row = blockIdx.x; row <= m; row += gridDim.x) {
        uint32_t* a = row < m ? A + (long long)row * lda : reinterpret_cast<uint32_t*>(colperm);
        const uint32_t saved = a[j];
        for (int hi = j + 1; hi > c + 1; hi -= blockDim.x) {
            const int pos = hi - 1 - tid;
            const uint32_t v = pos > c ? a[pos - 1] : 0u;
            __syncthreads();
            if (pos > c) a[pos] = v;
            __syncthreads();
        }
        if (tid == 0) a[c] = saved;
        __syncthreads();
    }
}

// Rows [a, b) reversed (full width n) together with rowperm.
__global__ void __launch_bounds__(kThreads) lqup_rowrev_kernel(uint32_t* __restrict__ A, long long lda, int n, int a,
                                                               int b, int32_t* __restrict__ rowperm) {
    const int npairs = (b - a) / 2;
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        uint32_t* r0 = A + (long long)(a + pr) * lda;
        uint32_t* r1 = A + (long long)(b - 1 - pr) * lda;
        for (int col = blockIdx.y * blockDim.x + threadIdx.x; col < n; col += gridDim.y * blockDim.x) {
            const uint32_t x = r0[col];
            r0[col] = r1[col];
            r1[col] = x;
        }
        if (blockIdx.y == 0 && threadIdx.x == 0) {
            const int32_t x = rowperm[a + pr];
            rowperm[a + pr] = rowperm[b - 1 - pr];
            rowperm[b - 1 - pr] = x;
        }
    }
}

// out[0] = 1 / a[0] mod p (a pivot found by the whole-row search).
__global__ void inv1_kernel(const uint32_t* a, uint32_t p, uint32_t* out) {
    if (threadIdx.x == 0) out[0] = inv_mod_dev(a[0], p);
}

__global__ void iota_kernel(int32_t* v, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

// Parity of a permutation: the number of inversions mod 2, xor-ed into *parity.
__global__ void __launch_bounds__(kThreads) perm_parity_kernel(const int32_t* __restrict__ perm, int n,
                                                               unsigned* parity) {
    __shared__ int32_t tile[kThreads];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t pi = i < n ? perm[i] : 0;
    unsigned cnt = 0;
    for (int j0 = blockIdx.x * blockDim.x; j0 < n; j0 += blockDim.x) {
        const int jj = j0 + threadIdx.x;
        tile[threadIdx.x] = jj < n ? perm[jj] : INT_MAX;
        __syncthreads();
        const int lim = min((int)blockDim.x, n - j0);
        for (int x = 0; x < lim; ++x)
            if (j0 + x > i && tile[x] < pi) cnt ^= 1u;
        __syncthreads();
    }
    if (i < n && cnt) atomicXor(parity, 1u);
}

// det = (-1)^parity * prod_i M[i][i] mod p (one CTA); rank deficiency handled on the host.
__global__ void __launch_bounds__(1024) lqup_det_kernel(const uint32_t* __restrict__ M, long long ld, int n, uint32_t p,
                                                        unsigned long long mu, const unsigned* parity, uint32_t* out) {
    __shared__ uint32_t red[1024];
    uint32_t acc = 1u % p;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        acc = mod_u64((unsigned long long)acc * __ldg(M + (long long)i * ld + i), p, mu);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = mod_u64((unsigned long long)red[threadIdx.x] * red[threadIdx.x + s], p, mu);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint32_t d = red[0];
        out[0] = (*parity & 1u) && d ? p - d : d;
    }
}

__global__ void identity_kernel(uint32_t* X, long long ld, int n) {
    const long long total = (long long)n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / n), c = (int)(i - (long long)r * n);
        X[(long long)r * ld + c] = r == c ? 1u : 0u;
    }
}

// X[perm[j]][:] = Y[j][:]
__global__ void __launch_bounds__(kThreads) row_scatter_kernel(const uint32_t* __restrict__ Y, long long ldy,
                                                               uint32_t* __restrict__ X, long long ldx, int n,
                                                               const int32_t* __restrict__ perm) {
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const uint32_t* src = Y + (long long)j * ldy;
        uint32_t* dst = X + (long long)perm[j] * ldx;
        for (int c = threadIdx.x; c < n; c += blockDim.x) dst[c] = src[c];
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int grid_rows(int64_t rows) { return (int)std::max<int64_t>(1, std::min<int64_t>(rows, 152 * 16)); }

// Host mirror of a leaf's outcome (pinned, one per host thread).
int* pinned_words() {
    thread_local int* buf = nullptr;
    if (!buf && cudaMallocHost(&buf, 64) != cudaSuccess) buf = nullptr;
    return buf;
}

// Split of h rows: on a leaf boundary above the leaf size, in halves below it.
int64_t split_rows(int64_t h) {
    if (h <= kLeafRows) return h / 2;
    const int64_t nb = (h + kLeafRows - 1) / kLeafRows;
    return (nb / 2) * kLeafRows;
}

// Window width: wide enough for a leaf's pivots plus the columns that small
// fields skip (a zero Schur entry has probability 1/p: above 2^16 a 64-row
// leaf meets one with probability below 10^-3, and then only splits).
int window_for(uint32_t p) { return p > 65536 ? kLeafRows : p > 64 ? kLeafRows + 32 : kMaxWin; }

struct Layout {
    size_t rows, e, usp, t1, g, info, words, rest;  // byte offsets; rest = products' workspace
    size_t prod;                             // bytes the products need
    size_t side;                             // the look-ahead products' workspace (prod bytes)
};

// Products of the recursion with the top half at full rank and the whole
// width: the largest shapes a call can meet (a smaller rank shortens the inner
// dimension; the width is at most n).  Every call checks its need again.
void products_bound(int64_t h, int64_t n, uint32_t p, int sms, size_t& best) {
    if (h <= 1) return;
    const int64_t h1 = split_rows(h), h2 = h - h1;
    const int64_t r1 = std::min(h1, n), r2 = std::min(h2, n);
    if (r1 > 0) {
        best = std::max(best, fgemm_ws_bytes(h2, n, r1, p, sms));   // G and the update
        best = std::max(best, fgemm_ws_bytes(r1, r2, r2, p, sms));  // Y' U_b^{-1}
        best = std::max(best, fgemm_ws_bytes(r1, r2, r1, p, sms));  // -U_a^{-1} (Y' U_b^{-1})
    }
    products_bound(h1, n, p, sms, best);
    if (h2 != h1) products_bound(h2, n, p, sms, best);
}

Layout layout(int64_t m, int64_t n, uint32_t p, int sms) {
    Layout Y;
    Y.rows = 0;
    Y.e = align256(size_t(kLeafRows) * std::max<int64_t>(n, 1) * 4);
    // inverses of pivot blocks: at most min(top half of the rows, n) square
    const size_t cap = (size_t)std::max<int64_t>(1, std::min(m > 1 ? split_rows(m) : 1, std::max<int64_t>(n, 1)));
    Y.usp = Y.e + align256(size_t(kLeafRows) * kLeafRows * 4);
    Y.t1 = Y.usp + align256(cap * cap * 4);
    Y.g = Y.t1 + align256(cap * cap * 4);
    Y.info = Y.g + align256(size_t(kGWords) * 4);
    Y.words = Y.info + align256(sizeof(LeafInfo));
    Y.rest = Y.words + 256;
    Y.prod = 0;
    products_bound(m, n, p, sms, Y.prod);
    Y.side = Y.rest + align256(Y.prod);
    return Y;
}

struct Ctx {
    uint32_t p;
    unsigned long long mu;
    uint32_t two64p;
    int64_t m, n;
    uint32_t* A;
    int64_t lda;
    int32_t* rowperm;
    int32_t* colperm;
    uint32_t* rows;
    uint32_t* E;
    uint32_t* Usp;  // inverse of a top half's pivot block when no caller asked for it
    uint32_t* T1;   // scratch for Y' U_b^{-1}
    uint32_t* G;    // scratch for a small product G = X U_a^{-1} that cannot be formed in place
    LeafInfo* info;
    void* ws;
    size_t ws_bytes;
    int* err;
    cudaStream_t s;
    int win;
    int* host;
    int sms;
    // look-ahead (null s2: off): the update of a bottom half's rows below its
    // first leaf runs on s2, with its own workspace, while that leaf is
    // factored; pending until the main stream has waited for ev_done
    cudaStream_t s2;
    cudaEvent_t ev_go, ev_done;
    void* ws2;
    size_t ws2_bytes;
    mutable bool pending;
};

// The main stream waits for the pending side-stream update (a no-op when
// none is pending).  Called before any launch that may touch rows other than
// the current leaf's.
ffgpu_status join(const Ctx& x) {
    if (!x.pending) return FFGPU_OK;
    x.pending = false;
    return cudaStreamWaitEvent(x.s, x.ev_done, 0) == cudaSuccess ? FFGPU_OK : FFGPU_ERR_CUDA;
}

// One side stream and two events per host thread and device, created on
// first use and kept for the thread's lifetime.
struct SideRes {
    cudaStream_t s = nullptr;
    cudaEvent_t go = nullptr, done = nullptr;
};

const SideRes* side_resources() {
    thread_local std::map<int, SideRes> all;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    SideRes& r = all[dev];
    if (!r.s) {
        SideRes t;
        if (cudaStreamCreateWithFlags(&t.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&t.go, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess) {
            if (t.done) cudaEventDestroy(t.done);
            if (t.go) cudaEventDestroy(t.go);
            if (t.s) cudaStreamDestroy(t.s);
            return nullptr;
        }
        r = t;
    }
    return &r;
}

ffgpu_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? FFGPU_OK : FFGPU_ERR_CUDA; }

size_t smem_window(int h, int WS) { return (size_t(h) * WS + 4 * size_t(h) * h + 2 * size_t(kTmWords)) * 4; }
size_t smem_rest(int h) { return size_t(h) * kRestCols * 4 + size_t(h) * h * 4; }

ffgpu_status set_attrs() {
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, [] {
        e = cudaFuncSetAttribute(lqup_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_window(kLeafRows, kMaxWin));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(lqup_rest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_rest(kLeafRows));
    });
    return cuda_ok(e);
}

// Rows [rb, rb + h) on the active columns [c, n).  Sets *ok = false (nothing
// written) when a pivot lies beyond the window and h > 1.
ffgpu_status leaf(const Ctx& x, int64_t rb, int64_t h, int64_t c, int64_t* rank, bool* ok, uint32_t* Uo,
                  int64_t ldu) {
    const int64_t w = x.n - c;
    const int W = (int)std::min<int64_t>(x.win, w);
    const int WS = (W + 31) & ~31;
    uint32_t* Ab = x.A + rb * x.lda;
    ffgpu_status st = cuda_ok(timed_launch("lqup_window", x.s, [&] {
        lqup_window_kernel<<<1, kWinThreads, smem_window((int)h, WS), x.s>>>(
            Ab + c, x.lda, (int)h, W, WS, x.p, x.mu, x.two64p, x.E, Uo, ldu, x.rows + c, x.n, x.info);
        return cudaGetLastError();
    }));
    if (st != FFGPU_OK) return st;
    // The window's outcome first: with every row a pivot no residual can be
    // non-zero, so the rest of the leaf needs no second round trip.  (A
    // pending side-stream update runs meanwhile: the window kernel reads and
    // writes only this leaf's rows and the leaf's scratch.)
    if ((st = cuda_ok(cudaMemcpyAsync(x.host, x.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, x.s))) != FFGPU_OK)
        return st;
    if ((st = cuda_ok(cudaStreamSynchronize(x.s))) != FFGPU_OK) return st;
    const int r = x.host[0];
    if ((st = join(x)) != FFGPU_OK) return st;
    const int nleft = (int)((c + kThreads - 1) / kThreads);
    const int nright = w > W ? (int)((w - W + kRestCols - 1) / kRestCols) : 0;
    if (nleft + nright > 0) {
        st = cuda_ok(timed_launch("lqup_rest", x.s, [&] {
            lqup_rest_kernel<<<nleft + nright, kThreads, smem_rest((int)h), x.s>>>(
                Ab, x.lda, (int)h, (int)c, W, (int)x.n, nleft, x.p, x.mu, x.two64p, x.E, x.rows, x.n, x.info);
            return cudaGetLastError();
        }));
        if (st != FFGPU_OK) return st;
    }
    int fail = 0, ident = x.host[2], firstnz = INT_MAX;
    if (r < h && nright > 0) {
        // non-pivot rows: their residuals beyond the window decide
        if ((st = cuda_ok(cudaMemcpyAsync(x.host, x.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, x.s))) !=
            FFGPU_OK)
            return st;
        if ((st = cuda_ok(cudaStreamSynchronize(x.s))) != FFGPU_OK) return st;
        fail = x.host[1];
        ident = x.host[2];
        firstnz = x.host[3];
    }
    if (fail) {
        if (h > 1) {
            *ok = false;
            return FFGPU_OK;
        }
        // one row, zero on the window: its pivot is the first non-zero column
        st = cuda_ok(timed_launch("lqup_colrot", x.s, [&] {
            lqup_colrot_kernel<<<grid_rows(x.m + 1), kThreads, 0, x.s>>>(x.A, x.lda, (int)x.m, (int)c, firstnz,
                                                                         x.colperm);
            if (Uo) inv1_kernel<<<1, 32, 0, x.s>>>(Ab + c, x.p, Uo);
            return cudaGetLastError();
        }));
        *rank = 1;
        *ok = true;
        return st;
    }
    if ((st = cuda_ok(cudaMemcpy2DAsync(Ab, x.lda * 4, x.rows, x.n * 4, x.n * 4, h, cudaMemcpyDeviceToDevice,
                                        x.s))) != FFGPU_OK)
        return st;
    st = cuda_ok(timed_launch("lqup_rowperm", x.s, [&] {
        lqup_rowperm_kernel<<<1, kThreads, 0, x.s>>>(x.rowperm + rb, (int)h, x.info);
        return cudaGetLastError();
    }));
    if (st != FFGPU_OK) return st;
    if (!ident && x.m > h) {
        st = cuda_ok(timed_launch("lqup_colperm", x.s, [&] {
            lqup_colperm_kernel<<<grid_rows(x.m), kThreads, 0, x.s>>>(x.A, x.lda, (int)x.m, (int)rb, (int)(rb + h),
                                                                      (int)c, W, x.info, x.colperm);
            return cudaGetLastError();
        }));
        if (st != FFGPU_OK) return st;
    } else if (!ident) {
        // no row outside the leaf: colperm alone
        st = cuda_ok(timed_launch("lqup_colperm", x.s, [&] {
            lqup_colperm_kernel<<<1, kThreads, 0, x.s>>>(x.A, x.lda, 0, 0, 0, (int)c, W, x.info, x.colperm);
            return cudaGetLastError();
        }));
        if (st != FFGPU_OK) return st;
    }
    *rank = r;
    *ok = true;
    return FFGPU_OK;
}

ffgpu_status reverse_rows(const Ctx& x, int64_t a, int64_t b) {
    if (b - a < 2) return FFGPU_OK;
    const dim3 grid((unsigned)std::min<int64_t>((b - a) / 2, 65535), (unsigned)std::min<int64_t>((x.n + 1023) / 1024, 8));
    return cuda_ok(timed_launch("lqup_rowrev", x.s, [&] {
        lqup_rowrev_kernel<<<grid, kThreads, 0, x.s>>>(x.A, x.lda, (int)x.n, (int)a, (int)b, x.rowperm);
        return cudaGetLastError();
    }));
}

// Rows [rb, rb + h) on the active columns [c, n); *rank receives their rank r.
// With Uo not null, the inverse of their pivot block (U restricted to these
// rows and their pivot columns: r x r, upper triangular) is written to Uo
// (leading dimension ldu), zeros below its diagonal.
//
// After the top half (rank r1, pivot block U_a), the bottom half's
// multipliers are G = X U_a^{-1}: one product written over X (fgemm converts
// both operands before it writes, so the output may overlap A).  The inverse
// of the whole pivot block [[U_a, Y'], [0, U_b]] is assembled from the
// halves' inverses: its off-diagonal block is -U_a^{-1} Y' U_b^{-1}, two
// products (Y' = the top rows on the bottom half's pivot columns).
ffgpu_status rec(const Ctx& x, int64_t rb, int64_t h, int64_t c, int64_t* rank, uint32_t* Uo, int64_t ldu) {
    *rank = 0;
    if (h == 0 || c >= x.n) return FFGPU_OK;
    ffgpu_status st;
    if (h <= kLeafRows) {
        bool ok = false;
        if ((st = leaf(x, rb, h, c, rank, &ok, Uo, ldu)) != FFGPU_OK || ok) return st;
    }
    const int64_t h1 = split_rows(h), h2 = h - h1;
    int64_t r1 = 0, r2 = 0;
    // the top half's inverse: into Uo's leading block, else into the scratch
    // (only this node reads it, before the bottom half runs)
    uint32_t* Ua = Uo ? Uo : x.Usp;
    const int64_t lda_u = Uo ? ldu : std::min(h1, x.n - c);  // r1 <= min(h1, n - c)
    if ((st = rec(x, rb, h1, c, &r1, Ua, lda_u)) != FFGPU_OK) return st;
    if ((st = join(x)) != FFGPU_OK) return st;
    const int sms = x.sms;
    auto product = [&](int64_t m, int64_t n, int64_t k, uint32_t alpha, const uint32_t* Ap, int64_t la,
                       const uint32_t* Bp, int64_t lb, uint32_t beta, uint32_t* Cp, int64_t lc) -> ffgpu_status {
        if (m == 0 || n == 0 || k == 0) return FFGPU_OK;
        if (fgemm_ws_bytes(m, n, k, x.p, sms) > x.ws_bytes) return FFGPU_ERR_NOMEM;
        return fgemm_run(m, n, k, x.p, alpha, Ap, la, Bp, lb, beta, Cp, lc, x.ws, x.ws_bytes, x.err, x.s, 0, false);
    };
    if (r1 > 0) {
        uint32_t* top = x.A + rb * x.lda + c;
        uint32_t* bot = x.A + (rb + h1) * x.lda + c;
        // G = X U_a^{-1}, in place when the product reads all of X before it
        // writes (the tensor-core route converts its operands first; the
        // CUDA-core kernel does when one column tile covers G), else through
        // a scratch (a small product: h2 r1 <= 2^27 / r1 < kGWords)
        if (fgemm_small(h2, r1, r1) ? r1 <= 64 : fgemm_single_pass(x.p, r1)) {
            if ((st = product(h2, r1, r1, 1, bot, x.lda, Ua, lda_u, 0, bot, x.lda)) != FFGPU_OK) return st;
        } else {
            if (!fgemm_small(h2, r1, r1) || h2 * r1 > kGWords) return FFGPU_ERR_INVALID;
            if ((st = product(h2, r1, r1, 1, bot, x.lda, Ua, lda_u, 0, x.G, r1)) != FFGPU_OK) return st;
            if (cudaMemcpy2DAsync(bot, x.lda * 4, x.G, r1 * 4, r1 * 4, h2, cudaMemcpyDeviceToDevice, x.s) !=
                cudaSuccess)
                return FFGPU_ERR_CUDA;
        }
        // Z <- Z - G Y
        const int64_t w = x.n - c - r1;
        const int64_t wz = std::min<int64_t>(w, x.win);  // the bottom half's first window
        if (w > wz && x.s2 && h2 > kLeafRows && !fgemm_small(h2, w - wz, r1) &&
            fgemm_ws_bytes(h2, w - wz, r1, x.p, sms) <= x.ws2_bytes) {
            // look-ahead: the columns of the bottom half's first window here,
            // the others on the side stream, on all but two SMs, while that
            // window is factored on one of the two (its kernel touches only
            // the first leaf's rows on those columns; every later launch
            // joins the side stream first).  A product on the CUDA-core
            // route would take every SM, so it stays on this stream.
            if ((st = product(h2, wz, r1, x.p - 1, bot, x.lda, top + r1, x.lda, 1, bot + r1, x.lda)) != FFGPU_OK)
                return st;
            if (cudaEventRecord(x.ev_go, x.s) != cudaSuccess || cudaStreamWaitEvent(x.s2, x.ev_go, 0) != cudaSuccess)
                return FFGPU_ERR_CUDA;
            if ((st = fgemm_run(h2, w - wz, r1, x.p, x.p - 1, bot, x.lda, top + r1 + wz, x.lda, 1, bot + r1 + wz,
                                x.lda, x.ws2, x.ws2_bytes, x.err, x.s2, std::max(2, sms - 2), false)) != FFGPU_OK)
                return st;
            if (cudaEventRecord(x.ev_done, x.s2) != cudaSuccess) return FFGPU_ERR_CUDA;
            x.pending = true;
        } else if (w > 0 &&
                   (st = product(h2, w, r1, x.p - 1, bot, x.lda, top + r1, x.lda, 1, bot + r1, x.lda)) != FFGPU_OK) {
            return st;
        }
    }
    uint32_t* Ub = Uo ? Uo + r1 * ldu + r1 : nullptr;
    if ((st = rec(x, rb + h1, h2, c + r1, &r2, Ub, ldu)) != FFGPU_OK) return st;
    if ((st = join(x)) != FFGPU_OK) return st;
    if (r2 > 0 && h1 > r1) {
        // [top non-pivot rows | bottom pivot rows] -> [bottom pivot rows | top non-pivot rows]
        if ((st = reverse_rows(x, rb + r1, rb + h1)) != FFGPU_OK) return st;
        if ((st = reverse_rows(x, rb + h1, rb + h1 + r2)) != FFGPU_OK) return st;
        if ((st = reverse_rows(x, rb + r1, rb + h1 + r2)) != FFGPU_OK) return st;
    }
    if (Uo && r1 > 0 && r2 > 0) {
        // [[U_a^{-1}, -U_a^{-1} Y' U_b^{-1}], [0, U_b^{-1}]]
        if (cudaMemset2DAsync(Uo + r1 * ldu, ldu * 4, 0, r1 * 4, r2, x.s) != cudaSuccess) return FFGPU_ERR_CUDA;
        const uint32_t* Yp = x.A + rb * x.lda + c + r1;
        if ((st = product(r1, r2, r2, 1, Yp, x.lda, Ub, ldu, 0, x.T1, r2)) != FFGPU_OK) return st;
        if ((st = product(r1, r2, r1, x.p - 1, Uo, ldu, x.T1, r2, 0, Uo + r1, ldu)) != FFGPU_OK) return st;
    }
    *rank = r1 + r2;
    return FFGPU_OK;
}

unsigned long long mulmod_host(unsigned long long a, unsigned long long b, unsigned long long p) {
    return (unsigned long long)((unsigned __int128)a * b % p);
}

}  // namespace

// Deterministic Miller-Rabin for 32-bit n (bases 2, 3, 5, 7 suffice below 3.2e9).
bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    for (uint32_t b : {2u, 3u, 5u, 7u})
        if (n % b == 0) return n == b;
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    for (unsigned long long a : {2ull, 3ull, 5ull, 7ull}) {
        unsigned long long x = 1, base = a % n, e = d;
        while (e) {
            if (e & 1) x = mulmod_host(x, base, n);
            base = mulmod_host(base, base, n);
            e >>= 1;
        }
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; ++i) {
            x = mulmod_host(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

size_t lqup_ws_bytes(int64_t m, int64_t n, uint32_t p, int sms) {
    const Layout Y = layout(m, n, p, sms);
    return Y.side + align256(Y.prod);
}

// In-place LQUP of the m x n matrix A (entries reduced mod p first).
// rowperm (m) and colperm (n) are device arrays; ws holds lqup_ws_bytes.
ffgpu_status lqup_run(int64_t m, int64_t n, uint32_t p, uint32_t* A, int64_t lda, int64_t* rank, int32_t* rowperm,
                      int32_t* colperm, void* ws, size_t ws_bytes, int* err, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    const int sms = sm_count(dev);
    const Layout Y = layout(m, n, p, sms);
    if (ws_bytes < Y.rest) return FFGPU_ERR_NOMEM;
    ffgpu_status st = set_attrs();
    if (st != FFGPU_OK) return st;
    unsigned char* w = static_cast<unsigned char*>(ws);
    Ctx x;
    x.p = p;
    x.mu = ~0ull / p;
    x.two64p = (uint32_t)(((unsigned __int128)1 << 64) % p);
    x.m = m;
    x.n = n;
    x.A = A;
    x.lda = lda;
    x.rowperm = rowperm;
    x.colperm = colperm;
    x.rows = reinterpret_cast<uint32_t*>(w + Y.rows);
    x.E = reinterpret_cast<uint32_t*>(w + Y.e);
    x.Usp = reinterpret_cast<uint32_t*>(w + Y.usp);
    x.T1 = reinterpret_cast<uint32_t*>(w + Y.t1);
    x.G = reinterpret_cast<uint32_t*>(w + Y.g);
    x.info = reinterpret_cast<LeafInfo*>(w + Y.info);
    x.err = err;
    x.s = s;
    x.win = window_for(p);
    x.host = pinned_words();
    if (!x.host) return FFGPU_ERR_NOMEM;
    x.sms = sms;
    x.pending = false;
    x.s2 = nullptr;
    x.ev_go = x.ev_done = nullptr;
    x.ws2 = nullptr;
    x.ws2_bytes = 0;
    const SideRes* sr = ws_bytes >= Y.side + align256(Y.prod) ? side_resources() : nullptr;
    if (sr) {
        x.ws = w + Y.rest;
        x.ws_bytes = Y.side - Y.rest;
        x.s2 = sr->s;
        x.ev_go = sr->go;
        x.ev_done = sr->done;
        x.ws2 = w + Y.side;
        x.ws2_bytes = ws_bytes - Y.side;
    } else {
        x.ws = w + Y.rest;
        x.ws_bytes = ws_bytes - Y.rest;
    }
    if (m > 0)
        iota_kernel<<<grid_rows((m + 255) / 256), 256, 0, s>>>(rowperm, (int)m);
    if (n > 0)
        iota_kernel<<<grid_rows((n + 255) / 256), 256, 0, s>>>(colperm, (int)n);
    if ((st = cuda_ok(cudaGetLastError())) != FFGPU_OK) return st;
    if (m > 0 && n > 0) {
        if (timed_launch("scale_mod_p", s, [&] { return launch_scale(A, lda, (int)m, (int)n, p, 1, x.mu, s); }) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
    }
    int64_t r = 0;
    st = rec(x, 0, m, 0, &r, nullptr, 0);
    if (x.pending) {
        // an error left the side stream's update in flight: let it finish
        // before the workspace is handed back
        cudaStreamSynchronize(x.s2);
        x.pending = false;
    }
    if (st != FFGPU_OK) return st;
    if ((st = cuda_ok(cudaMemcpyAsync(x.host, err, sizeof(int), cudaMemcpyDeviceToHost, s))) != FFGPU_OK) return st;
    if ((st = cuda_ok(cudaStreamSynchronize(s))) != FFGPU_OK) return st;
    if (x.host[0] != 0) return FFGPU_ERR_TIMEOUT;
    *rank = r;
    return FFGPU_OK;
}

// Workspace of the derived routines: the matrix copy M (m x n), rowperm,
// colperm, [Y (n x n) for the inverse], then the factorization's workspace.
struct DerivedLayout {
    size_t M, rp, cp, Yb, words, lq, total;
};

DerivedLayout derived_layout(int64_t m, int64_t n, uint32_t p, bool inverse, int sms) {
    DerivedLayout D;
    D.M = 0;
    D.rp = align256(size_t(m) * n * 4 + 4);
    D.cp = D.rp + align256(size_t(m) * 4 + 4);
    D.Yb = D.cp + align256(size_t(n) * 4 + 4);
    D.words = D.Yb + (inverse ? align256(size_t(n) * n * 4 + 4) : 0);
    D.lq = D.words + 256;
    size_t need = lqup_ws_bytes(m, n, p, sms);
    if (inverse) {
        need = std::max(need, ftrsm_ws_bytes(0, 0, FFGPU_TRSM_DEFAULT, n, n, p, sms));
        need = std::max(need, ftrsm_ws_bytes(0, 1, FFGPU_TRSM_DEFAULT, n, n, p, sms));
    }
    D.total = D.lq + align256(need);
    return D;
}

// Factor a copy of A into the workspace; returns the rank.
ffgpu_status derived_factor(int64_t m, int64_t n, uint32_t p, const uint32_t* A, int64_t lda, const DerivedLayout& D,
                            unsigned char* w, size_t ws_bytes, int* err, cudaStream_t s, int64_t* rank) {
    uint32_t* M = reinterpret_cast<uint32_t*>(w + D.M);
    if (cudaMemcpy2DAsync(M, size_t(n) * 4, A, size_t(lda) * 4, size_t(n) * 4, m, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return FFGPU_ERR_CUDA;
    return lqup_run(m, n, p, M, n, rank, reinterpret_cast<int32_t*>(w + D.rp), reinterpret_cast<int32_t*>(w + D.cp),
                    w + D.lq, ws_bytes - D.lq, err, s);
}

ffgpu_status rank_run(int64_t m, int64_t n, uint32_t p, const uint32_t* A, int64_t lda, int64_t* rank, void* ws,
                      size_t ws_bytes, int* err, cudaStream_t s, int sms) {
    const DerivedLayout D = derived_layout(m, n, p, false, sms);
    if (ws_bytes < D.total) return FFGPU_ERR_NOMEM;
    return derived_factor(m, n, p, A, lda, D, static_cast<unsigned char*>(ws), ws_bytes, err, s, rank);
}

ffgpu_status det_run(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* det, void* ws, size_t ws_bytes,
                     int* err, cudaStream_t s, int sms) {
    const DerivedLayout D = derived_layout(n, n, p, false, sms);
    if (ws_bytes < D.total) return FFGPU_ERR_NOMEM;
    unsigned char* w = static_cast<unsigned char*>(ws);
    int64_t r = 0;
    ffgpu_status st = derived_factor(n, n, p, A, lda, D, w, ws_bytes, err, s, &r);
    if (st != FFGPU_OK) return st;
    if (r < n) {
        *det = 0;
        return FFGPU_OK;
    }
    // full rank: every row is a pivot row (rowperm is the identity), so the
    // sign is colperm's parity
    unsigned* words = reinterpret_cast<unsigned*>(w + D.words);
    if (cudaMemsetAsync(words, 0, 16, s) != cudaSuccess) return FFGPU_ERR_CUDA;
    st = cuda_ok(timed_launch("perm_parity", s, [&] {
        perm_parity_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            reinterpret_cast<const int32_t*>(w + D.cp), (int)n, words);
        return cudaGetLastError();
    }));
    if (st != FFGPU_OK) return st;
    st = cuda_ok(timed_launch("lqup_det", s, [&] {
        lqup_det_kernel<<<1, 1024, 0, s>>>(reinterpret_cast<const uint32_t*>(w + D.M), n, (int)n, p, ~0ull / p, words,
                                           words + 1);
        return cudaGetLastError();
    }));
    if (st != FFGPU_OK) return st;
    if (cudaMemcpyAsync(det, words + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return FFGPU_ERR_CUDA;
    return cuda_ok(cudaStreamSynchronize(s));
}

ffgpu_status inverse_run(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* X, int64_t ldx, void* ws,
                         size_t ws_bytes, int* err, cudaStream_t s, int sms) {
    const DerivedLayout D = derived_layout(n, n, p, true, sms);
    if (ws_bytes < D.total) return FFGPU_ERR_NOMEM;
    unsigned char* w = static_cast<unsigned char*>(ws);
    int64_t r = 0;
    ffgpu_status st = derived_factor(n, n, p, A, lda, D, w, ws_bytes, err, s, &r);
    if (st != FFGPU_OK) return st;
    if (r < n) return FFGPU_ERR_SINGULAR;
    // A = L U P^{-1} (rowperm is the identity at full rank), so
    // A^{-1} = P U^{-1} L^{-1}: Y = I, Y <- L^{-1} Y, Y <- U^{-1} Y, X[colperm[j]] = Y[j]
    const uint32_t* M = reinterpret_cast<const uint32_t*>(w + D.M);
    uint32_t* Yv = reinterpret_cast<uint32_t*>(w + D.Yb);
    st = cuda_ok(timed_launch("identity", s, [&] {
        identity_kernel<<<grid_rows(((int64_t)n * n + 255) / 256), 256, 0, s>>>(Yv, n, (int)n);
        return cudaGetLastError();
    }));
    if (st != FFGPU_OK) return st;
    if ((st = ftrsm_run(0, 0, 1, FFGPU_TRSM_DEFAULT, n, n, p, 1, M, n, Yv, n, w + D.lq, ws_bytes - D.lq, err, s)) !=
        FFGPU_OK)
        return st;
    if ((st = ftrsm_run(0, 1, 0, FFGPU_TRSM_DEFAULT, n, n, p, 1, M, n, Yv, n, w + D.lq, ws_bytes - D.lq, err, s)) !=
        FFGPU_OK)
        return st;
    st = cuda_ok(timed_launch("row_scatter", s, [&] {
        row_scatter_kernel<<<grid_rows(n), kThreads, 0, s>>>(Yv, n, X, ldx, (int)n,
                                                             reinterpret_cast<const int32_t*>(w + D.cp));
        return cudaGetLastError();
    }));
    if (st != FFGPU_OK) return st;
    int* host = pinned_words();
    if (!host) return FFGPU_ERR_NOMEM;
    if (cudaMemcpyAsync(host, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FFGPU_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FFGPU_ERR_CUDA;
    return host[0] ? FFGPU_ERR_TIMEOUT : FFGPU_OK;
}

size_t derived_ws_bytes(int64_t m, int64_t n, uint32_t p, bool inverse, int sms) {
    return derived_layout(m, n, p, inverse, sms).total;
}

}  // namespace ffgpu

using namespace ffgpu;

namespace {

ffgpu_status check_field(uint32_t p) {
    if (p < 2 || p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
    return is_prime_u32(p) ? FFGPU_OK : FFGPU_ERR_UNSUPPORTED_P;
}

ffgpu_status device_and_sms(int* sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    *sms = sm_count(dev);
    return FFGPU_OK;
}

}  // namespace

extern "C" {

ffgpu_status ffgpu_lqup(int64_t m, int64_t n, uint32_t p, uint32_t* A, int64_t lda, int64_t* rank, int32_t* rowperm,
                        int32_t* colperm, void* stream) {
    ffgpu_status st = check_field(p);
    if (st != FFGPU_OK) return st;
    if (m < 0 || n < 0 || m > INT32_MAX / 2 || n > INT32_MAX / 2 || !rank) return FFGPU_ERR_INVALID;
    if ((m > 0 && n > 0 && (!A || lda < n)) || (m > 0 && !rowperm) || (n > 0 && !colperm)) return FFGPU_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    if ((st = device_and_sms(&sms)) != FFGPU_OK) return st;
    Pool* pool = nullptr;
    if ((st = pool_get(s, lqup_ws_bytes(m, n, p, sms), &pool)) != FFGPU_OK) return st;
    return lqup_run(m, n, p, A, lda, rank, rowperm, colperm, pool->ptr, pool->bytes, pool->err, s);
}

ffgpu_status ffgpu_rank(int64_t m, int64_t n, uint32_t p, const uint32_t* A, int64_t lda, int64_t* rank,
                        void* stream) {
    ffgpu_status st = check_field(p);
    if (st != FFGPU_OK) return st;
    if (m < 0 || n < 0 || m > INT32_MAX / 2 || n > INT32_MAX / 2 || !rank) return FFGPU_ERR_INVALID;
    if (m > 0 && n > 0 && (!A || lda < n)) return FFGPU_ERR_INVALID;
    if (m == 0 || n == 0) {
        *rank = 0;
        return FFGPU_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    if ((st = device_and_sms(&sms)) != FFGPU_OK) return st;
    Pool* pool = nullptr;
    if ((st = pool_get(s, derived_ws_bytes(m, n, p, false, sms), &pool)) != FFGPU_OK) return st;
    return rank_run(m, n, p, A, lda, rank, pool->ptr, pool->bytes, pool->err, s, sms);
}

ffgpu_status ffgpu_det(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* det, void* stream) {
    ffgpu_status st = check_field(p);
    if (st != FFGPU_OK) return st;
    if (n < 0 || n > INT32_MAX / 2 || !det) return FFGPU_ERR_INVALID;
    if (n > 0 && (!A || lda < n)) return FFGPU_ERR_INVALID;
    if (n == 0) {
        *det = 1;
        return FFGPU_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    if ((st = device_and_sms(&sms)) != FFGPU_OK) return st;
    Pool* pool = nullptr;
    if ((st = pool_get(s, derived_ws_bytes(n, n, p, false, sms), &pool)) != FFGPU_OK) return st;
    return det_run(n, p, A, lda, det, pool->ptr, pool->bytes, pool->err, s, sms);
}

ffgpu_status ffgpu_inverse(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* X, int64_t ldx,
                           void* stream) {
    ffgpu_status st = check_field(p);
    if (st != FFGPU_OK) return st;
    if (n < 0 || n > INT32_MAX / 2) return FFGPU_ERR_INVALID;
    if (n > 0 && (!A || !X || lda < n || ldx < n)) return FFGPU_ERR_INVALID;
    if (n == 0) return FFGPU_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    if ((st = device_and_sms(&sms)) != FFGPU_OK) return st;
    Pool* pool = nullptr;
    if ((st = pool_get(s, derived_ws_bytes(n, n, p, true, sms), &pool)) != FFGPU_OK) return st;
    return inverse_run(n, p, A, lda, X, ldx, pool->ptr, pool->bytes, pool->err, s, sms);
}

}  // extern "C"
