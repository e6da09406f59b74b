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
// column the check found.  A leaf whose rows are all pivots commits whatever
// lies beyond the window, so both kernels then write A in place (and the rest
// kernel reorders rowperm); otherwise they write scratch rows, copied to A on
// commit.  The host reads every leaf's outcome (rank, commit or split) before
// it issues the next step: the calls are host-synchronous.
//
// Look-ahead.  Where a node's update Z <- Z - G Y takes the tensor-core route
// and its bottom half has more than one leaf, the columns of the bottom
// half's first window are updated first on the caller's stream and the
// others on a side stream (its own workspace, all but two SMs), so that the
// first leaf's window kernel runs while the rest of the update does; every
// later launch makes the caller's stream wait for the side stream first.
#include <algorithm>
#include <chrono>
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
// the rest kernel); the first five ints are read back by the host.
struct LeafInfo {
    int rank;                 // pivots found in the window
    int fail;                 // some non-pivot row has a non-zero residual beyond the window
    int ident;                // the window's columns keep their order
    int firstnz;              // smallest column of such a residual (absolute index)
    int timeout;              // a bounded wait of the window kernel ran out
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

// Window factorization of one leaf (one CTA of kWinThreads).  A points at
// (rb, c); the leaf's tile is h x W (zero padding up to WS, a multiple of 32).
//
// Arithmetic.  For odd p the kernel works in Montgomery form with R = 2^32
// (x held as x R mod p): a product is one 64-bit multiply and one reduction,
// with no precomputed quotient of either factor, and the update
// P v - a u of an entry is a single reduction of P v + a (p - u) < 2 p^2 < p R.
// p = 2 works on plain bits (product AND, difference XOR).
//
// Elimination.  Fraction-free and row by row, so that no row waits for a
// modular inverse: row t' below pivot k (row t, column j, stored value P)
// becomes P row_t' - a row_t with a its stored entry in column j, and its
// scale d_t' (the factor by which the stored row exceeds the true Schur
// complement) is multiplied by P.  Each row is extended by the identity row
// of the leaf, so that the same operations turn the extension into d_t times
// row t of the leaf's elimination matrix E (E times the leaf's rows gives its
// eliminated rows).  Warp w holds rows w, w + 16, w + 32, w + 48 in registers
// (lane l columns l, l + 32, ...).  Rows are published in shared memory once
// final: row t is final after the pivots of rows 0 .. t-1, and its owner
// publishes it (values, pivot column, stored pivot, scale) and arrives on
// row t's mbarrier.  Every warp takes the rows in order, waits for each on its
// mbarrier (a bounded wait), and updates its own rows below it; the owner of
// row t + 1 updates that row first and publishes it at once, so that the chain
// of pivot decisions passes from warp to warp without a barrier of the CTA.
//
// Afterwards one batched inversion of the pivots (prefix and suffix products
// over a warp, one extended-Euclid inverse) gives the true multipliers
// l_t'k = a d_t / (P d_t') (prefix products of the inverse pivots per row),
// the true U rows and E (each stored row times 1 / d_t).  The inverse of the
// pivot block U11 (r x r, upper triangular) is left to the rest kernel's last
// CTA (u11_inverse), which runs beside the rest of the rows.
//
// Writes the leaf's new rows on the window (over A's window when every row
// is a pivot, else to the scratch rows: rows points at their column c), E
// (h x h, original row order), the LeafInfo and, when the caller asks for
// the inverse of the pivot block (Uig not null), U11 and the inverse of its
// diagonal to Usc.
constexpr int kWinWarps = kWinThreads / 32;
constexpr int kRowsPerWarp = kLeafRows / kWinWarps;
constexpr int kExt = kLeafRows;              // columns of the identity extension
constexpr int kTmWords = kLeafRows * kLeafRows / 4;  // doubling products of one level (npairs s^2 <= 32 s)

template <bool kBin>
struct WinField {
    uint32_t p, pinv, r2, one;  // pinv = -p^{-1} mod 2^32, r2 = R^2 mod p, one = R mod p
    __device__ __forceinline__ WinField(uint32_t p_, uint32_t two64p, unsigned long long mu) : p(p_) {
        if (kBin) {
            pinv = 0u;
            r2 = one = 1u;
        } else {
            uint32_t x = p;  // Newton's iteration for p^{-1} mod 2^32 (3, 6, 12, 24, 48 bits)
#pragma unroll
            for (int i = 0; i < 4; ++i) x *= 2u - p * x;
            pinv = 0u - x;
            r2 = two64p;
            one = mod_u64(1ull << 32, p, mu);
        }
    }
    __device__ __forceinline__ uint32_t redc(unsigned long long t) const {  // t < p R
        const uint32_t m = (uint32_t)t * pinv;
        const unsigned long long u = (t + (unsigned long long)m * p) >> 32;
        return u >= p ? (uint32_t)(u - p) : (uint32_t)u;
    }
    __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const {
        return kBin ? (a & b) : redc((unsigned long long)a * b);
    }
    // P v + a w (w = neg(u)): the update P v - a u
    __device__ __forceinline__ uint32_t fma2(uint32_t P, uint32_t v, uint32_t a, uint32_t w) const {
        return kBin ? ((P & v) ^ (a & w)) : redc((unsigned long long)P * v + (unsigned long long)a * w);
    }
    __device__ __forceinline__ uint32_t neg(uint32_t u) const { return kBin || u == 0u ? u : p - u; }
    __device__ __forceinline__ uint32_t to(uint32_t x) const { return kBin ? x : redc((unsigned long long)x * r2); }
    __device__ __forceinline__ uint32_t from(uint32_t x) const { return kBin ? x : redc(x); }
    __device__ __forceinline__ uint32_t inv(uint32_t x) const { return kBin ? x : to(inv_mod_dev(from(x), p)); }
};

template <int N, int NA>
__device__ __forceinline__ uint32_t pick(const uint32_t (&v)[NA], int c) {
    uint32_t x = 0u;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i == c) x = v[i];
    return x;
}

// Shared state of the elimination.
struct WinState {
    uint32_t* U;     // [h][WA]: published rows (window, then the identity extension)
    uint32_t* Lsm;   // [h][h]: numerators a (row t, pivot k), then the true multipliers
    uint64_t* bar;   // [h]: row t published
    int* jp;         // pivot column of row t (-1: none)
    uint32_t* Pv;    // stored pivot of row t
    uint32_t* dv;    // scale of row t
    int* pre;        // pivots above row t
    int* prow;       // pivot k's row
    int* pcol;       // pivot k's column
    uint32_t* P;     // pivot k's stored value
    int* colpiv;     // window column -> pivot number (-1: none)
    int* rowpiv;     // row -> pivot number (-1: none)
    volatile int* abort_flag;
};

// Publish row t (this warp's registers v; kk pivots above it; scale d).
template <int NCW, int NCA>
__device__ __forceinline__ void win_publish(const uint32_t (&v)[NCA], int t, int kk, uint32_t d, const WinState& S,
                                            int WA) {
    const int lane = threadIdx.x & 31;
    int j = -1;
#pragma unroll
    for (int c = 0; c < NCW; ++c) {
        const unsigned bal = __ballot_sync(0xffffffffu, v[c] != 0u);
        if (j < 0 && bal) j = 32 * c + __ffs(bal) - 1;
    }
#pragma unroll
    for (int c = 0; c < NCA; ++c) S.U[t * WA + lane + 32 * c] = v[c];
    const uint32_t P = j >= 0 ? __shfl_sync(0xffffffffu, pick<NCW>(v, j >> 5), j & 31) : 0u;
    if (lane == 0) {
        S.jp[t] = j;
        S.Pv[t] = P;
        S.dv[t] = d;
        S.pre[t] = kk;
        if (j >= 0) {
            S.prow[kk] = t;
            S.pcol[kk] = j;
            S.P[kk] = P;
            S.colpiv[j] = kk;
            S.rowpiv[t] = kk;
        }
    }
    __syncwarp();
    mbar_arrive(&S.bar[t]);  // each lane releases its own stores
}

// Row update by pivot row u (w = its negated values): v <- P v - a u with
// a = v[j]; the numerator goes to *lnum.  Nothing when a = 0.
template <bool kBin, int NCW, int NCA>
__device__ __forceinline__ void win_update(const WinField<kBin>& F, uint32_t (&v)[NCA], uint32_t& d,
                                           const uint32_t (&w)[NCA], int j, uint32_t P, uint32_t* lnum) {
    const uint32_t a = __shfl_sync(0xffffffffu, pick<NCW>(v, j >> 5), j & 31);
    if (a == 0u) return;
    if ((threadIdx.x & 31) == 0) *lnum = a;
#pragma unroll
    for (int c = 0; c < NCA; ++c) v[c] = F.fma2(P, v[c], a, w[c]);
    d = F.mul(d, P);
}

// The elimination; returns the rank on the window, or -1 if a wait ran out.
template <bool kBin, int NCW>
__device__ int win_eliminate(const WinField<kBin>& F, const uint32_t* A, long long lda, int h, int W,
                             const WinState& S, int* timeout) {
    constexpr int NCA = NCW + kExt / 32;
    constexpr int WA = 32 * NCA;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v[kRowsPerWarp][NCA], d[kRowsPerWarp];
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp; ++rr) {
        const int tt = warp + kWinWarps * rr;
        d[rr] = F.one;
#pragma unroll
        for (int c = 0; c < NCW; ++c) {
            const int q = lane + 32 * c;
            v[rr][c] = (tt < h && q < W) ? F.to(A[(long long)tt * lda + q]) : 0u;
        }
#pragma unroll
        for (int c = NCW; c < NCA; ++c) v[rr][c] = (lane + 32 * (c - NCW) == tt) ? F.one : 0u;
    }
    if (warp == 0) win_publish<NCW, NCA>(v[0], 0, 0, d[0], S, WA);
    int k = 0;
    for (int t = 0; t < h; ++t) {
        if (t % kWinWarps != warp && !mbar_wait(&S.bar[t], 0u, S.abort_flag, timeout, 1)) return -1;
        const int j = S.jp[t];
        const int tn = t + 1;
        const bool own_next = tn < h && tn % kWinWarps == warp;
        const int rn = tn / kWinWarps;
        if (j >= 0) {  // same value in every thread
            const uint32_t P = S.Pv[t];
            uint32_t w[NCA];
#pragma unroll
            for (int c = 0; c < NCA; ++c) w[c] = F.neg(S.U[t * WA + lane + 32 * c]);
            // the next row first (published right away), then the others
#pragma unroll
            for (int rr = 0; rr < kRowsPerWarp; ++rr) {
                if (!(own_next && rr == rn)) continue;
                win_update<kBin, NCW, NCA>(F, v[rr], d[rr], w, j, P, S.Lsm + tn * h + k);
                win_publish<NCW, NCA>(v[rr], tn, k + 1, d[rr], S, WA);
            }
#pragma unroll
            for (int rr = 0; rr < kRowsPerWarp; ++rr) {
                const int tt = warp + kWinWarps * rr;
                if (tt <= tn || tt >= h) continue;  // warp-uniform
                win_update<kBin, NCW, NCA>(F, v[rr], d[rr], w, j, P, S.Lsm + tt * h + k);
            }
            ++k;
        } else if (own_next) {
#pragma unroll
            for (int rr = 0; rr < kRowsPerWarp; ++rr)
                if (rr == rn) win_publish<NCW, NCA>(v[rr], tn, k, d[rr], S, WA);
        }
    }
    return k;
}

// The leaf's outcome (rank, whether the window's columns keep their order, a
// wait that ran out) straight into the host's mapped mailbox, then the
// sequence number that tells the host the words are there (the host polls it
// instead of copying the record back and synchronising the stream).
__device__ __forceinline__ void post_outcome(int* mbox, int seq, int rank, int ident, int timeout) {
    volatile int* m = mbox;
    m[0] = rank;
    m[1] = ident;
    m[2] = timeout;
    __threadfence_system();
    m[3] = seq;
}

template <bool kBin>
__device__ __forceinline__ void window_body(uint32_t* A, long long lda, int h, int W, int WS,
                                            uint32_t p, unsigned long long mu, uint32_t two64p,
                                            uint32_t* __restrict__ Eg, const uint32_t* Uig, uint32_t* __restrict__ Usc,
                                            uint32_t* __restrict__ rows, long long ldr,
                                            LeafInfo* __restrict__ info, int* mbox, int seq) {
    extern __shared__ uint32_t sm[];
    const int WA = WS + kExt;
    uint32_t* U = sm;                          // [h][WA]
    uint32_t* Lsm = U + h * WA;                // [h][h]
    __shared__ uint64_t s_bar[kLeafRows];
    __shared__ uint32_t s_Pv[kLeafRows], s_dv[kLeafRows], s_P[kLeafRows], s_invP[kLeafRows];
    __shared__ int s_jp[kLeafRows], s_pre[kLeafRows], s_prow[kLeafRows], s_pcol[kLeafRows];
    __shared__ int s_rowpiv[kLeafRows], s_colpiv[kMaxWin];
    __shared__ int s_newrow[kLeafRows], s_newcol[kMaxWin];
    __shared__ int s_cnt[kWinWarps];
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const WinField<kBin> F(p, two64p, mu);

    for (int idx = tid; idx < h * h; idx += blockDim.x) Lsm[idx] = 0u;
    for (int x = tid; x < h; x += blockDim.x) {
        s_rowpiv[x] = -1;
        mbar_init(&s_bar[x], 32);
    }
    for (int x = tid; x < kMaxWin; x += blockDim.x) s_colpiv[x] = -1;
    if (tid == 0) {
        s_abort = 0;
        info->timeout = 0;
    }
    __syncthreads();

    const WinState S{U, Lsm, s_bar, s_jp, s_Pv, s_dv, s_pre, s_prow, s_pcol, s_P, s_colpiv, s_rowpiv, &s_abort};
    int r;
    if (kBin)
        r = win_eliminate<kBin, 8>(F, A, lda, h, W, S, &info->timeout);
    else
        r = WS <= 64   ? win_eliminate<kBin, 2>(F, A, lda, h, W, S, &info->timeout)
            : WS <= 96 ? win_eliminate<kBin, 3>(F, A, lda, h, W, S, &info->timeout)
                       : win_eliminate<kBin, 8>(F, A, lda, h, W, S, &info->timeout);
    __syncthreads();
    if (s_abort) {  // a wait ran out (info->timeout is set): nothing else is written
        if (tid == 0) {
            info->rank = 0;
            info->fail = 0;
            info->ident = 1;
            info->firstnz = INT_MAX;
            post_outcome(mbox, seq, 0, 1, 1);
        }
        return;
    }

    // 1 / P_k for every pivot: prefix and suffix products over warp 0 (two per lane), one inverse
    if (warp == 0) {
        const uint32_t v0 = 2 * lane < r ? s_P[2 * lane] : F.one;
        const uint32_t v1 = 2 * lane + 1 < r ? s_P[2 * lane + 1] : F.one;
        const uint32_t loc = F.mul(v0, v1);
        uint32_t inc = loc, sinc = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = F.mul(inc, x);
            const uint32_t y = __shfl_down_sync(0xffffffffu, sinc, o);
            if (lane + o < 32) sinc = F.mul(sinc, y);
        }
        uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
        uint32_t sexc = __shfl_down_sync(0xffffffffu, sinc, 1);
        if (lane == 0) exc = F.one;
        if (lane == 31) sexc = F.one;
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        uint32_t itot = lane == 0 ? F.inv(total) : 0u;
        itot = __shfl_sync(0xffffffffu, itot, 0);
        const uint32_t base = F.mul(F.mul(itot, exc), sexc);
        if (2 * lane < r) s_invP[2 * lane] = F.mul(base, v1);
        if (2 * lane + 1 < r) s_invP[2 * lane + 1] = F.mul(base, v0);
    }
    __syncthreads();
    // per row (one warp each): the true multipliers l_tk = a_tk c_k / (d_t
    // before step k), c_k = d_{prow k} / P_k = 1 / (true pivot k); 1 / d_t
    // before step k is the product of 1 / P_k' over the earlier steps that
    // touched row t (exclusive prefix products); then the stored row times
    // 1 / d_t: the true U row (pivot rows) and row t of E
    for (int t = warp; t < h; t += kWinWarps) {
        const int pre = s_pre[t];
        const uint32_t n0 = lane < pre ? Lsm[t * h + lane] : 0u;
        const uint32_t n1 = lane + 32 < pre ? Lsm[t * h + lane + 32] : 0u;
        const uint32_t f0 = n0 ? s_invP[lane] : F.one, f1 = n1 ? s_invP[lane + 32] : F.one;
        uint32_t i0 = f0, i1 = f1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x0 = __shfl_up_sync(0xffffffffu, i0, o);
            const uint32_t x1 = __shfl_up_sync(0xffffffffu, i1, o);
            if (lane >= o) {
                i0 = F.mul(i0, x0);
                i1 = F.mul(i1, x1);
            }
        }
        const uint32_t tot0 = __shfl_sync(0xffffffffu, i0, 31), tot1 = __shfl_sync(0xffffffffu, i1, 31);
        uint32_t e0 = __shfl_up_sync(0xffffffffu, i0, 1), e1 = __shfl_up_sync(0xffffffffu, i1, 1);
        if (lane == 0) e0 = e1 = F.one;
        e1 = F.mul(e1, tot0);
        if (n0) Lsm[t * h + lane] = F.mul(F.mul(n0, F.mul(s_dv[s_prow[lane]], s_invP[lane])), e0);
        if (n1) Lsm[t * h + lane + 32] = F.mul(F.mul(n1, F.mul(s_dv[s_prow[lane + 32]], s_invP[lane + 32])), e1);
        const uint32_t invd = F.mul(tot0, tot1);
        for (int q = lane; q < WA; q += 32) U[t * WA + q] = F.mul(U[t * WA + q], invd);
    }
    __syncthreads();
    // U11 (plain form, on and above the diagonal) and the diagonal of its
    // inverse, for the rest kernel's last CTA, which forms U11^{-1} by
    // doubling while the other CTAs compute the rest of the rows
    if (Uig) {
        for (int idx = tid; idx < r * r; idx += blockDim.x) {
            const int i = idx / r, q = idx - i * r;
            if (q >= i) Usc[i * kLeafRows + q] = F.from(U[s_prow[i] * WA + s_pcol[q]]);
        }
        for (int i = tid; i < r; i += blockDim.x)
            Usc[kLeafRows * kLeafRows + i] = F.from(F.mul(s_dv[s_prow[i]], s_invP[i]));
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
        post_outcome(mbox, seq, r, ident, 0);
    }
    for (int x = tid; x < h; x += blockDim.x) {
        info->newrow[x] = s_newrow[x];
        if (x < r) info->prow[x] = s_prow[x];
    }
    for (int x = tid; x < W; x += blockDim.x) info->newcol[x] = s_newcol[x];
    for (int idx = tid; idx < h * h; idx += blockDim.x) {
        const int t = idx / h, q = idx - t * h;
        Eg[idx] = F.from(U[t * WA + WS + q]);
    }
    // the leaf's new rows on the window: multipliers left of the diagonal of
    // the first r columns, the pivot rows' values on and right of it; in place
    // when every row is a pivot (the leaf then commits: no residual is left to
    // check), else to the scratch rows
    uint32_t* const dst = r == h ? A : rows;
    const long long ldd = r == h ? lda : ldr;
    for (int idx = tid; idx < h * W; idx += blockDim.x) {
        const int i = idx / W, q = idx - i * W;
        const int t = s_newrow[i];
        uint32_t v;
        if (q < min(i, r))
            v = F.from(Lsm[t * h + q]);
        else
            v = i < r ? F.from(U[t * WA + s_newcol[q]]) : 0u;
        dst[(long long)i * ldd + q] = v;
    }
}

__global__ void __launch_bounds__(kWinThreads, 1) lqup_window_kernel(uint32_t* A, long long lda,
                                                                  int h, int W, int WS, uint32_t p,
                                                                  unsigned long long mu, uint32_t two64p,
                                                                  uint32_t* __restrict__ Eg, const uint32_t* Uig,
                                                                  uint32_t* __restrict__ Usc, uint32_t* __restrict__ rows,
                                                                  long long ldr, LeafInfo* __restrict__ info,
                                                                  int* mbox, int seq) {
    if (p == 2u)
        window_body<true>(A, lda, h, W, WS, p, mu, two64p, Eg, Uig, Usc, rows, ldr, info, mbox, seq);
    else
        window_body<false>(A, lda, h, W, WS, p, mu, two64p, Eg, Uig, Usc, rows, ldr, info, mbox, seq);
}

// U11^{-1} (r x r, upper triangular, plain form) from U11 and the inverse of
// its diagonal in Usc (written by the window kernel), into Uig (leading
// dimension ldu, zeros below the diagonal), by one CTA.  Doubling:
// [[A, C], [0, D]]^{-1} has off-diagonal block -A^{-1} C D^{-1}; level s pairs
// the blocks [b0, b0 + s) and [b0 + s, b0 + 2 s), b0 = 2 s pr, each level two
// products over all pairs at once, on 64 x 64 zero-padded blocks so that every
// dot product has the level's full length and no bounds (b0 + 2 s <= 64 at
// every level).  sm holds 2 x 64 x 64 + kTmWords words.
__device__ void u11_inverse(int r, const uint32_t* __restrict__ Usc, uint32_t* __restrict__ Uig, long long ldu,
                            uint32_t p, unsigned long long mu, uint32_t two64p, uint32_t* sm) {
    uint32_t* Us = sm;                          // [64][64]: U11
    uint32_t* Ui = Us + kLeafRows * kLeafRows;  // [64][64]: U11^{-1}
    uint32_t* Tm = Ui + kLeafRows * kLeafRows;  // [kTmWords]: one level's products
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kLeafRows * kLeafRows; idx += blockDim.x) {
        const int i = idx / kLeafRows, q = idx % kLeafRows;
        const bool in = i < r && q < r;
        Us[idx] = in && q >= i ? __ldg(Usc + idx) : 0u;
        Ui[idx] = in && q == i ? __ldg(Usc + kLeafRows * kLeafRows + i) : 0u;
    }
    __syncthreads();
    for (int ls = 0; (1 << ls) < r; ++ls) {
        const int s = 1 << ls;
        const int np = (r - s + 2 * s - 1) / (2 * s);
        const int nout = np << (2 * ls);
        // Tm = C D^{-1} (s x s per pair)
        for (int idx = tid; idx < nout; idx += blockDim.x) {
            const int pr = idx >> (2 * ls), rem = idx & ((s << ls) - 1);
            const int i = rem >> ls, jj = rem & (s - 1);
            const int b0 = 2 * s * pr;
            const uint32_t* crow = Us + (b0 + i) * kLeafRows + b0 + s;
            const uint32_t* dcol = Ui + (b0 + s) * kLeafRows + b0 + s + jj;
            Acc128 acc;
#pragma unroll 8
            for (int l = 0; l < s; ++l) acc.add((unsigned long long)crow[l] * dcol[l * kLeafRows]);
            Tm[idx] = acc.mod(p, mu, two64p);
        }
        __syncthreads();
        // (U11^{-1})12 = -A^{-1} Tm
        for (int idx = tid; idx < nout; idx += blockDim.x) {
            const int pr = idx >> (2 * ls), rem = idx & ((s << ls) - 1);
            const int i = rem >> ls, jj = rem & (s - 1);
            const int b0 = 2 * s * pr;
            const uint32_t* arow = Ui + (b0 + i) * kLeafRows + b0;
            const uint32_t* tcol = Tm + (pr << (2 * ls)) + jj;
            Acc128 acc;
#pragma unroll 8
            for (int l = 0; l < s; ++l) acc.add((unsigned long long)arow[l] * tcol[l << ls]);
            const uint32_t v = acc.mod(p, mu, two64p);
            Ui[(b0 + i) * kLeafRows + b0 + s + jj] = v ? p - v : 0u;
        }
        __syncthreads();
    }
    for (int idx = tid; idx < r * r; idx += blockDim.x) {
        const int i = idx / r, q = idx - i * r;
        Uig[(long long)i * ldu + q] = Ui[i * kLeafRows + q];
    }
}

// The rest of the leaf's rows.  Blocks [0, nleft): columns [0, c), the rows
// only reordered.  Blocks from nleft on: kRestCols columns each from c + W
// on: new row i = E[newrow[i]] times the original columns, a 64 x 64 x h
// product per block (each thread 4 rows x 4 columns, exact 96-bit sums); the
// non-pivot rows' residuals must be zero, else the leaf fails and the
// smallest such column is recorded.  A points at (rb, 0).  Out of place
// (inplace = 0) the new rows go to the scratch rows (column 0 at rows, leading
// dimension ldr); in place (every row of the leaf a pivot, so the leaf
// commits) they overwrite A's rows (every block reads all its columns before
// it writes them) and block 0 also applies the row order to rowperm.  With
// dbl set, one more block (the last) forms U11^{-1} into Uig meanwhile.
__device__ __forceinline__ void mac96(uint32_t& lo, uint32_t& mid, uint32_t& hi, uint32_t a, uint32_t b) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"(a), "r"(b));
}

__global__ void __launch_bounds__(kThreads) lqup_rest_kernel(uint32_t* A, long long lda, int h, int c, int W, int n,
                                                             int nleft, uint32_t p, unsigned long long mu,
                                                             uint32_t two64p, const uint32_t* __restrict__ Eg,
                                                             uint32_t* rows, long long ldr, int inplace,
                                                             int32_t* rowperm, LeafInfo* __restrict__ info,
                                                             const uint32_t* __restrict__ Usc, uint32_t* Uig,
                                                             long long ldu, int dbl) {
    extern __shared__ uint32_t sm[];
    __shared__ int s_newrow[kLeafRows];
    __shared__ int32_t s_perm[kLeafRows];
    if (dbl && blockIdx.x == gridDim.x - 1) {
        u11_inverse(info->rank, Usc, Uig, ldu, p, mu, two64p, sm);
        return;
    }
    const int tid = threadIdx.x;
    const int r = info->rank;
    for (int x = tid; x < h; x += blockDim.x) s_newrow[x] = info->newrow[x];
    __syncthreads();
    uint32_t* out = inplace ? A : rows;
    const long long ldo = inplace ? lda : ldr;
    if (inplace && blockIdx.x == 0) {
        for (int x = tid; x < h; x += blockDim.x) s_perm[x] = rowperm[s_newrow[x]];
        __syncthreads();
        for (int x = tid; x < h; x += blockDim.x) rowperm[x] = s_perm[x];
    }
    if ((int)blockIdx.x < nleft) {
        // one column per thread, every row of it read before any is written
        const int col = blockIdx.x * blockDim.x + tid;
        if (col < c) {
            uint32_t v[kLeafRows];
#pragma unroll
            for (int e = 0; e < kLeafRows; ++e) v[e] = e < h ? A[(long long)s_newrow[e] * lda + col] : 0u;
#pragma unroll
            for (int e = 0; e < kLeafRows; ++e)
                if (e < h) out[(long long)e * ldo + col] = v[e];
        }
        return;
    }
    const int q0 = c + W + (blockIdx.x - nleft) * kRestCols;
    const int nq = min(kRestCols, n - q0);
    uint32_t* R = sm;                           // [kLeafRows][kRestCols]: the original columns
    uint32_t* Et = R + kLeafRows * kRestCols;   // [kLeafRows][kLeafRows]: Et[s][i] = E[newrow[i]][s]
    for (int idx = tid; idx < kLeafRows * kRestCols; idx += blockDim.x) {
        const int i = idx / kRestCols, q = idx % kRestCols;
        R[idx] = (i < h && q < nq) ? A[(long long)i * lda + q0 + q] : 0u;
    }
    for (int idx = tid; idx < kLeafRows * kLeafRows; idx += blockDim.x) {
        const int sr = idx / kLeafRows, i = idx % kLeafRows;
        Et[idx] = (sr < h && i < h) ? __ldg(Eg + s_newrow[i] * h + sr) : 0u;
    }
    __syncthreads();
    const int tx = tid % 16, ty = tid / 16;  // columns 4 tx .. 4 tx + 3, rows 4 ty .. 4 ty + 3
    uint32_t lo[4][4], mid[4][4], hi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) lo[i][j] = mid[i][j] = hi[i][j] = 0u;
#pragma unroll 4
    for (int sr = 0; sr < h; ++sr) {
        const uint4 ea = *reinterpret_cast<const uint4*>(Et + sr * kLeafRows + 4 * ty);
        const uint4 rb = *reinterpret_cast<const uint4*>(R + sr * kRestCols + 4 * tx);
        const uint32_t ev[4] = {ea.x, ea.y, ea.z, ea.w}, rv[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mac96(lo[i][j], mid[i][j], hi[i][j], ev[i], rv[j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = 4 * ty + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = 4 * tx + j;
            const uint32_t th = mod_u64((unsigned long long)mod_u64(hi[i][j], p, mu) * two64p, p, mu);
            const uint32_t tl = mod_u64(((unsigned long long)mid[i][j] << 32) | lo[i][j], p, mu);
            const uint32_t v = th + tl >= p ? th + tl - p : th + tl;
            if (row < h && q < nq) {
                if (row >= r && v != 0u) {
                    info->fail = 1;
                    atomicMin(&info->firstnz, q0 + q);
                }
                out[(long long)row * ldo + q0 + q] = row < r ? v : 0u;
            }
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

// Products of the recursion's smallest blocks (every dimension at most
// kTiny), one launch in place of a k-split product and its reduction kernel
// (two launches each on the pivot chain), spread over a few CTAs.  Stage 1
// forms T = P1 Q1 (m x n, inner dimension k1); with P2 given, stage 2 forms
// P2 T (m2 x n, inner dimension m).  The result times alpha goes to C.
// Without P2 the CTAs split the rows (CTA j: rows [j kTinyPart, ...)), so C
// may be P1 itself: each CTA reads and writes only its own rows.  With P2
// they split the columns (CTA j: columns [j kTinyPart, ...)), and C must not
// overlap the operands.  With zr > 0 the first CTA also sets the zr x zc
// block at Z to zero.  Each entry's products of residues are summed four at
// a time in 64 bits (4 (p - 1)^2 < 2^64) and folded into 96 bits before one
// reduction.
constexpr int kTiny = 64;
constexpr int kTinyPart = 8;
constexpr int kTinyThreads = 512;

__device__ __forceinline__ void tiny_add96(uint32_t& lo, uint32_t& mid, uint32_t& hi, unsigned long long v) {
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(lo), "+r"(mid), "+r"(hi)
        : "r"((uint32_t)v), "r"((uint32_t)(v >> 32)));
}

// out (m x n, row stride n) = A (m x k, row stride k) B (k x n, row stride n)
// mod p; out is none of A, B.
__device__ void tiny_mm(uint32_t* out, const uint32_t* A, const uint32_t* B, int m, int n, int k, uint32_t p,
                        unsigned long long mu, uint32_t two64p) {
    for (int o = threadIdx.x; o < m * n; o += blockDim.x) {
        const int r = o / n, c = o - r * n;
        const uint32_t* a = A + r * k;
        const uint32_t* b = B + c;
        uint32_t lo = 0u, mid = 0u, hi = 0u;
        int l = 0;
        for (; l + 4 <= k; l += 4) {
            unsigned long long acc = (unsigned long long)a[l] * b[l * n];
            acc += (unsigned long long)a[l + 1] * b[(l + 1) * n];
            acc += (unsigned long long)a[l + 2] * b[(l + 2) * n];
            acc += (unsigned long long)a[l + 3] * b[(l + 3) * n];
            tiny_add96(lo, mid, hi, acc);
        }
        unsigned long long acc = 0ull;
        for (; l < k; ++l) acc += (unsigned long long)a[l] * b[l * n];
        tiny_add96(lo, mid, hi, acc);
        const uint32_t th = mod_u64((unsigned long long)mod_u64(hi, p, mu) * two64p, p, mu);
        const uint32_t tl = mod_u64(((unsigned long long)mid << 32) | lo, p, mu);
        out[o] = th + tl >= p ? th + tl - p : th + tl;
    }
}

// rows x cols block of a row-major matrix (leading dimension ld) into shared
// memory (row stride cols), reduced mod p
__device__ __forceinline__ void tiny_load(uint32_t* dst, const uint32_t* src, long long ld, int rows, int cols,
                                          uint32_t p, unsigned long long mu) {
    for (int i = threadIdx.x; i < rows * cols; i += blockDim.x) {
        const int r = i / cols, c = i - r * cols;
        dst[i] = mod_u64(src[(long long)r * ld + c], p, mu);
    }
}

__global__ void __launch_bounds__(kTinyThreads) lqup_tiny_kernel(int m, int n, int k1, const uint32_t* P1,
                                                                 long long ld1, const uint32_t* Q1, long long ldq1,
                                                                 int m2, const uint32_t* P2, long long ld2,
                                                                 uint32_t alpha, uint32_t* C, long long ldc,
                                                                 uint32_t* Z, long long ldz, int zr, int zc,
                                                                 uint32_t p, unsigned long long mu, uint32_t two64p) {
    __shared__ uint32_t sA[kTiny * kTiny], sB[kTiny * kTiny], sT[kTiny * kTiny];
    const int part = blockIdx.x * kTinyPart;
    const uint32_t* R = sT;
    int rows, cols, r0 = 0, c0 = 0;
    if (P2 == nullptr) {  // rows [part, part + rows) of P1 Q1
        r0 = part;
        rows = min(kTinyPart, m - part);
        cols = n;
        tiny_load(sA, P1 + (long long)r0 * ld1, ld1, rows, k1, p, mu);
        tiny_load(sB, Q1, ldq1, k1, n, p, mu);
        __syncthreads();
        tiny_mm(sT, sA, sB, rows, n, k1, p, mu, two64p);
    } else {  // columns [part, part + cols) of P2 (P1 Q1)
        c0 = part;
        cols = min(kTinyPart, n - part);
        tiny_load(sA, P1, ld1, m, k1, p, mu);
        tiny_load(sB, Q1 + c0, ldq1, k1, cols, p, mu);
        __syncthreads();
        tiny_mm(sT, sA, sB, m, cols, k1, p, mu, two64p);
        __syncthreads();  // stage 1 has read sA and sB
        tiny_load(sA, P2, ld2, m2, m, p, mu);
        __syncthreads();
        tiny_mm(sB, sA, sT, m2, cols, m, p, mu, two64p);
        R = sB;
        rows = m2;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows * cols; i += blockDim.x) {
        const int r = i / cols, c = i - r * cols;
        C[(long long)(r0 + r) * ldc + c0 + c] = alpha == 1u ? R[i] : mod_u64((unsigned long long)R[i] * alpha, p, mu);
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < zr * zc; i += blockDim.x) {
            const int r = i / zc, c = i - r * zc;
            Z[(long long)r * ldz + c] = 0u;
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

// The window kernel's mailbox in mapped pinned memory (one per host thread):
// words rank, ident, timeout, then the sequence number of the leaf that wrote
// them; dev is the same memory as the kernel addresses it.
struct Mailbox {
    int* host = nullptr;
    int* dev = nullptr;
    int seq = 0;
};

Mailbox* mailbox() {
    thread_local Mailbox mb;
    if (!mb.host) {
        int* h = nullptr;
        if (cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) return nullptr;
        int* d = nullptr;
        if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaFreeHost(h);
            return nullptr;
        }
        std::memset(h, 0, 64);
        mb.host = h;
        mb.dev = d;
    }
    return &mb;
}

// Polls the mailbox for leaf seq.  Nothing else is queued on s behind the
// window kernel, so once the stream is idle the words must be there; the poll
// is also bounded in time.
ffgpu_status wait_outcome(const Mailbox& mb, int seq, cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned it = 1;; ++it) {
        if (__atomic_load_n(&mb.host[3], __ATOMIC_ACQUIRE) == seq) return FFGPU_OK;
        if ((it & 255u) == 0) {
            const cudaError_t e = cudaStreamQuery(s);
            if (e == cudaSuccess) return __atomic_load_n(&mb.host[3], __ATOMIC_ACQUIRE) == seq ? FFGPU_OK : FFGPU_ERR_CUDA;
            if (e != cudaErrorNotReady) return FFGPU_ERR_CUDA;
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) return FFGPU_ERR_TIMEOUT;
        }
    }
}

// Split of h rows: on a leaf boundary above the leaf size, in halves below it.
int64_t split_rows(int64_t h) {
    if (h <= kLeafRows) return h / 2;
    const int64_t nb = (h + kLeafRows - 1) / kLeafRows;
    return (nb / 2) * kLeafRows;
}

// Window width: wide enough for a leaf's pivots plus the columns that small
// fields skip (a zero Schur entry has probability 1/p: above 2^10 a 64-row
// leaf of uniform entries meets one with probability about 1/p < 10^-3, and
// then only splits, while 96 columns cost every leaf an eighth more time).
int window_for(uint32_t p) { return p > 1024 ? kLeafRows : p > 64 ? kLeafRows + 32 : kMaxWin; }

struct Layout {
    size_t rows, e, usp, t1, g, info, usc, words, rest;  // byte offsets; rest = products' workspace
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
    Y.usc = Y.info + align256(sizeof(LeafInfo));
    Y.words = Y.usc + align256((size_t(kLeafRows) * kLeafRows + kLeafRows) * 4);
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
    uint32_t* Usc;  // a leaf's U11 and the inverse of its diagonal, for the rest kernel's last block
    void* ws;
    size_t ws_bytes;
    int* err;
    cudaStream_t s;
    int win;
    int* host;
    Mailbox* mbox;
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

size_t smem_window(int h, int WS) {
    return (size_t(h) * (WS + kExt) + size_t(h) * h) * 4;
}
size_t smem_rest(int) {
    // the rows' blocks: R and Et; the U11 block: U11, its inverse, one level's products
    return std::max(size_t(kLeafRows) * kRestCols * 4 + size_t(kLeafRows) * kLeafRows * 4,
                    (2 * size_t(kLeafRows) * kLeafRows + size_t(kTmWords)) * 4);
}

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
    // the kernel's register layouts: 64, 96 or 256 window columns (p = 2: 256)
    const int WS = x.p == 2 ? kMaxWin : W <= 64 ? 64 : W <= 96 ? 96 : kMaxWin;
    uint32_t* Ab = x.A + rb * x.lda;
    const int seq = ++x.mbox->seq;
    ffgpu_status st = cuda_ok(timed_launch("lqup_window", x.s, [&] {
        lqup_window_kernel<<<1, kWinThreads, smem_window((int)h, WS), x.s>>>(
            Ab + c, x.lda, (int)h, W, WS, x.p, x.mu, x.two64p, x.E, Uo, x.Usc, x.rows + c, x.n, x.info,
            x.mbox->dev, seq);
        return cudaGetLastError();
    }));
    if (st != FFGPU_OK) return st;
    // The window's outcome first: with every row a pivot no residual can be
    // non-zero, so the rest of the leaf needs no second round trip.  (A
    // pending side-stream update runs meanwhile: the window kernel reads and
    // writes only this leaf's rows and the leaf's scratch.)
    if ((st = wait_outcome(*x.mbox, seq, x.s)) != FFGPU_OK) return st;
    if (x.mbox->host[2]) return FFGPU_ERR_TIMEOUT;
    const int r = x.mbox->host[0];
    const int ident0 = x.mbox->host[1];
    if ((st = join(x)) != FFGPU_OK) return st;
    const int nleft = (int)((c + kThreads - 1) / kThreads);
    const int nright = w > W ? (int)((w - W + kRestCols - 1) / kRestCols) : 0;
    // every row a pivot: the window kernel wrote its columns in place, the rest
    // follows in place (and applies the row order to rowperm)
    const bool inplace = r == h;
    // one more block forms the inverse of the pivot block when it is asked for
    const int dbl = Uo ? 1 : 0;
    if (nleft + nright + dbl > 0) {
        st = cuda_ok(timed_launch("lqup_rest", x.s, [&] {
            lqup_rest_kernel<<<nleft + nright + dbl, kThreads, smem_rest((int)h), x.s>>>(
                Ab, x.lda, (int)h, (int)c, W, (int)x.n, nleft, x.p, x.mu, x.two64p, x.E, x.rows, x.n, inplace ? 1 : 0,
                x.rowperm + rb, x.info, x.Usc, Uo, ldu, dbl);
            return cudaGetLastError();
        }));
        if (st != FFGPU_OK) return st;
    }
    int fail = 0, ident = ident0, firstnz = INT_MAX;
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
    if (!inplace &&
        (st = cuda_ok(cudaMemcpy2DAsync(Ab, x.lda * 4, x.rows, x.n * 4, x.n * 4, h, cudaMemcpyDeviceToDevice,
                                        x.s))) != FFGPU_OK)
        return st;
    if (!inplace || nleft + nright == 0) {
        st = cuda_ok(timed_launch("lqup_rowperm", x.s, [&] {
            lqup_rowperm_kernel<<<1, kThreads, 0, x.s>>>(x.rowperm + rb, (int)h, x.info);
            return cudaGetLastError();
        }));
        if (st != FFGPU_OK) return st;
    }
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
    // one-CTA products of blocks of at most kTiny (see lqup_tiny_kernel)
    auto tiny = [&](int m, int n, int k1, const uint32_t* P1, int64_t ld1, const uint32_t* Q1, int64_t ldq1, int m2,
                    const uint32_t* P2, int64_t ld2, uint32_t alpha, uint32_t* Cp, int64_t ldc, uint32_t* Zp,
                    int64_t ldz, int zr, int zc) -> ffgpu_status {
        return cuda_ok(timed_launch("lqup_tiny", x.s, [&] {
            const int parts = ((P2 ? n : m) + kTinyPart - 1) / kTinyPart;
            lqup_tiny_kernel<<<parts, kTinyThreads, 0, x.s>>>(m, n, k1, P1, ld1, Q1, ldq1, m2, P2, ld2, alpha, Cp, ldc,
                                                              Zp, ldz, zr, zc, x.p, x.mu, x.two64p);
            return cudaGetLastError();
        }));
    };
    if (r1 > 0) {
        uint32_t* top = x.A + rb * x.lda + c;
        uint32_t* bot = x.A + (rb + h1) * x.lda + c;
        // G = X U_a^{-1}, in place when the product reads all of X before it
        // writes (the tensor-core route converts its operands first; the
        // CUDA-core kernel does when one column tile covers G), else through
        // a scratch (a small product: h2 r1 <= 2^27 / r1 < kGWords)
        if (h2 <= kTiny && r1 <= kTiny) {
            if ((st = tiny((int)h2, (int)r1, (int)r1, bot, x.lda, Ua, lda_u, 0, nullptr, 0, 1, bot, x.lda, nullptr, 0,
                           0, 0)) != FFGPU_OK)
                return st;
        } else if (fgemm_small(h2, r1, r1) ? r1 <= 64 : fgemm_single_pass(x.p, r1)) {
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
    if (Uo && r1 > 0 && r2 > 0 && r1 <= kTiny && r2 <= kTiny) {
        // [[U_a^{-1}, -U_a^{-1} Y' U_b^{-1}], [0, U_b^{-1}]] in one launch
        const uint32_t* Yp = x.A + rb * x.lda + c + r1;
        if ((st = tiny((int)r1, (int)r2, (int)r2, Yp, x.lda, Ub, ldu, (int)r1, Uo, ldu, x.p - 1, Uo + r1, ldu,
                       Uo + r1 * ldu, ldu, (int)r2, (int)r1)) != FFGPU_OK)
            return st;
    } else if (Uo && r1 > 0 && r2 > 0) {
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
    x.Usc = reinterpret_cast<uint32_t*>(w + Y.usc);
    x.err = err;
    x.s = s;
    x.win = window_for(p);
    x.host = pinned_words();
    if (!x.host) return FFGPU_ERR_NOMEM;
    x.mbox = mailbox();
    if (!x.mbox) return FFGPU_ERR_NOMEM;
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
