// Strassen-Winograd levels over residues mod p (section 3.2) on top of any
// base path, and the ffgpu_fgemm_ex entry point.
//
// One level follows the schedule of Table 2 for C <- alpha*A*B + beta*C with
// three temporaries X1 (m/2 x k/2), X2 (k/2 x n/2), X3 (m/2 x n/2): the eight
// pre-additions S1..S4, T1..T4 and the post-additions are elementwise kernels
// mod p (so, unlike the paper's delayed version, intermediate values do not
// grow: Theorem 3.1's bound is not needed), the seven products recurse.
// On the residue-number-system path the last level's pre-additions are not
// written out at all: each product's operands are passed down as signed sums
// of quadrants (S4 = A12 - A21 - A22 + A11, ...), summed mod p inside the
// conversion that writes the product's channel planes, so that level costs its
// seven products' conversions and the post-additions only.  (Fusing two levels
// was measured slower: the deepest operands are sums of up to 16 blocks, each
// read by every product that uses it.)
// Row 16 is taken with A22 (P4 = alpha*A22*T4 - beta*C21), the reading under
// which the schedule computes A*B.  Odd dimensions are handled by dynamic
// peeling (appendix, "case of an arbitrary k"): the even top-left block by
// Winograd, then a rank-1 update for an odd k, and the last column / last row
// by the base path.
#include <algorithm>
#include <cstring>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

uint32_t dmma_max_p();
uint32_t sgemm_max_p();
cudaError_t launch_dmma_fgemm(int m, int n, int k, const uint32_t* A, long long lda, const uint32_t* B,
                              long long ldb, uint32_t* C, long long ldc, uint32_t p, uint32_t al, uint32_t be,
                              cudaStream_t s);
cudaError_t launch_sgemm_fgemm(int m, int n, int k, const uint32_t* A, long long lda, const uint32_t* B,
                               long long ldb, uint32_t* C, long long ldc, uint32_t p, uint32_t al, uint32_t be,
                               void* ws, cudaStream_t s);
size_t sgemm_ws_bytes(int64_t m, int64_t n, int64_t k);

namespace {

// Z = (X + c*Y) mod p elementwise (any uint32 words; Z may alias X or Y).
__global__ void __launch_bounds__(256) axpy_mod_kernel(int rows, int cols, const uint32_t* X, long long ldx,
                                                       const uint32_t* Y, long long ldy, uint32_t* Z,
                                                       long long ldz, uint32_t c, uint32_t p,
                                                       unsigned long long mu) {
    const long long total = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), q = (int)(i - (long long)r * cols);
        const unsigned long long x = X[(long long)r * ldx + q], y = Y[(long long)r * ldy + q];
        Z[(long long)r * ldz + q] = mod_u64(x + (unsigned long long)c * y, p, mu);
    }
}

struct WinoCtx {
    int path;
    uint32_t p;
    unsigned long long mu;
    void* fg_ws;
    size_t fg_ws_bytes;
    unsigned char* tmp;
    int* err;
    cudaStream_t s;
    int sms;
    bool dry;            // size the workspace only
    size_t need_fg;      // dry run: largest base-path workspace
    size_t need_tmp;     // dry run: temporaries
};

ffgpu_status axpy(WinoCtx& c, int64_t rows, int64_t cols, const uint32_t* X, int64_t ldx, const uint32_t* Y,
                  int64_t ldy, uint32_t* Z, int64_t ldz, uint32_t coef) {
    if (c.dry || rows == 0 || cols == 0) return FFGPU_OK;
    long long g = (rows * cols + 255) / 256;
    g = std::min<long long>(std::max<long long>(g, 1), 152 * 16);
    return timed_launch("winograd_axpy", c.s, [&] {
               axpy_mod_kernel<<<(int)g, 256, 0, c.s>>>((int)rows, (int)cols, X, ldx, Y, ldy, Z, ldz, coef, c.p,
                                                        c.mu);
               return cudaGetLastError();
           }) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

ffgpu_status base(WinoCtx& c, int64_t m, int64_t n, int64_t k, uint32_t al, const uint32_t* A, int64_t lda,
                  const uint32_t* B, int64_t ldb, uint32_t be, uint32_t* C, int64_t ldc) {
    if (m == 0 || n == 0) return FFGPU_OK;
    if (c.path == 0) {
        if (c.dry) {
            c.need_fg = std::max(c.need_fg, fgemm_ws_bytes(m, n, k, c.p, c.sms));
            return FFGPU_OK;
        }
        return fgemm_run(m, n, k, c.p, al, A, lda, B, ldb, be, C, ldc, c.fg_ws, c.fg_ws_bytes, c.err, c.s, 0,
                         false);
    }
    if (c.path == 3) {
        if (c.dry || k == 0) {
            if (!c.dry)
                return launch_scale(C, ldc, (int)m, (int)n, c.p, be, c.mu, c.s) == cudaSuccess ? FFGPU_OK
                                                                                              : FFGPU_ERR_CUDA;
            return FFGPU_OK;
        }
        if (m > int64_t(65535) * 64) return FFGPU_ERR_INVALID;
        return timed_launch("small_gemm", c.s, [&] {
                   return launch_small_gemm(m, n, k, A, lda, B, ldb, C, ldc, c.p, al, be, nullptr, 0, c.sms, c.s);
               }) == cudaSuccess
                   ? FFGPU_OK
                   : FFGPU_ERR_CUDA;
    }
    if (c.dry) {
        if (c.path == 2 && k > 0) c.need_fg = std::max(c.need_fg, sgemm_ws_bytes(m, n, k));
        return FFGPU_OK;
    }
    if (k == 0)
        return timed_launch("scale_mod_p", c.s, [&] { return launch_scale(C, ldc, (int)m, (int)n, c.p, be, c.mu, c.s); }) ==
                       cudaSuccess
                   ? FFGPU_OK
                   : FFGPU_ERR_CUDA;
    cudaError_t e;
    if (c.path == 1)
        e = timed_launch("dmma_fgemm", c.s, [&] {
            return launch_dmma_fgemm((int)m, (int)n, (int)k, A, lda, B, ldb, C, ldc, c.p, al, be, c.s);
        });
    else
        e = timed_launch("sgemm_fgemm", c.s, [&] {
            return launch_sgemm_fgemm((int)m, (int)n, (int)k, A, lda, B, ldb, C, ldc, c.p, al, be, c.fg_ws, c.s);
        });
    return e == cudaSuccess ? FFGPU_OK : FFGPU_ERR_CUDA;
}

#define FF_TRY(x)                             \
    do {                                      \
        const ffgpu_status st_ = (x);         \
        if (st_ != FFGPU_OK) return st_;      \
    } while (0)

SumSrc src_of(const uint32_t* X, int64_t ld);
ffgpu_status wino_src(WinoCtx& c, int level, int64_t m, int64_t n, int64_t k, uint32_t al, const SumSrc& A,
                      const SumSrc& B, uint32_t be, uint32_t* C, int64_t ldc, size_t tmp_off);

ffgpu_status wino(WinoCtx& c, int level, int64_t m, int64_t n, int64_t k, uint32_t al, const uint32_t* A,
                  int64_t lda, const uint32_t* B, int64_t ldb, uint32_t be, uint32_t* C, int64_t ldc,
                  size_t tmp_off) {
    if (level == 0 || m < 2 || n < 2 || k < 2) return base(c, m, n, k, al, A, lda, B, ldb, be, C, ldc);
    // the residue path's last level: pre-additions summed inside the conversions
    // (deeper sums would read up to 4^levels blocks per entry; the levels above
    // write their S and T out once)
    if (c.path == 0 && level == 1)
        return wino_src(c, 1, m, n, k, al, src_of(A, lda), src_of(B, ldb), be, C, ldc, tmp_off);
    const int64_t m2 = m & ~int64_t(1), n2 = n & ~int64_t(1), k2 = k & ~int64_t(1);
    if (m2 != m || n2 != n || k2 != k) {  // dynamic peeling
        FF_TRY(wino(c, level, m2, n2, k2, al, A, lda, B, ldb, be, C, ldc, tmp_off));
        if (k2 != k) FF_TRY(base(c, m2, n2, 1, al, A + k2, lda, B + k2 * ldb, ldb, 1, C, ldc));
        if (n2 != n) FF_TRY(base(c, m2, 1, k, al, A, lda, B + n2, ldb, be, C + n2, ldc));
        if (m2 != m) FF_TRY(base(c, 1, n, k, al, A + m2 * lda, lda, B, ldb, be, C + m2 * ldc, ldc));
        return FFGPU_OK;
    }
    const int64_t h = m / 2, kh = k / 2, w = n / 2;
    const uint32_t p = c.p, neg1 = p - 1;
    const uint32_t *A11 = A, *A12 = A + kh, *A21 = A + h * lda, *A22 = A + h * lda + kh;
    const uint32_t *B11 = B, *B12 = B + w, *B21 = B + kh * ldb, *B22 = B + kh * ldb + w;
    uint32_t *C11 = C, *C12 = C + w, *C21 = C + h * ldc, *C22 = C + h * ldc + w;
    // temporaries of this level, then the next level's
    const size_t b1 = size_t(h) * kh * 4, b2 = size_t(kh) * w * 4, b3 = size_t(h) * w * 4;
    const size_t o1 = tmp_off, o2 = o1 + ((b1 + 255) & ~size_t(255)), o3 = o2 + ((b2 + 255) & ~size_t(255));
    const size_t next = o3 + ((b3 + 255) & ~size_t(255));
    if (c.dry) c.need_tmp = std::max(c.need_tmp, next);
    uint32_t* X1 = c.dry ? nullptr : reinterpret_cast<uint32_t*>(c.tmp + o1);
    uint32_t* X2 = c.dry ? nullptr : reinterpret_cast<uint32_t*>(c.tmp + o2);
    uint32_t* X3 = c.dry ? nullptr : reinterpret_cast<uint32_t*>(c.tmp + o3);
    const int L = level - 1;
    FF_TRY(axpy(c, h, kh, A21, lda, A22, lda, X1, kh, 1));                    // 1  S1 = A21 + A22
    FF_TRY(axpy(c, kh, w, B12, ldb, B11, ldb, X2, w, neg1));                  // 2  T1 = B12 - B11
    FF_TRY(wino(c, L, h, w, kh, al, X1, kh, X2, w, 0, X3, w, next));          // 3  P5 = a S1 T1
    FF_TRY(axpy(c, h, w, X3, w, C22, ldc, C22, ldc, be));                     // 4  C22 = P5 + b C22
    FF_TRY(axpy(c, h, w, X3, w, C12, ldc, C12, ldc, be));                     // 5  C12 = P5 + b C12
    FF_TRY(axpy(c, h, kh, X1, kh, A11, lda, X1, kh, neg1));                   // 6  S2 = S1 - A11
    FF_TRY(axpy(c, kh, w, B22, ldb, X2, w, X2, w, neg1));                     // 7  T2 = B22 - T1
    FF_TRY(wino(c, L, h, w, kh, al, A11, lda, B11, ldb, 0, X3, w, next));     // 8  P1 = a A11 B11
    FF_TRY(axpy(c, h, w, X3, w, C11, ldc, C11, ldc, be));                     // 9  C11 = P1 + b C11
    FF_TRY(wino(c, L, h, w, kh, al, X1, kh, X2, w, 1, X3, w, next));          // 10 U2 = a S2 T2 + P1
    FF_TRY(wino(c, L, h, w, kh, al, A12, lda, B21, ldb, 1, C11, ldc, next));  // 11 U1 = a A12 B21 + C11
    FF_TRY(axpy(c, h, kh, A12, lda, X1, kh, X1, kh, neg1));                   // 12 S4 = A12 - S2
    FF_TRY(axpy(c, kh, w, X2, w, B21, ldb, X2, w, neg1));                     // 13 T4 = T2 - B21
    FF_TRY(wino(c, L, h, w, kh, al, X1, kh, B22, ldb, 1, C12, ldc, next));    // 14 C12 = a S4 B22 + C12
    FF_TRY(axpy(c, h, w, X3, w, C12, ldc, C12, ldc, 1));                      // 15 U5 = U2 + C12
    FF_TRY(wino(c, L, h, w, kh, al, A22, lda, X2, w, (p - be) % p, C21, ldc, next));  // 16 P4 = a A22 T4 - b C21
    FF_TRY(axpy(c, h, kh, A11, lda, A21, lda, X1, kh, neg1));                 // 17 S3 = A11 - A21
    FF_TRY(axpy(c, kh, w, B22, ldb, B12, ldb, X2, w, neg1));                  // 18 T3 = B22 - B12
    FF_TRY(wino(c, L, h, w, kh, al, X1, kh, X2, w, 1, X3, w, next));          // 19 U3 = a S3 T3 + U2
    FF_TRY(axpy(c, h, w, X3, w, C22, ldc, C22, ldc, 1));                      // 20 U7 = U3 + C22
    FF_TRY(axpy(c, h, w, X3, w, C21, ldc, C21, ldc, neg1));                   // 21 U6 = U3 - C21
    return FFGPU_OK;
}

// ---------------------------------------------------------------------------
// The residue-number-system path with fused pre-additions.
// ---------------------------------------------------------------------------

SumSrc src_of(const uint32_t* X, int64_t ld) {
    SumSrc S;
    std::memset(&S, 0, sizeof(S));
    S.X[0] = X;
    S.ld[0] = ld;
    S.n = 1;
    return S;
}

// Block (r, c) of every term.
SumSrc sub(const SumSrc& S, int64_t r, int64_t c) {
    SumSrc T = S;
    for (int t = 0; t < S.n; ++t) T.X[t] = S.X[t] + r * S.ld[t] + c;
    return T;
}

// a + b or a - b (term lists concatenated; at most kMaxTerms terms).
SumSrc combine(const SumSrc& a, const SumSrc& b, bool minus) {
    SumSrc r = a;
    for (int t = 0; t < b.n; ++t) {
        r.X[r.n] = b.X[t];
        r.ld[r.n] = b.ld[t];
        r.neg[r.n] = minus ? 1u - b.neg[t] : b.neg[t];
        ++r.n;
    }
    return r;
}

// One product of the level's leaves: a single-term pair is an ordinary
// fgemm (any route); sums go through the tensor-core route's summing
// conversions, or, for a product small enough for the CUDA cores, are first
// written out into the temporaries at tmp_off.
ffgpu_status base_src(WinoCtx& c, int64_t m, int64_t n, int64_t k, uint32_t al, const SumSrc& A, const SumSrc& B,
                      uint32_t be, uint32_t* C, int64_t ldc, size_t tmp_off) {
    if (m == 0 || n == 0) return FFGPU_OK;
    if (A.n == 1 && B.n == 1) return base(c, m, n, k, al, A.X[0], A.ld[0], B.X[0], B.ld[0], be, C, ldc);
    if (k > 0 && !fgemm_small(m, n, k)) {
        if (c.dry) {
            c.need_fg = std::max(c.need_fg, fgemm_ws_bytes(m, n, k, c.p, c.sms));
            return FFGPU_OK;
        }
        return fgemm_run_rns_src(m, n, k, c.p, al, A, B, be, C, ldc, c.fg_ws, c.fg_ws_bytes, c.err, c.s, 0, false);
    }
    const size_t ba = (size_t(m) * k * 4 + 255) & ~size_t(255), bb = (size_t(k) * n * 4 + 255) & ~size_t(255);
    if (c.dry) {
        c.need_tmp = std::max(c.need_tmp, tmp_off + ba + bb);
        return base(c, m, n, k, al, nullptr, k, nullptr, n, be, C, ldc);
    }
    uint32_t* Ta = reinterpret_cast<uint32_t*>(c.tmp + tmp_off);
    uint32_t* Tb = reinterpret_cast<uint32_t*>(c.tmp + tmp_off + ba);
    const uint32_t* a = A.X[0];
    int64_t lda = A.ld[0];
    const uint32_t* b = B.X[0];
    int64_t ldb = B.ld[0];
    if (A.n > 1) {
        if (timed_launch("winograd_sum", c.s, [&] { return launch_sum_mod(A, (int)m, (int)k, c.p, Ta, k, c.s); }) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
        a = Ta;
        lda = k;
    }
    if (B.n > 1) {
        if (timed_launch("winograd_sum", c.s, [&] { return launch_sum_mod(B, (int)k, (int)n, c.p, Tb, n, c.s); }) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
        b = Tb;
        ldb = n;
    }
    return base(c, m, n, k, al, a, lda, b, ldb, be, C, ldc);
}

// Table 2's schedule with the operands as sums (rows 1-2, 6-7, 12-13, 17-18
// are term lists, no kernel); the products and post-additions as in wino.
ffgpu_status wino_src(WinoCtx& c, int level, int64_t m, int64_t n, int64_t k, uint32_t al, const SumSrc& A,
                      const SumSrc& B, uint32_t be, uint32_t* C, int64_t ldc, size_t tmp_off) {
    if (level == 0 || m < 2 || n < 2 || k < 2) return base_src(c, m, n, k, al, A, B, be, C, ldc, tmp_off);
    const int64_t m2 = m & ~int64_t(1), n2 = n & ~int64_t(1), k2 = k & ~int64_t(1);
    if (m2 != m || n2 != n || k2 != k) {  // dynamic peeling
        FF_TRY(wino_src(c, level, m2, n2, k2, al, A, B, be, C, ldc, tmp_off));
        if (k2 != k) FF_TRY(base_src(c, m2, n2, 1, al, sub(A, 0, k2), sub(B, k2, 0), 1, C, ldc, tmp_off));
        if (n2 != n) FF_TRY(base_src(c, m2, 1, k, al, A, sub(B, 0, n2), be, C + n2, ldc, tmp_off));
        if (m2 != m) FF_TRY(base_src(c, 1, n, k, al, sub(A, m2, 0), B, be, C + m2 * ldc, ldc, tmp_off));
        return FFGPU_OK;
    }
    const int64_t h = m / 2, kh = k / 2, w = n / 2;
    const uint32_t p = c.p, neg1 = p - 1;
    const SumSrc A11 = sub(A, 0, 0), A12 = sub(A, 0, kh), A21 = sub(A, h, 0), A22 = sub(A, h, kh);
    const SumSrc B11 = sub(B, 0, 0), B12 = sub(B, 0, w), B21 = sub(B, kh, 0), B22 = sub(B, kh, w);
    uint32_t *C11 = C, *C12 = C + w, *C21 = C + h * ldc, *C22 = C + h * ldc + w;
    const SumSrc S1 = combine(A21, A22, false), T1 = combine(B12, B11, true);   // rows 1-2
    const SumSrc S2 = combine(S1, A11, true), T2 = combine(B22, T1, true);      // rows 6-7
    const SumSrc S4 = combine(A12, S2, true), T4 = combine(T2, B21, true);      // rows 12-13
    const SumSrc S3 = combine(A11, A21, true), T3 = combine(B22, B12, true);    // rows 17-18
    const size_t b3 = size_t(h) * w * 4;
    const size_t o3 = tmp_off, next = o3 + ((b3 + 255) & ~size_t(255));
    if (c.dry) c.need_tmp = std::max(c.need_tmp, next);
    uint32_t* X3 = c.dry ? nullptr : reinterpret_cast<uint32_t*>(c.tmp + o3);
    const int L = level - 1;
    FF_TRY(wino_src(c, L, h, w, kh, al, S1, T1, 0, X3, w, next));              // 3  P5 = a S1 T1
    FF_TRY(axpy(c, h, w, X3, w, C22, ldc, C22, ldc, be));                     // 4  C22 = P5 + b C22
    FF_TRY(axpy(c, h, w, X3, w, C12, ldc, C12, ldc, be));                     // 5  C12 = P5 + b C12
    FF_TRY(wino_src(c, L, h, w, kh, al, A11, B11, 0, X3, w, next));            // 8  P1 = a A11 B11
    FF_TRY(axpy(c, h, w, X3, w, C11, ldc, C11, ldc, be));                     // 9  C11 = P1 + b C11
    FF_TRY(wino_src(c, L, h, w, kh, al, S2, T2, 1, X3, w, next));              // 10 U2 = a S2 T2 + P1
    FF_TRY(wino_src(c, L, h, w, kh, al, A12, B21, 1, C11, ldc, next));         // 11 U1 = a A12 B21 + C11
    FF_TRY(wino_src(c, L, h, w, kh, al, S4, B22, 1, C12, ldc, next));          // 14 C12 = a S4 B22 + C12
    FF_TRY(axpy(c, h, w, X3, w, C12, ldc, C12, ldc, 1));                      // 15 U5 = U2 + C12
    FF_TRY(wino_src(c, L, h, w, kh, al, A22, T4, (p - be) % p, C21, ldc, next));  // 16 P4 = a A22 T4 - b C21
    FF_TRY(wino_src(c, L, h, w, kh, al, S3, T3, 1, X3, w, next));              // 19 U3 = a S3 T3 + U2
    FF_TRY(axpy(c, h, w, X3, w, C22, ldc, C22, ldc, 1));                      // 20 U7 = U3 + C22
    FF_TRY(axpy(c, h, w, X3, w, C21, ldc, C21, ldc, neg1));                   // 21 U6 = U3 - C21
    return FFGPU_OK;
}

}  // namespace

ffgpu_status fgemm_ex_run(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const uint32_t* A,
                          int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta, uint32_t* C, int64_t ldc,
                          int path, int levels, cudaStream_t s) {
    if (path < 0 || path > 3 || levels < 0 || levels > 8) return FFGPU_ERR_INVALID;
    if (path == 1 && p > dmma_max_p()) return FFGPU_ERR_UNSUPPORTED_P;
    if (path == 2 && p > sgemm_max_p()) return FFGPU_ERR_UNSUPPORTED_P;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    WinoCtx c;
    c.path = path;
    c.p = p;
    c.mu = ~0ull / p;
    c.fg_ws = nullptr;
    c.fg_ws_bytes = 0;
    c.tmp = nullptr;
    c.err = nullptr;
    c.s = s;
    c.sms = sm_count(dev);
    c.dry = true;
    c.need_fg = 0;
    c.need_tmp = 0;
    const uint32_t al = alpha % p, be = beta % p;
    auto run = [&]() { return wino(c, levels, m, n, k, al, A, lda, B, ldb, be, C, ldc, 0); };
    FF_TRY(run());
    const size_t fg = (c.need_fg + 255) & ~size_t(255);
    Pool* pool = nullptr;
    FF_TRY(pool_get(s, fg + c.need_tmp, &pool));
    c.dry = false;
    c.fg_ws = pool->ptr;
    c.fg_ws_bytes = fg;
    c.tmp = static_cast<unsigned char*>(pool->ptr) + fg;
    c.err = pool->err;
    return run();
}

}  // namespace ffgpu
