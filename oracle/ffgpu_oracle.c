/*
 * CPU oracle for fgemm / ftrsm / LQUP (rank, determinant, inverse) over Z/pZ.
 * TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously correct definition of what the GPU
 * path computes.  It is called by tests/, by __graft_entry__.smoke() and by the
 * CPU-baseline leg of bench.py, and by nothing else.  It shares no code, header,
 * table or constant with the CUDA library and includes none of it.
 *
 * Arithmetic: every input is first reduced mod p (the paper embeds Z/pZ into Z
 * and maps back by reduction mod p, section 2.1.2); products of residues
 * (< 2^62) are summed exactly in unsigned 128-bit integers and reduced once per
 * output entry.  Outputs are canonical representatives in [0, p).
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define OR_OK 0
#define OR_INVALID (-1)
#define OR_NOMEM (-3)

/* (a*b + c*d) mod p for residues a,b,c,d < p < 2^32, exact. */
static uint64_t addmul2(uint64_t a, uint64_t b, uint64_t c, uint64_t d, uint64_t p)
{
    u128 s = (u128)a * b + (u128)c * d;
    return (uint64_t)(s % p);
}

/*
 * fgemm definition (section 3, the problem statement C <- alpha*A*B + beta*C
 * over Z/pZ; ring homomorphism Z -> Z/pZ of section 2.1.2):
 *   C[i][j] = (alpha * sum_t A[i][t]*B[t][j] + beta * C[i][j]) mod p,
 * all operands reduced mod p first.  Row-major with leading dimensions.
 * i-t-j loop order, one exact 128-bit accumulator per output entry of row i.
 */
int oracle_fgemm(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                 const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                 uint32_t beta, uint32_t* C, int64_t ldc)
{
    if (p < 2 || m < 0 || n < 0 || k < 0) return OR_INVALID;
    if (m == 0 || n == 0) return OR_OK;
    if ((k > 0 && (lda < k || ldb < n)) || ldc < n) return OR_INVALID;
    const uint64_t P = p, al = alpha % p, be = beta % p;
    int status = OR_OK;
#pragma omp parallel
    {
        u128* acc = (u128*)malloc(sizeof(u128) * (size_t)n);
        if (!acc) {
#pragma omp atomic write
            status = OR_NOMEM;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < m; i++) {
            if (!acc) continue;
            memset(acc, 0, sizeof(u128) * (size_t)n);
            for (int64_t t = 0; t < k; t++) {
                const uint64_t a = A[i * lda + t] % P;
                if (a == 0) continue;
                const uint32_t* brow = B + t * ldb;
                for (int64_t j = 0; j < n; j++) acc[j] += (u128)(a * (uint64_t)(brow[j] % P));
            }
            uint32_t* crow = C + i * ldc;
            for (int64_t j = 0; j < n; j++) {
                const uint64_t s = (uint64_t)(acc[j] % P);
                crow[j] = (uint32_t)addmul2(al, s, be, crow[j] % P, P);
            }
        }
        free(acc);
    }
    return status;
}

/*
 * Selected entries of the same definition: out[e] = C_new[rows[e]][cols[e]]
 * where C_new is what oracle_fgemm would write.  C is only read.  Used to
 * check the full-size GPU runs entry by entry without the cubic cost.
 */
int oracle_fgemm_entries(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                         const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                         uint32_t beta, const uint32_t* C, int64_t ldc,
                         int64_t count, const int64_t* rows, const int64_t* cols,
                         uint32_t* out)
{
    if (p < 2 || count < 0) return OR_INVALID;
    const uint64_t P = p, al = alpha % p, be = beta % p;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; e++) {
        const int64_t i = rows[e], j = cols[e];
        if (i < 0 || i >= m || j < 0 || j >= n) { out[e] = 0xFFFFFFFFu; continue; }
        u128 acc = 0;
        for (int64_t t = 0; t < k; t++)
            acc += (u128)((uint64_t)(A[i * lda + t] % P) * (uint64_t)(B[t * ldb + j] % P));
        out[e] = (uint32_t)addmul2(al, (uint64_t)(acc % P), be, C[i * ldc + j] % P, P);
    }
    return OR_OK;
}

/* y = M x mod p, M of size rows x cols (ld), exact.  Used for Freivalds checks. */
int oracle_matvec(int64_t rows, int64_t cols, uint32_t p, const uint32_t* M, int64_t ld,
                  const uint32_t* x, uint32_t* y)
{
    if (p < 2 || rows < 0 || cols < 0) return OR_INVALID;
    const uint64_t P = p;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; i++) {
        u128 acc = 0;
        const uint32_t* r = M + i * ld;
        for (int64_t j = 0; j < cols; j++) acc += (u128)((uint64_t)(r[j] % P) * (uint64_t)(x[j] % P));
        y[i] = (uint32_t)(acc % P);
    }
    return OR_OK;
}

/* Modular inverse by the extended Euclidean algorithm (the classical
 * representation's division, section 2.1.1).  Returns 0 if a is not
 * invertible mod p. */
static uint64_t inv_mod(uint64_t a, uint64_t p)
{
    int64_t r0 = (int64_t)p, r1 = (int64_t)(a % p), s0 = 0, s1 = 1;
    while (r1 != 0) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    if (r0 != 1) return 0;
    if (s0 < 0) s0 += (int64_t)p;
    return (uint64_t)s0;
}

/*
 * ftrsm definition (section 4: solve a triangular system with a matrix
 * right-hand side; X = A^{-1} B for the left side, the transposed statement
 * for the right side).  B is overwritten by X:
 *   side 0 (Left):  op(T) X = alpha B, T is m x m
 *   side 1 (Right): X op(T) = alpha B, T is n x n
 *   uplo 0 = Lower, 1 = Upper;  diag 0 = NonUnit, 1 = Unit (diagonal taken as 1).
 * Plain substitution mod p, one 128-bit accumulator per unknown.  Returns
 * OR_INVALID if a diagonal entry is not invertible mod p (NonUnit).
 */
int oracle_ftrsm(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p,
                 uint32_t alpha, const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb)
{
    if (p < 2 || m < 0 || n < 0 || side < 0 || side > 1 || uplo < 0 || uplo > 1 ||
        diag < 0 || diag > 1)
        return OR_INVALID;
    if (m == 0 || n == 0) return OR_OK;
    const int64_t nt = side == 0 ? m : n;
    if (ldt < nt || ldb < n) return OR_INVALID;
    const uint64_t P = p, al = alpha % p;
    uint64_t* dinv = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nt);
    if (!dinv) return OR_NOMEM;
    for (int64_t i = 0; i < nt; i++) {
        dinv[i] = diag ? 1 : inv_mod(T[i * ldt + i] % P, P);
        if (dinv[i] == 0) { free(dinv); return OR_INVALID; }
    }
    if (side == 0) {
        /* Each column j of B is an independent system T x = alpha b. */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) {
            for (int64_t s = 0; s < m; s++) {
                const int64_t i = uplo == 0 ? s : m - 1 - s; /* forward / back substitution */
                u128 acc = 0;
                const int64_t lo = uplo == 0 ? 0 : i + 1, hi = uplo == 0 ? i : m;
                for (int64_t l = lo; l < hi; l++)
                    acc += (u128)((uint64_t)(T[i * ldt + l] % P) * (uint64_t)B[l * ldb + j]);
                const uint64_t rhs = (uint64_t)(((u128)al * (B[i * ldb + j] % P)) % P);
                const uint64_t sum = (uint64_t)(acc % P);
                const uint64_t v = (rhs + P - sum) % P;
                B[i * ldb + j] = (uint32_t)((v * dinv[i]) % P);
            }
        }
    } else {
        /* Each row i of B is an independent system x T = alpha b, i.e. T^t x^t = alpha b^t. */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; i++) {
            uint32_t* row = B + i * ldb;
            for (int64_t s = 0; s < n; s++) {
                /* x T = b: column j of T gives x_j T_jj = b_j - sum_{l != j} x_l T_lj,
                   with l < j for Upper (solve left to right), l > j for Lower. */
                const int64_t j = uplo == 1 ? s : n - 1 - s;
                u128 acc = 0;
                const int64_t lo = uplo == 1 ? 0 : j + 1, hi = uplo == 1 ? j : n;
                for (int64_t l = lo; l < hi; l++)
                    acc += (u128)((uint64_t)row[l] * (uint64_t)(T[l * ldt + j] % P));
                const uint64_t rhs = (uint64_t)(((u128)al * (row[j] % P)) % P);
                const uint64_t sum = (uint64_t)(acc % P);
                const uint64_t v = (rhs + P - sum) % P;
                row[j] = (uint32_t)((v * dinv[j]) % P);
            }
        }
    }
    free(dinv);
    return OR_OK;
}

/*
 * LQUP (section 5: A = L Q U P with L lower triangular, P and Q permutations
 * and U upper triangular of rank r whose first r rows are non-zero; section 6:
 * rank, determinant and inverse derived from it), in packed form.
 *
 * Elimination row by row, top to bottom (the order in which the block
 * recursion of section 5 meets the rows).  When row i is reached it holds its
 * Schur complement s_i (every earlier pivot row has been subtracted from it).
 * If s_i is zero, row i is not a pivot row.  Otherwise it becomes pivot number
 * k with pivot column j = the smallest original column index with
 * s_i[j] != 0; U_k = s_i; every later row t gets the multiplier
 * l_tk = s_t[j] / s_i[j] and loses l_tk U_k.  The paper leaves the pivot
 * choice to the implementation; this rule (first non-zero in original column
 * order) makes the factorization unique, so a fast implementation that follows
 * it must produce exactly this output.
 *
 * Output (p prime, every input first reduced mod p):
 *   rowperm[0..m): the pivot rows in order, then the other rows ascending;
 *   colperm[0..n): the pivot columns in pivot order, then the other columns
 *                  ascending;
 *   A overwritten by M with M[a][b] = L[a][b] for b < min(a, r) and
 *   U[a][b] otherwise (zero for a >= r), where A[rowperm][:, colperm] = L U,
 *   L m x r unit lower trapezoidal (its unit diagonal is not stored), U r x n
 *   upper trapezoidal with non-zero diagonal.
 * Returns the rank r, or a negative OR_* code.
 */
int64_t oracle_lqup(int64_t m, int64_t n, uint32_t p, uint32_t* A, int64_t lda,
                    int32_t* rowperm, int32_t* colperm)
{
    if (p < 2 || m < 0 || n < 0 || (m > 0 && lda < n)) return OR_INVALID;
    const uint64_t P = p;
    const int64_t mn = m < n ? m : n;
    uint32_t* W = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m * n + 1));
    uint32_t* Lm = (uint32_t*)calloc((size_t)(m * mn + 1), sizeof(uint32_t));
    int64_t* prow = (int64_t*)malloc(sizeof(int64_t) * (size_t)(mn + 1));
    int64_t* pcol = (int64_t*)malloc(sizeof(int64_t) * (size_t)(mn + 1));
    char* used = (char*)calloc((size_t)(m + n + 1), 1);
    if (!W || !Lm || !prow || !pcol || !used) {
        free(W); free(Lm); free(prow); free(pcol); free(used);
        return OR_NOMEM;
    }
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) W[i * n + j] = (uint32_t)(A[i * lda + j] % P);
    int64_t r = 0;
    for (int64_t i = 0; i < m && r < mn; i++) {
        const uint32_t* wi = W + i * n;
        int64_t j = 0;
        while (j < n && wi[j] == 0) j++;
        if (j == n) continue;                    /* zero Schur complement: not a pivot row */
        const uint64_t inv = inv_mod(wi[j], P);
        if (inv == 0) { r = OR_INVALID; break; } /* p not prime */
        prow[r] = i;
        pcol[r] = j;
#pragma omp parallel for schedule(static)
        for (int64_t t = i + 1; t < m; t++) {
            uint32_t* wt = W + t * n;
            if (wt[j] == 0) continue;
            const uint64_t l = ((uint64_t)wt[j] * inv) % P;
            Lm[t * mn + r] = (uint32_t)l;
            const uint64_t nl = P - l;
            for (int64_t q = 0; q < n; q++) wt[q] = (uint32_t)(((uint64_t)wt[q] + nl * wi[q]) % P);
        }
        r++;
    }
    if (r >= 0) {
        int64_t a = 0;
        for (int64_t k = 0; k < r; k++) { rowperm[a++] = (int32_t)prow[k]; used[prow[k]] = 1; }
        for (int64_t i = 0; i < m; i++) if (!used[i]) rowperm[a++] = (int32_t)i;
        int64_t b = 0;
        for (int64_t k = 0; k < r; k++) { colperm[b++] = (int32_t)pcol[k]; used[m + pcol[k]] = 1; }
        for (int64_t j = 0; j < n; j++) if (!used[m + j]) colperm[b++] = (int32_t)j;
        for (int64_t a2 = 0; a2 < m; a2++) {
            const int64_t t = rowperm[a2];
            for (int64_t b2 = 0; b2 < n; b2++) {
                uint32_t v;
                if (b2 < (a2 < r ? a2 : r)) v = Lm[t * mn + b2];
                else v = a2 < r ? W[t * n + colperm[b2]] : 0u;
                A[a2 * lda + b2] = v;
            }
        }
    }
    free(W); free(Lm); free(prow); free(pcol); free(used);
    return r;
}

/*
 * Rank by the textbook column-by-column reduction to row echelon form (an
 * algorithm other than the one above): for each column, take the first
 * remaining row with a non-zero entry as the pivot, swap it up, clear the
 * column below it.  p prime.  Returns the rank, or a negative OR_* code.
 */
int64_t oracle_rank(int64_t m, int64_t n, uint32_t p, const uint32_t* A, int64_t lda)
{
    if (p < 2 || m < 0 || n < 0 || (m > 0 && lda < n)) return OR_INVALID;
    const uint64_t P = p;
    uint32_t* W = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m * n + 1));
    if (!W) return OR_NOMEM;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) W[i * n + j] = (uint32_t)(A[i * lda + j] % P);
    int64_t row = 0;
    for (int64_t col = 0; col < n && row < m; col++) {
        int64_t piv = row;
        while (piv < m && W[piv * n + col] == 0) piv++;
        if (piv == m) continue;
        if (piv != row)
            for (int64_t q = 0; q < n; q++) {
                const uint32_t x = W[row * n + q];
                W[row * n + q] = W[piv * n + q];
                W[piv * n + q] = x;
            }
        const uint64_t inv = inv_mod(W[row * n + col], P);
        if (inv == 0) { free(W); return OR_INVALID; }
#pragma omp parallel for schedule(static)
        for (int64_t t = row + 1; t < m; t++) {
            const uint64_t f = ((uint64_t)W[t * n + col] * inv) % P;
            if (f == 0) continue;
            for (int64_t q = col; q < n; q++)
                W[t * n + q] = (uint32_t)(((uint64_t)W[t * n + q] + (P - f) * W[row * n + q]) % P);
        }
        row++;
    }
    free(W);
    return row;
}

/*
 * Determinant by textbook Gaussian elimination with row swaps (each swap
 * negates it; section 6 defines the determinant through LQUP as the product of
 * U's diagonal, this is the independent classical route).  p prime.
 */
int oracle_det(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* det)
{
    if (p < 2 || n < 0 || (n > 0 && lda < n) || !det) return OR_INVALID;
    const uint64_t P = p;
    uint32_t* W = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n * n + 1));
    if (!W) return OR_NOMEM;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) W[i * n + j] = (uint32_t)(A[i * lda + j] % P);
    uint64_t d = 1 % P;
    for (int64_t c = 0; c < n; c++) {
        int64_t piv = c;
        while (piv < n && W[piv * n + c] == 0) piv++;
        if (piv == n) { d = 0; break; }
        if (piv != c) {
            for (int64_t q = 0; q < n; q++) {
                const uint32_t x = W[c * n + q];
                W[c * n + q] = W[piv * n + q];
                W[piv * n + q] = x;
            }
            d = (P - d) % P;
        }
        const uint64_t pv = W[c * n + c], inv = inv_mod(pv, P);
        if (inv == 0) { free(W); return OR_INVALID; }
        d = (d * pv) % P;
#pragma omp parallel for schedule(static)
        for (int64_t t = c + 1; t < n; t++) {
            const uint64_t f = ((uint64_t)W[t * n + c] * inv) % P;
            if (f == 0) continue;
            for (int64_t q = c; q < n; q++)
                W[t * n + q] = (uint32_t)(((uint64_t)W[t * n + q] + (P - f) * W[c * n + q]) % P);
        }
    }
    free(W);
    *det = (uint32_t)d;
    return OR_OK;
}

/*
 * Inverse by Gauss-Jordan elimination on [A | I] (the classical definition;
 * section 6 derives it from LQUP and two triangular solves).  X receives
 * A^{-1} mod p.  Returns OR_OK, OR_SINGULAR if A is singular mod p (X is then
 * unspecified), or another negative OR_* code.  p prime.
 */
#define OR_SINGULAR 1
int oracle_inverse(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* X, int64_t ldx)
{
    if (p < 2 || n < 0 || (n > 0 && (lda < n || ldx < n))) return OR_INVALID;
    const uint64_t P = p;
    const int64_t w = 2 * n;
    uint32_t* W = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n * w + 1));
    if (!W) return OR_NOMEM;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) {
            W[i * w + j] = (uint32_t)(A[i * lda + j] % P);
            W[i * w + n + j] = (i == j) ? (uint32_t)(1 % P) : 0u;
        }
    for (int64_t c = 0; c < n; c++) {
        int64_t piv = c;
        while (piv < n && W[piv * w + c] == 0) piv++;
        if (piv == n) { free(W); return OR_SINGULAR; }
        if (piv != c)
            for (int64_t q = 0; q < w; q++) {
                const uint32_t x = W[c * w + q];
                W[c * w + q] = W[piv * w + q];
                W[piv * w + q] = x;
            }
        const uint64_t inv = inv_mod(W[c * w + c], P);
        if (inv == 0) { free(W); return OR_INVALID; }
        for (int64_t q = 0; q < w; q++) W[c * w + q] = (uint32_t)(((uint64_t)W[c * w + q] * inv) % P);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < n; t++) {
            if (t == c) continue;
            const uint64_t f = W[t * w + c];
            if (f == 0) continue;
            for (int64_t q = 0; q < w; q++)
                W[t * w + q] = (uint32_t)(((uint64_t)W[t * w + q] + (P - f) * W[c * w + q]) % P);
        }
    }
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) X[i * ldx + j] = W[i * w + n + j];
    free(W);
    return OR_OK;
}

/* Number of OpenMP threads the oracle runs with (reported as "cores"). */
int oracle_num_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}
