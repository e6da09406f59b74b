/*
 * ffgpu -- exact dense linear algebra over Z/pZ on one GB300 GPU (sm_103a).
 *
 * C ABI of the library libffgpu.so.  Plain pointers and sizes only.
 *
 * The operations follow Dumas, Giorgi and Pernet, "Dense linear algebra over
 * word-size prime fields: the FFLAS and FFPACK packages":
 *   fgemm  (section 3):   C <- alpha*A*B + beta*C over Z/pZ;
 *   ftrsm  (section 4):   B <- alpha*op(T)^{-1}*B (left) or alpha*B*op(T)^{-1} (right).
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major; lda, ldb, ldc, ldt are leading dimensions in
 *     elements (ld >= number of columns).  A is m x k, B is k x n, C is m x n.
 *   - Matrix pointers are DEVICE pointers owned by the caller; the library
 *     never frees them.  Elements are uint32 words; any word is accepted and
 *     taken mod p, as are alpha and beta.  Outputs are canonical residues in
 *     [0, p).
 *   - 2 <= p <= 2^31 - 1.  p need not be prime for fgemm.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Every call is asynchronous on that stream; argument errors are
 *     returned synchronously and nothing is enqueued.  A failure inside a
 *     kernel (a bounded wait that ran out) is recorded in a device error word
 *     read by ffgpu_last_device_error().
 *   - m, n or k may be 0: k = 0 gives C <- beta*C mod p; m = 0 or n = 0 is a
 *     no-op.  C must not overlap A or B.
 *   - Workspace: calls without an explicit workspace use a pool the library
 *     keeps per (device, stream), grown with stream-ordered allocation.  Two
 *     calls on the same stream are ordered and share it; calls on different
 *     streams use different pools.
 */
#ifndef FFGPU_H
#define FFGPU_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FFGPU_API __attribute__((visibility("default")))
#else
#define FFGPU_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FFGPU_OK = 0,
    FFGPU_ERR_INVALID = -1,       /* bad argument (shape, ld, null pointer, p out of range) */
    FFGPU_ERR_UNSUPPORTED_P = -2, /* p outside [2, 2^31-1] */
    FFGPU_ERR_NOMEM = -3,         /* workspace allocation failed or caller workspace too small */
    FFGPU_ERR_CUDA = -4,          /* a CUDA runtime call failed (launch, copy, no device) */
    FFGPU_ERR_TIMEOUT = -5,       /* a kernel's bounded wait ran out; its results are invalid */
    FFGPU_ERR_BUDGET = -6,        /* request exceeds a configured memory budget */
    FFGPU_ERR_SINGULAR = -7       /* the matrix is singular mod p (ffgpu_inverse) */
} ffgpu_status;

/* Human-readable name of a status code (static storage). */
FFGPU_API const char* ffgpu_status_string(ffgpu_status s);

/* Library version: major*10000 + minor*100 + patch. */
FFGPU_API int ffgpu_version(void);

/*
 * fgemm (section 3, the problem statement; eqs. 1-2 for the delayed
 * reduction that the kernel restates for its accumulator):
 *     C <- (alpha * A * B + beta * C) mod p.
 * A: m x k (lda), B: k x n (ldb), C: m x n (ldc), all device memory.
 * Path: residues are mapped to a residue number system of small moduli
 * (<= 256, bf16-exact), one tensor-core product per modulus with the
 * accumulator reduced in place before it can lose exactness, and a fused
 * epilogue that reconstructs the value mod p and applies alpha and beta.
 * Bit-exact: the result is the unique canonical residue.
 */
FFGPU_API ffgpu_status ffgpu_fgemm(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                         const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                         uint32_t beta, uint32_t* C, int64_t ldc, void* stream);

/*
 * fgemm with a choice of arithmetic path and Winograd levels (section 3.2):
 *   path FFGPU_PATH_RNS  (0): the default route of ffgpu_fgemm: the residue-number-
 *                             system tensor-core path, small products on the
 *                             CUDA cores (ffgpu_set_small_threshold);
 *   path FFGPU_PATH_FP64 (1): residues carried in doubles on the FP64 DMMA unit,
 *                             reduced after every 16 products (eq. 2, gamma = 53),
 *                             p < 2^25;
 *   path FFGPU_PATH_FP32 (2): residues carried in floats (SIMT FFMA), reduced
 *                             before the sum can reach 2^24 (eq. 1-2, gamma = 24),
 *                             p <= 256;
 *   path FFGPU_PATH_SIMT (3): exact 96-bit integer dot products on the CUDA
 *                             cores, one reduction per output (what ffgpu_fgemm
 *                             uses for small products, see
 *                             ffgpu_set_small_threshold); m below 4194240.
 * winograd_levels (0..8): recursive levels of Winograd's variant with the
 * schedule of Table 2 (additions mod p, products by the chosen path) and
 * dynamic peeling of odd dimensions.  Every combination gives the same exact
 * result as ffgpu_fgemm.  p outside a path's range: FFGPU_ERR_UNSUPPORTED_P.
 * unreduced = 1 (with winograd_levels >= 1; path ignored): the variant that
 * section 3.2 analyses -- the levels run over Z on balanced residues (int32
 * operands, exact int64 products and sums) and the result is reduced once
 * at the end; admitted only when Theorem 3.1's bound on every intermediate
 * value, (3^l (p-1)/2)^2 floor(k/2^l), is below 2^62 and the operands
 * (at most 4^l (p-1)/2) fit int32, else FFGPU_ERR_UNSUPPORTED_P
 * (ffgpu_winograd_unreduced_kmax gives the largest admitted k).
 */
typedef struct {
    int32_t path;
    int32_t winograd_levels;
    int32_t unreduced;     /* 1: the levels' additions over Z, no reduction until the end (below) */
    int32_t reserved[5];   /* must be zero */
} ffgpu_options;
#define FFGPU_PATH_RNS 0
#define FFGPU_PATH_FP64 1
#define FFGPU_PATH_FP32 2
#define FFGPU_PATH_SIMT 3

/* Largest inner dimension k that l unreduced Winograd levels admit for p
 * (Theorem 3.1 / Corollary 3.4 with a 62-bit exact range, int32 operands);
 * 0 if none.  Host-only.  FFGPU_ERR_INVALID for p outside [2, 2^31 - 1] or
 * l outside [1, 8]. */
FFGPU_API ffgpu_status ffgpu_winograd_unreduced_kmax(uint32_t p, int levels, int64_t* kmax);

/*
 * Products with m*n*k at most max_macs multiply-adds (default 2^27) are
 * computed by ffgpu_fgemm, ffgpu_ftrsm and the LQUP routines on the CUDA
 * cores (path FFGPU_PATH_SIMT): for them the tensor-core path's fixed costs
 * (conversions, one product per channel, the CRT epilogue) exceed the
 * arithmetic.  0 sends every product to the tensor cores.  Process-wide; not
 * in the paper.  FFGPU_ERR_INVALID for a negative value.
 */
FFGPU_API ffgpu_status ffgpu_set_small_threshold(int64_t max_macs);
FFGPU_API int64_t ffgpu_get_small_threshold(void);

FFGPU_API ffgpu_status ffgpu_fgemm_ex(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                                      const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                                      uint32_t beta, uint32_t* C, int64_t ldc, const ffgpu_options* opt,
                                      void* stream);

/*
 * Autotuner (the paper tunes its Winograd threshold experimentally, section
 * 3.2.1, and names self-adapting thresholds as further development, section
 * 7).  For a problem shape (m, n, k each bucketed to a multiple of 256), a
 * modulus p and a path, ffgpu_autotune times every candidate plan on the
 * device on scratch data it allocates (the route: tensor cores or, for
 * products of at most 2^31 multiply-adds, the CUDA-core kernel; the tensor
 * cores' tile shape, 128 x 256 on one CTA or 256 x 256 on a CTA pair; the
 * tile order, in bands of 4, 16 or 64 tile rows; the chunk length between
 * in-place reductions; 0-2 Winograd levels) and stores the fastest in an
 * in-memory plan cache.  ffgpu_fgemm then runs every product of that bucket
 * and modulus with the cached plan (Winograd levels included);
 * ffgpu_fgemm_ws and the request server apply the plan's route, tile shape,
 * tile order and chunk length (their workspace has no room for Winograd's
 * temporaries); the batched launch sends an instance to the CUDA cores or the
 * tensor cores as its cached plan says.  With an empty cache every call uses
 * the default rules.  ffgpu_fgemm_auto computes like ffgpu_fgemm_ex with the
 * cached plan (tuning first on a miss).  The cache can be saved to and
 * loaded from a JSON file.  Results never depend on the plan (every plan is
 * exact).
 */
typedef struct {
    int32_t kernel;            /* 0 = one-CTA 128x256 tiles, 1 = CTA-pair 256x256 tiles, -1 = default rule */
    int32_t winograd_levels;
    int32_t chunk_steps;       /* 64-long k-steps between in-place reductions (0 = longest exact) */
    int32_t route;             /* 0 = tensor cores, 1 = CUDA-core kernel, -1 = default size rule */
    int32_t raster_rows;       /* tile rows per band of the tile order (0 = 16) */
    int32_t reserved[3];
    double ms;                 /* measured time of the plan */
} ffgpu_tuned;

FFGPU_API ffgpu_status ffgpu_autotune(int64_t m, int64_t n, int64_t k, uint32_t p, int path, void* stream,
                                      ffgpu_tuned* out);
/* FFGPU_OK and *out if the cache holds a plan for the problem's bucket, else FFGPU_ERR_INVALID. */
FFGPU_API ffgpu_status ffgpu_autotune_lookup(int64_t m, int64_t n, int64_t k, uint32_t p, int path,
                                             ffgpu_tuned* out);
FFGPU_API ffgpu_status ffgpu_autotune_save(const char* json_path);
FFGPU_API ffgpu_status ffgpu_autotune_load(const char* json_path);
FFGPU_API ffgpu_status ffgpu_autotune_clear(void);
FFGPU_API ffgpu_status ffgpu_fgemm_auto(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                                        const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                                        uint32_t beta, uint32_t* C, int64_t ldc, int path, void* stream);

/* Bytes of device workspace ffgpu_fgemm_ws needs for this problem. */
FFGPU_API ffgpu_status ffgpu_fgemm_workspace_size(int64_t m, int64_t n, int64_t k, uint32_t p,
                                        size_t* bytes);

/*
 * ffgpu_fgemm with a caller-owned device workspace of at least
 * ffgpu_fgemm_workspace_size() bytes (256-byte aligned).  The workspace must
 * not be used by anything else until the call has completed on `stream`.
 * Kernel errors are reported through the device error word of `stream`'s pool.
 */
FFGPU_API ffgpu_status ffgpu_fgemm_ws(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                            const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                            uint32_t beta, uint32_t* C, int64_t ldc,
                            void* workspace, size_t workspace_bytes, void* stream);

/*
 * ffgpu_fgemm for callers that cannot let the library allocate device memory.
 * The paper has no counterpart: this is a deployment variant of fgemm.
 *
 * Who needs it: code whose host framework owns all device memory and forbids
 * allocation in its execution path, latency-critical paths that cannot afford
 * an allocation's implicit synchronisation or its failure, and processes that
 * have already reserved the whole device.  The call computes the same result
 * as ffgpu_fgemm (same arguments, same output, bit for bit) but takes its
 * scratch from a static device array of FFGPU_NOALLOC_SCRATCH_BYTES that the
 * library holds on every GPU that loads it, until the process exits.  It calls
 * no cudaMalloc, cudaFree or allocating library routine and records no
 * profiling events.
 *
 * Limit: a problem whose scratch exceeds the array returns FFGPU_ERR_NOMEM
 * and enqueues nothing.  A product that runs on the CUDA cores (at most
 * ffgpu_get_small_threshold() multiply-adds) needs only its k-split partial
 * sums, a few MB at most.  Any other product needs the bf16 channel planes of
 * A and B plus the residue slots of at most 32 persistent CTAs: for p < 2^31
 * about 20*(m+n)*k + 21 MB bytes, so m = n = 1024 fits up to k = 1088.
 *
 * Set-up: the first call on a device looks up the array's device address on
 * that device (which may load the library's GPU code there); make that first
 * call before any stream capture.  Every call shares the one array and it
 * keeps the previous call's contents: calls whose work may overlap on the GPU
 * (different streams, or different host threads) race and must be ordered by
 * the caller.  A bounded wait that runs out inside the kernel ends it early and
 * leaves C undefined; this entry point does not report such a failure.
 */
#define FFGPU_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
FFGPU_API ffgpu_status ffgpu_fgemm_noalloc(int64_t m, int64_t n, int64_t k, uint32_t p,
                                           uint32_t alpha, const uint32_t* A, int64_t lda,
                                           const uint32_t* B, int64_t ldb, uint32_t beta,
                                           uint32_t* C, int64_t ldc, void* stream);

/*
 * ftrsm (section 4, Algorithm 1: block recursive triangular solve with a
 * matrix right-hand side), in place on B:
 *     side 0 (left):  B <- alpha * T^{-1} * B,  T is m x m;
 *     side 1 (right): B <- alpha * B * T^{-1},  T is n x n.
 * uplo 0 = lower, 1 = upper triangle of T is used (the other is not read);
 * diag 0 = non-unit, 1 = unit diagonal (diagonal entries are not read).
 * T (ldt) and B (ldb) are row-major device arrays; B is m x n.
 * The recursion stops at diagonal blocks of 128 to 1024 rows, whose inverses
 * are formed first (substitution mod p on 128-row blocks, then doubling with
 * batched products); each such block is then one product with its inverse,
 * and every other step is an fgemm update on the same stream.  A
 * non-invertible diagonal entry
 * (non-unit) cannot be detected before the kernels run: it is recorded on the
 * device and ffgpu_last_device_error then returns FFGPU_ERR_INVALID (B is
 * undefined).
 */
FFGPU_API ffgpu_status ffgpu_ftrsm(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p,
                                   uint32_t alpha, const uint32_t* T, int64_t ldt, uint32_t* B,
                                   int64_t ldb, void* stream);

/*
 * ftrsm with the algorithm chosen (ffgpu_ftrsm uses FFGPU_TRSM_DEFAULT):
 *   FFGPU_TRSM_RECURSIVE  Algorithm 1 (section 4.1): split the triangle in two,
 *                         solve, update the other half with one fgemm, solve;
 *                         every level's update is reduced mod p.
 *   FFGPU_TRSM_DELAYED    the delayed-reduction idea of Algorithms 2-3
 *                         (section 4.2) restated: left-looking, each block of
 *                         X computed by ONE product over all earlier blocks at
 *                         once, X_i = [Inv_i | -Inv_i T_i,prev] [B_i ; X_prev],
 *                         so every output block is reduced exactly once (the
 *                         residue system keeps the whole accumulation exact).
 *   FFGPU_TRSM_CASCADE    Algorithms 2-3 (section 4.3) as the paper states
 *                         them: blocks of t_split rows (Algorithm 2), each
 *                         solved by the recursion of Algorithm 3 with its
 *                         updates over Z (int64, exact products on the tensor
 *                         cores, no reduction) and leaves of t_del rows solved
 *                         over Z (eq. trsmboundcen), then reduced mod p; the
 *                         rows below a block updated by one fgemm mod p.
 *                         Non-unit diagonals are normalised first (T = D U,
 *                         section 4.2).  ffgpu_ftrsm_cascade_params gives
 *                         t_del, t_update and t_split for p.
 *   FFGPU_TRSM_DEFAULT    the recursive algorithm (measured the fastest at
 *                         every size tried, n = 2048 to 8192).
 * Same arguments, results and errors as ffgpu_ftrsm; FFGPU_ERR_INVALID for an
 * unknown algorithm.
 */
#define FFGPU_TRSM_DEFAULT (-1)
#define FFGPU_TRSM_RECURSIVE 0
#define FFGPU_TRSM_DELAYED 1
#define FFGPU_TRSM_CASCADE 2
FFGPU_API ffgpu_status ffgpu_ftrsm_ex(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                                      const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, int algorithm,
                                      void* stream);

/*
 * The thresholds of FFGPU_TRSM_CASCADE for p (section 4.2-4.3, balanced
 * residues |x| <= h = floor(p/2), carried in 64-bit signed integers):
 *   t_del    the largest n with h (h+1)^n < 2^63 (eq. trsmboundcen with
 *            gamma = 63): rows of a leaf solved over Z with no reduction;
 *   t_update the largest t with t h^2 + h < 2^62 (eq. 2 with gamma = 63, one
 *            term reserved for the right-hand side itself): products a
 *            right-hand side entry accumulates over Z between reductions;
 *   t_split  floor(t_update / t_del) t_del (Algorithm 2).
 * t_del is capped at 128 rows and t_update at 2^31 - 1.  Host-only; no device
 * is touched.  FFGPU_ERR_UNSUPPORTED_P outside 2 <= p < 2^31,
 * FFGPU_ERR_INVALID for a null output pointer.
 */
FFGPU_API ffgpu_status ffgpu_ftrsm_cascade_params(uint32_t p, int64_t* t_del, int64_t* t_update, int64_t* t_split);

/*
 * LQUP factorization over Z/pZ (section 5: A = L Q U P, L lower triangular,
 * Q and P permutations, U upper triangular of rank r with its first r rows
 * non-zero; block recursion on the rows, reduced to ftrsm and fgemm).
 * In place and packed: afterwards A[rowperm][:, colperm] = L U mod p with
 *   L  m x r, unit lower trapezoidal, stored strictly below the diagonal of
 *      A's first r columns (its unit diagonal is not stored);
 *   U  r x n, upper trapezoidal with a non-zero diagonal, stored on and above
 *      the diagonal of A's first r rows;
 *   A's rows r..m-1 are zero from column r on.
 * Pivot rule (the paper leaves it open): rows are met top to bottom; a row
 * whose Schur complement is non-zero is the next pivot row and its pivot
 * column is the first non-zero one in original column order.  rowperm
 * (device, m entries) lists the pivot rows in order, then the other rows
 * ascending; colperm (device, n entries) the pivot columns in pivot order,
 * then the other columns ascending.  With this rule the result is unique.
 * *rank (host) receives r.
 * A: device, row-major, lda >= n, entries any uint32 (taken mod p).  p must
 * be a prime in [2, 2^31 - 1], else FFGPU_ERR_UNSUPPORTED_P.  The call is
 * host-synchronous: pivot decisions are read back as the recursion proceeds
 * (workspace from the stream's pool).  Part of some updates runs on a
 * library-owned side stream of the calling thread; the call returns only
 * after that stream's work is done.  Errors: FFGPU_ERR_INVALID (shapes,
 * null pointers, m or n above 2^30), FFGPU_ERR_NOMEM, FFGPU_ERR_CUDA,
 * FFGPU_ERR_TIMEOUT (a product's bounded wait ran out); after an error other
 * than an argument check, A, rowperm and colperm are unspecified.
 */
FFGPU_API ffgpu_status ffgpu_lqup(int64_t m, int64_t n, uint32_t p, uint32_t* A, int64_t lda, int64_t* rank,
                                  int32_t* rowperm, int32_t* colperm, void* stream);

/*
 * Rank of A mod p (section 6: the number of non-zero rows of U), from the
 * LQUP of a copy of A; A (device, lda >= n) is not modified; *rank on the
 * host.  Same p rule, synchronization and errors as ffgpu_lqup.
 */
FFGPU_API ffgpu_status ffgpu_rank(int64_t m, int64_t n, uint32_t p, const uint32_t* A, int64_t lda, int64_t* rank,
                                  void* stream);

/*
 * Determinant of the n x n matrix A mod p (section 6: the product of U's
 * diagonal, zero as soon as the rank is below n), signed by the column
 * permutation; *det on the host, in [0, p); n = 0 gives 1.  A (device) is not
 * modified.  Same p rule, synchronization and errors as ffgpu_lqup.
 */
FFGPU_API ffgpu_status ffgpu_det(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* det,
                                 void* stream);

/*
 * Inverse of the n x n matrix A mod p (section 6, "Matrix inverse": LQUP,
 * then X = P^{-1} U^{-1} L^{-1} Q^{-1} by two triangular solves and a row
 * permutation).  X (device, ldx >= n, must not overlap A) receives A^{-1};
 * A is not modified.  FFGPU_ERR_SINGULAR if A is singular mod p (X is then
 * unchanged).  Same p rule, synchronization and other errors as ffgpu_lqup.
 */
FFGPU_API ffgpu_status ffgpu_inverse(int64_t n, uint32_t p, const uint32_t* A, int64_t lda, uint32_t* X,
                                     int64_t ldx, void* stream);

/* One independent fgemm of a batch: C <- (alpha*A*B + beta*C) mod p. */
typedef struct {
    int64_t m, n, k;
    uint32_t p, alpha, beta;
    const uint32_t* A;
    int64_t lda;
    const uint32_t* B;
    int64_t ldb;
    uint32_t* C;
    int64_t ldc;
} ffgpu_fgemm_desc;

/*
 * Batched fgemm: `count` independent problems of any shapes and moduli
 * (descs is a HOST array; every matrix is device memory).  Problems are
 * grouped by padded inner length; for each group of at most a few GiB of
 * channel planes the library enqueues one grouped conversion of all A's, one
 * of all B's, and ONE persistent tensor-core launch whose CTAs walk a job
 * list (instance, tile, modulus) balanced by cost (longest first).  Results
 * equal ffgpu_fgemm on each descriptor.  No C may overlap an A, a B or
 * another C of the batch.  Invalid descriptors fail the whole call before
 * anything is enqueued.
 */
FFGPU_API ffgpu_status ffgpu_fgemm_batched(int64_t count, const ffgpu_fgemm_desc* descs, void* stream);

/*
 * The batched launch's own threshold: products of at most that many
 * multiply-adds (2^23 by default) run in the grouped CUDA-core launch, the
 * rest in grouped tensor-core launches.  ffgpu_autotune_batched times this
 * batch (as ffgpu_fgemm_batched would run it) for thresholds 2^20 .. 2^26,
 * keeps the fastest for every later batched call (and in saved plan files),
 * and returns it in *best_macs.  Every descriptor's C receives alpha A B
 * (beta is taken as 0 so that the repeated runs agree): call it before the
 * real computation.  Synchronous.
 */
FFGPU_API ffgpu_status ffgpu_autotune_batched(int64_t count, const ffgpu_fgemm_desc* descs, void* stream,
                                              int64_t* best_macs);

/*
 * Batched plan: the launch sequence of ffgpu_fgemm_batched for one fixed
 * batch, laid out once and captured in a CUDA graph (the repeated-batch use of
 * the multi-modular products the paper's section 7 points to: the same shapes
 * and buffers, new contents each time).
 *
 * ffgpu_fgemm_batched_plan_create validates the descriptors (host array,
 * copied; the matrices are device memory on the current device), plans the
 * waves, allocates the plan's device memory (the largest wave's channel
 * planes and residue slots, every wave's tables, a workspace for products that
 * run outside the grouped launch, an error word), uploads the tables and
 * captures the conversions and tensor-core launches of every wave into a
 * graph.  It synchronizes the device.  Errors: FFGPU_ERR_INVALID /
 * FFGPU_ERR_UNSUPPORTED_P for a bad descriptor, FFGPU_ERR_NOMEM, FFGPU_ERR_CUDA;
 * *plan is NULL on failure.
 *
 * ffgpu_fgemm_batched_plan_run enqueues the graph on `stream` (current device
 * must be the plan's, else FFGPU_ERR_INVALID): every C of the batch becomes
 * (alpha*A*B + beta*C) mod p from the CURRENT contents of its A, B and C.
 * The pointers in the descriptors must stay valid while the plan lives.  Runs
 * of one plan share its workspace: two runs must not overlap (same stream, or
 * ordered by events).
 *
 * ffgpu_fgemm_batched_plan_error synchronizes the device and returns (and
 * clears) the plan's device error word: FFGPU_ERR_TIMEOUT after a bounded
 * wait expired in a run.  ffgpu_fgemm_batched_plan_info reports the wave
 * count, the products run outside the grouped launch, the graph's node count
 * and the plan's device bytes (any pointer may be NULL).
 * ffgpu_fgemm_batched_plan_destroy synchronizes the device and frees the plan
 * (NULL is accepted).
 */
/*
 * Multi-modular products from one exact integer product: for integer
 * matrices A (m x k) and B (k x n), int32 row-major on the device, every entry
 * of magnitude at most 2^bits (1 <= bits <= 30, and k 2^(2 bits) < 2^62 so
 * that A B fits in int64), writes C_i = (A B) mod p_i in [0, p_i) for each of
 * the nprimes moduli (1 <= nprimes <= 64, 2 <= p_i < 2^31; primes is a HOST
 * array, C a HOST array of nprimes device pointers, each an m x n uint32
 * matrix with leading dimension ldc).  Computes the integer product once
 * (channel residues of A and B, the tensor-core channel products, the exact
 * 64-bit reconstruction) and then reduces it modulo every p_i -- the
 * multi-modular use the paper cites for its routines (introduction; section 7:
 * the Chinese remainder algorithm) -- instead of one fgemm per prime.  Entries
 * beyond 2^bits in magnitude give undefined results.  Asynchronous on
 * `stream`; workspace from the stream's pool.  Errors: FFGPU_ERR_INVALID
 * (shapes, bits, the int64 bound, null pointers), FFGPU_ERR_UNSUPPORTED_P,
 * FFGPU_ERR_NOMEM, FFGPU_ERR_CUDA.  No C_i may overlap A, B or another C_j.
 */
FFGPU_API ffgpu_status ffgpu_fgemm_multimod(int64_t m, int64_t n, int64_t k, int bits, const int32_t* A, int64_t lda,
                                            const int32_t* B, int64_t ldb, int nprimes, const uint32_t* primes,
                                            uint32_t* const* C, int64_t ldc, void* stream);

/*
 * Batched multi-modular products (the configuration of many integer
 * instances, each reduced modulo the same primes): for every descriptor,
 * C[i] = (A B) mod primes[i] as ffgpu_fgemm_multimod would compute it, with
 * the instances' exact products done in grouped launches (one grouped
 * conversion per operand, one persistent integer-mode tensor-core launch and
 * one grouped fan-out per wave of instances).  descs is a HOST array; each
 * descriptor's C is a HOST array of nprimes device pointers (m x n uint32,
 * leading dimension ldc).  Same bounds and errors as ffgpu_fgemm_multimod,
 * checked for every descriptor before anything is enqueued.
 */
typedef struct {
    int64_t m, n, k;
    const int32_t* A;
    int64_t lda;
    const int32_t* B;
    int64_t ldb;
    uint32_t* const* C;
    int64_t ldc;
} ffgpu_multimod_desc;
FFGPU_API ffgpu_status ffgpu_fgemm_multimod_batched(int64_t count, const ffgpu_multimod_desc* descs, int bits,
                                                    int nprimes, const uint32_t* primes, void* stream);

typedef struct ffgpu_batched_plan ffgpu_batched_plan;
FFGPU_API ffgpu_status ffgpu_fgemm_batched_plan_create(int64_t count, const ffgpu_fgemm_desc* descs,
                                                       ffgpu_batched_plan** plan);
FFGPU_API ffgpu_status ffgpu_fgemm_batched_plan_run(ffgpu_batched_plan* plan, void* stream);
FFGPU_API ffgpu_status ffgpu_fgemm_batched_plan_error(ffgpu_batched_plan* plan);
FFGPU_API ffgpu_status ffgpu_fgemm_batched_plan_info(const ffgpu_batched_plan* plan, int* waves, int* singles,
                                                     size_t* graph_nodes, size_t* device_bytes);
FFGPU_API ffgpu_status ffgpu_fgemm_batched_plan_destroy(ffgpu_batched_plan* plan);

/*
 * Request server (continuous batching).  Not in the paper: the deployment of
 * fgemm / ftrsm as a service.  Requests carry HOST operands (pinned memory
 * for overlap) and a host output buffer.  An engine thread admits pending
 * requests in arrival order whenever one of `streams` worker streams is free
 * and a device arena of `budget_bytes` (allocated at creation, the HBM budget)
 * holds the request's operands and workspace; the admitted request is copied
 * in, computed and copied out on its stream, overlapping with the others.
 * Each result equals what ffgpu_fgemm / ffgpu_ftrsm give alone.
 */
typedef struct ffgpu_server ffgpu_server;

typedef struct {
    int32_t kind;            /* 0 = fgemm, 1 = ftrsm */
    int32_t side, uplo, diag;  /* ftrsm: as in ffgpu_ftrsm */
    int64_t m, n, k;         /* fgemm: A m x k, B k x n;  ftrsm: B m x n (k unused) */
    uint32_t p, alpha, beta;
    const uint32_t* A;       /* host; fgemm A, ftrsm T */
    int64_t lda;
    const uint32_t* B;       /* host; fgemm B, ftrsm right-hand sides */
    int64_t ldb;
    const uint32_t* C_in;    /* host; fgemm C when beta != 0 (else may be NULL) */
    int64_t ldc_in;
    uint32_t* out;           /* host; result m x n (fgemm C, ftrsm X) */
    int64_t ldo;
    uint64_t tag;            /* caller's identifier, echoed in the completion */
} ffgpu_request;

typedef struct {
    uint64_t tag;
    int32_t status;          /* ffgpu_status of the request */
    double t_submit_us, t_admit_us, t_done_us;  /* CLOCK_MONOTONIC, microseconds */
} ffgpu_completion;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    int64_t pending, inflight, peak_inflight;
    int64_t peak_bytes, budget_bytes, used_bytes;
} ffgpu_server_stats;

/* Creates a server on the current device (1..64 streams, budget >= 1 MiB). */
FFGPU_API ffgpu_status ffgpu_server_create(int streams, size_t budget_bytes, ffgpu_server** out);
/* Queues a request (returns at once).  FFGPU_ERR_BUDGET if it can never fit the budget. */
FFGPU_API ffgpu_status ffgpu_server_submit(ffgpu_server* server, const ffgpu_request* req);
/* Up to `cap` completions; waits up to wait_ms for the first one. */
FFGPU_API ffgpu_status ffgpu_server_poll(ffgpu_server* server, ffgpu_completion* out, int cap, int* count,
                                         int wait_ms);
FFGPU_API ffgpu_status ffgpu_server_get_stats(ffgpu_server* server, ffgpu_server_stats* out);
/* Drops pending requests, waits for admitted ones, frees everything. */
FFGPU_API ffgpu_status ffgpu_server_destroy(ffgpu_server* server);

/* Description of how ffgpu_fgemm computes a problem (for benchmarks and tests). */
typedef struct {
    int32_t mode;         /* 1 = single modulus p (p <= 256); 2 = residue number system */
    int32_t channels;     /* number of moduli, i.e. tensor-core products per output tile */
    uint32_t moduli[16];  /* the moduli in use */
    int32_t k_chunk;      /* inner-dimension length summed between in-place reductions */
    int32_t k_slices;     /* > 1 when k is split into several launches */
    int32_t tile_m, tile_n, tile_k;
    double mma_flops;     /* 2*m*n*k*channels: tensor-core operations issued */
} ffgpu_plan_info;

FFGPU_API ffgpu_status ffgpu_fgemm_plan(int64_t m, int64_t n, int64_t k, uint32_t p, ffgpu_plan_info* out);

/*
 * Synchronizes `stream`, returns FFGPU_ERR_TIMEOUT if a kernel launched on it
 * since the last call recorded a timed-out wait, FFGPU_ERR_INVALID if an
 * ftrsm met a non-invertible diagonal entry (and clears the record), FFGPU_OK
 * otherwise, or FFGPU_ERR_CUDA if the stream reports a CUDA error.
 */
FFGPU_API ffgpu_status ffgpu_last_device_error(void* stream);

/*
 * Kernel timing.  While enabled, every kernel the library launches is
 * bracketed by two CUDA events recorded on its launching stream.
 * ffgpu_profile_read synchronizes those events, sums their durations per
 * kernel name into out[0..cap) (sorted by name), sets *count to the number of
 * distinct kernels, and clears the record.  Off by default; costs two event
 * records per launch when on.
 */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} ffgpu_kernel_time;

FFGPU_API ffgpu_status ffgpu_profile_enable(int on);
FFGPU_API ffgpu_status ffgpu_profile_read(ffgpu_kernel_time* out, int cap, int* count);

/*
 * Self-test of failure detection (not in the paper): launches on `stream` a
 * kernel whose single wait targets a barrier that nothing completes, with a
 * limit of `limit_cycles` SM clock cycles (1 .. 2e9).  The wait gives up, the
 * kernel records a timeout and returns; ffgpu_last_device_error(stream) then
 * reports FFGPU_ERR_TIMEOUT and the context stays usable.  Every wait in the
 * library's kernels uses the same bounded mechanism (limit about one second).
 */
FFGPU_API ffgpu_status ffgpu_selftest_wait_timeout(int64_t limit_cycles, void* stream);

/*
 * Peak rate of a warp-level MMA unit, measured now on the current device:
 * register-only mma.sync chains on every SM for `iters` iterations (1 .. 2^24),
 * timed with CUDA events.  kind 0: int8 (m16n8k32, s8 x s8 -> s32), 1: bf16
 * (m16n8k16 -> f32), 2: FP64 DMMA (m8n8k4).  *ops_per_second counts 2 M N K
 * per MMA.  tcgen05 has no int8 kind on sm_103a, so kind 0 is this GPU's int8
 * tensor rate, the reference point beside the bf16 tensor-core roofline.
 * Synchronizes `stream`.  Not in the paper.
 */
FFGPU_API ffgpu_status ffgpu_peak_probe(int kind, int64_t iters, double* ops_per_second, void* stream);

/* Frees every workspace pool of the calling process (synchronizes the device). */
FFGPU_API ffgpu_status ffgpu_release_workspaces(void);

#ifdef __cplusplus
}
#endif

#endif /* FFGPU_H */
