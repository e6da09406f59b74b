// Internal declarations shared by the CUDA translation units of libffgpu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ffgpu.h"

namespace ffgpu {

// ---------------------------------------------------------------------------
// Residue number system.  Odd moduli <= 255 whose balanced residues
// (|r| <= 127) are exact bfloat16 values; pairwise coprime; in decreasing
// order so that the first c of them give the largest product for c channels.
// ---------------------------------------------------------------------------
constexpr int kMaxChannels = 12;
constexpr uint32_t kModuli[kMaxChannels] = {255, 253, 251, 247, 241, 239,
                                            233, 229, 227, 223, 211, 199};
// Largest modulus handled as a single channel (residues |x| <= 127).
constexpr uint32_t kDirectMaxP = 255;

// Tile of the tensor-core kernel.
constexpr int kTileM = 128;
constexpr int kTileN = 256;
constexpr int kTileK = 64;       // one 128-byte swizzle row of bf16
constexpr int kChunkSteps = 16;  // default: 16 x 64 = 1024 products summed between in-place reductions
constexpr int kStages = 4;

// Error codes written to the device error word.
enum DevErr : int {
    kDevOk = 0,
    kDevTimeoutProducer = 1,
    kDevTimeoutMma = 2,
    kDevTimeoutEpilogue = 3,
    kDevTimeoutDrain = 4,
    kDevSingular = 5,  // a non-unit triangular solve met a non-invertible diagonal entry
    kDevTimeoutStreamK = 6,  // a cut tile's head waited too long for its tail's residues
};

struct RnsPlan {
    int mode;        // 1 = direct (modulus p itself), 2 = RNS
    int nch;         // channels
    uint32_t p;
    uint32_t mod[kMaxChannels];
    uint32_t u[kMaxChannels];      // (M/m_c)^{-1} mod m_c
    uint32_t W[kMaxChannels];      // (M/m_c) mod p
    uint32_t negMp;                // (p - (M mod p)) mod p
    int64_t k_slice;               // largest inner length one launch may sum
};

// One fgemm instance as the tensor-core kernel sees it.
struct InstInfo {
    int m, n;
    int ksteps;                    // kp / 64
    int chunk_steps;               // k-steps summed between in-place reductions
    int nch;
    int direct;
    int vec_ok;                    // 16-byte vector access to C is legal
    uint32_t p;
    uint32_t alpha, beta;          // reduced mod p
    uint32_t negMpa;               // alpha * (p - M mod p) mod p
    uint32_t R32, R32s;            // 2^32 mod p and its Shoup quotient floor(R32 2^32 / p)
    uint32_t one_s;                // floor(2^32 / p): Shoup quotient of 1
    uint32_t beta_s;               // floor(beta 2^32 / p)
    uint32_t Kfix;                 // (-128 sum_c Wa_c - 6 negMpa) mod p: start value of the CRT sum
    uint32_t Finit;                // 6 2^14 + 2^13 - 128 sum_c fr_c (mod 2^32): start value of the quotient sum
    int int_out;                   // 1: integer mode -- C is an int64 array receiving the exact product
    unsigned long long Mfull;      // integer mode: M = prod m_c
    unsigned long long Xoff;       // integer mode: 128 sum_c M/m_c + 6 M (removed from the offset sums)
    uint32_t* C;
    long long ldc;
    int bucket;                    // grouped launch: tensor-map pair of this instance
    int rowA, rowB;                // grouped launch: first plane row of this instance
    float modf[kMaxChannels];
    float inv_m[kMaxChannels];
    uint32_t modu[kMaxChannels];
    uint32_t u[kMaxChannels];      // (M/m_c)^{-1} mod m_c (1 in direct mode)
    uint32_t Wa[kMaxChannels];     // alpha * (M/m_c) mod p (integer mode: low 32 bits of M/m_c)
    uint32_t fr[kMaxChannels];     // round(2^14 / m_c): fixed-point weight of b_c / m_c
    uint32_t Mhi[kMaxChannels];    // integer mode: high 32 bits of M/m_c
};

// Parameters of the single-instance tensor-core kernel (passed by value).
struct RnsGemmParams {
    InstInfo inst;
    int tiles_m, tiles_n, num_tiles;
    unsigned char* slots;          // per-CTA residue slots: 2 x slot_stride bytes per CTA
    size_t slot_stride;            // bytes of one slot: channels x 128 x 256
    int* err;                      // device error word
    int raster;                    // tile rows per band of the tile order (> 0)
    // CTA-pair kernel, cut last wave (sk_split > 1): the sk_rem tiles from
    // sk_dp on, each in sk_split parts of its chunks
    int sk_dp, sk_split, sk_rem;
    short* sk_part;                // tails' residues: pairs x 2 x channels x 128 x 256 int16
    int* sk_flags;                 // pairs x 2 x channels x kSkFlagsPerCta, zero at launch
};
constexpr int kSkFlagsPerCta = 8;  // one per epilogue warp

// Grouped launch: jobs (instance, tile, channel), listed per CTA, with
// everything the producer, MMA and epilogue roles need packed in 32 bytes so
// that one (prefetched) load per job suffices:
//   tmtn = tile row (bits 0-15) | tile column (bits 16-31)
//   cfg  = channel (bits 0-7) | residue slot of the tile (bit 8) |
//          channel count (bits 12-15) | k-bucket of the instance (bits 16-31)
//   modc = modulus m_c (bits 0-7) | (M/m_c)^{-1} mod m_c (bits 8-15) |
//          chunk length in k-steps (bits 16-23)
struct alignas(32) GroupJob {
    int inst;
    uint32_t tmtn;
    uint32_t cfg;
    uint32_t modc;
    int ksteps;        // k-steps of the instance
    int H;             // chunks
    int rowA, rowB;    // first plane rows of the tile's A and B blocks in the bucket's pools
};
struct GroupGemmParams {
    const InstInfo* insts;
    const GroupJob* jobs;
    const int* cta_begin;          // jobs of CTA b: [cta_begin[b], cta_begin[b+1])
    const CUtensorMap* maps;       // 2 per k-bucket: A planes, B planes (64-byte aligned)
    unsigned char* slots;          // 2 x slot_stride bytes per CTA
    size_t slot_stride;
    int* err;
};

constexpr size_t kSlotBytesPerCta = size_t(kMaxChannels) * kTileM * kTileN;  // one slot, any channel count
constexpr int kSlotsPerCta = 2;  // double buffered: residues of one tile, reconstruction of the previous

// Conversion parameters: uint32 words -> bf16 channel planes.
struct ConvertParams {
    uint32_t p;
    uint32_t half_p;                 // floor(p/2): residues above it are centred to x - p
    uint32_t mu32;                   // floor((2^32-1)/p)
    int nch;
    int direct;
    int signed_input;                // 1: words are int32 integers (|x| < 2^31), taken as they are, not mod p
    uint32_t mod[kMaxChannels];      // odd moduli <= 255
    uint32_t magic32[kMaxChannels];  // ceil(2^39 / m_c) < 2^32
};

// One matrix of a grouped conversion.  A (rows mode): X is rows (= m) x cols
// (= k), written to dst[c][r][kp] for r < rows_pad (m padded).  B (transposed
// mode): X is rows (= k) x cols (= n), written to dst[c][j][kp] for
// j < rows_pad (n padded).  Padding is written as zeros.
struct ConvJob {
    const uint32_t* X;
    long long ldx;
    int rows, cols;
    int rows_pad;
    int kp;
    int vec_ok;
    uint4* dst;            // this matrix's first plane row (channel 0) in its bucket pool
    size_t plane16;        // channel stride of the bucket pool, in 16-byte units
    ConvertParams cp;
};

// An operand given as a signed sum of up to kMaxTerms blocks of the same
// shape, sum_t (-1)^neg[t] X_t mod p (entries any uint32 words): the pre-added
// operands of Winograd's levels (S1..S4, T1..T4 of Table 2 and, two levels
// deep, their quadrants' sums), converted to channel planes in one pass
// without being written out.
constexpr int kMaxTerms = 16;
struct SumSrc {
    const uint32_t* X[kMaxTerms];
    long long ld[kMaxTerms];
    uint32_t neg[kMaxTerms];
    int n;
};

// host launchers (implemented in the .cu files)
long long convert_rows_grouped_blocks(int rows_pad);
long long convert_transpose_grouped_blocks(int cols_pad, int kp);
cudaError_t launch_convert_rows_grouped(const ConvJob* jobs, const long long* block_begin, int njobs,
                                        long long nblocks, cudaStream_t s);
cudaError_t launch_convert_transpose_grouped(const ConvJob* jobs, const long long* block_begin, int njobs,
                                             long long nblocks, cudaStream_t s);
cudaError_t launch_convert_rows(const uint32_t* X, long long ldx, int rows, int cols, int colsp,
                                const ConvertParams& cp, void* planes, cudaStream_t s);
cudaError_t launch_convert_transpose(const uint32_t* X, long long ldx, int rows, int cols, int rowsp,
                                     const ConvertParams& cp, void* planes, cudaStream_t s);
cudaError_t launch_scale(uint32_t* C, long long ldc, int m, int n, uint32_t p, uint32_t beta,
                         unsigned long long mu, cudaStream_t s);
// the same conversions with the words formed as a signed sum of blocks
cudaError_t launch_convert_rows_sum(const SumSrc& X, int rows, int cols, int colsp, const ConvertParams& cp,
                                    void* planes, cudaStream_t s);
cudaError_t launch_convert_transpose_sum(const SumSrc& X, int rows, int cols, int rowsp, const ConvertParams& cp,
                                         void* planes, cudaStream_t s);
// Z = the sum (rows x cols) mod p, written out (canonical residues)
cudaError_t launch_sum_mod(const SumSrc& X, int rows, int cols, uint32_t p, uint32_t* Z, long long ldz,
                           cudaStream_t s);
cudaError_t launch_rns_gemm(const CUtensorMap& mapA, const CUtensorMap& mapB,
                            const RnsGemmParams& prm, int grid, cudaStream_t s);
cudaError_t launch_rns_gemm_grouped(const GroupGemmParams& prm, int grid, cudaStream_t s, bool int_out = false);
cudaError_t launch_rns_gemm_int(const CUtensorMap& mapA, const CUtensorMap& mapB, const RnsGemmParams& prm,
                                int grid, cudaStream_t s);
cudaError_t launch_rns_gemm_pair(const CUtensorMap& mapA, const CUtensorMap& mapB, const RnsGemmParams& prm,
                                 int grid, cudaStream_t s);
bool use_pair_kernel(int64_t m, int grid);

// Plan settings for the calling thread (autotune.cu): set while a tuned plan
// or a tuning candidate runs.
//   kernel       0 = one-CTA kernel (128 x 256 tiles), 1 = CTA pair (256 x 256), -1 = default choice
//   chunk_steps  > 0 caps the chunk length between in-place reductions
//   route        0 = tensor cores, 1 = CUDA-core kernel, -1 = the size rule (fgemm_small)
//   raster       tile rows per band of the tile order (0 = kRasterRows)
struct TuneOverride {
    int kernel = -1;
    int chunk_steps = 0;
    int route = -1;
    int raster = 0;
};
extern thread_local TuneOverride g_tune_override;
// Installs a plan's settings for the calling thread until the scope ends.
struct ScopedTune {
    TuneOverride saved;
    explicit ScopedTune(const TuneOverride& t) : saved(g_tune_override) { g_tune_override = t; }
    ~ScopedTune() { g_tune_override = saved; }
};
// The cached plan for a product (path 0), if the plan cache holds one for its
// shape bucket and modulus: its settings and Winograd depth.
bool autotune_settings(int64_t m, int64_t n, int64_t k, uint32_t p, TuneOverride& o, int& levels);
// Route the cache gives a product (-1: no entry, 0 tensor cores, 1 CUDA cores).
int autotune_route(int64_t m, int64_t n, int64_t k, uint32_t p);
// Largest product (multiply-adds) the batched launch sends to the grouped CUDA-core kernel.
int64_t batched_small_macs();
void set_batched_small_macs(int64_t macs);
// A threshold for the calling thread's batched launches until the scope ends
// (the ftrsm's doubling products: one batch of equal products, where the
// single-product crossover applies rather than the mixed batch's).
extern thread_local int64_t g_batch_small_scoped;
struct ScopedBatchSmall {
    int64_t saved;
    explicit ScopedBatchSmall(int64_t macs) : saved(g_batch_small_scoped) { g_batch_small_scoped = macs; }
    ~ScopedBatchSmall() { g_batch_small_scoped = saved; }
};
constexpr int kRasterRows = 16;  // default tile rows per band of the tile order
int rns_gemm_pair_max_clusters();
size_t rns_gemm_smem_bytes();

// Workspace pool of one (device, stream).
struct Pool {
    void* ptr = nullptr;
    size_t bytes = 0;
    int* err = nullptr;
};
ffgpu_status pool_get(cudaStream_t s, size_t need, Pool** out);

// fgemm launch sequence shared by the entry points (ffgpu_host.cu).  ws is a
// 256-byte aligned workspace of ws_bytes; max_grid > 0 caps the number of
// persistent CTAs (and so the residue slots the workspace must hold); untimed
// launches skip the optional profiling events.
ffgpu_status fgemm_run(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                       const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                       uint32_t beta, uint32_t* C, int64_t ldc, void* ws, size_t ws_bytes,
                       int* err, cudaStream_t s, int max_grid, bool untimed);
size_t fgemm_ws_bytes(int64_t m, int64_t n, int64_t k, uint32_t p, int sms);
size_t fgemm_ws_bytes_min(int64_t m, int64_t n, int64_t k, uint32_t p, int sms);  // without stream-K residues
// The tensor-core route alone (fgemm_run dispatches small products to the
// CUDA-core kernel of small_gemm.cu, everything else here).
ffgpu_status fgemm_run_rns(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                           const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                           uint32_t beta, uint32_t* C, int64_t ldc, void* ws, size_t ws_bytes,
                           int* err, cudaStream_t s, int max_grid, bool untimed);
// The tensor-core route with operands given as sums of blocks.
ffgpu_status fgemm_run_rns_src(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const SumSrc& A,
                               const SumSrc& B, uint32_t beta, uint32_t* C, int64_t ldc, void* ws, size_t ws_bytes,
                               int* err, cudaStream_t s, int max_grid, bool untimed);
// small contractions on the CUDA cores (small_gemm.cu)
bool fgemm_small(int64_t m, int64_t n, int64_t k);
void set_small_threshold(int64_t macs);
int64_t small_threshold();
size_t small_ws_bytes(int64_t m, int64_t n, int64_t k, int sms);
// one small product of a grouped CUDA-core launch (batched fgemm)
struct SmallJob {
    const uint32_t* A;
    const uint32_t* B;
    uint32_t* C;
    long long lda, ldb, ldc;
    unsigned long long mu;
    int m, n, k, tiles_n, tile0;
    uint32_t p, alpha, beta, two64p;
};
void small_job(SmallJob& J, const ffgpu_fgemm_desc& d, int tile0, int tile);
int64_t small_tiles(int64_t m, int64_t n, int tile);
cudaError_t launch_small_grouped(const SmallJob* jobs, const int* tile_job, int64_t tiles, int tile, cudaStream_t s);
// ws may be null (then no k-split); C may overlap A or B when the launch
// splits k (partial sums first) or when n <= 64 (each CTA reads only the rows
// it writes).
cudaError_t launch_small_gemm(int64_t m, int64_t n, int64_t k, const uint32_t* A, int64_t lda, const uint32_t* B,
                              int64_t ldb, uint32_t* C, int64_t ldc, uint32_t p, uint32_t alpha, uint32_t beta,
                              void* ws, size_t ws_bytes, int sms, cudaStream_t s);
ffgpu_status check_args(int64_t m, int64_t n, int64_t k, uint32_t p, const void* A, int64_t lda,
                        const void* B, int64_t ldb, const void* C, int64_t ldc);
int sm_count(int dev);

void make_plan(uint32_t p, int64_t k, RnsPlan& pl);
bool fgemm_single_pass(uint32_t p, int64_t k);
int chunk_steps_for(const RnsPlan& pl);
unsigned long long barrett_mu(uint32_t p);
void fill_inst(InstInfo& I, int64_t m, int64_t n, int64_t kp, const RnsPlan& pl, uint32_t al, uint32_t be,
               uint32_t* C, int64_t ldc);
bool encode_planes(CUtensorMap* map, void* base, uint64_t kp, uint64_t rows, uint64_t nch, uint32_t box_rows);

// paths and Winograd levels (winograd.cu)
ffgpu_status fgemm_ex_run(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const uint32_t* A,
                          int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta, uint32_t* C, int64_t ldc,
                          int path, int levels, cudaStream_t s);

// Winograd levels over Z, one reduction at the end (winograd_z.cu)
int64_t winograd_z_kmax(uint32_t p, int levels);
ffgpu_status winograd_z_run(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const uint32_t* A,
                            int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta, uint32_t* C, int64_t ldc,
                            int levels, cudaStream_t s);

// multi-modular products from one exact integer product (multimod.cu)
constexpr int kMaxFanoutPrimes = 64;
// Per prime of a fan-out: p, R = 2^32 mod p and the Shoup quotients
// floor(R 2^32 / p) and floor(2^32 / p), so that a 62-bit magnitude
// u = u_hi 2^32 + u_lo reduces as u_hi R + u_lo with 32-bit products.
struct FanPrime {
    uint32_t p, R, Rs, one_s;
};
struct FanoutParams {              // X mod p_i for every prime (passed by value)
    int nprimes;
    long long ldc;
    FanPrime pr[kMaxFanoutPrimes];
    uint32_t* C[kMaxFanoutPrimes];
    unsigned char vec_ok[kMaxFanoutPrimes];   // 16-byte stores legal
};
inline FanPrime fan_prime(uint32_t p) {
    FanPrime f;
    f.p = p;
    f.R = (uint32_t)((1ull << 32) % p);
    f.Rs = (uint32_t)(((unsigned long long)f.R << 32) / p);
    f.one_s = (uint32_t)((1ull << 32) / p);
    return f;
}
void fill_inst_int(InstInfo& I, int64_t m, int64_t n, int64_t kp, const RnsPlan& pl, long long* X, int64_t ldx);
ffgpu_status multimod_check(int64_t m, int64_t n, int64_t k, int bits, const void* A, int64_t lda, const void* B,
                            int64_t ldb, int nprimes, const uint32_t* primes, uint32_t* const* C, int64_t ldc);
size_t multimod_ws_bytes(int64_t m, int64_t n, int64_t k, int bits, int sms);
void fanout_params(int nprimes, const uint32_t* primes, uint32_t* const* C, int64_t ldc, FanoutParams& F);
cudaError_t launch_multimod_fanout(const long long* X, long long ldx, int m, int n, const FanoutParams& F,
                                   cudaStream_t s);
ffgpu_status multimod_run(int64_t m, int64_t n, int64_t k, int bits, const int32_t* A, int64_t lda, const int32_t* B,
                          int64_t ldb, int nprimes, const uint32_t* primes, uint32_t* const* C, int64_t ldc,
                          void* ws, size_t ws_bytes, int* err, cudaStream_t s);
uint32_t multimod_plan_modulus(int bits);
// one exact integer product into (or added to) an int64 array (multimod.cu)
size_t int_gemm_ws_bytes(int64_t m, int64_t n, int64_t k, int bits, int sms);
ffgpu_status int_gemm_run(int64_t m, int64_t n, int64_t k, int bits, const int32_t* A, int64_t lda,
                          const int32_t* B, int64_t ldb, long long* X, int64_t ldx, bool accumulate, void* ws,
                          size_t ws_bytes, int* err, cudaStream_t s);
// grouped fan-out over the instances of a batch (one wave)
struct FanInst {
    const long long* X;
    long long ldx, ldc;
    int m, n;
    int cbase;  // first of this instance's nprimes output pointers in the pointer table
    int pad;
};
struct FanPrimes {
    int nprimes;
    FanPrime pr[kMaxFanoutPrimes];
};
long long multimod_fanout_blocks(int m, int n);
cudaError_t launch_multimod_fanout_grouped(const FanInst* insts, const long long* block_begin, int n_inst,
                                           long long nblocks, uint32_t* const* cptrs, const FanPrimes& P,
                                           cudaStream_t s);
// an integer-mode batch: every instance's exact product, fanned out to the primes
struct MultiCtx {
    int bits;
    int nprimes;
    const uint32_t* primes;
    const ffgpu_multimod_desc* mdescs;
    const ffgpu_fgemm_desc* pseudo;  // the planner's view: p = the plan's modulus, C = the int64 result
};
ffgpu_status batched_multimod_run(int64_t count, const ffgpu_multimod_desc* d, int bits, int nprimes,
                                  const uint32_t* primes, cudaStream_t s);

// batched fgemm (batched.cu)
ffgpu_status batched_run(int64_t count, const ffgpu_fgemm_desc* d, cudaStream_t s);
ffgpu_status batched_run_ws(int64_t count, const ffgpu_fgemm_desc* d, void* ws, size_t ws_bytes, int* err,
                            cudaStream_t s);
size_t batched_ws_bytes(int64_t count, const ffgpu_fgemm_desc* d, int sms);
struct BatchedPlan;
ffgpu_status batched_plan_create(int64_t count, const ffgpu_fgemm_desc* d, BatchedPlan** out);
ffgpu_status batched_plan_run(BatchedPlan* plan, cudaStream_t s);
ffgpu_status batched_plan_error(BatchedPlan* plan);
void batched_plan_destroy(BatchedPlan* plan);
void batched_plan_info(const BatchedPlan* plan, int* waves, int* singles, size_t* nodes, size_t* device_bytes);

// ftrsm: the double cascade of Algorithms 2-3 (ftrsm_cascade.cu)
struct CascadeParams {
    int64_t t_del;     // rows of a leaf solved over Z with no reduction (eq. trsmboundcen, 63-bit carrier)
    int64_t t_update;  // products an entry may accumulate over Z between reductions (eq. 2, 63-bit carrier)
    int64_t t_split;   // floor(t_update / t_del) t_del: rows of one delayed block
};
CascadeParams cascade_params(uint32_t p);
size_t cascade_ws_bytes(int side, int64_t m, int64_t n, uint32_t p, int sms);
ffgpu_status cascade_run(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                         const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, void* ws, size_t ws_bytes,
                         int* err, cudaStream_t s);

// ftrsm (ftrsm.cu)
int ftrsm_algo(int algo);
size_t ftrsm_ws_bytes(int side, int uplo, int algo, int64_t m, int64_t n, uint32_t p, int sms);
ffgpu_status ftrsm_run(int side, int uplo, int diag, int algo, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                       const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, void* ws, size_t ws_bytes,
                       int* err, cudaStream_t s);

// Kernel timing (ffgpu_profile_*): brackets a launch with events on `s`.
bool profiling_on();
void profile_record(const char* name, cudaEvent_t start, cudaEvent_t stop);

// Set while this thread captures a launch sequence into a CUDA graph: launches
// are then recorded without the profiling events.
extern thread_local bool g_capturing;

template <class F>
cudaError_t timed_launch(const char* name, cudaStream_t s, F&& launch) {
    if (!profiling_on() || g_capturing) return launch();
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return cudaErrorUnknown;
    cudaEventRecord(a, s);
    const cudaError_t e = launch();
    cudaEventRecord(b, s);
    profile_record(name, a, b);
    return e;
}

}  // namespace ffgpu
