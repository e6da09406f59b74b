// Host side of libffgpu: the C ABI, argument checks, the plan (which moduli,
// how the inner dimension is split), per-stream workspace pools, TMA
// descriptors and the launch sequence.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace ffgpu {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------

static uint32_t inv_small(uint32_t a, uint32_t m) {
    // inverse of a mod m for m <= 256 (a coprime to m), by exhaustive search
    a %= m;
    for (uint32_t x = 1; x < m; ++x)
        if ((a * x) % m == 1) return x;
    return 0;
}

// Largest inner length that c channels can sum exactly: 4 * k * h^2 <= M with
// h = floor(p/2), the largest magnitude of a centred residue.  The factor 4
// keeps |sum| <= M/4, the margin the reconstruction's rounding step needs.
static u128 moduli_product(int c) {
    u128 M = 1;
    for (int i = 0; i < c; ++i) M *= kModuli[i];
    return M;
}

static int64_t k_capacity(uint32_t p, int c) {
    const u128 h = p / 2;
    const u128 cap = moduli_product(c) / (4 * h * h);
    return cap > (u128)INT64_MAX ? INT64_MAX : (int64_t)cap;
}

// Plan for one launch summing `k` products (computed by build_plan, cached
// per modulus: the channel count is the only part that depends on k).
static void build_plan(uint32_t p, int64_t k, RnsPlan& pl);

namespace {
struct PlanCacheEntry {
    int64_t cap[kMaxChannels + 1];  // cap[c]: largest k that c channels sum exactly
    RnsPlan plans[kMaxChannels + 1];
    bool have[kMaxChannels + 1];
};
std::mutex g_plan_mu;
std::map<uint32_t, PlanCacheEntry> g_plan_cache;
}  // namespace

// True when fgemm_run(..., k, ...) converts all of A and B before its product
// kernel writes C (a single k-slice): C may then overlap A or B.
bool fgemm_single_pass(uint32_t p, int64_t k) {
    RnsPlan pl;
    make_plan(p, std::max<int64_t>(k, 1), pl);
    return k <= pl.k_slice;
}

void make_plan(uint32_t p, int64_t k, RnsPlan& pl) {
    if (p <= kDirectMaxP) {
        build_plan(p, k, pl);
        return;
    }
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plan_cache.find(p);
    if (it == g_plan_cache.end()) {
        if (g_plan_cache.size() > 4096) g_plan_cache.clear();  // bounded
        PlanCacheEntry e;
        std::memset(&e, 0, sizeof(e));
        for (int c = 1; c <= kMaxChannels; ++c) e.cap[c] = k_capacity(p, c);
        it = g_plan_cache.emplace(p, e).first;
    }
    PlanCacheEntry& e = it->second;
    const int64_t ks = std::min<int64_t>(std::max<int64_t>(k, 1), e.cap[kMaxChannels]);
    int c = 1;
    while (c < kMaxChannels && e.cap[c] < ks) ++c;
    if (!e.have[c]) {
        build_plan(p, e.cap[c], e.plans[c]);  // k = cap[c] selects exactly c channels
        e.have[c] = true;
    }
    pl = e.plans[c];
}

static void build_plan(uint32_t p, int64_t k, RnsPlan& pl) {
    std::memset(&pl, 0, sizeof(pl));
    pl.p = p;
    if (p <= kDirectMaxP) {
        pl.mode = 1;
        pl.nch = 1;
        pl.mod[0] = p;
        pl.u[0] = 1;  // M = p: X = b_0 - q p, so the general reconstruction applies with
        pl.W[0] = 1;  // M/m_0 = 1 and M mod p = 0
        pl.negMp = 0;
        pl.k_slice = INT64_MAX;
        return;
    }
    pl.mode = 2;
    pl.k_slice = k_capacity(p, kMaxChannels);
    const int64_t ks = std::min<int64_t>(std::max<int64_t>(k, 1), pl.k_slice);
    int c = 1;
    while (c < kMaxChannels && k_capacity(p, c) < ks) ++c;
    pl.nch = c;
    const u128 M = moduli_product(c);
    for (int i = 0; i < c; ++i) {
        const uint32_t m = kModuli[i];
        const u128 Mi = M / m;
        pl.mod[i] = m;
        pl.u[i] = inv_small((uint32_t)(Mi % m), m);
        pl.W[i] = (uint32_t)(Mi % p);
    }
    pl.negMp = (uint32_t)((p - (uint32_t)(M % p)) % p);
}

unsigned long long barrett_mu(uint32_t p) { return ~0ull / p; }

// Longest chunk of k-steps (64 products each) the f32 accumulator can sum
// exactly: with R the largest residue magnitude, a reduced value |v| <= R + 1
// plus 64*steps products of magnitude <= R^2 must stay below 2^24 (eq. 1 with
// gamma = 24).  FFGPU_CHUNK_STEPS may ask for fewer (tuning).
int chunk_steps_for(const RnsPlan& pl) {
    uint32_t R = 0;
    for (int c = 0; c < pl.nch; ++c) R = std::max(R, pl.mod[c] / 2);
    const unsigned long long r2 = std::max<unsigned long long>(1ull, (unsigned long long)R * R);
    unsigned long long steps = ((1ull << 24) - R - 2) / r2 / 64;
    steps = std::min<unsigned long long>(std::max<unsigned long long>(steps, 1ull), 64ull);
    if (const char* e = std::getenv("FFGPU_CHUNK_STEPS")) {
        const long long want = std::atoll(e);
        if (want >= 1 && (unsigned long long)want < steps) steps = (unsigned long long)want;
    }
    if (g_tune_override.chunk_steps > 0 && (unsigned long long)g_tune_override.chunk_steps < steps)
        steps = (unsigned long long)g_tune_override.chunk_steps;
    return (int)steps;
}

// ---------------------------------------------------------------------------
// Kernel timing
// ---------------------------------------------------------------------------
struct ProfEntry {
    std::string name;
    cudaEvent_t start, stop;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfEntry> g_prof;

bool profiling_on() { return g_prof_on; }
thread_local bool g_capturing = false;

void profile_record(const char* name, cudaEvent_t start, cudaEvent_t stop) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(ProfEntry{name, start, stop});
}

// ---------------------------------------------------------------------------
// Devices, pools, descriptors
// ---------------------------------------------------------------------------

static std::mutex g_mu;
static std::map<std::pair<int, cudaStream_t>, Pool> g_pools;
static std::map<int, int> g_sms;

int sm_count(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sms.find(dev);
    if (it != g_sms.end()) return it->second;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    g_sms[dev] = v;
    return v;
}

// Pool of (current device, stream); allocates the error word on first use and
// grows the buffer to `need` bytes with stream-ordered allocation.
// Host-side fault injection for tests: while FFGPU_INJECT_ALLOC_FAIL is set to
// a non-empty value other than "0", every workspace growth fails as an
// allocation failure would (FFGPU_ERR_NOMEM, the stream's pool left empty), so
// the error path and the recovery after it can be exercised without a fault.
static bool inject_alloc_failure() {
    const char* e = std::getenv("FFGPU_INJECT_ALLOC_FAIL");
    return e && *e && std::strcmp(e, "0") != 0;
}

ffgpu_status pool_get(cudaStream_t s, size_t need, Pool** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    Pool& pl = g_pools[std::make_pair(dev, s)];
    if (!pl.err) {
        if (cudaMalloc(&pl.err, 256) != cudaSuccess) {
            pl.err = nullptr;
            return FFGPU_ERR_NOMEM;
        }
        if (cudaMemset(pl.err, 0, 256) != cudaSuccess) return FFGPU_ERR_CUDA;
    }
    if (need > pl.bytes) {
        if (pl.ptr) {
            cudaFreeAsync(pl.ptr, s);
            pl.ptr = nullptr;
            pl.bytes = 0;
        }
        const size_t want = (need + (size_t(1) << 21) - 1) & ~((size_t(1) << 21) - 1);
        if (inject_alloc_failure()) return FFGPU_ERR_NOMEM;
        if (cudaMallocAsync(&pl.ptr, want, s) != cudaSuccess) {
            cudaGetLastError();
            pl.ptr = nullptr;
            return FFGPU_ERR_NOMEM;
        }
        pl.bytes = want;
    }
    *out = &pl;
    return FFGPU_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D map over channel planes [nch][rows][kp] of bf16, box 64 x box_rows x 1,
// 128-byte swizzle (the layout the tensor-core descriptors expect).
bool encode_planes(CUtensorMap* map, void* base, uint64_t kp, uint64_t rows, uint64_t nch,
                          uint32_t box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {kp, rows, nch};
    cuuint64_t strides[2] = {kp * 2, rows * kp * 2};
    cuuint32_t box[3] = {64, box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t slots, planesA, planesB, total;
};

size_t slot_stride_for(int nch) { return size_t(nch) * kTileM * kTileN; }

static Layout layout_for(int64_t m, int64_t n, int64_t kp, int nch, int grid) {
    Layout L;
    L.slots = 0;
    L.planesA = align256(size_t(grid) * kSlotsPerCta * slot_stride_for(nch));
    L.planesB = L.planesA + align256(size_t(nch) * m * kp * 2);
    L.total = L.planesB + align256(size_t(nch) * n * kp * 2);
    return L;
}

static int64_t round64(int64_t x) { return (x + 63) / 64 * 64; }

static int grid_for_tiles(int64_t m, int64_t n, int dev_sms) {
    const int64_t tiles = ((m + kTileM - 1) / kTileM) * ((n + kTileN - 1) / kTileN);
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, dev_sms));
}

ffgpu_status check_args(int64_t m, int64_t n, int64_t k, uint32_t p, const void* A, int64_t lda,
                               const void* B, int64_t ldb, const void* C, int64_t ldc) {
    if (p < 2 || p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
    if (m < 0 || n < 0 || k < 0) return FFGPU_ERR_INVALID;
    if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > INT32_MAX / 2) return FFGPU_ERR_INVALID;
    if (m == 0 || n == 0) return FFGPU_OK;
    if (!C || ldc < n) return FFGPU_ERR_INVALID;
    if (k > 0 && (!A || !B || lda < k || ldb < n)) return FFGPU_ERR_INVALID;
    return FFGPU_OK;
}

// Kernel view of one instance (everything but the grouped-launch placement).
void fill_inst(InstInfo& I, int64_t m, int64_t n, int64_t kp, const RnsPlan& pl, uint32_t al, uint32_t be,
               uint32_t* C, int64_t ldc) {
    std::memset(&I, 0, sizeof(I));
    I.m = (int)m;
    I.n = (int)n;
    I.ksteps = (int)(kp / kTileK);
    I.chunk_steps = chunk_steps_for(pl);
    I.nch = pl.nch;
    I.direct = pl.mode == 1;
    I.vec_ok = ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && (ldc % 4 == 0);
    I.p = pl.p;
    I.alpha = al;
    I.beta = be;
    const unsigned long long p = pl.p;
    I.negMpa = (uint32_t)((unsigned long long)al * pl.negMp % p);
    I.R32 = (uint32_t)((1ull << 32) % p);
    I.R32s = (uint32_t)(((unsigned long long)I.R32 << 32) / p);
    I.one_s = (uint32_t)((1ull << 32) / p);
    I.beta_s = (uint32_t)(((unsigned long long)be << 32) / p);
    I.C = C;
    I.ldc = ldc;
    unsigned long long sumW = 0;
    uint32_t sumF = 0;
    for (int c = 0; c < pl.nch; ++c) {
        const uint32_t m = pl.mod[c];
        I.modf[c] = (float)m;
        I.inv_m[c] = 1.0f / (float)m;
        I.modu[c] = m;
        I.u[c] = pl.u[c];
        I.Wa[c] = (uint32_t)((unsigned long long)al * pl.W[c] % p);
        I.fr[c] = ((1u << 14) + m / 2) / m;
        sumW += I.Wa[c];
        sumF += I.fr[c];
    }
    // digits arrive as b_c + 128 (b_c balanced); the offsets, and the +6 that
    // keeps the quotient non-negative, are undone by these start values
    const unsigned long long neg = (128ull * (sumW % p) + 6ull * I.negMpa) % p;
    I.Kfix = (uint32_t)((p - neg) % p);
    I.Finit = 6u * (1u << 14) + (1u << 13) - 128u * sumF;
}

// Kernel choice: the CTA-pair kernel for problems with more than one 128-row
// block (and a grid of at least one pair); FFGPU_KERNEL=single|pair forces one.
bool use_pair_kernel(int64_t m, int grid) {
    if (g_tune_override.kernel == 0) return false;
    const char* f = std::getenv("FFGPU_KERNEL");
    if (f && std::strcmp(f, "single") == 0) return false;
    if (grid < 2 || rns_gemm_pair_max_clusters() < 1) return false;
    if (g_tune_override.kernel == 1) return true;
    if (f && std::strcmp(f, "pair") == 0) return true;
    return m > kTileM;
}

// Schedule of a CTA-pair launch: np pairs, tiles dealt round-robin, and a
// cut last wave (split > 1): when the last wave has rem tiles, at most half
// the pairs, each of them is cut into split = min(pairs / rem, ksteps /
// kMinPartSteps, 4) parts of its ksteps k-steps, so that that wave takes
// about ksteps / split k-steps instead of ksteps.
// A problem with fewer tiles than pairs is one such wave, on rem x split
// pairs.  An even channel count is required (the kernel's job pairs never
// mix two segments).  FFGPU_STREAMK=0 keeps the round-robin schedule.
struct PairSched {
    int np = 1;
    int dp = 0, split = 0, rem = 0;
};

static int64_t pair_tiles(int64_t m, int64_t n) {
    return ((m + 2 * kTileM - 1) / (2 * kTileM)) * ((n + kTileN - 1) / kTileN);
}

// k-steps of a part of a cut tile: one chunk (1024 products).  Shorter parts
// lose more than they gain: their heads' epilogues wait on the tails'
// residues in L2 for every channel with little tensor work to overlap it
// (1024^3 with four parts of 4 k-steps: 161 us against 87.5 round-robin).
constexpr int64_t kMinPartSteps = 16;

// T tiles, at most np_max pairs, ksteps k-steps per tile, nch channels; cut =
// false gives the round-robin schedule.
static PairSched pair_sched(int64_t T, int np_max, int64_t ksteps, int nch, bool cut) {
    PairSched s;
    np_max = std::max(1, np_max);
    s.np = (int)std::max<int64_t>(1, std::min<int64_t>(T, np_max));
    const char* e = std::getenv("FFGPU_STREAMK");
    if (!cut || (e && std::strcmp(e, "0") == 0) || np_max < 2 || ksteps < 2 * kMinPartSteps || (nch & 1)) return s;
    const int64_t rem = T < np_max ? T : T % np_max;
    if (rem == 0) return s;
    const int64_t split = std::min<int64_t>(std::min<int64_t>(np_max / rem, ksteps / kMinPartSteps), 4);
    if (split < 2) return s;
    if (T < np_max) s.np = (int)(T * split);
    s.dp = (int)(T - rem);
    s.split = (int)split;
    s.rem = (int)rem;
    return s;
}

// Pairs a launch may use: at most cap CTAs, and no more clusters than fit at once.
static int pair_limit(int cap) { return std::max(1, std::min(cap / 2, rns_gemm_pair_max_clusters())); }

// Bytes of the cut tiles' residues and flags for np pairs (one flag per
// pair, CTA, channel and epilogue warp).
static size_t sk_part_bytes(int np, int nch) { return size_t(np) * 2 * nch * kTileM * kTileN * sizeof(short); }
static size_t sk_flag_bytes(int np, int nch) { return size_t(np) * 2 * nch * kSkFlagsPerCta * sizeof(int); }

// Workspace of a launch: the layout (residue slots for max(grid, 2 np) CTAs,
// the planes), then the residues and flags of a cut last wave.
struct LaunchLayout {
    Layout L;
    size_t part_off = 0, flag_off = 0, total = 0;
};

static LaunchLayout launch_layout(int64_t m, int64_t n, int64_t kp, int nch, int grid, bool pair,
                                  const PairSched& ps) {
    LaunchLayout X;
    X.L = layout_for(m, n, kp, nch, pair ? std::max(grid, 2 * ps.np) : grid);
    X.total = X.L.total;
    if (pair && ps.split > 1) {
        X.part_off = align256(X.total);
        X.flag_off = X.part_off + align256(sk_part_bytes(ps.np, nch));
        X.total = X.flag_off + align256(sk_flag_bytes(ps.np, nch));
    }
    return X;
}

static size_t fgemm_ws_bytes_impl(int64_t m, int64_t n, int64_t k, uint32_t p, int sms, bool cut) {
    if (m == 0 || n == 0 || k == 0) return 0;
    RnsPlan pl;
    make_plan(p, k, pl);
    const int64_t ks = std::min<int64_t>(k, pl.k_slice), kp = round64(ks);
    const int grid = grid_for_tiles(m, n, sms);
    const bool pair = use_pair_kernel(m, grid);
    const PairSched ps = pair ? pair_sched(pair_tiles(m, n), pair_limit(sms), kp / kTileK, pl.nch, cut) : PairSched();
    const size_t rns = launch_layout(m, n, kp, pl.nch, grid, pair, ps).total;
    // a small product runs on the CUDA cores, its k-split partial sums in the workspace
    return fgemm_small(m, n, k) ? std::max(rns, small_ws_bytes(m, n, k, sms)) : rns;
}

// Workspace bytes for the largest launch of a problem (with the residues of a
// cut last wave where that schedule applies).
size_t fgemm_ws_bytes(int64_t m, int64_t n, int64_t k, uint32_t p, int sms) {
    return fgemm_ws_bytes_impl(m, n, k, p, sms, true);
}

// The same for the round-robin schedule: a launch whose workspace has no room
// for a cut last wave keeps that schedule.
size_t fgemm_ws_bytes_min(int64_t m, int64_t n, int64_t k, uint32_t p, int sms) {
    return fgemm_ws_bytes_impl(m, n, k, p, sms, false);
}

// The launch sequence: per slice of the inner dimension, convert A and B to
// channel planes and run the tensor-core kernel (beta applies to the first
// slice only; later slices accumulate with beta = 1).
ffgpu_status fgemm_run(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                       const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                       uint32_t beta, uint32_t* C, int64_t ldc, void* ws, size_t ws_bytes,
                       int* err, cudaStream_t s, int max_grid, bool untimed) {
    if (m > 0 && n > 0 && fgemm_small(m, n, k)) {
        int dev = 0;
        cudaGetDevice(&dev);
        const int sms = sm_count(dev);
        auto f = [&] { return launch_small_gemm(m, n, k, A, lda, B, ldb, C, ldc, p, alpha, beta, ws, ws_bytes, sms, s); };
        return (untimed ? f() : timed_launch("small_gemm", s, f)) == cudaSuccess ? FFGPU_OK : FFGPU_ERR_CUDA;
    }
    return fgemm_run_rns(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, ws, ws_bytes, err, s, max_grid, untimed);
}

static SumSrc single_src(const uint32_t* X, int64_t ld) {
    SumSrc S;
    std::memset(&S, 0, sizeof(S));
    S.X[0] = X;
    S.ld[0] = ld;
    S.n = 1;
    return S;
}

// The sum with every block shifted by (r rows, c columns).
static SumSrc shifted(const SumSrc& S, int64_t r, int64_t c) {
    SumSrc T = S;
    for (int t = 0; t < S.n; ++t) T.X[t] = S.X[t] + r * S.ld[t] + c;
    return T;
}

ffgpu_status fgemm_run_rns(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                           const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                           uint32_t beta, uint32_t* C, int64_t ldc, void* ws, size_t ws_bytes,
                           int* err, cudaStream_t s, int max_grid, bool untimed) {
    return fgemm_run_rns_src(m, n, k, p, alpha, single_src(A, lda), single_src(B, ldb), beta, C, ldc, ws, ws_bytes,
                             err, s, max_grid, untimed);
}

ffgpu_status fgemm_run_rns_src(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const SumSrc& A,
                               const SumSrc& B, uint32_t beta, uint32_t* C, int64_t ldc, void* ws, size_t ws_bytes,
                               int* err, cudaStream_t s, int max_grid, bool untimed) {
    const unsigned long long mu = barrett_mu(p);
    auto launch = [&](const char* name, auto&& f) { return untimed ? f() : timed_launch(name, s, f); };
    const uint32_t al = alpha % p;
    uint32_t be = beta % p;
    if (k == 0)
        return launch("scale_mod_p", [&] { return launch_scale(C, ldc, (int)m, (int)n, p, be, mu, s); }) ==
                       cudaSuccess
                   ? FFGPU_OK
                   : FFGPU_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    int grid = grid_for_tiles(m, n, sm_count(dev));
    if (max_grid > 0 && grid > max_grid) grid = max_grid;
    RnsPlan pl0;
    make_plan(p, k, pl0);
    const int64_t kslice = std::min<int64_t>(k, pl0.k_slice);
    for (int64_t k0 = 0; k0 < k; k0 += kslice) {
        const int64_t ks = std::min<int64_t>(kslice, k - k0);
        RnsPlan pl;
        make_plan(p, ks, pl);
        const int64_t kp = round64(ks);
        // CTA-pair kernel (256 x 256 tiles) unless the problem has a single row
        // block or the caller forces the one-CTA kernel; its schedule sets the
        // number of residue slots, so it is chosen before the layout
        const bool pair = use_pair_kernel(m, grid);
        const int64_t ksteps = kp / kTileK;
        const int cap = max_grid > 0 ? std::min(sm_count(dev), max_grid) : sm_count(dev);
        PairSched ps = pair ? pair_sched(pair_tiles(m, n), pair_limit(cap), ksteps, pl.nch, true) : PairSched();
        LaunchLayout X = launch_layout(m, n, kp, pl.nch, grid, pair, ps);
        if (X.total > ws_bytes && ps.split > 1) {  // no room for a cut last wave: round-robin
            ps = pair_sched(pair_tiles(m, n), pair_limit(cap), ksteps, pl.nch, false);
            X = launch_layout(m, n, kp, pl.nch, grid, pair, ps);
        }
        if (X.total > ws_bytes) return FFGPU_ERR_NOMEM;
        const Layout& L = X.L;
        unsigned char* wsb = static_cast<unsigned char*>(ws);

        ConvertParams cp;
        std::memset(&cp, 0, sizeof(cp));
        cp.p = p;
        cp.half_p = p / 2;
        cp.mu32 = 0xFFFFFFFFu / cp.p;
        cp.nch = pl.nch;
        cp.direct = pl.mode == 1;
        for (int c = 0; c < pl.nch; ++c) {
            cp.mod[c] = pl.mod[c];
            cp.magic32[c] = (uint32_t)(((1ull << 39) + pl.mod[c] - 1) / pl.mod[c]);
        }
        // one term: the caller's matrix; several: Winograd's pre-additions,
        // summed mod p inside the conversion
        if (A.n == 1) {
            if (launch("convert_rows", [&] {
                    return launch_convert_rows(A.X[0] + k0, A.ld[0], (int)m, (int)ks, (int)kp, cp, wsb + L.planesA, s);
                }) != cudaSuccess)
                return FFGPU_ERR_CUDA;
        } else if (launch("convert_rows_sum", [&] {
                       return launch_convert_rows_sum(shifted(A, 0, k0), (int)m, (int)ks, (int)kp, cp,
                                                      wsb + L.planesA, s);
                   }) != cudaSuccess) {
            return FFGPU_ERR_CUDA;
        }
        if (B.n == 1) {
            if (launch("convert_transpose", [&] {
                    return launch_convert_transpose(B.X[0] + k0 * B.ld[0], B.ld[0], (int)ks, (int)n, (int)kp, cp,
                                                    wsb + L.planesB, s);
                }) != cudaSuccess)
                return FFGPU_ERR_CUDA;
        } else if (launch("convert_transpose_sum", [&] {
                       return launch_convert_transpose_sum(shifted(B, k0, 0), (int)ks, (int)n, (int)kp, cp,
                                                           wsb + L.planesB, s);
                   }) != cudaSuccess) {
            return FFGPU_ERR_CUDA;
        }

        CUtensorMap mapA, mapB;
        if (!encode_planes(&mapA, wsb + L.planesA, kp, m, pl.nch, kTileM) ||
            !encode_planes(&mapB, wsb + L.planesB, kp, n, pl.nch, pair ? 128 : kTileN))
            return FFGPU_ERR_CUDA;

        RnsGemmParams P;
        std::memset(&P, 0, sizeof(P));
        fill_inst(P.inst, m, n, kp, pl, al, be, C, ldc);
        const int tile_rows = pair ? 2 * kTileM : kTileM;
        P.tiles_m = (int)((m + tile_rows - 1) / tile_rows);
        P.tiles_n = (int)((n + kTileN - 1) / kTileN);
        P.num_tiles = P.tiles_m * P.tiles_n;
        P.slots = wsb + L.slots;
        P.slot_stride = slot_stride_for(pl.nch);
        P.err = err;
        P.raster = g_tune_override.raster > 0 ? g_tune_override.raster : kRasterRows;
        if (pair) {
            if (ps.split > 1) {
                P.sk_dp = ps.dp;
                P.sk_split = ps.split;
                P.sk_rem = ps.rem;
                P.sk_part = reinterpret_cast<short*>(wsb + X.part_off);
                P.sk_flags = reinterpret_cast<int*>(wsb + X.flag_off);
                if (cudaMemsetAsync(P.sk_flags, 0, sk_flag_bytes(ps.np, pl.nch), s) != cudaSuccess)
                    return FFGPU_ERR_CUDA;
            }
            const int np = ps.np;
            if (launch("rns_gemm_pair", [&] { return launch_rns_gemm_pair(mapA, mapB, P, 2 * np, s); }) != cudaSuccess)
                return FFGPU_ERR_CUDA;
        } else if (launch("rns_gemm", [&] { return launch_rns_gemm(mapA, mapB, P, grid, s); }) != cudaSuccess) {
            return FFGPU_ERR_CUDA;
        }
        be = 1;  // later slices accumulate onto the partial result
    }
    return FFGPU_OK;
}

}  // namespace ffgpu

using namespace ffgpu;

extern "C" {

const char* ffgpu_status_string(ffgpu_status s) {
    switch (s) {
        case FFGPU_OK: return "FFGPU_OK";
        case FFGPU_ERR_INVALID: return "FFGPU_ERR_INVALID";
        case FFGPU_ERR_UNSUPPORTED_P: return "FFGPU_ERR_UNSUPPORTED_P";
        case FFGPU_ERR_NOMEM: return "FFGPU_ERR_NOMEM";
        case FFGPU_ERR_CUDA: return "FFGPU_ERR_CUDA";
        case FFGPU_ERR_TIMEOUT: return "FFGPU_ERR_TIMEOUT";
        case FFGPU_ERR_BUDGET: return "FFGPU_ERR_BUDGET";
        case FFGPU_ERR_SINGULAR: return "FFGPU_ERR_SINGULAR";
    }
    return "FFGPU_UNKNOWN_STATUS";
}

int ffgpu_version(void) { return 100; }

ffgpu_status ffgpu_set_small_threshold(int64_t max_macs) {
    if (max_macs < 0) return FFGPU_ERR_INVALID;
    set_small_threshold(max_macs);
    return FFGPU_OK;
}

int64_t ffgpu_get_small_threshold(void) { return small_threshold(); }

ffgpu_status ffgpu_fgemm_workspace_size(int64_t m, int64_t n, int64_t k, uint32_t p, size_t* bytes) {
    if (!bytes) return FFGPU_ERR_INVALID;
    const ffgpu_status st = check_args(m, n, k, p, (const void*)1, std::max<int64_t>(k, 1), (const void*)1,
                                       std::max<int64_t>(n, 1), (const void*)1, std::max<int64_t>(n, 1));
    if (st != FFGPU_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        *bytes = fgemm_ws_bytes(m, n, k, p, 256);
        return FFGPU_OK;
    }
    *bytes = fgemm_ws_bytes(m, n, k, p, sm_count(dev));
    return FFGPU_OK;
}

ffgpu_status ffgpu_fgemm_plan(int64_t m, int64_t n, int64_t k, uint32_t p, ffgpu_plan_info* out) {
    if (!out) return FFGPU_ERR_INVALID;
    if (p < 2 || p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
    if (m < 0 || n < 0 || k < 0) return FFGPU_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    RnsPlan pl;
    make_plan(p, std::max<int64_t>(k, 1), pl);
    const int64_t ks = std::min<int64_t>(std::max<int64_t>(k, 1), pl.k_slice);
    out->mode = pl.mode;
    out->channels = pl.nch;
    for (int c = 0; c < pl.nch; ++c) out->moduli[c] = pl.mod[c];
    out->k_chunk = chunk_steps_for(pl) * kTileK;
    out->k_slices = (int32_t)((std::max<int64_t>(k, 1) + ks - 1) / ks);
    out->tile_m = kTileM;
    out->tile_n = kTileN;
    out->tile_k = kTileK;
    out->mma_flops = 2.0 * (double)m * (double)n * (double)round64(k) * (double)pl.nch;
    return FFGPU_OK;
}

ffgpu_status ffgpu_fgemm_ws(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                            const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                            uint32_t beta, uint32_t* C, int64_t ldc, void* workspace,
                            size_t workspace_bytes, void* stream) {
    ffgpu_status st = check_args(m, n, k, p, A, lda, B, ldb, C, ldc);
    if (st != FFGPU_OK || m == 0 || n == 0) return st;
    // a cached plan's kernel, chunk, route and tile order (its Winograd depth
    // needs workspace beyond the caller's and is not applied here)
    TuneOverride tuned;
    int levels = 0;
    bool have = k > 0 && autotune_settings(m, n, k, p, tuned, levels);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Pool* pool = nullptr;
    st = pool_get(s, 0, &pool);
    if (st != FFGPU_OK) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    if (have) {  // a plan whose route needs more than the workspace sized by the default rules is not used
        ScopedTune probe(tuned);
        have = workspace_bytes >= fgemm_ws_bytes(m, n, k, p, sm_count(dev));
    }
    ScopedTune scope(have ? tuned : g_tune_override);
    if (workspace_bytes < fgemm_ws_bytes(m, n, k, p, sm_count(dev))) return FFGPU_ERR_NOMEM;
    if (workspace_bytes && (reinterpret_cast<uintptr_t>(workspace) & 255)) return FFGPU_ERR_INVALID;
    return fgemm_run(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, workspace, workspace_bytes,
                     pool->err, s, 0, false);
}

ffgpu_status ffgpu_fgemm(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha,
                         const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta,
                         uint32_t* C, int64_t ldc, void* stream) {
    ffgpu_status st = check_args(m, n, k, p, A, lda, B, ldb, C, ldc);
    if (st != FFGPU_OK || m == 0 || n == 0) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the plan cache (filled by ffgpu_autotune or ffgpu_autotune_load): its
    // kernel, chunk, route, tile order and Winograd depth for this shape
    // bucket and modulus, when it holds one
    TuneOverride tuned;
    int levels = 0;
    const bool have = k > 0 && autotune_settings(m, n, k, p, tuned, levels);
    ScopedTune scope(have ? tuned : g_tune_override);
    if (have && levels > 0) return fgemm_ex_run(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, 0, levels, s);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    const size_t need = fgemm_ws_bytes(m, n, k, p, sm_count(dev));
    Pool* pool = nullptr;
    st = pool_get(s, need, &pool);
    if (st != FFGPU_OK) return st;
    return fgemm_run(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, pool->ptr, pool->bytes, pool->err,
                     s, 0, false);
}

ffgpu_status ffgpu_fgemm_ex(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const uint32_t* A,
                            int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta, uint32_t* C, int64_t ldc,
                            const ffgpu_options* opt, void* stream) {
    ffgpu_status st = check_args(m, n, k, p, A, lda, B, ldb, C, ldc);
    if (st != FFGPU_OK || m == 0 || n == 0) return st;
    const int path = opt ? opt->path : 0, levels = opt ? opt->winograd_levels : 0;
    if (opt) {
        for (int i = 0; i < 5; ++i)
            if (opt->reserved[i] != 0) return FFGPU_ERR_INVALID;
        if (opt->unreduced != 0 && opt->unreduced != 1) return FFGPU_ERR_INVALID;
        if (opt->unreduced)
            return winograd_z_run(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, levels,
                                  static_cast<cudaStream_t>(stream));
    }
    if (path == 0 && levels == 0)
        return ffgpu_fgemm(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, stream);
    return fgemm_ex_run(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, path, levels,
                        static_cast<cudaStream_t>(stream));
}

ffgpu_status ffgpu_fgemm_batched(int64_t count, const ffgpu_fgemm_desc* descs, void* stream) {
    if (count < 0 || (count > 0 && !descs)) return FFGPU_ERR_INVALID;
    for (int64_t i = 0; i < count; ++i) {
        const ffgpu_fgemm_desc& d = descs[i];
        const ffgpu_status st = check_args(d.m, d.n, d.k, d.p, d.A, d.lda, d.B, d.ldb, d.C, d.ldc);
        if (st != FFGPU_OK) return st;
    }
    if (count == 0) return FFGPU_OK;
    return batched_run(count, descs, static_cast<cudaStream_t>(stream));
}

ffgpu_status ffgpu_ftrsm_ex(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                            const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, int algorithm, void* stream) {
    if (p < 2 || p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
    if (side < 0 || side > 1 || uplo < 0 || uplo > 1 || diag < 0 || diag > 1) return FFGPU_ERR_INVALID;
    if (algorithm != FFGPU_TRSM_DEFAULT && algorithm != FFGPU_TRSM_RECURSIVE && algorithm != FFGPU_TRSM_DELAYED &&
        algorithm != FFGPU_TRSM_CASCADE)
        return FFGPU_ERR_INVALID;
    if (m < 0 || n < 0 || m > INT32_MAX / 2 || n > INT32_MAX / 2) return FFGPU_ERR_INVALID;
    if (m == 0 || n == 0) return FFGPU_OK;
    const int64_t nt = side == 0 ? m : n;
    if (!T || !B || ldt < nt || ldb < n) return FFGPU_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    Pool* pool = nullptr;
    ffgpu_status st = pool_get(s, ftrsm_ws_bytes(side, uplo, algorithm, m, n, p, sm_count(dev)), &pool);
    if (st != FFGPU_OK) return st;
    return ftrsm_run(side, uplo, diag, algorithm, m, n, p, alpha, T, ldt, B, ldb, pool->ptr, pool->bytes, pool->err,
                     s);
}

ffgpu_status ffgpu_ftrsm(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                         const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, void* stream) {
    return ffgpu_ftrsm_ex(side, uplo, diag, m, n, p, alpha, T, ldt, B, ldb, FFGPU_TRSM_DEFAULT, stream);
}

ffgpu_status ffgpu_fgemm_batched_plan_create(int64_t count, const ffgpu_fgemm_desc* descs,
                                             ffgpu_batched_plan** plan) {
    if (!plan || count < 0 || (count > 0 && !descs)) return FFGPU_ERR_INVALID;
    for (int64_t i = 0; i < count; ++i) {
        const ffgpu_fgemm_desc& d = descs[i];
        if (d.p < 2 || d.p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
        const ffgpu_status st = check_args(d.m, d.n, d.k, d.p, d.A, d.lda, d.B, d.ldb, d.C, d.ldc);
        if (st != FFGPU_OK) return st;
    }
    BatchedPlan* p = nullptr;
    const ffgpu_status st = batched_plan_create(count, descs, &p);
    *plan = reinterpret_cast<ffgpu_batched_plan*>(p);
    return st;
}

ffgpu_status ffgpu_fgemm_batched_plan_run(ffgpu_batched_plan* plan, void* stream) {
    if (!plan) return FFGPU_ERR_INVALID;
    return batched_plan_run(reinterpret_cast<BatchedPlan*>(plan), static_cast<cudaStream_t>(stream));
}

ffgpu_status ffgpu_fgemm_batched_plan_error(ffgpu_batched_plan* plan) {
    if (!plan) return FFGPU_ERR_INVALID;
    return batched_plan_error(reinterpret_cast<BatchedPlan*>(plan));
}

ffgpu_status ffgpu_fgemm_batched_plan_info(const ffgpu_batched_plan* plan, int* waves, int* singles,
                                           size_t* graph_nodes, size_t* device_bytes) {
    if (!plan) return FFGPU_ERR_INVALID;
    batched_plan_info(reinterpret_cast<const BatchedPlan*>(plan), waves, singles, graph_nodes, device_bytes);
    return FFGPU_OK;
}

ffgpu_status ffgpu_fgemm_batched_plan_destroy(ffgpu_batched_plan* plan) {
    batched_plan_destroy(reinterpret_cast<BatchedPlan*>(plan));
    return FFGPU_OK;
}

ffgpu_status ffgpu_fgemm_multimod(int64_t m, int64_t n, int64_t k, int bits, const int32_t* A, int64_t lda,
                                  const int32_t* B, int64_t ldb, int nprimes, const uint32_t* primes,
                                  uint32_t* const* C, int64_t ldc, void* stream) {
    ffgpu_status st = multimod_check(m, n, k, bits, A, lda, B, ldb, nprimes, primes, C, ldc);
    if (st != FFGPU_OK || m == 0 || n == 0) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    Pool* pool = nullptr;
    st = pool_get(s, multimod_ws_bytes(m, n, k, bits, sm_count(dev)), &pool);
    if (st != FFGPU_OK) return st;
    return multimod_run(m, n, k, bits, A, lda, B, ldb, nprimes, primes, C, ldc, pool->ptr, pool->bytes, pool->err, s);
}

ffgpu_status ffgpu_fgemm_multimod_batched(int64_t count, const ffgpu_multimod_desc* descs, int bits, int nprimes,
                                          const uint32_t* primes, void* stream) {
    if (count < 0 || (count > 0 && !descs)) return FFGPU_ERR_INVALID;
    for (int64_t i = 0; i < count; ++i) {
        const ffgpu_multimod_desc& d = descs[i];
        const ffgpu_status st =
            multimod_check(d.m, d.n, d.k, bits, d.A, d.lda, d.B, d.ldb, nprimes, primes, d.C, d.ldc);
        if (st != FFGPU_OK) return st;
    }
    if (count == 0) return FFGPU_OK;
    return batched_multimod_run(count, descs, bits, nprimes, primes, static_cast<cudaStream_t>(stream));
}

ffgpu_status ffgpu_last_device_error(void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    int* err = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_pools.find(std::make_pair(dev, s));
        if (it == g_pools.end() || !it->second.err) return FFGPU_OK;
        err = it->second.err;
    }
    int v = 0;
    if (cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FFGPU_ERR_CUDA;
    if (v != 0) {
        cudaMemset(err, 0, sizeof(int));
        return v == kDevSingular ? FFGPU_ERR_INVALID : FFGPU_ERR_TIMEOUT;
    }
    return FFGPU_OK;
}

ffgpu_status ffgpu_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return FFGPU_OK;
}

ffgpu_status ffgpu_profile_read(ffgpu_kernel_time* out, int cap, int* count) {
    if (cap < 0 || (cap > 0 && !out) || !count) return FFGPU_ERR_INVALID;
    std::vector<ProfEntry> entries;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        entries.swap(g_prof);
    }
    std::map<std::string, std::pair<int64_t, double>> acc;
    ffgpu_status st = FFGPU_OK;
    for (auto& e : entries) {
        float ms = 0.f;
        if (cudaEventSynchronize(e.stop) != cudaSuccess || cudaEventElapsedTime(&ms, e.start, e.stop) != cudaSuccess) {
            cudaGetLastError();
            st = FFGPU_ERR_CUDA;
        }
        auto& a = acc[e.name];
        a.first += 1;
        a.second += ms;
        cudaEventDestroy(e.start);
        cudaEventDestroy(e.stop);
    }
    int i = 0;
    for (auto& kv : acc) {
        if (i < cap) {
            std::memset(&out[i], 0, sizeof(out[i]));
            std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.first;
            out[i].total_ms = kv.second.second;
        }
        ++i;
    }
    *count = i;
    return st;
}

ffgpu_status ffgpu_release_workspaces(void) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_pools) {
        if (kv.second.ptr) cudaFree(kv.second.ptr);
        if (kv.second.err) cudaFree(kv.second.err);
    }
    g_pools.clear();
    return FFGPU_OK;
}

}  // extern "C"
