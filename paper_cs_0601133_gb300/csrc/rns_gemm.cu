// Tensor-core product over a residue number system, with the reduction mod p
// fused into the epilogue.
//
// What it computes (section 3, C <- alpha*A*B + beta*C over Z/pZ): A and B
// arrive as "channel planes": for each small modulus m_c (<= 256) the
// balanced residues of the centred inputs, stored as bf16 (exact, |r| <= 128).
// For every 128 x 256 output tile and every channel c the kernel forms
// S_c = sum_t A_c[i][t] * B_c[j][t] on the tcgen05 tensor cores with an f32
// accumulator in tensor memory.  This is the delayed reduction of section
// 2.1.2 restated for the accumulator: products of balanced residues are at
// most 127^2 in magnitude, so 1024 of them plus a reduced value (|v| <= 128)
// stay below 2^24, where every f32 sum of integers is exact (eq. 1 with
// gamma = 24).  After each chunk of that length the epilogue warps reduce the
// accumulator mod m_c in place (tcgen05.ld -> fma -> tcgen05.st) and the MMAs
// continue on top of it.
// After the last chunk each channel yields S mod m_c; the last channel of a
// tile triggers the reconstruction of S mod p from all residues (Chinese
// remainder theorem, the multi-modular route to p > 2^26 the paper lists as
// future work in section 7), then C = (alpha*S + beta*C) mod p.
//
// Roles (one CTA per SM, persistent over tiles):
//   warp 0      TMA producer: channel tiles of A (128x64) and B (256x64), 4 stages
//   warp 1      TMEM allocator and single-thread MMA issuer (M=128, N=256, K=16)
//   warps 2..9  epilogue: lane quarter (warp % 4) x column half ((warp-2) / 4)
// Two 256-column accumulators: the jobs (tile, channel) of a CTA are paired and
// their chunks interleaved, so one accumulator is reduced while the tensor
// cores fill the other.
//
// Two schedulers share the kernel body: one instance with tiles dealt
// round-robin to the persistent CTAs, and a grouped launch where the host lists
// each CTA's jobs (instance, tile, channel) over many instances of different
// shapes and moduli (section 8 of the build's scope: one launch for a batch).
#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kThreads = 448;   // 2 control warps, 8 epilogue warps, 4 combine warps
constexpr int kEpiWarps = 8;
constexpr int kFirstCombineWarp = 10;
constexpr uint32_t kABytes = kTileM * kTileK * 2;
constexpr uint32_t kBBytes = kTileN * kTileK * 2;
constexpr uint32_t kStageBytes = kABytes + kBBytes;
constexpr uint32_t kTmemCols = 512;
constexpr int kGroupM = 16;  // tile rasterisation: bands of 16 tile rows
// reconstruction tables of the combine warps (see combine_block): per channel
// and residue value, b*(M/m_c) mod p and b/m_c
constexpr size_t kTabBytes = size_t(kMaxChannels) * 256 * 8;
constexpr size_t kSmemBytes = 1024 + size_t(kStages) * kStageBytes + kTabBytes + 256;

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
    const int per_group = kGroupM * tiles_n;
    const int g = t / per_group;
    const int first = g * kGroupM;
    const int gm = min(tiles_m - first, kGroupM);
    const int r = t - g * per_group;
    tm = first + r % gm;
    tn = r / gm;
}

// Wait that ignores the abort flag (used to drain in-flight asynchronous work
// before the CTA releases shared and tensor memory); still bounded in time.
__device__ __forceinline__ void mbar_drain_wait(uint64_t* bar, uint32_t parity, int* err) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitLimitCycles) {
            atomicCAS(err, 0, (int)kDevTimeoutDrain);
            return;
        }
    }
}

// Exact residue in [0, m) of an f32 holding an integer of magnitude < 2^24.
__device__ __forceinline__ uint32_t f32_residue(float x, float m, float inv_m, int mi) {
    const float q = rintf(x * inv_m);
    int r = (int)fmaf(-q, m, x);
    if (r < 0) r += mi;
    if (r >= mi) r -= mi;
    return (uint32_t)r;
}

// Reconstruction of X mod p from the residues r_c of the channels, and the C
// update, for the 128 x 256 block of one CTA.  With M = prod m_c and
// b_c = r_c * (M/m_c)^{-1} mod m_c, X = sum_c b_c (M/m_c) - q M where
// q = round(sum_c b_c / m_c), valid because the plan guarantees |X| <= M/4 (the
// fraction is within 1/4 of an integer, far above f32 error); then X mod p =
// (sum_c b_c (M/m_c mod p) + q (p - M mod p)) mod p in 64-bit integers.
// b_c depends on r_c only, so for every channel the combine warps tabulate,
// for each of the 256 residue values, tabW = b_c (M/m_c mod p) mod p and
// tabF = b_c / m_c in shared memory (rebuilt when the tile's instance
// changes); an output then costs two table reads and two additions per
// channel.  Done by one of the kCombineWarps combine warps: warp cw takes rows
// [32 cw, 32 cw + 32); the lanes of a warp cover 128 consecutive columns (4
// each), so the residue loads (128 B per channel) and the C accesses (512 B)
// are coalesced; a thread handles kCombineRows x 4 outputs at a time.
constexpr int kCombineWarps = 4;
constexpr int kCombineRows = 4;

struct CombTables {
    uint32_t w[kMaxChannels][256];
    float f[kMaxChannels][256];
};

// Builds the tables of instance I (all combine warps, then a barrier among them).
__device__ __forceinline__ void build_tables(const InstInfo& I, CombTables* T, int tid) {
    asm volatile("bar.sync 1, %0;" ::"r"(kCombineWarps * 32) : "memory");
    if (!I.direct) {
        for (int idx = tid; idx < I.nch * 256; idx += kCombineWarps * 32) {
            const int c = idx >> 8, r = idx & 255;
            const uint32_t m = I.modu[c];
            if ((uint32_t)r < m) {
                const uint32_t b = (uint32_t)((r * I.u[c]) % m);
                T->w[c][r] = mod_u64((unsigned long long)b * I.W[c], I.p, I.mu);
                T->f[c][r] = (float)b / (float)m;
            }
        }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kCombineWarps * 32) : "memory");
}

__device__ __forceinline__ void combine_block(const InstInfo& I, const CombTables* T, int row0, int col0,
                                              const unsigned char* slot, size_t chan_stride, int cw, int lane) {
    const int nch = I.nch, m = I.m, n = I.n;
    const uint32_t p = I.p, negMp = I.negMp, alpha = I.alpha, beta = I.beta;
    const unsigned long long mu = I.mu;
    const bool direct = I.direct != 0, vec_ok = I.vec_ok != 0;
    uint32_t* const C = I.C;
    const long long ldc = I.ldc;
#pragma unroll 1
    for (int rg = cw * 32; rg < cw * 32 + 32; rg += kCombineRows) {
        if (row0 + rg >= m) break;
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            const int lc = pass * 128 + 4 * lane;
            const int col = col0 + lc;
            if (col >= n) continue;
            const bool full4 = col + 3 < n;
            const unsigned char* src = slot + size_t(rg) * kTileN + lc;
            uint32_t old[kCombineRows][4];
            unsigned long long S[kCombineRows][4];
            float G[kCombineRows][4];
#pragma unroll
            for (int rr = 0; rr < kCombineRows; ++rr) {
                const bool rok = row0 + rg + rr < m;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    old[rr][e] = 0u;
                    S[rr][e] = 0ull;
                    G[rr][e] = 0.f;
                }
                if (rok && beta != 0) {
                    const uint32_t* crow = C + (long long)(row0 + rg + rr) * ldc;
                    if (full4 && vec_ok) {
                        const uint4 v = *reinterpret_cast<const uint4*>(crow + col);
                        old[rr][0] = v.x; old[rr][1] = v.y; old[rr][2] = v.z; old[rr][3] = v.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (col + e < n) old[rr][e] = crow[col + e];
                    }
                }
            }
            if (direct) {
#pragma unroll
                for (int rr = 0; rr < kCombineRows; ++rr) {
                    const uint32_t w = *reinterpret_cast<const uint32_t*>(src + size_t(rr) * kTileN);
#pragma unroll
                    for (int e = 0; e < 4; ++e) S[rr][e] = (w >> (8 * e)) & 255u;
                }
            } else {
#pragma unroll 1
                for (int c = 0; c < nch; ++c) {
                    uint32_t w[kCombineRows];
#pragma unroll
                    for (int rr = 0; rr < kCombineRows; ++rr)
                        w[rr] = *reinterpret_cast<const uint32_t*>(src + size_t(c) * chan_stride + size_t(rr) * kTileN);
                    const uint32_t* tw = T->w[c];
                    const float* tf = T->f[c];
#pragma unroll
                    for (int rr = 0; rr < kCombineRows; ++rr)
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const uint32_t r = (w[rr] >> (8 * e)) & 255u;
                            S[rr][e] += tw[r];
                            G[rr][e] += tf[r];
                        }
                }
            }
#pragma unroll 1
            for (int rr = 0; rr < kCombineRows; ++rr) {
                const int row = row0 + rg + rr;
                if (row >= m) continue;
                uint32_t out[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t X;
                    if (direct) {
                        X = (uint32_t)S[rr][e];
                    } else {
                        const unsigned long long q = (unsigned long long)rintf(G[rr][e]);
                        X = mod_u64(S[rr][e] + q * negMp, p, mu);
                    }
                    out[e] = mod_u64((unsigned long long)alpha * X + (unsigned long long)beta * old[rr][e], p, mu);
                }
                uint32_t* crow = C + (long long)row * ldc;
                if (full4 && vec_ok) {
                    *reinterpret_cast<uint4*>(crow + col) = make_uint4(out[0], out[1], out[2], out[3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (col + e < n) crow[col + e] = out[e];
                }
            }
        }
    }
}

// A job of the kernel: one channel of one output tile of one instance.
struct Job {
    const InstInfo* inst;
    const CUtensorMap* mapA;
    const CUtensorMap* mapB;
    int tm, tn, c;
    int H;        // chunks of kChunkSteps k-steps
    int slot;     // residue slot of the job's tile
};

// Single instance, tiles dealt round-robin to the CTAs, channels in order.
struct SingleSched {
    const RnsGemmParams& P;
    const CUtensorMap* mA;
    const CUtensorMap* mB;
    int my_tiles;
    __device__ SingleSched(const RnsGemmParams& p, const CUtensorMap* a, const CUtensorMap* b)
        : P(p), mA(a), mB(b) {
        my_tiles = (int)blockIdx.x < P.num_tiles
                       ? (P.num_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                       : 0;
    }
    __device__ int num_jobs() const { return my_tiles * P.inst.nch; }
    __device__ void job(int j, Job& d) const {
        const int nch = P.inst.nch;
        const int t = (int)blockIdx.x + (j / nch) * (int)gridDim.x;
        d.inst = &P.inst;
        d.mapA = mA;
        d.mapB = mB;
        d.c = j % nch;
        tile_coords(t, P.tiles_m, P.tiles_n, d.tm, d.tn);
        d.H = (P.inst.ksteps + P.inst.chunk_steps - 1) / P.inst.chunk_steps;
        d.slot = (j / nch) & 1;  // tiles alternate the two residue slots
    }
    __device__ unsigned char* slots() const { return P.slots; }
    __device__ size_t slot_stride() const { return P.slot_stride; }
    __device__ int* err() const { return P.err; }
};

// Grouped launch: the host lists every CTA's jobs.
struct GroupSched {
    const GroupGemmParams& P;
    int begin, count;
    __device__ GroupSched(const GroupGemmParams& p, const CUtensorMap*, const CUtensorMap*) : P(p) {
        begin = P.cta_begin[blockIdx.x];
        count = P.cta_begin[blockIdx.x + 1] - begin;
    }
    __device__ int num_jobs() const { return count; }
    __device__ void job(int j, Job& d) const {
        const GroupJob g = P.jobs[begin + j];
        const InstInfo* I = P.insts + g.inst;
        d.inst = I;
        d.mapA = P.maps + 2 * I->bucket;
        d.mapB = P.maps + 2 * I->bucket + 1;
        d.tm = g.tm;
        d.tn = g.tn;
        d.c = g.c & 0xFF;
        d.H = (I->ksteps + I->chunk_steps - 1) / I->chunk_steps;
        d.slot = (g.c >> 8) & 1;  // tiles alternate the two residue slots
    }
    __device__ unsigned char* slots() const { return P.slots; }
    __device__ size_t slot_stride() const { return P.slot_stride; }
    __device__ int* err() const { return P.err; }
};

template <class Sched, class Params>
__device__ __forceinline__ void rns_gemm_body(const CUtensorMap* mapA, const CUtensorMap* mapB,
                                              const Params& P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = base;
    unsigned char* sB = base + kStages * kABytes;
    CombTables* tabs = reinterpret_cast<CombTables*>(sB + kStages * kBBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(tabs) + kTabBytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* acc_full = bars + 2 * kStages;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint64_t* slot_full = drain + 1;    // [2] epilogue -> combine warps: a tile's residues are complete
    uint64_t* slot_empty = slot_full + 2;  // [2] combine -> epilogue warps: the slot may be rewritten
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(slot_empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    const Sched S(P, mapA, mapB);
    const int J = S.num_jobs();   // jobs (tile, channel) of this CTA
    int* err = S.err();

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], kEpiWarps);
            mbar_init(&slot_full[a], kEpiWarps);
            mbar_init(&slot_empty[a], kCombineWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tc_alloc(tmem_slot, kTmemCols);
    if (warp == 0 && lane == 0 && mapA != nullptr) {
        tma_prefetch_desc(mapA);
        tma_prefetch_desc(mapB);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued = 0, last_parity = 0;
            bool ok = true;
            for (int pi = 0; 2 * pi < J && ok; ++pi) {
                const int nj = min(2, J - 2 * pi);
                Job jb[2];
                S.job(2 * pi, jb[0]);
                if (nj > 1) S.job(2 * pi + 1, jb[1]);
                const int Hmax = nj > 1 ? max(jb[0].H, jb[1].H) : jb[0].H;
                for (int h = 0; h < Hmax && ok; ++h) {
                    for (int s = 0; s < nj && ok; ++s) {
                        const Job& d = jb[s];
                        if (h >= d.H) continue;
                        const int cs = d.inst->chunk_steps;
                        const int k0 = h * cs;
                        const int steps = min(cs, d.inst->ksteps - k0);
                        const int rowA = d.inst->rowA + d.tm * kTileM;
                        const int rowB = d.inst->rowB + d.tn * kTileN;
                        for (int st = 0; st < steps; ++st) {
                            if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err, kDevTimeoutProducer)) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_expect_tx(&full[stage], kStageBytes);
                            const int kx = (k0 + st) * kTileK;
                            tma_load_3d(sA + stage * kABytes, d.mapA, kx, rowA, d.c, &full[stage]);
                            tma_load_3d(sB + stage * kBBytes, d.mapB, kx, rowB, d.c, &full[stage]);
                            issued |= 1u << stage;
                            last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                }
            }
            // every issued copy must have landed before shared memory is released
            for (int s2 = 0; s2 < kStages; ++s2)
                if (issued & (1u << s2)) mbar_drain_wait(&full[s2], (last_parity >> s2) & 1u, err);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t accp[2] = {0u, 0u};
            const uint32_t idesc = idesc_bf16_f32(kTileM, kTileN);
            bool ok = true;
            bool any = false;
            for (int pi = 0; 2 * pi < J && ok; ++pi) {
                const int nj = min(2, J - 2 * pi);
                Job jb[2];
                S.job(2 * pi, jb[0]);
                if (nj > 1) S.job(2 * pi + 1, jb[1]);
                const int Hmax = nj > 1 ? max(jb[0].H, jb[1].H) : jb[0].H;
                for (int h = 0; h < Hmax && ok; ++h) {
                    for (int s = 0; s < nj && ok; ++s) {
                        const Job& d = jb[s];
                        if (h >= d.H) continue;
                        const int cs = d.inst->chunk_steps;
                        const int steps = min(cs, d.inst->ksteps - h * cs);
                        if (!mbar_wait(&acc_empty[s], accp[s] ^ 1u, abort_flag, err, kDevTimeoutMma)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dt = tmem + (uint32_t)(s * kTileN);
                        for (int st = 0; st < steps; ++st) {
                            if (!mbar_wait(&full[stage], phase, abort_flag, err, kDevTimeoutMma)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t a0 = smem_addr(sA + stage * kABytes);
                            const uint32_t b0 = smem_addr(sB + stage * kBBytes);
#pragma unroll
                            for (int kk = 0; kk < kTileK / 16; ++kk) {
                                const uint32_t acc = (h > 0 || st > 0 || kk > 0) ? 1u : 0u;
                                tc_mma_bf16(dt, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32),
                                            idesc, acc);
                            }
                            tc_commit(&empty[stage]);
                            any = true;
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                        if (!ok) break;
                        tc_commit(&acc_full[s]);
                        accp[s] ^= 1u;
                    }
                }
            }
            // all issued MMAs must complete before tensor memory is released
            if (any) {
                tc_commit(drain);
                mbar_drain_wait(drain, 0u, err);
            }
        }
    } else if (warp < kFirstCombineWarp) {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_local = q * 32 + lane;
        const size_t sstride = S.slot_stride();
        unsigned char* slot_base = S.slots() + size_t(blockIdx.x) * 2 * sstride;
        const size_t row_off = size_t(row_local) * kTileN + half * 128;
        uint32_t accp[2] = {0u, 0u};
        uint32_t sep[2] = {0u, 0u};  // slot_empty phases
        bool ok = true;
        for (int pi = 0; 2 * pi < J && ok; ++pi) {
            const int nj = min(2, J - 2 * pi);
            Job jb[2];
            S.job(2 * pi, jb[0]);
            if (nj > 1) S.job(2 * pi + 1, jb[1]);
            const int Hmax = nj > 1 ? max(jb[0].H, jb[1].H) : jb[0].H;
            for (int h = 0; h < Hmax && ok; ++h) {
                for (int s = 0; s < nj; ++s) {
                    const Job& d = jb[s];
                    if (h >= d.H) continue;
                    const bool last_chunk = (h == d.H - 1);
                    const InstInfo& I = *d.inst;
                    const int c = d.c;
                    unsigned char* slot_row = slot_base + size_t(d.slot) * sstride + row_off;
                    if (!mbar_wait(&acc_full[s], accp[s], abort_flag, err, kDevTimeoutEpilogue)) {
                        ok = false;
                        break;
                    }
                    accp[s] ^= 1u;
                    tc_fence_after();
                    const uint32_t tbase =
                        tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * kTileN + half * 128);
                    const float mf = I.modf[c], im = I.inv_m[c];
                    const int mi = (int)I.modu[c];
                    if (!last_chunk) {
#pragma unroll 1
                        for (int cc = 0; cc < 4; ++cc) {
                            uint32_t v[32];
                            tc_ld32(tbase + cc * 32, v);
                            tc_wait_ld();
#pragma unroll
                            for (int i = 0; i < 32; ++i) {
                                const float x = __uint_as_float(v[i]);
                                const float qq = rintf(x * im);
                                v[i] = __float_as_uint(fmaf(-qq, mf, x));
                            }
                            tc_st32(tbase + cc * 32, v);
                        }
                        tc_wait_st();
                    } else {
                        // the tile's first residues: wait until the combine warps released this slot
                        if (c == 0) {
                            if (!mbar_wait(&slot_empty[d.slot], sep[d.slot] ^ 1u, abort_flag, err,
                                           kDevTimeoutEpilogue)) {
                                ok = false;
                                break;
                            }
                            sep[d.slot] ^= 1u;
                        }
                        unsigned char* dst = slot_row + size_t(c) * kTileM * kTileN;
#pragma unroll 1
                        for (int cc = 0; cc < 4; ++cc) {
                            uint32_t v[32];
                            tc_ld32(tbase + cc * 32, v);
                            tc_wait_ld();
                            uint32_t w[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                uint32_t packed = 0;
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    packed |= f32_residue(__uint_as_float(v[4 * i + e]), mf, im, mi)
                                              << (8 * e);
                                w[i] = packed;
                            }
                            uint4* d4 = reinterpret_cast<uint4*>(dst + cc * 32);
                            d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
                            d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
                        }
                    }
                    tc_fence_before();
                    if (last_chunk && c == I.nch - 1) __threadfence_block();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&acc_empty[s]);
                        if (last_chunk && c == I.nch - 1) mbar_arrive(&slot_full[d.slot]);
                    }
                }
            }
        }
    } else {
        // ------------------------------------------------------------ combine warps
        const int cw = warp - kFirstCombineWarp;
        const size_t sstride = S.slot_stride();
        unsigned char* slot_base = S.slots() + size_t(blockIdx.x) * 2 * sstride;
        uint32_t sfp[2] = {0u, 0u};
        const InstInfo* loaded = nullptr;
        for (int j = 0; j < J; ++j) {
            Job d;
            S.job(j, d);
            if (d.c != d.inst->nch - 1) continue;  // one reconstruction per tile
            if (d.inst != loaded) {
                // every combine warp is done with the previous tables (barrier inside)
                build_tables(*d.inst, tabs, cw * 32 + lane);
                loaded = d.inst;
            }
            if (!mbar_wait(&slot_full[d.slot], sfp[d.slot], abort_flag, err, kDevTimeoutEpilogue)) break;
            sfp[d.slot] ^= 1u;
            combine_block(*d.inst, tabs, d.tm * kTileM, d.tn * kTileN, slot_base + size_t(d.slot) * sstride,
                          size_t(kTileM) * kTileN, cw, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&slot_empty[d.slot]);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tc_dealloc(tmem, kTmemCols);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    rns_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                    const __grid_constant__ CUtensorMap mapB,
                    const __grid_constant__ RnsGemmParams P) {
    rns_gemm_body<SingleSched>(&mapA, &mapB, P);
}

__global__ void __launch_bounds__(kThreads, 1)
    rns_gemm_grouped_kernel(const __grid_constant__ GroupGemmParams P) {
    rns_gemm_body<GroupSched>(nullptr, nullptr, P);
}


// ---------------------------------------------------------------------------
// CTA-pair variant (cluster of 2, tcgen05 cta_group::2): one 256 x 256 output
// tile per pair; CTA rank r owns rows [128 r, 128 r + 128) of the tile and
// column half r of the B tile.  The leader (rank 0) issues M=256 N=256 MMAs
// that read A from each CTA's own shared memory and B from both halves, and
// writes each CTA's 128 x 256 accumulator into that CTA's tensor memory.  Per
// SM and stage the TMA moves 32 KB instead of 48 KB for the same tensor work,
// which leaves room for 6 stages.  Barriers: both CTAs' copies complete on the
// leader's full[] barrier; the leader's commits arrive on empty[] and
// acc_full[] in both CTAs; both CTAs' epilogues arrive on the leader's
// acc_empty[] (16 warps).
constexpr int kPStages = 6;
constexpr uint32_t kPABytes = 128 * kTileK * 2;
constexpr uint32_t kPBBytes = 128 * kTileK * 2;
constexpr uint32_t kPStageBytes = kPABytes + kPBBytes;
constexpr size_t kPairSmemBytes = 1024 + size_t(kPStages) * kPStageBytes + kTabBytes + 256;
constexpr int kPairTile = 256;

__global__ void __launch_bounds__(kThreads, 1)
    rns_gemm_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                         const __grid_constant__ RnsGemmParams P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = base;
    unsigned char* sB = base + kPStages * kPABytes;
    CombTables* tabs = reinterpret_cast<CombTables*>(sB + kPStages * kPBBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(tabs) + kTabBytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kPStages;
    uint64_t* acc_full = bars + 2 * kPStages;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint64_t* slot_full = drain + 1;       // [2] epilogue -> combine warps (this CTA)
    uint64_t* slot_empty = slot_full + 2;  // [2] combine -> epilogue warps (this CTA)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(slot_empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const InstInfo& I = P.inst;
    int* err = P.err;

    const int pair = (int)blockIdx.x >> 1, npairs = (int)gridDim.x >> 1;
    const int my_tiles = pair < P.num_tiles ? (P.num_tiles - 1 - pair) / npairs + 1 : 0;
    const int nch = I.nch;
    const int J = my_tiles * nch;
    const int CS = I.chunk_steps;
    const int H = (I.ksteps + CS - 1) / CS;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kPStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 2 * kEpiWarps);
            mbar_init(&slot_full[a], kEpiWarps);
            mbar_init(&slot_empty[a], kCombineWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) tc_alloc_pair(tmem_slot, kTmemCols);
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
    }
    tc_fence_before();
    cluster_sync();  // barriers of both CTAs initialised, tensor memory allocated
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------- producer (both CTAs)
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued = 0, last_parity = 0;
            bool ok = true;
            for (int pi = 0; 2 * pi < J && ok; ++pi) {
                const int nj = min(2, J - 2 * pi);
                for (int h = 0; h < H && ok; ++h) {
                    const int k0 = h * CS;
                    const int steps = min(CS, I.ksteps - k0);
                    for (int s = 0; s < nj && ok; ++s) {
                        const int j = 2 * pi + s;
                        const int t = pair + (j / nch) * npairs;
                        const int c = j % nch;
                        int tm, tn;
                        tile_coords(t, P.tiles_m, P.tiles_n, tm, tn);
                        const int rowA = tm * kPairTile + (int)rank * 128;
                        const int rowB = tn * kPairTile + (int)rank * 128;
                        for (int st = 0; st < steps; ++st) {
                            if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err, kDevTimeoutProducer)) {
                                ok = false;
                                break;
                            }
                            if (leader) mbar_arrive_expect_tx(&full[stage], 2 * kPStageBytes);
                            const uint32_t fb = cluster_addr(&full[stage], 0);
                            const int kx = (k0 + st) * kTileK;
                            tma_load_3d_pair(sA + stage * kPABytes, &mapA, kx, rowA, c, fb);
                            tma_load_3d_pair(sB + stage * kPBBytes, &mapB, kx, rowB, c, fb);
                            issued |= 1u << stage;
                            last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
                            if (++stage == kPStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                }
            }
            // the leader's full[] barriers count both CTAs' copies: draining them
            // covers every copy into either CTA's shared memory
            if (leader)
                for (int s2 = 0; s2 < kPStages; ++s2)
                    if (issued & (1u << s2)) mbar_drain_wait(&full[s2], (last_parity >> s2) & 1u, err);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer (leader)
        if (lane == 0 && leader) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t accp[2] = {0u, 0u};
            const uint32_t idesc = idesc_bf16_f32(2 * kTileM, kTileN);
            bool ok = true;
            bool any = false;
            for (int pi = 0; 2 * pi < J && ok; ++pi) {
                const int nj = min(2, J - 2 * pi);
                for (int h = 0; h < H && ok; ++h) {
                    const int steps = min(CS, I.ksteps - h * CS);
                    for (int s = 0; s < nj && ok; ++s) {
                        if (!mbar_wait(&acc_empty[s], accp[s] ^ 1u, abort_flag, err, kDevTimeoutMma)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dt = tmem + (uint32_t)(s * kTileN);
                        for (int st = 0; st < steps; ++st) {
                            if (!mbar_wait(&full[stage], phase, abort_flag, err, kDevTimeoutMma)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t a0 = smem_addr(sA + stage * kPABytes);
                            const uint32_t b0 = smem_addr(sB + stage * kPBBytes);
#pragma unroll
                            for (int kk = 0; kk < kTileK / 16; ++kk) {
                                const uint32_t acc = (h > 0 || st > 0 || kk > 0) ? 1u : 0u;
                                tc_mma_bf16_pair(dt, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc,
                                                 acc);
                            }
                            tc_commit_pair_both(&empty[stage]);
                            any = true;
                            if (++stage == kPStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                        if (!ok) break;
                        tc_commit_pair_both(&acc_full[s]);
                        accp[s] ^= 1u;
                    }
                }
            }
            if (any) {
                tc_commit_pair_local(drain);
                mbar_drain_wait(drain, 0u, err);
            }
        }
    } else if (warp < kFirstCombineWarp) {
        // ---------------------------------------------------- epilogue (both CTAs)
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_local = q * 32 + lane;
        unsigned char* slot_base = P.slots + size_t(blockIdx.x) * 2 * P.slot_stride;
        const size_t row_off = size_t(row_local) * kTileN + half * 128;
        const uint32_t acc_empty_leader[2] = {cluster_addr(&acc_empty[0], 0), cluster_addr(&acc_empty[1], 0)};
        uint32_t accp[2] = {0u, 0u};
        uint32_t sep[2] = {0u, 0u};
        bool ok = true;
        for (int pi = 0; 2 * pi < J && ok; ++pi) {
            const int nj = min(2, J - 2 * pi);
            for (int h = 0; h < H && ok; ++h) {
                const bool last_chunk = (h == H - 1);
                for (int s = 0; s < nj; ++s) {
                    const int j = 2 * pi + s;
                    const int c = j % nch;
                    const int slot = (j / nch) & 1;
                    unsigned char* slot_row = slot_base + size_t(slot) * P.slot_stride + row_off;
                    if (!mbar_wait(&acc_full[s], accp[s], abort_flag, err, kDevTimeoutEpilogue)) {
                        ok = false;
                        break;
                    }
                    accp[s] ^= 1u;
                    tc_fence_after();
                    const uint32_t tbase =
                        tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * kTileN + half * 128);
                    const float mf = I.modf[c], im = I.inv_m[c];
                    const int mi = (int)I.modu[c];
                    if (!last_chunk) {
#pragma unroll 1
                        for (int cc = 0; cc < 4; ++cc) {
                            uint32_t v[32];
                            tc_ld32(tbase + cc * 32, v);
                            tc_wait_ld();
#pragma unroll
                            for (int i = 0; i < 32; ++i) {
                                const float x = __uint_as_float(v[i]);
                                const float qq = rintf(x * im);
                                v[i] = __float_as_uint(fmaf(-qq, mf, x));
                            }
                            tc_st32(tbase + cc * 32, v);
                        }
                        tc_wait_st();
                    } else {
                        if (c == 0) {
                            if (!mbar_wait(&slot_empty[slot], sep[slot] ^ 1u, abort_flag, err, kDevTimeoutEpilogue)) {
                                ok = false;
                                break;
                            }
                            sep[slot] ^= 1u;
                        }
                        unsigned char* dst = slot_row + size_t(c) * kTileM * kTileN;
#pragma unroll 1
                        for (int cc = 0; cc < 4; ++cc) {
                            uint32_t v[32];
                            tc_ld32(tbase + cc * 32, v);
                            tc_wait_ld();
                            uint32_t w[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                uint32_t packed = 0;
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    packed |= f32_residue(__uint_as_float(v[4 * i + e]), mf, im, mi) << (8 * e);
                                w[i] = packed;
                            }
                            uint4* d4 = reinterpret_cast<uint4*>(dst + cc * 32);
                            d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
                            d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
                        }
                    }
                    tc_fence_before();
                    if (last_chunk && c == nch - 1) __threadfence_block();
                    __syncwarp();
                    if (lane == 0) {
                        if (leader)
                            mbar_arrive(&acc_empty[s]);
                        else
                            mbar_arrive_cluster(acc_empty_leader[s]);
                        if (last_chunk && c == nch - 1) mbar_arrive(&slot_full[slot]);
                    }
                }
            }
        }
    } else {
        // ---------------------------------------------------- combine warps (both CTAs)
        const int cw = warp - kFirstCombineWarp;
        unsigned char* slot_base = P.slots + size_t(blockIdx.x) * 2 * P.slot_stride;
        uint32_t sfp[2] = {0u, 0u};
        if (my_tiles > 0) build_tables(I, tabs, cw * 32 + lane);
        for (int ti = 0; ti < my_tiles; ++ti) {
            const int slot = ti & 1;
            if (!mbar_wait(&slot_full[slot], sfp[slot], abort_flag, err, kDevTimeoutEpilogue)) break;
            sfp[slot] ^= 1u;
            int tm, tn;
            tile_coords(pair + ti * npairs, P.tiles_m, P.tiles_n, tm, tn);
            // rows of this CTA: the 128-row block 2 tm + rank
            combine_block(I, tabs, (2 * tm + (int)rank) * kTileM, tn * kTileN, slot_base + size_t(slot) * P.slot_stride,
                          size_t(kTileM) * kTileN, cw, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&slot_empty[slot]);
        }
    }

    tc_fence_before();
    cluster_sync();  // no CTA leaves while its peer may still read its shared memory
    if (warp == 1) {
        tc_fence_after();
        tc_dealloc_pair(tmem, kTmemCols);
    }
}

}  // namespace

size_t rns_gemm_smem_bytes() { return kSmemBytes; }

static cudaLaunchConfig_t pair_config(int grid, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = kPairSmemBytes;
    cfg.stream = s;
    attr->id = cudaLaunchAttributeClusterDimension;
    attr->val.clusterDim.x = 2;
    attr->val.clusterDim.y = 1;
    attr->val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

static cudaError_t pair_attr() {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(rns_gemm_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kPairSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return cudaSuccess;
}

// Number of CTA pairs that can be resident at once (GPCs with an odd number of
// SMs leave one SM out): the persistent grid must not exceed it.
int rns_gemm_pair_max_clusters() {
    static int cached = -1;
    if (cached < 0) {
        if (pair_attr() != cudaSuccess) return 0;
        cudaLaunchAttribute attr;
        cudaLaunchConfig_t cfg = pair_config(2, 0, &attr);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, rns_gemm_pair_kernel, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        cached = n;
    }
    return cached;
}

cudaError_t launch_rns_gemm_pair(const CUtensorMap& mapA, const CUtensorMap& mapB, const RnsGemmParams& prm,
                                 int grid, cudaStream_t s) {
    cudaError_t e = pair_attr();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr;
    cudaLaunchConfig_t cfg = pair_config(grid, s, &attr);
    return cudaLaunchKernelEx(&cfg, rns_gemm_pair_kernel, mapA, mapB, prm);
}

cudaError_t launch_rns_gemm(const CUtensorMap& mapA, const CUtensorMap& mapB,
                            const RnsGemmParams& prm, int grid, cudaStream_t s) {
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(rns_gemm_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    rns_gemm_kernel<<<grid, kThreads, kSmemBytes, s>>>(mapA, mapB, prm);
    return cudaGetLastError();
}

cudaError_t launch_rns_gemm_grouped(const GroupGemmParams& prm, int grid, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(rns_gemm_grouped_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    rns_gemm_grouped_kernel<<<grid, kThreads, kSmemBytes, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace ffgpu
