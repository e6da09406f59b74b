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
// After the last chunk each channel yields its CRT digit b_c (S mod m_c times
// (M/m_c)^{-1} mod m_c, one byte per entry, written to a per-CTA residue slot);
// the last channel of a tile hands the slot to the combine warps, which
// reconstruct S mod p from all digits (Chinese remainder theorem, the
// multi-modular route to p > 2^26 the paper lists as future work in section 7)
// and write C = (alpha*S + beta*C) mod p.
//
// Roles (one CTA per SM, persistent over tiles):
//   warp 0      TMA producer: channel tiles of A (128x64) and B (256x64), 4 stages
//   warp 1      TMEM allocator and single-thread MMA issuer (M=128, N=256, K=16)
//   warps 2..9  epilogue: lane quarter (warp % 4) x column half ((warp-2) / 4)
//   warps 10-15 combine: reconstruction of the previous tile (two residue slots)
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

constexpr int kEpiWarps = 8;
static_assert(kEpiWarps == kSkFlagsPerCta, "one stream-K flag per epilogue warp");
constexpr int kCombineWarps = 6;
constexpr int kThreads = 32 * (2 + kEpiWarps + kCombineWarps);  // 2 control warps
constexpr int kFirstCombineWarp = 10;
constexpr uint32_t kABytes = kTileM * kTileK * 2;
constexpr uint32_t kBBytes = kTileN * kTileK * 2;
constexpr uint32_t kStageBytes = kABytes + kBBytes;
constexpr uint32_t kTmemCols = 512;
// per-instance constants of the reconstruction (see stage_consts): one copy for
// the combine warps, one per epilogue warp
constexpr size_t kConstBytes = size_t(1 + kEpiWarps) * kMaxChannels * 16;
constexpr size_t kSmemBytes = 1024 + size_t(kStages) * kStageBytes + kConstBytes + 256;

// Tile order: bands of `band` tile rows, column by column within a band (the
// tiles running at once share B columns and A rows in L2).
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int band, int& tm, int& tn) {
    const int per_group = band * tiles_n;
    const int g = t / per_group;
    const int first = g * band;
    const int gm = min(tiles_m - first, band);
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

// Rounding to the nearest integer without the (slow) float-to-integral
// conversion: for |z| < 2^22, z + 1.5 2^23 lands in [2^23, 2^24), where the
// float spacing is 1, so the fused add rounds z (taken exactly, before any
// rounding of a product inside the fma) to an integer.
constexpr float kRoundMagic = 12582912.f;  // 1.5 * 2^23

// CRT digit of one accumulator entry: with r = x mod m_c (x an f32 integer,
// |x| / m_c < 2^22), b = r u_c mod m_c in balanced form, |b| <= 127, returned
// as the f32 bit pattern of 1.5 2^23 + 128 + b, whose low byte is b + 128.
// Exactness: |r| <= 129 (the quotient x/m_c is rounded from a product with
// relative error < 2^-24 of a value below 2^22), so r u_c (< 2^15) and every
// intermediate below are integers exact in f32; r u_c / m_c is rounded from a
// value within 2^-14 of it, while for odd m_c its fractional part, a multiple
// of 1/m_c, stays 1/(2 m_c) away from 1/2, so b = r u_c - m_c round(r u_c /
// m_c) is the balanced residue (for even moduli, direct mode only, a tie may
// give +-m_c/2 <= 127).  Seven full-rate float operations, no conversion.
__device__ __forceinline__ uint32_t crt_digit_bits(float x, float mf, float im, float uf, float uim) {
    const float q1 = fmaf(x, im, kRoundMagic) - kRoundMagic;
    const float r = fmaf(-q1, mf, x);
    const float q2 = fmaf(r, uim, kRoundMagic) - kRoundMagic;
    return __float_as_uint(fmaf(r, uf, fmaf(-q2, mf, kRoundMagic + 128.f)));
}

// Low bytes of four digit patterns, packed.
__device__ __forceinline__ uint32_t pack_digits(uint32_t d0, uint32_t d1, uint32_t d2, uint32_t d3) {
    return __byte_perm(__byte_perm(d0, d1, 0x0040u), __byte_perm(d2, d3, 0x0040u), 0x5410u);
}

// [0, 2p) -> [0, p) (unsigned wrap-around makes t - p huge when t < p).
__device__ __forceinline__ uint32_t fold_p(uint32_t t, uint32_t p) { return min(t, t - p); }

// x w mod p up to one p (result in [0, 2p)) for any x < 2^32 and w < p < 2^31,
// given ws = floor(w 2^32 / p): Shoup's precomputed-quotient product, all in
// 32-bit arithmetic (x w / p - floor(x ws / 2^32) lies in [0, 2)).
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint32_t w, uint32_t ws, uint32_t p) {
    return x * w - __umulhi(x, ws) * p;
}

// Reconstruction of alpha X + beta C mod p from the CRT digits, for the
// 128 x 256 block of one CTA.  With M = prod m_c and b_c = r_c (M/m_c)^{-1}
// mod m_c in balanced form (the epilogue stores b_c + 128, see
// crt_digit_bits), X = sum_c b_c M/m_c - q M where q = round(sum_c b_c / m_c),
// valid because the plan guarantees |X| <= M/4; |q| <= 6.  q comes from a
// 14-bit fixed-point sum F = sum_c b_c fr_c with fr_c = round(2^14/m_c): each
// term is off by at most 128/2 units of 2^-14, twelve of them by < 0.05, so
// F / 2^14 stays within 0.3 of q.  Then alpha X mod p = (sum_c b_c Wa_c +
// q negMpa) mod p with Wa_c = alpha (M/m_c) mod p and negMpa = alpha (-M)
// mod p.  Both sums run over the stored bytes b_c + 128 in unsigned
// arithmetic, started at Kfix and Finit, which cancel the offsets mod p and
// make the quotient sum yield q + 6 >= 0: Y = S + (q + 6) negMpa < 2^44,
// congruent to alpha X, accumulated with one wide multiply-add per channel and
// reduced as Y_hi (2^32 mod p) + Y_lo with Shoup products; beta C mod p
// likewise.  Per output and channel: one byte extraction and two integer
// multiply-adds.
//
// Done by the kCombineWarps combine warps, joined for a CTA's last tile by the
// kEpiWarps epilogue warps (then idle): of nw participating warps, warp vw takes
// rows vw, vw + nw, ...; lane l takes columns [8 l, 8 l + 8), so a warp reads
// 256 contiguous digit bytes per channel and row and 1 KB of C.  The next
// row's digits and C entries are loaded while the current row is reduced (two
// register buffers); the loads are latency-bound, hence the extra warps.
struct CombRow {
    uint2 w[kMaxChannels];  // digits of columns 8l .. 8l+7, per channel
    uint32_t o[8];          // the old entries of C
};

__device__ __forceinline__ void comb_load(const unsigned char* src, size_t chan_stride, int nch,
                                          const uint32_t* crow, int col, int n, bool full8, bool ldo,
                                          CombRow& R) {
#pragma unroll
    for (int c = 0; c < kMaxChannels; ++c)
        if (c < nch) R.w[c] = *reinterpret_cast<const uint2*>(src + size_t(c) * chan_stride);
#pragma unroll
    for (int e = 0; e < 8; ++e) R.o[e] = 0u;
    if (ldo) {
        if (full8) {
            const uint4 v0 = *reinterpret_cast<const uint4*>(crow + col);
            const uint4 v1 = *reinterpret_cast<const uint4*>(crow + col + 4);
            R.o[0] = v0.x; R.o[1] = v0.y; R.o[2] = v0.z; R.o[3] = v0.w;
            R.o[4] = v1.x; R.o[5] = v1.y; R.o[6] = v1.z; R.o[7] = v1.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (col + e < n) R.o[e] = crow[col + e];
        }
    }
}

// Integer mode: the exact product, X = sum_c d_c (M/m_c) - Xoff - (q + 6) M
// over the stored bytes d_c = b_c + 128, all mod 2^64 (exact: |X| < 2^63 by
// the plan), written as int64 (C points to an int64 array).
__device__ __forceinline__ void comb_row_int(const InstInfo& I, const uint4* kc, int nch, const CombRow& R,
                                         uint32_t* crow32, int col, int n, bool full8) {
    unsigned long long X[8];
    uint32_t F[8];
    const uint32_t Finit = I.Finit;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        X[e] = 0ull;
        F[e] = Finit;
    }
#pragma unroll
    for (int c = 0; c < kMaxChannels; ++c) {
        if (c < nch) {
            const uint4 k = kc[c];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t d = __byte_perm(e < 4 ? R.w[c].x : R.w[c].y, 0u, 0x4440u | (uint32_t)(e & 3));
                X[e] += (unsigned long long)d * k.x + ((unsigned long long)(d * k.z) << 32);
                F[e] += d * k.y;
            }
        }
    }
    const unsigned long long Xoff = I.Xoff, M = I.Mfull;
    long long out[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) out[e] = (long long)(X[e] - Xoff - (unsigned long long)(F[e] >> 14) * M);
    long long* crow = reinterpret_cast<long long*>(crow32);
    if (I.beta != 0) {  // a later slice of the inner dimension adds to the earlier ones
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (col + e < n) out[e] += crow[col + e];
    }
    if (full8) {
#pragma unroll
        for (int e = 0; e < 8; e += 2)
            *reinterpret_cast<longlong2*>(crow + col + e) = make_longlong2(out[e], out[e + 1]);
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (col + e < n) crow[col + e] = out[e];
    }
}

template <bool kInt>
__device__ __forceinline__ void comb_row(const InstInfo& I, const uint4* kc, int nch, const CombRow& R,
                                         uint32_t* crow, int col, int n, bool full8) {
    if constexpr (kInt) {
        comb_row_int(I, kc, nch, R, crow, col, n, full8);
        return;
    }
    unsigned long long S[8];
    uint32_t F[8];
    const uint32_t Kfix = I.Kfix, Finit = I.Finit;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        S[e] = Kfix;
        F[e] = Finit;
    }
#pragma unroll
    for (int c = 0; c < kMaxChannels; ++c) {
        if (c < nch) {
            const uint4 k = kc[c];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t b = __byte_perm(e < 4 ? R.w[c].x : R.w[c].y, 0u, 0x4440u | (uint32_t)(e & 3));
                S[e] += (unsigned long long)b * k.x;
                F[e] += b * k.y;
            }
        }
    }
    const uint32_t p = I.p, negMpa = I.negMpa, R32 = I.R32, R32s = I.R32s, one_s = I.one_s;
    const uint32_t beta = I.beta, beta_s = I.beta_s;
    uint32_t out[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const uint32_t q = F[e] >> 14;  // q + 6
        const unsigned long long Y = S[e] + (unsigned long long)q * negMpa;
        const uint32_t t1 = fold_p(mul_shoup((uint32_t)(Y >> 32), R32, R32s, p), p);
        const uint32_t lo = (uint32_t)Y;
        const uint32_t t2 = fold_p(lo - __umulhi(lo, one_s) * p, p);
        const uint32_t x = fold_p(t1 + t2, p);
        const uint32_t t3 = fold_p(mul_shoup(R.o[e], beta, beta_s, p), p);
        out[e] = fold_p(x + t3, p);
    }
    if (full8) {
        *reinterpret_cast<uint4*>(crow + col) = make_uint4(out[0], out[1], out[2], out[3]);
        *reinterpret_cast<uint4*>(crow + col + 4) = make_uint4(out[4], out[5], out[6], out[7]);
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (col + e < n) crow[col + e] = out[e];
    }
}

template <bool kInt>
__device__ __forceinline__ void combine_block(const InstInfo& I, const uint4* kc, int row0, int col0,
                                              const unsigned char* slot, size_t chan_stride, int vw, int nw,
                                              int lane) {
    const int rows = min(kTileM, I.m - row0);
    const int n = I.n;
    const int col = col0 + 8 * lane;
    if (vw >= rows || col >= n) return;  // nothing below is warp-collective
    const int nch = I.nch;
    const bool full8 = (col + 7 < n) && I.vec_ok;
    const bool ldo = I.beta != 0 && !kInt;  // integer mode reads its int64 partial itself
    const long long ldc = I.ldc;
    uint32_t* const C = I.C + (long long)row0 * ldc;
    const unsigned char* const src = slot + 8 * lane;
    CombRow A, B;
    int r = vw;
    comb_load(src + size_t(r) * kTileN, chan_stride, nch, C + r * ldc, col, n, full8, ldo, A);
#pragma unroll 1
    while (true) {
        if (r + nw < rows)
            comb_load(src + size_t(r + nw) * kTileN, chan_stride, nch, C + (r + nw) * ldc, col, n, full8, ldo, B);
        comb_row<kInt>(I, kc, nch, A, C + r * ldc, col, n, full8);
        r += nw;
        if (r >= rows) break;
        if (r + nw < rows)
            comb_load(src + size_t(r + nw) * kTileN, chan_stride, nch, C + (r + nw) * ldc, col, n, full8, ldo, A);
        comb_row<kInt>(I, kc, nch, B, C + r * ldc, col, n, full8);
        r += nw;
        if (r >= rows) break;
    }
}

// The constants for one warp's own use (an epilogue warp joining a reconstruction).
__device__ __forceinline__ void stage_consts_warp(const InstInfo& I, uint4* kc, int lane) {
    if (lane < I.nch) kc[lane] = make_uint4(I.Wa[lane], I.fr[lane], I.Mhi[lane], 0u);
    __syncwarp();
}

// Per-instance constants of the reconstruction, {Wa_c, fr_c}, staged in shared
// memory by the combine warps (barriers among them on both sides).
__device__ __forceinline__ void stage_consts(const InstInfo& I, uint4* kc, int tid) {
    asm volatile("bar.sync 1, %0;" ::"r"(kCombineWarps * 32) : "memory");
    if (tid < I.nch) kc[tid] = make_uint4(I.Wa[tid], I.fr[tid], I.Mhi[tid], 0u);
    asm volatile("bar.sync 1, %0;" ::"r"(kCombineWarps * 32) : "memory");
}

// Epilogue of one warp on its 32 lanes x 128 columns of an accumulator, two
// 32-column loads in flight per tensor-memory wait.
// In-place reduction mod m_c (|result| <= m_c/2 + 1), between chunks; |x| / m_c
// < 2^22 (chunk lengths keep |x| < 2^24, and m_c >= 4 unless |residues| <= 1).
__device__ __forceinline__ void epi_reduce(uint32_t tbase, float mf, float im) {
#pragma unroll 1
    for (int cc = 0; cc < 4; cc += 2) {
        uint32_t v[32], v2[32];
        tc_ld32(tbase + cc * 32, v);
        tc_ld32(tbase + cc * 32 + 32, v2);
        tc_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float x = __uint_as_float(v[i]);
            v[i] = __float_as_uint(fmaf(-(fmaf(x, im, kRoundMagic) - kRoundMagic), mf, x));
            const float y = __uint_as_float(v2[i]);
            v2[i] = __float_as_uint(fmaf(-(fmaf(y, im, kRoundMagic) - kRoundMagic), mf, y));
        }
        tc_st32(tbase + cc * 32, v);
        tc_st32(tbase + cc * 32 + 32, v2);
    }
    tc_wait_st();
}

__device__ __forceinline__ void store_digits(const uint32_t* v, float mf, float im, float uf, float uim,
                                             unsigned char* dst) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        w[i] = pack_digits(crt_digit_bits(__uint_as_float(v[4 * i]), mf, im, uf, uim),
                           crt_digit_bits(__uint_as_float(v[4 * i + 1]), mf, im, uf, uim),
                           crt_digit_bits(__uint_as_float(v[4 * i + 2]), mf, im, uf, uim),
                           crt_digit_bits(__uint_as_float(v[4 * i + 3]), mf, im, uf, uim));
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// After the last chunk: CRT digits (one byte per entry) to the residue slot.
// Only what the reconstruction reads is stored: nothing for a row at or past
// the instance's last row (row_ok false), nothing for a 32-column group that
// starts at or past col_lim (columns counted from this warp's first one); the
// tensor-memory loads stay warp-wide.
__device__ __forceinline__ void epi_digits(uint32_t tbase, float mf, float im, float uf, float uim,
                                           unsigned char* dst, bool row_ok, int col_lim) {
#pragma unroll 1
    for (int cc = 0; cc < 4; cc += 2) {
        uint32_t v[32], v2[32];
        tc_ld32(tbase + cc * 32, v);
        tc_ld32(tbase + cc * 32 + 32, v2);
        tc_wait_ld();
        if (row_ok && cc * 32 < col_lim) store_digits(v, mf, im, uf, uim, dst + cc * 32);
        if (row_ok && cc * 32 + 32 < col_lim) store_digits(v2, mf, im, uf, uim, dst + cc * 32 + 32);
    }
}

// A job of the kernel: one channel of one output tile of one instance.  Every
// role walks its CTA's jobs in the same order with its own iterator, so the
// per-job work on the single-thread producer and MMA paths is a few moves:
// those threads share their SM sub-partitions with the epilogue warps' dense
// float code and get few issue slots while it runs.
struct Job {
    const InstInfo* inst;
    const CUtensorMap* mapA;
    const CUtensorMap* mapB;
    int tm, tn;
    int c, nch;
    int H;           // chunks of cs k-steps
    int cs, ksteps;
    int rowA, rowB;  // first plane rows of the tile's A and B blocks
    int slot;        // residue slot of the job's tile
    float mf, im, uf;  // m_c, 1/m_c, (M/m_c)^{-1} mod m_c
};

// Single instance, tiles dealt round-robin to the CTAs, channels in order.
struct SingleSched {
    const RnsGemmParams& P;
    const CUtensorMap* mA;
    const CUtensorMap* mB;
    int my_tiles, H;
    int ti, c, tm, tn;  // iteration state
    __device__ SingleSched(const RnsGemmParams& p, const CUtensorMap* a, const CUtensorMap* b)
        : P(p), mA(a), mB(b), ti(0), c(0), tm(0), tn(0) {
        my_tiles = (int)blockIdx.x < P.num_tiles
                       ? (P.num_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                       : 0;
        H = (P.inst.ksteps + P.inst.chunk_steps - 1) / P.inst.chunk_steps;
        if (my_tiles > 0) tile_coords((int)blockIdx.x, P.tiles_m, P.tiles_n, P.raster, tm, tn);
    }
    __device__ int num_jobs() const { return my_tiles * P.inst.nch; }
    __device__ void fill(Job& d, int tile_ord, int ch, int tm_, int tn_) const {
        const InstInfo& I = P.inst;
        d.inst = &I;
        d.mapA = mA;
        d.mapB = mB;
        d.tm = tm_;
        d.tn = tn_;
        d.c = ch;
        d.nch = I.nch;
        d.H = H;
        d.cs = I.chunk_steps;
        d.ksteps = I.ksteps;
        d.rowA = I.rowA + tm_ * kTileM;
        d.rowB = I.rowB + tn_ * kTileN;
        d.slot = tile_ord & 1;  // tiles alternate the two residue slots
        d.mf = I.modf[ch];
        d.im = I.inv_m[ch];
        d.uf = (float)I.u[ch];
    }
    __device__ void next(Job& d) {
        fill(d, ti, c, tm, tn);
        if (++c == P.inst.nch) {
            c = 0;
            if (++ti < my_tiles) tile_coords((int)blockIdx.x + ti * (int)gridDim.x, P.tiles_m, P.tiles_n, P.raster, tm, tn);
        }
    }
    __device__ void last_job(Job& d) const {
        int a, b;
        tile_coords((int)blockIdx.x + (my_tiles - 1) * (int)gridDim.x, P.tiles_m, P.tiles_n, P.raster, a, b);
        fill(d, my_tiles - 1, P.inst.nch - 1, a, b);
    }
    __device__ unsigned char* slots() const { return P.slots; }
    __device__ size_t slot_stride() const { return P.slot_stride; }
    __device__ int* err() const { return P.err; }
};

// Grouped launch: the host lists every CTA's jobs; the next record is loaded
// one job ahead.
struct GroupSched {
    const GroupGemmParams& P;
    int begin, count, j;
    GroupJob nxt;
    __device__ GroupSched(const GroupGemmParams& p, const CUtensorMap*, const CUtensorMap*) : P(p), j(0) {
        begin = P.cta_begin[blockIdx.x];
        count = P.cta_begin[blockIdx.x + 1] - begin;
        if (count > 0) nxt = P.jobs[begin];
    }
    __device__ int num_jobs() const { return count; }
    __device__ void decode(const GroupJob& g, Job& d) const {
        d.inst = P.insts + g.inst;
        const int bucket = (int)(g.cfg >> 16);
        d.mapA = P.maps + 2 * bucket;
        d.mapB = P.maps + 2 * bucket + 1;
        d.tm = (int)(g.tmtn & 0xFFFFu);
        d.tn = (int)(g.tmtn >> 16);
        d.c = (int)(g.cfg & 0xFFu);
        d.slot = (int)((g.cfg >> 8) & 1u);
        d.nch = (int)((g.cfg >> 12) & 0xFu);
        d.H = g.H;
        d.cs = (int)((g.modc >> 16) & 0xFFu);
        d.ksteps = g.ksteps;
        d.rowA = g.rowA;
        d.rowB = g.rowB;
        d.mf = (float)(g.modc & 0xFFu);
        d.im = __frcp_rn(d.mf);
        d.uf = (float)((g.modc >> 8) & 0xFFu);
    }
    __device__ void next(Job& d) {
        const GroupJob g = nxt;
        if (++j < count) nxt = P.jobs[begin + j];
        decode(g, d);
    }
    __device__ void last_job(Job& d) const { decode(P.jobs[begin + count - 1], d); }
    __device__ unsigned char* slots() const { return P.slots; }
    __device__ size_t slot_stride() const { return P.slot_stride; }
    __device__ int* err() const { return P.err; }
};

template <class Sched, bool kInt, class Params>
__device__ __forceinline__ void rns_gemm_body(const CUtensorMap* mapA, const CUtensorMap* mapB,
                                              const Params& P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = base;
    unsigned char* sB = base + kStages * kABytes;
    uint4* kc = reinterpret_cast<uint4*>(sB + kStages * kBBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(kc) + kConstBytes);
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

    Sched S(P, mapA, mapB);       // per-thread iterator over this CTA's jobs
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
                S.next(jb[0]);
                if (nj > 1) S.next(jb[1]);
                const int Hmax = nj > 1 ? max(jb[0].H, jb[1].H) : jb[0].H;
                for (int h = 0; h < Hmax && ok; ++h) {
                    for (int s = 0; s < nj && ok; ++s) {
                        const Job& d = jb[s];
                        if (h >= d.H) continue;
                        const int cs = d.cs;
                        const int k0 = h * cs;
                        const int steps = min(cs, d.ksteps - k0);
                        const int rowA = d.rowA;
                        const int rowB = d.rowB;
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
                S.next(jb[0]);
                if (nj > 1) S.next(jb[1]);
                const int Hmax = nj > 1 ? max(jb[0].H, jb[1].H) : jb[0].H;
                for (int h = 0; h < Hmax && ok; ++h) {
                    for (int s = 0; s < nj && ok; ++s) {
                        const Job& d = jb[s];
                        if (h >= d.H) continue;
                        const int cs = d.cs;
                        const int steps = min(cs, d.ksteps - h * cs);
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
        int tiles_on[2] = {0, 0};    // tiles handed to each slot so far
        bool ok = true;
        for (int pi = 0; 2 * pi < J && ok; ++pi) {
            const int nj = min(2, J - 2 * pi);
            Job jb[2];
            S.next(jb[0]);
            if (nj > 1) S.next(jb[1]);
            const int Hmax = nj > 1 ? max(jb[0].H, jb[1].H) : jb[0].H;
            for (int h = 0; h < Hmax && ok; ++h) {
                for (int s = 0; s < nj; ++s) {
                    const Job& d = jb[s];
                    if (h >= d.H) continue;
                    const bool last_chunk = (h == d.H - 1);
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
                    const float mf = d.mf, im = d.im;
                    const float uf = d.uf, uim = uf * im;
                    if (!last_chunk) {
                        epi_reduce(tbase, mf, im);
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
                        const InstInfo& I = *d.inst;
                        epi_digits(tbase, mf, im, uf, uim, dst, d.tm * kTileM + row_local < I.m,
                                   I.n - d.tn * kTileN - half * 128);
                    }
                    tc_fence_before();
                    if (last_chunk && c == d.nch - 1) __threadfence_block();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&acc_empty[s]);
                        if (last_chunk && c == d.nch - 1) mbar_arrive(&slot_full[d.slot]);
                    }
                    if (last_chunk && c == d.nch - 1) ++tiles_on[d.slot];
                }
            }
        }
        if (ok && J > 0) {
            // the CTA's last tile: take 8 of the 12 row shares of its reconstruction
            Job d;
            S.last_job(d);
            uint4* kcw = kc + (1 + (warp - 2)) * kMaxChannels;
            stage_consts_warp(*d.inst, kcw, lane);
            if (mbar_wait(&slot_full[d.slot], (uint32_t)(tiles_on[d.slot] - 1) & 1u, abort_flag, err,
                          kDevTimeoutEpilogue))
                combine_block<kInt>(*d.inst, kcw, d.tm * kTileM, d.tn * kTileN, slot_base + size_t(d.slot) * sstride,
                              size_t(kTileM) * kTileN, kCombineWarps + (warp - 2), kCombineWarps + kEpiWarps, lane);
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
            S.next(d);
            if (d.c != d.nch - 1) continue;  // one reconstruction per tile
            if (d.inst != loaded) {
                // every combine warp is done with the previous constants (barrier inside)
                stage_consts(*d.inst, kc, cw * 32 + lane);
                loaded = d.inst;
            }
            if (!mbar_wait(&slot_full[d.slot], sfp[d.slot], abort_flag, err, kDevTimeoutEpilogue)) break;
            sfp[d.slot] ^= 1u;
            const bool last = j == J - 1;  // the epilogue warps join the last tile's reconstruction
            combine_block<kInt>(*d.inst, kc, d.tm * kTileM, d.tn * kTileN, slot_base + size_t(d.slot) * sstride,
                          size_t(kTileM) * kTileN, cw, last ? kCombineWarps + kEpiWarps : kCombineWarps, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&slot_empty[d.slot]);
        }
    }

    tc_fence_before();
    __syncwarp();  // warps 0 and 1 reconverge (lane 0 ran the producer / MMA loop) before the aligned barrier
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
    rns_gemm_body<SingleSched, false>(&mapA, &mapB, P);
}

__global__ void __launch_bounds__(kThreads, 1)
    rns_gemm_int_kernel(const __grid_constant__ CUtensorMap mapA,
                        const __grid_constant__ CUtensorMap mapB,
                        const __grid_constant__ RnsGemmParams P) {
    rns_gemm_body<SingleSched, true>(&mapA, &mapB, P);
}

__global__ void __launch_bounds__(kThreads, 1)
    rns_gemm_grouped_kernel(const __grid_constant__ GroupGemmParams P) {
    rns_gemm_body<GroupSched, false>(nullptr, nullptr, P);
}

__global__ void __launch_bounds__(kThreads, 1)
    rns_gemm_grouped_int_kernel(const __grid_constant__ GroupGemmParams P) {
    rns_gemm_body<GroupSched, true>(nullptr, nullptr, P);
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
//
// Schedule.  Tiles are dealt round-robin to the pairs.  When the last wave
// has fewer tiles (rem) than half the pairs, its tiles are instead cut along
// the inner dimension into sk_split equal parts of their k-steps (each part
// taken in chunks of at most chunk_steps), part j of tile r on pair r + j rem, so that the last wave keeps rem x sk_split pairs
// busy for a fraction of the time.  The parts of a wave run together, at the
// same offsets of the inner dimension, as the tiles of a full wave do (their
// operand blocks are shared through L2 the same way).  Parts j > 0 ("tails")
// reduce each channel's accumulator mod m_c and hand the residues (int16) to
// part 0 (the "head") through global memory, raising a flag per channel and
// epilogue warp; the head adds them to its own accumulators before that
// channel's CRT digits.
// The head's wait is bounded and nothing waits on a head.
constexpr int kPStages = 6;
constexpr uint32_t kPABytes = 128 * kTileK * 2;
constexpr uint32_t kPBBytes = 128 * kTileK * 2;
constexpr uint32_t kPStageBytes = kPABytes + kPBBytes;
constexpr size_t kPairSmemBytes = 1024 + size_t(kPStages) * kPStageBytes + kConstBytes + 256;
constexpr int kPairTile = 256;

// The segments of one pair (the same in every role of both CTAs): its
// round-robin tiles, then, in a cut last wave, one part of a tile.
struct PairSegs {
    int pair, np, KS, ndp, split, rem;
    __device__ PairSegs(const RnsGemmParams& P, int pair_, int np_, int KS_) : pair(pair_), np(np_), KS(KS_) {
        if (P.sk_split > 1) {
            ndp = P.sk_dp / np;
            split = P.sk_split;
            rem = P.sk_rem;
        } else {
            ndp = pair < P.num_tiles ? (P.num_tiles - 1 - pair) / np + 1 : 0;
            split = 0;
            rem = 1;
        }
    }
    __device__ bool in_split() const { return split > 1 && pair < rem * split; }
    __device__ int count() const { return ndp + (in_split() ? 1 : 0); }
    // segment j: tile t, k-steps [sb, se), kind 0 whole, 1 head, 2 tail
    __device__ void get(int j, int& t, int& sb, int& se, int& kind) const {
        if (j < ndp) {
            t = pair + j * np;
            sb = 0;
            se = KS;
            kind = 0;
            return;
        }
        const int part = pair / rem;
        t = ndp * np + pair % rem;
        sb = part * KS / split;
        se = (part + 1) * KS / split;
        kind = part == 0 ? 1 : 2;
    }
    __device__ bool has_tail() const { return in_split() && pair >= rem; }  // the last segment
    __device__ int digit_ord(int j) const { return j; }
    __device__ int digit_tiles() const { return count() - (has_tail() ? 1 : 0); }
};

// Partial residues of a tail: int16 per entry, [pair][rank][channel][128][256].
__device__ __forceinline__ short* sk_part_at(const RnsGemmParams& P, int pair, uint32_t rank, int c) {
    return P.sk_part + ((size_t(pair) * 2 + rank) * P.inst.nch + c) * size_t(kTileM) * kTileN;
}

__device__ __forceinline__ uint32_t pack_s16(float a, float b) {
    return (uint32_t)(uint16_t)(short)__float2int_rn(a) | ((uint32_t)(uint16_t)(short)__float2int_rn(b) << 16);
}

// Tail of a cut tile: this lane's 128 columns reduced mod m_c (|r| <= m_c/2 + 1)
// and stored as int16 at dst.
__device__ __forceinline__ void epi_partial(uint32_t tbase, float mf, float im, short* dst) {
#pragma unroll 1
    for (int cc = 0; cc < 4; cc += 2) {
        uint32_t v[32], v2[32];
        tc_ld32(tbase + cc * 32, v);
        tc_ld32(tbase + cc * 32 + 32, v2);
        tc_wait_ld();
        uint32_t w[32];
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
            const float x0 = __uint_as_float(v[i]), x1 = __uint_as_float(v[i + 1]);
            const float y0 = __uint_as_float(v2[i]), y1 = __uint_as_float(v2[i + 1]);
            w[i / 2] = pack_s16(fmaf(-(fmaf(x0, im, kRoundMagic) - kRoundMagic), mf, x0),
                                fmaf(-(fmaf(x1, im, kRoundMagic) - kRoundMagic), mf, x1));
            w[16 + i / 2] = pack_s16(fmaf(-(fmaf(y0, im, kRoundMagic) - kRoundMagic), mf, y0),
                                     fmaf(-(fmaf(y1, im, kRoundMagic) - kRoundMagic), mf, y1));
        }
        uint4* d4 = reinterpret_cast<uint4*>(dst + cc * 32);
#pragma unroll
        for (int i = 0; i < 8; ++i) d4[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    }
}

__device__ __forceinline__ void add_s16(uint32_t (&v)[32], const uint4* src) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 q = __ldcg(src + i);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 8 * i + 2 * e;
            v[j] = __float_as_uint(__uint_as_float(v[j]) + (float)(short)(w[e] & 0xFFFFu));
            v[j + 1] = __float_as_uint(__uint_as_float(v[j + 1]) + (float)(short)(w[e] >> 16));
        }
    }
}

// Head of a cut tile: epi_digits on the accumulator plus the residues of the
// tails on pairs tp0, tp0 + step, ... below tp_end (this lane's 128 int16 of
// each), one 32-column load at a time (a head is at most one tile per pair).
// The sums stay below 2^24 in magnitude (at most three tails of |r| <= 129).
__device__ __forceinline__ void epi_digits_sk(uint32_t tbase, float mf, float im, float uf, float uim,
                                              unsigned char* dst, bool row_ok, int col_lim, const RnsGemmParams& P,
                                              int tp0, int tp_end, int step, uint32_t rank, int c, size_t row_off) {
#pragma unroll 1
    for (int cc = 0; cc < 4; ++cc) {
        uint32_t v[32];
        tc_ld32(tbase + cc * 32, v);
        tc_wait_ld();
#pragma unroll 1
        for (int tp = tp0; tp < tp_end; tp += step)
            add_s16(v, reinterpret_cast<const uint4*>(sk_part_at(P, tp, rank, c) + row_off + cc * 32));
        if (row_ok && cc * 32 < col_lim) store_digits(v, mf, im, uf, uim, dst + cc * 32);
    }
}

__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait for a tail's flag (every lane polls); false on timeout or abort.
__device__ __forceinline__ bool sk_wait(const int* flag, volatile int* abort_flag, int* err) {
    if (ld_acquire_gpu(flag)) return true;
    const long long t0 = clock64();
    uint32_t it = 0;
    while (true) {
        if (ld_acquire_gpu(flag)) return true;
        if ((++it & 63u) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitLimitCycles) {
                *abort_flag = 1;
                atomicCAS(err, 0, (int)kDevTimeoutStreamK);
                return false;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    rns_gemm_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                         const __grid_constant__ RnsGemmParams P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = base;
    unsigned char* sB = base + kPStages * kPABytes;
    uint4* kc = reinterpret_cast<uint4*>(sB + kPStages * kPBBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(kc) + kConstBytes);
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
    const int nch = I.nch;
    const int CS = I.chunk_steps;
    const PairSegs G(P, pair, npairs, I.ksteps);
    const int nseg = G.count();
    const int J = nseg * nch;  // jobs: (segment, channel); a job pair never mixes two chunk ranges

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
                int jc[2], jrA[2], jrB[2], sb = 0, se = I.ksteps;
                for (int s = 0; s < nj; ++s) {
                    const int j = (2 * pi + s) / nch;
                    int t, kind, tm, tn;
                    G.get(j, t, sb, se, kind);
                    tile_coords(t, P.tiles_m, P.tiles_n, P.raster, tm, tn);
                    jc[s] = (2 * pi + s) % nch;
                    jrA[s] = tm * kPairTile + (int)rank * 128;
                    jrB[s] = tn * kPairTile + (int)rank * 128;
                }
                const int nh = (se - sb + CS - 1) / CS;
                for (int h = 0; h < nh && ok; ++h) {
                    const int k0 = sb + h * CS;
                    const int steps = min(CS, se - k0);
                    for (int s = 0; s < nj && ok; ++s) {
                        const int c = jc[s];
                        const int rowA = jrA[s];
                        const int rowB = jrB[s];
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
                int t, kind, sb, se;
                G.get((2 * pi) / nch, t, sb, se, kind);
                const int nh = (se - sb + CS - 1) / CS;
                for (int h = 0; h < nh && ok; ++h) {
                    const int steps = min(CS, se - (sb + h * CS));
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
            int jc[2], jslot[2], jtm[2], jtn[2], jkind[2], sb = 0, se = I.ksteps;
            for (int s = 0; s < nj; ++s) {
                const int j = (2 * pi + s) / nch;
                int t;
                G.get(j, t, sb, se, jkind[s]);
                tile_coords(t, P.tiles_m, P.tiles_n, P.raster, jtm[s], jtn[s]);
                jc[s] = (2 * pi + s) % nch;
                jslot[s] = G.digit_ord(j) & 1;
            }
            const int nh = (se - sb + CS - 1) / CS;
            for (int h = 0; h < nh && ok; ++h) {
                const bool last_chunk = (h == nh - 1);
                for (int s = 0; s < nj; ++s) {
                    const int c = jc[s];
                    const int slot = jslot[s];
                    const int kind = jkind[s];
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
                    const float uf = (float)I.u[c], uim = uf * im;
                    if (!last_chunk) {
                        epi_reduce(tbase, mf, im);
                    } else if (kind == 2) {
                        epi_partial(tbase, mf, im, sk_part_at(P, pair, rank, c) + row_off);
                    } else {
                        if (c == 0) {
                            if (!mbar_wait(&slot_empty[slot], sep[slot] ^ 1u, abort_flag, err, kDevTimeoutEpilogue)) {
                                ok = false;
                                break;
                            }
                            sep[slot] ^= 1u;
                        }
                        // a head: this channel's residues of every tail first
                        for (int tp = pair + G.rem; kind == 1 && tp < G.rem * G.split && ok; tp += G.rem)
                            ok = sk_wait(P.sk_flags + ((size_t(tp) * 2 + rank) * nch + c) * kEpiWarps + (warp - 2),
                                         abort_flag, err);
                        if (!ok) break;
                        unsigned char* dst = slot_row + size_t(c) * kTileM * kTileN;
                        const bool row_ok = (2 * jtm[s] + (int)rank) * kTileM + row_local < I.m;
                        const int col_lim = I.n - jtn[s] * kTileN - half * 128;
                        if (kind == 1)
                            epi_digits_sk(tbase, mf, im, uf, uim, dst, row_ok, col_lim, P, pair + G.rem,
                                          G.rem * G.split, G.rem, rank, c, row_off);
                        else
                            epi_digits(tbase, mf, im, uf, uim, dst, row_ok, col_lim);
                    }
                    tc_fence_before();
                    if (last_chunk && c == nch - 1) __threadfence_block();
                    __syncwarp();
                    if (lane == 0) {
                        if (leader)
                            mbar_arrive(&acc_empty[s]);
                        else
                            mbar_arrive_cluster(acc_empty_leader[s]);
                        if (last_chunk && c == nch - 1 && kind != 2) mbar_arrive(&slot_full[slot]);
                    }
                    if (last_chunk && kind == 2) {
                        // this warp's residues of channel c are out: release them to the head
                        __threadfence();
                        __syncwarp();
                        if (lane == 0)
                            st_release_gpu(P.sk_flags + ((size_t(pair) * 2 + rank) * nch + c) * kEpiWarps + (warp - 2),
                                           1);
                    }
                }
            }
        }
        const int nd = G.digit_tiles();
        if (ok && nd > 0) {
            // the CTA's last digit tile: take 8 of the 12 row shares of its reconstruction
            const int ti = nd - 1;
            int jl = nseg - 1;
            if (G.has_tail() && jl == G.ndp) --jl;  // a range that is one tail only: the last round-robin tile
            int t, sb, se, kind, tm, tn;
            G.get(jl, t, sb, se, kind);
            tile_coords(t, P.tiles_m, P.tiles_n, P.raster, tm, tn);
            uint4* kcw = kc + (1 + (warp - 2)) * kMaxChannels;
            stage_consts_warp(I, kcw, lane);
            if (mbar_wait(&slot_full[ti & 1], (uint32_t)(ti >> 1) & 1u, abort_flag, err, kDevTimeoutEpilogue))
                combine_block<false>(I, kcw, (2 * tm + (int)rank) * kTileM, tn * kTileN,
                              slot_base + size_t(ti & 1) * P.slot_stride, size_t(kTileM) * kTileN,
                              kCombineWarps + (warp - 2), kCombineWarps + kEpiWarps, lane);
        }
    } else {
        // ---------------------------------------------------- combine warps (both CTAs)
        const int cw = warp - kFirstCombineWarp;
        unsigned char* slot_base = P.slots + size_t(blockIdx.x) * 2 * P.slot_stride;
        uint32_t sfp[2] = {0u, 0u};
        const int nd = G.digit_tiles();
        if (nd > 0) stage_consts(I, kc, cw * 32 + lane);
        for (int j = 0, ti = 0; j < nseg; ++j) {
            int t, sb, se, kind, tm, tn;
            G.get(j, t, sb, se, kind);
            if (kind == 2) continue;
            const int slot = ti & 1;
            if (!mbar_wait(&slot_full[slot], sfp[slot], abort_flag, err, kDevTimeoutEpilogue)) break;
            sfp[slot] ^= 1u;
            tile_coords(t, P.tiles_m, P.tiles_n, P.raster, tm, tn);
            // rows of this CTA: the 128-row block 2 tm + rank
            combine_block<false>(I, kc, (2 * tm + (int)rank) * kTileM, tn * kTileN, slot_base + size_t(slot) * P.slot_stride,
                          size_t(kTileM) * kTileN, cw, ti == nd - 1 ? kCombineWarps + kEpiWarps : kCombineWarps,
                          lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&slot_empty[slot]);
            ++ti;
        }
    }

    tc_fence_before();
    __syncwarp();    // warps 0 and 1 reconverge before the aligned cluster barrier
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

cudaError_t launch_rns_gemm_grouped(const GroupGemmParams& prm, int grid, cudaStream_t s, bool int_out) {
    static bool attr_set = false, attr_set_int = false;
    if (!(int_out ? attr_set_int : attr_set)) {
        cudaError_t e = cudaFuncSetAttribute(int_out ? rns_gemm_grouped_int_kernel : rns_gemm_grouped_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        (int_out ? attr_set_int : attr_set) = true;
    }
    if (int_out)
        rns_gemm_grouped_int_kernel<<<grid, kThreads, kSmemBytes, s>>>(prm);
    else
        rns_gemm_grouped_kernel<<<grid, kThreads, kSmemBytes, s>>>(prm);
    return cudaGetLastError();
}

cudaError_t launch_rns_gemm_int(const CUtensorMap& mapA, const CUtensorMap& mapB, const RnsGemmParams& prm,
                                int grid, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(rns_gemm_int_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    rns_gemm_int_kernel<<<grid, kThreads, kSmemBytes, s>>>(mapA, mapB, prm);
    return cudaGetLastError();
}

}  // namespace ffgpu
