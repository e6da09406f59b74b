// Multi-modular products from one exact integer product.
//
// The paper's introduction motivates word-size finite-field routines by their
// use inside multi-modular (Chinese remainder) computations over Z, and
// section 7 names the Chinese remainder algorithm as the route beyond one
// word.  For integer matrices A (m x k) and B (k x n) whose entries are below
// 2^bits in magnitude, the products C_i = (A B) mod p_i for many primes p_i
// are all images of the one integer product X = A B.  This file computes X
// once, exactly -- the residues of A and B modulo the channel moduli (no
// reduction mod any prime), the channel products on the tensor cores, the
// reconstruction of X as a 64-bit integer in the combine warps (integer mode
// of the tensor-core kernel) -- and then writes X mod p_i for every prime with
// one memory-bound fan-out kernel.  The per-prime route repeats the whole
// product for each prime.
#include <algorithm>
#include <cstring>
#include <vector>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

typedef unsigned __int128 u128;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// u mod p for a magnitude u < 2^62: u_hi R + u_lo with Shoup products (each in
// [0, 2p)), folded to [0, p) -- 32-bit arithmetic only.
__device__ __forceinline__ uint32_t fan_mod(unsigned long long u, const FanPrime& f) {
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    uint32_t t1 = hi * f.R - __umulhi(hi, f.Rs) * f.p;
    t1 = min(t1, t1 - f.p);
    uint32_t t2 = lo - __umulhi(lo, f.one_s) * f.p;
    t2 = min(t2, t2 - f.p);
    const uint32_t t = t1 + t2;
    return min(t, t - f.p);
}

// X (int64, m x n, ldx) -> C_i = X mod p_i in [0, p_i), 4 columns per thread.
__global__ void __launch_bounds__(256) multimod_fanout_kernel(const long long* __restrict__ X, long long ldx, int m,
                                                              int n, const __grid_constant__ FanoutParams P) {
    const int n4 = (n + 3) / 4;
    const long long total = (long long)m * n4;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(g / n4);
        const int c0 = (int)(g - (long long)r * n4) * 4;
        const long long* src = X + (long long)r * ldx + c0;
        unsigned long long u[4];
        bool neg[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long v = (c0 + e < n) ? __ldg(src + e) : 0ll;
            neg[e] = v < 0;
            u[e] = neg[e] ? 0ull - (unsigned long long)v : (unsigned long long)v;
        }
        const bool full4 = c0 + 3 < n;
#pragma unroll 1
        for (int i = 0; i < P.nprimes; ++i) {
            const FanPrime f = P.pr[i];
            uint32_t out[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t t = fan_mod(u[e], f);
                out[e] = (neg[e] && t != 0u) ? f.p - t : t;
            }
            uint32_t* dst = P.C[i] + (long long)r * P.ldc + c0;
            if (full4 && P.vec_ok[i]) {
                *reinterpret_cast<uint4*>(dst) = make_uint4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (c0 + e < n) dst[e] = out[e];
            }
        }
    }
}

constexpr int kFanThreads = 256;

__device__ __forceinline__ int fan_find(const long long* __restrict__ begin, int n, long long b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Every instance of a wave: block -> instance by binary search over the
// prefix table; each thread 4 columns of one row, all primes.
__global__ void __launch_bounds__(kFanThreads) multimod_fanout_grouped_kernel(
    const FanInst* __restrict__ insts, const long long* __restrict__ block_begin, int n_inst,
    uint32_t* const* __restrict__ cptrs, const __grid_constant__ FanPrimes P) {
    const int i = fan_find(block_begin, n_inst, blockIdx.x);
    const FanInst F = insts[i];
    const int n4 = (F.n + 3) / 4;
    const long long g = (blockIdx.x - block_begin[i]) * (long long)kFanThreads + threadIdx.x;
    if (g >= (long long)F.m * n4) return;
    const int r = (int)(g / n4);
    const int c0 = (int)(g - (long long)r * n4) * 4;
    const long long* src = F.X + (long long)r * F.ldx + c0;
    unsigned long long u[4];
    bool neg[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const long long v = (c0 + e < F.n) ? __ldg(src + e) : 0ll;
        neg[e] = v < 0;
        u[e] = neg[e] ? 0ull - (unsigned long long)v : (unsigned long long)v;
    }
    const bool full4 = c0 + 3 < F.n;
#pragma unroll 1
    for (int q = 0; q < P.nprimes; ++q) {
        const FanPrime f = P.pr[q];
        uint32_t out[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t t = fan_mod(u[e], f);
            out[e] = (neg[e] && t != 0u) ? f.p - t : t;
        }
        uint32_t* dst = cptrs[F.cbase + q] + (long long)r * F.ldc + c0;
        if (full4 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
            *reinterpret_cast<uint4*>(dst) = make_uint4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c0 + e < F.n) dst[e] = out[e];
        }
    }
}

}  // namespace

long long multimod_fanout_blocks(int m, int n) {
    return ((long long)m * ((n + 3) / 4) + kFanThreads - 1) / kFanThreads;
}

cudaError_t launch_multimod_fanout_grouped(const FanInst* insts, const long long* block_begin, int n_inst,
                                           long long nblocks, uint32_t* const* cptrs, const FanPrimes& P,
                                           cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    multimod_fanout_grouped_kernel<<<(unsigned)nblocks, kFanThreads, 0, s>>>(insts, block_begin, n_inst, cptrs, P);
    return cudaGetLastError();
}

// Kernel view of an integer-mode product (see comb_row_int): the CRT weights
// M/m_c and M are needed only mod 2^64, because the exact product fits in
// int64 and the reconstruction is a ring computation mod 2^64.
void fill_inst_int(InstInfo& I, int64_t m, int64_t n, int64_t kp, const RnsPlan& pl, long long* X, int64_t ldx) {
    std::memset(&I, 0, sizeof(I));
    I.m = (int)m;
    I.n = (int)n;
    I.ksteps = (int)(kp / kTileK);
    I.chunk_steps = chunk_steps_for(pl);
    I.nch = pl.nch;
    I.direct = 0;
    I.vec_ok = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 2 == 0);
    I.p = pl.p;
    I.alpha = 1;
    I.beta = 0;
    I.int_out = 1;
    I.C = reinterpret_cast<uint32_t*>(X);
    I.ldc = 2 * ldx;  // in 32-bit words
    u128 M = 1;
    for (int c = 0; c < pl.nch; ++c) M *= pl.mod[c];
    unsigned long long sumMi = 0;
    uint32_t sumF = 0;
    for (int c = 0; c < pl.nch; ++c) {
        const uint32_t mc = pl.mod[c];
        const unsigned long long Mi = (unsigned long long)(M / mc);  // mod 2^64
        I.modf[c] = (float)mc;
        I.inv_m[c] = 1.0f / (float)mc;
        I.modu[c] = mc;
        I.u[c] = pl.u[c];
        I.Wa[c] = (uint32_t)Mi;
        I.Mhi[c] = (uint32_t)(Mi >> 32);
        I.fr[c] = ((1u << 14) + mc / 2) / mc;
        sumMi += Mi;
        sumF += I.fr[c];
    }
    I.Mfull = (unsigned long long)M;
    I.Xoff = 128ull * sumMi - 6ull * (unsigned long long)M;
    I.Finit = 6u * (1u << 14) + (1u << 13) - 128u * sumF;
}

ffgpu_status multimod_check(int64_t m, int64_t n, int64_t k, int bits, const void* A, int64_t lda, const void* B,
                            int64_t ldb, int nprimes, const uint32_t* primes, uint32_t* const* C, int64_t ldc) {
    if (m < 0 || n < 0 || k < 0 || m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > INT32_MAX / 2)
        return FFGPU_ERR_INVALID;
    if (bits < 1 || bits > 30) return FFGPU_ERR_INVALID;
    if (nprimes < 1 || nprimes > kMaxFanoutPrimes || !primes || !C) return FFGPU_ERR_INVALID;
    for (int i = 0; i < nprimes; ++i) {
        if (primes[i] < 2 || primes[i] > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
        if (m > 0 && n > 0 && !C[i]) return FFGPU_ERR_INVALID;
    }
    if (m == 0 || n == 0) return FFGPU_OK;
    if (ldc < n) return FFGPU_ERR_INVALID;
    if (k > 0 && (!A || !B || lda < k || ldb < n)) return FFGPU_ERR_INVALID;
    // the exact product must fit in int64 with a margin: k 2^(2 bits) < 2^62
    if (k > 0 && (2 * bits >= 62 || (uint64_t)k >= (1ull << (62 - 2 * bits)))) return FFGPU_ERR_INVALID;
    return FFGPU_OK;
}

// The plan's magnitude bound: 2^bits, at least 2^7 so that the plan is a
// residue system (a larger bound is still a valid one).
uint32_t multimod_plan_modulus(int bits) { return 2u << std::max(bits, 7); }

size_t multimod_ws_bytes(int64_t m, int64_t n, int64_t k, int bits, int sms) {
    if (m == 0 || n == 0) return 0;
    RnsPlan pl;
    make_plan(multimod_plan_modulus(bits), std::max<int64_t>(k, 1), pl);
    const int64_t kp = (std::max<int64_t>(k, 1) + kTileK - 1) / kTileK * kTileK;
    const int64_t tiles = ((m + kTileM - 1) / kTileM) * ((n + kTileN - 1) / kTileN);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
    const int64_t ldx = (n + 1) / 2 * 2;
    return align256(size_t(grid) * kSlotsPerCta * size_t(pl.nch) * kTileM * kTileN) +
           align256(size_t(pl.nch) * m * kp * 2) + align256(size_t(pl.nch) * n * kp * 2) +
           align256(size_t(m) * ldx * 8);
}

void fanout_params(int nprimes, const uint32_t* primes, uint32_t* const* C, int64_t ldc, FanoutParams& F) {
    std::memset(&F, 0, sizeof(F));
    F.nprimes = nprimes;
    F.ldc = ldc;
    for (int i = 0; i < nprimes; ++i) {
        F.pr[i] = fan_prime(primes[i]);
        F.C[i] = C[i];
        F.vec_ok[i] = ((reinterpret_cast<uintptr_t>(C[i]) & 15) == 0) && (ldc % 4 == 0);
    }
}

cudaError_t launch_multimod_fanout(const long long* X, long long ldx, int m, int n, const FanoutParams& F,
                                   cudaStream_t s) {
    const long long work = (long long)m * ((n + 3) / 4);
    int dev = 0;
    cudaGetDevice(&dev);
    const int grid = (int)std::min<long long>((work + 255) / 256, (long long)sm_count(dev) * 16);
    multimod_fanout_kernel<<<std::max(grid, 1), 256, 0, s>>>(X, ldx, m, n, F);
    return cudaGetLastError();
}

// Workspace of one exact integer product (planes and residue slots; the
// int64 result is the caller's).
size_t int_gemm_ws_bytes(int64_t m, int64_t n, int64_t k, int bits, int sms) {
    if (m == 0 || n == 0) return 0;
    RnsPlan pl;
    make_plan(multimod_plan_modulus(bits), std::max<int64_t>(k, 1), pl);
    const int64_t kp = (std::max<int64_t>(k, 1) + kTileK - 1) / kTileK * kTileK;
    const int64_t tiles = ((m + kTileM - 1) / kTileM) * ((n + kTileN - 1) / kTileN);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
    return align256(size_t(grid) * kSlotsPerCta * size_t(pl.nch) * kTileM * kTileN) +
           align256(size_t(pl.nch) * m * kp * 2) + align256(size_t(pl.nch) * n * kp * 2);
}

// The exact integer product X = A B (int32 words taken as they are, |entries|
// <= 2^bits, k 2^(2 bits) < 2^62) written to X (int64, ldx even and X 16-byte
// aligned for vector stores), or added to it when accumulate is set (the sum
// must stay below 2^63 in magnitude).  Conversions of both operands, then the
// integer-mode tensor-core kernel.
ffgpu_status int_gemm_run(int64_t m, int64_t n, int64_t k, int bits, const int32_t* A, int64_t lda,
                          const int32_t* B, int64_t ldb, long long* X, int64_t ldx, bool accumulate, void* ws,
                          size_t ws_bytes, int* err, cudaStream_t s) {
    if (m == 0 || n == 0 || k == 0) return FFGPU_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = sm_count(dev);
    RnsPlan pl;
    make_plan(multimod_plan_modulus(bits), k, pl);  // magnitudes up to 2^bits play the centred residues' part
    if (pl.mode != 2 || k > pl.k_slice) return FFGPU_ERR_INVALID;
    const int64_t kp = (k + kTileK - 1) / kTileK * kTileK;
    const int64_t tiles = ((m + kTileM - 1) / kTileM) * ((n + kTileN - 1) / kTileN);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
    unsigned char* w = static_cast<unsigned char*>(ws);
    const size_t o_slots = 0;
    const size_t o_A = o_slots + align256(size_t(grid) * kSlotsPerCta * size_t(pl.nch) * kTileM * kTileN);
    const size_t o_B = o_A + align256(size_t(pl.nch) * m * kp * 2);
    if (ws_bytes < o_B + align256(size_t(pl.nch) * n * kp * 2)) return FFGPU_ERR_NOMEM;

    ConvertParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.p = pl.p;
    cp.half_p = pl.p / 2;
    cp.mu32 = 0xFFFFFFFFu / pl.p;
    cp.nch = pl.nch;
    cp.direct = 0;
    cp.signed_input = 1;
    for (int c = 0; c < pl.nch; ++c) {
        cp.mod[c] = pl.mod[c];
        cp.magic32[c] = (uint32_t)(((1ull << 39) + pl.mod[c] - 1) / pl.mod[c]);
    }
    if (timed_launch("convert_rows", s, [&] {
            return launch_convert_rows(reinterpret_cast<const uint32_t*>(A), lda, (int)m, (int)k, (int)kp, cp,
                                       w + o_A, s);
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    if (timed_launch("convert_transpose", s, [&] {
            return launch_convert_transpose(reinterpret_cast<const uint32_t*>(B), ldb, (int)k, (int)n, (int)kp, cp,
                                            w + o_B, s);
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    CUtensorMap mapA, mapB;
    if (!encode_planes(&mapA, w + o_A, kp, m, pl.nch, kTileM) || !encode_planes(&mapB, w + o_B, kp, n, pl.nch, kTileN))
        return FFGPU_ERR_CUDA;
    RnsGemmParams P;
    std::memset(&P, 0, sizeof(P));
    fill_inst_int(P.inst, m, n, kp, pl, X, ldx);
    P.inst.beta = accumulate ? 1u : 0u;  // integer mode: add the int64 values already in X
    P.tiles_m = (int)((m + kTileM - 1) / kTileM);
    P.tiles_n = (int)((n + kTileN - 1) / kTileN);
    P.num_tiles = P.tiles_m * P.tiles_n;
    P.slots = w + o_slots;
    P.slot_stride = size_t(pl.nch) * kTileM * kTileN;
    P.err = err;
    P.raster = kRasterRows;
    return timed_launch("rns_gemm_int", s, [&] { return launch_rns_gemm_int(mapA, mapB, P, grid, s); }) ==
                   cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

ffgpu_status multimod_run(int64_t m, int64_t n, int64_t k, int bits, const int32_t* A, int64_t lda, const int32_t* B,
                          int64_t ldb, int nprimes, const uint32_t* primes, uint32_t* const* C, int64_t ldc,
                          void* ws, size_t ws_bytes, int* err, cudaStream_t s) {
    if (m == 0 || n == 0) return FFGPU_OK;
    FanoutParams F;
    fanout_params(nprimes, primes, C, ldc, F);
    const int64_t ldx = (n + 1) / 2 * 2;
    if (k == 0) {  // X = 0
        if (cudaMemsetAsync(ws, 0, size_t(m) * ldx * 8, s) != cudaSuccess) return FFGPU_ERR_CUDA;
        return timed_launch("multimod_fanout", s, [&] {
                   return launch_multimod_fanout(static_cast<const long long*>(ws), ldx, (int)m, (int)n, F, s);
               }) == cudaSuccess
                   ? FFGPU_OK
                   : FFGPU_ERR_CUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    // the product's planes and slots first, then the int64 result (the layout
    // multimod_ws_bytes sizes)
    const size_t o_X = int_gemm_ws_bytes(m, n, k, bits, sm_count(dev));
    if (ws_bytes < o_X + align256(size_t(m) * ldx * 8)) return FFGPU_ERR_NOMEM;
    long long* X = reinterpret_cast<long long*>(static_cast<unsigned char*>(ws) + o_X);
    const ffgpu_status st = int_gemm_run(m, n, k, bits, A, lda, B, ldb, X, ldx, false, ws, o_X, err, s);
    if (st != FFGPU_OK) return st;
    return timed_launch("multimod_fanout", s, [&] {
               return launch_multimod_fanout(X, ldx, (int)m, (int)n, F, s);
           }) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

}  // namespace ffgpu
