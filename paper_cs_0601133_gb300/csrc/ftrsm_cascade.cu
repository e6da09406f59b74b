// ftrsm by the double cascade of section 4.3: Algorithm 2
// (trsm-rec-BLAS-delayed) over Algorithm 3 (trsm-partial-delayed).
//
// Every variant (side, uplo, diag) is first mapped onto one system, unit lower
// triangular with the right-hand sides as columns, T'' Y = W:
//   * side R is transposed (X T = B  <=>  T^T X^T = B^T),
//   * an upper triangle is turned into a lower one by reversing the order of
//     rows and columns,
//   * a non-unit diagonal is normalised away (section 4.2: T = D U with U unit
//     diagonal; here row i of the system is multiplied by t_ii^{-1}, so only
//     ring operations remain), alpha folded into the same scaling of W.
// The solve then follows the paper's two cascades:
//   Algorithm 2: W is cut into blocks of t_split rows.  Each block is solved
//     by Algorithm 3, reduced mod p, and the rows below it are updated with
//     one fgemm mod p (W_rest <- W_rest - V_i X_i).
//   Algorithm 3 (a block of at most t_update rows): the block's right-hand
//     sides are held over Z as int64 (balanced residues of W to start with);
//     the block is split in two, the first half solved, the second half's
//     right-hand sides updated over Z with NO reduction (B_2 <- B_2 - A_21 X_1,
//     an exact integer product on the tensor cores, added to the int64
//     values), then the second half solved.  Below 128 rows a panel kernel
//     finishes the recursion on the CUDA cores: leaves of t_del rows, each
//     reduced mod p ("B = B mod p"), solved over Z in int64 with no
//     reduction ("dtrsm"), reduced mod p again ("X = X mod p"), and the
//     remaining rows of the panel updated over Z by the leaf's solution.
// Bounds (63-bit signed carrier, balanced residues |x| <= h = floor(p/2)):
//   t_del    largest n with h (h+1)^n < 2^63 (eq. trsmboundcen, exponent n):
//            a leaf's solution over Z stays within int64 (Corollary 4.5);
//   t_update largest t with t h^2 + h < 2^62: a right-hand side that starts
//            at |b| <= h and receives t products of residues stays below
//            2^62 (eq. 2 with one term reserved, as the paper's t_update
//            column reads), also the exact product's own limit;
//   t_split  floor(t_update / t_del) t_del (Algorithm 2).
// For large p the blocks are small (p = 2^31 - 1: t_del = 1, t_split = 2):
// the reductions the paper delays are then needed after almost every step,
// which is the regime where it reports the algorithm's speed dropping.
#include <algorithm>
#include <cstring>

#include "devutil.cuh"
#include "internal.h"

namespace ffgpu {

namespace {

typedef unsigned __int128 u128;

constexpr int kPanel = 128;        // rows a panel kernel solves
constexpr int kPanelCols = 32;     // right-hand sides per CTA (one per lane)
constexpr int kPanelThreads = 256; // 8 warps: warp w updates rows r = w mod 8
constexpr int kTile = 32;          // transposing copies

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

// Balanced residue of a signed 64-bit integer (|z| < 2^63): z mod p in
// (-p/2, p/2], the centred representation of section 2.1.1.
__device__ __forceinline__ long long bal_mod(long long z, uint32_t p, unsigned long long mu) {
    const bool neg = z < 0;
    const unsigned long long u = neg ? 0ull - (unsigned long long)z : (unsigned long long)z;
    uint32_t r = mod_u64(u, p, mu);
    if (neg && r != 0u) r = p - r;
    return r > p / 2 ? (long long)r - (long long)p : (long long)r;
}

// Index of the source entry behind row i of the working system: rows (and
// columns) are reversed for an upper triangle.
__device__ __forceinline__ int src_index(int i, int sz, int rev) { return rev ? sz - 1 - i : i; }

// d[i] = inverse of the diagonal entry behind working row i (1 for a unit
// diagonal); a non-invertible entry sets kDevSingular.
__global__ void casc_diag_kernel(const uint32_t* __restrict__ T, long long ldt, int sz, int rev, int unit, uint32_t p,
                                 unsigned long long mu, uint32_t* __restrict__ d, int* err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sz; i += gridDim.x * blockDim.x) {
        if (unit) {
            d[i] = 1u;
            continue;
        }
        const int a = src_index(i, sz, rev);
        const uint32_t v = inv_mod_dev(mod_u64(__ldg(T + (long long)a * ldt + a), p, mu), p);
        if (v == 0u) atomicCAS(err, 0, (int)kDevSingular);
        d[i] = v;
    }
}

// The strictly lower part of the working triangle, T''(i, j) = d_i T(src),
// as negated balanced int32 (Tn, for the products over Z) and, when Tc is not
// null, as canonical residues (for Algorithm 2's updates mod p).  One 32 x 32
// tile of (i, j) per CTA, through shared memory when the source is read
// transposed (side R), so that both reads and writes are coalesced.
__global__ void __launch_bounds__(kTile * 8) casc_prep_t_kernel(const uint32_t* __restrict__ T, long long ldt, int sz,
                                                                 int rev, int trans, uint32_t p, unsigned long long mu,
                                                                 const uint32_t* __restrict__ d, int32_t* __restrict__ Tn,
                                                                 uint32_t* __restrict__ Tc) {
    __shared__ uint32_t tile[kTile][kTile + 1];
    const int I0 = blockIdx.y * kTile, J0 = blockIdx.x * kTile;
    if (J0 > I0 + kTile - 1) return;  // entirely above the diagonal: never read
    const int tx = threadIdx.x & (kTile - 1), ty = threadIdx.x / kTile;
    for (int yy = ty; yy < kTile; yy += 8) {
        uint32_t v = 0u;
        if (trans) {  // element (i = I0 + tx, j = J0 + yy) is T[b(j)][a(i)]: contiguous in tx
            const int i = I0 + tx, j = J0 + yy;
            if (i < sz && j < sz && j < i)
                v = __ldg(T + (long long)src_index(j, sz, rev) * ldt + src_index(i, sz, rev));
            tile[yy][tx] = v;  // tile[j - J0][i - I0]
        } else {      // element (i = I0 + yy, j = J0 + tx) is T[a(i)][b(j)]
            const int i = I0 + yy, j = J0 + tx;
            if (i < sz && j < sz && j < i)
                v = __ldg(T + (long long)src_index(i, sz, rev) * ldt + src_index(j, sz, rev));
            tile[tx][yy] = v;  // tile[j - J0][i - I0]
        }
    }
    __syncthreads();
    const uint32_t h = p / 2;
    for (int yy = ty; yy < kTile; yy += 8) {
        const int i = I0 + yy, j = J0 + tx;
        if (i >= sz || j >= i) continue;
        const uint32_t c = mod_u64((unsigned long long)mod_u64(tile[tx][yy], p, mu) * d[i], p, mu);
        const long long bal = c > h ? (long long)c - (long long)p : (long long)c;
        Tn[(long long)i * sz + j] = (int32_t)(-bal);
        if (Tc) Tc[(long long)i * sz + j] = c;
    }
}

// W (sz x N, row-major) from B: row i of W is row a(i) of B (side L) or
// column a(i) of B (side R), times alpha d_i mod p.  dir = 0: B -> W;
// dir = 1: W -> B (the solution written back, no scaling).
__global__ void __launch_bounds__(kTile * 8) casc_move_b_kernel(uint32_t* __restrict__ B, long long ldb, int sz, int N,
                                                                 int rev, int trans, uint32_t p, unsigned long long mu,
                                                                 uint32_t alpha, const uint32_t* __restrict__ d,
                                                                 uint32_t* __restrict__ W, int dir) {
    __shared__ uint32_t tile[kTile][kTile + 1];
    const int I0 = blockIdx.y * kTile, C0 = blockIdx.x * kTile;  // W rows [I0, I0+32), columns [C0, C0+32)
    const int tx = threadIdx.x & (kTile - 1), ty = threadIdx.x / kTile;
    if (!trans) {  // B row a(i), contiguous in the column index
        for (int yy = ty; yy < kTile; yy += 8) {
            const int i = I0 + yy, c = C0 + tx;
            if (i >= sz || c >= N) continue;
            uint32_t* bp = B + (long long)src_index(i, sz, rev) * ldb + c;
            uint32_t* wp = W + (long long)i * N + c;
            if (dir == 0) {
                const uint32_t s = mod_u64((unsigned long long)alpha * d[i], p, mu);
                *wp = mod_u64((unsigned long long)mod_u64(*bp, p, mu) * s, p, mu);
            } else {
                *bp = *wp;
            }
        }
        return;
    }
    // side R: W(i, c) is B[c][a(i)]; B is read / written contiguous in i
    if (dir == 0) {
        for (int yy = ty; yy < kTile; yy += 8) {
            const int c = C0 + yy, i = I0 + tx;
            tile[yy][tx] = (c < N && i < sz) ? B[(long long)c * ldb + src_index(i, sz, rev)] : 0u;
        }
        __syncthreads();
        for (int yy = ty; yy < kTile; yy += 8) {
            const int i = I0 + yy, c = C0 + tx;
            if (i >= sz || c >= N) continue;
            const uint32_t s = mod_u64((unsigned long long)alpha * d[i], p, mu);
            W[(long long)i * N + c] = mod_u64((unsigned long long)mod_u64(tile[tx][yy], p, mu) * s, p, mu);
        }
    } else {
        for (int yy = ty; yy < kTile; yy += 8) {
            const int i = I0 + yy, c = C0 + tx;
            tile[yy][tx] = (i < sz && c < N) ? W[(long long)i * N + c] : 0u;
        }
        __syncthreads();
        for (int yy = ty; yy < kTile; yy += 8) {
            const int c = C0 + yy, i = I0 + tx;
            if (c < N && i < sz) B[(long long)c * ldb + src_index(i, sz, rev)] = tile[tx][yy];
        }
    }
}

// A block's right-hand sides over Z: Z[r][c] = the balanced residue of W[r][c].
__global__ void casc_to_z_kernel(const uint32_t* __restrict__ W, int rows, int N, uint32_t p,
                                 long long* __restrict__ Z, long long ldz) {
    const long long total = (long long)rows * N;
    const uint32_t h = p / 2;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(g / N), c = (int)(g - (long long)r * N);
        const uint32_t w = W[g];
        Z[(long long)r * ldz + c] = w > h ? (long long)w - (long long)p : (long long)w;
    }
}

// The end of Algorithm 3's recursion for one panel of P <= kPanel rows
// (absolute rows [r0, r0 + P) of the working triangle) and 32 right-hand
// sides per CTA.  Z holds the panel's right-hand sides over Z (int64, all
// updates from outside the panel already added, |z| < 2^62).  Leaves of td
// rows in order; for each: its rows reduced mod p (balanced), solved over Z
// by forward substitution with no reduction (warp 0, one lane per right-hand
// side; |x| < 2^63 by t_del), reduced mod p; then every later row of the
// panel updated over Z with the leaf's reduced solution (all 8 warps).  Writes
// the solution as canonical residues (W) and balanced int32 (Xz, the operand
// of the next products over Z).
__global__ void __launch_bounds__(kPanelThreads) casc_panel_kernel(const int32_t* __restrict__ Tn, long long ldt,
                                                                   int r0, int P, const long long* __restrict__ Z,
                                                                   long long ldz, uint32_t* __restrict__ W,
                                                                   int32_t* __restrict__ Xz, int N, int td,
                                                                   uint32_t p, unsigned long long mu) {
    extern __shared__ unsigned char smem[];
    long long* Zs = reinterpret_cast<long long*>(smem);                        // [kPanel][32]
    int32_t* Xs = reinterpret_cast<int32_t*>(Zs + kPanel * kPanelCols);         // [kPanel][32]
    int32_t* Ts = Xs + kPanel * kPanelCols;                                     // [kPanel][kPanel]
    const int tx = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int col = blockIdx.x * kPanelCols + tx;
    const bool valid = col < N;
    for (int r = g; r < P; r += kPanelThreads / 32) Zs[r * kPanelCols + tx] = valid ? Z[(long long)r * ldz + col] : 0ll;
    for (int idx = threadIdx.x; idx < P * P; idx += kPanelThreads) {
        const int r = idx / P, j = idx - r * P;
        Ts[r * kPanel + j] = j < r ? __ldg(Tn + (long long)(r0 + r) * ldt + r0 + j) : 0;
    }
    __syncthreads();
    for (int a = 0; a < P; a += td) {
        const int e = min(a + td, P);
        if (g == 0) {
            // the leaf: B = B mod p, X = T^{-1} B over Z, X = X mod p
            for (int i = a; i < e; ++i) {
                long long x = bal_mod(Zs[i * kPanelCols + tx], p, mu);
                for (int j = a; j < i; ++j) x += (long long)Ts[i * kPanel + j] * Zs[j * kPanelCols + tx];
                Zs[i * kPanelCols + tx] = x;
            }
            for (int i = a; i < e; ++i) {
                const long long x = bal_mod(Zs[i * kPanelCols + tx], p, mu);
                Zs[i * kPanelCols + tx] = x;
                Xs[i * kPanelCols + tx] = (int32_t)x;
            }
        }
        __syncthreads();
        // the rest of the panel over Z: z_r += sum_j (-T_rj) x_j, no reduction
        for (int r = e + g; r < P; r += kPanelThreads / 32) {
            long long acc = Zs[r * kPanelCols + tx];
            for (int j = a; j < e; ++j) acc += (long long)Ts[r * kPanel + j] * (long long)Xs[j * kPanelCols + tx];
            Zs[r * kPanelCols + tx] = acc;
        }
        __syncthreads();
    }
    if (!valid) return;
    for (int r = g; r < P; r += kPanelThreads / 32) {
        const int32_t x = Xs[r * kPanelCols + tx];
        W[(long long)r * N + col] = x < 0 ? (uint32_t)(x + (int32_t)p) : (uint32_t)x;
        Xz[(long long)r * N + col] = x;
    }
}

constexpr size_t kPanelSmem = size_t(kPanel) * kPanelCols * 8 + size_t(kPanel) * kPanelCols * 4 +
                              size_t(kPanel) * kPanel * 4;

struct CascLayout {
    int64_t sz, N, S, ldz;
    size_t d, tn, tc, w, z, xz, prod, total;
    bool need_tc;
};

CascLayout casc_layout(int side, int64_t m, int64_t n, uint32_t p, int sms) {
    CascLayout L;
    L.sz = side == 0 ? m : n;
    L.N = side == 0 ? n : m;
    const CascadeParams cp = cascade_params(p);
    L.S = std::min<int64_t>(cp.t_split, L.sz);
    L.ldz = (L.N + 1) / 2 * 2;
    L.need_tc = L.S < L.sz;
    const int bits = bit_length(p / 2);
    L.d = 0;
    L.tn = L.d + align256(size_t(L.sz) * 4);
    L.tc = L.tn + align256(size_t(L.sz) * L.sz * 4);
    L.w = L.tc + (L.need_tc ? align256(size_t(L.sz) * L.sz * 4) : 0);
    L.z = L.w + align256(size_t(L.sz) * L.N * 4);
    L.xz = L.z + align256(size_t(L.S) * L.ldz * 8);
    L.prod = L.xz + align256(size_t(L.S) * L.N * 4);
    size_t pw = L.S > kPanel ? int_gemm_ws_bytes(L.S, L.N, L.S, bits, sms) : 0;
    for (int64_t b0 = 0; b0 + L.S < L.sz; b0 += L.S)  // Algorithm 2's updates, one per block but the last
        pw = std::max(pw, fgemm_ws_bytes(L.sz - b0 - L.S, L.N, L.S, p, sms));
    L.total = L.prod + align256(pw);
    return L;
}

struct CascCtx {
    const CascLayout* L;
    int bits, td;
    uint32_t p;
    unsigned long long mu;
    const int32_t* Tn;
    uint32_t* W;
    long long* Z;   // rows of the current block
    int32_t* Xz;    // rows of the current block
    int64_t b0;     // first row of the current block
    void* ws;
    size_t ws_bytes;
    int* err;
    cudaStream_t s;
};

// Algorithm 3 on the rows [r0, r0 + S) of the current block.
ffgpu_status partial_delayed(const CascCtx& c, int64_t r0, int64_t S) {
    const CascLayout& L = *c.L;
    if (S <= kPanel) {
        const int grid = (int)((L.N + kPanelCols - 1) / kPanelCols);
        return timed_launch("trsm_cascade_panel", c.s, [&] {
                   casc_panel_kernel<<<grid, kPanelThreads, kPanelSmem, c.s>>>(
                       c.Tn, L.sz, (int)r0, (int)S, c.Z + (r0 - c.b0) * L.ldz, L.ldz, c.W + r0 * L.N,
                       c.Xz + (r0 - c.b0) * L.N, (int)L.N, c.td, c.p, c.mu);
                   return cudaGetLastError();
               }) == cudaSuccess
                   ? FFGPU_OK
                   : FFGPU_ERR_CUDA;
    }
    const int64_t panels = (S + kPanel - 1) / kPanel;
    const int64_t h = (panels / 2) * kPanel;
    ffgpu_status st = partial_delayed(c, r0, h);
    if (st != FFGPU_OK) return st;
    // B_2 <- B_2 - A_21 X_1 over Z (Tn holds -A), added to the int64 values
    st = int_gemm_run(S - h, L.N, h, c.bits, c.Tn + (r0 + h) * L.sz + r0, L.sz, c.Xz + (r0 - c.b0) * L.N, L.N,
                      c.Z + (r0 + h - c.b0) * L.ldz, L.ldz, true, c.ws, c.ws_bytes, c.err, c.s);
    if (st != FFGPU_OK) return st;
    return partial_delayed(c, r0 + h, S - h);
}

}  // namespace

CascadeParams cascade_params(uint32_t p) {
    CascadeParams cp;
    const u128 h = p / 2;  // the largest centred magnitude (1 for p = 2)
    const u128 lim63 = (u128)1 << 63, lim62 = (u128)1 << 62;
    int64_t n = 0;
    u128 v = h;
    while (n < kPanel && v * (h + 1) < lim63) {
        v *= h + 1;
        ++n;
    }
    cp.t_del = std::max<int64_t>(n, 1);
    const u128 t = (lim62 - 1 - h) / (h * h);
    cp.t_update = t > (u128)INT32_MAX ? (int64_t)INT32_MAX : (int64_t)t;
    cp.t_split = std::max<int64_t>(cp.t_update / cp.t_del * cp.t_del, 1);
    return cp;
}

size_t cascade_ws_bytes(int side, int64_t m, int64_t n, uint32_t p, int sms) {
    return casc_layout(side, m, n, p, sms).total;
}

ffgpu_status cascade_run(int side, int uplo, int diag, int64_t m, int64_t n, uint32_t p, uint32_t alpha,
                         const uint32_t* T, int64_t ldt, uint32_t* B, int64_t ldb, void* ws, size_t ws_bytes,
                         int* err, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    const CascLayout L = casc_layout(side, m, n, p, sm_count(dev));
    if (ws_bytes < L.total) return FFGPU_ERR_NOMEM;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(casc_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmem) !=
            cudaSuccess)
            return FFGPU_ERR_CUDA;
        attr_set = true;
    }
    unsigned char* w = static_cast<unsigned char*>(ws);
    uint32_t* d = reinterpret_cast<uint32_t*>(w + L.d);
    int32_t* Tn = reinterpret_cast<int32_t*>(w + L.tn);
    uint32_t* Tc = L.need_tc ? reinterpret_cast<uint32_t*>(w + L.tc) : nullptr;
    uint32_t* W = reinterpret_cast<uint32_t*>(w + L.w);
    // working orientation: side R transposed, an upper triangle (after the
    // transposition) reversed into a lower one
    const int trans = side == 1;
    const int rev = (uplo == 1) != (side == 1);
    const unsigned long long mu = ~0ull / p;
    const int sz = (int)L.sz, N = (int)L.N;
    const CascadeParams cp = cascade_params(p);
    const dim3 tgrid((unsigned)((sz + kTile - 1) / kTile), (unsigned)((sz + kTile - 1) / kTile));
    const dim3 bgrid((unsigned)((N + kTile - 1) / kTile), (unsigned)((sz + kTile - 1) / kTile));
    if (timed_launch("trsm_cascade_prep", s, [&] {
            casc_diag_kernel<<<(sz + 255) / 256, 256, 0, s>>>(T, ldt, sz, rev, diag, p, mu, d, err);
            casc_prep_t_kernel<<<tgrid, kTile * 8, 0, s>>>(T, ldt, sz, rev, trans, p, mu, d, Tn, Tc);
            casc_move_b_kernel<<<bgrid, kTile * 8, 0, s>>>(B, ldb, sz, N, rev, trans, p, mu, alpha % p, d, W, 0);
            return cudaGetLastError();
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    CascCtx c;
    c.L = &L;
    c.bits = bit_length(p / 2);
    c.td = (int)cp.t_del;
    c.p = p;
    c.mu = mu;
    c.Tn = Tn;
    c.W = W;
    c.Z = reinterpret_cast<long long*>(w + L.z);
    c.Xz = reinterpret_cast<int32_t*>(w + L.xz);
    c.ws = w + L.prod;
    c.ws_bytes = ws_bytes - L.prod;
    c.err = err;
    c.s = s;
    // Algorithm 2: blocks of t_split rows
    for (int64_t b0 = 0; b0 < sz; b0 += L.S) {
        const int64_t S = std::min<int64_t>(L.S, sz - b0);
        c.b0 = b0;
        const long long total = S * (long long)N;
        if (timed_launch("trsm_cascade_to_z", s, [&] {
                casc_to_z_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 65535), 256, 0, s>>>(
                    W + b0 * N, (int)S, N, p, c.Z, L.ldz);
                return cudaGetLastError();
            }) != cudaSuccess)
            return FFGPU_ERR_CUDA;
        ffgpu_status st = partial_delayed(c, b0, S);  // X_i, reduced mod p in W
        if (st != FFGPU_OK) return st;
        const int64_t rest = sz - b0 - S;
        if (rest > 0) {  // W_rest <- W_rest - V_i X_i mod p
            st = fgemm_run(rest, N, S, p, p - 1, Tc + (b0 + S) * sz + b0, sz, W + b0 * N, N, 1, W + (b0 + S) * N, N,
                           c.ws, c.ws_bytes, err, s, 0, false);
            if (st != FFGPU_OK) return st;
        }
    }
    return timed_launch("trsm_cascade_unprep", s, [&] {
               casc_move_b_kernel<<<bgrid, kTile * 8, 0, s>>>(B, ldb, sz, N, rev, trans, p, mu, 1u, d, W, 1);
               return cudaGetLastError();
           }) == cudaSuccess
               ? FFGPU_OK
               : FFGPU_ERR_CUDA;
}

}  // namespace ffgpu

using namespace ffgpu;

extern "C" ffgpu_status ffgpu_ftrsm_cascade_params(uint32_t p, int64_t* t_del, int64_t* t_update, int64_t* t_split) {
    if (p < 2 || p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
    if (!t_del || !t_update || !t_split) return FFGPU_ERR_INVALID;
    const CascadeParams cp = cascade_params(p);
    *t_del = cp.t_del;
    *t_update = cp.t_update;
    *t_split = cp.t_split;
    return FFGPU_OK;
}
