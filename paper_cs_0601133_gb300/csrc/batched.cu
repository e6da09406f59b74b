// Batched fgemm: many independent products of different shapes and moduli in
// one grouped conversion per operand and one persistent tensor-core launch per
// wave.  Host side only: plans, placement of every instance's channel planes in
// per-k pools, cost-balanced job lists, tables copied to the device.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <queue>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#include "internal.h"

namespace ffgpu {

namespace {

// Channel-plane bytes per wave (FFGPU_BATCH_WAVE_GB overrides): fewer, larger
// waves mean fewer launch tails and table uploads.
size_t wave_plane_budget() {
    static size_t v = 0;
    if (v == 0) {
        size_t gb = 12;
        if (const char* e = std::getenv("FFGPU_BATCH_WAVE_GB")) {
            const long long x = std::atoll(e);
            if (x >= 1 && x <= 200) gb = (size_t)x;
        }
        v = gb << 30;
    }
    return v;
}

// Pinned, double-buffered host staging for the per-wave tables: the copy of
// wave w runs while the host fills wave w+1, and a buffer is rewritten only
// after the event recorded behind its copy has completed.
struct StageBuf {
    unsigned char* p = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
};
// One pair per device: a buffer's event belongs to the device whose stream
// records it.
struct StageSet {
    StageBuf buf[2];
    int next = 0;
};
std::mutex g_stage_mu;  // held from stage_get to stage_done
std::map<int, StageSet> g_stage_sets;

StageSet& stage_set() {
    int dev = 0;
    cudaGetDevice(&dev);
    return g_stage_sets[dev];
}

unsigned char* stage_get(size_t bytes, int* idx) {
    StageSet& S = stage_set();
    StageBuf& b = S.buf[S.next];
    if (b.pending) {
        cudaEventSynchronize(b.ev);
        b.pending = false;
    }
    if (!b.ev && cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        b.ev = nullptr;
        return nullptr;
    }
    if (b.bytes < bytes) {
        if (b.p) cudaFreeHost(b.p);
        b.p = nullptr;
        b.bytes = 0;
        const size_t want = std::max(bytes, size_t(1) << 20);
        if (cudaHostAlloc(reinterpret_cast<void**>(&b.p), want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return nullptr;
        }
        b.bytes = want;
    }
    *idx = S.next;
    S.next ^= 1;
    return b.p;
}

// Called with g_stage_mu held, right after the copy from buffer idx was
// enqueued on s.  If the event cannot be recorded (for instance on a stream of
// another device), the copy is waited for here instead, so that the next
// stage_get cannot overwrite a buffer a copy still reads.
void stage_done(int idx, cudaStream_t s) {
    StageBuf& b = stage_set().buf[idx];
    if (cudaEventRecord(b.ev, s) == cudaSuccess) {
        b.pending = true;
        return;
    }
    cudaGetLastError();
    cudaStreamSynchronize(s);
    b.pending = false;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// One tensor-core instance of a wave.  mpad / npad: the rows and columns its
// tiles cover (whole 128 x 256 tiles); mst / nst: the plane rows it stores
// (m and n rounded to 8).  A tile that reaches past the stored rows reads the
// next instance's planes (or the pool's zero fill): those rows and columns
// of the tile are never reconstructed, so only the inner dimension's padding
// must be zeros -- and the conversions write it.
struct BInst {
    const ffgpu_fgemm_desc* d;
    RnsPlan pl;
    int64_t kp, mpad, npad, mst, nst;
    int bucket;
    int64_t rowA, rowB;
};

struct Bucket {
    int64_t kp;
    int nch;
    int64_t rowsA, rowsB;
    size_t offA, offB;  // byte offsets of the pools from the plane base
};

// Host plan of one wave: pools by padded inner length, cost-balanced job
// lists, and the layout of the two device regions it needs -- the planes
// (residue slots, then the pools) and the tables (tensor maps, instances, jobs,
// conversion jobs, block prefix sums).
struct WaveLayout {
    std::vector<Bucket> buckets;
    std::vector<GroupJob> jobs;
    std::vector<int> cta_begin;
    int grid = 1;
    size_t plane_bytes = 0;
    size_t t_inst = 0, t_jobs = 0, t_cta = 0, t_convA = 0, t_convB = 0, t_bbA = 0, t_bbB = 0, tab_bytes = 0;
    long long nbA = 0, nbB = 0;  // conversion blocks
    // integer mode: per-instance int64 results (in the plane region) and the fan-out tables
    std::vector<size_t> xoff;
    size_t t_fan = 0, t_fanbb = 0, t_cptr = 0;
    long long nbF = 0;
};

int64_t x_ld(int64_t n) { return (n + 1) / 2 * 2; }

void layout_wave(std::vector<BInst>& w, int sms, WaveLayout& L, const MultiCtx* mc) {
    std::unordered_map<int64_t, int> bucket_of;
    for (auto& b : w) {
        int idx;
        auto it = bucket_of.find(b.kp);
        if (it == bucket_of.end()) {
            L.buckets.push_back(Bucket{b.kp, 0, 0, 0, 0, 0});
            idx = (int)L.buckets.size() - 1;
            bucket_of.emplace(b.kp, idx);
        } else {
            idx = it->second;
        }
        Bucket& B = L.buckets[idx];
        b.bucket = idx;
        B.nch = std::max(B.nch, b.pl.nch);
        b.rowA = B.rowsA;
        b.rowB = B.rowsB;
        B.rowsA += b.mst;
        B.rowsB += b.nst;
    }
    // tiles and their cost (channels x k-steps), longest first onto the least-loaded CTA
    struct Tile {
        int inst, tm, tn;
        double cost;
    };
    std::vector<Tile> tiles;
    for (size_t i = 0; i < w.size(); ++i) {
        const auto& b = w[i];
        const int tmn = (int)(b.mpad / kTileM), tnn = (int)(b.npad / kTileN);
        const double cost = (double)b.pl.nch * (double)(b.kp / kTileK) + 4.0;
        for (int tm = 0; tm < tmn; ++tm)
            for (int tn = 0; tn < tnn; ++tn) tiles.push_back(Tile{(int)i, tm, tn, cost});
    }
    L.grid = (int)std::max<size_t>(1, std::min<size_t>(tiles.size(), (size_t)sms));
    std::stable_sort(tiles.begin(), tiles.end(), [](const Tile& a, const Tile& b) { return a.cost > b.cost; });
    std::vector<std::vector<int>> per_cta(L.grid);
    {
        typedef std::pair<double, int> Load;
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int c = 0; c < L.grid; ++c) heap.push(Load(0.0, c));
        for (size_t t = 0; t < tiles.size(); ++t) {
            Load l = heap.top();
            heap.pop();
            per_cta[l.second].push_back((int)t);
            l.first += tiles[t].cost;
            heap.push(l);
        }
    }
    L.cta_begin.assign(L.grid + 1, 0);
    for (int c = 0; c < L.grid; ++c) {
        L.cta_begin[c] = (int)L.jobs.size();
        uint32_t parity = 0;
        for (int t : per_cta[c]) {
            const Tile& T = tiles[t];
            const BInst& b = w[T.inst];
            const int ksteps = (int)(b.kp / kTileK);
            const int cs = chunk_steps_for(b.pl);
            for (int ch = 0; ch < b.pl.nch; ++ch) {
                GroupJob g;
                g.inst = T.inst;
                g.tmtn = (uint32_t)T.tm | ((uint32_t)T.tn << 16);
                g.cfg = (uint32_t)ch | (parity << 8) | ((uint32_t)b.pl.nch << 12) | ((uint32_t)b.bucket << 16);
                g.modc = b.pl.mod[ch] | (b.pl.u[ch] << 8) | ((uint32_t)cs << 16);
                g.ksteps = ksteps;
                g.H = (ksteps + cs - 1) / cs;
                g.rowA = (int)b.rowA + T.tm * kTileM;
                g.rowB = (int)b.rowB + T.tn * kTileN;
                L.jobs.push_back(g);
            }
            parity ^= 1u;
        }
    }
    L.cta_begin[L.grid] = (int)L.jobs.size();

    // planes: slots | pools
    size_t off = align_up(size_t(L.grid) * kSlotsPerCta * kSlotBytesPerCta, 256);
    for (auto& B : L.buckets) {
        B.offA = off;
        off = align_up(off + size_t(B.nch) * B.rowsA * B.kp * 2, 256);
        B.offB = off;
        off = align_up(off + size_t(B.nch) * B.rowsB * B.kp * 2, 256);
    }
    if (mc) {  // exact int64 products
        L.xoff.resize(w.size());
        for (size_t i = 0; i < w.size(); ++i) {
            L.xoff[i] = off;
            off = align_up(off + size_t(w[i].d->m) * x_ld(w[i].d->n) * 8, 256);
        }
    }
    L.plane_bytes = off;
    // tables: maps | instances | jobs | cta_begin | conversion jobs | prefix sums [| fan-out tables]
    const size_t n_inst = w.size();
    L.t_inst = align_up(2 * L.buckets.size() * sizeof(CUtensorMap), 64);
    L.t_jobs = align_up(L.t_inst + n_inst * sizeof(InstInfo), 64);
    L.t_cta = align_up(L.t_jobs + L.jobs.size() * sizeof(GroupJob), 64);
    L.t_convA = align_up(L.t_cta + L.cta_begin.size() * sizeof(int), 64);
    L.t_convB = align_up(L.t_convA + n_inst * sizeof(ConvJob), 64);
    L.t_bbA = align_up(L.t_convB + n_inst * sizeof(ConvJob), 64);
    L.t_bbB = align_up(L.t_bbA + (n_inst + 1) * sizeof(long long), 64);
    L.tab_bytes = align_up(L.t_bbB + (n_inst + 1) * sizeof(long long), 256);
    if (mc) {
        L.t_fan = L.tab_bytes;
        L.t_fanbb = align_up(L.t_fan + n_inst * sizeof(FanInst), 64);
        L.t_cptr = align_up(L.t_fanbb + (n_inst + 1) * sizeof(long long), 64);
        L.tab_bytes = align_up(L.t_cptr + n_inst * size_t(mc->nprimes) * sizeof(uint32_t*), 256);
    }
}

// Host image of the tables (L.tab_bytes at `host`, zeroed by the caller) for
// planes at `planes` on the device.
ffgpu_status fill_wave_tables(const std::vector<BInst>& w, WaveLayout& L, unsigned char* planes,
                              unsigned char* host, const MultiCtx* mc) {
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host);
    for (size_t bi = 0; bi < L.buckets.size(); ++bi) {
        const Bucket& B = L.buckets[bi];
        if (!encode_planes(&maps[2 * bi], planes + B.offA, B.kp, B.rowsA, B.nch, kTileM) ||
            !encode_planes(&maps[2 * bi + 1], planes + B.offB, B.kp, B.rowsB, B.nch, kTileN))
            return FFGPU_ERR_CUDA;
    }
    const size_t n_inst = w.size();
    InstInfo* infos = reinterpret_cast<InstInfo*>(host + L.t_inst);
    ConvJob* convA = reinterpret_cast<ConvJob*>(host + L.t_convA);
    ConvJob* convB = reinterpret_cast<ConvJob*>(host + L.t_convB);
    long long* bbA = reinterpret_cast<long long*>(host + L.t_bbA);
    long long* bbB = reinterpret_cast<long long*>(host + L.t_bbB);
    long long nbA = 0, nbB = 0;
    for (size_t i = 0; i < n_inst; ++i) {
        const BInst& b = w[i];
        const ffgpu_fgemm_desc& d = *b.d;
        const Bucket& B = L.buckets[b.bucket];
        if (mc)
            fill_inst_int(infos[i], d.m, d.n, b.kp, b.pl, reinterpret_cast<long long*>(planes + L.xoff[i]), x_ld(d.n));
        else
            fill_inst(infos[i], d.m, d.n, b.kp, b.pl, d.alpha % d.p, d.beta % d.p, d.C, d.ldc);
        infos[i].bucket = b.bucket;
        infos[i].rowA = (int)b.rowA;
        infos[i].rowB = (int)b.rowB;

        ConvertParams cp;
        std::memset(&cp, 0, sizeof(cp));
        cp.p = d.p;
        cp.half_p = d.p / 2;
        cp.mu32 = 0xFFFFFFFFu / cp.p;
        cp.nch = b.pl.nch;
        cp.direct = b.pl.mode == 1;
        cp.signed_input = mc ? 1 : 0;
        for (int c = 0; c < b.pl.nch; ++c) {
            cp.mod[c] = b.pl.mod[c];
            cp.magic32[c] = (uint32_t)(((1ull << 39) + b.pl.mod[c] - 1) / b.pl.mod[c]);
        }
        ConvJob& a = convA[i];
        a.X = d.A;
        a.ldx = d.lda;
        a.rows = (int)d.m;
        a.cols = (int)d.k;
        a.rows_pad = (int)b.mst;
        a.kp = (int)b.kp;
        a.vec_ok = ((reinterpret_cast<uintptr_t>(d.A) & 15) == 0) && (d.lda % 4 == 0);
        a.dst = reinterpret_cast<uint4*>(planes + B.offA + size_t(b.rowA) * b.kp * 2);
        a.plane16 = size_t(B.rowsA) * b.kp / 8;
        a.cp = cp;
        ConvJob& c2 = convB[i];
        c2.X = d.B;
        c2.ldx = d.ldb;
        c2.rows = (int)d.k;
        c2.cols = (int)d.n;
        c2.rows_pad = (int)b.nst;
        c2.kp = (int)b.kp;
        c2.vec_ok = 0;
        c2.dst = reinterpret_cast<uint4*>(planes + B.offB + size_t(b.rowB) * b.kp * 2);
        c2.plane16 = size_t(B.rowsB) * b.kp / 8;
        c2.cp = cp;
        bbA[i] = nbA;
        bbB[i] = nbB;
        nbA += convert_rows_grouped_blocks((int)b.mst);
        nbB += convert_transpose_grouped_blocks((int)b.nst, (int)b.kp);
    }
    bbA[n_inst] = nbA;
    bbB[n_inst] = nbB;
    L.nbA = nbA;
    L.nbB = nbB;
    if (mc) {
        FanInst* fan = reinterpret_cast<FanInst*>(host + L.t_fan);
        long long* fbb = reinterpret_cast<long long*>(host + L.t_fanbb);
        uint32_t** cp = reinterpret_cast<uint32_t**>(host + L.t_cptr);
        long long nbF = 0;
        for (size_t i = 0; i < n_inst; ++i) {
            const ffgpu_fgemm_desc& d = *w[i].d;
            const ffgpu_multimod_desc& md = mc->mdescs[w[i].d - mc->pseudo];
            fan[i].X = reinterpret_cast<const long long*>(planes + L.xoff[i]);
            fan[i].ldx = x_ld(d.n);
            fan[i].ldc = md.ldc;
            fan[i].m = (int)d.m;
            fan[i].n = (int)d.n;
            fan[i].cbase = (int)(i * mc->nprimes);
            for (int q = 0; q < mc->nprimes; ++q) cp[i * mc->nprimes + q] = md.C[q];
            fbb[i] = nbF;
            nbF += multimod_fanout_blocks((int)d.m, (int)d.n);
        }
        fbb[n_inst] = nbF;
        L.nbF = nbF;
    }
    std::memcpy(host + L.t_jobs, L.jobs.data(), L.jobs.size() * sizeof(GroupJob));
    std::memcpy(host + L.t_cta, L.cta_begin.data(), L.cta_begin.size() * sizeof(int));
    return FFGPU_OK;
}

// The wave's three kernels, its tables already at `tabs` on the device.
ffgpu_status launch_wave(const std::vector<BInst>& w, const WaveLayout& L, unsigned char* planes,
                         unsigned char* tabs, int* err, cudaStream_t s, const MultiCtx* mc) {
    const int n_inst = (int)w.size();
    if (timed_launch("convert_rows_grouped", s, [&] {
            return launch_convert_rows_grouped(reinterpret_cast<const ConvJob*>(tabs + L.t_convA),
                                               reinterpret_cast<const long long*>(tabs + L.t_bbA), n_inst, L.nbA,
                                               s);
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    if (timed_launch("convert_transpose_grouped", s, [&] {
            return launch_convert_transpose_grouped(reinterpret_cast<const ConvJob*>(tabs + L.t_convB),
                                                    reinterpret_cast<const long long*>(tabs + L.t_bbB), n_inst,
                                                    L.nbB, s);
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    GroupGemmParams P;
    P.insts = reinterpret_cast<const InstInfo*>(tabs + L.t_inst);
    P.jobs = reinterpret_cast<const GroupJob*>(tabs + L.t_jobs);
    P.cta_begin = reinterpret_cast<const int*>(tabs + L.t_cta);
    P.maps = reinterpret_cast<const CUtensorMap*>(tabs);
    P.slots = planes;
    P.slot_stride = kSlotBytesPerCta;
    P.err = err;
    if (timed_launch(mc ? "rns_gemm_grouped_int" : "rns_gemm_grouped", s,
                     [&] { return launch_rns_gemm_grouped(P, L.grid, s, mc != nullptr); }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    if (mc) {
        FanPrimes F;
        std::memset(&F, 0, sizeof(F));
        F.nprimes = mc->nprimes;
        for (int q = 0; q < mc->nprimes; ++q) F.pr[q] = fan_prime(mc->primes[q]);
        if (timed_launch("multimod_fanout_grouped", s, [&] {
                return launch_multimod_fanout_grouped(reinterpret_cast<const FanInst*>(tabs + L.t_fan),
                                                      reinterpret_cast<const long long*>(tabs + L.t_fanbb), n_inst,
                                                      L.nbF, reinterpret_cast<uint32_t* const*>(tabs + L.t_cptr), F,
                                                      s);
            }) != cudaSuccess)
            return FFGPU_ERR_CUDA;
    }
    return FFGPU_OK;
}

// Immediate execution of one wave: workspace (planes, then tables) from the
// caller (ws != nullptr) or the stream's pool, table image staged in pinned
// memory and copied in stream order.
ffgpu_status run_wave(std::vector<BInst>& w, cudaStream_t s, int sms, void* ws_in, size_t ws_bytes, int* err_in,
                      const MultiCtx* mc = nullptr) {
    WaveLayout L;
    layout_wave(w, sms, L, mc);
    const size_t t0 = align_up(L.plane_bytes, 128);
    unsigned char* ws = nullptr;
    int* errw = err_in;
    if (ws_in) {
        if (ws_bytes < t0 + L.tab_bytes) return FFGPU_ERR_NOMEM;
        ws = static_cast<unsigned char*>(ws_in);
    } else {
        Pool* pool = nullptr;
        ffgpu_status st = pool_get(s, t0 + L.tab_bytes, &pool);
        if (st != FFGPU_OK) return st;
        ws = static_cast<unsigned char*>(pool->ptr);
        errw = pool->err;
    }
    ffgpu_status st;
    std::unique_lock<std::mutex> stage_lk(g_stage_mu);
    int stage_idx = -1;
    std::vector<unsigned char> fallback;
    unsigned char* host = stage_get(L.tab_bytes, &stage_idx);
    if (!host) {
        fallback.resize(L.tab_bytes);
        host = fallback.data();
    }
    std::memset(host, 0, L.tab_bytes);
    st = fill_wave_tables(w, L, ws, host, mc);
    if (st != FFGPU_OK) return st;
    if (cudaMemcpyAsync(ws + t0, host, L.tab_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return FFGPU_ERR_CUDA;
    if (stage_idx >= 0) stage_done(stage_idx, s);
    stage_lk.unlock();
    return launch_wave(w, L, ws, ws + t0, errw, s, mc);
}

// Small products of a batch: one grouped CUDA-core launch, one CTA per 64 x 64
// output tile (the tensor-core route would spend a whole 128 x 256 tile and
// its reconstruction on each).  Tables: the job records, then the tile -> job
// map.
// Products of at most this many multiply-adds take the grouped CUDA-core
// launch: 2^23 measured best for the multi-modular batch (2^19 .. 2^24);
// ffgpu_autotune_batched re-measures it for a given batch.
static std::atomic<int64_t> g_batch_small_macs{int64_t(1) << 23};

}  // namespace

thread_local int64_t g_batch_small_scoped = -1;
int64_t batched_small_macs() { return g_batch_small_scoped >= 0 ? g_batch_small_scoped : g_batch_small_macs.load(); }
void set_batched_small_macs(int64_t macs) { g_batch_small_macs.store(macs < 0 ? 0 : macs); }

namespace {

// Two launches by tile size: products with a dimension of at most 32, or
// whose output pads less on 32 x 32 tiles (small_on_32), on 32 x 32 tiles, the
// others on 64 x 64 tiles.  Tables: per size the job records, then the tile ->
// job map.
struct SmallGroup {
    std::vector<const ffgpu_fgemm_desc*> d;
    std::vector<const ffgpu_fgemm_desc*> by[2];  // [0]: 64 x 64 tiles, [1]: 32 x 32 tiles
    int64_t tiles[2] = {0, 0};
    size_t t_jobs[2] = {0, 0}, t_map[2] = {0, 0}, bytes = 0;
};

constexpr int kSmallTile[2] = {64, 32};

// 32 x 32 tiles for a product with a dimension of at most 32, or whose output
// padded to 32 x 32 tiles, weighted by kSmall32Cost (a 32 x 32 tile stages
// twice the words per multiply-add of a 64 x 64 one), is smaller than padded
// to 64 x 64 tiles.  Measured on the 131,072-product multi-modular batch
// (ms for the whole batch, weights 1.0 / 1.25 / 1.5 / the first rule alone):
// 215.0 / 214.8 / 217.4 / 216.7.
constexpr double kSmall32Cost = 1.25;
bool small_on_32(int64_t m, int64_t n) {
    if (std::min(m, n) <= 32) return true;
    const double p32 = double((m + 31) / 32 * 32) * double((n + 31) / 32 * 32);
    const double p64 = double((m + 63) / 64 * 64) * double((n + 63) / 64 * 64);
    return p32 * kSmall32Cost < p64;
}

void layout_small(SmallGroup& G) {
    G.by[0].clear();
    G.by[1].clear();
    for (const ffgpu_fgemm_desc* d : G.d) G.by[small_on_32(d->m, d->n) ? 1 : 0].push_back(d);
    size_t off = 0;
    for (int g = 0; g < 2; ++g) {
        G.tiles[g] = 0;
        for (const ffgpu_fgemm_desc* d : G.by[g]) G.tiles[g] += small_tiles(d->m, d->n, kSmallTile[g]);
        G.t_jobs[g] = off;
        off += align_up(G.by[g].size() * sizeof(SmallJob), 256);
        G.t_map[g] = off;
        off += align_up(size_t(G.tiles[g]) * sizeof(int), 256);
    }
    G.bytes = off;
}

void fill_small(const SmallGroup& G, unsigned char* host) {
    for (int g = 0; g < 2; ++g) {
        SmallJob* jobs = reinterpret_cast<SmallJob*>(host + G.t_jobs[g]);
        int* map = reinterpret_cast<int*>(host + G.t_map[g]);
        int64_t t = 0;
        for (size_t j = 0; j < G.by[g].size(); ++j) {
            small_job(jobs[j], *G.by[g][j], (int)t, kSmallTile[g]);
            const int64_t nt = small_tiles(G.by[g][j]->m, G.by[g][j]->n, kSmallTile[g]);
            for (int64_t q = 0; q < nt; ++q) map[t++] = (int)j;
        }
    }
}

ffgpu_status launch_small(const SmallGroup& G, const unsigned char* tabs, cudaStream_t s) {
    for (int g = 0; g < 2; ++g) {
        if (G.tiles[g] == 0) continue;
        if (timed_launch("small_gemm_grouped", s, [&] {
                return launch_small_grouped(reinterpret_cast<const SmallJob*>(tabs + G.t_jobs[g]),
                                            reinterpret_cast<const int*>(tabs + G.t_map[g]), G.tiles[g],
                                            kSmallTile[g], s);
            }) != cudaSuccess)
            return FFGPU_ERR_CUDA;
    }
    return FFGPU_OK;
}

// Immediate execution: tables staged in pinned memory, copied into the
// workspace (the caller's or the stream's pool) in stream order.
ffgpu_status run_small(SmallGroup& G, cudaStream_t s, void* ws_in, size_t ws_bytes) {
    if (G.d.empty()) return FFGPU_OK;
    layout_small(G);
    unsigned char* ws = nullptr;
    if (ws_in) {
        if (ws_bytes < G.bytes) return FFGPU_ERR_NOMEM;
        ws = static_cast<unsigned char*>(ws_in);
    } else {
        Pool* pool = nullptr;
        ffgpu_status st = pool_get(s, G.bytes, &pool);
        if (st != FFGPU_OK) return st;
        ws = static_cast<unsigned char*>(pool->ptr);
    }
    std::unique_lock<std::mutex> stage_lk(g_stage_mu);
    int stage_idx = -1;
    std::vector<unsigned char> fallback;
    unsigned char* host = stage_get(G.bytes, &stage_idx);
    if (!host) {
        fallback.resize(G.bytes);
        host = fallback.data();
    }
    fill_small(G, host);
    if (cudaMemcpyAsync(ws, host, G.bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return FFGPU_ERR_CUDA;
    if (stage_idx >= 0) stage_done(stage_idx, s);
    stage_lk.unlock();
    return launch_small(G, ws, s);
}

// Splits a batch into small products (CUDA cores, when `small` is given),
// waves (bounded plane bytes, at most 0xFFFF inner lengths) and single
// products (k = 0, k beyond one launch's capacity, huge m or n).
void split_batch(int64_t count, const ffgpu_fgemm_desc* descs, std::vector<std::vector<BInst>>& waves,
                 std::vector<const ffgpu_fgemm_desc*>& singles, SmallGroup* small = nullptr) {
    std::vector<BInst> wave;
    std::unordered_set<int64_t> wave_k;
    size_t wave_bytes = 0;
    const int64_t small_limit = std::min<int64_t>(batched_small_macs(), small_threshold());
    for (int64_t i = 0; i < count; ++i) {
        const ffgpu_fgemm_desc& d = descs[i];
        if (d.m == 0 || d.n == 0) continue;
        // a cached plan for the instance's shape bucket and modulus decides its
        // route; otherwise the size rule
        const int tuned_route = autotune_route(d.m, d.n, d.k, d.p);
        const bool to_small = tuned_route >= 0 ? tuned_route == 1
                                               : double(d.m) * double(d.n) * double(d.k) <= double(small_limit);
        if (small && d.k > 0 && to_small) {
            small->d.push_back(&d);
            continue;
        }
        RnsPlan pl;
        make_plan(d.p, d.k, pl);
        if (d.k == 0 || d.k > pl.k_slice) {
            singles.push_back(&d);
            continue;
        }
        BInst b;
        b.d = &d;
        b.pl = pl;
        b.kp = round_up(d.k, kTileK);
        b.mpad = round_up(d.m, kTileM);
        b.npad = round_up(d.n, kTileN);
        b.mst = round_up(d.m, 8);
        b.nst = round_up(d.n, 8);
        b.bucket = 0;
        b.rowA = b.rowB = 0;
        if (b.mpad / kTileM > 0xFFFF || b.npad / kTileN > 0xFFFF) {  // tile indices are packed in 16 bits
            singles.push_back(&d);
            continue;
        }
        const size_t bytes = size_t(pl.nch) * (b.mst + b.nst) * b.kp * 2;
        const bool new_k = wave_k.find(b.kp) == wave_k.end();
        if (!wave.empty() && (wave_bytes + bytes > wave_plane_budget() || (new_k && wave_k.size() >= 0xFFFF))) {
            waves.push_back(std::move(wave));
            wave.clear();
            wave_k.clear();
            wave_bytes = 0;
        }
        wave.push_back(b);
        wave_k.insert(b.kp);
        wave_bytes += bytes;
    }
    if (!wave.empty()) waves.push_back(std::move(wave));
}

}  // namespace

ffgpu_status batched_run(int64_t count, const ffgpu_fgemm_desc* descs, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    const int sms = sm_count(dev);
    std::vector<std::vector<BInst>> waves;
    std::vector<const ffgpu_fgemm_desc*> singles;
    SmallGroup small;
    split_batch(count, descs, waves, singles, &small);
    ffgpu_status st0 = run_small(small, s, nullptr, 0);
    if (st0 != FFGPU_OK) return st0;
    for (auto& w : waves) {
        ffgpu_status st = run_wave(w, s, sms, nullptr, 0, nullptr);
        if (st != FFGPU_OK) return st;
    }
    for (const ffgpu_fgemm_desc* d : singles) {
        Pool* pool = nullptr;
        ffgpu_status st = pool_get(s, fgemm_ws_bytes(d->m, d->n, d->k, d->p, sms), &pool);
        if (st != FFGPU_OK) return st;
        st = fgemm_run(d->m, d->n, d->k, d->p, d->alpha, d->A, d->lda, d->B, d->ldb, d->beta, d->C, d->ldc,
                       pool->ptr, pool->bytes, pool->err, s, 0, false);
        if (st != FFGPU_OK) return st;
    }
    return FFGPU_OK;
}

// The same with a caller workspace (for library-internal batches that must
// stay inside a workspace sized by batched_ws_bytes, e.g. ftrsm's inversion).
ffgpu_status batched_run_ws(int64_t count, const ffgpu_fgemm_desc* descs, void* ws, size_t ws_bytes, int* err,
                            cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    const int sms = sm_count(dev);
    std::vector<std::vector<BInst>> waves;
    std::vector<const ffgpu_fgemm_desc*> singles;
    SmallGroup small;
    split_batch(count, descs, waves, singles, &small);
    ffgpu_status st0 = run_small(small, s, ws, ws_bytes);
    if (st0 != FFGPU_OK) return st0;
    for (auto& w : waves) {
        ffgpu_status st = run_wave(w, s, sms, ws, ws_bytes, err);
        if (st != FFGPU_OK) return st;
    }
    for (const ffgpu_fgemm_desc* d : singles) {
        ffgpu_status st = fgemm_run(d->m, d->n, d->k, d->p, d->alpha, d->A, d->lda, d->B, d->ldb, d->beta, d->C,
                                    d->ldc, ws, ws_bytes, err, s, 0, false);
        if (st != FFGPU_OK) return st;
    }
    return FFGPU_OK;
}

// Integer-mode batch: the planner sees each instance as a product "mod" the
// plan's magnitude modulus writing to an int64 result; the waves fan the
// results out to the primes.
ffgpu_status batched_multimod_run(int64_t count, const ffgpu_multimod_desc* md, int bits, int nprimes,
                                  const uint32_t* primes, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    const int sms = sm_count(dev);
    std::vector<ffgpu_fgemm_desc> pseudo((size_t)count);
    const uint32_t pm = multimod_plan_modulus(bits);
    for (int64_t i = 0; i < count; ++i) {
        ffgpu_fgemm_desc& d = pseudo[i];
        std::memset(&d, 0, sizeof(d));
        d.m = md[i].m;
        d.n = md[i].n;
        d.k = md[i].k;
        d.p = pm;
        d.alpha = 1;
        d.A = reinterpret_cast<const uint32_t*>(md[i].A);
        d.lda = md[i].lda;
        d.B = reinterpret_cast<const uint32_t*>(md[i].B);
        d.ldb = md[i].ldb;
    }
    MultiCtx mc;
    mc.bits = bits;
    mc.nprimes = nprimes;
    mc.primes = primes;
    mc.mdescs = md;
    mc.pseudo = pseudo.data();
    std::vector<std::vector<BInst>> waves;
    std::vector<const ffgpu_fgemm_desc*> singles;
    split_batch(count, pseudo.data(), waves, singles);
    for (auto& w : waves) {
        ffgpu_status st = run_wave(w, s, sms, nullptr, 0, nullptr, &mc);
        if (st != FFGPU_OK) return st;
    }
    for (const ffgpu_fgemm_desc* d : singles) {  // k = 0 or shapes beyond the grouped launch
        const ffgpu_multimod_desc& x = md[d - pseudo.data()];
        Pool* pool = nullptr;
        ffgpu_status st = pool_get(s, multimod_ws_bytes(x.m, x.n, x.k, bits, sms), &pool);
        if (st != FFGPU_OK) return st;
        st = multimod_run(x.m, x.n, x.k, bits, x.A, x.lda, x.B, x.ldb, nprimes, primes, x.C, x.ldc, pool->ptr,
                          pool->bytes, pool->err, s);
        if (st != FFGPU_OK) return st;
    }
    return FFGPU_OK;
}

// Workspace batched_run_ws needs for a batch (shapes and moduli only).
size_t batched_ws_bytes(int64_t count, const ffgpu_fgemm_desc* descs, int sms) {
    std::vector<std::vector<BInst>> waves;
    std::vector<const ffgpu_fgemm_desc*> singles;
    SmallGroup small;
    split_batch(count, descs, waves, singles, &small);
    layout_small(small);
    size_t need = small.d.empty() ? 0 : small.bytes;
    for (auto& w : waves) {
        WaveLayout L;
        layout_wave(w, sms, L, nullptr);
        need = std::max(need, align_up(L.plane_bytes, 128) + L.tab_bytes);
    }
    for (const ffgpu_fgemm_desc* d : singles) need = std::max(need, fgemm_ws_bytes(d->m, d->n, d->k, d->p, sms));
    return need;
}

// ---------------------------------------------------------------------------
// Batched plan: the same batch laid out once, its tables uploaded once, and
// its whole launch sequence captured in a CUDA graph; a run is one graph
// launch.  The plan owns one plane region (the largest wave's), the tables of
// every wave, a workspace for the single products, and its error word.
// ---------------------------------------------------------------------------
struct BatchedPlan {
    int dev = 0;
    void* planes = nullptr;
    void* tabs = nullptr;
    void* single_ws = nullptr;
    size_t plane_bytes = 0, tab_bytes = 0, single_bytes = 0;
    int* err = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int waves = 0, singles = 0;
    size_t nodes = 0;
};

namespace {
void plan_free(BatchedPlan* P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->planes) cudaFree(P->planes);
    if (P->tabs) cudaFree(P->tabs);
    if (P->single_ws) cudaFree(P->single_ws);
    if (P->err) cudaFree(P->err);
    delete P;
}
}  // namespace

ffgpu_status batched_plan_create(int64_t count, const ffgpu_fgemm_desc* descs, BatchedPlan** out) {
    *out = nullptr;
    BatchedPlan* P = new BatchedPlan();
    if (cudaGetDevice(&P->dev) != cudaSuccess) {
        delete P;
        return FFGPU_ERR_CUDA;
    }
    const int sms = sm_count(P->dev);
    std::vector<std::vector<BInst>> waves;
    std::vector<const ffgpu_fgemm_desc*> singles;
    SmallGroup small;
    split_batch(count, descs, waves, singles, &small);
    layout_small(small);
    std::vector<WaveLayout> layouts(waves.size());
    std::vector<size_t> tab_off(waves.size());
    const size_t small_off = 0;
    if (!small.d.empty()) P->tab_bytes = align_up(small.bytes, 256);
    for (size_t i = 0; i < waves.size(); ++i) {
        layout_wave(waves[i], sms, layouts[i], nullptr);
        P->plane_bytes = std::max(P->plane_bytes, layouts[i].plane_bytes);
        tab_off[i] = P->tab_bytes;
        P->tab_bytes = align_up(P->tab_bytes + layouts[i].tab_bytes, 256);
    }
    for (const ffgpu_fgemm_desc* d : singles)
        P->single_bytes = std::max(P->single_bytes, fgemm_ws_bytes(d->m, d->n, d->k, d->p, sms));
    ffgpu_status st = FFGPU_OK;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (bytes == 0) return true;
        if (cudaMalloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            return false;
        }
        return true;
    };
    if (!alloc(&P->planes, P->plane_bytes) || !alloc(&P->tabs, P->tab_bytes) ||
        !alloc(&P->single_ws, P->single_bytes) || !alloc(reinterpret_cast<void**>(&P->err), sizeof(int))) {
        plan_free(P);
        return FFGPU_ERR_NOMEM;
    }
    cudaMemset(P->err, 0, sizeof(int));
    // every wave's tables, uploaded once
    std::vector<unsigned char> host(P->tab_bytes, 0);
    unsigned char* planes = static_cast<unsigned char*>(P->planes);
    unsigned char* tabs = static_cast<unsigned char*>(P->tabs);
    if (!small.d.empty()) fill_small(small, host.data() + small_off);
    for (size_t i = 0; i < waves.size() && st == FFGPU_OK; ++i)
        st = fill_wave_tables(waves[i], layouts[i], planes, host.data() + tab_off[i], nullptr);
    if (st == FFGPU_OK && P->tab_bytes > 0 &&
        cudaMemcpy(tabs, host.data(), P->tab_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        st = FFGPU_ERR_CUDA;
    if (st != FFGPU_OK) {
        plan_free(P);
        return st;
    }
    // capture the launch sequence on a private stream
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        plan_free(P);
        return FFGPU_ERR_CUDA;
    }
    g_capturing = true;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = FFGPU_ERR_CUDA;
    if (st == FFGPU_OK && !small.d.empty()) st = launch_small(small, tabs + small_off, cs);
    for (size_t i = 0; i < waves.size() && st == FFGPU_OK; ++i)
        st = launch_wave(waves[i], layouts[i], planes, tabs + tab_off[i], P->err, cs, nullptr);
    for (size_t i = 0; i < singles.size() && st == FFGPU_OK; ++i) {
        const ffgpu_fgemm_desc* d = singles[i];
        st = fgemm_run(d->m, d->n, d->k, d->p, d->alpha, d->A, d->lda, d->B, d->ldb, d->beta, d->C, d->ldc,
                       P->single_ws, P->single_bytes, P->err, cs, 0, true);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    g_capturing = false;
    cudaStreamDestroy(cs);
    if (st == FFGPU_OK && (ce != cudaSuccess || g == nullptr)) st = FFGPU_ERR_CUDA;
    if (st != FFGPU_OK) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        plan_free(P);
        return st;
    }
    P->graph = g;
    if (cudaGraphInstantiate(&P->exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        plan_free(P);
        return FFGPU_ERR_CUDA;
    }
    cudaGraphGetNodes(g, nullptr, &P->nodes);
    P->waves = (int)waves.size();
    P->singles = (int)singles.size();
    *out = P;
    return FFGPU_OK;
}

ffgpu_status batched_plan_run(BatchedPlan* P, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    if (dev != P->dev) return FFGPU_ERR_INVALID;
    if (cudaGraphLaunch(P->exec, s) != cudaSuccess) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    return FFGPU_OK;
}

ffgpu_status batched_plan_error(BatchedPlan* P) {
    int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return FFGPU_ERR_CUDA;
    }
    if (cudaMemcpy(&v, P->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FFGPU_ERR_CUDA;
    if (v != 0) {
        cudaMemset(P->err, 0, sizeof(int));
        return v == kDevSingular ? FFGPU_ERR_INVALID : FFGPU_ERR_TIMEOUT;
    }
    return FFGPU_OK;
}

void batched_plan_destroy(BatchedPlan* P) {
    if (!P) return;
    cudaDeviceSynchronize();  // no graph launch of this plan may still be running
    plan_free(P);
}

void batched_plan_info(const BatchedPlan* P, int* waves, int* singles, size_t* nodes, size_t* device_bytes) {
    if (waves) *waves = P->waves;
    if (singles) *singles = P->singles;
    if (nodes) *nodes = P->nodes;
    if (device_bytes) *device_bytes = P->plane_bytes + P->tab_bytes + P->single_bytes + sizeof(int);
}

}  // namespace ffgpu
