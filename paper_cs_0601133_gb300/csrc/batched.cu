// Batched fgemm: many independent products of different shapes and moduli in
// one grouped conversion per operand and one persistent tensor-core launch per
// wave.  Host side only: plans, placement of every instance's channel planes in
// per-k pools, cost-balanced job lists, tables copied to the device.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <functional>
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
std::mutex g_stage_mu;  // held from stage_get to stage_done
StageBuf g_stage[2];
int g_stage_next = 0;

unsigned char* stage_get(size_t bytes, int* idx) {
    StageBuf& b = g_stage[g_stage_next];
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
    *idx = g_stage_next;
    g_stage_next ^= 1;
    return b.p;
}

void stage_done(int idx, cudaStream_t s) {
    if (cudaEventRecord(g_stage[idx].ev, s) == cudaSuccess) g_stage[idx].pending = true;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct BInst {
    const ffgpu_fgemm_desc* d;
    RnsPlan pl;
    int64_t kp, mpad, npad;
    int bucket;
    int64_t rowA, rowB;
};

struct Bucket {
    int64_t kp;
    int nch;
    int64_t rowsA, rowsB;
    size_t offA, offB;  // byte offsets of the pools in the workspace
};

ffgpu_status run_wave(std::vector<BInst>& w, cudaStream_t s, int sms) {
    // buckets by padded inner length
    std::vector<Bucket> buckets;
    std::unordered_map<int64_t, int> bucket_of;
    for (auto& b : w) {
        int idx;
        auto it = bucket_of.find(b.kp);
        if (it == bucket_of.end()) {
            buckets.push_back(Bucket{b.kp, 0, 0, 0, 0, 0});
            idx = (int)buckets.size() - 1;
            bucket_of.emplace(b.kp, idx);
        } else {
            idx = it->second;
        }
        Bucket& B = buckets[idx];
        b.bucket = idx;
        B.nch = std::max(B.nch, b.pl.nch);
        b.rowA = B.rowsA;
        b.rowB = B.rowsB;
        B.rowsA += b.mpad;
        B.rowsB += b.npad;
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
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(tiles.size(), (size_t)sms));
    std::stable_sort(tiles.begin(), tiles.end(), [](const Tile& a, const Tile& b) { return a.cost > b.cost; });
    std::vector<std::vector<int>> per_cta(grid);
    {
        typedef std::pair<double, int> Load;
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int c = 0; c < grid; ++c) heap.push(Load(0.0, c));
        for (size_t t = 0; t < tiles.size(); ++t) {
            Load l = heap.top();
            heap.pop();
            per_cta[l.second].push_back((int)t);
            l.first += tiles[t].cost;
            heap.push(l);
        }
    }
    std::vector<GroupJob> jobs;
    std::vector<int> cta_begin(grid + 1, 0);
    for (int c = 0; c < grid; ++c) {
        cta_begin[c] = (int)jobs.size();
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
                jobs.push_back(g);
            }
            parity ^= 1u;
        }
    }
    cta_begin[grid] = (int)jobs.size();

    // workspace layout: slots | pools | tables
    size_t off = align_up(size_t(grid) * kSlotsPerCta * kSlotBytesPerCta, 256);
    for (auto& B : buckets) {
        B.offA = off;
        off = align_up(off + size_t(B.nch) * B.rowsA * B.kp * 2, 256);
        B.offB = off;
        off = align_up(off + size_t(B.nch) * B.rowsB * B.kp * 2, 256);
    }
    const size_t n_inst = w.size();
    const size_t t_maps = align_up(off, 128);
    const size_t t_inst = align_up(t_maps + 2 * buckets.size() * sizeof(CUtensorMap), 64);
    const size_t t_jobs = align_up(t_inst + n_inst * sizeof(InstInfo), 64);
    const size_t t_cta = align_up(t_jobs + jobs.size() * sizeof(GroupJob), 64);
    const size_t t_convA = align_up(t_cta + cta_begin.size() * sizeof(int), 64);
    const size_t t_convB = align_up(t_convA + n_inst * sizeof(ConvJob), 64);
    const size_t t_bbA = align_up(t_convB + n_inst * sizeof(ConvJob), 64);
    const size_t t_bbB = align_up(t_bbA + (n_inst + 1) * sizeof(long long), 64);
    const size_t t_end = align_up(t_bbB + (n_inst + 1) * sizeof(long long), 256);

    Pool* pool = nullptr;
    ffgpu_status st = pool_get(s, t_end, &pool);
    if (st != FFGPU_OK) return st;
    unsigned char* ws = static_cast<unsigned char*>(pool->ptr);

    // host image of the tables [t_maps, t_end), in pinned staging when available
    const size_t tab_bytes = t_end - t_maps;
    std::unique_lock<std::mutex> stage_lk(g_stage_mu);
    int stage_idx = -1;
    std::vector<unsigned char> fallback;
    unsigned char* host = stage_get(tab_bytes, &stage_idx);
    if (!host) {
        fallback.resize(tab_bytes);
        host = fallback.data();
    }
    std::memset(host, 0, tab_bytes);
    auto at = [&](size_t o) { return host + (o - t_maps); };
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(at(t_maps));
    for (size_t bi = 0; bi < buckets.size(); ++bi) {
        const Bucket& B = buckets[bi];
        if (!encode_planes(&maps[2 * bi], ws + B.offA, B.kp, B.rowsA, B.nch, kTileM) ||
            !encode_planes(&maps[2 * bi + 1], ws + B.offB, B.kp, B.rowsB, B.nch, kTileN))
            return FFGPU_ERR_CUDA;
    }
    InstInfo* infos = reinterpret_cast<InstInfo*>(at(t_inst));
    ConvJob* convA = reinterpret_cast<ConvJob*>(at(t_convA));
    ConvJob* convB = reinterpret_cast<ConvJob*>(at(t_convB));
    long long* bbA = reinterpret_cast<long long*>(at(t_bbA));
    long long* bbB = reinterpret_cast<long long*>(at(t_bbB));
    long long nbA = 0, nbB = 0;
    for (size_t i = 0; i < n_inst; ++i) {
        const BInst& b = w[i];
        const ffgpu_fgemm_desc& d = *b.d;
        const Bucket& B = buckets[b.bucket];
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
        for (int c = 0; c < b.pl.nch; ++c) {
            cp.mod[c] = b.pl.mod[c];
            cp.magic32[c] = (uint32_t)(((1ull << 39) + b.pl.mod[c] - 1) / b.pl.mod[c]);
        }
        ConvJob& a = convA[i];
        a.X = d.A;
        a.ldx = d.lda;
        a.rows = (int)d.m;
        a.cols = (int)d.k;
        a.rows_pad = (int)b.mpad;
        a.kp = (int)b.kp;
        a.vec_ok = ((reinterpret_cast<uintptr_t>(d.A) & 15) == 0) && (d.lda % 4 == 0);
        a.dst = reinterpret_cast<uint4*>(ws + B.offA + size_t(b.rowA) * b.kp * 2);
        a.plane16 = size_t(B.rowsA) * b.kp / 8;
        a.cp = cp;
        ConvJob& c2 = convB[i];
        c2.X = d.B;
        c2.ldx = d.ldb;
        c2.rows = (int)d.k;
        c2.cols = (int)d.n;
        c2.rows_pad = (int)b.npad;
        c2.kp = (int)b.kp;
        c2.vec_ok = 0;
        c2.dst = reinterpret_cast<uint4*>(ws + B.offB + size_t(b.rowB) * b.kp * 2);
        c2.plane16 = size_t(B.rowsB) * b.kp / 8;
        c2.cp = cp;
        bbA[i] = nbA;
        bbB[i] = nbB;
        nbA += convert_rows_grouped_blocks((int)b.mpad);
        nbB += convert_transpose_grouped_blocks((int)b.npad, (int)b.kp);
    }
    bbA[n_inst] = nbA;
    bbB[n_inst] = nbB;
    std::memcpy(at(t_jobs), jobs.data(), jobs.size() * sizeof(GroupJob));
    std::memcpy(at(t_cta), cta_begin.data(), cta_begin.size() * sizeof(int));
    if (cudaMemcpyAsync(ws + t_maps, host, tab_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    if (stage_idx >= 0) stage_done(stage_idx, s);
    stage_lk.unlock();

    if (timed_launch("convert_rows_grouped", s, [&] {
            return launch_convert_rows_grouped(reinterpret_cast<const ConvJob*>(ws + t_convA),
                                               reinterpret_cast<const long long*>(ws + t_bbA), (int)n_inst, nbA, s);
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    if (timed_launch("convert_transpose_grouped", s, [&] {
            return launch_convert_transpose_grouped(reinterpret_cast<const ConvJob*>(ws + t_convB),
                                                    reinterpret_cast<const long long*>(ws + t_bbB), (int)n_inst,
                                                    nbB, s);
        }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    GroupGemmParams P;
    P.insts = reinterpret_cast<const InstInfo*>(ws + t_inst);
    P.jobs = reinterpret_cast<const GroupJob*>(ws + t_jobs);
    P.cta_begin = reinterpret_cast<const int*>(ws + t_cta);
    P.maps = reinterpret_cast<const CUtensorMap*>(ws + t_maps);
    P.slots = ws;
    P.slot_stride = kSlotBytesPerCta;
    P.err = pool->err;
    if (timed_launch("rns_gemm_grouped", s, [&] { return launch_rns_gemm_grouped(P, grid, s); }) != cudaSuccess)
        return FFGPU_ERR_CUDA;
    return FFGPU_OK;
}

}  // namespace

ffgpu_status batched_run(int64_t count, const ffgpu_fgemm_desc* descs, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    const int sms = sm_count(dev);
    std::vector<BInst> wave;
    std::unordered_set<int64_t> wave_k;
    std::vector<const ffgpu_fgemm_desc*> singles;  // k = 0, k beyond one launch's capacity, huge m or n
    size_t wave_bytes = 0;
    for (int64_t i = 0; i < count; ++i) {
        const ffgpu_fgemm_desc& d = descs[i];
        if (d.m == 0 || d.n == 0) continue;
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
        if (b.mpad / kTileM > 0xFFFF || b.npad / kTileN > 0xFFFF) {  // tile indices are packed in 16 bits
            singles.push_back(&d);
            continue;
        }
        b.bucket = 0;
        b.rowA = b.rowB = 0;
        const size_t bytes = size_t(pl.nch) * (b.mpad + b.npad) * b.kp * 2;
        // a wave holds at most 0xFFFF distinct inner lengths (k-bucket indices are packed in 16 bits)
        const bool new_k = wave_k.find(b.kp) == wave_k.end();
        if (!wave.empty() && (wave_bytes + bytes > wave_plane_budget() || (new_k && wave_k.size() >= 0xFFFF))) {
            ffgpu_status st = run_wave(wave, s, sms);
            if (st != FFGPU_OK) return st;
            wave.clear();
            wave_k.clear();
            wave_bytes = 0;
        }
        wave.push_back(b);
        wave_k.insert(b.kp);
        wave_bytes += bytes;
    }
    if (!wave.empty()) {
        ffgpu_status st = run_wave(wave, s, sms);
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

}  // namespace ffgpu
