// Autotuner: per (path, shape bucket, modulus) choice of the route (tensor
// cores or the CUDA-core kernel), the tensor-core tile shape (one-CTA kernel,
// 128 x 256 tiles, or CTA pair, 256 x 256), the tile order (rows per band),
// the chunk length between in-place reductions and the number of Winograd
// levels (section 3.2.1: the threshold "must be determined experimentally"),
// by timing the candidates on the device -- the "self-adapting" thresholds
// the paper lists as further development (section 7).  Choices live in an
// in-memory plan cache that ffgpu_fgemm, ffgpu_fgemm_ws, the request server
// and the batched launch consult, and that can be saved to and loaded from
// JSON.  For a batch, ffgpu_autotune_batched measures the size below which
// products take the grouped CUDA-core launch.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace ffgpu {

thread_local TuneOverride g_tune_override;

namespace {

struct Entry {
    int kernel, levels, chunk, route, raster;
    double ms;
};

std::mutex g_tune_mu;
std::map<std::string, Entry> g_cache;
std::atomic<size_t> g_cache_size{0};
thread_local bool g_tuning = false;  // set while candidates run: no cache consults

int64_t bucket(int64_t x) { return (x + 255) / 256 * 256; }

std::string key_for(int path, int64_t m, int64_t n, int64_t k, uint32_t p) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "%d:%lld:%lld:%lld:%u", path, (long long)bucket(m), (long long)bucket(n),
                  (long long)bucket(k), p);
    return buf;
}

bool lookup(int path, int64_t m, int64_t n, int64_t k, uint32_t p, Entry& e) {
    if (g_tuning || g_cache_size.load(std::memory_order_relaxed) == 0) return false;
    const std::string key = key_for(path, m, n, k, p);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    e = it->second;
    return true;
}

void store(const std::string& key, const Entry& e) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_cache[key] = e;
    g_cache_size.store(g_cache.size());
}

void to_public(const Entry& e, ffgpu_tuned* out) {
    std::memset(out, 0, sizeof(*out));
    out->kernel = e.kernel;
    out->winograd_levels = e.levels;
    out->chunk_steps = e.chunk;
    out->route = e.route;
    out->raster_rows = e.raster;
    out->ms = e.ms;
}

TuneOverride to_override(const Entry& e) {
    TuneOverride o;
    o.kernel = e.kernel;
    o.chunk_steps = e.chunk;
    o.route = e.route;
    o.raster = e.raster;
    return o;
}

__global__ void fill_words_kernel(uint32_t* x, size_t n, uint32_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u ^ seed;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        x[i] = h;
    }
}

ffgpu_status run_candidate(int path, int levels, int64_t m, int64_t n, int64_t k, uint32_t p, const uint32_t* A,
                           const uint32_t* B, uint32_t* C, cudaStream_t s) {
    if (path == 0 && levels == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        Pool* pool = nullptr;
        ffgpu_status st = pool_get(s, fgemm_ws_bytes(m, n, k, p, sm_count(dev)), &pool);
        if (st != FFGPU_OK) return st;
        return fgemm_run(m, n, k, p, 1, A, k, B, n, 0, C, n, pool->ptr, pool->bytes, pool->err, s, 0, true);
    }
    return fgemm_ex_run(m, n, k, p, 1, A, k, B, n, 0, C, n, path, levels, s);
}

struct Cand {
    int kernel, levels, chunk, route, raster;
};

// Best of three timed runs (after one untimed) of `fn` on stream s, in ms.
template <class F>
ffgpu_status time_best(cudaStream_t s, F&& fn, float& best_ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FFGPU_ERR_CUDA;
    ffgpu_status st = fn();
    best_ms = 1e30f;
    for (int r = 0; r < 3 && st == FFGPU_OK; ++r) {
        cudaEventRecord(e0, s);
        st = fn();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = FFGPU_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best_ms = std::min(best_ms, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace

bool autotune_settings(int64_t m, int64_t n, int64_t k, uint32_t p, TuneOverride& o, int& levels) {
    Entry e;
    if (!lookup(0, m, n, k, p, e)) return false;
    o = to_override(e);
    levels = e.route == 1 ? 0 : e.levels;
    return true;
}

int autotune_route(int64_t m, int64_t n, int64_t k, uint32_t p) {
    Entry e;
    return lookup(0, m, n, k, p, e) ? e.route : -1;
}

ffgpu_status autotune_run(int path, int64_t m, int64_t n, int64_t k, uint32_t p, cudaStream_t s,
                          ffgpu_tuned* out) {
    if (m <= 0 || n <= 0 || k <= 0 || path < 0 || path > 2) return FFGPU_ERR_INVALID;
    uint32_t *A = nullptr, *B = nullptr, *C = nullptr;
    if (cudaMalloc(&A, size_t(m) * k * 4) != cudaSuccess || cudaMalloc(&B, size_t(k) * n * 4) != cudaSuccess ||
        cudaMalloc(&C, size_t(m) * n * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(A);
        cudaFree(B);
        cudaFree(C);
        return FFGPU_ERR_NOMEM;
    }
    fill_words_kernel<<<1024, 256, 0, s>>>(A, size_t(m) * k, 12345u);
    fill_words_kernel<<<1024, 256, 0, s>>>(B, size_t(k) * n, 67890u);
    RnsPlan pl;
    make_plan(p, k, pl);
    const int max_chunk = chunk_steps_for(pl);
    std::vector<Cand> cands;
    const int64_t mn = std::min(std::min(m, n), k);
    if (path == 0) {
        // the CUDA-core kernel, for products small enough to be worth trying there
        if (double(m) * double(n) * double(k) <= double(int64_t(1) << 31) && m <= int64_t(65535) * 64)
            cands.push_back(Cand{-1, 0, 0, 1, 0});
        for (int kernel = 0; kernel <= 1; ++kernel) {
            if (kernel == 1 && m <= kTileM) continue;  // a CTA pair needs two row blocks
            cands.push_back(Cand{kernel, 0, max_chunk, 0, kRasterRows});
            if (max_chunk >= 2) cands.push_back(Cand{kernel, 0, max_chunk / 2, 0, kRasterRows});
            cands.push_back(Cand{kernel, 0, max_chunk, 0, 4});
            cands.push_back(Cand{kernel, 0, max_chunk, 0, 64});
        }
        for (int levels = 1; levels <= 2; ++levels) {
            if ((mn >> levels) < 256) break;
            cands.push_back(Cand{-1, levels, 0, -1, 0});
        }
    } else {
        for (int levels = 0; levels <= 2; ++levels) {
            if (levels > 0 && (mn >> levels) < 256) break;
            cands.push_back(Cand{-1, levels, 0, -1, 0});
        }
    }
    Entry best{-1, 0, 0, -1, 0, 1e30};
    ffgpu_status st = FFGPU_OK;
    g_tuning = true;
    for (const Cand& c : cands) {
        TuneOverride o;
        o.kernel = c.kernel;
        o.chunk_steps = c.chunk;
        o.route = c.route;
        o.raster = c.raster;
        ScopedTune scope(o);
        float ms = 0.f;
        st = time_best(s, [&] { return run_candidate(path, c.levels, m, n, k, p, A, B, C, s); }, ms);
        if (st != FFGPU_OK) break;
        if (ms < best.ms) best = Entry{c.kernel, c.levels, c.chunk, c.route, c.raster, ms};
    }
    g_tuning = false;
    cudaStreamSynchronize(s);
    cudaFree(A);
    cudaFree(B);
    cudaFree(C);
    if (st != FFGPU_OK) return st;
    store(key_for(path, m, n, k, p), best);
    if (out) to_public(best, out);
    return FFGPU_OK;
}

bool autotune_lookup(int path, int64_t m, int64_t n, int64_t k, uint32_t p, ffgpu_tuned* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_cache.find(key_for(path, m, n, k, p));
    if (it == g_cache.end()) return false;
    if (out) to_public(it->second, out);
    return true;
}

ffgpu_status autotune_save(const char* path) {
    FILE* f = std::fopen(path, "w");
    if (!f) return FFGPU_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::fprintf(f, "{\"version\": 2, \"batched_small_macs\": %lld, \"plans\": [\n", (long long)batched_small_macs());
    size_t i = 0;
    for (const auto& kv : g_cache) {
        const Entry& e = kv.second;
        std::fprintf(f,
                     "  {\"key\": \"%s\", \"kernel\": %d, \"winograd_levels\": %d, \"chunk_steps\": %d, "
                     "\"route\": %d, \"raster_rows\": %d, \"ms\": %.6f}%s\n",
                     kv.first.c_str(), e.kernel, e.levels, e.chunk, e.route, e.raster, e.ms,
                     ++i < g_cache.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    return std::fclose(f) == 0 ? FFGPU_OK : FFGPU_ERR_INVALID;
}

// Reads the file written by autotune_save (one plan object per line).
ffgpu_status autotune_load(const char* path) {
    FILE* f = std::fopen(path, "r");
    if (!f) return FFGPU_ERR_INVALID;
    char line[512];
    std::map<std::string, Entry> loaded;
    long long batch_macs = -1;
    bool ok = true;
    while (std::fgets(line, sizeof(line), f)) {
        if (const char* bp = std::strstr(line, "\"batched_small_macs\"")) {
            if (std::sscanf(bp, "\"batched_small_macs\": %lld", &batch_macs) != 1) ok = false;
        }
        const char* kp = std::strstr(line, "\"key\"");
        if (!kp) continue;
        char key[128];
        Entry e;
        if (std::sscanf(kp,
                        "\"key\": \"%127[^\"]\", \"kernel\": %d, \"winograd_levels\": %d, \"chunk_steps\": %d, "
                        "\"route\": %d, \"raster_rows\": %d, \"ms\": %lf",
                        key, &e.kernel, &e.levels, &e.chunk, &e.route, &e.raster, &e.ms) != 7 ||
            e.kernel < -1 || e.kernel > 1 || e.levels < 0 || e.levels > 8 || e.chunk < 0 || e.route < -1 ||
            e.route > 1 || e.raster < 0) {
            ok = false;
            break;
        }
        loaded[key] = e;
    }
    std::fclose(f);
    if (!ok) return FFGPU_ERR_INVALID;
    if (batch_macs >= 0) set_batched_small_macs(batch_macs);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : loaded) g_cache[kv.first] = kv.second;
    g_cache_size.store(g_cache.size());
    return FFGPU_OK;
}

void autotune_clear() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_cache.clear();
    g_cache_size.store(0);
}

}  // namespace ffgpu

using namespace ffgpu;

extern "C" {

ffgpu_status ffgpu_autotune(int64_t m, int64_t n, int64_t k, uint32_t p, int path, void* stream, ffgpu_tuned* out) {
    if (p < 2 || p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
    return autotune_run(path, m, n, k, p, static_cast<cudaStream_t>(stream), out);
}

ffgpu_status ffgpu_autotune_lookup(int64_t m, int64_t n, int64_t k, uint32_t p, int path, ffgpu_tuned* out) {
    if (p < 2 || p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
    return autotune_lookup(path, m, n, k, p, out) ? FFGPU_OK : FFGPU_ERR_INVALID;
}

ffgpu_status ffgpu_autotune_save(const char* path) { return path ? autotune_save(path) : FFGPU_ERR_INVALID; }
ffgpu_status ffgpu_autotune_load(const char* path) { return path ? autotune_load(path) : FFGPU_ERR_INVALID; }
ffgpu_status ffgpu_autotune_clear(void) {
    autotune_clear();
    return FFGPU_OK;
}

ffgpu_status ffgpu_autotune_batched(int64_t count, const ffgpu_fgemm_desc* descs, void* stream, int64_t* best_macs) {
    if (count <= 0 || !descs || !best_macs) return FFGPU_ERR_INVALID;
    for (int64_t i = 0; i < count; ++i) {
        const ffgpu_fgemm_desc& d = descs[i];
        const ffgpu_status st = check_args(d.m, d.n, d.k, d.p, d.A, d.lda, d.B, d.ldb, d.C, d.ldc);
        if (st != FFGPU_OK) return st;
    }
    // every candidate computes C = alpha A B (beta taken as 0, so repeated runs agree)
    std::vector<ffgpu_fgemm_desc> d(descs, descs + count);
    for (auto& x : d) x.beta = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t old = batched_small_macs();
    int64_t best = old;
    float best_ms = 1e30f;
    ffgpu_status st = FFGPU_OK;
    g_tuning = true;
    for (int e = 20; e <= 26 && st == FFGPU_OK; ++e) {
        set_batched_small_macs(int64_t(1) << e);
        float ms = 0.f;
        st = time_best(s, [&] { return batched_run(count, d.data(), s); }, ms);
        if (st == FFGPU_OK && ms < best_ms) {
            best_ms = ms;
            best = int64_t(1) << e;
        }
    }
    g_tuning = false;
    set_batched_small_macs(st == FFGPU_OK ? best : old);
    if (st != FFGPU_OK) return st;
    *best_macs = best;
    return FFGPU_OK;
}

ffgpu_status ffgpu_fgemm_auto(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const uint32_t* A,
                              int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta, uint32_t* C, int64_t ldc,
                              int path, void* stream) {
    ffgpu_status st = check_args(m, n, k, p, A, lda, B, ldb, C, ldc);
    if (st != FFGPU_OK || m == 0 || n == 0) return st;
    ffgpu_tuned t;
    std::memset(&t, 0, sizeof(t));
    if (k > 0 && !autotune_lookup(path, m, n, k, p, &t)) {
        st = autotune_run(path, m, n, k, p, static_cast<cudaStream_t>(stream), &t);
        if (st != FFGPU_OK) return st;
    }
    if (path == 0) return ffgpu_fgemm(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, stream);  // applies the plan
    ffgpu_options opt;
    std::memset(&opt, 0, sizeof(opt));
    opt.path = path;
    opt.winograd_levels = t.winograd_levels;
    return ffgpu_fgemm_ex(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, &opt, stream);
}

}  // extern "C"
