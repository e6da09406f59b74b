// Autotuner: per (path, shape bucket, channel count) choice of the tensor-core
// kernel variant, the number of Winograd levels (section 3.2.1: the threshold
// "must be determined experimentally") and the chunk length between in-place
// reductions, by timing the candidates on the device (the "self-adapting"
// thresholds the paper lists as further development, section 7).  Choices
// live in an in-memory plan cache that can be saved to and loaded from JSON.
#include <algorithm>
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
    int kernel, levels, chunk;
    double ms;
};

std::mutex g_tune_mu;
std::map<std::string, Entry> g_cache;

int64_t bucket(int64_t x) { return (x + 255) / 256 * 256; }

std::string key_for(int path, int64_t m, int64_t n, int64_t k, uint32_t p) {
    RnsPlan pl;
    make_plan(p, std::max<int64_t>(k, 1), pl);
    char buf[128];
    std::snprintf(buf, sizeof(buf), "%d:%lld:%lld:%lld:%d:%d", path, (long long)bucket(m), (long long)bucket(n),
                  (long long)bucket(k), pl.mode, pl.nch);
    return buf;
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

}  // namespace

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
    struct Cand {
        int kernel, levels, chunk;
    };
    std::vector<Cand> cands;
    const int64_t mn = std::min(std::min(m, n), k);
    for (int levels = 0; levels <= 2; ++levels) {
        if (levels > 0 && (mn >> levels) < 256) break;
        if (path == 0) {
            for (int kernel = 0; kernel <= 1; ++kernel) {
                cands.push_back(Cand{kernel, levels, max_chunk});
                if (levels == 0 && max_chunk >= 2) cands.push_back(Cand{kernel, levels, max_chunk / 2});
            }
        } else {
            cands.push_back(Cand{0, levels, 0});
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Entry best{-1, 0, 0, 1e30};
    ffgpu_status st = FFGPU_OK;
    for (const Cand& c : cands) {
        g_tune_override.kernel = c.kernel;
        g_tune_override.chunk_steps = c.chunk;
        st = run_candidate(path, c.levels, m, n, k, p, A, B, C, s);  // warm-up
        if (st != FFGPU_OK) break;
        float best_ms = 1e30f;
        for (int r = 0; r < 3 && st == FFGPU_OK; ++r) {
            cudaEventRecord(e0, s);
            st = run_candidate(path, c.levels, m, n, k, p, A, B, C, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_ms = std::min(best_ms, ms);
        }
        if (st != FFGPU_OK) break;
        if (best_ms < best.ms) best = Entry{c.kernel, c.levels, c.chunk, best_ms};
    }
    g_tune_override = TuneOverride();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(A);
    cudaFree(B);
    cudaFree(C);
    if (st != FFGPU_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_cache[key_for(path, m, n, k, p)] = best;
    }
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->kernel = best.kernel;
        out->winograd_levels = best.levels;
        out->chunk_steps = best.chunk;
        out->ms = best.ms;
    }
    return FFGPU_OK;
}

bool autotune_lookup(int path, int64_t m, int64_t n, int64_t k, uint32_t p, ffgpu_tuned* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_cache.find(key_for(path, m, n, k, p));
    if (it == g_cache.end()) return false;
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->kernel = it->second.kernel;
        out->winograd_levels = it->second.levels;
        out->chunk_steps = it->second.chunk;
        out->ms = it->second.ms;
    }
    return true;
}

ffgpu_status autotune_save(const char* path) {
    FILE* f = std::fopen(path, "w");
    if (!f) return FFGPU_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::fprintf(f, "{\"version\": 1, \"plans\": [\n");
    size_t i = 0;
    for (const auto& kv : g_cache) {
        std::fprintf(f, "  {\"key\": \"%s\", \"kernel\": %d, \"winograd_levels\": %d, \"chunk_steps\": %d, \"ms\": %.6f}%s\n",
                     kv.first.c_str(), kv.second.kernel, kv.second.levels, kv.second.chunk, kv.second.ms,
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
    bool ok = true;
    while (std::fgets(line, sizeof(line), f)) {
        const char* kp = std::strstr(line, "\"key\"");
        if (!kp) continue;
        char key[128];
        Entry e;
        if (std::sscanf(kp, "\"key\": \"%127[^\"]\", \"kernel\": %d, \"winograd_levels\": %d, \"chunk_steps\": %d, \"ms\": %lf",
                        key, &e.kernel, &e.levels, &e.chunk, &e.ms) != 5) {
            ok = false;
            break;
        }
        loaded[key] = e;
    }
    std::fclose(f);
    if (!ok) return FFGPU_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : loaded) g_cache[kv.first] = kv.second;
    return FFGPU_OK;
}

void autotune_clear() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_cache.clear();
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

ffgpu_status ffgpu_fgemm_auto(int64_t m, int64_t n, int64_t k, uint32_t p, uint32_t alpha, const uint32_t* A,
                              int64_t lda, const uint32_t* B, int64_t ldb, uint32_t beta, uint32_t* C, int64_t ldc,
                              int path, void* stream) {
    ffgpu_status st = check_args(m, n, k, p, A, lda, B, ldb, C, ldc);
    if (st != FFGPU_OK || m == 0 || n == 0) return st;
    ffgpu_tuned t;
    if (k > 0 && !autotune_lookup(path, m, n, k, p, &t)) {
        st = autotune_run(path, m, n, k, p, static_cast<cudaStream_t>(stream), &t);
        if (st != FFGPU_OK) return st;
    }
    if (k == 0) std::memset(&t, 0, sizeof(t));
    g_tune_override.kernel = t.kernel;
    g_tune_override.chunk_steps = t.chunk_steps;
    ffgpu_options opt;
    std::memset(&opt, 0, sizeof(opt));
    opt.path = path;
    opt.winograd_levels = t.winograd_levels;
    st = ffgpu_fgemm_ex(m, n, k, p, alpha, A, lda, B, ldb, beta, C, ldc, &opt, stream);
    g_tune_override = TuneOverride();
    return st;
}

}  // extern "C"
