// Continuous-batching request server for fgemm / ftrsm.
//
// Requests arrive with host operands.  An engine thread admits them in
// arrival order whenever a worker stream is free and the device arena (a
// fixed HBM budget) has room for the request's operands and workspace; each
// admitted request is copied in, computed and copied out on its own stream, so
// the work of requests admitted at different times overlaps on the device.
// Completion is detected with CUDA events; the request's memory and stream are
// then returned and the next pending requests admitted.  Times are
// CLOCK_MONOTONIC microseconds.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace ffgpu {


namespace {

double now_us() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec * 1e6 + ts.tv_nsec * 1e-3;
}

// First-fit allocator over one device arena, with coalescing of free blocks.
class Arena {
  public:
    bool init(size_t bytes) {
        bytes_ = bytes;
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        free_[0] = bytes;
        return true;
    }
    void release() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    // offset of a block of `n` bytes (256-aligned), or -1
    long long alloc(size_t n) {
        n = (n + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                used_ += n;
                return (long long)off;
            }
        }
        return -1;
    }
    void free_block(size_t off, size_t n) {
        n = (n + 255) & ~size_t(255);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    unsigned char* base() const { return static_cast<unsigned char*>(base_); }
    size_t capacity() const { return bytes_; }
    size_t used() const { return used_; }

  private:
    void* base_ = nullptr;
    size_t bytes_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Req {
    ffgpu_request r;
    size_t bytes = 0;
    long long off = -1;
    int stream = -1;
    cudaEvent_t done = nullptr;
    double t_submit = 0, t_admit = 0;
    int status = 0;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct Server {
    int nstreams = 0;
    std::vector<cudaStream_t> streams;
    std::vector<int*> errs;
    std::vector<int> free_streams;
    Arena arena;
    int dev = 0, sms = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> pending;
    std::vector<Req*> inflight;
    std::deque<ffgpu_completion> completed;
    std::thread engine;
    std::atomic<bool> stop{false};
    ffgpu_server_stats stats{};

    size_t need_bytes(const ffgpu_request& q) const {
        if (q.kind == 0) {
            return align256(size_t(q.m) * q.k * 4) + align256(size_t(q.k) * q.n * 4) + align256(size_t(q.m) * q.n * 4) +
                   align256(fgemm_ws_bytes(q.m, q.n, q.k, q.p, sms));
        }
        const int64_t nt = q.side == 0 ? q.m : q.n;
        return align256(size_t(nt) * nt * 4) + align256(size_t(q.m) * q.n * 4) +
               align256(ftrsm_ws_bytes(q.side, q.uplo, FFGPU_TRSM_DEFAULT, q.m, q.n, q.p, sms));
    }

    // enqueue the whole request on stream `si` using arena block `off`
    int launch(Req* q, int si) {
        cudaStream_t s = streams[si];
        const ffgpu_request& r = q->r;
        unsigned char* blk = arena.base() + q->off;
        ffgpu_status st;
        if (r.kind == 0) {
            uint32_t* dA = reinterpret_cast<uint32_t*>(blk);
            uint32_t* dB = reinterpret_cast<uint32_t*>(blk + align256(size_t(r.m) * r.k * 4));
            uint32_t* dC = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(dB) + align256(size_t(r.k) * r.n * 4));
            unsigned char* ws = reinterpret_cast<unsigned char*>(dC) + align256(size_t(r.m) * r.n * 4);
            const size_t ws_bytes = q->bytes - size_t(ws - blk);
            if (r.k > 0) {
                cudaMemcpy2DAsync(dA, r.k * 4, r.A, r.lda * 4, r.k * 4, r.m, cudaMemcpyHostToDevice, s);
                cudaMemcpy2DAsync(dB, r.n * 4, r.B, r.ldb * 4, r.n * 4, r.k, cudaMemcpyHostToDevice, s);
            }
            if (r.beta % r.p != 0 && r.C_in)
                cudaMemcpy2DAsync(dC, r.n * 4, r.C_in, r.ldc_in * 4, r.n * 4, r.m, cudaMemcpyHostToDevice, s);
            else
                cudaMemsetAsync(dC, 0, size_t(r.m) * r.n * 4, s);
            {
                // the request's cached plan, if any (kernel, chunk, route, tile order; the
                // arena block holds no room for Winograd's temporaries)
                TuneOverride tuned;
                int levels = 0;
                const bool have = r.k > 0 && autotune_settings(r.m, r.n, r.k, r.p, tuned, levels);
                ScopedTune scope(have ? tuned : g_tune_override);
                st = fgemm_run(r.m, r.n, r.k, r.p, r.alpha, dA, std::max<int64_t>(r.k, 1), dB, r.n, r.beta, dC, r.n,
                               ws, ws_bytes, errs[si], s, 0, false);
            }
            cudaMemcpy2DAsync(r.out, r.ldo * 4, dC, r.n * 4, r.n * 4, r.m, cudaMemcpyDeviceToHost, s);
        } else {
            const int64_t nt = r.side == 0 ? r.m : r.n;
            uint32_t* dT = reinterpret_cast<uint32_t*>(blk);
            uint32_t* dB = reinterpret_cast<uint32_t*>(blk + align256(size_t(nt) * nt * 4));
            unsigned char* ws = reinterpret_cast<unsigned char*>(dB) + align256(size_t(r.m) * r.n * 4);
            const size_t ws_bytes = q->bytes - size_t(ws - blk);
            cudaMemcpy2DAsync(dT, nt * 4, r.A, r.lda * 4, nt * 4, nt, cudaMemcpyHostToDevice, s);
            cudaMemcpy2DAsync(dB, r.n * 4, r.B, r.ldb * 4, r.n * 4, r.m, cudaMemcpyHostToDevice, s);
            st = ftrsm_run(r.side, r.uplo, r.diag, FFGPU_TRSM_DEFAULT, r.m, r.n, r.p, r.alpha, dT, nt, dB, r.n, ws, ws_bytes,
                           errs[si], s);
            cudaMemcpy2DAsync(r.out, r.ldo * 4, dB, r.n * 4, r.n * 4, r.m, cudaMemcpyDeviceToHost, s);
        }
        cudaEventRecord(q->done, s);
        if (cudaGetLastError() != cudaSuccess && st == FFGPU_OK) st = FFGPU_ERR_CUDA;
        return (int)st;
    }

    void finish(Req* q, int status) {
        ffgpu_completion c;
        c.tag = q->r.tag;
        c.status = status;
        c.t_submit_us = q->t_submit;
        c.t_admit_us = q->t_admit;
        c.t_done_us = now_us();
        completed.push_back(c);
        stats.completed += 1;
        if (status != 0) stats.failed += 1;
    }

    void loop() {
        cudaSetDevice(dev);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop.load()) {
            bool progress = false;
            // completions
            for (size_t i = 0; i < inflight.size();) {
                Req* q = inflight[i];
                const cudaError_t e = cudaEventQuery(q->done);
                if (e == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                int status = q->status;
                if (e != cudaSuccess) status = FFGPU_ERR_CUDA;
                int hv = 0;
                if (status == 0 && cudaMemcpy(&hv, errs[q->stream], sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
                    hv != 0) {
                    status = hv == kDevSingular ? FFGPU_ERR_INVALID : FFGPU_ERR_TIMEOUT;
                    cudaMemset(errs[q->stream], 0, sizeof(int));
                }
                finish(q, status);
                arena.free_block((size_t)q->off, q->bytes);
                free_streams.push_back(q->stream);
                cudaEventDestroy(q->done);
                delete q;
                inflight[i] = inflight.back();
                inflight.pop_back();
                progress = true;
            }
            // admissions, in arrival order (the head waits for memory)
            while (!pending.empty() && !free_streams.empty()) {
                Req* q = pending.front();
                const long long off = arena.alloc(q->bytes);
                if (off < 0) break;
                pending.pop_front();
                q->off = off;
                q->stream = free_streams.back();
                free_streams.pop_back();
                q->t_admit = now_us();
                cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming);
                q->status = launch(q, q->stream);
                inflight.push_back(q);
                stats.admitted += 1;
                stats.peak_inflight = std::max<int64_t>(stats.peak_inflight, (int64_t)inflight.size());
                stats.peak_bytes = std::max<int64_t>(stats.peak_bytes, (int64_t)arena.used());
                progress = true;
            }
            if (progress) cv.notify_all();
            if (!progress) {
                if (inflight.empty())
                    cv.wait_for(lk, std::chrono::milliseconds(2));
                else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                    lk.lock();
                }
            }
        }
    }
};

}  // namespace ffgpu

using namespace ffgpu;

extern "C" {

ffgpu_status ffgpu_server_create(int streams, size_t budget_bytes, ffgpu_server** out) {
    if (!out || streams < 1 || streams > 64 || budget_bytes < (size_t(1) << 20)) return FFGPU_ERR_INVALID;
    Server* sv = new Server();
    if (cudaGetDevice(&sv->dev) != cudaSuccess) {
        delete sv;
        return FFGPU_ERR_CUDA;
    }
    sv->sms = sm_count(sv->dev);
    if (!sv->arena.init(budget_bytes)) {
        delete sv;
        return FFGPU_ERR_NOMEM;
    }
    sv->nstreams = streams;
    for (int i = 0; i < streams; ++i) {
        cudaStream_t s;
        int* e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaMalloc(&e, 256) != cudaSuccess) {
            cudaGetLastError();
            sv->arena.release();
            delete sv;
            return FFGPU_ERR_CUDA;
        }
        cudaMemset(e, 0, 256);
        sv->streams.push_back(s);
        sv->errs.push_back(e);
        sv->free_streams.push_back(i);
    }
    cudaDeviceSynchronize();
    sv->engine = std::thread([sv] { sv->loop(); });
    *out = reinterpret_cast<ffgpu_server*>(sv);
    return FFGPU_OK;
}

ffgpu_status ffgpu_server_submit(ffgpu_server* server, const ffgpu_request* req) {
    if (!server || !req) return FFGPU_ERR_INVALID;
    Server* sv = reinterpret_cast<Server*>(server);
    const ffgpu_request& r = *req;
    if (r.kind == 0) {
        const ffgpu_status st = check_args(r.m, r.n, r.k, r.p, r.A, r.lda, r.B, r.ldb, r.out, r.ldo);
        if (st != FFGPU_OK) return st;
        if (r.m == 0 || r.n == 0) return FFGPU_ERR_INVALID;
    } else if (r.kind == 1) {
        if (r.p < 2 || r.p > 0x7FFFFFFFu) return FFGPU_ERR_UNSUPPORTED_P;
        const int64_t nt = r.side == 0 ? r.m : r.n;
        if (r.side < 0 || r.side > 1 || r.uplo < 0 || r.uplo > 1 || r.diag < 0 || r.diag > 1 || r.m <= 0 ||
            r.n <= 0 || !r.A || !r.B || !r.out || r.lda < nt || r.ldb < r.n || r.ldo < r.n)
            return FFGPU_ERR_INVALID;
    } else {
        return FFGPU_ERR_INVALID;
    }
    Req* q = new Req();
    q->r = r;
    q->bytes = sv->need_bytes(r);
    if (q->bytes > sv->arena.capacity()) {
        delete q;
        return FFGPU_ERR_BUDGET;  // could never be admitted
    }
    q->t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->pending.push_back(q);
        sv->stats.submitted += 1;
    }
    sv->cv.notify_all();
    return FFGPU_OK;
}

ffgpu_status ffgpu_server_poll(ffgpu_server* server, ffgpu_completion* out, int cap, int* count, int wait_ms) {
    if (!server || !count || cap < 0 || (cap > 0 && !out)) return FFGPU_ERR_INVALID;
    Server* sv = reinterpret_cast<Server*>(server);
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->completed.empty() && wait_ms > 0)
        sv->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [sv] { return !sv->completed.empty(); });
    int n = 0;
    while (n < cap && !sv->completed.empty()) {
        out[n++] = sv->completed.front();
        sv->completed.pop_front();
    }
    *count = n;
    return FFGPU_OK;
}

ffgpu_status ffgpu_server_get_stats(ffgpu_server* server, ffgpu_server_stats* out) {
    if (!server || !out) return FFGPU_ERR_INVALID;
    Server* sv = reinterpret_cast<Server*>(server);
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->pending = (int64_t)sv->pending.size();
    out->inflight = (int64_t)sv->inflight.size();
    out->budget_bytes = (int64_t)sv->arena.capacity();
    out->used_bytes = (int64_t)sv->arena.used();
    return FFGPU_OK;
}

ffgpu_status ffgpu_server_destroy(ffgpu_server* server) {
    if (!server) return FFGPU_ERR_INVALID;
    Server* sv = reinterpret_cast<Server*>(server);
    // let admitted work finish; pending requests are dropped
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        for (Req* q : sv->pending) delete q;
        sv->pending.clear();
    }
    for (int i = 0; i < 100000; ++i) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (sv->inflight.empty()) break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    sv->stop.store(true);
    sv->cv.notify_all();
    if (sv->engine.joinable()) sv->engine.join();
    for (Req* q : sv->inflight) {
        cudaEventDestroy(q->done);
        delete q;
    }
    for (auto s : sv->streams) cudaStreamSynchronize(s);
    for (auto s : sv->streams) cudaStreamDestroy(s);
    for (auto e : sv->errs) cudaFree(e);
    sv->arena.release();
    delete sv;
    return FFGPU_OK;
}

}  // extern "C"
