// Peak rates of the legacy warp-level MMA units, measured on the device: the
// reference points reported beside the tensor-core roofline.  tcgen05 has no
// int8 kind on sm_103a, so the int8 rate of this GPU is the warp-level
// mma.sync rate; the bf16 and FP64 (DMMA) warp-level rates are measured the
// same way.  Each warp runs independent MMA chains on register operands (no
// memory traffic) for a fixed number of iterations on every SM; the rate is
// the operations issued over the CUDA-event time of the launch.
#include <algorithm>

#include "internal.h"

namespace ffgpu {

namespace {

constexpr int kChains = 4;       // independent accumulators per warp
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) probe_imma(int64_t iters, int* out) {
    uint32_t a[4], b[2];
    int32_t d[kChains][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = 0x01010101u * (threadIdx.x + i);
    b[0] = 0x02020202u;
    b[1] = 0x03030303u;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) d[c][i] = 0;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == 0x7fffffff) out[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) probe_hmma(int64_t iters, int* out) {
    uint32_t a[4], b[2];
    float d[kChains][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = 0x3f803f80u;  // two bf16 ones
    b[0] = b[1] = 0x3f803f80u;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) d[c][i] = 0.f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == -1.f) out[0] = 1;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dmma(int64_t iters, int* out) {
    double a = 1.0 + threadIdx.x, b = 0.5;
    double d[kChains][2];
#pragma unroll
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(d[c][0]), "+d"(d[c][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
    if (s == -1.0) out[0] = 1;
}

}  // namespace

}  // namespace ffgpu

// kind: 0 = int8 (s8 x s8 -> s32, m16n8k32), 1 = bf16 (-> f32, m16n8k16),
// 2 = FP64 DMMA (m8n8k4).  Operations per MMA: 2 M N K.
extern "C" ffgpu_status ffgpu_peak_probe(int kind, int64_t iters, double* ops_per_second, void* stream) {
    using namespace ffgpu;
    if (!ops_per_second || kind < 0 || kind > 2 || iters < 1 || iters > (int64_t(1) << 24)) return FFGPU_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFGPU_ERR_CUDA;
    const int sms = sm_count(dev);
    const int blocks = sms * 4;  // 32 warps per SM
    int* out = nullptr;
    if (cudaMallocAsync(&out, sizeof(int), s) != cudaSuccess) return FFGPU_ERR_NOMEM;
    auto launch = [&](int64_t n) {
        if (kind == 0) probe_imma<<<blocks, kProbeThreads, 0, s>>>(n, out);
        else if (kind == 1) probe_hmma<<<blocks, kProbeThreads, 0, s>>>(n, out);
        else probe_dmma<<<blocks, kProbeThreads, 0, s>>>(n, out);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ffgpu_status st = FFGPU_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = FFGPU_ERR_CUDA;
    if (st == FFGPU_OK) {
        launch(std::max<int64_t>(1, iters / 8));  // warm-up (clocks, code)
        cudaEventRecord(e0, s);
        launch(iters);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) st = FFGPU_ERR_CUDA;
    }
    if (st == FFGPU_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per_mma = kind == 0 ? 2.0 * 16 * 8 * 32 : kind == 1 ? 2.0 * 16 * 8 * 16 : 2.0 * 8 * 8 * 4;
        const double mmas = double(blocks) * (kProbeThreads / 32) * kChains * double(iters);
        *ops_per_second = ms > 0.f ? mmas * per_mma / (ms * 1e-3) : 0.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    return st;
}
