// FP32 FMA throughput calibration.  Every hot kernel of the library is bound by
// FP32 SIMT arithmetic, so the roofline denominator is the FMA rate this GPU
// actually sustains: many independent FMA chains per thread, enough resident
// warps to hide the pipe latency, timed with CUDA events on the caller's
// stream.  Scalar FFMA and the packed two-lane form are measured separately.
#include <cuda_runtime.h>

#include "mrpop_internal.cuh"

namespace mrpop {
namespace {

constexpr int kChains = 8;      // independent accumulators per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;  // 2,048 threads per SM

__device__ float g_peak_sink;

typedef unsigned long long pk2;

__device__ __forceinline__ pk2 pk2_fma(pk2 a, pk2 b, pk2 c) {
    pk2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// a <- a * b + c converges to c / (1 - b) = 1: no overflow, no subnormals.
template <bool PACKED>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(int iters, float b, float c) {
    const float seed = 1.f + 1e-7f * (float)(threadIdx.x & 31);
    float sum = 0.f;
    if (PACKED) {
        pk2 a[kChains], bb, cc;
        asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
        asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            const float v = seed + 1e-6f * (float)i;
            asm("mov.b64 %0, {%1, %1};" : "=l"(a[i]) : "f"(v));
        }
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = pk2_fma(a[i], bb, cc);
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i]));
            sum += lo + hi;
        }
    } else {
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = seed + 1e-6f * (float)i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = __fmaf_rn(a[i], b, c);
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) sum += a[i];
    }
    if (sum == -1.f) g_peak_sink = sum;  // never true; keeps the chains live
}

}  // namespace
}  // namespace mrpop

using namespace mrpop;

extern "C" mrpop_status mrpop_fp32_peak(int32_t packed, int32_t iters, double *tflops,
                                        void *cuda_stream) {
    if (!tflops) return set_error(MRPOP_EINVAL, "tflops is NULL");
    if (packed != 0 && packed != 1) return set_error(MRPOP_EINVAL, "packed must be 0 or 1");
    if (iters < 1 || iters > (1 << 24)) return set_error(MRPOP_EINVAL, "iters out of range");
    int dev = 0, sms = 0;
    MRPOP_CUDA_TRY(cudaGetDevice(&dev));
    MRPOP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const dim3 grid(sms * kBlocksPerSM), block(kThreads);
    const float b = 0.99999f, c = 1e-5f;
    auto launch = [&](int n) {
        if (packed)
            fma_peak_kernel<true><<<grid, block, 0, st>>>(n, b, c);
        else
            fma_peak_kernel<false><<<grid, block, 0, st>>>(n, b, c);
    };
    cudaEvent_t e0, e1;
    MRPOP_CUDA_TRY(cudaEventCreate(&e0));
    if (const cudaError_t ce = cudaEventCreate(&e1); ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_error(ce, "cudaEventCreate");
    }
    launch(iters);  // warm-up (clocks ramp, module load)
    constexpr int kReps = 5;
    cudaEventRecord(e0, st);
    for (int r = 0; r < kReps; ++r) launch(iters);
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_error(err, "fma_peak_kernel");
    const double flops = 2.0 * kChains * (packed ? 2.0 : 1.0) * (double)iters *
                         (double)grid.x * kThreads * kReps;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return MRPOP_OK;
}
