// measure.cu -- the FP32 and FP64 CUDA-core peaks that the descriptor
// kernels' roofline fractions are taken against, measured on the device the
// context runs on.
//
// Every thread runs independent chains of fused multiply-adds (eight scalar
// FP32 chains, eight chains of packed FP32x2 FMAs, or eight FP64 chains):
// enough independent work per scheduler to hide the pipe latency, nothing else
// in the loop.  The grid is a multiple of the SM count.  Time by CUDA events on
// the context's stream; the best of a few repetitions is returned, in FLOP/s
// with an FMA counted as two.
#include <cuda_runtime.h>

#include <algorithm>

#include "mala_internal.h"

namespace mala {

namespace {

constexpr int kFmaThreads = 256;
constexpr int kFmaBlocksPerSm = 4;
constexpr int kFmaIters = 16384;

__global__ void __launch_bounds__(kFmaThreads) k_fma_scalar(float a, float b, float* __restrict__ sink) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = b * (float)(threadIdx.x + i);
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(kFmaThreads) k_fma_packed(float a, float b, float* __restrict__ sink) {
    float2 x[8];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = make_float2(b * (float)(threadIdx.x + i), b * (float)(threadIdx.x - i));
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
    if (s == 1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kFmaIters64 = 1024;  // FP64 runs at a small fraction of the FP32 rate

__global__ void __launch_bounds__(kFmaThreads) k_fma_f64(double a, double b, double* __restrict__ sink) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = b * (double)(threadIdx.x + i);
    for (int it = 0; it < kFmaIters64; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1234.5) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int measure_peaks(Ctx* c, double* scalar_tflops, double* packed_tflops, double* fp64_tflops) {
    const int blocks = std::max(1, c->num_sms) * kFmaBlocksPerSm;
    const cudaStream_t st = c->stream;
    MALA_TRY(c->ws_misc.reserve(c, sizeof(double) * (size_t)blocks * kFmaThreads));
    float* sink = c->ws_misc.as<float>();
    cudaEvent_t e0, e1;
    MALA_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(MALA_ERR_CUDA, "cudaEventCreate failed");
    }
    double best[3] = {0.0, 0.0, 0.0};
    int rc = MALA_OK;
    for (int kind = 0; kind < 3 && rc == MALA_OK; ++kind) {
        const double fma_per_thread = kind == 2 ? (double)kFmaIters64 * 8.0 : (double)kFmaIters * 8.0 * (kind ? 2.0 : 1.0);
        const double flop = 2.0 * fma_per_thread * (double)blocks * kFmaThreads;
        for (int rep = 0; rep < 4; ++rep) {  // the first repetition warms clocks and caches
            cudaEventRecord(e0, st);
            if (kind == 0) k_fma_scalar<<<blocks, kFmaThreads, 0, st>>>(0.999999f, 1e-7f, sink);
            else if (kind == 1) k_fma_packed<<<blocks, kFmaThreads, 0, st>>>(0.999999f, 1e-7f, sink);
            else k_fma_f64<<<blocks, kFmaThreads, 0, st>>>(0.999999999, 1e-12, reinterpret_cast<double*>(sink));
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) {
                rc = fail(MALA_ERR_CUDA, "FMA probe failed: %s", cudaGetErrorString(e));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms > 0.f) best[kind] = std::max(best[kind], flop / (ms * 1e-3) / 1e12);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (scalar_tflops) *scalar_tflops = best[0];
    if (packed_tflops) *packed_tflops = best[1];
    if (fp64_tflops) *fp64_tflops = best[2];
    return rc;
}

}  // namespace mala

using namespace mala;

struct mala_ctx : public mala::Ctx {};

extern "C" int mala_measure_peaks(mala_ctx* c, double* fp32_scalar_tflops, double* fp32_packed_tflops,
                                  double* fp64_tflops) {
    if (!c) return fail(MALA_ERR_INVALID_ARG, "context is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    MALA_DEVICE_SCOPE(c->device);
    return measure_peaks(c, fp32_scalar_tflops, fp32_packed_tflops, fp64_tflops);
}
