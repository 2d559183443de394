// Arithmetic peaks of the GPU the library runs on, measured with dependent
// FMA chains (no counterpart in the paper: the H.psi kernels are compared
// with these rates, next to the HBM bandwidth).  Each thread runs kChains
// independent chains of `iters` fused multiply-adds; the grid fills every SM
// with 2048 threads, so each scheduler always has an independent FMA to
// issue.  The chains stay bounded (x <- x * b + c with |b| < 1).
#include "device_util.cuh"

namespace pq {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32(int iters, float b, float c,
                                                           float* sink) {
    float x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) x[i] = __fmaf_rn(x[i], b, c);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i];
    if (s == 12345.678f) sink[threadIdx.x] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f32x2(int iters, float b, float c,
                                                             float* sink) {
    float2 x[kPeakChains];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i)
        x[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i * 1e-3f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) x[i] = __ffma2_rn(x[i], b2, c2);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i].x + x[i].y;
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_f64(int iters, double b, double c,
                                                           double* sink) {
    double x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) x[i] = __fma_rn(x[i], b, c);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i];
    if (s == 12345.678) sink[threadIdx.x] = s;
}

}  // namespace pq

using namespace pq;

extern "C" __attribute__((visibility("default"))) pq_status pq_measure_peak(int kind, int iters,
                                                                            double* ms_out,
                                                                            double* flop_out) {
    clear_error();
    if (!ms_out || !flop_out || iters < 1 || kind < PQ_PEAK_FP32 || kind > PQ_PEAK_FP64) {
        set_error("bad peak request (kind, iters >= 1, outputs)");
        return PQ_EINVAL;
    }
    const int G = grid_size() * (2048 / kPeakThreads);
    double* sink = nullptr;
    PQ_CUDA_TRY(cudaMalloc(&sink, kPeakThreads * sizeof(double)));
    cudaEvent_t e0, e1;
    PQ_CUDA_TRY(cudaEventCreate(&e0));
    PQ_CUDA_TRY(cudaEventCreate(&e1));
    auto launch = [&]() {
        if (kind == PQ_PEAK_FP32)
            k_peak_f32<<<G, kPeakThreads>>>(iters, 0.999f, 1e-4f, (float*)sink);
        else if (kind == PQ_PEAK_FP32X2)
            k_peak_f32x2<<<G, kPeakThreads>>>(iters, 0.999f, 1e-4f, (float*)sink);
        else
            k_peak_f64<<<G, kPeakThreads>>>(iters, 0.999, 1e-4, sink);
    };
    launch();   // warm-up
    PQ_CUDA_TRY(cudaEventRecord(e0));
    launch();
    PQ_CUDA_TRY(cudaEventRecord(e1));
    PQ_CUDA_TRY(cudaEventSynchronize(e1));
    PQ_LAUNCHED();
    PQ_LAUNCHED();
    float ms = 0.f;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) {
        set_error("peak kernel: %s", cudaGetErrorString(e));
        return PQ_ECUDA;
    }
    const double lanes = kind == PQ_PEAK_FP32X2 ? 2.0 : 1.0;
    *ms_out = ms;
    *flop_out = 2.0 * lanes * kPeakChains * (double)iters * (double)G * kPeakThreads;
    return PQ_OK;
}
