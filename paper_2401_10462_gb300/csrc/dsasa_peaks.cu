// Microbenchmarks of the arithmetic roofs that bound the dSASA kernels (none of them is a
// dense contraction or HBM bound): FP32 FMA, FP64 FMA, the special-function unit (rsqrt)
// and the library atan2f that the area terms call, each measured with CUDA events on a
// private stream, with every SM busy (grid = a multiple of the SM count) and many
// independent dependency chains per thread.  No clock or device setting is touched.
//
// Built into its own library (libdsasa_peaks.so) so that the product library carries no
// benchmark code; bench.py calls it once per run and reports the measured roofs beside the
// HBM copy and tensor peaks recorded for the machine (MEASURED_PEAKS.json).
#include <cuda_runtime.h>

#include <stdint.h>

namespace {

constexpr int kChains = 8;      // independent accumulators per thread
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma32(float* out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true: keeps the work
}

__global__ void __launch_bounds__(kThreads) k_fma64(double* out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(kThreads) k_rsqrt(float* out, int iters, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = rsqrtf(a[k]) + c;   // one MUFU + one FADD
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_atan2(float* out, int iters, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 0.5f + (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = atan2f(a[k], c) + c;
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of `reps` timed launches (ms) of one kernel configuration
template <class F> float best_ms(F launch, cudaStream_t s, int reps) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    launch();   // warm-up
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

// out[0] FP32 FMA TFLOP/s (2 flop per FMA), out[1] FP64 FMA TFLOP/s, out[2] rsqrt Gop/s
// (special-function unit), out[3] atan2f Gop/s (the library function the area terms call),
// out[4] warp instructions per second issued by the FP32 FMA kernel (G/s; every FMA warp
// instruction is one issue slot), out[5] the SM count used.  Returns 0, or a CUDA error code.
extern "C" int dsasa_peaks_measure(int device, double* out) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return (int)e;
    const int blocks = sms * 8;   // 8 blocks of 256 threads per SM: 64 warps, full occupancy
    float* sink = nullptr;
    e = cudaMalloc(&sink, sizeof(double) * blocks * kThreads);
    if (e != cudaSuccess) { cudaStreamDestroy(s); return (int)e; }
    const double threads = (double)blocks * kThreads;
    const int it32 = 2048, it64 = 64, itr = 512, ita = 128;
    float ms = best_ms([&] { k_fma32<<<blocks, kThreads, 0, s>>>(sink, it32, 0.9999f, 1e-4f); }, s, 5);
    const double fma32 = threads * it32 * 16.0 * kChains;
    out[0] = 2.0 * fma32 / (ms * 1e-3) / 1e12;
    out[4] = fma32 / 32.0 / (ms * 1e-3) / 1e9;
    ms = best_ms([&] { k_fma64<<<blocks, kThreads, 0, s>>>((double*)sink, it64, 0.9999, 1e-4); }, s, 5);
    out[1] = 2.0 * threads * it64 * 4.0 * kChains / (ms * 1e-3) / 1e12;
    ms = best_ms([&] { k_rsqrt<<<blocks, kThreads, 0, s>>>(sink, itr, 0.5f); }, s, 5);
    out[2] = threads * itr * 4.0 * kChains / (ms * 1e-3) / 1e9;
    ms = best_ms([&] { k_atan2<<<blocks, kThreads, 0, s>>>(sink, ita, 0.7f); }, s, 5);
    out[3] = threads * ita * kChains / (ms * 1e-3) / 1e9;
    out[5] = sms;
    e = cudaGetLastError();
    cudaFree(sink);
    cudaStreamDestroy(s);
    return (int)e;
}
