// Measured peaks of the SM pipes the pair passes run on (the ALU roofline's
// denominators): independent chains of FP32 fused multiply-adds, FP64 fused
// multiply-adds, or FP32 reciprocal square roots (the special-function unit),
// enough warps and chains per warp to keep each pipe issuing every cycle.
#include <cuda_runtime.h>

#include "gz.h"

namespace {

constexpr int kChains = 8;    // independent dependency chains per thread
constexpr int kIters = 8192;  // chain steps per thread (FP64: 1/16, SFU: 1/4 of it)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_ffma(float* out, float x, float y) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (float)(threadIdx.x + c);
#pragma unroll 4
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], x, y);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_dfma(double* out, double x, double y) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (double)(threadIdx.x + c);
#pragma unroll 4
    for (int it = 0; it < kIters / 16; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_mufu(float* out, float y) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1.f + (float)(threadIdx.x + c);
#pragma unroll 4
    for (int it = 0; it < kIters / 4; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = rsqrtf(a[c] + y);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" gz_status gz_measure_alu(int32_t which, double* ops_per_s, void* cuda_stream) {
    if (!ops_per_s || which < 0 || which > 2) return GZ_E_INVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GZ_E_CUDA;
    const int grid = sms * 8;  // 8 blocks of 256 threads per SM: 64 warps
    void* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)grid * kThreads) != cudaSuccess) {
        cudaGetLastError();
        return GZ_E_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double per_thread = 0.0;
    float best = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // first launch warms up
        cudaEventRecord(e0, st);
        if (which == 0) {
            k_ffma<<<grid, kThreads, 0, st>>>((float*)buf, 0.9999999f, 1e-7f);
            per_thread = 2.0 * kChains * kIters;
        } else if (which == 1) {
            k_dfma<<<grid, kThreads, 0, st>>>((double*)buf, 0.9999999999, 1e-12);
            per_thread = 2.0 * kChains * (kIters / 16);
        } else {
            k_mufu<<<grid, kThreads, 0, st>>>((float*)buf, 1e-3f);
            per_thread = (double)kChains * (kIters / 4);
        }
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess) return GZ_E_CUDA;
    *ops_per_s = per_thread * grid * kThreads / (best * 1e-3);
    return GZ_OK;
}
