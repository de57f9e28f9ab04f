// k_probe.cu -- pipe-throughput probes used for the roofline of the
// FP64-bound kernels (the paper has no counterpart): DFMA and FFMA
// throughput, and the cost of the FP64 reciprocal, square root and logarithm
// that the FP64 flux arithmetic uses (idp_fastmath.cuh), in
// DFMA-equivalents. Every thread runs long chains of independent operations;
// the results are kept live by a data-dependent store. Also a test hook that
// evaluates those routines on device arrays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/idp_dgsem.h"
#include "idp_fastmath.cuh"

namespace idp {
void host_log_table(LogTab &T);   // idp_host.cu
}

namespace {

constexpr int kChains = 8;

__global__ void probe_dfma(double *sink, int iters, double a, double b) {
    double x[kChains];
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 123.456) sink[threadIdx.x] = s;
}

__global__ void probe_ffma(float *sink, int iters, float a, float b) {
    float x[kChains];
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 123.456f) sink[threadIdx.x] = s;
}

// op: 0 reciprocal, 1 square root, 2 natural logarithm (idp_fastmath.cuh)
__global__ void probe_op(double *sink, int iters, int op, const idp::LogTab *T) {
    double x[kChains];
    for (int c = 0; c < kChains; ++c) x[c] = 1.5 + threadIdx.x * 1e-4 + c * 0.1;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (op == 0) x[c] = idp::fast_rcp(x[c]) + 1.0;
            else if (op == 1) x[c] = idp::fast_sqrt(x[c]) + 1.0;
            else x[c] = idp::fast_log(x[c], T) + 1.75;
        }
    double s = 0.0;
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 123.456) sink[threadIdx.x] = s;
}

}  // namespace

static __global__ void eval_math(int fn, const double *x, double *y, long long n, const idp::LogTab *T) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fn == 0 ? idp::fast_rcp(x[i]) : (fn == 1 ? idp::fast_sqrt(x[i]) : idp::fast_log(x[i], T));
}

static idp::LogTab *device_log_table() {
    idp::LogTab h, *d = nullptr;
    idp::host_log_table(h);
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) { cudaFree(d); return nullptr; }
    return d;
}

extern "C" idp_status idp_eval_math(int32_t fn, const double *x, double *y, int64_t n, void *stream) {
    if (fn < 0 || fn > 2 || n < 0 || (n > 0 && (!x || !y))) return IDP_E_ARG;
    if (n == 0) return IDP_OK;
    idp::LogTab *T = device_log_table();
    if (!T) return IDP_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    eval_math<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(fn, x, y, n, T);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(T);
    return e == cudaSuccess ? IDP_OK : IDP_E_CUDA;
}

extern "C" idp_status idp_probe_pipes(double *out, void *stream) {
    if (!out) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return IDP_E_CUDA;
    double *sink = nullptr;
    if (cudaMalloc(&sink, 1024 * sizeof(double)) != cudaSuccess) return IDP_E_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    auto timed = [&](auto launch) {
        launch();   // warm-up
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return (double)ms * 1e-3;
    };
    idp::LogTab *T = device_log_table();
    if (!T) { cudaFree(sink); return IDP_E_CUDA; }
    const int it_d = 2048, it_f = 65536, it_op = 256;
    double td = timed([&] { probe_dfma<<<blocks, threads, 0, st>>>(sink, it_d, 0.999999, 1e-7); });
    double tf = timed([&] { probe_ffma<<<blocks, threads, 0, st>>>((float *)sink, it_f, 0.999999f, 1e-7f); });
    double nd = (double)blocks * threads * it_d * kChains, nf = (double)blocks * threads * it_f * kChains;
    out[0] = 2.0 * nd / td * 1e-12;   // FP64 TFLOP/s (FMA = 2 flops)
    out[1] = 2.0 * nf / tf * 1e-12;   // FP32 TFLOP/s
    double per_dfma = td / nd;
    for (int op = 0; op < 3; ++op) {
        double t = timed([&] { probe_op<<<blocks, threads, 0, st>>>(sink, it_op, op, T); });
        double n = (double)blocks * threads * it_op * kChains;
        out[2 + op] = (t / n) / per_dfma;   // DFMA-equivalents per operation (incl. its add)
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    cudaFree(sink);
    cudaFree(T);
    return e == cudaSuccess ? IDP_OK : IDP_E_CUDA;
}
