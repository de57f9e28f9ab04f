// k_noalloc.cu -- discrete integrals sum_i m_i u_i without any device
// allocation.
//
// Who needs this: code that may not call cudaMalloc -- a caller recording a
// CUDA graph (allocation is not allowed while a stream is being captured), a
// framework that owns a fixed device-memory budget and forbids further
// allocations once it has started, or a host callback, which must not make
// CUDA calls that allocate. Such a caller can still check conservation: it
// passes its own device arrays for the state, the element areas, the
// simulation offsets and the result, and the per-element partial sums go to
// a fixed-size array that is part of this library's device image.
//
// The scratch array below exists once per device for as long as the library
// is loaded. Every call reuses it, so calls that overlap on the GPU (two
// streams, or two threads) race on it; serialise them. Each call overwrites
// the partials for elements [0, n_elems) before reading them, so no clearing
// is needed between calls.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/idp_dgsem.h"

namespace idp {
void host_lgl_weights(int N, double *w);   // defined in idp_host.cu
}

namespace {

// per-element partials, [4][IDP_NOALLOC_MAX_ELEMS]
static __device__ __align__(256) double g_noalloc_partials[4 * (size_t)IDP_NOALLOC_MAX_ELEMS];

struct Weights {
    double w[8];
};

// sum over the element's nodes of (dx dy / 4) w_i w_j u_v, node order fixed
__global__ void k_partials_noalloc(const double *__restrict__ u, const double *__restrict__ area, int K, int NP,
                                   Weights W, double *part) {
    const int NN = NP * NP;
    const size_t KN = (size_t)K * NN;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        double J = area[e] / 4.0;
        for (int v = 0; v < 4; ++v) {
            double s = 0.0;
            for (int n = 0; n < NN; ++n) s += J * W.w[n % NP] * W.w[n / NP] * u[v * KN + (size_t)e * NN + n];
            part[(size_t)v * IDP_NOALLOC_MAX_ELEMS + e] = s;
        }
    }
}

// per simulation: fixed-order tree sum of the partials in [off[s], off[s+1]),
// the offsets clamped to [0, K] (the partials of this call), so that a bad
// offset sums fewer partials instead of stale ones or memory past the array
__global__ void k_segments_noalloc(const double *part, const int64_t *off, long long K, double *out) {
    __shared__ double red[4][256];
    const int s = blockIdx.x;
    long long b = off[s], e = off[s + 1];
    b = b < 0 ? 0 : (b > K ? K : b);
    e = e < b ? b : (e > K ? K : e);
    double acc[4] = {0, 0, 0, 0};
    for (long long k = b + threadIdx.x; k < e; k += blockDim.x)
        for (int v = 0; v < 4; ++v) acc[v] += part[(size_t)v * IDP_NOALLOC_MAX_ELEMS + k];
    for (int v = 0; v < 4; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int v = 0; v < 4; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int v = 0; v < 4; ++v) out[4 * s + v] = red[v][0];
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (the host-side symbol is only a stand-in, not a device
// pointer).
idp_status scratch_for_current_device(double **ptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IDP_E_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return IDP_E_CUDA;
        g_scratch[dev] = (double *)p;
    }
    *ptr = g_scratch[dev];
    return IDP_OK;
}

}  // namespace

extern "C" idp_status idp_integrals_noalloc(const double *u, const double *elem_area, int64_t n_elems, int32_t N,
                                            const int64_t *sim_elem_offsets, int32_t n_sims, double *out,
                                            void *stream) {
    if (!u || !elem_area || !sim_elem_offsets || !out || n_sims < 1 || N < 1 || N > 7 || n_elems < 1)
        return IDP_E_ARG;
    if (n_elems > IDP_NOALLOC_MAX_ELEMS) return IDP_E_ARG;   // beyond the fixed scratch
    double *part = nullptr;
    idp_status st = scratch_for_current_device(&part);
    if (st != IDP_OK) return st;
    Weights W = {};
    idp::host_lgl_weights(N, W.w);
    cudaStream_t s = (cudaStream_t)stream;
    int blocks = (int)((n_elems + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_partials_noalloc<<<blocks, 256, 0, s>>>(u, elem_area, (int)n_elems, N + 1, W, part);
    k_segments_noalloc<<<n_sims, 256, 0, s>>>(part, sim_elem_offsets, (long long)n_elems, out);
    return cudaGetLastError() == cudaSuccess ? IDP_OK : IDP_E_CUDA;
}
