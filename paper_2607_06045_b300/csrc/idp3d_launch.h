// idp3d_launch.h -- the per-degree launcher table of the 3D kernels
// (instantiated in k_inst3d.cu, one translation unit per N + 1).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "idp3d_mortar.cuh"

namespace idp3 {

struct Launchers3 {
    int np = 0, epb = 0, epb64 = 0, threads = 0;   // elements per block: time step and FP32 form; FP64 element kernel
    size_t smem = 0, smem32 = 0;   // dynamic shared memory of one element-kernel block (FP64 path, FP32 form)
    cudaError_t (*prepare)() = nullptr;
    // the element kernel: FP64 path, FP32 form
    void (*element)(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const Stage3 &A) = nullptr;
    void (*element32)(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const Stage3 &A) = nullptr;
    // the time step: FP64 path (its wave speeds first, into lam[3][K (N+1)^3]), FP32 form
    // dt: the FP64 path's two passes (dtmin: 2 entries, the minimum and the
    // FP32 pass's; emin: one value per element); dt32: the FP32 form
    void (*dt)(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const double *u, double gamma,
               unsigned long long *dtmin, unsigned *status, unsigned *emin) = nullptr;
    void (*dt32)(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const double *u, double gamma,
                 unsigned long long *dtmin, unsigned *status, unsigned *emin) = nullptr;
    // the mortar kernels (grid: one block per mortar; apply: its own grid)
    void (*mflux)(cudaStream_t st, const Grid3 &G, const MOps3 *mo, const double *u, double gamma) = nullptr;
    void (*mfactor)(cudaStream_t st, const Grid3 &G, const Stage3 &A) = nullptr;
    void (*mapply)(cudaStream_t st, const Grid3 &G, const Stage3 &A) = nullptr;
};

Launchers3 launchers3_np2();
Launchers3 launchers3_np3();
Launchers3 launchers3_np4();
Launchers3 launchers3_np5();

}  // namespace idp3
