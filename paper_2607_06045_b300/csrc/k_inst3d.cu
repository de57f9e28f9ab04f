// k_inst3d.cu -- the 3D kernels of one polynomial degree (IDP3_NP = N + 1 on
// the compiler command line) behind a launcher table.
#include "idp3d_launch.h"

#ifndef IDP3_NP
#error "IDP3_NP must be defined"
#endif

#define IDP3_CAT2(a, b) a##b
#define IDP3_CAT(a, b) IDP3_CAT2(a, b)

namespace idp3 {
namespace {

constexpr int NP = IDP3_NP;
// elements per block: about 128 threads, one per node
constexpr int EPB = NP == 2 ? 16 : (NP == 3 ? 4 : (NP == 4 ? 2 : 1));   // time step, FP32 form
constexpr int EPB64 = EPB;                                              // FP64 element kernel
using L3 = Launch3<NP, EPB>;
using L64 = Launch3<NP, EPB64>;

cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_element3d<NP, EPB64, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(Sm3<NP, double>) * EPB64));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_element3d<NP, EPB, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(Sm3<NP, float>) * EPB));
}

void element(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const Stage3 &A) {
    k_element3d<NP, EPB64, double><<<grid, L64::threads, sizeof(Sm3<NP, double>) * EPB64, st>>>(G, ops, A);
}

void element32(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const Stage3 &A) {
    k_element3d<NP, EPB, float><<<grid, L3::threads, sizeof(Sm3<NP, float>) * EPB, st>>>(G, ops, A);
}

// FP64 path: the FP32 pass into dtmin[1] (reset first) and the elements'
// minima, then the FP64 quotients of the picked elements into dtmin[0]
void dt(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const double *u, double gamma,
        unsigned long long *dtmin, unsigned *status, unsigned *emin) {
    k_inf3d<<<1, 32, 0, st>>>(dtmin + 1);
    k_dt3d<NP, EPB, float><<<grid, L3::threads, 0, st>>>(G, ops, u, gamma, dtmin + 1, status,
                                                          DtPick3{1, emin, nullptr});
    k_dt3d<NP, EPB, double><<<grid, L3::threads, 0, st>>>(G, ops, u, gamma, dtmin, status,
                                                           DtPick3{2, emin, dtmin + 1});
}

void dt32(int grid, cudaStream_t st, const Grid3 &G, const Ops3 *ops, const double *u, double gamma,
          unsigned long long *dtmin, unsigned *status, unsigned *) {
    k_dt3d<NP, EPB, float><<<grid, L3::threads, 0, st>>>(G, ops, u, gamma, dtmin, status,
                                                          DtPick3{0, nullptr, nullptr});
}

void mflux(cudaStream_t st, const Grid3 &G, const MOps3 *mo, const double *u, double gamma) {
    k_mflux3<NP><<<G.mort.M, kMortThreads3, 0, st>>>(G, mo, u, gamma);
}

void mfactor(cudaStream_t st, const Grid3 &G, const Stage3 &A) {
    k_mfactor3<NP><<<G.mort.M, kMortThreads3, 0, st>>>(G, A);
}

void mapply(cudaStream_t st, const Grid3 &G, const Stage3 &A) {
    const int blocks = (G.mort.MN + 255) / 256;
    k_mapply3<NP><<<blocks < 1184 ? blocks : 1184, 256, 0, st>>>(G, A);
}

}  // namespace

Launchers3 IDP3_CAT(launchers3_np, IDP3_NP)() {
    Launchers3 L;
    L.np = NP;
    L.epb = EPB;
    L.epb64 = EPB64;
    L.threads = L3::threads;
    L.smem = sizeof(Sm3<NP, double>) * EPB64;
    L.smem32 = sizeof(Sm3<NP, float>) * EPB;
    L.prepare = prepare;
    L.element = element;
    L.element32 = element32;
    L.dt = dt;
    L.dt32 = dt32;
    L.mflux = mflux;
    L.mfactor = mfactor;
    L.mapply = mapply;
    return L;
}

}  // namespace idp3
