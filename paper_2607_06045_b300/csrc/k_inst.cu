// k_inst.cu -- instantiates the kernels of one polynomial degree (IDP_NP =
// N + 1, set on the compiler command line) and exposes them as a launcher
// table.
#include <algorithm>

#include "idp_launch.cuh"

#ifndef IDP_NP
#error "IDP_NP must be defined"
#endif

#define IDP_CAT2(a, b) a##b
#define IDP_CAT(a, b) IDP_CAT2(a, b)

namespace idp {
namespace {

constexpr int NP = IDP_NP;

template <typename FT, int EPB, bool EXT>
void el_launch(int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s, const StageArgs &a) {
    size_t smem = sizeof(ElemSm<NP, FT, EXT>) * EPB;
    k_element<NP, FT, EPB, EXT><<<grid, ElemLaunch<NP, EPB>::threads, smem, st>>>(m, s, a);
}

template <typename FT, int EPB, bool EXT>
cudaError_t el_prepare(int *bps) {
    size_t smem = sizeof(ElemSm<NP, FT, EXT>) * EPB;
    cudaError_t e = cudaFuncSetAttribute(k_element<NP, FT, EPB, EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_element<NP, FT, EPB, EXT>,
                                                         ElemLaunch<NP, EPB>::threads, smem);
}

size_t element_smem(int fp32, int ext, int epb) {
    size_t per = ext ? (fp32 ? sizeof(ElemSm<NP, float, true>) : sizeof(ElemSm<NP, double, true>))
                     : (fp32 ? sizeof(ElemSm<NP, float>) : sizeof(ElemSm<NP, double>));
    return per * (size_t)epb;
}

int element_threads(int epb) {
    switch (epb) {
    case 1: return ElemLaunch<NP, 1>::threads;
    case 2: return ElemLaunch<NP, 2>::threads;
    case 4: return ElemLaunch<NP, 4>::threads;
    case 8: return ElemLaunch<NP, 8>::threads;
    default: return ElemLaunch<NP, 16>::threads;
    }
}

// dispatch on (precision, extended kernel, elements per block)
#define IDP_EPB_CASE(FN, E, ...)                                                               \
    case E:                                                                                    \
        if (ext) return fp32 ? FN<float, E, true>(__VA_ARGS__) : FN<double, E, true>(__VA_ARGS__); \
        return fp32 ? FN<float, E, false>(__VA_ARGS__) : FN<double, E, false>(__VA_ARGS__);
#define IDP_EPB_SWITCH(FN, ...)               \
    switch (epb) {                            \
    IDP_EPB_CASE(FN, 1, __VA_ARGS__)          \
    IDP_EPB_CASE(FN, 2, __VA_ARGS__)          \
    IDP_EPB_CASE(FN, 4, __VA_ARGS__)          \
    IDP_EPB_CASE(FN, 8, __VA_ARGS__)          \
    default:                                  \
        if (ext) return fp32 ? FN<float, 16, true>(__VA_ARGS__) : FN<double, 16, true>(__VA_ARGS__); \
        return fp32 ? FN<float, 16, false>(__VA_ARGS__) : FN<double, 16, false>(__VA_ARGS__); \
    }

cudaError_t element_prepare(int fp32, int ext, int epb, int *bps) {
    if (ElemLaunch<NP, 16>::threads > 1024 && epb == 16) return cudaErrorInvalidConfiguration;
    IDP_EPB_SWITCH(el_prepare, bps)
}

void element(int fp32, int ext, int epb, int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s,
             const StageArgs &a) {
    IDP_EPB_SWITCH(el_launch, grid, st, m, s, a)
}

void face(cudaStream_t st, const MeshDev &m, const double *u, const Gas &gas, const Ops *ops, double *fbuf,
          int num_sms) {
    const long long F = 2ll * m.K * NP;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((F + 255) / 256, (long long)num_sms * 16));
    k_face<NP><<<blocks, 256, 0, st>>>(m, u, gas, ops, fbuf);
}

void mortar_flux(int fp32, int ent, int a2a, int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s,
                 const double *u, const Gas &gas, const Ops *ops) {
    constexpr int T = 32 * MORTARS_PER_BLOCK;
    if (a2a) {
        if (fp32) k_mortar_flux<NP, float, true><<<grid, T, 0, st>>>(m, s, u, gas, ops, ent);
        else k_mortar_flux<NP, double, true><<<grid, T, 0, st>>>(m, s, u, gas, ops, ent);
    } else {
        if (fp32) k_mortar_flux<NP, float, false><<<grid, T, 0, st>>>(m, s, u, gas, ops, ent);
        else k_mortar_flux<NP, double, false><<<grid, T, 0, st>>>(m, s, u, gas, ops, ent);
    }
}

void mortar_lob(cudaStream_t st, const MeshDev &m, const SlotsDev &s, const Ops *ops, const double *lofv, int ent,
                int num_sms) {
    const int blocks = std::max(1, std::min((s.S + 127) / 128, num_sms * 16));
    k_mortar_lob<NP><<<blocks, 128, 0, st>>>(m, s, ops, lofv, ent);
}

void mortar_limit(int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s, const StageArgs &a) {
    (void)grid;
    if (m.mb_blocks > 0)
        k_mortar_limit_apply<NP><<<m.mb_blocks, MortarLaunch<NP>::threads, mortar_smem<NP>(m.mb_fmax), st>>>(m, s, a);
}

void dt_speed(int fp32, cudaStream_t st, const MeshDev &m, const double *u, const Gas &gamma, unsigned *status,
              void *lam, int num_sms) {
    const long long KN = (long long)m.K * NP * NP;
    const int sb = (int)std::max<long long>(1, std::min<long long>((KN + 255) / 256, (long long)num_sms * 32));
    if (fp32) k_dt_speed<NP, float><<<sb, 256, 0, st>>>(m, u, gamma, status, (float *)lam);
    else k_dt_speed<NP, double><<<sb, 256, 0, st>>>(m, u, gamma, status, (double *)lam);
}

void dt(int fp32, int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s, const double *u, const Gas &gamma,
        int rule, const Ops *ops, const double *t_sim, unsigned long long *dtmin, unsigned *status,
        const double *fbuf, const void *lam, int filt, unsigned *emin) {
    constexpr int EPB = NP * NP >= 64 ? 2 : (NP * NP >= 25 ? 4 : 8);
    int blocks = (m.K + EPB - 1) / EPB;
    const int n = m.n_sims;
    if (filt == 1) {
        // the FP64 path's two passes: FP32 minima into dtmin[n..2n) and emin,
        k_dt<NP, EPB, float><<<blocks, ElemLaunch<NP, EPB>::threads, 0, st>>>(
            m, s, u, gamma, rule, ops, t_sim, dtmin + n, status, fbuf, nullptr, DtFilter{1, emin, nullptr});
    } else if (filt == 2) {
        // then the FP64 quotients of the candidate elements into dtmin[0..n)
        k_dt<NP, EPB, double><<<blocks, ElemLaunch<NP, EPB>::threads, 0, st>>>(
            m, s, u, gamma, rule, ops, t_sim, dtmin, status, fbuf, nullptr, DtFilter{2, emin, dtmin + n});
    } else if (fp32) {
        k_dt<NP, EPB, float><<<blocks, ElemLaunch<NP, EPB>::threads, 0, st>>>(
            m, s, u, gamma, rule, ops, t_sim, dtmin, status, nullptr, (const float *)lam, DtFilter{0, nullptr, nullptr});
    } else {
        k_dt<NP, EPB, double><<<blocks, ElemLaunch<NP, EPB>::threads, 0, st>>>(
            m, s, u, gamma, rule, ops, t_sim, dtmin, status, fbuf, (const double *)lam, DtFilter{0, nullptr, nullptr});
    }
    (void)grid;
}

void integrals(int grid, cudaStream_t st, const MeshDev &m, const double *u, const Ops *ops, double *part) {
    k_elem_integrals<NP><<<grid, 256, 0, st>>>(m, u, ops, part);
}

void amr_indicator(cudaStream_t st, const double *u, int K, const Ops *ops, double gm1, int kind, int var, double filt,
                   double *ind, int num_sms) {
    const int blocks = std::max(1, std::min((K + 127) / 128, num_sms * 8));
    k_amr_indicator<NP><<<blocks, 128, 0, st>>>(u, K, ops, gm1, kind, var, filt, ind);
}

void amr_transfer(cudaStream_t st, const double *uo, int Ko, double *un, int Kn, const int *kind, const int4 *src,
                  const Ops *ops, int num_sms) {
    const long long nodes = (long long)Kn * NP * NP;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((nodes + 255) / 256, (long long)num_sms * 16));
    k_amr_transfer<NP><<<blocks, 256, 0, st>>>(uo, Ko, un, Kn, kind, src, ops);
}

void amr_zs(cudaStream_t st, double *un, int Kn, const double *uo, int Ko, const int4 *fam, int nfam, const Ops *ops,
            double gm1, double eps, unsigned long long *nscaled) {
    if (nfam <= 0) return;
    k_amr_zs<NP><<<(nfam + 3) / 4, 128, 0, st>>>(un, Kn, uo, Ko, fam, nfam, ops, gm1, eps, nscaled);
}

}  // namespace

Launchers IDP_CAT(launchers_np, IDP_NP)() {
    Launchers L;
    L.np = NP;
    L.element_smem = element_smem;
    L.element_threads = element_threads;
    L.element_prepare = element_prepare;
    L.element = element;
    L.face = face;
    L.mortar_flux = mortar_flux;
    L.mortar_lob = mortar_lob;
    L.mortar_limit = mortar_limit;
    L.mortar_w = MortarLaunch<NP>::W;
    L.dt = dt;
    L.dt_speed = dt_speed;
    L.integrals = integrals;
    L.amr_indicator = amr_indicator;
    L.amr_transfer = amr_transfer;
    L.amr_zs = amr_zs;
    return L;
}

}  // namespace idp
