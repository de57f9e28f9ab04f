// idp_launch.cuh -- per-degree kernel launchers. Each polynomial degree is
// compiled in its own translation unit (k_inst.cu with IDP_NP = N + 1); the
// host selects the table for its N at create time.
#pragma once

#include "idp_amr.cuh"
#include "idp_mortar.cuh"

namespace idp {

constexpr int kEpbChoices[] = {1, 2, 4, 8, 16};
constexpr int kNumEpb = 5;

struct Launchers {
    int np;
    // element pass: fp32 selects the FP32 form, ext the extended kernel of
    // the local-limiting variants; epb = elements per block
    size_t (*element_smem)(int fp32, int ext, int epb);
    int (*element_threads)(int epb);
    cudaError_t (*element_prepare)(int fp32, int ext, int epb, int *blocks_per_sm);
    void (*element)(int fp32, int ext, int epb, int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s,
                    const StageArgs &a);
    // conforming-face fluxes of the FP64 element pass (k_face)
    void (*face)(cudaStream_t st, const MeshDev &m, const double *u, const Gas &gas, const Ops *ops, double *fbuf,
                 int num_sms);
    void (*mortar_flux)(int fp32, int ent, int a2a, int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s,
                        const double *u, const Gas &gas, const Ops *ops);
    void (*mortar_lob)(cudaStream_t st, const MeshDev &m, const SlotsDev &s, const Ops *ops, const double *lofv,
                       int ent, int num_sms);
    // mortar limiting and the limited corrections (k_mortar_limit_apply),
    // mortar_w own mortars per block
    void (*mortar_limit)(int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s, const StageArgs &a);
    int mortar_w;
    // time step; lam (when not null): the wave speeds of every node,
    // 2 K (N+1)^2 values in the flux type, written by dt_speed first; filt
    // 1 and 2: the two passes of the FP64 path's time step with the face
    // buffer (k_dt's DtFilter; emin: one value per element; dtmin: 2 n_sims
    // entries)
    void (*dt)(int fp32, int grid, cudaStream_t st, const MeshDev &m, const SlotsDev &s, const double *u,
               const Gas &gas, int rule, const Ops *ops, const double *t_sim, unsigned long long *dtmin,
               unsigned *status, const double *fbuf, const void *lam, int filt, unsigned *emin);
    void (*dt_speed)(int fp32, cudaStream_t st, const MeshDev &m, const double *u, const Gas &gas,
                     unsigned *status, void *lam, int num_sms);
    void (*integrals)(int grid, cudaStream_t st, const MeshDev &m, const double *u, const Ops *ops, double *part);
    // adaptive mesh refinement (idp_amr.cuh)
    void (*amr_indicator)(cudaStream_t st, const double *u, int K, const Ops *ops, double gm1, int kind, int var,
                          double filt, double *ind, int num_sms);
    void (*amr_transfer)(cudaStream_t st, const double *uo, int Ko, double *un, int Kn, const int *kind,
                         const int4 *src, const Ops *ops, int num_sms);
    void (*amr_zs)(cudaStream_t st, double *un, int Kn, const double *uo, int Ko, const int4 *fam, int nfam,
                   const Ops *ops, double gm1, double eps, unsigned long long *nscaled);
};

Launchers launchers_np2();
Launchers launchers_np3();
Launchers launchers_np4();
Launchers launchers_np5();
Launchers launchers_np6();
Launchers launchers_np7();
Launchers launchers_np8();

}  // namespace idp
