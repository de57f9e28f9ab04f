// idp_mortar.cuh -- face-list kernels at nonconforming interfaces and the
// per-step reductions of the IDP LGL-DGSEM (arXiv 2607.06045).
//
//  k_mortar_flux   per block of mortars: high-order L2 mortar flux (Sec. 2.3,
//                  interpolate, LLF on the two small faces, project back) and
//                  the sparse low-order IDP mortar flux (Eq. interfaceflux_local)
//                  with its bar states and graph-viscosity sums.
//  k_mortar_limit_apply  one factor l_S per mortar after the volume
//                  correction, each node's correction budget scaled by its
//                  number of mortars n_i (Sec. 2.3, mortar limiting), then the
//                  limited corrections at the mortar nodes in mortar order and
//                  the stage there, in one launch.
//  k_dt            IDP time step (Eq. timestep_restriction) or the low-order
//                  CFL estimate (Eq. CFLcondition_lowordermethod), per simulation.
#pragma once

#include "idp_element.cuh"

namespace idp {

constexpr int MORTARS_PER_BLOCK = 4;   // mortars of one block (32 threads each)

// FT: flux arithmetic type (FP32 in the FP32 form). Interpolation, the
// admissibility test, bar states and all sums are FP64.
template <int NP, typename FT>
__device__ __forceinline__ Prim<FT> mortar_prim(const Gas &g, const double *q) {
    if constexpr (sizeof(FT) == 4) {
        float a, b;
        return make_prim_f32(g, q[0], q[1], q[2], q[3], false, a, b);
    } else {
        return make_prim<FT>(g, q[0], q[1], q[2], q[3], false);
    }
}

// MORTARS_PER_BLOCK mortars per block. Every phase is one loop of the whole
// block over the items of all its mortars -- (node, variable) items for the
// interpolation and the projection, one small-face node each for the LLF
// fluxes, one nonzero weight each for the low-order pair terms -- so the
// phases with few items per mortar still fill whole warps. Every pair term is
// formed once and summed into both of its slots in a fixed order.
// ent: also the minimum over each slot's bar states of s = ln p - gamma ln rho
// (entropy bound of local limiting with bar-state bounds).
// A2A: all-to-all weights (every large node with every small-face node).
template <int NP, typename FT, bool A2A>
__global__ void __launch_bounds__(32 * MORTARS_PER_BLOCK)
k_mortar_flux(MeshDev mesh, SlotsDev sl, const double *__restrict__ u, Gas gas, const Ops *ops, int ent) {
    constexpr int NN = NP * NP, Q = 3 * NP, NI = 2 * NP, MP = A2A ? 2 * NP * NP : 3 * NP, W = MORTARS_PER_BLOCK;
    constexpr int NT = 32 * W;
    __shared__ double s_u[W][Q][4];      // traces: large side, then the two small faces
    __shared__ FT s_uf[W][Q][4];         // the same in the flux type
    __shared__ FT s_pr[W][Q][3];         // normal velocity, p, c
    __shared__ double s_ui[W][NI][4];    // large trace interpolated to the small-face nodes
    __shared__ FT s_f[W][NI][4];         // LLF flux on the small faces
    __shared__ double s_term[W][MP][4];  // sparse low-order pair terms
    __shared__ double s_rb[W][MP];       // their bar-state densities
    __shared__ FT s_d2[W][MP];           // and 2 d
    __shared__ double s_sb[W][MP];       // and their s (entropy bound)
    __shared__ int s_info[W], s_L[W], s_bad[W];
    __shared__ int2 s_sm[W];
    __shared__ double s_halfL[W];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * W;
    const int nm = min(W, mesh.M - m0);   // mortars of this block
    if (nm <= 0) return;                  // uniform per block
    const size_t KN = (size_t)mesh.K * NN;
    const Gas &g = gas;
    constexpr bool F32 = sizeof(FT) == 4;
    if (tid < nm) {
        const int m = m0 + tid, info = mesh.m_info[m], L = mesh.m_large[m];
        const Geo geoL = mesh.geom[L];
        s_info[tid] = info;
        s_L[tid] = L;
        s_sm[tid] = mesh.m_small[m];
        s_halfL[tid] = (info & 1) == 0 ? 0.5 * geoL.w : 0.5 * geoL.z;
        s_bad[tid] = 0;
    }
    __syncthreads();
    // traces and their primitives
    for (int it = tid; it < nm * Q; it += NT) {
        const int mi = it / Q, q = it - mi * Q;
        const int info = s_info[mi], dir = info & 1, low = (info >> 1) & 1;
        const int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2), sS = sL ^ 1;
        int gnode;
        if (q < NP) gnode = s_L[mi] * NN + face_node<NP>(sL, q);
        else {
            int p = (q - NP) / NP, l = (q - NP) % NP;
            gnode = (p == 0 ? s_sm[mi].x : s_sm[mi].y) * NN + face_node<NP>(sS, l);
        }
        double qv[4];
        for (int v = 0; v < 4; ++v) { qv[v] = u[v * KN + gnode]; s_u[mi][q][v] = qv[v]; }
        Prim<FT> pr;
        if constexpr (F32) {
            float m1f, m2f;
            pr = make_prim_f32(g, qv[0], qv[1], qv[2], qv[3], false, m1f, m2f);
            s_uf[mi][q][0] = pr.rho; s_uf[mi][q][1] = m1f; s_uf[mi][q][2] = m2f;
            s_uf[mi][q][3] = pr.E;
        } else {
            pr = make_prim<FT>(g, qv[0], qv[1], qv[2], qv[3], false);
            for (int v = 0; v < 4; ++v) s_uf[mi][q][v] = qv[v];
        }
        s_pr[mi][q][0] = dir == 0 ? pr.v1 : pr.v2;
        s_pr[mi][q][1] = pr.p;
        s_pr[mi][q][2] = pr.c;
    }
    __syncthreads();
    // interpolation of the large trace to the small-face nodes (FP64)
    for (int it = tid; it < nm * NI * 4; it += NT) {
        const int mi = it / (NI * 4), rem = it - mi * (NI * 4), r = rem >> 2, v = rem & 3;
        double acc = 0.0;
        for (int k = 0; k < NP; ++k) acc += ops->I[r][k] * s_u[mi][k][v];
        s_ui[mi][r][v] = acc;
    }
    // low-order pair terms (Eq. interfaceflux_local) with their bar states
    // and 2 d; term enters the large slot with -, the small with +
    const int npair = ops->npair;
    for (int it = tid; it < nm * npair; it += NT) {
        const int mi = it / npair, pp = it - mi * npair;
        const int info = s_info[mi], dir = info & 1, low = (info >> 1) & 1;
        const double sg = low ? 1.0 : -1.0;   // large side's outward normal along +dir
        const int k = ops->pk[pp], r = ops->pr[pp];
        const double wt = ops->wt[k][r] * s_halfL[mi];
        const double *a = s_u[mi][k], *b = s_u[mi][NP + r];
        const FT *af = s_uf[mi][k], *bf = s_uf[mi][NP + r];
        const FT *pa = s_pr[mi][k], *pb = s_pr[mi][NP + r];
        FT la = fabs(pa[0]) + pa[2], lb = fabs(pb[0]) + pb[2];
        FT lam = speed_max(la, lb);
        FT fa[4], fb[4];
        phys_flux<FT>(af[1], af[2], af[3], pa[1], pa[0], dir, fa);
        phys_flux<FT>(bf[1], bf[2], bf[3], pb[1], pb[0], dir, fb);
        const FT sgf = low ? FT(1) : FT(-1);
        FT hw, i2l_f;
        double i2l;
        if constexpr (F32) { hw = d2f(0.5 * wt); i2l_f = 0.5f / lam; i2l = f2d(i2l_f); }
        else { hw = 0.5 * wt; i2l = 0.5 * fast_rcp(lam); }
        // the all-to-all weights can be negative: c_ij = omega n / 2 and
        // d_ij = |c_ij| lambda, so the bar state looks along sign(omega) n
        const double sgw = (A2A && wt < 0.0) ? -sg : sg;
        for (int v = 0; v < 4; ++v) {
            FT term;
            if constexpr (A2A) term = hw * (sgf * fa[v] + sgf * fb[v]) - fabs(hw) * lam * (bf[v] - af[v]);
            else term = hw * ((sgf * fa[v] + sgf * fb[v]) - lam * (bf[v] - af[v]));
            if constexpr (F32) s_term[mi][pp][v] = f2d(term);
            else s_term[mi][pp][v] = term;
        }
        s_rb[mi][pp] = 0.5 * (a[0] + b[0]) - sgw * (b[1 + dir] - a[1 + dir]) * i2l;
        if (ent) {
            const bool pos = sgw > 0.0;
            if constexpr (F32) s_sb[mi][pp] = bar_entropy<float>(g, af, fa, bf, fb, pos ? i2l_f : -i2l_f);
            else s_sb[mi][pp] = bar_entropy<double>(g, a, fa, b, fb, pos ? i2l : -i2l);
        }
        FT wtf;
        if constexpr (F32) wtf = d2f(fabs(wt));
        else wtf = fabs(wt);
        s_d2[mi][pp] = wtf * lam;
    }
    __syncthreads();
    // admissibility of the interpolated states; LLF on the small faces
    // (left/bottom state first); a mortar with an inadmissible interpolated
    // state keeps its low-order flux (its LLF values are not used)
    for (int it = tid; it < nm * NI; it += NT) {
        const int mi = it / NI, r = it - mi * NI;
        const int info = s_info[mi], dir = info & 1, low = (info >> 1) & 1;
        const double *acc = s_ui[mi][r];
        // rho > 0 and rho p > 0, without a division
        if (!dpos(acc[0]) || !dpos(acc[0] * acc[3] - 0.5 * (acc[1] * acc[1] + acc[2] * acc[2]))) {
            atomicOr(&s_bad[mi], 1);
            continue;
        }
        const Prim<FT> pint = mortar_prim<NP, FT>(g, acc);
        FT f[4];
        Prim<FT> ps{};
        ps.v1 = dir == 0 ? s_pr[mi][NP + r][0] : FT(0);
        ps.v2 = dir == 1 ? s_pr[mi][NP + r][0] : FT(0);
        ps.p = s_pr[mi][NP + r][1];
        ps.c = s_pr[mi][NP + r][2];
        const FT *us = s_uf[mi][NP + r];
        FT ui[4];
        for (int v = 0; v < 4; ++v) ui[v] = to_ft<FT>(s_ui[mi][r][v]);
        if constexpr (F32) {
            if (low) llf_prim<FT, FT>(ui, pint, us, ps, dir, f);
            else llf_prim<FT, FT>(us, ps, ui, pint, dir, f);
        } else {
            // operands selected per lane: the warp's mortars of either
            // orientation share one flux evaluation
            FT uL[4], uR[4];
            for (int v = 0; v < 4; ++v) {
                const FT o = us[v];
                uL[v] = low ? ui[v] : o;
                uR[v] = low ? o : ui[v];
            }
            llf_prim<FT, FT>(uL, pick_prim(low != 0, pint, ps), uR, pick_prim(low != 0, ps, pint), dir, f);
        }
        for (int v = 0; v < 4; ++v) s_f[mi][r][v] = f[v];
    }
    __syncthreads();
    // per (slot, variable): high-order contribution (projection summed in
    // FP64, so conservation across the mortar holds to FP64 rounding whatever
    // the flux type) and the low-order sum
    for (int it = tid; it < nm * Q * 4; it += NT) {
        const int mi = it / (Q * 4), rem = it - mi * (Q * 4), q = rem >> 2, v = rem & 3;
        const int m = m0 + mi;
        const double sg = ((s_info[mi] >> 1) & 1) ? 1.0 : -1.0;
        const double halfL = s_halfL[mi], halfS = 0.5 * halfL;
        double chi = 0.0, clo = 0.0;
        const int np_q = ops->slot_n[q];
        for (int t = 0; t < np_q; ++t) clo += s_term[mi][ops->slot_p[q][t]][v];
        if (q < NP) clo = -clo;
        if (!s_bad[mi]) {
            if (q < NP) {
                double acc = 0.0;
                for (int r = 0; r < NI; ++r) {
                    double fr;
                    if constexpr (F32) fr = f2d(s_f[mi][r][v]);
                    else fr = s_f[mi][r][v];
                    acc += ops->P[q][r] * fr;
                }
                chi = -sg * ops->w[q] * (halfL * acc);
            } else {
                const int l = (q - NP) % NP;
                double fr;
                if constexpr (F32) fr = f2d(s_f[mi][q - NP][v]);
                else fr = s_f[mi][q - NP][v];
                chi = sg * ops->w[l] * (halfS * fr);
            }
        } else {
            chi = clo;
        }
        const size_t si = (size_t)v * sl.S + (size_t)m * Q + q;
        sl.chi[si] = chi;
        sl.clo[si] = clo;
    }
    // per slot: bar-state range and 2 d sum over its pairs
    for (int it = tid; it < nm * Q; it += NT) {
        const int mi = it / Q, q = it - mi * Q;
        long long klo = okey(INFINITY), khi = okey(-INFINITY);
        FT ds = FT(0);
        double smin = INFINITY;
        const int np_q = ops->slot_n[q];
        for (int t = 0; t < np_q; ++t) {
            const int p = ops->slot_p[q][t];
            const long long kb = okey(s_rb[mi][p]);
            klo = kb < klo ? kb : klo;
            khi = kb > khi ? kb : khi;
            ds += s_d2[mi][p];
            if (ent) smin = dmin(smin, s_sb[mi][p]);
        }
        const int si = (m0 + mi) * Q + q;
        if (ent) sl.sbmin[si] = smin;
        sl.rbmin[si] = okey_value(klo);
        sl.rbmax[si] = okey_value(khi);
        if constexpr (F32) sl.dsum[si] = f2d(ds);
        else sl.dsum[si] = ds;
    }
    if (tid < nm) sl.bad[m0 + tid] = s_bad[tid] ? 1 : 0;
}

// Largest factor of slot s of mortar m (R9): its node stays inside the
// density interval and above the pressure bound (and, with the entropy bound,
// above it) for the correction scaled by n_i dt / m_i; th2 the same for the
// positivity bounds alone (combined limiting).
template <int NP>
__device__ __forceinline__ void mortar_slot_factor(const MeshDev &mesh, const SlotsDev &sl, const StageArgs &A, int m,
                                                   int s, double &th, double &th2) {
    {
        const int L = mesh.m_large[m];
        const double dt = stage_dt(A, mesh.sim[L]);
        double u0[4], av[4];
        const double f = (double)sl.nmort[s] * dt * fast_rcp(sl.mass[s]);   // n_i dt / m_i
        for (int v = 0; v < 4; ++v) {
            u0[v] = sl.uvol[(size_t)v * sl.S + s];
            av[v] = f * (sl.chi[(size_t)v * sl.S + s] - sl.clo[(size_t)v * sl.S + s]);
        }
        double lr = 1.0;
        const double tl = sl.tol[s];
        if (dpos(av[0])) { double t = (sl.rmax[s] + tl - u0[0]) * fast_rcp(av[0]); if (dlt(t, lr)) lr = t; }
        else if (dneg(av[0])) { double t = (sl.rmin[s] - tl - u0[0]) * fast_rcp(av[0]); if (dlt(t, lr)) lr = t; }
        if (!dpos(lr)) lr = 0.0;
        const double pmin = sl.pmin[s] * fast_rcp(sl.rfv[s]);
        const double pm = pmin - kTol * fabs(pmin);
        th = theta_max(A.gas.gm1, u0, av, A.gas.gm1, pm, g_zero(A.gas.gm1, u0, pm), lr);
        // entropy bound of local limiting (R21)
        if (A.entropy && A.limiting >= 2) th = theta_entropy(A.gas, u0, av, sl.lnK[s], th);
        th2 = 1.0;
        if (A.limiting == 3) {
            // the positivity bounds only: rho >= beta rho_FV, p >= p_min
            const double rfv = sl.rfv[s], rmin2 = dmin(A.beta * rfv, rfv);
            double lr2 = 1.0;
            if (dneg(av[0])) { double t = (rmin2 - tl - u0[0]) * fast_rcp(av[0]); if (dlt(t, lr2)) lr2 = t; }
            if (!dpos(lr2)) lr2 = 0.0;
            th2 = theta_max(A.gas.gm1, u0, av, A.gas.gm1, pm, g_zero(A.gas.gm1, u0, pm), lr2);
        }
    }
}

// Mortar limiting and the limited corrections in one launch. Block b owns
// the mortars [b W, b W + W) and the mortar nodes whose first mortar (in
// mortar order) is one of them; for a corner node whose second mortar lies in
// a later block, that mortar's factor is formed here too (its "foreign"
// mortars, listed per block by the host), so no block waits for another.
// Phase 1: one item per slot of the own and foreign mortars, the factor of a
// mortar the minimum over its slots (shared-memory minimum on the bits of
// the non-negative factors). Phase 2: the owned nodes' corrections in mortar
// order and the stage combination there.
template <int NP>
struct MortarLaunch {
    // own mortars per block: the slots of W mortars and two foreign ones fill
    // about 128 threads; the block has 256, so that the slots of the own and
    // foreign mortars (W + fmax of them) take one pass of the factor loop
    // (measured: 18.8 us per launch on the DMR workload against 21.0 with 128
    // threads, 22.2 with 256 threads and twice the mortars)
    static constexpr int Q = 3 * NP, threads = 256;
    static constexpr int W = (128 - 2 * Q) / Q > 0 ? (128 - 2 * Q) / Q : 1;
};

template <int NP>
__global__ void __launch_bounds__(MortarLaunch<NP>::threads) k_mortar_limit_apply(MeshDev mesh, SlotsDev sl, StageArgs A) {
    constexpr int NN = NP * NP, Q = 3 * NP, NT = MortarLaunch<NP>::threads, W = MortarLaunch<NP>::W;
    extern __shared__ __align__(16) unsigned char mort_smem[];
    const int LW = W + mesh.mb_fmax;                     // local mortars: own, then foreign
    unsigned long long *s_min = reinterpret_cast<unsigned long long *>(mort_smem);
    unsigned long long *s_min2 = s_min + LW;
    double *s_ell = reinterpret_cast<double *>(s_min2 + LW);
    const int b = blockIdx.x, m0 = b * W, tid = threadIdx.x;
    const int nown = min(W, mesh.M - m0);
    const int f0 = mesh.mb_for_off[b], nfor = mesh.mb_for_off[b + 1] - f0;
    const int nloc = nown + nfor;
    const bool combined = A.limiting == 3;
    auto mortar_of = [&](int lm) { return lm < nown ? m0 + lm : mesh.mb_foreign[f0 + lm - nown]; };
    for (int j = tid; j < nloc; j += NT) { s_min[j] = dbits(1.0); s_min2[j] = dbits(1.0); }
    __syncthreads();
    for (int k = tid; k < nloc * Q; k += NT) {
        const int lm = k / Q, q = k - lm * Q, m = mortar_of(lm);
        if (sl.bad[m] != 0) continue;
        double th, th2;
        mortar_slot_factor<NP>(mesh, sl, A, m, m * Q + q, th, th2);
        atomicMin(&s_min[lm], dbits(dpos(th) ? th : 0.0));
        if (combined) atomicMin(&s_min2[lm], dbits(dpos(th2) ? th2 : 0.0));
    }
    __syncthreads();
    for (int j = tid; j < nloc; j += NT) {
        const int mm = mortar_of(j);
        const bool bad = sl.bad[mm] != 0;
        double lS = bad ? 0.0 : __longlong_as_double((long long)s_min[j]);
        if (combined && !bad) {
            // Eq. combination_posLim_local with the largest indicator of the
            // mortar's three elements
            const int2 sm2 = mesh.m_small[mm];
            const double am = fmax(A.aind[mesh.m_large[mm]], fmax(A.aind[sm2.x], A.aind[sm2.y]));
            lS = (1.0 - am) * __longlong_as_double((long long)s_min2[j]) + am * lS;
        }
        s_ell[j] = lS;
        if (j < nown) sl.ell[mm] = lS;
    }
    __syncthreads();
    if (A.collect && tid < 32) {
        // statistics of the own mortars: face length (1 - l_S), active and
        // low-order-only mortars
        float am = 0.0f;
        unsigned nm = 0, nf = 0;
        for (int j = tid; j < nown; j += 32) {
            const int mm = m0 + j;
            const double lS = s_ell[j];
            const int info = mesh.m_info[mm], dir = info & 1;
            const GeoC gc = mesh.geoc[mesh.m_large[mm]];
            am += d2f(2.0 * (dir == 0 ? gc.hy : gc.hx)) * (1.0f - d2f(lS));
            nm += nn_lt(lS, 1.0);
            nf += sl.bad[mm] != 0;
        }
        for (int o = 16; o > 0; o >>= 1) am += __shfl_down_sync(0xffffffffu, am, o);
        nm = __reduce_add_sync(0xffffffffu, nm);
        nf = __reduce_add_sync(0xffffffffu, nf);
        if (tid == 0) {
            if (am > 0.0f) atomicAdd(&A.stats->alpha_mort_len, (double)am);
            if (nm) atomicAdd(&A.stats->n_mort, (unsigned long long)nm);
            if (nf) atomicAdd(&A.stats->n_fallback, (unsigned long long)nf);
        }
    }
    // the factor of the mortar of slot s (own or foreign)
    auto ell_of = [&](int s) {
        const int mm = s / Q;
        if (mm >= m0 && mm < m0 + nown) return s_ell[mm - m0];
        for (int f = 0; f < nfor; ++f)
            if (mesh.mb_foreign[f0 + f] == mm) return s_ell[nown + f];
        return 0.0;   // not reached: the host lists every foreign mortar
    };
    const size_t KN = (size_t)mesh.K * NN;
    double st_rmin = INFINITY;
    float st_pmin = 0.0f, st_one = 0.0f;   // minimum p (FP32 statistic) as the ratio st_pmin / st_one
    unsigned vr = 0, vp = 0, np_ = 0, ve = 0;
    const bool ent = A.entropy && A.limiting == 2;   // entropy bound checked (local limiting)
    const int n0 = mesh.mb_node_off[b], n1 = mesh.mb_node_off[b + 1];
    for (int k = n0 + tid; k < n1; k += NT) {
        const int gnode = mesh.mn_node[k];
        const int2 ss = mesh.mn_slot[k];
        const int s0 = ss.x;
        const int e = gnode / NN;
        const double dt = stage_dt(A, mesh.sim[e]);
        const double imi = fast_rcp(sl.mass[s0]);
        double corr[4] = {0, 0, 0, 0};
        for (int c = 0; c < 2; ++c) {
            int s = c == 0 ? ss.x : ss.y;
            if (s < 0) continue;
            double l = ell_of(s);
            for (int v = 0; v < 4; ++v) corr[v] += l * (sl.chi[(size_t)v * sl.S + s] - sl.clo[(size_t)v * sl.S + s]);
        }
        double ut[4];
        const double dtm = dt * imi;
        for (int v = 0; v < 4; ++v) {
            double uv = sl.uvol[(size_t)v * sl.S + s0];
            ut[v] = uv + dtm * corr[v];
            if (A.mode == 0) {
                A.out[v * KN + gnode] = (sl.un[(size_t)v * sl.S + s0] + corr[v]) * imi;
            } else {
                double o = ut[v];
                double un = sl.un[(size_t)v * sl.S + s0];
                if (A.comb == 1) o = 0.75 * un + 0.25 * ut[v];
                else if (A.comb == 2) o = un * (1.0 / 3.0) + 2.0 / 3.0 * ut[v];
                A.out[v * KN + gnode] = o;
            }
        }
        if (A.collect) {
            // rho p = (gamma-1)(rho E - |m|^2/2) against p_min rho, without division
            const double rp = A.gas.gm1 * (ut[0] * ut[3] - 0.5 * (ut[1] * ut[1] + ut[2] * ut[2]));
            const double pmin = sl.pmin[s0] * fast_rcp(sl.rfv[s0]);
            const double rmin = A.limiting == 3 ? dmin(A.beta * sl.rfv[s0], sl.rfv[s0]) : sl.rmin[s0];
            const double rmax = A.limiting == 3 ? INFINITY : sl.rmax[s0];
            if (dlt(ut[0], rmin - kViolTol * fabs(rmin)) || dlt(rmax + kViolTol * fabs(rmax), ut[0])) vr++;
            if (dlt(rp, (pmin - kViolTol * fabs(pmin)) * ut[0])) vp++;
            if (!dpos(ut[0]) || !dpos(rp)) np_++;
            if (ent && dlt(entropy_s(A.gas, ut[0], ut[1], ut[2], ut[3]), sl.lnK[s0] + A.gas.eviol)) ve++;
            st_rmin = dmin(st_rmin, ut[0]);
            const float pf = dpos(ut[0]) ? d2f(rp) / d2f(ut[0]) : 0.0f;
            if (pf > 0.0f && (st_one == 0.0f || pf < st_pmin)) { st_pmin = pf; st_one = 1.0f; }
        }
    }
    if (A.collect) block_stats(A, 0.0f, 0u, vr, vp, np_, st_rmin, st_pmin, st_one, ve);
    if ((vr | vp | np_ | ve) != 0u) atomicOr(A.status, ST_VIOLATION);
}

// shared memory of k_mortar_limit_apply for at most fmax foreign mortars per block
template <int NP>
constexpr size_t mortar_smem(int fmax) {
    return (size_t)(MortarLaunch<NP>::W + fmax) * (2 * sizeof(unsigned long long) + sizeof(double));
}

// Low-order-solution bounds across mortars (Eq. Bounds_LowOrder): per slot,
// the range of rho_FV and the minimum of s(u_FV) over the nodes on the other
// side of the mortar that share a nonzero local weight with it. One thread
// per slot; lofv is the element pre-pass output [2][K (N+1)^2].
template <int NP>
__global__ void __launch_bounds__(128) k_mortar_lob(MeshDev mesh, SlotsDev sl, const Ops *ops,
                                                    const double *__restrict__ lofv, int ent) {
    constexpr int NN = NP * NP, Q = 3 * NP;
    const size_t KN = (size_t)mesh.K * NN;
    for (int si = blockIdx.x * blockDim.x + threadIdx.x; si < sl.S; si += gridDim.x * blockDim.x) {
        const int m = si / Q, q = si - m * Q;
        const int info = mesh.m_info[m], dir = info & 1, low = (info >> 1) & 1;
        const int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2), sS = sL ^ 1;
        const int L = mesh.m_large[m];
        const int2 sm2 = mesh.m_small[m];
        long long klo = okey(INFINITY), khi = okey(-INFINITY);
        double smin = INFINITY;
        const int np_q = ops->slot_n[q];
        for (int t = 0; t < np_q; ++t) {
            const int p = ops->slot_p[q][t];
            // the pair's node on the other side: a small-face node for a
            // large slot, the large node for a small slot
            size_t g;
            if (q < NP) {
                const int r = ops->pr[p];
                g = (size_t)(r < NP ? sm2.x : sm2.y) * NN + face_node<NP>(sS, r % NP);
            } else {
                g = (size_t)L * NN + face_node<NP>(sL, ops->pk[p]);
            }
            const long long kb = okey(lofv[g]);
            klo = kb < klo ? kb : klo;
            khi = kb > khi ? kb : khi;
            if (ent) smin = dmin(smin, lofv[KN + g]);
        }
        sl.lbmin[si] = okey_value(klo);
        sl.lbmax[si] = okey_value(khi);
        if (ent) sl.lsmin[si] = smin;
    }
}

// Time step: per node m_i / sum_j 2 d_ij (rule 0) or min over directions of
// (w_i h / 2) / (|v| + c) (rule 1); minimum per simulation as ordered bits.
// One block holds EPB elements, one thread per node. Three uniform passes:
// each node's wave speeds |v_x| + c and |v_y| + c; per face node the outside
// wave speed along the face normal (conforming neighbour or ghost state) or
// the mortar's 2d sum; then the per-node sums. In the FP32 form (FT = float)
// the wave speeds, sums and the quotient are FP32 and the result is scaled by
// (1 - 4e-6), more than the FP32 rounding of these few operations, so the
// step never exceeds the FP64 limit.
// Wave speeds |v_x| + c and |v_y| + c of every node, lam[2][K (N+1)^2], for
// k_dt: one thread per node, so that the time step reads a conforming
// neighbour's speed (one value) instead of its state (four) and does not form
// the neighbour's primitives again.
template <int NP, typename FT>
__global__ void __launch_bounds__(256) k_dt_speed(MeshDev mesh, const double *__restrict__ u, Gas gas,
                                                  unsigned *status, FT *__restrict__ lam) {
    const size_t KN = (size_t)mesh.K * NP * NP;
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < KN; gi += (size_t)gridDim.x * blockDim.x) {
        double qd[4] = {u[gi], u[KN + gi], u[2 * KN + gi], u[3 * KN + gi]};
        Prim<FT> q = mortar_prim<NP, FT>(gas, qd);
        bool okp;
        if constexpr (sizeof(FT) == 4) okp = q.p > 0.0f;
        else okp = dpos(q.p);
        if (!dpos(qd[0]) || !okp) atomicOr(status, ST_BAD_INPUT);
        lam[gi] = fabs(q.v1) + q.c;
        lam[KN + gi] = fabs(q.v2) + q.c;
    }
}

// The FP64 path's time step in two passes. The first (FT = float, mode 1)
// forms every node's quotient in FP32 from the FP32 primitives and the face
// buffer's wave speeds and writes each element's minimum (emin) and, into
// its own dtmin array, each simulation's minimum; its quotients are within
// a relative 1e-5 of the FP64 ones (the FP32 form's scaling margin is 4e-6).
// The second (FT = double, mode 2) forms the FP64 quotients only in the
// elements whose FP32 minimum is within a relative 1e-4 of their
// simulation's, which hold the FP64 minimiser, so its minimum is the one-pass
// FP64 minimum bit for bit.
struct DtFilter {
    int mode;                          // 0: one pass; 1: FP32 pass; 2: FP64 pass over the candidates
    unsigned *emin;                    // per element: the FP32 pass's minimum (bits of a positive float)
    const unsigned long long *smin;    // mode 2: per simulation, the FP32 pass's minimum (bits of a double)
};
constexpr double kDtFilterMargin = 1e-4;

template <int NP, int EPB, typename FT>
__global__ void __launch_bounds__(ElemLaunch<NP, EPB>::threads)
k_dt(MeshDev mesh, SlotsDev sl, const double *__restrict__ u, Gas gas, int rule, const Ops *ops,
     const double *t_sim, unsigned long long *dtmin, unsigned *status, const double *__restrict__ fbuf,
     const FT *__restrict__ lam, DtFilter flt) {
    constexpr int NN = NP * NP, N = NP - 1, NT = ElemLaunch<NP, EPB>::threads;
    constexpr bool F32 = sizeof(FT) == 4;
    __shared__ FT s_l[EPB][2][NN];       // |v_x| + c, |v_y| + c per node
    __shared__ FT s_o[EPB][4][NP];       // outside wave speed, or 2d sum of a mortar side
    __shared__ double s_w[NP];
    __shared__ int s_wsim[NT / 32];                 // per warp: its lane 0's simulation
    __shared__ unsigned long long s_wbest[NT / 32];  // and that simulation's minimum
    __shared__ unsigned s_emin[EPB];                 // mode 1: per element minimum (float bits)
    __shared__ unsigned char s_cand[EPB];            // mode 2: the element is a candidate
    if (threadIdx.x < NP) s_w[threadIdx.x] = ops->w[threadIdx.x];
    const size_t KN = (size_t)mesh.K * NN;
    const Gas &g = gas;
    for (int e0 = blockIdx.x * EPB; e0 < mesh.K; e0 += gridDim.x * EPB) {
        if (flt.mode != 0) {
            // (EPB * NN <= NT: one node per thread)
            const int le = threadIdx.x / NN, e = e0 + le;
            bool cd = false;
            if (le < EPB && threadIdx.x % NN == 0) {
                if (flt.mode == 1) s_emin[le] = 0x7f800000u;   // +inf
                if (e < mesh.K && flt.mode == 2) {
                    const double smin = __longlong_as_double((long long)flt.smin[mesh.sim[e]]);
                    cd = (double)__uint_as_float(flt.emin[e]) <= smin * (1.0 + kDtFilterMargin);
                }
                s_cand[le] = cd;
            }
            // mode 2: a block without candidates has nothing to do (uniform)
            if (!__syncthreads_or(cd) && flt.mode == 2) continue;
        }
        for (int k = threadIdx.x; k < EPB * NN; k += NT) {
            int le = k / NN, n = k - le * NN, e = e0 + le;
            if (e >= mesh.K) continue;
            if (flt.mode == 2 && !s_cand[le]) continue;
            size_t gi = (size_t)e * NN + n;
            if (lam) {
                // from k_dt_speed
                s_l[le][0][n] = lam[gi];
                s_l[le][1][n] = lam[KN + gi];
                continue;
            }
            double qd[4] = {u[gi], u[KN + gi], u[2 * KN + gi], u[3 * KN + gi]};
            Prim<FT> q = mortar_prim<NP, FT>(g, qd);
            bool okp;
            if constexpr (F32) okp = q.p > 0.0f;
            else okp = dpos(q.p);
            if (!dpos(qd[0]) || !okp) atomicOr(status, ST_BAD_INPUT);
            s_l[le][0][n] = fabs(q.v1) + q.c;
            s_l[le][1][n] = fabs(q.v2) + q.c;
        }
        if (rule == 0) {
            for (int k = threadIdx.x; k < EPB * 4 * NP; k += NT) {
                int le = k / (4 * NP), s = (k / NP) % 4, t = k % NP, e = e0 + le;
                if (e >= mesh.K) continue;
                if (flt.mode == 2 && !s_cand[le]) continue;
                const uchar4 ftv = mesh.ftype[e];
                const int4 nb4 = mesh.fnbr[e];
                const int ft = s == 0 ? ftv.x : (s == 1 ? ftv.y : (s == 2 ? ftv.z : ftv.w));
                const int nb = s == 0 ? nb4.x : (s == 1 ? nb4.y : (s == 2 ? nb4.z : nb4.w));
                if (ft == FT_CONF && fbuf != nullptr) {
                    // FP64 path: the face's lambda = max of both wave speeds
                    // from k_face on the same state (the entry of the element
                    // on the face's left/bottom); max(own, lambda) = lambda
                    const int owner = (s & 1) ? e : nb;
                    const long long F = 2ll * mesh.K * NP, q = (2ll * owner + (s >> 1)) * NP + t;
                    s_o[le][s][t] = to_ft<FT>(fbuf[5 * F + q]);
                } else if (ft == FT_CONF && lam) {
                    // the neighbour's wave speed along the face normal
                    const size_t ko = (size_t)nb * NN + face_node<NP>(s ^ 1, t);
                    s_o[le][s][t] = lam[(size_t)(s >> 1) * KN + ko];
                } else if (ft == FT_CONF || ft == FT_BND) {
                    double uo[4];
                    if (ft == FT_CONF) {
                        size_t ko = (size_t)nb * NN + face_node<NP>(s ^ 1, t);
                        for (int v = 0; v < 4; ++v) uo[v] = u[v * KN + ko];
                    } else {
                        const int n = face_node<NP>(s, t), i = n % NP, sim = mesh.sim[e];
                        const Geo geo = mesh.geom[e];
                        size_t gi = (size_t)e * NN + n;
                        double ui[4] = {u[gi], u[KN + gi], u[2 * KN + gi], u[3 * KN + gi]};
                        double xn = geo.x + 0.5 * geo.z * (1.0 + ops->xi[i]);
                        double yn = geo.y + 0.5 * geo.w * (1.0 + ops->xi[n / NP]);
                        ghost_state(mesh.siminfo[sim], s, ui, xn, yn, t_sim[sim], uo);
                    }
                    Prim<FT> po = mortar_prim<NP, FT>(g, uo);
                    s_o[le][s][t] = fabs((s >> 1) == 0 ? po.v1 : po.v2) + po.c;
                } else {
                    s_o[le][s][t] = to_ft<FT>(sl.dsum[slot_of<NP>(ft, nb, t)]);
                }
            }
        }
        __syncthreads();
        unsigned long long best = dbits(INFINITY);
        int bsim = -1;
        for (int k = threadIdx.x; k < EPB * NN; k += NT) {
            int le = k / NN, n = k - le * NN, e = e0 + le;
            if (e >= mesh.K) continue;
            if (flt.mode == 2 && !s_cand[le]) continue;
            const int i = n % NP, j = n / NP;
            const GeoC gc = mesh.geoc[e];
            const int sim = mesh.sim[e];
            double val;
            if (rule == 1) {
                if constexpr (F32)
                    val = f2d(fminf(d2f(s_w[i] * gc.hx) / s_l[le][0][n], d2f(s_w[j] * gc.hy) / s_l[le][1][n]) *
                              (1.0f - 4e-6f));
                else
                    val = fmin(s_w[i] * gc.hx * fast_rcp(s_l[le][0][n]), s_w[j] * gc.hy * fast_rcp(s_l[le][1][n]));
            } else {
                const uchar4 ftv = mesh.ftype[e];
                FT ds = FT(0);
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const int pos = d == 0 ? i : j, row = d == 0 ? j : i;
                    FT cc2;   // 2 c_ij = w_row |face| / 2
                    if constexpr (F32) cc2 = d2f(s_w[row]) * (d == 0 ? gc.hyf : gc.hxf);
                    else cc2 = s_w[row] * (d == 0 ? gc.hy : gc.hx);
                    const FT li = s_l[le][d][n];
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const bool interior = side == 0 ? pos > 0 : pos < N;
                        const int s = 2 * d + side;
                        const int ft = s == 0 ? ftv.x : (s == 1 ? ftv.y : (s == 2 ? ftv.z : ftv.w));
                        const int on = d == 0 ? n + (side == 0 ? -1 : 1) : n + (side == 0 ? -NP : NP);
                        const FT lo = interior ? s_l[le][d][interior ? on : n] : s_o[le][s][row];
                        const bool mort = !interior && ft != FT_CONF && ft != FT_BND;
                        ds += mort ? lo : cc2 * (li > lo ? li : lo);
                    }
                }
                if constexpr (F32) val = f2d(gc.A4f * d2f(s_w[i] * s_w[j]) / ds * (1.0f - 4e-6f));
                else val = gc.A4 * (s_w[i] * s_w[j]) * fast_rcp(ds);
            }
            // positive doubles order like their bits
            const unsigned long long vb = dbits(val);
            if (sim != bsim) {
                if (bsim >= 0 && best < dbits(INFINITY)) atomicMin(&dtmin[bsim], best);
                bsim = sim;
                best = dbits(INFINITY);
            }
            if (dpos(val) && vb < best) best = vb;
            if (flt.mode == 1 && dpos(val)) atomicMin(&s_emin[le], __float_as_uint((float)val));
        }
        // warp minimum among the lanes that share lane 0's simulation (other
        // simulations: one atomic per lane), then the block's warps of the
        // same simulation merged in shared memory, one atomic per block and
        // simulation (same-address atomics serialise in L2)
        {
            const int s0 = __shfl_sync(0xffffffffu, bsim, 0);
            const bool same = bsim == s0;
            unsigned long long bw = same ? best : dbits(INFINITY);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_down_sync(0xffffffffu, bw, o);
                bw = ob < bw ? ob : bw;
            }
            if ((threadIdx.x & 31) == 0) { s_wsim[threadIdx.x >> 5] = s0; s_wbest[threadIdx.x >> 5] = bw; }
            if (!same && bsim >= 0 && best < dbits(INFINITY)) atomicMin(&dtmin[bsim], best);
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 0; w < NT / 32; ++w) {
                    const int sw = s_wsim[w];
                    if (sw < 0) continue;
                    unsigned long long bm = s_wbest[w];
                    for (int w2 = w + 1; w2 < NT / 32; ++w2)
                        if (s_wsim[w2] == sw) { bm = s_wbest[w2] < bm ? s_wbest[w2] : bm; s_wsim[w2] = -1; }
                    if (bm < dbits(INFINITY)) atomicMin(&dtmin[sw], bm);
                }
            }
            if (flt.mode == 1 && threadIdx.x < EPB && e0 + (int)threadIdx.x < mesh.K)
                flt.emin[e0 + threadIdx.x] = s_emin[threadIdx.x];
        }
        __syncthreads();
    }
}

// dtmin holds 2 n entries: the time-step minimum per simulation, then the
// FP32 pass's minimum of the two-pass time step
static __global__ void k_dt_init(unsigned long long *dtmin, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 2 * n) dtmin[k] = dbits(INFINITY);
}

// The step's end: t += dt per simulation, and both time-step minima reset to
// +inf for the next step (which then needs no reset launch of its own).
static __global__ void k_time_advance(double *t_sim, unsigned long long *dtmin, double cfl, double *dt_last, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        double dt = cfl * __longlong_as_double((long long)dtmin[k]);
        t_sim[k] += dt;
        dt_last[k] = dt;
        dtmin[k] = dbits(INFINITY);
        dtmin[n + k] = dbits(INFINITY);
    }
}

// sum_i m_i u_i per element (fixed order over its nodes)
template <int NP>
__global__ void k_elem_integrals(MeshDev mesh, const double *__restrict__ u, const Ops *ops, double *part) {
    constexpr int NN = NP * NP;
    const size_t KN = (size_t)mesh.K * NN;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < mesh.K; e += gridDim.x * blockDim.x) {
        Geo geo = mesh.geom[e];
        double J = geo.z * geo.w / 4.0;
        for (int v = 0; v < 4; ++v) {
            double s = 0.0;
            for (int n = 0; n < NN; ++n) s += J * ops->w[n % NP] * ops->w[n / NP] * u[v * KN + (size_t)e * NN + n];
            part[(size_t)v * mesh.K + e] = s;
        }
    }
}

// per simulation: fixed-order tree sum of the element partials in [off[s], off[s+1])
static __global__ void k_sum_segments(const double *part, int K, const long long *off, double *out) {
    __shared__ double red[4][256];
    const int s = blockIdx.x;
    const long long b = off[s], e = off[s + 1];
    double acc[4] = {0, 0, 0, 0};
    for (long long k = b + threadIdx.x; k < e; k += blockDim.x)
        for (int v = 0; v < 4; ++v) acc[v] += part[(size_t)v * K + k];
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

}  // namespace idp
