// idp3d_mortar.cuh -- the nonconforming faces of the 3D IDP LGL-DGSEM
// (arXiv 2607.06045, Sec. 2.2 and 2.3 with d = 3) on 2:1 octrees: one face
// between a leaf and four finer ones is a mortar with 2 x 2 small faces.
//
//  k_mflux3    per mortar, from the stage input: the high-order L2 mortar flux
//              as the tensor product of the 1D interpolation and exact L2
//              projection (interpolate the large face to the four small
//              faces' nodes, LLF there, project back), the sparse low-order
//              mortar flux of Eq. interfaceflux_local with the local weights
//              taken as products of the 1D overlap weights, the pairs' bar-state
//              densities and 2 d_ij sums; a mortar whose interpolated states
//              leave the admissible set keeps its low-order flux (R16).
//  k_mfactor3  one factor l_S per mortar after the volume correction: the
//              largest factor that keeps every node of the mortar inside its
//              density interval and above its pressure bound for the
//              correction scaled by n_i dt / m_i (R9 with the n_i budget).
//  k_mapply3   per mortar node: u_vol plus the limited corrections of its
//              mortars (in mortar order), the stage combination, statistics.
#pragma once

#include "idp3d.cuh"

namespace idp3 {

// 1D mortar operators (degree N, reference units): interpolation to the two
// half-faces' nodes, exact L2 projection back, the local overlap weights of
// App. A as a pair list (large node k, half-face node r = e (N+1) + l) with,
// per 1D slot (large nodes, then the half-faces' nodes), its pairs in order
struct MOps3 {
    double w[NPMAX3];
    double I[2 * NPMAX3][NPMAX3];
    double P[NPMAX3][2 * NPMAX3];
    double wt[NPMAX3][2 * NPMAX3];
    int n1;
    int pk[4 * NPMAX3], pr[4 * NPMAX3];
    int sn[3 * NPMAX3];
    int sp[3 * NPMAX3][2 * NPMAX3];
};

// mortar kernels: one mortar per block
constexpr int kMortThreads3 = 128;

template <int NP>
struct MortSize3 {
    static constexpr int NR = NP * NP, Q = 5 * NR, NI = 4 * NR;
    static constexpr int P1 = 3 * NP - 1;   // at most 3 N + 2 nonzero 1D overlaps
    static constexpr int PP = P1 * P1;
};

// per-mortar geometry: quarter area of the large face and its sign
__device__ __forceinline__ double mort_qarea(const Grid3 &G, int L, int d) {
    double h[3];
    extents3(G, L, h);
    return h[(d + 1) % 3] * h[(d + 2) % 3] / 4.0;
}

template <int NP>
__global__ void __launch_bounds__(kMortThreads3) k_mflux3(Grid3 G, const MOps3 *__restrict__ mo, const double *__restrict__ u,
                                                          double gamma) {
    using MS = MortSize3<NP>;
    constexpr int N = NP - 1, NR = MS::NR, Q = MS::Q, NI = MS::NI, PP = MS::PP, NT = kMortThreads3;
    constexpr int NN = NP * NP * NP;
    __shared__ double s_u[Q][NV];       // traces: large face, then the four small faces
    __shared__ double s_pr[Q][3];       // normal velocity, pressure, wave speed |v_d| + c
    __shared__ double s_ui[NI][NV];     // the large trace interpolated to the small faces' nodes
    __shared__ double s_f[NI][NV];      // LLF fluxes on the small faces (along +d)
    __shared__ double s_term[PP][NV];   // low-order pair terms
    __shared__ double s_rb[PP], s_d2[PP];
    __shared__ int s_bad;
    const Mort3 &MO = G.mort;
    const int m = blockIdx.x, tid = threadIdx.x;
    const int *inf = MO.info + 7 * m;
    const int d = inf[0], L = inf[1], low = inf[2];
    const int sL = 2 * d + low;
    const double sg = low ? 1.0 : -1.0;   // the large side's outward normal along +d
    const double qaL = mort_qarea(G, L, d), qaS = qaL / 4.0;
    const size_t KN = (size_t)G.K * NN;
    const double gm1 = gamma - 1.0;
    const int n1 = mo->n1;
    if (tid == 0) s_bad = 0;
    // traces and their primitives
    for (int q = tid; q < Q; q += NT) {
        const int f = q / NR, t = q - f * NR;
        const int e = f == 0 ? L : inf[3 + f - 1];
        const int pos = (f == 0) == (low != 0) ? N : 0;   // the large face is its +d side when low
        const int n = node_of<NP>(d, t, pos);
        double o[NV];
        for (int v = 0; v < NV; ++v) { o[v] = u[v * KN + (size_t)e * NN + n]; s_u[q][v] = o[v]; }
        const double ir = idp::fast_rcp(o[0]);
        const double vd = o[1 + d] * ir;
        const double p = gm1 * (o[4] - 0.5 * (o[1] * o[1] + o[2] * o[2] + o[3] * o[3]) * ir);
        s_pr[q][0] = vd;
        s_pr[q][1] = p;
        s_pr[q][2] = (o[0] > 0.0 && p > 0.0) ? fabs(vd) + idp::fast_sqrt(gamma * p * ir) : 0.0;
    }
    __syncthreads();
    // interpolation to the small faces' nodes (tensor product of the 1D one)
    for (int it = tid; it < NI * NV; it += NT) {
        const int r = it / NV, v = it - r * NV;
        const int p = r / NR, t = r - p * NR, l1 = t % NP, l2 = t / NP;
        const double *I1 = mo->I[(p & 1) * NP + l1], *I2 = mo->I[(p >> 1) * NP + l2];
        double acc = 0.0;
        for (int k2 = 0; k2 < NP; ++k2) {
            double a2 = 0.0;
            for (int k1 = 0; k1 < NP; ++k1) a2 += I1[k1] * s_u[k1 + NP * k2][v];
            acc += I2[k2] * a2;
        }
        s_ui[r][v] = acc;
    }
    // low-order pair terms (Eq. interfaceflux_local): term enters the large
    // node's slot with -, the small one's with +; bar-state density and 2 d
    for (int pp = tid; pp < n1 * n1; pp += NT) {
        const int t1 = pp / n1, t2 = pp - t1 * n1;
        const int k1 = mo->pk[t1], r1 = mo->pr[t1], k2 = mo->pk[t2], r2 = mo->pr[t2];
        const int qa = k1 + NP * k2;
        const int qs = NR + ((r1 / NP) + 2 * (r2 / NP)) * NR + (r1 % NP) + NP * (r2 % NP);
        const double wgt = mo->wt[k1][r1] * mo->wt[k2][r2] * qaL;
        const double *a = s_u[qa], *b = s_u[qs];
        const double lam = fmax(s_pr[qa][2], s_pr[qs][2]);
        double fa[NV], fb[NV];
        flux_p(a, s_pr[qa][0], s_pr[qa][1], d, fa);
        flux_p(b, s_pr[qs][0], s_pr[qs][1], d, fb);
        for (int v = 0; v < NV; ++v) s_term[pp][v] = 0.5 * (wgt * sg * (fa[v] + fb[v]) - wgt * lam * (b[v] - a[v]));
        s_rb[pp] = 0.5 * (a[0] + b[0]) - sg * (b[1 + d] - a[1 + d]) * (0.5 * idp::fast_rcp(lam));
        s_d2[pp] = wgt * lam;
    }
    __syncthreads();
    // admissibility of the interpolated states; LLF on the small faces
    // (the lower state along +d first)
    for (int r = tid; r < NI; r += NT) {
        const double *x = s_ui[r];
        if (!(x[0] > 0.0) || !(x[0] * x[4] - 0.5 * (x[1] * x[1] + x[2] * x[2] + x[3] * x[3]) > 0.0)) {
            atomicOr(&s_bad, 1);
            continue;
        }
        const double ir = idp::fast_rcp(x[0]);
        const double vi = x[1 + d] * ir;
        const double pi = gm1 * (x[4] - 0.5 * (x[1] * x[1] + x[2] * x[2] + x[3] * x[3]) * ir);
        const double li = fabs(vi) + idp::fast_sqrt(gamma * pi * ir);
        const int qs = NR + r;
        const double *us = s_u[qs];
        double fi[NV], fs[NV];
        flux_p(x, vi, pi, d, fi);
        flux_p(us, s_pr[qs][0], s_pr[qs][1], d, fs);
        const double lam = fmax(li, s_pr[qs][2]);
        const double *uL = low ? x : us, *uR = low ? us : x, *fL = low ? fi : fs, *fR = low ? fs : fi;
        for (int v = 0; v < NV; ++v) s_f[r][v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
    }
    __syncthreads();
    const int bad = s_bad;
    // per (slot, variable): the low-order sum over the slot's pairs in a fixed
    // order and the high-order contribution (projection for the large face)
    for (int it = tid; it < Q * NV; it += NT) {
        const int q = it / NV, v = it - q * NV;
        int a1, a2;   // the slot's 1D slots along the two tangential directions
        if (q < NR) { a1 = q % NP; a2 = q / NP; }
        else {
            const int p = (q - NR) / NR, t = (q - NR) - p * NR;
            a1 = NP + (p & 1) * NP + t % NP;
            a2 = NP + (p >> 1) * NP + t / NP;
        }
        double clo = 0.0;
        for (int i1 = 0; i1 < mo->sn[a1]; ++i1)
            for (int i2 = 0; i2 < mo->sn[a2]; ++i2) clo += s_term[mo->sp[a1][i1] * n1 + mo->sp[a2][i2]][v];
        if (q < NR) clo = -clo;
        double chi;
        if (bad) {
            chi = clo;
        } else if (q < NR) {
            const int k1 = q % NP, k2 = q / NP;
            double acc = 0.0;
            for (int p = 0; p < 4; ++p) {
                const double *P1 = mo->P[k1] + (p & 1) * NP, *P2 = mo->P[k2] + (p >> 1) * NP;
                for (int l2 = 0; l2 < NP; ++l2) {
                    double a = 0.0;
                    for (int l1 = 0; l1 < NP; ++l1) a += P1[l1] * s_f[p * NR + l1 + NP * l2][v];
                    acc += P2[l2] * a;
                }
            }
            chi = -sg * (mo->w[k1] * mo->w[k2]) * (qaL * acc);
        } else {
            const int t = (q - NR) % NR;
            chi = sg * (mo->w[t % NP] * mo->w[t / NP]) * (qaS * s_f[q - NR][v]);
        }
        const size_t si = (size_t)v * MO.S + (size_t)m * Q + q;
        MO.chi[si] = chi;
        MO.clo[si] = clo;
    }
    // per slot: bar-state density range and sum of 2 d_ij
    for (int q = tid; q < Q; q += NT) {
        int a1, a2;
        if (q < NR) { a1 = q % NP; a2 = q / NP; }
        else {
            const int p = (q - NR) / NR, t = (q - NR) - p * NR;
            a1 = NP + (p & 1) * NP + t % NP;
            a2 = NP + (p >> 1) * NP + t / NP;
        }
        double lo = INFINITY, hi = -INFINITY, ds = 0.0;
        for (int i1 = 0; i1 < mo->sn[a1]; ++i1)
            for (int i2 = 0; i2 < mo->sn[a2]; ++i2) {
                const int pp = mo->sp[a1][i1] * n1 + mo->sp[a2][i2];
                lo = idp::dmin(lo, s_rb[pp]);
                hi = idp::dmax(hi, s_rb[pp]);
                ds += s_d2[pp];
            }
        const size_t si = (size_t)m * Q + q;
        MO.rbmin[si] = lo;
        MO.rbmax[si] = hi;
        MO.dsum[si] = ds;
    }
    if (tid == 0) MO.bad[m] = bad;
}

// one factor per mortar (R9): the minimum over its slots of the largest
// factor that keeps the slot's node admissible for u_vol + l n_i dt / m_i H
template <int NP>
__global__ void __launch_bounds__(kMortThreads3) k_mfactor3(Grid3 G, Stage3 A) {
    using MS = MortSize3<NP>;
    constexpr int Q = MS::Q, NT = kMortThreads3;
    __shared__ unsigned long long s_min, s_min2;
    const Mort3 &MO = G.mort;
    const int m = blockIdx.x, tid = threadIdx.x;
    const double g = A.gamma, dt = stage_dt3(A);
    const bool bad = MO.bad[m] != 0, comb = A.limiting == 3;
    if (tid == 0) s_min = s_min2 = (unsigned long long)__double_as_longlong(1.0);
    __syncthreads();
    if (A.limiting > 0 && !bad) {
        unsigned long long best = (unsigned long long)__double_as_longlong(1.0), best2 = best;
        for (int q = tid; q < Q; q += NT) {
            const int s = m * Q + q, mn = MO.slot_mn[s];
            const size_t MN = MO.MN;
            const double f = (double)MO.mn_cnt[mn] * dt * MO.h_b[4 * MN + mn];   // n_i dt / m_i
            double u0[NV], av[NV];
            for (int v = 0; v < NV; ++v) {
                u0[v] = MO.h_uvol[v * MN + mn];
                av[v] = f * (MO.chi[(size_t)v * MO.S + s] - MO.clo[(size_t)v * MO.S + s]);
            }
            const double tolr = kTol3 * fabs(MO.h_b[3 * MN + mn]);
            // R15 per slot: a density change below 1e-14 |rho_FV| is exempt from the density bounds
            const bool exs = fabs(av[0]) <= tolr;
            double lr = 1.0;
            if (!exs && av[0] > 0.0) { const double t = (MO.h_b[1 * MN + mn] + tolr - u0[0]) / av[0]; if (t < lr) lr = t; }
            else if (!exs && av[0] < 0.0) { const double t = (MO.h_b[0 * MN + mn] - tolr - u0[0]) / av[0]; if (t < lr) lr = t; }
            if (!(lr > 0.0)) lr = 0.0;
            const double pm = MO.h_b[2 * MN + mn];
            double th = theta3(g, u0, av, pm - kTol3 * fabs(pm), lr);
            if (!(th > 0.0)) th = 0.0;
            const unsigned long long tb = (unsigned long long)__double_as_longlong(th);
            best = tb < best ? tb : best;
            if (comb) {
                // the positivity bounds alone: rho >= min(beta rho_FV, rho_FV), p >= p_min
                const double rf = MO.h_b[3 * MN + mn], rmin2 = idp::dmin(A.beta * rf, rf);
                double lr2 = 1.0;
                if (!exs && av[0] < 0.0) { const double t = (rmin2 - tolr - u0[0]) / av[0]; if (t < lr2) lr2 = t; }
                if (!(lr2 > 0.0)) lr2 = 0.0;
                double th2 = theta3(g, u0, av, pm - kTol3 * fabs(pm), lr2);
                if (!(th2 > 0.0)) th2 = 0.0;
                const unsigned long long tb2 = (unsigned long long)__double_as_longlong(th2);
                best2 = tb2 < best2 ? tb2 : best2;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
            best = ob < best ? ob : best;
            const unsigned long long ob2 = __shfl_down_sync(0xffffffffu, best2, o);
            best2 = ob2 < best2 ? ob2 : best2;
        }
        if ((tid & 31) == 0) { atomicMin(&s_min, best); atomicMin(&s_min2, best2); }
    }
    __syncthreads();
    if (tid == 0) {
        double lS = bad ? 0.0 : (A.limiting > 0 ? __longlong_as_double((long long)s_min) : 1.0);
        if (comb && !bad) {
            // Eq. combination_posLim_local with the largest indicator of the mortar's five elements
            const int *inf = MO.info + 7 * m;
            double am = A.aind[inf[1]];
            for (int p = 0; p < 4; ++p) am = fmax(am, A.aind[inf[3 + p]]);
            lS = (1.0 - am) * __longlong_as_double((long long)s_min2) + am * lS;
        }
        MO.ell[m] = lS;
        if (A.collect && A.limiting > 0) {
            const int *inf = MO.info + 7 * m;
            const double area = 4.0 * mort_qarea(G, inf[1], inf[0]);
            atomicAdd(&A.stats->alpha_mort_a, area * (1.0 - lS));
            atomicAdd(&A.stats->mort_area, area);
            if (lS < 1.0) atomicAdd(&A.stats->n_mort, 1ull);
            if (bad) atomicAdd(&A.stats->n_mort_fallback, 1ull);
        }
    }
}

// the mortar nodes: u_vol plus the limited corrections of their mortars in
// mortar order, then the residual or the stage combination, and statistics
template <int NP>
__global__ void __launch_bounds__(256) k_mapply3(Grid3 G, Stage3 A) {
    constexpr int Q = MortSize3<NP>::Q, NN = NP * NP * NP;
    const Mort3 &MO = G.mort;
    const size_t KN = (size_t)G.K * NN, MN = MO.MN;
    const double g = A.gamma, dt = stage_dt3(A);
    unsigned vr = 0, vp = 0, np_ = 0;
    double rmin_st = INFINITY, pmin_st = INFINITY;
    for (int mn = blockIdx.x * blockDim.x + threadIdx.x; mn < MO.MN; mn += gridDim.x * blockDim.x) {
        const int gi = MO.mn_node[mn], cnt = MO.mn_cnt[mn];
        double corr[NV] = {0, 0, 0, 0, 0};
        for (int c = 0; c < cnt; ++c) {
            const int s = MO.mn_slot[(size_t)c * MN + mn];
            const double l = MO.ell[s / Q];
            for (int v = 0; v < NV; ++v) corr[v] += l * (MO.chi[(size_t)v * MO.S + s] - MO.clo[(size_t)v * MO.S + s]);
        }
        const double im = MO.h_b[4 * MN + mn];
        double ut[NV];
        for (int v = 0; v < NV; ++v) {
            ut[v] = MO.h_uvol[v * MN + mn] + dt * im * corr[v];
            double o;
            if (A.mode == 0) o = (MO.h_res[v * MN + mn] + corr[v]) * im;
            else if (A.comb == 1) o = 0.75 * A.un[v * KN + gi] + 0.25 * ut[v];
            else if (A.comb == 2) o = A.un[v * KN + gi] * (1.0 / 3.0) + 2.0 / 3.0 * ut[v];
            else o = ut[v];
            A.out[v * KN + gi] = o;
        }
        if (A.collect && A.limiting > 0) {
            const double p = pres3(g, ut);
            // the bounds the stage keeps: the positivity ones under the combined limiting
            const double rf0 = MO.h_b[3 * MN + mn];
            const double rl = A.limiting == 3 ? idp::dmin(A.beta * rf0, rf0) : MO.h_b[0 * MN + mn];
            const double rh = A.limiting == 3 ? INFINITY : MO.h_b[1 * MN + mn], pl = MO.h_b[2 * MN + mn];
            if (ut[0] < rl - kViol3 * fabs(rl) || ut[0] > rh + kViol3 * fabs(rh)) vr++;
            if (p < pl - kViol3 * fabs(pl)) vp++;
            if (!(ut[0] > 0.0) || !(p > 0.0)) np_++;
            rmin_st = idp::dmin(rmin_st, ut[0]);
            pmin_st = idp::dmin(pmin_st, p);
        }
    }
    if (A.collect && A.limiting > 0) {
        const unsigned FULL = 0xffffffffu;
        vr = __reduce_add_sync(FULL, vr);
        vp = __reduce_add_sync(FULL, vp);
        np_ = __reduce_add_sync(FULL, np_);
        for (int o = 16; o > 0; o >>= 1) {
            rmin_st = idp::dmin(rmin_st, __shfl_down_sync(FULL, rmin_st, o));
            pmin_st = idp::dmin(pmin_st, __shfl_down_sync(FULL, pmin_st, o));
        }
        if ((threadIdx.x & 31) == 0) {
            if (vr) atomicAdd(&A.stats->n_vrho, (unsigned long long)vr);
            if (vp) atomicAdd(&A.stats->n_vp, (unsigned long long)vp);
            if (np_) atomicAdd(&A.stats->n_nonpos, (unsigned long long)np_);
            stat_min(&A.stats->min_rho_bits, rmin_st);
            stat_min(&A.stats->min_p_bits, pmin_st);
        }
        if ((vr | vp | np_) != 0u && (threadIdx.x & 31) == 0) atomicOr(A.status, S_VIOLATION);
    }
}

}  // namespace idp3
