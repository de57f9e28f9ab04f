// idp_element.cuh -- the per-element pass of one stage of the IDP LGL-DGSEM
// (arXiv 2607.06045, Sec. 2): volume two-point fluxes and their Sbar
// contraction into high-order subcell fluxes (Eq. fluxdifferencingform),
// low-order graph-viscosity subcell fluxes (Eq. FVmethod, c/d form of
// Eq. LowOrderScheme_globalIndices), conforming and boundary LLF fluxes, the
// low-order update, bar-state bounds (Eqs. Bounds_Positivity,
// Bounds_Barstates), Zalesak density and closed-form pressure limiting of the
// antidiffusive subcell fluxes (Sec. 2.3) and the SSP-RK stage combination.
//
// Mapping: one thread block holds EPB elements, one thread per LGL node; the
// (N+1)^2 nodal states, primitives, pair fluxes and subcell fluxes of each
// element live in shared memory. Mortar faces read the per-node slots written
// by the mortar-flux kernel; mortar nodes hand their post-volume state to the
// mortar-limiting kernels through the same slots.
#pragma once

#include "idp_device.cuh"

namespace idp {

struct StageArgs {
    const double *u;      // stage state u^(s)
    const double *un;     // step-start state (step mode)
    double *out;          // step mode: u^(s+1); rhs mode: right-hand side
    int mode;             // 0: rhs, 1: step
    int comb;             // step mode: 0 out = ut, 1 out = 3/4 un + 1/4 ut, 2 out = un/3 + 2/3 ut
    int limiting;         // 0 none, 1 positivity, 2 local
    int collect;          // statistics on/off
    double dt;            // rhs mode
    const unsigned long long *dtmin;  // step mode: per-sim min of m / sum 2d (ordered bits)
    double cfl;
    double t;             // rhs mode time
    const double *t_sim;  // step mode per-sim time
    double tstage;        // step mode: stage time = t_sim + tstage * dt
    double beta, gamma;
    const Ops *ops;
    unsigned *status;
    StatsAcc *stats;
};

__device__ __forceinline__ double stage_dt(const StageArgs &A, int sim) {
    return A.mode == 0 ? A.dt : A.cfl * __longlong_as_double((long long)A.dtmin[sim]);
}
__device__ __forceinline__ double stage_time(const StageArgs &A, int sim, double dt) {
    return A.mode == 0 ? A.t : A.t_sim[sim] + A.tstage * dt;
}

template <int NP, typename FT>
struct ElemSm {
    static constexpr int NN = NP * NP, N = NP - 1, NPAIR = NP * (NP - 1) / 2, NIF = 2 * NP * (NP - 1);
    double u[4][NN];
    double ufv[4][NN];
    double lfv[4][NN];
    double face[4][NP][4];   // J-weighted numerical flux along +x/+y (conforming, boundary)
    double outs[4][NP][4];   // outside state (conforming neighbour or ghost)
    double fbar[4][NP];      // bar-state density across the face
    double f2d[4][NP];       // 2 d_ij across the face
    FT Fdg[NIF][4];          // mass-weighted high-order subcell flux w_r * fhat (flux type)
    FT Ffv[NIF][4];          // mass-weighted low-order subcell flux (flux type)
    double Fv[NIF][4];       // the low-order subcell flux in FP64, for the residual sums
    double ibar[NIF], i2d[NIF], ell[NIF];
    double rmin[NN], rmax[NN], tol[NN], Rp[NN], Rm[NN];
    // pressure solve at u_FV in the form scaled by rho_FV: gm = (gamma-1) rho_FV,
    // pm = p_min rho_FV = beta (gamma-1)(rho E - |m|^2/2), c0 = g(0)
    double dtm[NN], gms[NN], pms[NN], c0[NN];
    float ufvf[4][NN];       // FP32 copies for the certified admissibility check
    float dtmf[NN], gmsf[NN], pmsf[NN], c0f[NN];
    unsigned char ex[NIF];   // density antidiffusion below the tolerance (R15)
    float uf[4][NN];         // FP32 state (FP32 form)
    double invA;             // 1 / (dx dy)
    FT pr[9][NN];            // rho, v1, v2, p, c, E, ln rho, ln beta, beta
    union {
        FT pair[2][NP][NPAIR][4];   // two-point fluxes (dead after the Sbar contraction)
        struct {
            double Ad[NIF][4];       // antidiffusive flux A = Fdg - Ffv in FP64
            float Af[NIF][4];        // and in FP32
        } a;
    } un;
};

template <int NP>
struct PairTab {
    // pair index -> (a, b), a < b, and (a, b) -> index
    __device__ __forceinline__ static void ab(int pi, int &a, int &b) {
        int k = pi;
        a = 0;
        while (k >= NP - 1 - a) { k -= NP - 1 - a; ++a; }
        b = a + 1 + k;
    }
    __device__ __forceinline__ static int idx(int a, int b) {
        // pairs are enumerated a-major: (0,1),(0,2),..,(0,N),(1,2),..
        return a * (2 * NP - a - 1) / 2 + (b - a - 1);
    }
};

template <int NP, typename FT>
__device__ __forceinline__ Prim<FT> load_prim(const ElemSm<NP, FT> &S, int n) {
    Prim<FT> q;
    q.rho = S.pr[0][n]; q.v1 = S.pr[1][n]; q.v2 = S.pr[2][n]; q.p = S.pr[3][n]; q.c = S.pr[4][n];
    q.E = S.pr[5][n]; q.lr = S.pr[6][n]; q.lb = S.pr[7][n]; q.beta = S.pr[8][n];
    return q;
}

// interface id (d, r, a): between nodes a and a+1 of row r (d = 0) or column r (d = 1)
template <int NP>
__device__ __forceinline__ int ifid(int d, int r, int a) { return (d * NP + r) * (NP - 1) + a; }
template <int NP>
__device__ __forceinline__ int nodeid(int d, int r, int a) { return d == 0 ? r * NP + a : a * NP + r; }

// Slot index of face node t on element side s of kind ft (mortar kinds only).
template <int NP>
__device__ __forceinline__ int slot_of(int ft, int m, int t) {
    int role = ft == FT_MLARGE ? 0 : (ft == FT_MSLO ? 1 : 2);
    return m * 3 * NP + role * NP + t;
}

__device__ __forceinline__ void block_stats(const StageArgs &A, double am, double mm, unsigned long long nact,
                                            unsigned long long nvr, unsigned long long nvp, unsigned long long nnp,
                                            unsigned long long ndx, double rmin_, double pmin_) {
    // warp reduction then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        am += __shfl_down_sync(0xffffffffu, am, o);
        mm += __shfl_down_sync(0xffffffffu, mm, o);
        nact += __shfl_down_sync(0xffffffffu, nact, o);
        nvr += __shfl_down_sync(0xffffffffu, nvr, o);
        nvp += __shfl_down_sync(0xffffffffu, nvp, o);
        nnp += __shfl_down_sync(0xffffffffu, nnp, o);
        ndx += __shfl_down_sync(0xffffffffu, ndx, o);
        rmin_ = fmin(rmin_, __shfl_down_sync(0xffffffffu, rmin_, o));
        pmin_ = fmin(pmin_, __shfl_down_sync(0xffffffffu, pmin_, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (mm > 0.0) { atomicAdd(&A.stats->alpha_vol_m, am); atomicAdd(&A.stats->mass, mm); }
        if (nact) atomicAdd(&A.stats->n_vol, nact);
        if (nvr) atomicAdd(&A.stats->n_vrho, nvr);
        if (nvp) atomicAdd(&A.stats->n_vp, nvp);
        if (nnp) atomicAdd(&A.stats->n_nonpos, nnp);
        if (ndx) atomicAdd(&A.stats->n_dtx, ndx);
        if (rmin_ > 0.0 && rmin_ < INFINITY) atomicMin(&A.stats->min_rho_bits, dbits(rmin_));
        if (pmin_ > 0.0 && pmin_ < INFINITY) atomicMin(&A.stats->min_p_bits, dbits(pmin_));
    }
}

template <int NP, int EPB>
struct ElemLaunch {
    // threads per block: one per node, rounded up to whole warps
    static constexpr int threads = ((EPB * NP * NP + 31) / 32) * 32;
};

template <int NP, typename FT, int EPB>
__global__ void __launch_bounds__(ElemLaunch<NP, EPB>::threads)
k_element(MeshDev mesh, SlotsDev sl, StageArgs A) {
    using SM = ElemSm<NP, FT>;
    constexpr int NN = NP * NP, N = NP - 1, NPAIR = SM::NPAIR, NIF = SM::NIF;
    constexpr int NT = ElemLaunch<NP, EPB>::threads;
    constexpr bool F32 = sizeof(FT) == 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    SM *sm = reinterpret_cast<SM *>(smraw);
    __shared__ double s_w[NP], s_iw[NP], s_S[NP][NP];

    const int tid = threadIdx.x;
    if (tid < NP) { s_w[tid] = A.ops->w[tid]; s_iw[tid] = A.ops->iw[tid]; }
    if (tid < NN) s_S[tid / NP][tid % NP] = A.ops->S[tid / NP][tid % NP];
    const double g = A.gamma;
    const FT ginv1 = FT(1.0 / (g - 1.0));
    const size_t KN = (size_t)mesh.K * NN;
    const bool limited = A.limiting > 0;
    const bool dgmode = (A.mode == 0 && A.dt == 0.0) || !limited;

    for (int e0 = blockIdx.x * EPB; e0 < mesh.K; e0 += gridDim.x * EPB) {
        // ---------------- P0: states, primitives, outside traces -------------
        for (int k = tid; k < EPB * NN; k += NT) {
            int le = k / NN, n = k - le * NN, e = e0 + le;
            if (e >= mesh.K) continue;
            SM &S = sm[le];
            size_t gi = (size_t)e * NN + n;
            double r = A.u[gi], m1 = A.u[KN + gi], m2 = A.u[2 * KN + gi], E = A.u[3 * KN + gi];
            S.u[0][n] = r; S.u[1][n] = m1; S.u[2][n] = m2; S.u[3][n] = E;
            Prim<FT> q;
            if constexpr (F32) {
                float m1f, m2f;
                q = make_prim_f32(g, r, m1, m2, E, true, m1f, m2f);
                S.uf[0][n] = q.rho; S.uf[1][n] = m1f; S.uf[2][n] = m2f; S.uf[3][n] = q.E;
            } else {
                q = make_prim<FT>(g, r, m1, m2, E, true);
            }
            if (!(r > 0.0) || !(q.p > FT(0)) || !isfinite(E) || !isfinite(m1) || !isfinite(m2))
                atomicOr(A.status, ST_BAD_INPUT);
            S.pr[0][n] = q.rho; S.pr[1][n] = q.v1; S.pr[2][n] = q.v2; S.pr[3][n] = q.p; S.pr[4][n] = q.c;
            S.pr[5][n] = q.E; S.pr[6][n] = q.lr; S.pr[7][n] = q.lb; S.pr[8][n] = q.beta;
            if (n == 0) { Geo geo = mesh.geom[e]; S.invA = 1.0 / (geo.z * geo.w); }
        }
        for (int k = tid; k < EPB * 4 * NP; k += NT) {
            int le = k / (4 * NP), s = (k / NP) % 4, t = k % NP, e = e0 + le;
            if (e >= mesh.K) continue;
            uchar4 ftv = mesh.ftype[e];
            int ft = s == 0 ? ftv.x : (s == 1 ? ftv.y : (s == 2 ? ftv.z : ftv.w));
            SM &S = sm[le];
            if (ft == FT_CONF) {
                int4 nb4 = mesh.fnbr[e];
                int nb = s == 0 ? nb4.x : (s == 1 ? nb4.y : (s == 2 ? nb4.z : nb4.w));
                size_t gi = (size_t)nb * NN + face_node<NP>(s ^ 1, t);
                for (int v = 0; v < 4; ++v) S.outs[s][t][v] = A.u[v * KN + gi];
            } else if (ft == FT_BND) {
                size_t gi = (size_t)e * NN + face_node<NP>(s, t);
                double in[4] = {A.u[gi], A.u[KN + gi], A.u[2 * KN + gi], A.u[3 * KN + gi]};
                int sim = mesh.sim[e];
                Geo geo = mesh.geom[e];
                int ii = face_node<NP>(s, t) % NP;
                double dtt = stage_dt(A, sim);
                double tt = stage_time(A, sim, dtt);
                double xn = geo.x + 0.5 * geo.z * (1.0 + A.ops->xi[ii]);
                double gst[4];
                ghost_state(mesh.siminfo[sim], s, in, xn, tt, gst);
                for (int v = 0; v < 4; ++v) S.outs[s][t][v] = gst[v];
            }
        }
        __syncthreads();

        // ---------------- P1: pair fluxes, face fluxes, interior FV ----------
        for (int k = tid; k < EPB * 2 * NP * NPAIR; k += NT) {
            int le = k / (2 * NP * NPAIR), rem = k - le * (2 * NP * NPAIR);
            int d = rem / (NP * NPAIR), r = (rem / NPAIR) % NP, pi = rem % NPAIR;
            if (e0 + le >= mesh.K) continue;
            SM &S = sm[le];
            int a, b;
            PairTab<NP>::ab(pi, a, b);
            Prim<FT> pa = load_prim<NP, FT>(S, nodeid<NP>(d, r, a)), pb = load_prim<NP, FT>(S, nodeid<NP>(d, r, b));
            FT f[4];
            ranocha<FT>(pa, pb, d, ginv1, f);
            for (int v = 0; v < 4; ++v) S.un.pair[d][r][pi][v] = f[v];
        }
        for (int k = tid; k < EPB * 4 * NP; k += NT) {
            int le = k / (4 * NP), s = (k / NP) % 4, t = k % NP, e = e0 + le;
            if (e >= mesh.K) continue;
            uchar4 ftv = mesh.ftype[e];
            int ft = s == 0 ? ftv.x : (s == 1 ? ftv.y : (s == 2 ? ftv.z : ftv.w));
            if (ft != FT_CONF && ft != FT_BND) continue;
            SM &S = sm[le];
            int d = s >> 1, n = face_node<NP>(s, t);
            double in[4] = {S.u[0][n], S.u[1][n], S.u[2][n], S.u[3][n]};
            double out[4] = {S.outs[s][t][0], S.outs[s][t][1], S.outs[s][t][2], S.outs[s][t][3]};
            Prim<FT> pi = load_prim<NP, FT>(S, n);
            Prim<FT> po;
            if constexpr (F32) {
                float m1f, m2f;
                po = make_prim_f32(g, out[0], out[1], out[2], out[3], false, m1f, m2f);
            } else {
                po = make_prim<FT>(g, out[0], out[1], out[2], out[3], false);
            }
            FT f[4];
            FT lam = (s == 0 || s == 2) ? llf_prim<FT>(out, po, in, pi, d, f) : llf_prim<FT>(in, pi, out, po, d, f);
            Geo geo = mesh.geom[e];
            double half = d == 0 ? 0.5 * geo.w : 0.5 * geo.z;
            for (int v = 0; v < 4; ++v) S.face[s][t][v] = half * (double)f[v];
            double sg = (s == 1 || s == 3) ? 1.0 : -1.0;
            double ld = (double)lam;
            double i2l = (double)(FT(0.5) / lam);
            S.fbar[s][t] = 0.5 * (in[0] + out[0]) - sg * (out[1 + d] - in[1 + d]) * i2l;
            S.f2d[s][t] = 2.0 * (s_w[t] * half / 2.0) * ld;
        }
        if (!dgmode) {
            for (int k = tid; k < EPB * NIF; k += NT) {
                int le = k / NIF, id = k - le * NIF, e = e0 + le;
                if (e >= mesh.K) continue;
                int d = id / (NP * N), r = (id / N) % NP, a = id % N;
                SM &S = sm[le];
                int na = nodeid<NP>(d, r, a), nb = nodeid<NP>(d, r, a + 1);
                Prim<FT> pa = load_prim<NP, FT>(S, na), pb = load_prim<NP, FT>(S, nb);
                FT vna = d == 0 ? pa.v1 : pa.v2, vnb = d == 0 ? pb.v1 : pb.v2;
                FT la = fabs(vna) + pa.c, lb = fabs(vnb) + pb.c;
                FT lam = la > lb ? la : lb;
                FT ua[4], ub[4];
                for (int v = 0; v < 4; ++v) {
                    ua[v] = F32 ? (FT)S.uf[v][na] : (FT)S.u[v][na];
                    ub[v] = F32 ? (FT)S.uf[v][nb] : (FT)S.u[v][nb];
                }
                FT fa[4], fb[4];
                phys_flux<FT>(ua[1], ua[2], ua[3], pa.p, vna, d, fa);
                phys_flux<FT>(ub[1], ub[2], ub[3], pb.p, vnb, d, fb);
                Geo geo = mesh.geom[e];
                double cc = s_w[r] * (d == 0 ? geo.w : geo.z) / 4.0;
                FT ccf = (FT)cc;
                for (int v = 0; v < 4; ++v) {
                    FT fv = ccf * (fa[v] + fb[v]) - ccf * lam * (ub[v] - ua[v]);
                    S.Ffv[id][v] = fv;
                    S.Fv[id][v] = (double)fv;
                }
                double ld = (double)lam;
                double i2l = (double)(FT(0.5) / lam);
                S.i2d[id] = 2.0 * cc * ld;
                S.ibar[id] = 0.5 * (S.u[0][na] + S.u[0][nb]) - (S.u[1 + d][nb] - S.u[1 + d][na]) * i2l;
            }
        }
        __syncthreads();

        // ---------------- P2: high-order subcell fluxes; low-order update ----
        for (int k = tid; k < EPB * NIF; k += NT) {
            int le = k / NIF, id = k - le * NIF, e = e0 + le;
            if (e >= mesh.K) continue;
            int d = id / (NP * N), r = (id / N) % NP, a = id % N;
            SM &S = sm[le];
            FT acc[4] = {FT(0), FT(0), FT(0), FT(0)};
            for (int l = 0; l <= a; ++l)
                for (int kk = a + 1; kk < NP; ++kk) {
                    FT sv = (FT)s_S[l][kk];
                    int pi = PairTab<NP>::idx(l, kk);
                    for (int v = 0; v < 4; ++v) acc[v] += sv * S.un.pair[d][r][pi][v];
                }
            Geo geo = mesh.geom[e];
            FT wh = (FT)(s_w[r] * (d == 0 ? 0.5 * geo.w : 0.5 * geo.z));
            for (int v = 0; v < 4; ++v) S.Fdg[id][v] = wh * acc[v];
        }
        if (!dgmode) {
            for (int k = tid; k < EPB * NN; k += NT) {
                int le = k / NN, n = k - le * NN, e = e0 + le;
                if (e >= mesh.K) continue;
                SM &S = sm[le];
                int i = n % NP, j = n / NP;
                int sim = mesh.sim[e];
                double dt = stage_dt(A, sim);
                double dtm = dt * (4.0 * S.invA) * s_iw[i] * s_iw[j];
                double L[4] = {0, 0, 0, 0};
                double lo = S.u[0][n], hi = S.u[0][n], ds = 0.0;
                uchar4 ftv = mesh.ftype[e];
                int4 nb4 = mesh.fnbr[e];
                // x direction: left then right; y: bottom then top
                for (int d = 0; d < 2; ++d) {
                    int pos = d == 0 ? i : j, row = d == 0 ? j : i;
                    for (int side = 0; side < 2; ++side) {
                        bool interior = side == 0 ? pos > 0 : pos < N;
                        if (interior) {
                            int id = ifid<NP>(d, row, side == 0 ? pos - 1 : pos);
                            double sgn = side == 0 ? 1.0 : -1.0;
                            for (int v = 0; v < 4; ++v) L[v] += sgn * S.Fv[id][v];
                            lo = fmin(lo, S.ibar[id]); hi = fmax(hi, S.ibar[id]);
                            ds += S.i2d[id];
                        } else {
                            int s = 2 * d + side;
                            int ft = s == 0 ? ftv.x : (s == 1 ? ftv.y : (s == 2 ? ftv.z : ftv.w));
                            if (ft == FT_CONF || ft == FT_BND) {
                                double sgn = side == 0 ? 1.0 : -1.0;
                                for (int v = 0; v < 4; ++v) L[v] += sgn * (s_w[row] * S.face[s][row][v]);
                                lo = fmin(lo, S.fbar[s][row]); hi = fmax(hi, S.fbar[s][row]);
                                ds += S.f2d[s][row];
                            } else {
                                int m = s == 0 ? nb4.x : (s == 1 ? nb4.y : (s == 2 ? nb4.z : nb4.w));
                                int q = slot_of<NP>(ft, m, row);
                                for (int v = 0; v < 4; ++v) L[v] += sl.clo[(size_t)v * sl.S + q];
                                lo = fmin(lo, sl.rbmin[q]); hi = fmax(hi, sl.rbmax[q]);
                                ds += sl.dsum[q];
                            }
                        }
                    }
                }
                double q[4];
                S.dtm[n] = dtm;
                for (int v = 0; v < 4; ++v) {
                    S.lfv[v][n] = L[v];
                    q[v] = S.u[v][n] + dtm * L[v];
                    S.ufv[v][n] = q[v];
                    S.ufvf[v][n] = (float)q[v];
                }
                double rmin, rmax;
                if (A.limiting == 2) { rmin = fmax(lo, A.beta * q[0]); rmax = hi; }
                else { rmin = A.beta * q[0]; rmax = INFINITY; }
                if (q[0] < rmin) rmin = q[0];
                if (q[0] > rmax) rmax = q[0];
                S.rmin[n] = rmin; S.rmax[n] = rmax;
                double rp = (g - 1.0) * (q[0] * q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]));   // rho p
                double gms = (g - 1.0) * q[0], pms = A.beta * rp;
                double c0 = g_zero(gms, q, pms);
                S.gms[n] = gms; S.pms[n] = pms; S.c0[n] = c0;
                S.tol[n] = kTol * fabs(q[0]);
                S.dtmf[n] = (float)dtm; S.gmsf[n] = (float)gms; S.pmsf[n] = (float)pms; S.c0f[n] = (float)c0;
                if (A.collect && dtm * ds > 1.0) atomicAdd(&A.stats->n_dtx, 1ull);
            }
        }
        __syncthreads();

        if (dgmode) {
            // ------------- unlimited high-order residual (Eq. evolutionformula)
            for (int k = tid; k < EPB * NN; k += NT) {
                int le = k / NN, n = k - le * NN, e = e0 + le;
                if (e >= mesh.K) continue;
                SM &S = sm[le];
                int i = n % NP, j = n / NP;
                Geo geo = mesh.geom[e];
                int sim = mesh.sim[e];
                double mi = geo.z * geo.w / 4.0 * s_w[i] * s_w[j];
                double L[4] = {0, 0, 0, 0};
                uchar4 ftv = mesh.ftype[e];
                int4 nb4 = mesh.fnbr[e];
                for (int d = 0; d < 2; ++d) {
                    int pos = d == 0 ? i : j, row = d == 0 ? j : i;
                    for (int side = 0; side < 2; ++side) {
                        bool interior = side == 0 ? pos > 0 : pos < N;
                        double sgn = side == 0 ? 1.0 : -1.0;
                        if (interior) {
                            int id = ifid<NP>(d, row, side == 0 ? pos - 1 : pos);
                            for (int v = 0; v < 4; ++v) L[v] += sgn * (double)S.Fdg[id][v];
                        } else {
                            int s = 2 * d + side;
                            int ft = s == 0 ? ftv.x : (s == 1 ? ftv.y : (s == 2 ? ftv.z : ftv.w));
                            if (ft == FT_CONF || ft == FT_BND) {
                                for (int v = 0; v < 4; ++v) L[v] += sgn * (s_w[row] * S.face[s][row][v]);
                            } else {
                                int m = s == 0 ? nb4.x : (s == 1 ? nb4.y : (s == 2 ? nb4.z : nb4.w));
                                int q = slot_of<NP>(ft, m, row);
                                for (int v = 0; v < 4; ++v) L[v] += sl.chi[(size_t)v * sl.S + q];
                            }
                        }
                    }
                }
                size_t gi = (size_t)e * NN + n;
                if (A.mode == 0) {
                    for (int v = 0; v < 4; ++v) A.out[v * KN + gi] = L[v] / mi;
                } else {
                    double dt = stage_dt(A, sim);
                    for (int v = 0; v < 4; ++v) {
                        double ut = S.u[v][n] + dt / mi * L[v];
                        double o = ut;
                        if (A.comb == 1) o = 0.75 * A.un[v * KN + gi] + 0.25 * ut;
                        else if (A.comb == 2) o = A.un[v * KN + gi] * (1.0 / 3.0) + 2.0 / 3.0 * ut;
                        A.out[v * KN + gi] = o;
                    }
                }
            }
            __syncthreads();
            continue;
        }

        // ---------------- P2b: antidiffusive fluxes A = Fdg - Ffv ------------
        for (int k = tid; k < EPB * NIF; k += NT) {
            int le = k / NIF, id = k - le * NIF;
            if (e0 + le >= mesh.K) continue;
            SM &S = sm[le];
            int d = id / (NP * N), r = (id / N) % NP, a = id % N;
            for (int v = 0; v < 4; ++v) {
                FT fd = S.Fdg[id][v], ff = S.Ffv[id][v];
                S.un.a.Ad[id][v] = (double)fd - S.Fv[id][v];
                S.un.a.Af[id][v] = (float)(fd - ff);
            }
            int nl = nodeid<NP>(d, r, a), nr = nodeid<NP>(d, r, a + 1);
            double aa = fabs(S.un.a.Ad[id][0]);
            S.ex[id] = (S.dtm[nl] * aa <= S.tol[nl]) && (S.dtm[nr] * aa <= S.tol[nr]);
        }
        __syncthreads();

        // ---------------- P3: Zalesak factors for density (R7) -------------
        // R+ = min(1, Q+/P+) with Q+ = (m/dt)(rho_max - rho_FV), written with
        // dt/m so that only an active bound costs a division
        for (int k = tid; k < EPB * NN; k += NT) {
            int le = k / NN, n = k - le * NN, e = e0 + le;
            if (e >= mesh.K) continue;
            SM &S = sm[le];
            int i = n % NP, j = n / NP;
            double dtm = S.dtm[n];
            double Pp = 0.0, Pm = 0.0;
            for (int d = 0; d < 2; ++d) {
                int pos = d == 0 ? i : j, row = d == 0 ? j : i;
                for (int side = 0; side < 2; ++side) {
                    if (side == 0 ? pos == 0 : pos == N) continue;
                    int a = side == 0 ? pos - 1 : pos;
                    int id = ifid<NP>(d, row, a);
                    if (S.ex[id]) continue;
                    double Ar = S.un.a.Ad[id][0];
                    double G = side == 0 ? Ar : -Ar;
                    Pp += G > 0 ? G : 0.0;
                    Pm += G < 0 ? G : 0.0;
                }
            }
            double rfv = S.ufv[0][n];
            double qp = S.rmax[n] - rfv, qm = S.rmin[n] - rfv;   // Q / (m/dt)
            double pp = dtm * Pp, pmm = dtm * Pm;
            double Rp = (pp > qp) ? qp / pp : 1.0;
            double Rm = (pmm < qm) ? qm / pmm : 1.0;
            S.Rp[n] = Rp < 0.0 ? 0.0 : Rp;
            S.Rm[n] = Rm < 0.0 ? 0.0 : Rm;
        }
        __syncthreads();

        // ---------------- P4: per interface factor (R7, R8; Gamma = 4) -----
        for (int k = tid; k < EPB * NIF; k += NT) {
            int le = k / NIF, id = k - le * NIF, e = e0 + le;
            if (e >= mesh.K) continue;
            int d = id / (NP * N), r = (id / N) % NP, a = id % N;
            SM &S = sm[le];
            int nl = nodeid<NP>(d, r, a), nr = nodeid<NP>(d, r, a + 1);
            double Ar = S.un.a.Ad[id][0];
            double lr = S.ex[id] ? 1.0
                           : (-Ar > 0.0) ? fmin(S.Rp[nl], S.Rm[nr]) : fmin(S.Rm[nl], S.Rp[nr]);
            double th = lr;
            // left end point: Gamma-scaled increment -4 dt/m A; right: +4 dt/m A
            for (int side = 0; side < 2 && th > 0.0; ++side) {
                int nd = side == 0 ? nl : nr;
                float sgf = side == 0 ? -4.0f : 4.0f;
                float u0f[4], af[4];
                float sdf = sgf * S.dtmf[nd];
                for (int v = 0; v < 4; ++v) { u0f[v] = S.ufvf[v][nd]; af[v] = sdf * S.un.a.Af[id][v]; }
                if (admissible_f32(S.gmsf[nd], u0f, af, S.pmsf[nd], S.c0f[nd], (float)th) && S.c0[nd] > 0.0 &&
                    S.ufv[0][nd] > 0.0)
                    continue;   // the whole interval [0, th] is admissible
                double u0[4], av[4];
                double sd = (side == 0 ? -4.0 : 4.0) * S.dtm[nd];
                for (int v = 0; v < 4; ++v) { u0[v] = S.ufv[v][nd]; av[v] = sd * S.un.a.Ad[id][v]; }
                th = theta_max(g, u0, av, S.gms[nd], S.pms[nd], S.c0[nd], th);
            }
            S.ell[id] = th;   // min over both end points (each searched below the previous)
        }
        __syncthreads();

        // ---------------- P5: blend, outputs, mortar hand-off, stats --------
        {
            double st_am = 0.0, st_m = 0.0, st_rmin = INFINITY, st_pmin = INFINITY;
            unsigned long long st_act = 0, st_vr = 0, st_vp = 0, st_np = 0;
            for (int k = tid; k < EPB * NN; k += NT) {
                int le = k / NN, n = k - le * NN, e = e0 + le;
                if (e >= mesh.K) continue;
                SM &S = sm[le];
                int i = n % NP, j = n / NP;
                Geo geo = mesh.geom[e];
                double mi = geo.z * geo.w / 4.0 * s_w[i] * s_w[j];
                double dtm = S.dtm[n];
                double sacc[4] = {0, 0, 0, 0}, lmin = 1.0;
                for (int d = 0; d < 2; ++d) {
                    int pos = d == 0 ? i : j, row = d == 0 ? j : i;
                    if (pos > 0) {
                        int id = ifid<NP>(d, row, pos - 1);
                        double l = S.ell[id];
                        for (int v = 0; v < 4; ++v) sacc[v] += l * S.un.a.Ad[id][v];
                        lmin = fmin(lmin, l);
                    }
                    if (pos < N) {
                        int id = ifid<NP>(d, row, pos);
                        double l = S.ell[id];
                        for (int v = 0; v < 4; ++v) sacc[v] -= l * S.un.a.Ad[id][v];
                        lmin = fmin(lmin, l);
                    }
                }
                double uvol[4], resv[4] = {0, 0, 0, 0};
                for (int v = 0; v < 4; ++v) uvol[v] = S.ufv[v][n] + dtm * sacc[v];
                if (A.mode == 0)
                    for (int v = 0; v < 4; ++v) resv[v] = S.lfv[v][n] + sacc[v];
                size_t gi = (size_t)e * NN + n;
                // mortar hand-off
                uchar4 ftv = mesh.ftype[e];
                int4 nb4 = mesh.fnbr[e];
                int nmort = 0;
                int sides[2] = {-1, -1};
                if (i == 0 && ftv.x >= FT_MLARGE) sides[nmort++] = 0;
                if (i == N && ftv.y >= FT_MLARGE) sides[nmort++] = 1;
                if (j == 0 && ftv.z >= FT_MLARGE) sides[nmort++] = 2;
                if (j == N && ftv.w >= FT_MLARGE) sides[nmort++] = 3;
                for (int c = 0; c < nmort; ++c) {
                    int s = sides[c];
                    int ft = s == 0 ? ftv.x : (s == 1 ? ftv.y : (s == 2 ? ftv.z : ftv.w));
                    int m = s == 0 ? nb4.x : (s == 1 ? nb4.y : (s == 2 ? nb4.z : nb4.w));
                    int q = slot_of<NP>(ft, m, s < 2 ? j : i);
                    for (int v = 0; v < 4; ++v) {
                        sl.uvol[(size_t)v * sl.S + q] = uvol[v];
                        // rhs mode keeps the mass-weighted residual, step mode u^n
                        sl.un[(size_t)v * sl.S + q] = A.mode == 0 ? resv[v] : (A.comb != 0 ? A.un[v * KN + gi] : 0.0);
                    }
                    sl.rmin[q] = S.rmin[n]; sl.rmax[q] = S.rmax[n]; sl.pmin[q] = S.pms[n] / S.ufv[0][n];
                    sl.tol[q] = S.tol[n]; sl.mass[q] = mi; sl.nmort[q] = (float)nmort;
                }
                if (A.mode == 0) {
                    for (int v = 0; v < 4; ++v) A.out[v * KN + gi] = resv[v] / mi;
                } else {
                    for (int v = 0; v < 4; ++v) {
                        double o = uvol[v];
                        if (A.comb == 1) o = 0.75 * A.un[v * KN + gi] + 0.25 * uvol[v];
                        else if (A.comb == 2) o = A.un[v * KN + gi] * (1.0 / 3.0) + 2.0 / 3.0 * uvol[v];
                        A.out[v * KN + gi] = o;
                    }
                }
                if (A.collect) {
                    st_am += mi * (1.0 - lmin);
                    st_m += mi;
                    st_act += lmin < 1.0;
                    if (nmort == 0) {
                        // rho p = (gamma-1)(rho E - |m|^2/2): checks without division
                        double rp = (g - 1.0) * (uvol[0] * uvol[3] - 0.5 * (uvol[1] * uvol[1] + uvol[2] * uvol[2]));
                        // p >= p_min  <=>  rho p rho_FV >= (p_min rho_FV) rho
                        if (uvol[0] < S.rmin[n] - kViolTol * fabs(S.rmin[n]) ||
                            uvol[0] > S.rmax[n] + kViolTol * fabs(S.rmax[n])) st_vr++;
                        if (rp * S.ufv[0][n] < S.pms[n] * (1.0 - kViolTol) * uvol[0]) st_vp++;
                        if (!(uvol[0] > 0.0) || !(rp > 0.0)) st_np++;
                        st_rmin = fmin(st_rmin, uvol[0]);
                        if (lmin < 1.0) st_pmin = fmin(st_pmin, rp / uvol[0]);
                    }
                }
            }
            if (A.collect) block_stats(A, st_am, st_m, st_act, st_vr, st_vp, st_np, 0ull, st_rmin, st_pmin);
            if ((st_vr | st_vp | st_np) != 0ull) atomicOr(A.status, ST_VIOLATION);
        }
        __syncthreads();
    }
}

}  // namespace idp
