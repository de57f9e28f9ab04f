// idp_device.cuh -- device data structures and point functions of the IDP
// LGL-DGSEM right-hand side (arXiv 2607.06045, Sec. 2) for sm_103a.
//
// Arithmetic types: every routine is templated on the flux type FT (double
// for the FP64 path, float for the FP32 form). Bounds, limiter solves,
// blending and sums always use double.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "idp_bits.cuh"
#include "idp_fastmath.cuh"

namespace idp {

constexpr int NPMAX = 8;          // N <= 7
constexpr double kTol = 1e-14;    // limiter relaxation / exemption (reading R15)
constexpr double kViolTol = 1e-13;  // violation tolerance (reading R13)
constexpr double kEtaRelax = 1e-12;  // entropy bound: relative relaxation inside the limiter (R21)
constexpr double kEtaViol = 1e-11;   // entropy bound: tolerance of the violation count (R21)

// Face kinds of an element side (-x, +x, -y, +y).
enum : int { FT_CONF = 0, FT_BND = 1, FT_MLARGE = 2, FT_MSLO = 3, FT_MSHI = 4 };
// Boundary kinds (idp_bc)
enum : int { BC_PERIODIC = 0, BC_WALL = 1, BC_DIRICHLET = 2, BC_OUTFLOW = 3, BC_DMR = 4, BC_JET = 5 };
// status bits
enum : unsigned { ST_BAD_INPUT = 1u, ST_VIOLATION = 2u, ST_NONFINITE = 4u };

// Element geometry: x = left edge, y = bottom edge, z = dx, w = dy.
struct __align__(32) Geo {
    double x, y, z, w;
};

// Per-element constants formed once on the host: 4 / (dx dy), dx dy / 4,
// half and quarter edge lengths, and FP32 copies.
struct __align__(16) GeoC {
    double iA4, A4, hx, hy, qx, qy;
    float hxf, hyf, qxf, qyf, A4f, pad;
};

// Reference operators for NP = N + 1 nodes (Sec. 2.1, App. A).
struct Ops {
    double xi[NPMAX];                // LGL nodes
    double w[NPMAX];                 // LGL weights
    double iw[NPMAX];                // 1 / w
    double S[NPMAX][NPMAX];          // Sbar = 2 Qbar - Bbar
    double wt[NPMAX][2 * NPMAX];     // low-order mortar weights (reference units): local or all-to-all
    double I[2 * NPMAX][NPMAX];      // interpolation large -> small-face nodes
    double P[NPMAX][2 * NPMAX];      // projection small-face fluxes -> large
    // nonzero low-order mortar weights as a pair list (large node k,
    // small-face node r), k-major with r ascending, and per mortar slot (large
    // nodes first, then the small-face nodes) the pairs that touch it, in the
    // same order (at most 3 N + 2 pairs for the sparse local weights, all
    // 2 (N+1)^2 for the all-to-all weights)
    int npair;
    int pk[2 * NPMAX * NPMAX], pr[2 * NPMAX * NPMAX];
    int slot_n[3 * NPMAX];
    int slot_p[3 * NPMAX][2 * NPMAX];
    LogTab lg;                       // table of the FP64 logarithm
    // inverse of V_ik = sqrt((2k+1)/2) P_k(xi_i): nodal values to coefficients
    // of the orthonormal Legendre basis (shock indicator, combined limiting)
    double Vinv[NPMAX][NPMAX];
    // shock indicator: threshold T = 0.5 10^(-1.8 (N+1)^(1/4)), sharpness
    // s = ln((1 - 1e-4) / 1e-4)
    double ind_T, ind_s;
};

// Per simulation: boundary data (ghost states as conserved variables).
struct SimInfo {
    int32_t bc[4];
    int32_t pad[4];
    double bc_cons[4][4];
    double dmr_post[4];
    double dmr_pre[4];
    double y1;
    double pad2;
};

// Limiter statistics accumulators (device).
struct StatsAcc {
    double alpha_vol_m, mass, alpha_mort_len, len;
    unsigned long long n_vol, n_mort, n_fallback, n_vrho, n_vp, n_nonpos, n_dtx, n_stages;
    unsigned long long min_rho_bits, min_p_bits;   // positive doubles as ordered bits
    unsigned long long n_veta;                     // entropy-bound violations
};

struct MeshDev {
    int K, M, n_sims, n_mnodes;
    const Geo *geom;          // per element: x_left, y_bottom, dx, dy
    const GeoC *geoc;         // per element: derived constants
    const int32_t *sim;       // per element
    const int4 *fnbr;         // per element and side: neighbour element / mortar id / -1
    const uchar4 *ftype;      // per element and side: FT_*
    const int32_t *m_large;   // per mortar
    const int2 *m_small;      // per mortar: lower, upper small element
    const int32_t *m_info;    // per mortar: dir | (large_is_low << 1)
    const SimInfo *siminfo;
    const int32_t *mn_node;   // unique mortar nodes: global node index
    const int2 *mn_slot;      // their (first, second or -1) slot
    // mortar limiting blocks (k_mortar_limit_apply): per block its owned
    // nodes mn[mb_node_off[b] .. mb_node_off[b+1]) and its foreign mortars
    // mb_foreign[mb_for_off[b] .. mb_for_off[b+1]); mb_fmax their largest count
    const int32_t *mb_node_off, *mb_for_off, *mb_foreign;
    int mb_fmax, mb_blocks;
};

// Per-mortar-node scratch ("slots", index m * 3NP + q, large nodes first,
// then the lower and upper small element's face nodes).
struct SlotsDev {
    int S;                    // M * 3NP
    double *chi, *clo;        // [4][S] high/low-order contribution to m du/dt
    double *rbmin, *rbmax;    // bar-state density min/max over cross-mortar pairs
    double *dsum;             // sum_j 2 d_ij over cross-mortar pairs
    double *uvol, *un;        // [4][S] state after the volume step / at step start
    double *rmin, *rmax, *pmin, *tol, *mass;   // pmin: p_min rho_FV (divided by rfv where used)
    double *rfv;              // rho_FV
    float *nmort;             // n_i
    int32_t *bad;             // per mortar: interpolated state inadmissible
    double *ell;              // per mortar l_S
    // entropy bound and low-order bounds (local-limiting variants)
    double *lnK;              // ln K of the node's entropy bound, K = eta_min (1 - kEtaRelax)
    double *sbmin;            // min of s = ln p - gamma ln rho over the cross-mortar bar states
    double *lbmin, *lbmax;    // min/max of rho_FV over the nodes across the mortar
    double *lsmin;            // min of s(u_FV) over the nodes across the mortar
};

// ---------------------------------------------------------------------------
// point functions
// ---------------------------------------------------------------------------

// Ideal-gas constants, formed once on the host: gamma, gamma - 1,
// 1 / (gamma - 1) and their FP32 copies.
// The entropy bound works with s = ln p - gamma ln rho (ln eta = s - ln(gamma-1)):
// ln K = s_min + eoff, eoff = ln(1 - kEtaRelax) - ln(gamma - 1); a state
// violates the bound when s < ln K + eviol, eviol = ln(gamma - 1)
// - ln(1 - kEtaRelax) + ln(1 - kEtaViol).
struct Gas {
    double g, gm1, ginv1;
    float gf, gm1f, ginv1f;
    const LogTab *lg;   // device table of fast_log
    double eoff, eviol;
};
inline Gas make_gas(double gamma, const LogTab *lg) {
    Gas G;
    G.lg = lg;
    G.g = gamma; G.gm1 = gamma - 1.0; G.ginv1 = 1.0 / (gamma - 1.0);
    G.gf = (float)G.g; G.gm1f = (float)G.gm1; G.ginv1f = (float)G.ginv1;
    G.eoff = log1p(-kEtaRelax) - log(G.gm1);
    G.eviol = log(G.gm1) - log1p(-kEtaRelax) + log1p(-kEtaViol);
    return G;
}

__device__ __forceinline__ double pressure_d(double gm1, double r, double m1, double m2, double E) {
    return gm1 * (E - 0.5 * (m1 * m1 + m2 * m2) / r);
}

// max of two non-negative wave speeds: doubles by their bits (integer pipe),
// floats directly
__device__ __forceinline__ double speed_max(double a, double b) { return nn_lt(a, b) ? b : a; }
__device__ __forceinline__ float speed_max(float a, float b) { return a > b ? a : b; }

// Node primitives in the flux type.
template <typename FT> struct Prim {
    FT rho, v1, v2, p, c, E, lr, lb, beta;
};

// a where c holds, else b, field by field: per-lane selects on the integer
// pipe, so that lanes which need a two-point flux with their operands in
// either order share one inlined copy of it
template <typename FT>
__device__ __forceinline__ Prim<FT> pick_prim(bool c, const Prim<FT> &a, const Prim<FT> &b) {
    Prim<FT> r;
    r.rho = c ? a.rho : b.rho; r.v1 = c ? a.v1 : b.v1; r.v2 = c ? a.v2 : b.v2;
    r.p = c ? a.p : b.p; r.c = c ? a.c : b.c; r.E = c ? a.E : b.E;
    r.lr = c ? a.lr : b.lr; r.lb = c ? a.lb : b.lb; r.beta = c ? a.beta : b.beta;
    return r;
}

// Logarithmic means of Ranocha's flux with one division per pair: the
// density mean {rho}_ln and the inverse mean 1/{rho/p}_ln. For each mean the
// far branch is (a-b)/(ln a - ln b) from per-node logarithms (FP64) or
// ln(a/b) (FP32); for u = ((a-b)/(a+b))^2 below 1e-4 (FP64) or 1e-2 (FP32)
// the Ismail-Roe series (a+b)/(2 F(u)), F = 1 + u/3 + u^2/5 + u^3/7, with
// 1/F from the inverted series 1 - u/3 - 4u^2/45 - 44u^3/945. The two
// denominators share one reciprocal. HALVES: rho, beta and their logarithms
// are given halved (make_prim_half), which scales every quotient exactly and
// leaves the series' factors 1/2 and 2 to the data.
template <typename FT, bool HALVES = false>
__device__ __forceinline__ void log_means(const Prim<FT> &a, const Prim<FT> &b, FT &rho_ln, FT &ibeta) {
    constexpr bool dbl = sizeof(FT) == 8;
    const FT thr = dbl ? FT(1e-4) : FT(1e-2);
    FT dr = a.rho - b.rho, sr = a.rho + b.rho;
    FT db = a.beta - b.beta, sb = a.beta + b.beta;
    bool nr, nb;
    if constexpr (dbl) {
        // the test only picks between two forms that agree to rounding near
        // the threshold, so FP32 (converted on the integer pipe) suffices and
        // spares four FP64 operations per mean; <= keeps equal states that
        // flush to zero in FP32 on the series
        const float drf = d2f(dr), srf = d2f(sr), dbf = d2f(db), sbf = d2f(sb);
        nr = drf * drf <= 1e-4f * (srf * srf);
        nb = dbf * dbf <= 1e-4f * (sbf * sbf);
    } else {
        nr = dr * dr < thr * (sr * sr);
        nb = db * db < thr * (sb * sb);
    }
    FT lr, lb;
    if (dbl) { lr = a.lr - b.lr; lb = a.lb - b.lb; }
    else {
        lr = nr ? FT(0) : (FT)logf((float)(a.rho / b.rho));
        lb = nb ? FT(0) : (FT)logf((float)(a.beta / b.beta));
    }
    FT Xr = nr ? sr : lr, Xb = nb ? sb : db;
    FT R;
    if constexpr (dbl) R = fast_rcp(Xr * Xb);
    else R = FT(1) / (Xr * Xb);
    FT ixr = Xb * R, ixb = Xr * R;   // 1/Xr, 1/Xb
    if (nr) {
        FT f = dr * ixr, u = f * f;
        FT invF = FT(1) - u * (FT(1.0 / 3.0) + u * (FT(4.0 / 45.0) + u * FT(44.0 / 945.0)));
        rho_ln = HALVES ? sr * invF : FT(0.5) * sr * invF;
    } else {
        rho_ln = dr * ixr;
    }
    if (nb) {
        FT f = db * ixb, u = f * f;
        FT F = FT(1) + u * (FT(1.0 / 3.0) + u * (FT(1.0 / 5.0) + u * FT(1.0 / 7.0)));
        ibeta = HALVES ? F * ixb : FT(2) * F * ixb;
    } else {
        ibeta = lb * ixb;
    }
}

// Ranocha's entropy-conserving, kinetic-energy-preserving two-point flux
// along axis d (reading R1; the paper names it in Sec. 3).
template <typename FT>
__device__ __forceinline__ void ranocha(const Prim<FT> &a, const Prim<FT> &b, int d, FT ginv1, FT f[4]) {
    FT rho_ln, ibeta;
    log_means<FT>(a, b, rho_ln, ibeta);
    FT v1m = FT(0.5) * (a.v1 + b.v1), v2m = FT(0.5) * (a.v2 + b.v2), pm = FT(0.5) * (a.p + b.p);
    FT vna = d == 0 ? a.v1 : a.v2, vnb = d == 0 ? b.v1 : b.v2;
    FT fr = rho_ln * (FT(0.5) * (vna + vnb));
    f[0] = fr;
    f[1] = fr * v1m + (d == 0 ? pm : FT(0));
    f[2] = fr * v2m + (d == 1 ? pm : FT(0));
    f[3] = fr * (FT(0.5) * (a.v1 * b.v1 + a.v2 * b.v2) + ibeta * ginv1) + FT(0.5) * (a.p * vnb + b.p * vna);
}

// Physical flux along axis d from conserved momentum/energy and primitives.
template <typename FT>
__device__ __forceinline__ void phys_flux(FT m1, FT m2, FT E, FT p, FT vn, int d, FT f[4]) {
    f[0] = (d == 0 ? m1 : m2);
    f[1] = m1 * vn + (d == 0 ? p : FT(0));
    f[2] = m2 * vn + (d == 1 ? p : FT(0));
    f[3] = (E + p) * vn;
}

// Primitive state from a conserved state (double input). The pressure is
// always formed in FP64 (E - |m|^2 / 2 rho cancels at high Mach numbers) with
// one reciprocal of rho; with full = true also beta = rho / p and, in the
// FP64 path, ln rho and ln beta = ln rho - ln p. The velocity, pressure and
// sound speed use explicitly rounded operations so that every element that
// forms them for the same node gets the same bits.
template <typename FT>
__device__ __forceinline__ Prim<FT> make_prim(const Gas &G, double r, double m1, double m2, double E, bool full) {
    const double g = G.g;
    Prim<FT> q;
    double ri = fast_rcp(r);
    double v1 = __dmul_rn(m1, ri), v2 = __dmul_rn(m2, ri);
    double ke = __dmul_rn(0.5, __dadd_rn(__dmul_rn(m1, v1), __dmul_rn(m2, v2)));
    double p = __dmul_rn(G.gm1, __dadd_rn(E, -ke));
    q.rho = (FT)r; q.v1 = (FT)v1; q.v2 = (FT)v2; q.p = (FT)p; q.E = (FT)E;
    q.lr = q.lb = FT(0);
    if (sizeof(FT) == 8) {
        q.c = (FT)fast_sqrt(__dmul_rn(__dmul_rn(g, p), ri));
        if (full) {
            q.beta = (FT)__dmul_rn(r, fast_rcp(p));
            double lr = fast_log(r, G.lg);
            q.lr = (FT)lr;
            q.lb = (FT)(lr - fast_log(p, G.lg));
        } else {
            q.beta = FT(0);
        }
    } else {
        float pf = (float)p, rf = (float)r;
        q.c = (FT)__fsqrt_rn(__fdiv_rn(__fmul_rn(G.gf, pf), rf));
        q.beta = full ? (FT)__fdiv_rn(rf, pf) : FT(0);
    }
    return q;
}

// Node data of the FP64 element pass in halves: v1/2, v2/2 and p/2 (the
// same bits as make_prim's v1, v2, p scaled by 1/2, which is exact), rho/2,
// and beta'/2 with beta' = rho / (rho e) = (gamma - 1) rho / p, and the
// halves of ln rho and ln beta' (beta' rescales beta at rounding level; the
// logarithmic mean's quotient is homogeneous of degree -1 in beta, so
// 1/{beta'}_ln = 1/((gamma - 1) {beta}_ln)). The two-point flux's means
// become sums of halves, the logarithmic means lose their factors 1/2 and 2
// and the factor 1/(gamma - 1) sits in beta'; c is make_prim's.
// (full = false: v/2, p/2 and c only, rho whole)
__device__ __forceinline__ Prim<double> make_prim_half(const Gas &G, double r, double m1, double m2, double E,
                                                       bool full = true) {
    Prim<double> q;
    const double ri = fast_rcp(r), hri = 0.5 * ri;
    const double h1 = __dmul_rn(m1, hri), h2 = __dmul_rn(m2, hri);
    const double re = __dadd_rn(E, -__dadd_rn(__dmul_rn(m1, h1), __dmul_rn(m2, h2)));   // rho e
    const double hp = __dmul_rn(0.5 * G.gm1, re);
    q.rho = r; q.v1 = h1; q.v2 = h2; q.p = hp; q.E = E;
    q.c = fast_sqrt(__dmul_rn(__dmul_rn(2.0 * G.g, hp), ri));
    q.beta = q.lr = q.lb = 0.0;
    if (full) {
        q.rho = 0.5 * r;
        q.beta = q.rho * fast_rcp(re);
        q.lr = 0.5 * fast_log(r, G.lg);
        q.lb = q.lr - 0.5 * fast_log(re, G.lg);
    }
    return q;
}

// Half the physical flux along d (the mass flux m_d whole) from half the
// normal velocity and half the pressure.
__device__ __forceinline__ void phys_flux_half(double m1, double m2, double E, double hp, double hvn, int d,
                                               double f[4]) {
    f[0] = (d == 0 ? m1 : m2);
    f[1] = m1 * hvn + (d == 0 ? hp : 0.0);
    f[2] = m2 * hvn + (d == 1 ? hp : 0.0);
    f[3] = (E + 2.0 * hp) * hvn;
}

// Local Lax-Friedrichs flux along axis d (Davis wave speed, R3) from the
// conserved states and the halved data of make_prim_half; returns lambda.
__device__ __forceinline__ double llf_half(const double uL[4], const Prim<double> &a, const double uR[4],
                                           const Prim<double> &b, int d, double f[4]) {
    const double vna = d == 0 ? a.v1 : a.v2, vnb = d == 0 ? b.v1 : b.v2;
    const double lam = speed_max(2.0 * fabs(vna) + a.c, 2.0 * fabs(vnb) + b.c);
    double fa[4], fb[4];
    phys_flux_half(uL[1], uL[2], uL[3], a.p, vna, d, fa);
    phys_flux_half(uR[1], uR[2], uR[3], b.p, vnb, d, fb);
    const double hl = 0.5 * lam;
    f[0] = 0.5 * (fa[0] + fb[0]) - hl * (uR[0] - uL[0]);
    for (int v = 1; v < 4; ++v) f[v] = (fa[v] + fb[v]) - hl * (uR[v] - uL[v]);
    return lam;
}

// Ranocha's flux (R1) from the halved node data of make_prim_half.
__device__ __forceinline__ void ranocha_half(const Prim<double> &a, const Prim<double> &b, int d, double f[4]) {
    double rho_ln, ibeta;
    log_means<double, true>(a, b, rho_ln, ibeta);
    const double v1m = a.v1 + b.v1, v2m = a.v2 + b.v2, pm = a.p + b.p;
    const double vna = d == 0 ? a.v1 : a.v2, vnb = d == 0 ? b.v1 : b.v2;
    const double fr = rho_ln * (d == 0 ? v1m : v2m);
    f[0] = fr;
    f[1] = fr * v1m + (d == 0 ? pm : 0.0);
    f[2] = fr * v2m + (d == 1 ? pm : 0.0);
    f[3] = fr * (2.0 * (a.v1 * b.v1 + a.v2 * b.v2) + ibeta) + 2.0 * (a.p * vnb + b.p * vna);
}

// FP32 primitives of the FP32 form. When E - |m|^2/2rho keeps at least an
// eighth of E the pressure is formed in FP32: with the state rounded once,
// the kinetic energy carries at most 4 unit roundings and E one half, so the
// FP32 pressure is within (0.5 + 4 * 7/8) * 8 + 0.5 = 32.5 unit roundings
// (2e-6) of the pressure of the rounded state and positive for sure;
// otherwise it is formed in FP64 as above. The state is rounded to FP32 on
// the integer pipe (d2f); the same function serves every element that reads
// the node, so they all get the same bits.
__device__ __forceinline__ Prim<float> make_prim_f32(const Gas &G, double r, double m1, double m2, double E, bool full,
                                                     float &m1o, float &m2o) {
    float rf = d2f(r), m1f = d2f(m1), m2f = d2f(m2), Ef = d2f(E);
    float rif = __frcp_rn(rf);
    float v1 = __fmul_rn(m1f, rif), v2 = __fmul_rn(m2f, rif);
    float kef = __fmul_rn(0.5f, __fadd_rn(__fmul_rn(m1f, v1), __fmul_rn(m2f, v2)));
    float pef = __fadd_rn(Ef, -kef);
    Prim<float> q;
    if (rf > 0.0f && Ef > 0.0f && pef >= 0.125f * Ef) {
        q.rho = rf; q.v1 = v1; q.v2 = v2; q.E = Ef;
        q.p = __fmul_rn(G.gm1f, pef);
        q.lr = q.lb = 0.0f;
        q.c = __fsqrt_rn(__fmul_rn(__fmul_rn(G.gf, q.p), rif));
        q.beta = full ? __fmul_rn(rf, __frcp_rn(q.p)) : 0.0f;
    } else {
        q = make_prim<float>(G, r, m1, m2, E, full);
    }
    m1o = m1f;
    m2o = m2f;
    return q;
}

// Conserved-state component in the flux type (FP32 via the integer pipe).
template <typename FT>
__device__ __forceinline__ FT to_ft(double x) {
    if constexpr (sizeof(FT) == 4) return d2f(x);
    else return x;
}
template <typename FT>
__device__ __forceinline__ FT to_ft(float x) { return (FT)x; }

// Local Lax-Friedrichs flux along axis d from conserved states (double, or
// float in the FP32 form) and their primitives (Davis wave speed, R3);
// returns lambda.
template <typename FT, typename ST>
__device__ __forceinline__ FT llf_prim(const ST uL[4], const Prim<FT> &a, const ST uR[4], const Prim<FT> &b, int d,
                                       FT f[4]) {
    FT vna = d == 0 ? a.v1 : a.v2, vnb = d == 0 ? b.v1 : b.v2;
    FT la = fabs(vna) + a.c, lb = fabs(vnb) + b.c;
    FT lam = speed_max(la, lb);
    FT fa[4], fb[4], ul[4], ur[4];
    for (int v = 0; v < 4; ++v) { ul[v] = to_ft<FT>(uL[v]); ur[v] = to_ft<FT>(uR[v]); }
    phys_flux<FT>(ul[1], ul[2], ul[3], a.p, vna, d, fa);
    phys_flux<FT>(ur[1], ur[2], ur[3], b.p, vnb, d, fb);
    for (int v = 0; v < 4; ++v) f[v] = FT(0.5) * (fa[v] + fb[v]) - FT(0.5) * lam * (ur[v] - ul[v]);
    return lam;
}

// g(0) = gm (rho E - |m|^2/2) - pm rho of a state. With gm = gamma - 1 and
// pm = p_min this is rho (p - p_min); the element pass uses the same form
// scaled by rho_FV (gm = (gamma-1) rho_FV, pm = p_min rho_FV), whose roots are
// the same and which needs no division.
__device__ __forceinline__ double g_zero(double gm, const double u0[4], double pm) {
    return gm * (u0[0] * u0[3] - 0.5 * (u0[1] * u0[1] + u0[2] * u0[2])) - pm * u0[0];
}

// Certifies in FP32 that theta = hi is admissible (rho > 0 and g(hi) >= 0 in
// exact arithmetic) from FP32 inputs that carry at most three roundings each:
// every product and sum below then stays within 17 unit roundings of the sum
// S of the absolute terms, so g_f32 > 4e-6 S implies g(hi) > 0 with a
// fourfold margin, and the FP64 evaluation of the same decision agrees. When
// h is theta rounded to FP32, g(theta) - g(h) is below 2 unit roundings of S,
// well inside the margin, so theta itself is certified. Returns false when it
// cannot decide (near the bound, or magnitudes outside the FP32 range).
__device__ __forceinline__ bool admissible_f32(float gm, const float u0[4], const float a[4], float pm, float c0f,
                                               float h) {
    if (!(c0f > 0.0f) || !(u0[0] > 0.0f) || !(h > 0.0f)) return false;
    float r0 = u0[0], m1 = u0[1], m2 = u0[2], E0 = u0[3];
    float ar = a[0], am1 = a[1], am2 = a[2], aE = a[3];
    float t1 = r0 * aE, t2 = ar * E0, t3 = m1 * am1, t4 = m2 * am2, t5 = pm * ar;
    float c1 = gm * (t1 + t2 - t3 - t4) - t5;
    float s1 = gm * (fabsf(t1) + fabsf(t2) + fabsf(t3) + fabsf(t4)) + fabsf(t5);
    float q1 = ar * aE, q2 = am1 * am1 + am2 * am2;
    float c2 = gm * (q1 - 0.5f * q2);
    float s2 = gm * (fabsf(q1) + 0.5f * q2);
    float S = fabsf(c0f) + h * (s1 + h * s2);
    if (!(S > 1e-30f) || !(S < 1e30f)) return false;
    float gh = c0f + h * (c1 + h * c2);
    if (!(gh > 4e-6f * S)) return false;
    float rh = r0 + h * ar;
    return rh > 4e-6f * (r0 + h * fabsf(ar));
}

__device__ __forceinline__ bool admissible_f32(double gm, const double u0[4], const double a[4], double pm,
                                               double c0, double hi) {
    if (!(c0 > 0.0) || !(u0[0] > 0.0) || !(hi > 0.0)) return false;
    float uf[4] = {d2f(u0[0]), d2f(u0[1]), d2f(u0[2]), d2f(u0[3])};
    float af[4] = {d2f(a[0]), d2f(a[1]), d2f(a[2]), d2f(a[3])};
    return admissible_f32(d2f(gm), uf, af, d2f(pm), d2f(c0), d2f(hi));
}

// Reading R8: largest theta in [0, hi] such that u0 + theta a has rho > 0 and
// p >= p_min; the admissible set is convex so the feasible thetas form an
// interval [0, theta*]. g(theta) = gm (rho E - |m|^2/2) - pm rho with
// (gm, pm) = (gamma-1, p_min) or both scaled by the same positive factor
// (see g_zero); c0 = g(0); gm1 = gamma - 1, so p_min = pm gm1 / gm.
__device__ __forceinline__ double theta_max(double gm1, const double u0[4], const double a[4], double gm, double pm,
                                            double c0, double hi) {
    if (!(hi > 0.0)) return 0.0;
    if (!(c0 > 0.0) || !(u0[0] > 0.0)) return 0.0;
    if (admissible_f32(gm, u0, a, pm, c0, hi)) return hi;
    double c1 = gm * (u0[0] * a[3] + a[0] * u0[3] - (u0[1] * a[1] + u0[2] * a[2])) - pm * a[0];
    double c2 = gm * (a[0] * a[3] - 0.5 * (a[1] * a[1] + a[2] * a[2]));
    double rho_hi = u0[0] + hi * a[0];
    double g_hi = c0 + hi * (c1 + hi * c2);
    if (rho_hi > 0.0 && g_hi >= 0.0) return hi;
    double root = INFINITY;
    if (c2 == 0.0) {
        if (c1 < 0.0) root = -c0 / c1;
    } else {
        double disc = c1 * c1 - 4.0 * c2 * c0;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            double q = -0.5 * (c1 + (c1 >= 0.0 ? sq : -sq));
            double r1 = q / c2, r2 = c0 / q;
            if (r1 > 0.0 && r1 < root) root = r1;
            if (r2 > 0.0 && r2 < root) root = r2;
        }
    }
    double th = root < hi ? root * (1.0 - 1e-12) : hi;
    if (a[0] < 0.0) {
        double tr = -u0[0] / a[0];
        if (th >= tr) th = 0.5 * tr;
    }
    if (!(th > 0.0)) return 0.0;
    const double pmin = pm * gm1 / gm;
    for (int it = 0; it < 4; ++it) {
        double v0 = u0[0] + th * a[0], v1 = u0[1] + th * a[1], v2 = u0[2] + th * a[2], v3 = u0[3] + th * a[3];
        if (v0 > 0.0 && pressure_d(gm1, v0, v1, v2, v3) >= pmin * (1.0 - 1e-13)) return th;
        th *= 0.5;
    }
    return 0.0;
}

// Ghost state across boundary side s (readings R4, R24). in: interior
// conserved state at the face node, (x, y): its coordinates, t: time.
__device__ __forceinline__ void ghost_state(const SimInfo &si, int s, const double in[4], double x, double y,
                                            double t, double gst[4]) {
    int kind = si.bc[s];
    const double *dir = nullptr;
    if (kind == BC_JET) {
        // inflow band |y| <= 0.05 on -x, ambient state elsewhere on the x sides
        if (s == 0) dir = fabs(y) <= 0.05 ? si.dmr_post : si.dmr_pre;
        else if (s == 1) dir = si.dmr_pre;
        kind = dir ? BC_DIRICHLET : BC_OUTFLOW;
    } else if (kind == BC_DMR) {
        if (s == 0) dir = si.dmr_post;
        else if (s == 1) kind = BC_OUTFLOW;
        else if (s == 2) { if (x < 1.0 / 6.0) dir = si.dmr_post; else kind = BC_WALL; }
        else dir = (x < 1.0 / 6.0 + (si.y1 + 20.0 * t) / sqrt(3.0)) ? si.dmr_post : si.dmr_pre;
        if (dir) kind = BC_DIRICHLET;
    } else if (kind == BC_DIRICHLET) {
        dir = si.bc_cons[s];
    }
    if (kind == BC_WALL) {
        double nx = s == 0 ? -1.0 : (s == 1 ? 1.0 : 0.0), ny = s == 2 ? -1.0 : (s == 3 ? 1.0 : 0.0);
        double mn = in[1] * nx + in[2] * ny;
        gst[0] = in[0]; gst[1] = in[1] - 2.0 * mn * nx; gst[2] = in[2] - 2.0 * mn * ny; gst[3] = in[3];
    } else if (kind == BC_DIRICHLET) {
        for (int v = 0; v < 4; ++v) gst[v] = dir[v];
    } else {
        for (int v = 0; v < 4; ++v) gst[v] = in[v];
    }
}

// local face-node coordinates (i, j) of face index t on side s
template <int NP>
__device__ __forceinline__ int face_node(int s, int t) {
    int i = s == 0 ? 0 : (s == 1 ? NP - 1 : t);
    int j = s == 2 ? 0 : (s == 3 ? NP - 1 : t);
    return j * NP + i;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

}  // namespace idp
