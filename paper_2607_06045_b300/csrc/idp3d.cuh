// idp3d.cuh -- the IDP-limited LGL-DGSEM stage for the 3D Euler equations
// (d = 3 of arXiv 2607.06045, Sec. 2) on 2:1-balanced Cartesian octrees of
// hexahedra: one fused element kernel per stage and the IDP time step (the
// mortar kernels of the nonconforming faces are in idp3d_mortar.cuh).
//
// The stage is the 2D one with the third direction (Sec. 2.1-2.3 for
// d = 3): Ranocha's two-point fluxes along x, y and z within each element,
// the telescoped high-order subcell fluxes (Eq. fluxdifferencingform), the
// LLF faces, the low-order subcell fluxes with the graph viscosity
// (Eq. LowOrderScheme_globalIndices in flux form), bar-state density bounds
// and positivity (Eqs. Bounds_Positivity, Bounds_Barstates), Zalesak density
// limiting and the pressure factor with Gamma = 2d = 6, then the SSP-RK3
// combination. State u[5][K][N+1]^3 FP64 (rho, rho v1, rho v2, rho v3, rho e),
// x index fastest, leaves in the caller's order. At a mortar side the element
// takes its low-order face terms and bar-state ranges from the mortar's slots
// and hands the node's volume-corrected state to the mortar kernels, which
// finish it.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "idp_bits.cuh"
#include "idp_fastmath.cuh"

namespace idp3 {

constexpr int NV = 5;
constexpr int NPMAX3 = 8;
constexpr double kTol3 = 1e-14;       // R15
constexpr double kViol3 = 1e-13;      // R13
constexpr double kGamma3 = 6.0;       // Gamma = 2d (Sec. 2.3)
enum : int { B_PERIODIC = 0, B_WALL = 1, B_DIRICHLET = 2, B_OUTFLOW = 3 };
enum : unsigned { S_BAD_INPUT = 1u, S_VIOLATION = 2u };

// Mortars (a face between a leaf and four finer ones, 2 x 2 small faces p =
// p1 + 2 p2 by their offsets along the face's tangential directions (d+1) mod
// 3 and (d+2) mod 3). Each mortar has Q = 5 (N+1)^2 slots, one per node on
// it: the large face's nodes, then each small face's, node t = a + (N+1) b
// of a face with a along (d+1) mod 3. A "mortar node" is a node on at least
// one mortar (up to three); the element kernel hands it off and the mortar
// kernels finish it.
struct Mort3 {
    int M, S, MN;                    // mortars, slots (M Q), mortar nodes
    const int *info;                 // [M][7]: d, large element, large on the low side, small elements p = 0..3
    double *chi, *clo;               // [NV][S]: high- and low-order contribution to the node's mass-weighted residual
    double *rbmin, *rbmax, *dsum;    // [S]: bar-state density range over the slot's pairs and their sum of 2 d_ij
    int *bad;                        // [M]: the interpolated states left the admissible set (R16)
    double *ell;                     // [M]: the mortar's factor l_S
    const int *slot_mn;              // [S]: the slot's mortar node
    const int *mn_node;              // [MN]: its global node (e (N+1)^3 + n)
    const int *mn_slot;              // [3][MN]: its slots in mortar order, -1 past n_i
    const int *mn_cnt;               // [MN]: n_i, its number of mortars
    double *h_uvol, *h_res;          // [NV][MN]: u_vol and the residual before the mortar corrections (mass-weighted)
    double *h_b;                     // [5][MN]: rho_min, rho_max, p_min, rho_FV, 1 / m
};

// The mesh: K leaves, leaf e at level lev[e] with extents (dx, dy, dz) 2^-lev
// (dx, dy, dz of a level-0 cell); per side (-x, +x, -y, +y, -z, +z) of each
// leaf nbr[6 e + s]: the conforming neighbour (>= 0), -1 at a boundary, or
// -2 - (the first slot of the mortar face); boundary kinds per side of the
// box and the conserved Dirichlet states.
struct Grid3 {
    int nx, ny, nz, K;
    double dx, dy, dz;
    int bc[6];
    double bc_cons[6][NV];
    const int *nbr;
    const signed char *lev;
    const idp::LogTab *lg;           // table of the FP64 logarithm
    const double *ind;               // shock indicator: V^-1 [(N+1)^2] row-major, then T and s
    Mort3 mort;
};

// extents of leaf e
__device__ __forceinline__ void extents3(const Grid3 &G, int e, double *h) {
    const double sc = __int_as_float((127 - (int)G.lev[e]) << 23);   // 2^-lev, exact
    h[0] = G.dx * sc; h[1] = G.dy * sc; h[2] = G.dz * sc;
}

// LGL nodes and weights, Sbar (Sec. 2.1), 1 / w
struct Ops3 {
    double xi[NPMAX3], w[NPMAX3], iw[NPMAX3], S[NPMAX3][NPMAX3];
};

// statistics of the limited stages (atomics)
struct Stats3 {
    double alpha_m;                 // sum of m (1 - min factor at the node)
    unsigned long long n_active;    // nodes with a factor below one
    unsigned long long n_vrho, n_vp, n_nonpos;
    unsigned long long min_rho_bits, min_p_bits;
    double alpha_mort_a, mort_area;          // sum over mortars of area (1 - l_S), of area
    unsigned long long n_mort, n_mort_fallback;   // mortars with l_S < 1; with an inadmissible interpolation
};

struct Stage3 {
    const double *u;     // stage input u^(s)
    const double *un;    // u^n (stage combination)
    double *out;         // rhs (mode 0) or u^(s+1) (mode 1)
    double dt_host;      // time step when dtmin is null
    const unsigned long long *dtmin;   // device minimum of m_i / sum 2 d_ij (bits); dt = cfl * value
    double cfl;
    int mode;            // 0: residual per unit mass, 1: stage state
    int comb;            // 0: u~, 1: 3/4 u^n + 1/4 u~, 2: 1/3 u^n + 2/3 u~
    int limiting;        // 0 none (the high-order residual), 1 positivity, 2 local, 3 combined
    int collect;         // statistics on
    double beta, gamma;
    Stats3 *stats;
    unsigned *status;
    double *aind;        // combined limiting: per element shock indicator (written by the element kernel)
};

// a statistic's running minimum (positive doubles order like their bits)
__device__ __forceinline__ void stat_min(unsigned long long *slot, double v) {
    if (v > 0.0 && v < INFINITY) atomicMin(slot, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double stage_dt3(const Stage3 &A) {
    return A.dtmin ? A.cfl * __longlong_as_double((long long)*A.dtmin) : A.dt_host;
}

__device__ __forceinline__ double pres3(double g, const double *u) {
    return (g - 1.0) * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * idp::fast_rcp(u[0]));
}

// R8 with 5 variables: the largest theta <= hi with rho(u0 + theta a) > 0
// and p(u0 + theta a) >= pmin (closed-form root of the quadratic rho p -
// pmin rho, aimed 1e-12 inside, verified, halved at most four times)
__device__ __forceinline__ double theta3(double g, const double *u0, const double *a, double pmin, double hi) {
    if (!(hi > 0.0)) return 0.0;
    const double gm1 = g - 1.0;
    const double m0 = u0[1] * u0[1] + u0[2] * u0[2] + u0[3] * u0[3];
    const double ma = u0[1] * a[1] + u0[2] * a[2] + u0[3] * a[3];
    const double aa = a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
    const double c0 = gm1 * (u0[0] * u0[4] - 0.5 * m0) - pmin * u0[0];
    const double c1 = gm1 * (u0[0] * a[4] + a[0] * u0[4] - ma) - pmin * a[0];
    const double c2 = gm1 * (a[0] * a[4] - 0.5 * aa);
    if (!(u0[0] > 0.0) || !(c0 > 0.0)) return 0.0;
    const double rho_hi = u0[0] + hi * a[0], g_hi = c0 + hi * (c1 + hi * c2);
    if (rho_hi > 0.0 && g_hi >= 0.0) return hi;
    double root = INFINITY;
    if (c2 == 0.0) {
        if (c1 < 0.0) root = -c0 / c1;
    } else {
        const double disc = c1 * c1 - 4.0 * c2 * c0;
        if (disc >= 0.0) {
            const double sq = sqrt(disc);
            const double q = -0.5 * (c1 + (c1 >= 0.0 ? sq : -sq));
            const double r1 = q / c2, r2 = c0 / q;
            if (r1 > 0.0 && r1 < root) root = r1;
            if (r2 > 0.0 && r2 < root) root = r2;
        }
    }
    double th = root < hi ? root * (1.0 - 1e-12) : hi;
    if (a[0] < 0.0) {
        const double tr = -u0[0] / a[0];
        if (th >= tr) th = 0.5 * tr;
    }
    if (!(th > 0.0)) return 0.0;
    for (int it = 0; it < 4; ++it) {
        double v[NV];
        for (int k = 0; k < NV; ++k) v[k] = u0[k] + th * a[k];
        if (v[0] > 0.0 && pres3(g, v) >= pmin * (1.0 - 1e-13)) return th;
        th *= 0.5;
    }
    return 0.0;
}

// Certifies in FP32 that theta = h is admissible for u0 + theta a (rho > 0 and
// g(h) = (gamma-1)(rho E - |m|^2/2) - pmin rho >= 0 in exact arithmetic) from
// FP32 inputs that carry at most three roundings each (u_FV rounded once,
// a = Gamma dt/m A from two rounded factors, c0 = g(0) formed in FP64 and
// rounded): every FP32 product and sum below stays within 20 unit roundings
// (2^-24) of the sum S of the absolute terms, so g_f32 > 4e-6 S (67 unit
// roundings) implies g(h) > 0 with a threefold margin, and the same holds for
// the density. Returns false when it cannot decide (near the bound, or
// magnitudes outside the FP32 range); the FP64 solve then runs.
__device__ __forceinline__ bool admissible3_f32f(float gm, const float *u0, const float *a, float pm, float c0f,
                                                 float hf) {
    if (!(c0f > 0.0f) || !(u0[0] > 0.0f) || !(hf > 0.0f)) return false;
    const float t1 = u0[0] * a[4], t2 = a[0] * u0[4], t5 = pm * a[0];
    float tm = 0.0f, sm = 0.0f, q2 = 0.0f;
    for (int c = 1; c <= 3; ++c) {
        const float t = u0[c] * a[c];
        tm += t;
        sm += fabsf(t);
        q2 += a[c] * a[c];
    }
    const float c1 = gm * (t1 + t2 - tm) - t5;
    const float s1 = gm * (fabsf(t1) + fabsf(t2) + sm) + fabsf(t5);
    const float q1 = a[0] * a[4];
    const float c2 = gm * (q1 - 0.5f * q2);
    const float s2 = gm * (fabsf(q1) + 0.5f * q2);
    const float S = fabsf(c0f) + hf * (s1 + hf * s2);
    if (!(S > 1e-30f) || !(S < 1e30f)) return false;
    const float gh = c0f + hf * (c1 + hf * c2);
    if (!(gh > 4e-6f * S)) return false;
    const float rh = u0[0] + hf * a[0];
    return rh > 4e-6f * (u0[0] + hf * fabsf(a[0]));
}

// the ghost state across boundary side s (R4: wall, Dirichlet, outflow)
__device__ __forceinline__ void ghost3(const Grid3 &G, int s, const double *in, double *q) {
    const int kind = G.bc[s];
    if (kind == B_DIRICHLET) {
        for (int v = 0; v < NV; ++v) q[v] = G.bc_cons[s][v];
    } else {
        for (int v = 0; v < NV; ++v) q[v] = in[v];
        if (kind == B_WALL) q[1 + s / 2] = -in[1 + s / 2];
    }
}

template <int NP>
struct El3 {
    static constexpr int N = NP - 1, NR = NP * NP, NN = NP * NP * NP, NPAIR = NP * (NP - 1) / 2;
    static constexpr int NIF = 3 * NR * N, NF = 6 * NR;
};

// node index within an element of position a along d in row r (r = t1 + NP t2,
// t1, t2 the other two indices in cyclic order d+1, d+2)
template <int NP>
__device__ __forceinline__ int node_of(int d, int r, int a) {
    const int t1 = r % NP, t2 = r / NP;
    int idx[3];
    idx[d] = a; idx[(d + 1) % 3] = t1; idx[(d + 2) % 3] = t2;
    return (idx[2] * NP + idx[1]) * NP + idx[0];
}

// per-node flux data of the element kernel: in the FP64 path v1/2, v2/2,
// v3/2, p/2, ln rho, (ln beta')/2, beta'/2 with beta' = (gamma - 1) rho / p =
// rho / (rho e), and |v_d| + c (the halves and beta' are exact or
// rounding-level rescalings that fold the means' factors 1/2 and 2 and the
// 1/(gamma - 1) of the two-point flux into the node data); in the FP32 form the state rounded to FP32, v1, v2, v3, p,
// beta = rho / p and |v_d| + c in FP32
template <int NP, bool F32>
struct Node3 {
    static constexpr int NN = NP * NP * NP;
    double pr[7][NN];
    double lam[3][NN];
};
template <int NP>
struct Node3<NP, true> {
    static constexpr int NN = NP * NP * NP;
    float uf[NV][NN];
    float pr[5][NN];
    float lam[3][NN];
};

// shared memory of one element; arrays whose lifetimes do not overlap share
// storage (phases P0..P5 of k_element3d). FT: the flux type (float in the
// FP32 form): the per-node flux data, pair fluxes, outside primitives and
// low-order subcell fluxes; everything else is FP64.
template <int NP, typename FT = double>
struct Sm3 {
    using E = El3<NP>;
    static constexpr int NN = E::NN, NR = E::NR, NIF = E::NIF, NPAIR = E::NPAIR;
    union {
        double u[NV][NN];      // P0 - P2: the stage input
        double rfv[NV][NN];    // P2 - P5: low-order residual (each node overwrites only its own u)
    };
    union {
        struct {                          // P0 - P1
            Node3<NP, sizeof(FT) == 4> nd;
            FT outp[6][NR][3];            // outside states' normal velocity, pressure, wave speed
        };
        struct {                          // P2 - P5
            double ufv[NV][NN];           // the low-order update u_FV
            double rmin[NN], rmax[NN], pmin[NN];
            double im[NN];                // 1 / m
            // FP32 copies for the certificates (P2 - P4): u_FV, Gamma dt / m,
            // p_min and g(0) = (gamma-1)(rho E - |m|^2/2) - p_min rho at u_FV
            float ufvf[NV][NN], gdtf[NN], pmf[NN], c0f[NN];
        };
    };
    struct {                      // P2b - P5
        double Rp[NN], Rm[NN];       // Zalesak factors (P3 - P4)
        double ell[NIF];             // interface factors (P4 - P5)
        unsigned char ex[NIF];       // R15 exemption (P2b - P4)
    };
    union {
        FT pair[3][NR][NPAIR][NV];       // P1 - P2b: two-point fluxes of every row
        double iscr[2][NN];               // P0b: the combined limiting's modal transform
        struct {                          // P3 - P4: interface ends whose FP32 certificate
            unsigned short pend[NIF];     // did not decide (interface id | end << 15), for
            int npend;                    // the FP64 solve by whole warps
            double Rm2[NN];               // combined limiting: R- of the positivity bounds
        };
    };
    union {
        struct {                     // P0 - P2
            union {
                double outs[6][NR][NV];   // P0 - P1b: outside states of the six faces
                double ff[6][NR][NV];     // P1b - P2: face fluxes, mass-weighted, along +d (each
            };                            // P1b item reads its outside state, then writes its flux)
            double fbl[6][NR];       // bar-state density range across the face (one value
            double fbh[6][NR];       // at a conforming face, a mortar slot's range at a mortar)
            double ibar[NIF];        // bar-state density of the interior interfaces
        };
        double A[NIF][NV];           // P2b - P5: antidiffusive fluxes (mass-weighted)
    };
    FT fvf[NIF][NV];           // P1 - P2b: low-order subcell fluxes, mass-weighted, along +d
    double q[3], J, iJ;        // quarter face areas, dx dy dz / 8 and its inverse
    double aind;               // combined limiting: the element's shock indicator
    int nb[6];                 // the sides' neighbour entries (Grid3::nbr)
};

// a flux-type value in FP64 (FP32 converted on the integer pipe)
__device__ __forceinline__ double to_d3(double x) { return x; }
__device__ __forceinline__ double to_d3(float x) { return idp::f2d(x); }

// FP32 primitives of a state (the FP32 form): the state rounded to FP32 (on
// the integer pipe), v, p and 1 / rho. When E - |m|^2/2rho keeps at least an
// eighth of E the pressure is formed in FP32 (within 2e-6 of the rounded
// state's and positive for sure, as in 2D); otherwise v, p and 1/rho are
// formed in FP64 and rounded. False for a non-admissible state.
__device__ __forceinline__ bool prim3_f32(double gm1, const double *u, float *uf, float *v, float &p, float &ir) {
    for (int k = 0; k < NV; ++k) uf[k] = idp::d2f(u[k]);
    ir = __frcp_rn(uf[0]);
    for (int c = 0; c < 3; ++c) v[c] = __fmul_rn(uf[1 + c], ir);
    const float ke = 0.5f * (uf[1] * v[0] + uf[2] * v[1] + uf[3] * v[2]);
    const float pe = uf[4] - ke;
    if (uf[0] > 0.0f && uf[4] > 0.0f && pe >= 0.125f * uf[4]) {
        p = idp::d2f(gm1) * pe;
        return true;
    }
    const double ird = idp::fast_rcp(u[0]);
    double vd[3];
    for (int c = 0; c < 3; ++c) vd[c] = u[1 + c] * ird;
    const double pd = gm1 * (u[4] - 0.5 * (u[1] * vd[0] + u[2] * vd[1] + u[3] * vd[2]));
    for (int c = 0; c < 3; ++c) v[c] = idp::d2f(vd[c]);
    p = idp::d2f(pd);
    ir = idp::d2f(ird);
    return idp::dpos(u[0]) && idp::dpos(pd) && p > 0.0f;
}

// both logarithmic means of a pair in FP32 (the FP32 form): logarithms of
// the ratios, the Ismail-Roe series where ((a - b)/(a + b))^2 < 1e-2 (its
// truncation is below FP32 rounding there), one reciprocal for both
__device__ __forceinline__ void log_means3_f32(float ra, float rb, float ba, float bb, float &rho_ln, float &ibeta) {
    const float dr = ra - rb, sr = ra + rb, db = ba - bb, sb = ba + bb;
    const bool nr = dr * dr < 1e-2f * (sr * sr), nb = db * db < 1e-2f * (sb * sb);
    const float lr = nr ? 0.0f : logf(__fdiv_rn(ra, rb)), lb = nb ? 0.0f : logf(__fdiv_rn(ba, bb));
    const float Xr = nr ? sr : lr, Xb = nb ? sb : db;
    const float R = __frcp_rn(Xr * Xb);
    const float ixr = Xb * R, ixb = Xr * R;
    if (nr) {
        const float f = dr * ixr, uu = f * f;
        rho_ln = 0.5f * sr * (1.0f - uu * (1.0f / 3.0f + uu * (4.0f / 45.0f + uu * (44.0f / 945.0f))));
    } else {
        rho_ln = dr * ixr;
    }
    if (nb) {
        const float f = db * ixb, uu = f * f;
        ibeta = 2.0f * ixb * (1.0f + uu * (1.0f / 3.0f + uu * (1.0f / 5.0f + uu * (1.0f / 7.0f))));
    } else {
        ibeta = lb * ixb;
    }
}

// threads of a block of EPB elements: one per node, rounded up to whole warps
template <int NP, int EPB>
struct Launch3 {
    static constexpr int items = EPB * NP * NP * NP, threads = (items + 31) / 32 * 32;
};

// Both logarithmic means of a pair (R2) from the node logarithms, with one
// reciprocal: rho_ln = (ra - rb) / (ln ra - ln rb) and 1 / beta_ln = (ln ba -
// ln bb) / (ba - bb), each by the Ismail-Roe series where ((a - b)/(a + b))^2
// <= 1e-4 (the test in FP32, converted on the integer pipe: the two forms
// agree to rounding near the threshold). ba, bb and their logarithms come
// halved (the FP64 node data), which scales the quotient exactly and drops
// the series' factor 2.
__device__ __forceinline__ void log_means3(double ra, double rb, double lra, double lrb, double ba, double bb,
                                           double lba, double lbb, double &rho_ln, double &ibeta) {
    const double dr = ra - rb, sr = ra + rb, db = ba - bb, sb = ba + bb;
    const float drf = idp::d2f(dr), srf = idp::d2f(sr), dbf = idp::d2f(db), sbf = idp::d2f(sb);
    const bool nr = drf * drf <= 1e-4f * (srf * srf), nb = dbf * dbf <= 1e-4f * (sbf * sbf);
    const double Xr = nr ? sr : lra - lrb, Xb = nb ? sb : db;
    const double R = idp::fast_rcp(Xr * Xb);
    const double ixr = Xb * R, ixb = Xr * R;   // 1 / Xr, 1 / Xb
    if (nr) {
        const double f = dr * ixr, u = f * f;
        // sr / (2 F(u)) with 1/F = 1 - u/3 - 4u^2/45 - 44u^3/945
        rho_ln = 0.5 * sr * (1.0 - u * (1.0 / 3.0 + u * (4.0 / 45.0 + u * (44.0 / 945.0))));
    } else {
        rho_ln = dr * ixr;
    }
    if (nb) {
        const double f = db * ixb, u = f * f;
        // 2 F(u) / sb with F = 1 + u/3 + u^2/5 + u^3/7
        ibeta = ixb * (1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0))));
    } else {
        ibeta = (lba - lbb) * ixb;
    }
}

// half the physical flux along d (the mass flux m_d whole) from the state,
// half its velocity along d and half its pressure (the FP64 node data)
__device__ __forceinline__ void flux_h(const double *u, double hv, double hp, int d, double *f) {
    f[0] = u[1 + d];
    f[1] = u[1] * hv + (d == 0 ? hp : 0.0);
    f[2] = u[2] * hv + (d == 1 ? hp : 0.0);
    f[3] = u[3] * hv + (d == 2 ? hp : 0.0);
    f[4] = (u[4] + 2.0 * hp) * hv;
}

// physical flux along d from the state and its velocity along d and pressure
template <typename T>
__device__ __forceinline__ void flux_p(const T *u, T vd, T p, int d, T *f) {
    f[0] = u[1 + d];
    f[1] = u[1] * vd + (d == 0 ? p : T(0));
    f[2] = u[2] * vd + (d == 1 ? p : T(0));
    f[3] = u[3] * vd + (d == 2 ? p : T(0));
    f[4] = (u[4] + p) * vd;
}

// One block of EPB elements, one thread per node; items of each phase are
// spread over the block. Per node, its primitives, logarithms and wave
// speeds are formed once (P0); the pair, face and subcell fluxes take them
// from shared memory. FT = float: the FP32 form (R18): node primitives, the
// two-point, face and subcell fluxes in FP32; bar states, bounds, sums,
// limiting and the stage update in FP64.
template <int NP, int EPB, typename FT>
__global__ void __launch_bounds__(Launch3<NP, EPB>::threads)
k_element3d(Grid3 G, const Ops3 *__restrict__ ops_g, Stage3 A) {
    using E = El3<NP>;
    using SM = Sm3<NP, FT>;
    constexpr bool F32 = sizeof(FT) == 4;
    constexpr int N = E::N, NN = E::NN, NR = E::NR, NPAIR = E::NPAIR, NIF = E::NIF, NT = Launch3<NP, EPB>::threads;
    extern __shared__ __align__(16) unsigned char sm3_raw[];
    SM *S = reinterpret_cast<SM *>(sm3_raw);
    __shared__ Ops3 ops;
    __shared__ float Sf[NP][NP];   // Sbar in FP32 (the FP32 form)
    __shared__ double w3[NN], iw3[NN];   // w_i w_j w_k and its inverse per node of an element
    const int tid = threadIdx.x;
    for (int k = tid; k < (int)(sizeof(Ops3) / sizeof(double)); k += NT)
        reinterpret_cast<double *>(&ops)[k] = reinterpret_cast<const double *>(ops_g)[k];
    for (int k = tid; k < NN; k += NT) {
        const int i = k % NP, j = (k / NP) % NP, l = k / (NP * NP);
        w3[k] = ops_g->w[i] * ops_g->w[j] * ops_g->w[l];
        iw3[k] = (1.0 / ops_g->w[i]) * (1.0 / ops_g->w[j]) * (1.0 / ops_g->w[l]);
    }
    if (F32)
        for (int k = tid; k < NP * NP; k += NT) Sf[k / NP][k % NP] = idp::d2f(ops_g->S[k / NP][k % NP]);
    const size_t KN = (size_t)G.K * NN;
    const double g = A.gamma, gm1 = g - 1.0, igm1 = 1.0 / gm1, hgm1 = 0.5 * gm1, g2 = 2.0 * g;
    const double dt = stage_dt3(A), idt = 1.0 / dt;
    const int e0 = blockIdx.x * EPB;
    const Mort3 &MO = G.mort;
    // ---- P0: state, primitives, logarithms, wave speeds; outside states
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        if (n == 0) {
            double h[3];
            extents3(G, e, h);
            S[le].q[0] = h[1] * h[2] / 4.0; S[le].q[1] = h[0] * h[2] / 4.0; S[le].q[2] = h[0] * h[1] / 4.0;
            S[le].J = h[0] * h[1] * h[2] / 8.0;
            S[le].iJ = 8.0 / (h[0] * h[1] * h[2]);
        }
        double uv[NV];
        for (int v = 0; v < NV; ++v) { uv[v] = A.u[v * KN + (size_t)e * NN + n]; S[le].u[v][n] = uv[v]; }
        auto &nd = S[le].nd;
        if constexpr (F32) {
            float uf[NV], vf[3], pf, irf;
            const bool ok = prim3_f32(gm1, uv, uf, vf, pf, irf);
            for (int v = 0; v < NV; ++v) nd.uf[v][n] = uf[v];
            for (int c = 0; c < 3; ++c) nd.pr[c][n] = vf[c];
            nd.pr[3][n] = pf;
            if (!ok) {
                atomicOr(A.status, S_BAD_INPUT);
                nd.pr[4][n] = 1.0f;
                for (int d = 0; d < 3; ++d) nd.lam[d][n] = 0.0f;
                continue;
            }
            const float c = sqrtf(idp::d2f(g) * pf * irf);
            nd.pr[4][n] = uf[0] * __frcp_rn(pf);
            for (int d = 0; d < 3; ++d) nd.lam[d][n] = fabsf(vf[d]) + c;
        } else {
            // halves of v and p; rho e = E - |m|^2 / 2 rho = p / (gamma - 1)
            const double ir = idp::fast_rcp(uv[0]), hir = 0.5 * ir;
            const double h1 = uv[1] * hir, h2 = uv[2] * hir, h3 = uv[3] * hir;
            const double re = uv[4] - (uv[1] * h1 + uv[2] * h2 + uv[3] * h3);
            const double hp = hgm1 * re;
            nd.pr[0][n] = h1; nd.pr[1][n] = h2; nd.pr[2][n] = h3; nd.pr[3][n] = hp;
            if (!(uv[0] > 0.0) || !(re > 0.0)) {
                atomicOr(A.status, S_BAD_INPUT);
                nd.pr[4][n] = 0.0; nd.pr[5][n] = 0.0; nd.pr[6][n] = 1.0;
                for (int d = 0; d < 3; ++d) nd.lam[d][n] = 0.0;
                continue;
            }
            const double c = idp::fast_sqrt(g2 * hp * ir);
            const double bet = uv[0] * idp::fast_rcp(re);
            nd.pr[4][n] = idp::fast_log(uv[0], G.lg);
            nd.pr[5][n] = 0.5 * idp::fast_log(bet, G.lg);
            nd.pr[6][n] = 0.5 * bet;
            nd.lam[0][n] = 2.0 * fabs(h1) + c; nd.lam[1][n] = 2.0 * fabs(h2) + c; nd.lam[2][n] = 2.0 * fabs(h3) + c;
        }
    }
    for (int k = tid; k < EPB * 6 * NR; k += NT) {
        const int le = k / (6 * NR), r0 = k - le * 6 * NR, s = r0 / NR, t = r0 - s * NR, e = e0 + le;
        if (e >= G.K) continue;
        const int d = s / 2, side = s & 1;
        const int nb = G.nbr[6 * e + s];
        if (t == 0) S[le].nb[s] = nb;
        if (nb < -1) continue;   // a mortar: its slots carry the face terms
        const int nin = node_of<NP>(d, t, side ? N : 0);
        double o[NV];
        if (nb >= 0) {
            const int nout = node_of<NP>(d, t, side ? 0 : N);
            for (int v = 0; v < NV; ++v) o[v] = A.u[v * KN + (size_t)nb * NN + nout];
        } else {
            double in[NV];
            for (int v = 0; v < NV; ++v) in[v] = A.u[v * KN + (size_t)e * NN + nin];
            ghost3(G, s, in, o);
        }
        for (int v = 0; v < NV; ++v) S[le].outs[s][t][v] = o[v];
        // the outside state's normal velocity, pressure and wave speed
        if constexpr (F32) {
            float of[NV], vf[3], pf, irf;
            const bool ok = prim3_f32(gm1, o, of, vf, pf, irf);
            S[le].outp[s][t][0] = vf[d];
            S[le].outp[s][t][1] = pf;
            S[le].outp[s][t][2] = ok ? fabsf(vf[d]) + sqrtf(idp::d2f(g) * pf * irf) : 0.0f;
        } else {
            // halves of v_d and p, as the node data
            const double ir = idp::fast_rcp(o[0]), hir = 0.5 * ir;
            const double hvd = o[1 + d] * hir;
            const double re = o[4] - (o[1] * o[1] + o[2] * o[2] + o[3] * o[3]) * hir;
            const double hpo = hgm1 * re;
            S[le].outp[s][t][0] = hvd;
            S[le].outp[s][t][1] = hpo;
            S[le].outp[s][t][2] = (o[0] > 0.0 && re > 0.0) ? 2.0 * fabs(hvd) + idp::fast_sqrt(g2 * hpo * ir) : 0.0;
        }
    }
    __syncthreads();
    const bool comb = A.limiting == 3;
    if (comb) {
        // ---- P0b: the shock indicator of each element (Sec. 3.5, reading R34):
        // the pressure's modes in the orthonormal Legendre tensor basis, one
        // direction per pass, then the energies of the top two mode shells
        const double *Vi = G.ind;
        for (int k = tid; k < EPB * NN; k += NT) {
            const int le = k / NN, n = k - le * NN;
            if (e0 + le >= G.K) continue;
            const double r = S[le].u[0][n], m1 = S[le].u[1][n], m2 = S[le].u[2][n], m3 = S[le].u[3][n];
            S[le].iscr[0][n] = gm1 * (S[le].u[4][n] - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) * idp::fast_rcp(r));
        }
        for (int pass = 0; pass < 3; ++pass) {
            __syncthreads();
            const int src = pass & 1, dst = src ^ 1, stride = pass == 0 ? 1 : (pass == 1 ? NP : NP * NP);
            for (int k = tid; k < EPB * NN; k += NT) {
                const int le = k / NN, n = k - le * NN;
                if (e0 + le >= G.K) continue;
                const int mi = (n / stride) % NP, base = n - mi * stride;
                double acc = 0.0;
                for (int i = 0; i < NP; ++i) acc += Vi[mi * NP + i] * S[le].iscr[src][base + i * stride];
                S[le].iscr[dst][n] = acc;
            }
        }
        __syncthreads();
        for (int le = tid; le < EPB; le += NT) {
            if (e0 + le >= G.K) continue;
            double e0s = 0.0, e1s = 0.0, e2s = 0.0;
            for (int n = 0; n < NN; ++n) {
                const int i = n % NP, j = (n / NP) % NP, k = n / (NP * NP);
                const int top = max(max(i, j), k);
                const double m2 = S[le].iscr[1][n] * S[le].iscr[1][n];
                if (top == N) e1s += m2;
                else if (top == N - 1) e2s += m2;
                else e0s += m2;
            }
            double E = 0.0;
            if (e0s + e1s + e2s > 0.0) E = e1s / (e0s + e1s + e2s);
            if (e0s + e2s > 0.0 && e2s / (e0s + e2s) > E) E = e2s / (e0s + e2s);
            const double T = Vi[NP * NP], sh = Vi[NP * NP + 1];
            double a = 1.0 / (1.0 + exp(-sh / T * (E - T)));
            if (a < 1e-3) a = 0.0;
            if (a > 1.0 - 1e-3) a = 1.0;
            S[le].aind = a;
            A.aind[e0 + le] = a;
        }
        __syncthreads();
    }
    // ---- P1a: two-point fluxes of every row, each unordered pair once
    for (int k = tid; k < EPB * 3 * NR * NPAIR; k += NT) {
        const int le = k / (3 * NR * NPAIR), r0 = k - le * 3 * NR * NPAIR;
        const int d = r0 / (NR * NPAIR), r1 = r0 - d * NR * NPAIR, r = r1 / NPAIR, pp = r1 - r * NPAIR;
        if (e0 + le >= G.K) continue;
        // pair index -> (a, b), a < b, a-major
        int a = 0, rem = pp;
        while (rem >= N - a) { rem -= N - a; ++a; }
        const int b = a + 1 + rem;
        const int na = node_of<NP>(d, r, a), nb = node_of<NP>(d, r, b);
        const SM &X = S[le];
        FT rho_ln, iba, igm;
        if constexpr (F32) {
            log_means3_f32(X.nd.uf[0][na], X.nd.uf[0][nb], X.nd.pr[4][na], X.nd.pr[4][nb], rho_ln, iba);
            igm = idp::d2f(igm1);
        } else {
            log_means3(X.u[0][na], X.u[0][nb], X.nd.pr[4][na], X.nd.pr[4][nb], X.nd.pr[6][na], X.nd.pr[6][nb],
                       X.nd.pr[5][na], X.nd.pr[5][nb], rho_ln, iba);
            igm = igm1;
        }
        const FT pa = X.nd.pr[3][na], pb = X.nd.pr[3][nb];
        FT va[3], vb[3];
        for (int cc = 0; cc < 3; ++cc) { va[cc] = X.nd.pr[cc][na]; vb[cc] = X.nd.pr[cc][nb]; }
        // R1 (Ranocha) along d
        FT f[NV];
        if constexpr (F32) {
            const FT h = FT(0.5);
            const FT vdot = va[0] * vb[0] + va[1] * vb[1] + va[2] * vb[2];
            const FT fr = rho_ln * h * (va[d] + vb[d]);
            f[0] = fr;
            for (int cc = 0; cc < 3; ++cc) f[1 + cc] = fr * h * (va[cc] + vb[cc]) + (cc == d ? h * (pa + pb) : FT(0));
            f[4] = fr * (h * vdot + iba * igm) + h * (pa * vb[d] + pb * va[d]);
        } else {
            // halves of v and p: the means are sums; iba is already 1 / ((gamma - 1) beta_ln)
            (void)igm;
            const double hdot = va[0] * vb[0] + va[1] * vb[1] + va[2] * vb[2];
            const double fr = rho_ln * (va[d] + vb[d]);
            f[0] = fr;
            for (int cc = 0; cc < 3; ++cc) f[1 + cc] = fr * (va[cc] + vb[cc]) + (cc == d ? pa + pb : 0.0);
            f[4] = fr * (2.0 * hdot + iba) + 2.0 * (pa * vb[d] + pb * va[d]);
        }
        for (int v = 0; v < NV; ++v) S[le].pair[d][r][pp][v] = f[v];
    }
    // ---- P1b: LLF faces (mass-weighted, along +d) and their bar-state densities
    for (int k = tid; k < EPB * 6 * NR; k += NT) {
        const int le = k / (6 * NR), r0 = k - le * 6 * NR, s = r0 / NR, t = r0 - s * NR;
        if (e0 + le >= G.K) continue;
        const int d = s / 2, side = s & 1;
        const int nbv = S[le].nb[s];
        if (nbv < -1) {
            // mortar: the slot's low-order contribution to the node (ff enters
            // a low face with +, a high face with -) and its bar-state range
            const int slot = -2 - nbv + t;
            for (int v = 0; v < NV; ++v) {
                const double c = MO.clo[(size_t)v * MO.S + slot];
                S[le].ff[s][t][v] = side ? -c : c;
            }
            S[le].fbl[s][t] = MO.rbmin[slot];
            S[le].fbh[s][t] = MO.rbmax[slot];
            continue;
        }
        const int nin = node_of<NP>(d, t, side ? N : 0);
        const SM &X = S[le];
        const double *q = X.q;
        const double wt = ops.w[t % NP] * ops.w[t / NP], cw = wt * q[d];
        FT ui[NV], uo[NV], fi[NV], fo[NV];
        for (int v = 0; v < NV; ++v) {
            if constexpr (F32) { ui[v] = X.nd.uf[v][nin]; uo[v] = idp::d2f(X.outs[s][t][v]); }
            else { ui[v] = X.u[v][nin]; uo[v] = X.outs[s][t][v]; }
        }
        FT lam;
        if constexpr (F32) {
            flux_p<FT>(ui, X.nd.pr[d][nin], X.nd.pr[3][nin], d, fi);
            flux_p<FT>(uo, X.outp[s][t][0], X.outp[s][t][1], d, fo);
            lam = fmaxf(X.nd.lam[d][nin], X.outp[s][t][2]);
        } else {
            // half fluxes (the mass flux whole) from the halves of v_d and p
            flux_h(ui, X.nd.pr[d][nin], X.nd.pr[3][nin], d, fi);
            flux_h(uo, X.outp[s][t][0], X.outp[s][t][1], d, fo);
            lam = idp::dmax(X.nd.lam[d][nin], X.outp[s][t][2]);
        }
        const FT cwf = (FT)(F32 ? (double)idp::d2f(cw) : cw);
        // left state first: the outside is on the left of a low face
        const FT *uL = side ? ui : uo, *uR = side ? uo : ui, *fL = side ? fi : fo, *fR = side ? fo : fi;
        const FT hl = FT(0.5) * lam;
        for (int v = 0; v < NV; ++v) {
            const FT fm = (F32 || v == 0) ? FT(0.5) * (fL[v] + fR[v]) : fL[v] + fR[v];
            S[le].ff[s][t][v] = to_d3(cwf * (fm - hl * (uR[v] - uL[v])));
        }
        // ubar = (u_i + u_o)/2 - c.(f_o - f_i)/(2 |c| lambda), c along the outward normal
        double fb;
        if constexpr (F32) {
            const float sgf = side ? 0.5f : -0.5f;
            fb = idp::f2d(0.5f * (ui[0] + uo[0]) - sgf * (uo[1 + d] - ui[1 + d]) * __frcp_rn(lam));
        } else {
            const double dm = side ? uo[1 + d] - ui[1 + d] : ui[1 + d] - uo[1 + d];
            fb = 0.5 * ((ui[0] + uo[0]) - dm * idp::fast_rcp(lam));
        }
        S[le].fbl[s][t] = fb;
        S[le].fbh[s][t] = fb;
    }
    // ---- P1c: low-order subcell fluxes at the interior interfaces
    for (int k = tid; k < EPB * NIF; k += NT) {
        const int le = k / NIF, id = k - le * NIF;
        if (e0 + le >= G.K) continue;
        const int d = id / (NR * N), r1 = id - d * NR * N, r = r1 / N, a = r1 - r * N;
        const int nl = node_of<NP>(d, r, a), nr = node_of<NP>(d, r, a + 1);
        const SM &X = S[le];
        FT ul[NV], ur[NV], fl[NV], fr[NV];
        for (int v = 0; v < NV; ++v) {
            if constexpr (F32) { ul[v] = X.nd.uf[v][nl]; ur[v] = X.nd.uf[v][nr]; }
            else { ul[v] = X.u[v][nl]; ur[v] = X.u[v][nr]; }
        }
        FT lam;
        if constexpr (F32) {
            flux_p<FT>(ul, X.nd.pr[d][nl], X.nd.pr[3][nl], d, fl);
            flux_p<FT>(ur, X.nd.pr[d][nr], X.nd.pr[3][nr], d, fr);
            lam = fmaxf(X.nd.lam[d][nl], X.nd.lam[d][nr]);
        } else {
            flux_h(ul, X.nd.pr[d][nl], X.nd.pr[3][nl], d, fl);
            flux_h(ur, X.nd.pr[d][nr], X.nd.pr[3][nr], d, fr);
            lam = idp::dmax(X.nd.lam[d][nl], X.nd.lam[d][nr]);
        }
        const double cc2d = ops.w[r % NP] * ops.w[r / NP] * X.q[d], ccd = 0.5 * cc2d;
        const FT cc = (FT)(F32 ? (double)idp::d2f(ccd) : ccd);
        // FP64 path: half fluxes for v >= 1, so 2 cc multiplies their sum
        const FT cc2 = (FT)(F32 ? 0.0 : cc2d);
        for (int v = 0; v < NV; ++v)
            S[le].fvf[id][v] = ((F32 || v == 0) ? cc : cc2) * (fl[v] + fr[v]) - cc * lam * (ur[v] - ul[v]);
        if constexpr (F32) S[le].ibar[id] = idp::f2d(0.5f * (ul[0] + ur[0]) - 0.5f * (ur[1 + d] - ul[1 + d]) * __frcp_rn(lam));
        else S[le].ibar[id] = 0.5 * ((ul[0] + ur[0]) - (ur[1 + d] - ul[1 + d]) * idp::fast_rcp(lam));
    }
    __syncthreads();
    // ---- P2: low-order residual, low-order update and bounds per node
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN;
        if (e0 + le >= G.K) continue;
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        const double im = iw3[n] * S[le].iJ;
        double r[NV] = {0, 0, 0, 0, 0}, uv[NV];
        for (int v = 0; v < NV; ++v) uv[v] = S[le].u[v][n];
        double lo = uv[0], hi = uv[0];
        for (int d = 0; d < 3; ++d) {
            const int pos = idx[d], row = idx[(d + 1) % 3] + NP * idx[(d + 2) % 3];
            // low side: the interface (pos-1, pos) or the low face
            double b0l, b0h, b1l, b1h;
            if (pos > 0) {
                const int id = (d * NR + row) * N + pos - 1;
                for (int v = 0; v < NV; ++v) r[v] += to_d3(S[le].fvf[id][v]);
                b0l = b0h = S[le].ibar[id];
            } else {
                for (int v = 0; v < NV; ++v) r[v] += S[le].ff[2 * d][row][v];
                b0l = S[le].fbl[2 * d][row];
                b0h = S[le].fbh[2 * d][row];
            }
            if (pos < N) {
                const int id = (d * NR + row) * N + pos;
                for (int v = 0; v < NV; ++v) r[v] -= to_d3(S[le].fvf[id][v]);
                b1l = b1h = S[le].ibar[id];
            } else {
                for (int v = 0; v < NV; ++v) r[v] -= S[le].ff[2 * d + 1][row][v];
                b1l = S[le].fbl[2 * d + 1][row];
                b1h = S[le].fbh[2 * d + 1][row];
            }
            lo = idp::dmin(lo, idp::dmin(b0l, b1l));
            hi = idp::dmax(hi, idp::dmax(b0h, b1h));
        }
        double uf[NV];
        for (int v = 0; v < NV; ++v) {
            uf[v] = uv[v] + dt * im * r[v];
            S[le].ufv[v][n] = uf[v];
            S[le].rfv[v][n] = r[v];   // overwrites this node's own u only
        }
        double rmn, rmx;
        if (A.limiting >= 2) { rmn = idp::dmax(lo, A.beta * uf[0]); rmx = hi; }
        else { rmn = A.beta * uf[0]; rmx = INFINITY; }
        S[le].rmin[n] = idp::dmin(rmn, uf[0]);
        S[le].rmax[n] = idp::dmax(rmx, uf[0]);
        const double rhoe = uf[0] * uf[4] - 0.5 * (uf[1] * uf[1] + uf[2] * uf[2] + uf[3] * uf[3]);
        const double pm = A.beta * gm1 * rhoe * idp::fast_rcp(uf[0]);
        S[le].pmin[n] = pm;
        S[le].im[n] = im;
        for (int v = 0; v < NV; ++v) S[le].ufvf[v][n] = idp::d2f(uf[v]);
        S[le].gdtf[n] = idp::d2f(kGamma3 * dt * im);
        S[le].pmf[n] = idp::d2f(pm);
        S[le].c0f[n] = idp::d2f(gm1 * rhoe - pm * uf[0]);
    }
    __syncthreads();
    // ---- P2b: telescoped high-order subcell fluxes per row (summed in FP64),
    // then A = F_DG - F_FV (A takes the storage of the face data, the
    // exemption flags that of the outside states: both dead after P2)
    for (int k = tid; k < EPB * 3 * NR; k += NT) {
        const int le = k / (3 * NR), r0 = k - le * 3 * NR, d = r0 / NR, r = r0 - d * NR;
        if (e0 + le >= G.K) continue;
        const double wt = ops.w[r % NP] * ops.w[r / NP];
        // FP32 form: the contraction in FP32 (each interface's A is formed
        // once and enters both its nodes, so conservation is untouched)
        const float wqf = F32 ? idp::d2f(wt * S[le].q[d]) : 0.0f;
        double acc[NV] = {0, 0, 0, 0, 0};
        float accf[NV] = {0, 0, 0, 0, 0};
        for (int l = 0; l < N; ++l) {
            for (int mm = 0; mm < NP; ++mm) {
                if (mm == l) continue;   // Sbar has a zero diagonal
                const int lo_ = l < mm ? l : mm, hi_ = l < mm ? mm : l;
                const int pp = lo_ * (2 * NP - lo_ - 1) / 2 + (hi_ - lo_ - 1);
                if constexpr (F32) {
                    const float sf = Sf[l][mm];
                    for (int v = 0; v < NV; ++v) accf[v] += sf * S[le].pair[d][r][pp][v];
                } else {
                    const double sq = ops.S[l][mm] * S[le].q[d];
                    for (int v = 0; v < NV; ++v) acc[v] += sq * to_d3(S[le].pair[d][r][pp][v]);
                }
            }
            const int id = (d * NR + r) * N + l;
            const int nl = node_of<NP>(d, r, l), nr = node_of<NP>(d, r, l + 1);
            const double iml = S[le].im[nl], imr = S[le].im[nr];
            for (int v = 0; v < NV; ++v) {
                if constexpr (F32) S[le].A[id][v] = idp::f2d(wqf * accf[v] - S[le].fvf[id][v]);
                else S[le].A[id][v] = wt * acc[v] - S[le].fvf[id][v];
            }
            // R15 at both ends (dt/m |A| <= 1e-14 |rho_FV|, both sides times Gamma):
            // decided in FP32 where the two sides differ by more than 1e-3 (far
            // above the few FP32 roundings), else in FP64
            const double Ar = fabs(S[le].A[id][0]);
            const float af = fabsf(idp::d2f(Ar));
            constexpr float kTolG = (float)(kTol3 * kGamma3);
            bool exl, exr;
            {
                const float lf = S[le].gdtf[nl] * af, tf = kTolG * fabsf(S[le].ufvf[0][nl]);
                if (lf < 0.999f * tf) exl = true;
                else if (lf > 1.001f * tf) exl = false;
                else exl = dt * iml * Ar <= kTol3 * fabs(S[le].ufv[0][nl]);
            }
            {
                const float lf = S[le].gdtf[nr] * af, tf = kTolG * fabsf(S[le].ufvf[0][nr]);
                if (lf < 0.999f * tf) exr = true;
                else if (lf > 1.001f * tf) exr = false;
                else exr = dt * imr * Ar <= kTol3 * fabs(S[le].ufv[0][nr]);
            }
            S[le].ex[id] = exl && exr;
        }
    }
    __syncthreads();
    // ---- P3: Zalesak (R7) per node
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN;
        if (e0 + le >= G.K) continue;
        if (n == 0) S[le].npend = 0;   // the pair fluxes are dead: P4's list takes their storage
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        const double m = w3[n] * S[le].J;
        double Pp = 0.0, Pm = 0.0;
        for (int d = 0; d < 3; ++d) {
            const int pos = idx[d], row = idx[(d + 1) % 3] + NP * idx[(d + 2) % 3];
            // the signs on the integer pipe: each inflow adds to one of the two sums
            if (pos > 0) {
                const int id = (d * NR + row) * N + pos - 1;
                const double Gv = S[le].A[id][0];
                if (!S[le].ex[id]) { if (idp::dpos(Gv)) Pp += Gv; else if (idp::dneg(Gv)) Pm += Gv; }
            }
            if (pos < N) {
                const int id = (d * NR + row) * N + pos;
                const double Gv = -S[le].A[id][0];
                if (!S[le].ex[id]) { if (idp::dpos(Gv)) Pp += Gv; else if (idp::dneg(Gv)) Pm += Gv; }
            }
        }
        const double rf = S[le].ufv[0][n];
        const double mdt = m * idt;
        const double Qp = mdt * (S[le].rmax[n] - rf), Qm = mdt * (S[le].rmin[n] - rf);
        // the quotients only where the bound has some room but less than the
        // inflow (0 < R < 1); a node on its bound takes R = 0 without one
        double Rp = 1.0, Rm = 1.0;
        if (idp::dpos(Pp) && idp::dlt(Qp, Pp)) Rp = idp::dpos(Qp) ? Qp * idp::fast_rcp(Pp) : 0.0;
        if (idp::dneg(Pm) && idp::dlt(Pm, Qm)) Rm = idp::dneg(Qm) ? Qm * idp::fast_rcp(Pm) : 0.0;
        S[le].Rp[n] = idp::dpos(Rp) ? Rp : 0.0;
        S[le].Rm[n] = idp::dpos(Rm) ? Rm : 0.0;
        if (comb) {
            // R- of the positivity bounds alone (rho >= beta rho_FV; no upper bound)
            const double Qm2 = mdt * (idp::dmin(A.beta * rf, rf) - rf);
            double Rm2 = 1.0;
            if (idp::dneg(Pm) && idp::dlt(Pm, Qm2)) Rm2 = idp::dneg(Qm2) ? Qm2 * idp::fast_rcp(Pm) : 0.0;
            S[le].Rm2[n] = idp::dpos(Rm2) ? Rm2 : 0.0;
        }
    }
    __syncthreads();
    // ---- P4: interface factors: Zalesak, then the pressure factor of both
    // ends with Gamma = 6, each end searched below the other's result. Pass 1
    // certifies the ends in FP32 from the per-node FP32 copies; the first end
    // it leaves undecided goes to its element's list with the factor reached
    // so far, and pass 2 runs those FP64 solves (R8) by whole warps.
    // the FP32 certificate of end `side` of interface id at th
    auto cert_end = [&](const SM &X, int id, int side, const float *af, double th) {
        const int d = id / (NR * N), r1 = id - d * NR * N, r = r1 / N, a = r1 - r * N;
        const int nd = node_of<NP>(d, r, side ? a + 1 : a);
        float u0f[NV], avf[NV];
        const float sg = side ? X.gdtf[nd] : -X.gdtf[nd];
        for (int v = 0; v < NV; ++v) { u0f[v] = X.ufvf[v][nd]; avf[v] = sg * af[v]; }
        return admissible3_f32f(idp::d2f(gm1), u0f, avf, X.pmf[nd], X.c0f[nd], idp::d2f(th));
    };
    // the FP64 solve of end `side` of interface id below th
    auto solve_end = [&](const SM &X, int id, int side, double th) {
        const int d = id / (NR * N), r1 = id - d * NR * N, r = r1 / N, a = r1 - r * N;
        const int nd = node_of<NP>(d, r, side ? a + 1 : a);
        double u0[NV], av[NV];
        const double sg = (side ? kGamma3 : -kGamma3) * dt * X.im[nd];
        for (int v = 0; v < NV; ++v) { u0[v] = X.ufv[v][nd]; av[v] = sg * X.A[id][v]; }
        return theta3(g, u0, av, X.pmin[nd], th);
    };
    // the pressure factor of both ends below lr (certificate, else FP64 solve)
    auto pressure_factor = [&](const SM &X, int id, const float *af, double lr) {
        double th = lr;
        for (int side = 0; side < 2 && idp::dpos(th); ++side)
            if (!cert_end(X, id, side, af, th)) th = solve_end(X, id, side, th);
        return th;
    };
    if (comb) {
        // Eq. combination_posLim_local: l = (1 - a) l_positivity + a l_local
        for (int k = tid; k < EPB * NIF; k += NT) {
            const int le = k / NIF, id = k - le * NIF;
            if (e0 + le >= G.K) continue;
            const int d = id / (NR * N), r1 = id - d * NR * N, r = r1 / N, a = r1 - r * N;
            const int nl = node_of<NP>(d, r, a), nr = node_of<NP>(d, r, a + 1);
            const SM &X = S[le];
            const double *Ai = X.A[id];
            const bool neg = idp::dneg(Ai[0]);
            const double lr = X.ex[id] ? 1.0 : neg ? idp::dmin(X.Rp[nl], X.Rm[nr]) : idp::dmin(X.Rm[nl], X.Rp[nr]);
            const double lr2 = X.ex[id] ? 1.0 : neg ? X.Rm2[nr] : X.Rm2[nl];
            float af[NV];
            for (int v = 0; v < NV; ++v) af[v] = idp::d2f(Ai[v]);
            const double th = pressure_factor(X, id, af, lr), th2 = pressure_factor(X, id, af, lr2);
            S[le].ell[id] = (1.0 - X.aind) * th2 + X.aind * th;
        }
    }
    for (int k = tid; k < EPB * NIF && !comb; k += NT) {
        const int le = k / NIF, id = k - le * NIF;
        if (e0 + le >= G.K) continue;
        double th = 1.0;
        if (A.limiting > 0) {
            const int d = id / (NR * N), r1 = id - d * NR * N, r = r1 / N, a = r1 - r * N;
            const int nl = node_of<NP>(d, r, a), nr = node_of<NP>(d, r, a + 1);
            const double *Ai = S[le].A[id];
            th = S[le].ex[id] ? 1.0
               : idp::dneg(Ai[0]) ? idp::dmin(S[le].Rp[nl], S[le].Rm[nr]) : idp::dmin(S[le].Rm[nl], S[le].Rp[nr]);
            float af[NV];
            for (int v = 0; v < NV; ++v) af[v] = idp::d2f(Ai[v]);
            int pend = -1;
            for (int side = 0; side < 2 && idp::dpos(th); ++side)
                if (!cert_end(S[le], id, side, af, th)) { pend = side; break; }
            if (pend >= 0) S[le].pend[atomicAdd(&S[le].npend, 1)] = (unsigned short)(id | (pend << 15));
        }
        S[le].ell[id] = th;
    }
    __syncthreads();
    if (A.limiting > 0 && !comb) {
        int tot = 0;
        for (int le = 0; le < EPB; ++le) tot += (e0 + le < G.K) ? S[le].npend : 0;
        for (int k = tid; k < tot; k += NT) {
            int le = 0, j = k;
            while (j >= S[le].npend) { j -= S[le].npend; ++le; }
            const SM &X = S[le];
            const int item = X.pend[j], id = item & 0x7fff, side0 = item >> 15;
            double th = solve_end(X, id, side0, X.ell[id]);
            if (side0 == 0 && idp::dpos(th)) {
                float af[NV];
                for (int v = 0; v < NV; ++v) af[v] = idp::d2f(X.A[id][v]);
                if (!cert_end(X, id, 1, af, th)) th = solve_end(X, id, 1, th);
            }
            S[le].ell[id] = th;
        }
    }
    __syncthreads();
    // ---- P5: limited update, stage combination, statistics
    unsigned vr = 0, vp = 0, np_ = 0, nact = 0;
    double am = 0.0, rmin_st = INFINITY, pmin_st = INFINITY;
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        const double im = S[le].im[n];
        double s[NV] = {0, 0, 0, 0, 0}, lm = 1.0;
        // the node's interfaces in a fixed order: x low, x high, y low, y high, z low, z high
        for (int d = 0; d < 3; ++d) {
            const int pos = idx[d], row = idx[(d + 1) % 3] + NP * idx[(d + 2) % 3];
            if (pos > 0) {
                const int id = (d * NR + row) * N + pos - 1;
                const double l = S[le].ell[id];
                lm = idp::dmin(lm, l);
                for (int v = 0; v < NV; ++v) s[v] += l * S[le].A[id][v];
            }
            if (pos < N) {
                const int id = (d * NR + row) * N + pos;
                const double l = S[le].ell[id];
                lm = idp::dmin(lm, l);
                for (int v = 0; v < NV; ++v) s[v] -= l * S[le].A[id][v];
            }
        }
        // a node on a mortar side: its first mortar slot (x, y, z order)
        int mslot = -1;
        for (int d = 0; d < 3 && mslot < 0; ++d) {
            const int pos = idx[d], row = idx[(d + 1) % 3] + NP * idx[(d + 2) % 3];
            const int nbv = pos == 0 ? S[le].nb[2 * d] : (pos == N ? S[le].nb[2 * d + 1] : 0);
            if (nbv < -1) mslot = -2 - nbv + row;
        }
        const size_t gi = (size_t)e * NN + n;
        double ut[NV];
        if (mslot >= 0) {
            // hand-off: the mortar kernels add the limited mortar corrections
            // and write the node
            const int mn = MO.slot_mn[mslot];
            for (int v = 0; v < NV; ++v) {
                ut[v] = S[le].ufv[v][n] + dt * im * s[v];
                MO.h_uvol[(size_t)v * MO.MN + mn] = ut[v];
                MO.h_res[(size_t)v * MO.MN + mn] = S[le].rfv[v][n] + s[v];
            }
            MO.h_b[0 * (size_t)MO.MN + mn] = S[le].rmin[n];
            MO.h_b[1 * (size_t)MO.MN + mn] = S[le].rmax[n];
            MO.h_b[2 * (size_t)MO.MN + mn] = S[le].pmin[n];
            MO.h_b[3 * (size_t)MO.MN + mn] = S[le].ufv[0][n];
            MO.h_b[4 * (size_t)MO.MN + mn] = im;
        } else {
            for (int v = 0; v < NV; ++v) {
                const double res = S[le].rfv[v][n] + s[v];
                ut[v] = S[le].ufv[v][n] + dt * im * s[v];
                double o;
                if (A.mode == 0) o = res * im;
                else if (A.comb == 1) o = 0.75 * A.un[v * KN + gi] + 0.25 * ut[v];
                else if (A.comb == 2) o = A.un[v * KN + gi] * (1.0 / 3.0) + 2.0 / 3.0 * ut[v];
                else o = ut[v];
                A.out[v * KN + gi] = o;
            }
        }
        if (A.collect && A.limiting > 0) {
            if (idp::dlt(lm, 1.0)) {
                am += w3[n] * S[le].J * (1.0 - lm);
                nact++;
            }
            if (mslot < 0) {
                // the bounds the stage keeps: the positivity ones under the combined limiting
                const double rf0 = S[le].ufv[0][n];
                const double rl = comb ? idp::dmin(A.beta * rf0, rf0) : S[le].rmin[n];
                const double rh = comb ? INFINITY : S[le].rmax[n], pl = S[le].pmin[n];
                // the density bounds: the exact comparison first, the tolerance only past a bound
                if ((idp::dlt(ut[0], rl) && idp::dlt(ut[0], rl - kViol3 * fabs(rl))) ||
                    (idp::dlt(rh, ut[0]) && idp::dlt(rh + kViol3 * fabs(rh), ut[0])))
                    vr++;
                // rho p = (gamma-1)(rho E - |m|^2/2) against p_min rho: certified in
                // FP32 when it clears the bound by 1e-5 of its terms (far above the
                // FP32 rounding of these few operations), else decided in FP64
                float q[NV];
                for (int v = 0; v < NV; ++v) q[v] = idp::d2f(ut[v]);
                const float kef = 0.5f * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]), ref = q[0] * q[4];
                const float gf = idp::d2f(gm1), rpf = gf * (ref - kef), lim = idp::d2f(pl) * q[0];
                if (q[0] > 0.0f && rpf - lim > 1e-5f * (gf * (fabsf(ref) + kef) + fabsf(lim))) {
                    pmin_st = idp::dmin(pmin_st, idp::f2d(__fdiv_rn(rpf, q[0])));
                } else {
                    const double rp = gm1 * (ut[0] * ut[4] - 0.5 * (ut[1] * ut[1] + ut[2] * ut[2] + ut[3] * ut[3]));
                    if (idp::dlt(rp, (pl - kViol3 * fabs(pl)) * ut[0])) vp++;
                    if (!idp::dpos(ut[0]) || !idp::dpos(rp)) np_++;
                    else pmin_st = idp::dmin(pmin_st, idp::f2d(__fdiv_rn(idp::d2f(rp), q[0])));
                }
                rmin_st = idp::dmin(rmin_st, ut[0]);
            }
        }
    }
    if (A.collect && A.limiting > 0) {
        const unsigned FULL = 0xffffffffu;
        vr = __reduce_add_sync(FULL, vr);
        vp = __reduce_add_sync(FULL, vp);
        np_ = __reduce_add_sync(FULL, np_);
        nact = __reduce_add_sync(FULL, nact);
        for (int o = 16; o > 0; o >>= 1) {
            am += __shfl_down_sync(FULL, am, o);
            rmin_st = idp::dmin(rmin_st, __shfl_down_sync(FULL, rmin_st, o));
            pmin_st = idp::dmin(pmin_st, __shfl_down_sync(FULL, pmin_st, o));
        }
        if ((tid & 31) == 0) {
            if (am > 0.0) atomicAdd(&A.stats->alpha_m, am);
            if (nact) atomicAdd(&A.stats->n_active, (unsigned long long)nact);
            if (vr) atomicAdd(&A.stats->n_vrho, (unsigned long long)vr);
            if (vp) atomicAdd(&A.stats->n_vp, (unsigned long long)vp);
            if (np_) atomicAdd(&A.stats->n_nonpos, (unsigned long long)np_);
            stat_min(&A.stats->min_rho_bits, rmin_st);
            stat_min(&A.stats->min_p_bits, pmin_st);
        }
    }
    if (A.collect && (vr | vp | np_) != 0u && (tid & 31) == 0) atomicOr(A.status, S_VIOLATION);
}

// |v_d| + c of a state along the three axes, with one fast reciprocal and
// square root; false for a non-admissible state
__device__ __forceinline__ bool wave_speeds3(double g, const double *u, double *lam) {
    const double ir = idp::fast_rcp(u[0]);
    const double p = (g - 1.0) * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * ir);
    if (!idp::dpos(u[0]) || !idp::dpos(p)) {
        lam[0] = lam[1] = lam[2] = 0.0;
        return false;
    }
    const double c = idp::fast_sqrt(g * p * ir);
    for (int d = 0; d < 3; ++d) lam[d] = fabs(u[1 + d] * ir) + c;
    return true;
}

// the same in FP32 from the certified FP32 primitives (the FP32 form)
__device__ __forceinline__ bool wave_speeds3(double g, const double *u, float *lam) {
    float uf[NV], v[3], p, ir;
    const bool ok = prim3_f32(g - 1.0, u, uf, v, p, ir);
    const float c = ok ? sqrtf(idp::d2f(g) * p * ir) : 0.0f;
    for (int d = 0; d < 3; ++d) lam[d] = ok ? fabsf(v[d]) + c : 0.0f;
    return ok;
}

// The FP32 form's time step is formed in FP32 and scaled by (1 - 8e-6):
// its wave speeds carry the certified FP32 pressure (within 2.5e-6 of the
// rounded state's), a square root and a few roundings, so the scaled
// quotient stays below the FP64 one.
constexpr double kDtSafe32 = 1.0 - 8e-6;

// IDP time step (Eq. timestep_restriction): per node m_i / sum_j 2 d_ij over
// its subcell and face neighbours (at a mortar side the slot's sum over its
// pairs, formed by the mortar flux kernel from the same state); minimum per
// block, one atomic per block. 2 d_ij of a subcell or conforming pair is
// w_t1 w_t2 (A_d / 4) max(lambda_i, lambda_j). FT = float: wave speeds, sums
// and the quotient in FP32 (the FP32 form).
// The FP64 path's time step in two passes (pk): the FP32 kernel (mode 1)
// also writes each element's minimum (emin, bits of a positive float); the
// FP64 kernel (mode 2) then forms the FP64 quotients only in the
// elements whose FP32 minimum lies within a relative 1e-4 of the FP32
// pass's overall minimum (smin). The FP32 quotients are within about 1e-5
// of the FP64 ones (the FP32 form's margin kDtSafe32 is 8e-6), so the FP64
// minimiser's element is always formed and the result is the one-pass FP64
// minimum bit for bit.
struct DtPick3 {
    int mode;                          // 0: one pass; 1: FP32 pass; 2: FP64 pass over the picked elements
    unsigned *emin;                    // per element: the FP32 pass's minimum
    const unsigned long long *smin;    // mode 2: the FP32 pass's minimum (bits of a double)
};
constexpr double kPickMargin3 = 1e-4;

static __global__ void k_inf3d(unsigned long long *p) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = (unsigned long long)__double_as_longlong(INFINITY);
}

template <int NP, int EPB, typename FT>
__global__ void __launch_bounds__(Launch3<NP, EPB>::threads)
k_dt3d(Grid3 G, const Ops3 *__restrict__ ops_g, const double *__restrict__ u, double gamma,
       unsigned long long *dtmin, unsigned *status, DtPick3 pk) {
    using E = El3<NP>;
    constexpr bool F32 = sizeof(FT) == 4;
    constexpr int N = E::N, NN = E::NN, NT = Launch3<NP, EPB>::threads;
    __shared__ FT lam[EPB][3][NN];
    __shared__ FT w[NP];
    __shared__ FT geo[EPB][4];   // quarter face areas, dx dy dz / 8
    __shared__ unsigned long long best_s[NT / 32];
    __shared__ unsigned s_emin[EPB];
    __shared__ unsigned char s_cand[EPB];
    if (threadIdx.x < NP) w[threadIdx.x] = (FT)(F32 ? (double)idp::d2f(ops_g->w[threadIdx.x]) : ops_g->w[threadIdx.x]);
    const size_t KN = (size_t)G.K * NN;
    const int e0 = blockIdx.x * EPB, tid = threadIdx.x;
    if (pk.mode != 0) {
        // (EPB * NN <= NT: one node per thread)
        const int le = tid / NN, e = e0 + le;
        bool cd = false;
        if (le < EPB && tid % NN == 0) {
            if (pk.mode == 1) s_emin[le] = 0x7f800000u;   // +inf
            if (pk.mode == 2 && e < G.K)
                cd = (double)__uint_as_float(pk.emin[e]) <= __longlong_as_double((long long)*pk.smin) * (1.0 + kPickMargin3);
            s_cand[le] = cd;
        }
        // mode 2: a block without picked elements has nothing to do (uniform)
        if (!__syncthreads_or(cd) && pk.mode == 2) return;
    }
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        if (pk.mode == 2 && !s_cand[le]) continue;
        if (n == 0) {
            double h[3];
            extents3(G, e, h);
            const double gd[4] = {h[1] * h[2] / 4.0, h[0] * h[2] / 4.0, h[0] * h[1] / 4.0, h[0] * h[1] * h[2] / 8.0};
            for (int c = 0; c < 4; ++c) geo[le][c] = (FT)(F32 ? (double)idp::d2f(gd[c]) : gd[c]);
        }
        double uv[NV];
        FT l3[3];
        for (int v = 0; v < NV; ++v) uv[v] = u[v * KN + (size_t)e * NN + n];
        if (!wave_speeds3(gamma, uv, l3)) atomicOr(status, S_BAD_INPUT);
        for (int d = 0; d < 3; ++d) lam[le][d][n] = l3[d];
    }
    __syncthreads();
    unsigned long long best = (unsigned long long)__double_as_longlong(INFINITY);
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        if (pk.mode == 2 && !s_cand[le]) continue;
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        FT s2d = FT(0);
        double smort = 0.0;   // the mortar slots' sums (FP64)
        for (int d = 0; d < 3; ++d) {
            const int pos = idx[d];
            const FT li = lam[le][d][n];
            FT lsum = FT(0);
            for (int side = 0; side < 2; ++side) {
                FT lo;
                if (side == 0 ? pos > 0 : pos < N) {
                    const int nn2 = n + (side == 0 ? -1 : 1) * (d == 0 ? 1 : (d == 1 ? NP : NP * NP));
                    lo = lam[le][d][nn2];
                } else {
                    const int s = 2 * d + side, nb = G.nbr[6 * e + s];
                    if (nb < -1) {
                        smort += G.mort.dsum[-2 - nb + idx[(d + 1) % 3] + NP * idx[(d + 2) % 3]];
                        continue;
                    }
                    double o[NV];
                    if (nb >= 0) {
                        int jdx[3] = {idx[0], idx[1], idx[2]};
                        jdx[d] = side ? 0 : N;
                        const int nout = (jdx[2] * NP + jdx[1]) * NP + jdx[0];
                        for (int v = 0; v < NV; ++v) o[v] = u[v * KN + (size_t)nb * NN + nout];
                    } else {
                        double in[NV];
                        for (int v = 0; v < NV; ++v) in[v] = u[v * KN + (size_t)e * NN + n];
                        ghost3(G, s, in, o);
                    }
                    FT l3[3];
                    wave_speeds3(gamma, o, l3);
                    lo = l3[d];
                }
                if constexpr (F32) lsum += fmaxf(li, lo);
                else lsum += idp::dmax(li, lo);
            }
            s2d += w[idx[(d + 1) % 3]] * w[idx[(d + 2) % 3]] * geo[le][d] * lsum;
        }
        const FT m = w[idx[0]] * w[idx[1]] * w[idx[2]] * geo[le][3];
        double val;
        if constexpr (F32) {
            const float tot = smort == 0.0 ? s2d : (float)(idp::f2d(s2d) + smort) ;
            val = idp::f2d(__fdiv_rn(m, tot)) * kDtSafe32;
        } else {
            val = m * idp::fast_rcp(s2d + smort);
        }
        const unsigned long long vb = (unsigned long long)__double_as_longlong(val);
        if (val > 0.0 && vb < best) best = vb;
        if (pk.mode == 1 && val > 0.0) atomicMin(&s_emin[le], __float_as_uint((float)val));
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
        best = ob < best ? ob : best;
    }
    if ((tid & 31) == 0) best_s[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
        unsigned long long b = best_s[0];
        for (int k = 1; k < NT / 32; ++k) b = best_s[k] < b ? best_s[k] : b;
        if (b < (unsigned long long)__double_as_longlong(INFINITY)) atomicMin(dtmin, b);
    }
    if (pk.mode == 1 && tid < EPB && e0 + tid < G.K) pk.emin[e0 + tid] = s_emin[tid];
}

// the step's end: t += cfl * min, the minimum reset to +inf for the next step
static __global__ void k_advance3d(double *t, unsigned long long *dtmin, double cfl, double *dt_last) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double dt = cfl * __longlong_as_double((long long)*dtmin);
        *t += dt;
        *dt_last = dt;
        *dtmin = (unsigned long long)__double_as_longlong(INFINITY);
    }
}

}  // namespace idp3
