// idp3d.cuh -- the IDP-limited LGL-DGSEM stage for the 3D Euler equations
// (d = 3 of arXiv 2607.06045, Sec. 2) on a conforming Cartesian grid of
// hexahedra: one fused element kernel per stage and the IDP time step.
//
// The stage is the 2D one with the third direction (Sec. 2.1-2.3 for
// d = 3): Ranocha's two-point fluxes along x, y and z within each element,
// the telescoped high-order subcell fluxes (Eq. fluxdifferencingform), the
// LLF faces, the low-order subcell fluxes with the graph viscosity
// (Eq. LowOrderScheme_globalIndices in flux form), bar-state density bounds
// and positivity (Eqs. Bounds_Positivity, Bounds_Barstates), Zalesak density
// limiting and the pressure factor with Gamma = 2d = 6, then the SSP-RK3
// combination. State u[5][K][N+1]^3 FP64 (rho, rho v1, rho v2, rho v3, rho e),
// x index fastest; element e = (ez ny + ey) nx + ex.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "idp_bits.cuh"

namespace idp3 {

constexpr int NV = 5;
constexpr int NPMAX3 = 8;
constexpr double kTol3 = 1e-14;       // R15
constexpr double kViol3 = 1e-13;      // R13
constexpr double kGamma3 = 6.0;       // Gamma = 2d (Sec. 2.3)
enum : int { B_PERIODIC = 0, B_WALL = 1, B_DIRICHLET = 2, B_OUTFLOW = 3 };
enum : unsigned { S_BAD_INPUT = 1u, S_VIOLATION = 2u };

// the grid, its boundary kinds per side (-x, +x, -y, +y, -z, +z) and the
// conserved Dirichlet states
struct Grid3 {
    int nx, ny, nz, K;
    double dx, dy, dz;
    int bc[6];
    double bc_cons[6][NV];
};

// LGL nodes and weights, Sbar (Sec. 2.1), 1 / w
struct Ops3 {
    double xi[NPMAX3], w[NPMAX3], S[NPMAX3][NPMAX3];
};

// statistics of the limited stages (atomics)
struct Stats3 {
    double alpha_m;                 // sum of m (1 - min factor at the node)
    unsigned long long n_active;    // nodes with a factor below one
    unsigned long long n_vrho, n_vp, n_nonpos;
    unsigned long long min_rho_bits, min_p_bits;
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
    int limiting;        // 0 none (the high-order residual), 1 positivity, 2 local
    int collect;         // statistics on
    double beta, gamma;
    Stats3 *stats;
    unsigned *status;
};

__device__ __forceinline__ double stage_dt3(const Stage3 &A) {
    return A.dtmin ? A.cfl * __longlong_as_double((long long)*A.dtmin) : A.dt_host;
}

__device__ __forceinline__ double pres3(double g, const double *u) {
    return (g - 1.0) * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0]);
}

__device__ __forceinline__ void flux3(double g, const double *u, int d, double *f) {
    const double p = pres3(g, u), vn = u[1 + d] / u[0];
    f[0] = u[1 + d];
    f[1] = u[1] * vn + (d == 0 ? p : 0.0);
    f[2] = u[2] * vn + (d == 1 ? p : 0.0);
    f[3] = u[3] * vn + (d == 2 ? p : 0.0);
    f[4] = (u[4] + p) * vn;
}

__device__ __forceinline__ double wave3(double g, const double *u, int d) {
    return fabs(u[1 + d] / u[0]) + sqrt(g * pres3(g, u) / u[0]);
}

// R2: logarithmic mean, Ismail-Roe series below u = 1e-4
__device__ __forceinline__ double logmean3(double a, double b) {
    const double f = (a - b) / (a + b), uu = f * f;
    if (uu < 1e-4) return (a + b) / (2.0 * (1.0 + uu / 3.0 + uu * uu / 5.0 + uu * uu * uu / 7.0));
    return (a - b) / log(a / b);
}

// R1 along axis d from the two states and their primitives (v, p)
__device__ __forceinline__ void ranocha3(double g, const double *uL, const double *vL, double pL,
                                         const double *uR, const double *vR, double pR, int d, double *f) {
    const double rho_ln = logmean3(uL[0], uR[0]);
    const double bet_ln = logmean3(uL[0] / pL, uR[0] / pR);
    const double vdot = vL[0] * vR[0] + vL[1] * vR[1] + vL[2] * vR[2];
    const double fr = rho_ln * 0.5 * (vL[d] + vR[d]);
    f[0] = fr;
    for (int a = 0; a < 3; ++a) f[1 + a] = fr * 0.5 * (vL[a] + vR[a]) + (a == d ? 0.5 * (pL + pR) : 0.0);
    f[4] = fr * (0.5 * vdot + 1.0 / ((g - 1.0) * bet_ln)) + 0.5 * (pL * vR[d] + pR * vL[d]);
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

// neighbour element across side s of element e, or -1 at a non-periodic boundary
__device__ __forceinline__ int nbr3(const Grid3 &G, int e, int s) {
    int ex = e % G.nx, ey = (e / G.nx) % G.ny, ez = e / (G.nx * G.ny);
    const int d = s / 2, step = (s & 1) ? 1 : -1;
    int c[3] = {ex, ey, ez};
    const int n[3] = {G.nx, G.ny, G.nz};
    c[d] += step;
    if (c[d] < 0 || c[d] >= n[d]) {
        if (G.bc[s] != B_PERIODIC) return -1;
        c[d] = (c[d] + n[d]) % n[d];
    }
    return (c[2] * G.ny + c[1]) * G.nx + c[0];
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

// shared memory of one element; arrays whose lifetimes do not overlap share
// storage (phases P0..P5 of k_element3d)
template <int NP>
struct Sm3 {
    using E = El3<NP>;
    static constexpr int NN = E::NN, NR = E::NR, NIF = E::NIF, NPAIR = E::NPAIR;
    union {
        double u[NV][NN];      // P0 - P2: the stage input
        double rfv[NV][NN];    // P2 - P5: low-order residual (each node overwrites only its own u)
    };
    double pr[4][NN];          // P0 - P1: v1, v2, v3, p
    union {
        double outs[6][NR][NV];   // P0 - P1: outside states of the six faces
        struct {                  // P2b - P5
            double Rp[NN], Rm[NN];       // Zalesak factors (P3 - P4)
            double ell[NIF];             // interface factors (P4 - P5)
            unsigned char ex[NIF];       // R15 exemption (P2b - P4)
        };
    };
    double pair[3][NR][NPAIR][NV];   // P1 - P2b: two-point fluxes of every row
    union {
        struct {                     // P1 - P2
            double ff[6][NR][NV];    // face fluxes, mass-weighted, along +d
            double fbar[6][NR];      // bar-state density across the face
            double ibar[NIF];        // bar-state density of the interior interfaces
        };
        double A[NIF][NV];           // P2b - P5: antidiffusive fluxes (mass-weighted)
    };
    double fvf[NIF][NV];       // P1 - P2b: low-order subcell fluxes, mass-weighted, along +d
    double ufv[NV][NN];        // P2 - P5
    double rmin[NN], rmax[NN], pmin[NN];
};

// threads of a block of EPB elements: one per node, rounded up to whole warps
template <int NP, int EPB>
struct Launch3 {
    static constexpr int items = EPB * NP * NP * NP, threads = (items + 31) / 32 * 32;
};

// One block of EPB elements, one thread per node; items of each phase are
// spread over the block.
template <int NP, int EPB>
__global__ void __launch_bounds__(Launch3<NP, EPB>::threads)
k_element3d(Grid3 G, const Ops3 *__restrict__ ops_g, Stage3 A) {
    using E = El3<NP>;
    using SM = Sm3<NP>;
    constexpr int N = E::N, NN = E::NN, NR = E::NR, NPAIR = E::NPAIR, NIF = E::NIF, NT = Launch3<NP, EPB>::threads;
    extern __shared__ __align__(16) unsigned char sm3_raw[];
    SM *S = reinterpret_cast<SM *>(sm3_raw);
    __shared__ Ops3 ops;
    const int tid = threadIdx.x;
    for (int k = tid; k < (int)(sizeof(Ops3) / sizeof(double)); k += NT)
        reinterpret_cast<double *>(&ops)[k] = reinterpret_cast<const double *>(ops_g)[k];
    const size_t KN = (size_t)G.K * NN;
    const double g = A.gamma;
    const double dt = stage_dt3(A);
    const double q[3] = {G.dy * G.dz / 4.0, G.dx * G.dz / 4.0, G.dx * G.dy / 4.0};   // quarter face areas
    const double J = G.dx * G.dy * G.dz / 8.0;
    const int e0 = blockIdx.x * EPB;
    // ---- P0: state, primitives, outside states
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        double uv[NV];
        for (int v = 0; v < NV; ++v) { uv[v] = A.u[v * KN + (size_t)e * NN + n]; S[le].u[v][n] = uv[v]; }
        const double p = pres3(g, uv);
        for (int a = 0; a < 3; ++a) S[le].pr[a][n] = uv[1 + a] / uv[0];
        S[le].pr[3][n] = p;
        if (!(uv[0] > 0.0) || !(p > 0.0)) atomicOr(A.status, S_BAD_INPUT);
    }
    for (int k = tid; k < EPB * 6 * NR; k += NT) {
        const int le = k / (6 * NR), r0 = k - le * 6 * NR, s = r0 / NR, t = r0 - s * NR, e = e0 + le;
        if (e >= G.K) continue;
        const int d = s / 2, side = s & 1;
        const int nb = nbr3(G, e, s);
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
    }
    __syncthreads();
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
        double ua[NV], ub[NV], va[3], vb[3], f[NV];
        for (int v = 0; v < NV; ++v) { ua[v] = S[le].u[v][na]; ub[v] = S[le].u[v][nb]; }
        for (int c = 0; c < 3; ++c) { va[c] = S[le].pr[c][na]; vb[c] = S[le].pr[c][nb]; }
        ranocha3(g, ua, va, S[le].pr[3][na], ub, vb, S[le].pr[3][nb], d, f);
        for (int v = 0; v < NV; ++v) S[le].pair[d][r][pp][v] = f[v];
    }
    // ---- P1b: LLF faces (mass-weighted, along +d) and their bar-state densities
    for (int k = tid; k < EPB * 6 * NR; k += NT) {
        const int le = k / (6 * NR), r0 = k - le * 6 * NR, s = r0 / NR, t = r0 - s * NR;
        if (e0 + le >= G.K) continue;
        const int d = s / 2, side = s & 1;
        const int nin = node_of<NP>(d, t, side ? N : 0);
        double ui[NV], uo[NV], fi[NV], fo[NV];
        for (int v = 0; v < NV; ++v) { ui[v] = S[le].u[v][nin]; uo[v] = S[le].outs[s][t][v]; }
        flux3(g, ui, d, fi);
        flux3(g, uo, d, fo);
        const double lam = fmax(wave3(g, ui, d), wave3(g, uo, d));
        const double wt = ops.w[t % NP] * ops.w[t / NP], cw = wt * q[d];
        // left state first: the outside is on the left of a low face
        const double *uL = side ? ui : uo, *uR = side ? uo : ui, *fL = side ? fi : fo, *fR = side ? fo : fi;
        for (int v = 0; v < NV; ++v) S[le].ff[s][t][v] = cw * (0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]));
        // ubar = (u_i + u_o)/2 - c.(f_o - f_i)/(2 |c| lambda), c along the outward normal
        const double sg = side ? 1.0 : -1.0;
        S[le].fbar[s][t] = 0.5 * (ui[0] + uo[0]) - sg * (fo[0] - fi[0]) / (2.0 * lam);
    }
    // ---- P1c: low-order subcell fluxes at the interior interfaces
    for (int k = tid; k < EPB * NIF; k += NT) {
        const int le = k / NIF, id = k - le * NIF;
        if (e0 + le >= G.K) continue;
        const int d = id / (NR * N), r1 = id - d * NR * N, r = r1 / N, a = r1 - r * N;
        const int nl = node_of<NP>(d, r, a), nr = node_of<NP>(d, r, a + 1);
        double ul[NV], ur[NV], fl[NV], fr[NV];
        for (int v = 0; v < NV; ++v) { ul[v] = S[le].u[v][nl]; ur[v] = S[le].u[v][nr]; }
        flux3(g, ul, d, fl);
        flux3(g, ur, d, fr);
        const double lam = fmax(wave3(g, ul, d), wave3(g, ur, d));
        const double cc = ops.w[r % NP] * ops.w[r / NP] * q[d] / 2.0;
        for (int v = 0; v < NV; ++v) S[le].fvf[id][v] = cc * (fl[v] + fr[v]) - cc * lam * (ur[v] - ul[v]);
        S[le].ibar[id] = 0.5 * (ul[0] + ur[0]) - (fr[0] - fl[0]) / (2.0 * lam);
    }
    __syncthreads();
    // ---- P2: low-order residual, low-order update and bounds per node
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN;
        if (e0 + le >= G.K) continue;
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        const double m = ops.w[idx[0]] * ops.w[idx[1]] * ops.w[idx[2]] * J;
        double r[NV] = {0, 0, 0, 0, 0}, uv[NV];
        for (int v = 0; v < NV; ++v) uv[v] = S[le].u[v][n];
        double lo = uv[0], hi = uv[0];
        for (int d = 0; d < 3; ++d) {
            const int pos = idx[d], row = idx[(d + 1) % 3] + NP * idx[(d + 2) % 3];
            // low side: the interface (pos-1, pos) or the low face
            if (pos > 0) {
                const int id = (d * NR + row) * N + pos - 1;
                for (int v = 0; v < NV; ++v) r[v] += S[le].fvf[id][v];
                lo = fmin(lo, S[le].ibar[id]); hi = fmax(hi, S[le].ibar[id]);
            } else {
                for (int v = 0; v < NV; ++v) r[v] += S[le].ff[2 * d][row][v];
                lo = fmin(lo, S[le].fbar[2 * d][row]); hi = fmax(hi, S[le].fbar[2 * d][row]);
            }
            if (pos < N) {
                const int id = (d * NR + row) * N + pos;
                for (int v = 0; v < NV; ++v) r[v] -= S[le].fvf[id][v];
                lo = fmin(lo, S[le].ibar[id]); hi = fmax(hi, S[le].ibar[id]);
            } else {
                for (int v = 0; v < NV; ++v) r[v] -= S[le].ff[2 * d + 1][row][v];
                lo = fmin(lo, S[le].fbar[2 * d + 1][row]); hi = fmax(hi, S[le].fbar[2 * d + 1][row]);
            }
        }
        double uf[NV];
        for (int v = 0; v < NV; ++v) {
            uf[v] = uv[v] + dt / m * r[v];
            S[le].ufv[v][n] = uf[v];
            S[le].rfv[v][n] = r[v];   // overwrites this node's own u only
        }
        double rmn, rmx;
        if (A.limiting >= 2) { rmn = fmax(lo, A.beta * uf[0]); rmx = hi; }
        else { rmn = A.beta * uf[0]; rmx = INFINITY; }
        S[le].rmin[n] = fmin(rmn, uf[0]);
        S[le].rmax[n] = fmax(rmx, uf[0]);
        S[le].pmin[n] = A.beta * pres3(g, uf);
    }
    __syncthreads();
    // ---- P2b: telescoped high-order subcell fluxes per row, then A = F_DG - F_FV
    // (A takes the storage of the face data, the exemption flags that of the
    // outside states: both dead after P2)
    for (int k = tid; k < EPB * 3 * NR; k += NT) {
        const int le = k / (3 * NR), r0 = k - le * 3 * NR, d = r0 / NR, r = r0 - d * NR;
        if (e0 + le >= G.K) continue;
        const double wt = ops.w[r % NP] * ops.w[r / NP];
        double acc[NV] = {0, 0, 0, 0, 0};
        for (int l = 0; l < N; ++l) {
            for (int mm = 0; mm < NP; ++mm) {
                if (mm == l) continue;   // Sbar has a zero diagonal
                const int lo_ = l < mm ? l : mm, hi_ = l < mm ? mm : l;
                const int pp = lo_ * (2 * NP - lo_ - 1) / 2 + (hi_ - lo_ - 1);
                const double sq = ops.S[l][mm] * q[d];
                for (int v = 0; v < NV; ++v) acc[v] += sq * S[le].pair[d][r][pp][v];
            }
            const int id = (d * NR + r) * N + l;
            const int nl = node_of<NP>(d, r, l), nr = node_of<NP>(d, r, l + 1);
            const int il[3] = {nl % NP, (nl / NP) % NP, nl / (NP * NP)}, ir[3] = {nr % NP, (nr / NP) % NP, nr / (NP * NP)};
            const double ml = ops.w[il[0]] * ops.w[il[1]] * ops.w[il[2]] * J;
            const double mr = ops.w[ir[0]] * ops.w[ir[1]] * ops.w[ir[2]] * J;
            for (int v = 0; v < NV; ++v) S[le].A[id][v] = wt * acc[v] - S[le].fvf[id][v];
            const double Ar = fabs(S[le].A[id][0]);
            S[le].ex[id] = (dt / ml * Ar <= kTol3 * fabs(S[le].ufv[0][nl])) && (dt / mr * Ar <= kTol3 * fabs(S[le].ufv[0][nr]));
        }
    }
    __syncthreads();
    // ---- P3: Zalesak (R7) per node
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN;
        if (e0 + le >= G.K) continue;
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        const double m = ops.w[idx[0]] * ops.w[idx[1]] * ops.w[idx[2]] * J;
        double Pp = 0.0, Pm = 0.0;
        for (int d = 0; d < 3; ++d) {
            const int pos = idx[d], row = idx[(d + 1) % 3] + NP * idx[(d + 2) % 3];
            if (pos > 0) {
                const int id = (d * NR + row) * N + pos - 1;
                const double Gv = S[le].A[id][0];
                if (!S[le].ex[id]) { Pp += Gv > 0 ? Gv : 0.0; Pm += Gv < 0 ? Gv : 0.0; }
            }
            if (pos < N) {
                const int id = (d * NR + row) * N + pos;
                const double Gv = -S[le].A[id][0];
                if (!S[le].ex[id]) { Pp += Gv > 0 ? Gv : 0.0; Pm += Gv < 0 ? Gv : 0.0; }
            }
        }
        const double rf = S[le].ufv[0][n];
        const double Qp = m / dt * (S[le].rmax[n] - rf), Qm = m / dt * (S[le].rmin[n] - rf);
        double Rp = (Pp > 0.0) ? fmin(Qp / Pp, 1.0) : 1.0, Rm = (Pm < 0.0) ? fmin(Qm / Pm, 1.0) : 1.0;
        S[le].Rp[n] = Rp > 0.0 ? Rp : 0.0;
        S[le].Rm[n] = Rm > 0.0 ? Rm : 0.0;
    }
    __syncthreads();
    // ---- P4: interface factors: Zalesak, then the pressure factor of both
    // ends with Gamma = 6
    for (int k = tid; k < EPB * NIF; k += NT) {
        const int le = k / NIF, id = k - le * NIF;
        if (e0 + le >= G.K) continue;
        double l = 1.0;
        if (A.limiting > 0) {
            const int d = id / (NR * N), r1 = id - d * NR * N, r = r1 / N, a = r1 - r * N;
            const int nl = node_of<NP>(d, r, a), nr = node_of<NP>(d, r, a + 1);
            const double *Ai = S[le].A[id];
            const double lr = S[le].ex[id] ? 1.0
                            : (-Ai[0] > 0.0) ? fmin(S[le].Rp[nl], S[le].Rm[nr]) : fmin(S[le].Rm[nl], S[le].Rp[nr]);
            const int il[3] = {nl % NP, (nl / NP) % NP, nl / (NP * NP)}, ir[3] = {nr % NP, (nr / NP) % NP, nr / (NP * NP)};
            const double ml = ops.w[il[0]] * ops.w[il[1]] * ops.w[il[2]] * J;
            const double mr = ops.w[ir[0]] * ops.w[ir[1]] * ops.w[ir[2]] * J;
            double u0[NV], av[NV];
            for (int v = 0; v < NV; ++v) { u0[v] = S[le].ufv[v][nl]; av[v] = -kGamma3 * dt / ml * Ai[v]; }
            const double thl = theta3(g, u0, av, S[le].pmin[nl], lr);
            for (int v = 0; v < NV; ++v) { u0[v] = S[le].ufv[v][nr]; av[v] = kGamma3 * dt / mr * Ai[v]; }
            const double thr = theta3(g, u0, av, S[le].pmin[nr], lr);
            l = fmin(thl, thr);
        }
        S[le].ell[id] = l;
    }
    __syncthreads();
    // ---- P5: limited update, stage combination, statistics
    unsigned vr = 0, vp = 0, np_ = 0, nact = 0;
    double am = 0.0, rmin_st = INFINITY, pmin_st = INFINITY;
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        const double m = ops.w[idx[0]] * ops.w[idx[1]] * ops.w[idx[2]] * J;
        double s[NV] = {0, 0, 0, 0, 0}, lm = 1.0;
        // the node's interfaces in a fixed order: x low, x high, y low, y high, z low, z high
        for (int d = 0; d < 3; ++d) {
            const int pos = idx[d], row = idx[(d + 1) % 3] + NP * idx[(d + 2) % 3];
            if (pos > 0) {
                const int id = (d * NR + row) * N + pos - 1;
                const double l = S[le].ell[id];
                lm = fmin(lm, l);
                for (int v = 0; v < NV; ++v) s[v] += l * S[le].A[id][v];
            }
            if (pos < N) {
                const int id = (d * NR + row) * N + pos;
                const double l = S[le].ell[id];
                lm = fmin(lm, l);
                for (int v = 0; v < NV; ++v) s[v] -= l * S[le].A[id][v];
            }
        }
        const size_t gi = (size_t)e * NN + n;
        double ut[NV];
        for (int v = 0; v < NV; ++v) {
            const double res = S[le].rfv[v][n] + s[v];
            ut[v] = S[le].ufv[v][n] + dt / m * s[v];
            double o;
            if (A.mode == 0) o = res / m;
            else if (A.comb == 1) o = 0.75 * A.un[v * KN + gi] + 0.25 * ut[v];
            else if (A.comb == 2) o = A.un[v * KN + gi] * (1.0 / 3.0) + 2.0 / 3.0 * ut[v];
            else o = ut[v];
            A.out[v * KN + gi] = o;
        }
        if (A.collect && A.limiting > 0) {
            const double p = pres3(g, ut);
            const double rl = S[le].rmin[n], rh = S[le].rmax[n], pl = S[le].pmin[n];
            if (ut[0] < rl - kViol3 * fabs(rl) || ut[0] > rh + kViol3 * fabs(rh)) vr++;
            if (p < pl - kViol3 * fabs(pl)) vp++;
            if (!(ut[0] > 0.0) || !(p > 0.0)) np_++;
            am += m * (1.0 - lm);
            if (lm < 1.0) nact++;
            rmin_st = fmin(rmin_st, ut[0]);
            pmin_st = fmin(pmin_st, p);
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
            rmin_st = fmin(rmin_st, __shfl_down_sync(FULL, rmin_st, o));
            pmin_st = fmin(pmin_st, __shfl_down_sync(FULL, pmin_st, o));
        }
        if ((tid & 31) == 0) {
            if (am > 0.0) atomicAdd(&A.stats->alpha_m, am);
            if (nact) atomicAdd(&A.stats->n_active, (unsigned long long)nact);
            if (vr) atomicAdd(&A.stats->n_vrho, (unsigned long long)vr);
            if (vp) atomicAdd(&A.stats->n_vp, (unsigned long long)vp);
            if (np_) atomicAdd(&A.stats->n_nonpos, (unsigned long long)np_);
            if (rmin_st > 0.0 && rmin_st < INFINITY) atomicMin(&A.stats->min_rho_bits, (unsigned long long)__double_as_longlong(rmin_st));
            if (pmin_st > 0.0 && pmin_st < INFINITY) atomicMin(&A.stats->min_p_bits, (unsigned long long)__double_as_longlong(pmin_st));
        }
    }
    if (A.collect && (vr | vp | np_) != 0u && (tid & 31) == 0) atomicOr(A.status, S_VIOLATION);
}

// IDP time step (Eq. timestep_restriction): per node m_i / sum_j 2 d_ij over
// its subcell and face neighbours; minimum per block, one atomic per block
template <int NP, int EPB>
__global__ void __launch_bounds__(Launch3<NP, EPB>::threads)
k_dt3d(Grid3 G, const Ops3 *__restrict__ ops_g, const double *__restrict__ u, double gamma,
       unsigned long long *dtmin, unsigned *status) {
    using E = El3<NP>;
    constexpr int N = E::N, NN = E::NN, NT = Launch3<NP, EPB>::threads;
    __shared__ double lam[EPB][3][NN];
    __shared__ double w[NP];
    __shared__ unsigned long long best_s[NT / 32];
    if (threadIdx.x < NP) w[threadIdx.x] = ops_g->w[threadIdx.x];
    const size_t KN = (size_t)G.K * NN;
    const int e0 = blockIdx.x * EPB, tid = threadIdx.x;
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        double uv[NV];
        for (int v = 0; v < NV; ++v) uv[v] = u[v * KN + (size_t)e * NN + n];
        if (!(uv[0] > 0.0) || !(pres3(gamma, uv) > 0.0)) atomicOr(status, S_BAD_INPUT);
        for (int d = 0; d < 3; ++d) lam[le][d][n] = wave3(gamma, uv, d);
    }
    __syncthreads();
    const double q[3] = {G.dy * G.dz / 4.0, G.dx * G.dz / 4.0, G.dx * G.dy / 4.0};
    const double J = G.dx * G.dy * G.dz / 8.0;
    unsigned long long best = (unsigned long long)__double_as_longlong(INFINITY);
    for (int k = tid; k < EPB * NN; k += NT) {
        const int le = k / NN, n = k - le * NN, e = e0 + le;
        if (e >= G.K) continue;
        const int idx[3] = {n % NP, (n / NP) % NP, n / (NP * NP)};
        double s2d = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double cd = w[idx[(d + 1) % 3]] * w[idx[(d + 2) % 3]] * q[d] / 2.0;
            const double li = lam[le][d][n];
            for (int side = 0; side < 2; ++side) {
                const int pos = idx[d];
                double lo;
                if (side == 0 ? pos > 0 : pos < N) {
                    const int nn2 = n + (side == 0 ? -1 : 1) * (d == 0 ? 1 : (d == 1 ? NP : NP * NP));
                    lo = lam[le][d][nn2];
                } else {
                    const int s = 2 * d + side, nb = nbr3(G, e, s);
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
                    lo = wave3(gamma, o, d);
                }
                s2d += 2.0 * cd * fmax(li, lo);
            }
        }
        const double m = w[idx[0]] * w[idx[1]] * w[idx[2]] * J;
        const double val = m / s2d;
        const unsigned long long vb = (unsigned long long)__double_as_longlong(val);
        if (val > 0.0 && vb < best) best = vb;
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
