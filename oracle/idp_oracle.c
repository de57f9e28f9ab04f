/*
 * idp_oracle.c -- plain, slow FP64 CPU oracle of the IDP-limited LGL-DGSEM
 * right-hand side and SSP-RK3 step for the 2D Euler equations on a 2:1
 * quadtree (Bolm, Rueda-Ramirez, Kuzmin, Gassner, arXiv 2607.06045).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library. It shares no code with the
 * CUDA path.
 *
 * Structure, in the paper's order:
 *   - reference operators: LGL nodes and weights (Sec. 2.1), the Lagrange
 *     basis and its derivative, Qbar = diag(w) D, Bbar, Sbar = 2 Qbar - Bbar
 *     (Sec. 2.1, volume integral);
 *   - local mortar weights by subcell overlap (Eq. local_weights, App. A);
 *   - the high-order residual in the form of Eq. evolutionformula, and the
 *     high-order subcell fluxes of Eq. fluxdifferencingform;
 *   - the low-order residual written literally in the global graph form of
 *     Eq. LowOrderScheme_globalIndices with the c/d coefficients of Sec. 2.1
 *     and, at mortars, Eq. c_nonconforming;
 *   - bar states (Sec. 2.2, IDP property), bounds (Eqs. Bounds_Positivity,
 *     Bounds_Barstates), FCT volume limiting and mortar limiting (Sec. 2.3);
 *   - the IDP time step (Eq. timestep_restriction) and SSP-RK3.
 *
 * Readings where the paper is silent (numbered as in the design notes):
 *   R1 Ranocha's entropy-conserving, kinetic-energy-preserving volume flux;
 *   R2 logarithmic mean with the Ismail-Roe series below u = 1e-4;
 *   R3 Davis wave speed lambda = max(|v_n,L| + c_L, |v_n,R| + c_R);
 *   R4 ghost states for the boundary kinds;
 *   R5 L2 mortar: interpolate, LLF on the small faces, project back
 *      (LGL-weighted adjoint of interpolation, or exact L2 projection);
 *   R6 the node itself is one of its bar states;
 *   R7 Zalesak limiting of density;
 *   R8 closed-form largest admissible factor for pressure, Gamma = 2d = 4;
 *   R9 mortar factor after the volume correction with budget n_i;
 *   R10 dt evaluated once per step;  R11 low-order CFL variant;
 *   R12 mass-/length-weighted mean limiting factors;
 *   R13 violation tolerance 1e-13 relative;
 *   R15 volume density antidiffusion below 1e-14 relative is not
 *      density-limited, and the mortar step aims at bounds relaxed by 1e-14
 *      relative, so that rounding noise (exactly cancelling high- and
 *      low-order fluxes, e.g. at the end nodes of a mortar, at a node the
 *      volume step left on its bound) cannot switch a factor between 0 and 1;
 *   R16 a mortar whose interpolated large-side states are not admissible
 *      uses its low-order flux (alpha_S = 1), as the paper reports for
 *      interpolation near vacuum (Sec. 3.2).
 *   R20 the combined limiting's indicator (Hennemann et al.'s modal energy
 *      indicator of the pressure);
 *   R21 entropy bound (Eq. Bounds_Barstates, right part): the largest
 *      factor keeping eta >= eta_min (1 - 1e-12) for the Gamma-scaled
 *      update with a margin of 1e-14 of the terms of the entropy function
 *      above rounding, found by bisection, verified;
 *   R22 low-order-solution bounds (Eq. Bounds_LowOrder): the node and its
 *      graph neighbours' low-order states; ghost states are not neighbours;
 *   R23 Chandrashekar's volume flux (the paper's astrophysical jet);
 *   R24 the jet's boundary: inflow band |y| <= 0.05 on the -x side, the
 *      ambient state elsewhere on the x sides;
 *   R25 all-to-all mortar weights by the LGL quadrature of the small face;
 *   R26 AMR transfer: interpolation (refinement), exact L2 projection
 *      (coarsening), Zhang-Shu scaling toward the parent's mean with one
 *      factor per family;
 *   R27 Loehner-type second-difference indicator.
 * Every bound interval is widened to contain the low-order value, which in
 * exact arithmetic it already does (Eq. convex_combination).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Built with -fopenmp (the all-cores CPU baseline), the loops marked
   ORC_PARALLEL run their iterations on all threads: each iteration writes
   only its own node's, interface's or element's outputs, so the results are
   the same bits as the serial build's. Every sum across iterations stays
   serial. */
#define ORC_PRAGMA(x) _Pragma(#x)
#ifdef _OPENMP
#define ORC_PARALLEL ORC_PRAGMA(omp parallel for schedule(static))
#else
#define ORC_PARALLEL
#endif

#define NPMAX 9
#define NSTAT 16

/* Work accounting. The op-counting build (opcount.cpp) compiles this file
   with a counted scalar type in place of double and defines these hooks:
   ORC_ROW(r) attributes the following arithmetic to a step of the hot path;
   ORC_PURE(id, ...) at the top of a pure function counts its arithmetic only
   the first time the function sees the same arguments within a stage
   (ORC_PURE_PAIR: the same unordered pair of states, ORC_PURE2: the same
   ordered pair), so that each distinct
   evaluation of a primitive is counted once. A state identifies as node g
   when it was fetched from the solution (ORC_TAG); evaluations on other
   states (low-order, bar, interpolated states) are all counted. ORC_SCOPE
   opens the accounting of one state at one time (a time step and its first
   stage share one). ORC_CONST(x) marks a value formed once per step (the
   time step) as a constant of the stages that use it. In this build they do
   nothing. */
enum { ROW_OTHER = 0, ROW_NODE_PREP, ROW_VOLUME_FLUX, ROW_SUBCELL_FV, ROW_FACE_FLUX, ROW_MORTAR_FLUX,
       ROW_LOW_UPDATE, ROW_BOUNDS, ROW_VOLUME_LIMIT, ROW_MORTAR_LIMIT, ROW_STAGE, ROW_DT,
       ROW_REFORM /* a quantity formed again that an earlier step already holds */,
       ROW_STATS /* statistics and violation counts, not part of the method */, ROW_COUNT };
enum { PF_PRESSURE = 1, PF_VELOCITY, PF_BETA, PF_SOUND, PF_WAVE, PF_FLUX, PF_LOGMEAN, PF_RANOCHA,
       PF_CHANDRASHEKAR, PF_LLF, PF_ETA, PF_BAR };
#define ORC_ROWS_DEFINED 1
#ifndef ORC_ROW
#define ORC_ROW(r) ((void)0)
#define ORC_PURE(...) ((void)0)
#define ORC_PURE_PAIR(...) ((void)0)
#define ORC_PURE2(...) ((void)0)
#define ORC_TAG(q, g) ((void)0)
#define ORC_TAG_N(q, g, n) ((void)0)
#define ORC_SCOPE(u, t) ((void)0)
#define ORC_CONST(x) ((void)0)
#endif
#define TOL 1e-14   /* R15: relative bound relaxation inside the limiter */

/* ------------------------------------------------------------------------ */
/* context                                                                   */
/* ------------------------------------------------------------------------ */

enum { F_CONF = 0, F_BND = 1, F_MORT_LARGE = 2, F_MORT_SMALL = 3 };
enum { BC_PERIODIC = 0, BC_WALL = 1, BC_DIRICHLET = 2, BC_OUTFLOW = 3, BC_DMR = 4, BC_JET = 5 };

typedef struct {
    int j;          /* neighbour global node index, or -1-g for ghost g */
    double cx, cy;  /* c_(i,j) */
} orc_nb;

typedef struct {
    int N, np, proj;
    double gamma;
    double xi[NPMAX], w[NPMAX];
    double D[NPMAX][NPMAX], S[NPMAX][NPMAX];
    double wt[NPMAX][2 * NPMAX];   /* local weights, reference units */
    double mw[NPMAX][2 * NPMAX];   /* weights of the low-order mortar flux: wt, or all-to-all (R25) */
    double Iint[2 * NPMAX][NPMAX]; /* interpolation large -> small nodes */
    double P[NPMAX][2 * NPMAX];    /* projection small -> large */

    /* mesh */
    int nx0, ny0;
    double x0, y0, x1, y1;
    int bc[4];
    double bc_prim[4][4], dmr_post[4], dmr_pre[4];
    int K;
    int *lev, *ix, *iy;
    double *dx, *dy, *xc, *yc;
    int *ftype;   /* [K][4] */
    int *fnbr;    /* [K][4] neighbour element or mortar id */
    int *fpos;    /* [K][4] small element position 0 lower / 1 upper */
    int M;
    int *mort;    /* [M][5]: dir(0 x,1 y), large, large_is_low(1 if large on -side), small_lo, small_hi */

    /* global node graph */
    int nn;       /* K*np*np */
    int *nb_off;  /* [nn+1] */
    orc_nb *nb;
    int ng;       /* ghost count */
    int *g_elem, *g_side, *g_t;  /* ghost owner element, side, face index */
    int *ghost_of;                /* [K][4][np] ghost index or -1 */
    int *mcount;  /* number of mortars incident on node */
    int vflux;    /* volume flux: 0 Ranocha (R1), 1 Chandrashekar (R23) */
} orc_ctx;

#ifdef ORC_COUNTING
static void orc_count_node_prep(const orc_ctx *c, const double *u);
#endif

/* ------------------------------------------------------------------------ */
/* reference operators (Sec. 2.1)                                           */
/* ------------------------------------------------------------------------ */

/* Legendre P_n and its first two derivatives by the three-term recurrence. */
static void legendre(int n, double x, double *P, double *dP, double *d2P) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { *P = 1.0; *dP = 0.0; *d2P = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1; p1 = p2;
    }
    *P = p1;
    /* derivatives for |x| < 1 from (x^2-1) P_n' = n (x P_n - P_{n-1}) and the
       Legendre equation (1-x^2) P'' - 2x P' + n(n+1) P = 0 */
    *dP = n * (x * p1 - p0) / (x * x - 1.0);
    *d2P = (2.0 * x * (*dP) - n * (n + 1.0) * p1) / (1.0 - x * x);
}

/* LGL nodes: -1, the roots of P_N' (Newton from Chebyshev-Lobatto guesses), +1;
   weights w = 2 / (N (N+1) P_N(x)^2). */
void orc_lgl(int N, double *xi, double *w) {
    xi[0] = -1.0; xi[N] = 1.0;
    for (int k = 1; k < N; ++k) {
        double x = -cos(M_PI * k / N);
        for (int it = 0; it < 100; ++it) {
            double P, dP, d2P;
            legendre(N, x, &P, &dP, &d2P);
            double dxn = dP / d2P;
            x -= dxn;
            if (fabs(dxn) < 1e-16) break;
        }
        xi[k] = x;
    }
    for (int k = 0; k <= N; ++k) {
        double P = 1.0;   /* |P_N(+-1)| = 1 */
        if (k > 0 && k < N) { double dP, d2P; legendre(N, xi[k], &P, &dP, &d2P); }
        w[k] = 2.0 / (N * (N + 1.0) * P * P);
    }
}

/* Lagrange basis phi_j(x) on the nodes xi (product definition). */
static double lagrange(int np, const double *xi, int j, double x) {
    double v = 1.0;
    for (int m = 0; m < np; ++m)
        if (m != j) v *= (x - xi[m]) / (xi[j] - xi[m]);
    return v;
}

/* phi_j'(x) by the product rule. */
static double lagrange_deriv(int np, const double *xi, int j, double x) {
    double s = 0.0;
    for (int m = 0; m < np; ++m) {
        if (m == j) continue;
        double t = 1.0 / (xi[j] - xi[m]);
        for (int l = 0; l < np; ++l)
            if (l != j && l != m) t *= (x - xi[l]) / (xi[j] - xi[l]);
        s += t;
    }
    return s;
}

/* Gauss-Legendre nodes by Newton on P_n (used only for exact L2 projection). */
static void gauss(int n, double *x, double *w) {
    for (int k = 0; k < n; ++k) {
        double t = -cos(M_PI * (k + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int m = 1; m < n; ++m) { double p2 = ((2.0 * m + 1.0) * t * p1 - m * p0) / (m + 1.0); p0 = p1; p1 = p2; }
            double dp = n * (t * p1 - p0) / (t * t - 1.0);
            double d = p1 / dp; t -= d;
            if (fabs(d) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int m = 1; m < n; ++m) { double p2 = ((2.0 * m + 1.0) * t * p1 - m * p0) / (m + 1.0); p0 = p1; p1 = p2; }
        double dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[k] = t; w[k] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* Solve A X = B (n x n, m right-hand sides) by Gaussian elimination with
   partial pivoting; A and B are overwritten. */
static void solve(int n, int m, double *A, double *B) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r) if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
            for (int k = 0; k < m; ++k) { double t = B[c * m + k]; B[c * m + k] = B[piv * m + k]; B[piv * m + k] = t; }
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = A[r * n + c] / A[c * n + c];
            for (int k = 0; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[c * m + k];
        }
    }
    for (int r = 0; r < n; ++r) for (int k = 0; k < m; ++k) B[r * m + k] /= A[r * n + r];
}

/* Operators for degree N: Sbar, local weights, mortar interpolation and
   projection (proj 0: LGL-weighted adjoint of interpolation; 1: exact L2). */
/* Local weights of Eq. local_weights (App. A) on one interface between a
   side with one face and a side with `ratio` faces (1: a conforming face,
   2: a 2:1 mortar) on the reference interval [-1, 1]: the length of the
   overlap of the LGL subcell [a_L, a_U] of node k of the single face with the
   subcell [b_L, b_U] of node l of face e of the other side, whose subcells are
   1/ratio as wide. wt[k][e np + l], np x ratio np. */
static void face_overlap_weights(int np, const double *w, int ratio, double *wt) {
    for (int k = 0; k < np; ++k) {
        double aL = -1.0, aU;
        for (int m = 0; m < k; ++m) aL += w[m];
        aU = aL + w[k];
        for (int e = 0; e < ratio; ++e) {
            for (int l = 0; l < np; ++l) {
                double bL = ratio == 1 ? -1.0 : (e == 0 ? -1.0 : 0.0), bU;
                double sc = ratio == 1 ? 1.0 : 0.5;
                for (int m = 0; m < l; ++m) bL += sc * w[m];
                bU = bL + sc * w[l];
                double lo = aL > bL ? aL : bL, hi = aU < bU ? aU : bU;
                /* subcells that only touch at a point (b_U = b_L in exact
                   arithmetic) do not overlap: rounding-level overlaps are 0 */
                wt[k * ratio * np + e * np + l] = hi - lo > 1e-13 ? hi - lo : 0.0;
            }
        }
    }
}

void orc_operators(int N, int proj, double *xi, double *w, double *D, double *S,
                   double *wt, double *Iint, double *P) {
    int np = N + 1;
    orc_lgl(N, xi, w);
    /* D_ij = phi_j'(xi_i), Qbar = diag(w) D, Bbar = diag(-1,0..0,1) */
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
            D[i * np + j] = lagrange_deriv(np, xi, j, xi[i]);
            double Q = w[i] * D[i * np + j];
            double B = (i == j) ? (i == 0 ? -1.0 : (i == N ? 1.0 : 0.0)) : 0.0;
            S[i * np + j] = 2.0 * Q - B;
        }
    /* the SBP property Qbar + Qbar^T = Bbar makes Sbar = 2 Qbar - Bbar
       skew-symmetric: its diagonal is zero exactly (rounding leaves ~1e-16) */
    for (int i = 0; i < np; ++i) S[i * np + i] = 0.0;
    /* local weights (App. A): overlap length of the LGL subcell of large node
       k and of small node (e, l), the small subcells being half as wide */
    face_overlap_weights(np, w, 2, wt);
    /* interpolation to the small-face nodes s = (xi_l -/+ 1)/2 */
    for (int e = 0; e < 2; ++e)
        for (int l = 0; l < np; ++l) {
            double s = 0.5 * (xi[l] + (e == 0 ? -1.0 : 1.0));
            for (int k = 0; k < np; ++k) Iint[(e * np + l) * np + k] = lagrange(np, xi, k, s);
        }
    if (proj == 0) {
        for (int k = 0; k < np; ++k)
            for (int e = 0; e < 2; ++e)
                for (int l = 0; l < np; ++l)
                    P[k * 2 * np + e * np + l] = 0.5 * w[l] * Iint[(e * np + l) * np + k] / w[k];
    } else {
        /* exact L2 projection with Gauss quadrature of 2N+2 points per half */
        int ng = 2 * np;
        double gx[2 * NPMAX], gw[2 * NPMAX];
        gauss(ng, gx, gw);
        double Mm[NPMAX * NPMAX], Bm[NPMAX * 2 * NPMAX];
        memset(Mm, 0, sizeof Mm); memset(Bm, 0, sizeof Bm);
        for (int q = 0; q < ng; ++q)
            for (int a = 0; a < np; ++a)
                for (int b = 0; b < np; ++b)
                    Mm[a * np + b] += gw[q] * lagrange(np, xi, a, gx[q]) * lagrange(np, xi, b, gx[q]);
        for (int e = 0; e < 2; ++e)
            for (int q = 0; q < ng; ++q) {
                double s = 0.5 * (gx[q] + (e == 0 ? -1.0 : 1.0));   /* point on the large face */
                for (int k = 0; k < np; ++k)
                    for (int l = 0; l < np; ++l)
                        Bm[k * 2 * np + e * np + l] += 0.5 * gw[q] * lagrange(np, xi, k, s) * lagrange(np, xi, l, gx[q]);
            }
        solve(np, 2 * np, Mm, Bm);
        /* P multiplies small-face nodal fluxes and gives large-face nodal
           values; the large element weights them by w_k */
        for (int k = 0; k < np; ++k)
            for (int c = 0; c < 2 * np; ++c) P[k * 2 * np + c] = Bm[k * 2 * np + c];
    }
}

/* ------------------------------------------------------------------------ */
/* Euler physics                                                            */
/* ------------------------------------------------------------------------ */

static double pressure(double g, const double *u) {
    ORC_PURE(PF_PRESSURE, u);
    return (g - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
}

/* velocity v = m / rho of a state */
static void velocity(const double *u, double *v1, double *v2) {
    ORC_PURE(PF_VELOCITY, u);
    *v1 = u[1] / u[0];
    *v2 = u[2] / u[0];
}

/* rho / p of a state */
static double rho_over_p(double g, const double *u) {
    ORC_PURE(PF_BETA, u);
    return u[0] / pressure(g, u);
}

/* speed of sound sqrt(gamma p / rho) */
static double sound_speed(double g, const double *u) {
    ORC_PURE(PF_SOUND, u);
    return sqrt(g * pressure(g, u) / u[0]);
}

/* physical flux f(u) . n for a unit normal n = (nx, ny) */
static void flux_n(double g, const double *u, double nx, double ny, double *f) {
    ORC_PURE(PF_FLUX, u, nx, ny);
    double v1, v2, p = pressure(g, u);
    velocity(u, &v1, &v2);
    double vn = v1 * nx + v2 * ny;
    f[0] = u[0] * vn;
    f[1] = u[1] * vn + p * nx;
    f[2] = u[2] * vn + p * ny;
    f[3] = (u[3] + p) * vn;
}

/* |v . n| + c of one state along the unit normal n */
static double wave_speed(double g, const double *a, double nx, double ny) {
    /* (|v . n| does not depend on the sign of n, and the negation is exact:
       the accounting treats n and -n as the same evaluation) */
    ORC_PURE(PF_WAVE, a, nx, ny);
    double va = (a[1] * nx + a[2] * ny) / a[0];
    return fabs(va) + sound_speed(g, a);
}

/* R3: Davis estimate of the maximum wave speed along n */
static double lambda_max(double g, const double *a, const double *b, double nx, double ny) {
    double la = wave_speed(g, a, nx, ny), lb = wave_speed(g, b, nx, ny);
    return la > lb ? la : lb;
}

/* One nonzero weight of the low-order interface flux (Eq. interfaceflux_local,
   Sec. 2.2): node i on the side the unit normal (nx, ny) points away from and
   node j across the interface, coupled by the weight wt (physical length;
   c_ij = wt n / 2, d_ij = aw lambda_ij / 2 with aw = |wt|, R25). Adds the
   pair's outward contributions to Fi (node i) and Fj (node j); they sum to
   zero (Eq. conservationProperty). */
static void sparse_pair_flux(double g, double wt, double aw, const double *ui, const double *uj,
                             double nx, double ny, double *Fi, double *Fj) {
    double fi[4], fj[4];
    flux_n(g, ui, nx, ny, fi); flux_n(g, uj, nx, ny, fj);
    double lam = lambda_max(g, ui, uj, nx, ny);
    for (int v = 0; v < 4; ++v) {
        Fi[v] += 0.5 * (wt * (fi[v] + fj[v]) - aw * lam * (uj[v] - ui[v]));
        Fj[v] += 0.5 * (-wt * (fi[v] + fj[v]) - aw * lam * (ui[v] - uj[v]));
    }
}

/* Bar state of the graph pair (i, j) with coefficient c_ij = (cx, cy)
   (Eq. barstateform): ubar = (u_i + u_j)/2 - c_ij . (f(u_j) - f(u_i)) / (2 d_ij),
   d_ij = |c_ij| lambda_ij. It is the same state for (j, i), c_ji = -c_ij.
   nvar: how many variables to form (1: the density alone). */
static void bar_state(double gm, const double *ui, const double *uj, double cx, double cy, int nvar,
                      double *ub) {
    ORC_PURE_PAIR(PF_BAR, ui, uj, cx, cy, nvar);
    double nrm = sqrt(cx * cx + cy * cy);
    double d = nrm * lambda_max(gm, ui, uj, cx / nrm, cy / nrm);
    double fi[4], fj[4], fiy[4], fjy[4];
    flux_n(gm, ui, 1.0, 0.0, fi); flux_n(gm, ui, 0.0, 1.0, fiy);
    flux_n(gm, uj, 1.0, 0.0, fj); flux_n(gm, uj, 0.0, 1.0, fjy);
    for (int v = 0; v < nvar; ++v) {
        double cdf = cx * (fj[v] - fi[v]) + cy * (fjy[v] - fiy[v]);
        ub[v] = 0.5 * (ui[v] + uj[v]) - cdf / (2.0 * d);
    }
}

/* local Lax-Friedrichs (Rusanov) flux along a unit normal */
void orc_llf(double g, const double *uL, const double *uR, double nx, double ny, double *f) {
    ORC_PURE2(PF_LLF, uL, uR, nx, ny);
    double fL[4], fR[4];
    flux_n(g, uL, nx, ny, fL);
    flux_n(g, uR, nx, ny, fR);
    double lam = lambda_max(g, uL, uR, nx, ny);
    for (int v = 0; v < 4; ++v) f[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

/* R2: logarithmic mean (a - b) / ln(a / b) in the Ismail-Roe form
   (a + b) / (2 F), F = ln(zeta) / (2 f), zeta = a / b, f = (zeta-1)/(zeta+1),
   with the series F = 1 + u/3 + u^2/5 + u^3/7, u = f^2, for u < 1e-4 */
double orc_logmean(double a, double b) {
    double f = (a - b) / (a + b), u = f * f;
    if (u < 1e-4) return (a + b) / (2.0 * (1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0));
    return (a - b) / log(a / b);
}

/* R1: Ranocha's EC/KEP two-point flux along the unit axis d (0 x, 1 y) */
void orc_ranocha(double g, const double *uL, const double *uR, int d, double *f) {
    ORC_PURE_PAIR(PF_RANOCHA, uL, uR, d);
    double rL = uL[0], rR = uR[0];
    double v1L, v2L, v1R, v2R;
    velocity(uL, &v1L, &v2L);
    velocity(uR, &v1R, &v2R);
    double pL = pressure(g, uL), pR = pressure(g, uR);
    double rho_ln = orc_logmean(rL, rR);
    double inv_beta = 1.0 / orc_logmean(rho_over_p(g, uL), rho_over_p(g, uR));   /* 1/{rho/p}_ln */
    double v1a = 0.5 * (v1L + v1R), v2a = 0.5 * (v2L + v2R), pa = 0.5 * (pL + pR);
    double vnL = d == 0 ? v1L : v2L, vnR = d == 0 ? v1R : v2R, vna = 0.5 * (vnL + vnR);
    double fr = rho_ln * vna;
    f[0] = fr;
    f[1] = fr * v1a + (d == 0 ? pa : 0.0);
    f[2] = fr * v2a + (d == 1 ? pa : 0.0);
    f[3] = fr * (0.5 * (v1L * v1R + v2L * v2R) + inv_beta / (g - 1.0)) + 0.5 * (pL * vnR + pR * vnL);
}

/* R23: Chandrashekar's EC/KEP two-point flux along the unit axis d, in his
   notation beta = rho / (2 p): f_rho = {rho}_ln {v_n}, f_m = f_rho {v}
   + p_hat n with p_hat = {rho} / (2 {beta}), f_E = f_rho (1 / (2 (gamma-1)
   {beta}_ln) - {|v|^2} / 2) + f_m . {v} (Sec. 3: the paper's astrophysical
   jet uses it for the volume fluxes). */
void orc_chandrashekar(double g, const double *uL, const double *uR, int d, double *f) {
    ORC_PURE_PAIR(PF_CHANDRASHEKAR, uL, uR, d);
    double rL = uL[0], rR = uR[0];
    double v1L, v2L, v1R, v2R;
    velocity(uL, &v1L, &v2L);
    velocity(uR, &v1R, &v2R);
    double pL = pressure(g, uL), pR = pressure(g, uR);
    double bL = rL / (2.0 * pL), bR = rR / (2.0 * pR);
    double rho_ln = orc_logmean(rL, rR), beta_ln = orc_logmean(bL, bR);
    double p_hat = 0.5 * (rL + rR) / (2.0 * 0.5 * (bL + bR));
    double v1a = 0.5 * (v1L + v1R), v2a = 0.5 * (v2L + v2R);
    double vna = d == 0 ? v1a : v2a;
    double v2avg = 0.5 * ((v1L * v1L + v2L * v2L) + (v1R * v1R + v2R * v2R));
    double fr = rho_ln * vna;
    f[0] = fr;
    f[1] = fr * v1a + (d == 0 ? p_hat : 0.0);
    f[2] = fr * v2a + (d == 1 ? p_hat : 0.0);
    f[3] = fr * (1.0 / (2.0 * (g - 1.0) * beta_ln) - 0.5 * v2avg) + f[1] * v1a + f[2] * v2a;
}

static void volume_flux(const orc_ctx *c, const double *uL, const double *uR, int d, double *f) {
    if (c->vflux == 1) orc_chandrashekar(c->gamma, uL, uR, d, f);
    else orc_ranocha(c->gamma, uL, uR, d, f);
}

void orc_set_volume_flux(orc_ctx *c, int k) { c->vflux = k; }

/* the weights of the low-order mortar flux, [np][2 np], reference units */
void orc_mortar_weights(const orc_ctx *c, double *out) {
    for (int a = 0; a < c->np; ++a)
        for (int b = 0; b < 2 * c->np; ++b) out[a * 2 * c->np + b] = c->mw[a][b];
}

/* ------------------------------------------------------------------------ */
/* mesh connectivity (naive: sorted leaf keys and binary search)            */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t key; int e; } leafkey;
static int cmp_key(const void *a, const void *b) {
    int64_t x = ((const leafkey *)a)->key, y = ((const leafkey *)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}
static int64_t mkkey(int l, int64_t x, int64_t y) { return ((int64_t)l << 58) | (x << 29) | y; }
static int find_leaf(const leafkey *t, int K, int l, int64_t x, int64_t y) {
    leafkey q; q.key = mkkey(l, x, y);
    const leafkey *r = bsearch(&q, t, K, sizeof(leafkey), cmp_key);
    return r ? r->e : -1;
}

void orc_destroy(orc_ctx *c) {
    if (!c) return;
    free(c->lev); free(c->ix); free(c->iy); free(c->dx); free(c->dy); free(c->xc); free(c->yc);
    free(c->ftype); free(c->fnbr); free(c->fpos); free(c->mort);
    free(c->nb_off); free(c->nb); free(c->g_elem); free(c->g_side); free(c->g_t); free(c->mcount); free(c->ghost_of);
    free(c);
}

static int gidx(const orc_ctx *c, int e, int i, int j) { return (e * c->np + j) * c->np + i; }

/* face node t of side s -> local (i, j) */
static void face_node(int np, int s, int t, int *i, int *j) {
    switch (s) {
    case 0: *i = 0; *j = t; break;
    case 1: *i = np - 1; *j = t; break;
    case 2: *i = t; *j = 0; break;
    default: *i = t; *j = np - 1; break;
    }
}

/* outward unit normal of side s */
static void side_normal(int s, double *nx, double *ny) {
    *nx = (s == 0) ? -1.0 : (s == 1 ? 1.0 : 0.0);
    *ny = (s == 2) ? -1.0 : (s == 3 ? 1.0 : 0.0);
}

static void push_nb(orc_nb **buf, int *n, int *cap, int j, double cx, double cy) {
    if (*n == *cap) { *cap = *cap ? 2 * *cap : 1024; *buf = realloc(*buf, sizeof(orc_nb) * (*cap)); }
    (*buf)[*n].j = j; (*buf)[*n].cx = cx; (*buf)[*n].cy = cy; ++*n;
}

orc_ctx *orc_create(int N, double gamma, int proj, int nx0, int ny0, double x0, double y0,
                    double x1, double y1, int K, const int8_t *level, const int32_t *ix,
                    const int32_t *iy, const int32_t *bc, const double *bc_prim,
                    const double *dmr_post, const double *dmr_pre, int a2a, int *err) {
    *err = 0;
    if (N < 1 || N + 1 > NPMAX || K < 1) { *err = 1; return NULL; }
    orc_ctx *c = calloc(1, sizeof(orc_ctx));
    c->N = N; c->np = N + 1; c->gamma = gamma; c->proj = proj;
    /* the operator routine writes dense np-strided arrays: repack to NPMAX strides */
    {
        double D[NPMAX * NPMAX], S[NPMAX * NPMAX], wt[NPMAX * 2 * NPMAX], I[2 * NPMAX * NPMAX], P[NPMAX * 2 * NPMAX];
        double xi[NPMAX], w[NPMAX];
        orc_operators(N, proj, xi, w, D, S, wt, I, P);
        int np = N + 1;
        for (int a = 0; a < np; ++a) { c->xi[a] = xi[a]; c->w[a] = w[a]; }
        for (int a = 0; a < np; ++a) for (int b = 0; b < np; ++b) { c->D[a][b] = D[a * np + b]; c->S[a][b] = S[a * np + b]; }
        for (int a = 0; a < np; ++a) for (int b = 0; b < 2 * np; ++b) { c->wt[a][b] = wt[a * 2 * np + b]; c->P[a][b] = P[a * 2 * np + b]; }
        for (int a = 0; a < 2 * np; ++a) for (int b = 0; b < np; ++b) c->Iint[a][b] = I[a * np + b];
        /* low-order mortar weights: the sparse local weights of Eq. local_weights,
           or the all-to-all weights of Eq. nonlocal_weight, omega_(i,j) =
           int_{S,N} phi_i^- phi_j^+ ds by the LGL quadrature of the small face S
           (R25): w_j |S|/2 phi_i(x_j), i.e. w_l / 2 * I[p np + l][k] in units of the
           large face's half length */
        for (int a = 0; a < np; ++a)
            for (int b = 0; b < 2 * np; ++b) {
                double x = 0.5 * w[b % np] * I[b * np + a];
                /* rounding-level values where a small-face node meets a large
                   node are zero (as R14 for the local weights) */
                if (fabs(x) < 1e-13) x = 0.0;
                c->mw[a][b] = a2a ? x : c->wt[a][b];
            }
    }
    c->nx0 = nx0; c->ny0 = ny0; c->x0 = x0; c->y0 = y0; c->x1 = x1; c->y1 = y1;
    for (int s = 0; s < 4; ++s) { c->bc[s] = bc[s]; for (int v = 0; v < 4; ++v) c->bc_prim[s][v] = bc_prim[4 * s + v]; }
    for (int v = 0; v < 4; ++v) { c->dmr_post[v] = dmr_post[v]; c->dmr_pre[v] = dmr_pre[v]; }
    c->K = K;
    c->lev = malloc(sizeof(int) * K); c->ix = malloc(sizeof(int) * K); c->iy = malloc(sizeof(int) * K);
    c->dx = malloc(sizeof(double) * K); c->dy = malloc(sizeof(double) * K);
    c->xc = malloc(sizeof(double) * K); c->yc = malloc(sizeof(double) * K);
    leafkey *tab = malloc(sizeof(leafkey) * K);
    for (int e = 0; e < K; ++e) {
        c->lev[e] = level[e]; c->ix[e] = ix[e]; c->iy[e] = iy[e];
        double n = (double)(1 << level[e]);
        c->dx[e] = (x1 - x0) / (nx0 * n); c->dy[e] = (y1 - y0) / (ny0 * n);
        c->xc[e] = x0 + (ix[e] + 0.5) * c->dx[e]; c->yc[e] = y0 + (iy[e] + 0.5) * c->dy[e];
        tab[e].key = mkkey(level[e], ix[e], iy[e]); tab[e].e = e;
    }
    qsort(tab, K, sizeof(leafkey), cmp_key);
    c->ftype = malloc(sizeof(int) * 4 * K); c->fnbr = malloc(sizeof(int) * 4 * K); c->fpos = malloc(sizeof(int) * 4 * K);
    c->mort = malloc(sizeof(int) * 5 * 4 * K);
    c->M = 0;
    for (int e = 0; e < K; ++e) for (int s = 0; s < 4; ++s) c->fpos[4 * e + s] = -1;
    /* pass 1: conforming, boundary and large-side mortar faces */
    for (int e = 0; e < K && !*err; ++e) {
        int l = c->lev[e];
        int64_t nxl = (int64_t)nx0 << l, nyl = (int64_t)ny0 << l;
        for (int s = 0; s < 4; ++s) {
            int dir = s / 2;
            int64_t qx = ix[e] + (s == 0 ? -1 : (s == 1 ? 1 : 0));
            int64_t qy = iy[e] + (s == 2 ? -1 : (s == 3 ? 1 : 0));
            int out = (qx < 0 || qx >= nxl || qy < 0 || qy >= nyl);
            if (out && bc[s] != BC_PERIODIC) { c->ftype[4 * e + s] = F_BND; c->fnbr[4 * e + s] = -1; continue; }
            qx = (qx + nxl) % nxl; qy = (qy + nyl) % nyl;
            int nb = find_leaf(tab, K, l, qx, qy);
            if (nb >= 0) { c->ftype[4 * e + s] = F_CONF; c->fnbr[4 * e + s] = nb; continue; }
            if (l > 0 && find_leaf(tab, K, l - 1, qx >> 1, qy >> 1) >= 0) {
                c->ftype[4 * e + s] = F_MORT_SMALL; c->fnbr[4 * e + s] = -1; continue;  /* filled in pass 2 */
            }
            /* two finer neighbours across the face */
            int64_t fx0, fy0, fx1, fy1;
            if (dir == 0) { fx0 = fx1 = 2 * qx + (s == 0 ? 1 : 0); fy0 = 2 * qy; fy1 = 2 * qy + 1; }
            else { fy0 = fy1 = 2 * qy + (s == 2 ? 1 : 0); fx0 = 2 * qx; fx1 = 2 * qx + 1; }
            int a = find_leaf(tab, K, l + 1, fx0, fy0), b = find_leaf(tab, K, l + 1, fx1, fy1);
            if (a < 0 || b < 0) { *err = 2; break; }   /* not 2:1 balanced, or a gap */
            int m = c->M++;
            c->mort[5 * m + 0] = dir; c->mort[5 * m + 1] = e;
            c->mort[5 * m + 2] = (s == 1 || s == 3) ? 1 : 0;  /* large on the low side */
            c->mort[5 * m + 3] = a; c->mort[5 * m + 4] = b;
            c->ftype[4 * e + s] = F_MORT_LARGE; c->fnbr[4 * e + s] = m;
        }
    }
    free(tab);
    if (*err) { orc_destroy(c); return NULL; }
    /* pass 2: small-side mortar faces */
    for (int m = 0; m < c->M; ++m) {
        int dir = c->mort[5 * m], low = c->mort[5 * m + 2];
        int s_small = dir == 0 ? (low ? 0 : 1) : (low ? 2 : 3);
        for (int p = 0; p < 2; ++p) {
            int e = c->mort[5 * m + 3 + p];
            c->ftype[4 * e + s_small] = F_MORT_SMALL; c->fnbr[4 * e + s_small] = m; c->fpos[4 * e + s_small] = p;
        }
    }
    for (int e = 0; e < K; ++e) for (int s = 0; s < 4; ++s)
        if (c->ftype[4 * e + s] == F_MORT_SMALL && c->fnbr[4 * e + s] < 0) { *err = 2; orc_destroy(c); return NULL; }

    /* global node graph with c_(i,j) (Sec. 2.1 and Eq. c_nonconforming) */
    int np = c->np;
    c->nn = K * np * np;
    c->nb_off = malloc(sizeof(int) * (c->nn + 1));
    c->mcount = calloc(c->nn, sizeof(int));
    c->g_elem = malloc(sizeof(int) * 4 * np * K); c->g_side = malloc(sizeof(int) * 4 * np * K); c->g_t = malloc(sizeof(int) * 4 * np * K);
    c->ng = 0;
    int cap = 0, cnt = 0;
    orc_nb *buf = NULL;
    /* ghost numbering first */
    int *ghost_of = malloc(sizeof(int) * 4 * np * K);
    for (int e = 0; e < K; ++e) for (int s = 0; s < 4; ++s) for (int t = 0; t < np; ++t) {
        int q = (4 * e + s) * np + t;
        ghost_of[q] = -1;
        if (c->ftype[4 * e + s] == F_BND) {
            ghost_of[q] = c->ng; c->g_elem[c->ng] = e; c->g_side[c->ng] = s; c->g_t[c->ng] = t; c->ng++;
        }
    }
    for (int e = 0; e < K; ++e) {
        for (int j = 0; j < np; ++j) for (int i = 0; i < np; ++i) {
            int g = gidx(c, e, i, j);
            c->nb_off[g] = cnt;
            double cxv = c->w[j] * c->dy[e] / 4.0, cyv = c->w[i] * c->dx[e] / 4.0;
            if (i > 0) push_nb(&buf, &cnt, &cap, gidx(c, e, i - 1, j), -cxv, 0.0);
            if (i < np - 1) push_nb(&buf, &cnt, &cap, gidx(c, e, i + 1, j), cxv, 0.0);
            if (j > 0) push_nb(&buf, &cnt, &cap, gidx(c, e, i, j - 1), 0.0, -cyv);
            if (j < np - 1) push_nb(&buf, &cnt, &cap, gidx(c, e, i, j + 1), 0.0, cyv);
            for (int s = 0; s < 4; ++s) {
                int on = (s == 0 && i == 0) || (s == 1 && i == np - 1) || (s == 2 && j == 0) || (s == 3 && j == np - 1);
                if (!on) continue;
                int t = s < 2 ? j : i;
                double nx, ny; side_normal(s, &nx, &ny);
                double half = (s < 2 ? c->dy[e] : c->dx[e]) / 2.0;   /* face Jacobian */
                int ft = c->ftype[4 * e + s];
                if (ft == F_CONF) {
                    int f = c->fnbr[4 * e + s], fi, fj;
                    face_node(np, s ^ 1, t, &fi, &fj);
                    double cc = c->w[t] * half / 2.0;
                    push_nb(&buf, &cnt, &cap, gidx(c, f, fi, fj), cc * nx, cc * ny);
                } else if (ft == F_BND) {
                    double cc = c->w[t] * half / 2.0;
                    push_nb(&buf, &cnt, &cap, -1 - ghost_of[(4 * e + s) * np + t], cc * nx, cc * ny);
                } else {
                    int m = c->fnbr[4 * e + s];
                    c->mcount[g]++;
                    int dir = c->mort[5 * m], low = c->mort[5 * m + 2];
                    int large = c->mort[5 * m + 1];
                    double halfL = (dir == 0 ? c->dy[large] : c->dx[large]) / 2.0;
                    if (ft == F_MORT_LARGE) {
                        int s_small = dir == 0 ? (low ? 0 : 1) : (low ? 2 : 3);
                        for (int p = 0; p < 2; ++p) {
                            int es = c->mort[5 * m + 3 + p];
                            for (int l = 0; l < np; ++l) {
                                double wt = c->mw[t][p * np + l];
                                if (wt == 0.0) continue;
                                int si, sj; face_node(np, s_small, l, &si, &sj);
                                double cc = wt * halfL / 2.0;
                                push_nb(&buf, &cnt, &cap, gidx(c, es, si, sj), cc * nx, cc * ny);
                            }
                        }
                    } else {
                        int p = c->fpos[4 * e + s];
                        int s_large = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2);
                        for (int k = 0; k < np; ++k) {
                            double wt = c->mw[k][p * np + t];
                            if (wt == 0.0) continue;
                            int li, lj; face_node(np, s_large, k, &li, &lj);
                            double cc = wt * halfL / 2.0;
                            push_nb(&buf, &cnt, &cap, gidx(c, large, li, lj), cc * nx, cc * ny);
                        }
                    }
                }
            }
        }
    }
    c->nb_off[c->nn] = cnt;
    c->nb = buf;
    c->ghost_of = ghost_of;
    return c;
}

int orc_n_mortars(const orc_ctx *c) { return c->M; }
void orc_mortars(const orc_ctx *c, int32_t *out) { for (int k = 0; k < 5 * c->M; ++k) out[k] = c->mort[k]; }
void orc_faces(const orc_ctx *c, int32_t *ftype, int32_t *fnbr) {
    for (int k = 0; k < 4 * c->K; ++k) { ftype[k] = c->ftype[k]; fnbr[k] = c->fnbr[k]; }
}
int orc_graph_size(const orc_ctx *c) { return c->nb_off[c->nn]; }
void orc_graph(const orc_ctx *c, int32_t *off, int32_t *nbj, double *cx, double *cy) {
    for (int g = 0; g <= c->nn; ++g) off[g] = c->nb_off[g];
    for (int k = 0; k < c->nb_off[c->nn]; ++k) { nbj[k] = c->nb[k].j; cx[k] = c->nb[k].cx; cy[k] = c->nb[k].cy; }
}

/* ------------------------------------------------------------------------ */
/* states, ghosts                                                           */
/* ------------------------------------------------------------------------ */

static void get_u(const orc_ctx *c, const double *u, int g, double *q) {
    for (int v = 0; v < 4; ++v) q[v] = u[(size_t)v * c->nn + g];
    ORC_TAG(q, g);
}

static void prim_to_cons(double gm, const double *w, double *q) {
    q[0] = w[0]; q[1] = w[0] * w[1]; q[2] = w[0] * w[2];
    q[3] = w[3] / (gm - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
}

/* R4: ghost state across boundary side s of element e at face node t */
static void ghost_state(const orc_ctx *c, const double *u, int e, int s, int t, double time, double *q) {
    int i, j; face_node(c->np, s, t, &i, &j);
    double in[4]; get_u(c, u, gidx(c, e, i, j), in);
    double nx, ny; side_normal(s, &nx, &ny);
    int kind = c->bc[s];
    double x = c->xc[e] + 0.5 * c->dx[e] * c->xi[i];
    double y = c->yc[e] + 0.5 * c->dy[e] * c->xi[j];
    if (kind == BC_JET) {
        /* R24: the jet inflow band |y| <= 0.05 of the -x side, the ambient
           state elsewhere on the x sides, outflow on the y sides */
        if (s == 0) kind = (fabs(y) <= 0.05) ? BC_DIRICHLET + 100 : BC_DIRICHLET + 200;
        else if (s == 1) kind = BC_DIRICHLET + 200;
        else kind = BC_OUTFLOW;
    }
    if (kind == BC_DMR) {
        if (s == 0) kind = BC_DIRICHLET + 100;        /* post-shock inflow */
        else if (s == 1) kind = BC_OUTFLOW;
        else if (s == 2) kind = (x < 1.0 / 6.0) ? BC_DIRICHLET + 100 : BC_WALL;
        else kind = (x < 1.0 / 6.0 + (c->y1 + 20.0 * time) / sqrt(3.0)) ? BC_DIRICHLET + 100 : BC_DIRICHLET + 200;
    }
    if (kind == BC_WALL) {
        double mn = in[1] * nx + in[2] * ny;
        q[0] = in[0]; q[1] = in[1] - 2.0 * mn * nx; q[2] = in[2] - 2.0 * mn * ny; q[3] = in[3];
    } else if (kind == BC_DIRICHLET) {
        prim_to_cons(c->gamma, c->bc_prim[s], q);
    } else if (kind == BC_DIRICHLET + 100) {
        prim_to_cons(c->gamma, c->dmr_post, q);
    } else if (kind == BC_DIRICHLET + 200) {
        prim_to_cons(c->gamma, c->dmr_pre, q);
    } else {
        for (int v = 0; v < 4; ++v) q[v] = in[v];
    }
}

static double *make_ghosts(const orc_ctx *c, const double *u, double time) {
    double *gh = malloc(sizeof(double) * 4 * (c->ng + 1));
    ORC_PARALLEL
    for (int k = 0; k < c->ng; ++k) ghost_state(c, u, c->g_elem[k], c->g_side[k], c->g_t[k], time, gh + 4 * k);
    return gh;
}

static void node_or_ghost(const orc_ctx *c, const double *u, const double *gh, int j, double *q) {
    if (j >= 0) get_u(c, u, j, q);
    else {
        for (int v = 0; v < 4; ++v) q[v] = gh[4 * (-1 - j) + v];
        ORC_TAG(q, j);
    }
}

static double mass(const orc_ctx *c, int g) {
    int np = c->np, e = g / (np * np), r = g % (np * np), i = r % np, j = r / np;
    return c->dx[e] * c->dy[e] / 4.0 * c->w[i] * c->w[j];
}

/* Mortar m: global node indices of its 3np nodes (large side first, then
   the lower and the upper small element) and the outward, mass-weighted
   low-order sparse fluxes of Eq. interfaceflux_local for each of them. */
static void mortar_nodes(const orc_ctx *c, int m, int *gnode) {
    int np = c->np;
    int dir = c->mort[5 * m], L = c->mort[5 * m + 1], low = c->mort[5 * m + 2];
    int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2), sS = sL ^ 1;
    for (int k = 0; k < np; ++k) { int li, lj; face_node(np, sL, k, &li, &lj); gnode[k] = gidx(c, L, li, lj); }
    for (int p = 0; p < 2; ++p) {
        int es = c->mort[5 * m + 3 + p];
        for (int l = 0; l < np; ++l) { int si, sj; face_node(np, sS, l, &si, &sj); gnode[np + p * np + l] = gidx(c, es, si, sj); }
    }
}

static void mortar_low(const orc_ctx *c, const double *u, int m, double Flo[][4]) {
    int np = c->np;
    double gm = c->gamma;
    int dir = c->mort[5 * m], L = c->mort[5 * m + 1], low = c->mort[5 * m + 2];
    int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2);
    double nxL, nyL; side_normal(sL, &nxL, &nyL);
    double halfL = (dir == 0 ? c->dy[L] : c->dx[L]) / 2.0;
    int gnode[3 * NPMAX];
    mortar_nodes(c, m, gnode);
    for (int q = 0; q < 3 * np; ++q) for (int v = 0; v < 4; ++v) Flo[q][v] = 0.0;
    for (int k = 0; k < np; ++k)
        for (int p = 0; p < 2; ++p)
            for (int l = 0; l < np; ++l) {
                double wt = c->mw[k][p * np + l] * halfL;
                if (wt == 0.0) continue;
                double ui[4], uj[4];
                get_u(c, u, gnode[k], ui); get_u(c, u, gnode[np + p * np + l], uj);
                /* c_ij = omega n / 2 and d_ij = |c_ij| lambda (the all-to-all
                   weights can be negative) */
                sparse_pair_flux(gm, wt, fabs(wt), ui, uj, nxL, nyL, Flo[k], Flo[np + p * np + l]);
            }
}

/* ------------------------------------------------------------------------ */
/* high-order DG residual (Eq. evolutionformula) and subcell fluxes          */
/* ------------------------------------------------------------------------ */

/* Surface fluxes of every element side, as J-weighted numerical fluxes in the
   +x (+y) direction, f_hat = (face length / 2) * flux, per face node: sf[e][s][t][v].
   Mortars use R5: interpolate, LLF on the small faces, project back. R16: a
   mortar whose interpolated large-side states are not admissible (rho <= 0
   or p <= 0) has no high-order flux; it uses its low-order sparse flux and
   is flagged in mbad (if given). */
static double *surface_fluxes_b(const orc_ctx *c, const double *u, const double *gh, char *mbad);
static double *surface_fluxes(const orc_ctx *c, const double *u, const double *gh) {
    return surface_fluxes_b(c, u, gh, NULL);
}
static double *surface_fluxes_b(const orc_ctx *c, const double *u, const double *gh, char *mbad) {
    int np = c->np, K = c->K;
    double *sf = calloc((size_t)K * 4 * np * 4, sizeof(double));
    double g = c->gamma;
    ORC_PARALLEL
    for (int e = 0; e < K; ++e)
        for (int s = 0; s < 4; ++s) {
            int ft = c->ftype[4 * e + s];
            if (ft == F_MORT_LARGE || ft == F_MORT_SMALL) continue;
            double ax = s < 2 ? 1.0 : 0.0, ay = 1.0 - ax, half = (s < 2 ? c->dy[e] : c->dx[e]) / 2.0;
            for (int t = 0; t < np; ++t) {
                int i, j; face_node(np, s, t, &i, &j);
                double in[4], out[4], f[4];
                get_u(c, u, gidx(c, e, i, j), in);
                if (ft == F_CONF) {
                    int fi, fj; face_node(np, s ^ 1, t, &fi, &fj);
                    get_u(c, u, gidx(c, c->fnbr[4 * e + s], fi, fj), out);
                } else {
                    int q = c->ghost_of[(4 * e + s) * np + t];
                    for (int v = 0; v < 4; ++v) out[v] = gh[4 * q + v];
                }
                /* left/bottom state first */
                if (s == 0 || s == 2) orc_llf(g, out, in, ax, ay, f); else orc_llf(g, in, out, ax, ay, f);
                for (int v = 0; v < 4; ++v) sf[((size_t)(4 * e + s) * np + t) * 4 + v] = half * f[v];
            }
        }
    for (int m = 0; m < c->M; ++m) {
        ORC_ROW(ROW_MORTAR_FLUX);
        int dir = c->mort[5 * m], L = c->mort[5 * m + 1], low = c->mort[5 * m + 2];
        int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2), sS = sL ^ 1;
        double ax = dir == 0 ? 1.0 : 0.0, ay = 1.0 - ax;
        double halfL = (dir == 0 ? c->dy[L] : c->dx[L]) / 2.0, halfS = halfL / 2.0;
        double fst[2 * NPMAX][4];
        int bad = 0;
        for (int p = 0; p < 2 && !bad; ++p)
            for (int l = 0; l < np; ++l) {
                double ui[4] = {0, 0, 0, 0};
                for (int k = 0; k < np; ++k) {
                    int li, lj; face_node(np, sL, k, &li, &lj);
                    double q[4]; get_u(c, u, gidx(c, L, li, lj), q);
                    for (int v = 0; v < 4; ++v) ui[v] += c->Iint[p * np + l][k] * q[v];
                }
                if (!(ui[0] > 0.0) || !(pressure(g, ui) > 0.0)) { bad = 1; break; }
            }
        if (mbad) mbad[m] = (char)bad;
        if (bad) {
            double Flo[3 * NPMAX][4];
            mortar_low(c, u, m, Flo);
            for (int k = 0; k < np; ++k)
                for (int v = 0; v < 4; ++v)
                    sf[((size_t)(4 * L + sL) * np + k) * 4 + v] = (low ? 1.0 : -1.0) * Flo[k][v] / c->w[k];
            for (int p = 0; p < 2; ++p) {
                int es = c->mort[5 * m + 3 + p];
                for (int l = 0; l < np; ++l)
                    for (int v = 0; v < 4; ++v)
                        sf[((size_t)(4 * es + sS) * np + l) * 4 + v] = (low ? -1.0 : 1.0) * Flo[np + p * np + l][v] / c->w[l];
            }
            continue;
        }
        for (int p = 0; p < 2; ++p) {
            int es = c->mort[5 * m + 3 + p];
            for (int l = 0; l < np; ++l) {
                double ui[4] = {0, 0, 0, 0}, us[4], f[4];
                for (int k = 0; k < np; ++k) {
                    int li, lj; face_node(np, sL, k, &li, &lj);
                    double q[4]; get_u(c, u, gidx(c, L, li, lj), q);
                    for (int v = 0; v < 4; ++v) ui[v] += c->Iint[p * np + l][k] * q[v];
                }
                int si, sj; face_node(np, sS, l, &si, &sj);
                get_u(c, u, gidx(c, es, si, sj), us);
                if (low) orc_llf(g, ui, us, ax, ay, f); else orc_llf(g, us, ui, ax, ay, f);
                for (int v = 0; v < 4; ++v) { fst[p * np + l][v] = f[v]; sf[((size_t)(4 * es + sS) * np + l) * 4 + v] = halfS * f[v]; }
            }
        }
        for (int k = 0; k < np; ++k)
            for (int v = 0; v < 4; ++v) {
                double acc = 0.0;
                for (int q = 0; q < 2 * np; ++q) acc += c->P[k][q] * fst[q][v];
                sf[((size_t)(4 * L + sL) * np + k) * 4 + v] = halfL * acc;
            }
    }
    ORC_ROW(ROW_FACE_FLUX);
    return sf;
}

/* mass-weighted high-order residual J w_i w_j du/dt (Eq. evolutionformula) */
static void dg_residual(const orc_ctx *c, const double *u, const double *sf, double *res) {
    int np = c->np, N = c->N;
    ORC_PARALLEL
    for (int e = 0; e < c->K; ++e)
        for (int j = 0; j < np; ++j)
            for (int i = 0; i < np; ++i) {
                double ui[4], uk[4], f[4], F1[4] = {0, 0, 0, 0}, F2[4] = {0, 0, 0, 0};
                get_u(c, u, gidx(c, e, i, j), ui);
                for (int k = 0; k < np; ++k) {
                    /* Sbar_ii = 0: the node's own pair adds nothing */
                    if (k != i) {
                        get_u(c, u, gidx(c, e, k, j), uk);
                        volume_flux(c, ui, uk, 0, f);
                        double sh = c->S[i][k] * (c->dy[e] / 2.0);
                        for (int v = 0; v < 4; ++v) F1[v] -= sh * f[v];
                    }
                    if (k != j) {
                        get_u(c, u, gidx(c, e, i, k), uk);
                        volume_flux(c, ui, uk, 1, f);
                        double sh = c->S[j][k] * (c->dx[e] / 2.0);
                        for (int v = 0; v < 4; ++v) F2[v] -= sh * f[v];
                    }
                }
                for (int v = 0; v < 4; ++v) {
                    double a = F1[v], b = F2[v];
                    if (i == 0) a += sf[((size_t)(4 * e + 0) * np + j) * 4 + v];
                    if (i == N) a -= sf[((size_t)(4 * e + 1) * np + j) * 4 + v];
                    if (j == 0) b += sf[((size_t)(4 * e + 2) * np + i) * 4 + v];
                    if (j == N) b -= sf[((size_t)(4 * e + 3) * np + i) * 4 + v];
                    res[(size_t)v * c->nn + gidx(c, e, i, j)] = c->w[j] * a + c->w[i] * b;
                }
            }
}

/* high-order subcell flux between nodes (l=a) and a+1 of a row/column
   (Eq. fluxdifferencingform), d = 0 for x rows (row index r = j), 1 for y */
/* all N high-order subcell fluxes of one row (d = 0) or column (d = 1) r of
   element e, fh[a] between nodes a and a+1: the same sums as
   dg_subcell_flux, in the same order, each extending the previous one
   (Eq. fluxdifferencingform). Sbar has a zero diagonal, so a node's own pair
   adds nothing and is skipped. */
static void dg_subcell_fluxes_row(const orc_ctx *c, const double *u, int e, int d, int r, double fh[][4]) {
    int np = c->np, N = c->N;
    double f[4], ul[4], uk[4], acc[4] = {0, 0, 0, 0};
    double half = (d == 0 ? c->dy[e] : c->dx[e]) / 2.0;
    for (int l = 0; l < N; ++l) {
        for (int k = 0; k < np; ++k) {
            if (k == l) continue;
            get_u(c, u, d == 0 ? gidx(c, e, l, r) : gidx(c, e, r, l), ul);
            get_u(c, u, d == 0 ? gidx(c, e, k, r) : gidx(c, e, r, k), uk);
            volume_flux(c, ul, uk, d, f);
            double sh = c->S[l][k] * half;
            for (int v = 0; v < 4; ++v) acc[v] += sh * f[v];
        }
        for (int v = 0; v < 4; ++v) fh[l][v] = acc[v];
    }
}

static void dg_subcell_flux(const orc_ctx *c, const double *u, int e, int d, int r, int a, double *fh) {
    int np = c->np;
    double f[4], ul[4], uk[4];
    for (int v = 0; v < 4; ++v) fh[v] = 0.0;
    double half = (d == 0 ? c->dy[e] : c->dx[e]) / 2.0;
    for (int l = 0; l <= a; ++l)
        for (int k = 0; k < np; ++k) {
            get_u(c, u, d == 0 ? gidx(c, e, l, r) : gidx(c, e, r, l), ul);
            get_u(c, u, d == 0 ? gidx(c, e, k, r) : gidx(c, e, r, k), uk);
            volume_flux(c, ul, uk, d, f);
            for (int v = 0; v < 4; ++v) fh[v] += c->S[l][k] * half * f[v];
        }
}

/* ------------------------------------------------------------------------ */
/* low-order residual in global form (Eq. LowOrderScheme_globalIndices)     */
/* ------------------------------------------------------------------------ */

static void fv_residual(const orc_ctx *c, const double *u, const double *gh, double *res, double *dsum) {
    double g = c->gamma;
    ORC_PARALLEL
    for (int i = 0; i < c->nn; ++i) {
        double ui[4], uj[4], acc[4] = {0, 0, 0, 0}, s2d = 0.0;
        get_u(c, u, i, ui);
        for (int k = c->nb_off[i]; k < c->nb_off[i + 1]; ++k) {
            const orc_nb *b = &c->nb[k];
            ORC_ROW(b->j >= 0 && b->j / (c->np * c->np) == i / (c->np * c->np) ? ROW_SUBCELL_FV
                    : b->j >= 0 && c->lev[b->j / (c->np * c->np)] != c->lev[i / (c->np * c->np)] ? ROW_MORTAR_FLUX
                    : ROW_FACE_FLUX);
            node_or_ghost(c, u, gh, b->j, uj);
            double nrm = sqrt(b->cx * b->cx + b->cy * b->cy);
            double fx[4], fy[4];
            flux_n(g, uj, 1.0, 0.0, fx);
            flux_n(g, uj, 0.0, 1.0, fy);
            double lam = lambda_max(g, ui, uj, b->cx / nrm, b->cy / nrm);
            double d = nrm * lam;
            for (int v = 0; v < 4; ++v) acc[v] += -(b->cx * fx[v] + b->cy * fy[v]) + d * (uj[v] - ui[v]);
            s2d += 2.0 * d;
        }
        ORC_ROW(ROW_SUBCELL_FV);
        for (int v = 0; v < 4; ++v) res[(size_t)v * c->nn + i] = acc[v];
        if (dsum) dsum[i] = s2d;
    }
}

/* IDP time step (Eq. timestep_restriction) or, for rule 1, the low-order CFL
   estimate (R11): min over nodes and directions of (w_i dx/2) / (|v| + c). */
double orc_dt(const orc_ctx *c, const double *u, double time, double cfl, int rule) {
    double best = INFINITY;
    ORC_SCOPE(u, time);
    ORC_ROW(ROW_DT);
    if (rule == 0) {
        double *gh = make_ghosts(c, u, time);
        double *tq = malloc(sizeof(double) * c->nn);
        ORC_PARALLEL
        for (int i = 0; i < c->nn; ++i) {
            /* sum_j 2 d_ij over the node's graph neighbours, as in the
               low-order residual */
            double ui[4], uj[4], s2d = 0.0;
            get_u(c, u, i, ui);
            for (int k = c->nb_off[i]; k < c->nb_off[i + 1]; ++k) {
                const orc_nb *b = &c->nb[k];
                node_or_ghost(c, u, gh, b->j, uj);
                double nrm = sqrt(b->cx * b->cx + b->cy * b->cy);
                double d = nrm * lambda_max(c->gamma, ui, uj, b->cx / nrm, b->cy / nrm);
                s2d += 2.0 * d;
            }
            tq[i] = mass(c, i) / s2d;
        }
        for (int i = 0; i < c->nn; ++i) if (tq[i] < best) best = tq[i];
        free(gh); free(tq);
    } else {
        int np = c->np;
        for (int i = 0; i < c->nn; ++i) {
            double q[4]; get_u(c, u, i, q);
            int e = i / (np * np), r = i % (np * np), a = r % np, b = r / np;
            double p = pressure(c->gamma, q), cs = sqrt(c->gamma * p / q[0]);
            double tx = c->w[a] * c->dx[e] / 2.0 / (fabs(q[1] / q[0]) + cs);
            double ty = c->w[b] * c->dy[e] / 2.0 / (fabs(q[2] / q[0]) + cs);
            if (tx < best) best = tx;
            if (ty < best) best = ty;
        }
    }
    return cfl * best;
}

/* ------------------------------------------------------------------------ */
/* shock indicator of the combined limiting (Sec. 3.5, Eq.                   */
/* combination_posLim_local): the modal-energy indicator of Hennemann et al.  */
/* applied to the pressure (reading R20)                                      */
/* ------------------------------------------------------------------------ */

/* alpha in [0, 1] from the nodal pressures p[j * np + i] of one element at
   the LGL nodes xi of degree N. The pressure is expanded in the orthonormal
   Legendre tensor basis, m = V^{-1} P V^{-T}; with e1 the energy of the modes
   with max(k, l) = N, e2 that of max(k, l) = N - 1 and e0 the rest, the
   energy fraction is E = max(e1 / (e0 + e1 + e2), e2 / (e0 + e2)); alpha is
   the logistic map 1 / (1 + exp(-(s / T)(E - T))) with the threshold
   T = 0.5 10^(-1.8 (N+1)^(1/4)) and s = ln((1 - 1e-4) / 1e-4), snapped to 0
   or 1 within 1e-3 of them. */
double orc_indicator(int N, const double *xi, const double *p) {
    int np = N + 1;
    double V[NPMAX * NPMAX], Vc[NPMAX * NPMAX], X[NPMAX * NPMAX], Xt[NPMAX * NPMAX];
    for (int i = 0; i < np; ++i)
        for (int k = 0; k < np; ++k) {
            double Pk, dP, d2P;
            legendre(k, xi[i], &Pk, &dP, &d2P);
            V[i * np + k] = sqrt((2.0 * k + 1.0) / 2.0) * Pk;
        }
    /* X = V^{-1} P with P[i][j] = p(x_i, y_j) */
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) X[i * np + j] = p[j * np + i];
    memcpy(Vc, V, sizeof(double) * np * np);
    solve(np, np, Vc, X);
    /* M^T = V^{-1} X^T, so Xt[l][k] = M[k][l] */
    for (int k = 0; k < np; ++k)
        for (int j = 0; j < np; ++j) Xt[j * np + k] = X[k * np + j];
    memcpy(Vc, V, sizeof(double) * np * np);
    solve(np, np, Vc, Xt);
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;
    for (int l = 0; l < np; ++l)
        for (int k = 0; k < np; ++k) {
            double m2 = Xt[l * np + k] * Xt[l * np + k];
            int top = k > l ? k : l;
            if (top == N) e1 += m2;
            else if (top == N - 1) e2 += m2;
            else e0 += m2;
        }
    double E = 0.0;
    if (e0 + e1 + e2 > 0.0) E = e1 / (e0 + e1 + e2);
    if (e0 + e2 > 0.0 && e2 / (e0 + e2) > E) E = e2 / (e0 + e2);
    double T = 0.5 * pow(10.0, -1.8 * pow(N + 1.0, 0.25));
    double sh = log((1.0 - 1e-4) / 1e-4);
    double a = 1.0 / (1.0 + exp(-sh / T * (E - T)));
    if (a < 1e-3) a = 0.0;
    if (a > 1.0 - 1e-3) a = 1.0;
    return a;
}

/* ------------------------------------------------------------------------ */
/* limiting (Sec. 2.3)                                                       */
/* ------------------------------------------------------------------------ */

/* R8: largest theta in [0, hi] such that v = u0 + theta a has rho > 0 and
   g(theta) = (gamma-1)(rho E - |m|^2/2) - pmin rho >= 0 (equivalently
   p >= pmin); the admissible set is convex, so the feasible thetas are an
   interval [0, theta*]. */
double orc_theta(double gm, const double *u0, const double *a, double pmin, double hi) {
    if (!(hi > 0.0)) return 0.0;
    double c0 = (gm - 1.0) * (u0[0] * u0[3] - 0.5 * (u0[1] * u0[1] + u0[2] * u0[2])) - pmin * u0[0];
    if (!(c0 > 0.0) || !(u0[0] > 0.0)) return 0.0;
    double c1 = (gm - 1.0) * (u0[0] * a[3] + a[0] * u0[3] - (u0[1] * a[1] + u0[2] * a[2])) - pmin * a[0];
    double c2 = (gm - 1.0) * (a[0] * a[3] - 0.5 * (a[1] * a[1] + a[2] * a[2]));
    double rho_hi = u0[0] + hi * a[0];
    double g_hi = c0 + hi * (c1 + hi * c2);
    if (rho_hi > 0.0 && g_hi >= 0.0) return hi;
    /* smallest positive root of c0 + c1 t + c2 t^2 (c0 > 0) */
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
    /* aim a relative 1e-12 inside the root so that rounding in the root and
       in the directly evaluated pressure does not cross the bound */
    double th = root < hi ? root * (1.0 - 1e-12) : hi;
    if (a[0] < 0.0) {
        double tr = -u0[0] / a[0];   /* density reaches zero */
        if (th >= tr) th = 0.5 * tr;
    }
    if (!(th > 0.0)) return 0.0;
    /* verification in FP64 against the directly evaluated pressure (R13
       tolerance): at most four halvings, then zero */
    for (int it = 0; it < 4; ++it) {
        double v[4];
        for (int k = 0; k < 4; ++k) v[k] = u0[k] + th * a[k];
        if (v[0] > 0.0 && pressure(gm, v) >= pmin * (1.0 - 1e-13)) return th;
        th *= 0.5;
    }
    return 0.0;
}

/* modified specific entropy of Eq. Bounds_Barstates: eta = p rho^-gamma / (gamma - 1) */
static double entropy_eta(double g, const double *u) {
    ORC_PURE(PF_ETA, u);
    return pressure(g, u) * pow(u[0], -g) / (g - 1.0);
}

/* relative relaxation of the entropy bound inside the limiter (R21) and the
   tolerance of the entropy violation count */
#define ETA_RELAX 1e-12
#define ETA_VIOL 1e-11

/* Psi(v) = rho e(v) - K rho(v)^gamma with rho e = E - |m|^2 / (2 rho): for
   rho > 0, Psi >= 0 exactly when eta(v) >= K. -inf where rho <= 0. */
static double entropy_psi(double g, const double *v, double K) {
    if (!(v[0] > 0.0)) return -INFINITY;
    return v[3] - 0.5 * (v[1] * v[1] + v[2] * v[2]) / v[0] - K * pow(v[0], g);
}

/* R21: the entropy factor. The target is Psi >= delta with
   delta = 1e-14 (|E_0| + K rho_0^gamma), a margin above the rounding of Psi
   (a few units in the last place of its terms), so that the decision and the
   root do not depend on that rounding; the set {Psi >= delta} is convex (Psi
   is concave), so the admissible thetas are an interval [0, theta*]. hi is
   returned when it meets the target; otherwise theta* by bisection to
   adjacent doubles, verified against Psi >= 0 and halved at most four times
   (a safeguard). */
double orc_theta_entropy(double g, const double *u0, const double *a, double K, double hi) {
    if (!(hi > 0.0) || !(u0[0] > 0.0)) return 0.0;
    const double delta = 1e-14 * (fabs(u0[3]) + K * pow(u0[0], g));
    double v[4];
    for (int k = 0; k < 4; ++k) v[k] = u0[k] + hi * a[k];
    if (entropy_psi(g, v, K) >= delta) return hi;
    if (!(entropy_psi(g, u0, K) >= delta)) return 0.0;
    double lo = 0.0, up = hi;
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + up);
        if (!(mid > lo && mid < up)) break;
        for (int k = 0; k < 4; ++k) v[k] = u0[k] + mid * a[k];
        if (entropy_psi(g, v, K) >= delta) lo = mid; else up = mid;
    }
    double th = lo;
    for (int it = 0; it < 4 && th > 0.0; ++it) {
        for (int k = 0; k < 4; ++k) v[k] = u0[k] + th * a[k];
        if (entropy_psi(g, v, K) >= 0.0) return th;
        th *= 0.5;
    }
    return 0.0;
}

double orc_entropy_eta(double g, const double *u) { return entropy_eta(g, u); }

/* optional per-mortar factor output (l_S) for inspection by the tests */
static double *g_mortar_ell = NULL;
void orc_set_mortar_ell_out(double *p) { g_mortar_ell = p; }
static double *g_mortar_dbg = NULL;   /* [M][3np][16]: node, lr, th, u0[4], av[4], rmin, rmax, pmin, n, H_rho */
void orc_set_mortar_dbg_out(double *p) { g_mortar_dbg = p; }
static double *g_node_dbg = NULL;     /* [nn][8]: rho_FV, rmin, rmax, pmin, rho_vol, lmin, R+, R- */
void orc_set_node_dbg_out(double *p) { g_node_dbg = p; }
static double *g_iface_dbg = NULL;    /* [nif][8]: gl, gr, A_rho, exempt, l_rho, theta_l, theta_r, l */
void orc_set_iface_dbg_out(double *p) { g_iface_dbg = p; }
/* Test hook: a value in [0, 1] replaces every volume interface factor and
   every mortar factor of the following stages (negative: off), so that the
   pins can compare the FCT assembly with the pure low-order (0) and the
   unlimited high-order (1) residuals. */
static double g_force_ell = -1.0;
void orc_set_force_ell(double v) { g_force_ell = v; }

/* statistics slots */
enum { ST_AVOL_M = 0, ST_M, ST_NVOL, ST_AMORT_L, ST_L, ST_NMORT, ST_VRHO, ST_VP, ST_NONPOS, ST_DTX, ST_MINRHO, ST_MINP,
       ST_VETA };

/* One limited forward-Euler stage: on return res holds the mass-weighted
   limited residual m_i du_i/dt and, if utilde != NULL, utilde the limited
   stage state u + dt/m * res written in the FCT form
   u_FV + dt/m (sum l G) + dt/m (sum_S l_S H_S).
   limiting: 0 none, 1 positivity, 2 local (bar-state density bounds),
   3 combined: per interface and per mortar the factor
   l = (1 - a) l_positivity + a l_local with a the shock indicator of the
   element (of the mortar: the largest of its three elements), Sec. 3.5
   Eq. combination_posLim_local.
   bounds (local limiting): 0 bar states (Eq. Bounds_Barstates), 1 the
   low-order solution of the node and its neighbours (Eq. Bounds_LowOrder).
   entropy (local limiting): 1 adds the lower bound on eta of the chosen kind
   of bounds (R21). */
int orc_stage(const orc_ctx *c, const double *u, double time, double dt, int limiting,
              double beta, int bounds, int entropy, double *res_out, double *utilde, double *stats) {
    int np = c->np, nn = c->nn, K = c->K, N = c->N;
    double gm = c->gamma;
    ORC_SCOPE(u, time);
#ifdef ORC_COUNTING
    orc_count_node_prep(c, u);
#endif
    ORC_ROW(ROW_FACE_FLUX);
    double *gh = make_ghosts(c, u, time);
    char *mbad = calloc(c->M + 1, 1);
    double *sf = surface_fluxes_b(c, u, gh, mbad);
    double *rdg = malloc(sizeof(double) * 4 * nn);
    if (dt == 0.0 || limiting == 0) {
        ORC_ROW(ROW_VOLUME_FLUX);
        dg_residual(c, u, sf, rdg);
        ORC_ROW(ROW_STAGE);
        free(mbad);
        for (int k = 0; k < 4 * nn; ++k) res_out[k] = rdg[k];
        if (utilde) for (int i = 0; i < nn; ++i) for (int v = 0; v < 4; ++v)
            utilde[(size_t)v * nn + i] = u[(size_t)v * nn + i] + dt / mass(c, i) * rdg[(size_t)v * nn + i];
        free(gh); free(sf); free(rdg);
        return 0;
    }
    double *rfv = malloc(sizeof(double) * 4 * nn), *ds = malloc(sizeof(double) * nn);
    fv_residual(c, u, gh, rfv, ds);
    /* low-order update */
    ORC_ROW(ROW_LOW_UPDATE);
    double *ufv = malloc(sizeof(double) * 4 * nn);
    ORC_PARALLEL
    for (int i = 0; i < nn; ++i) {
        double m = mass(c, i);
        for (int v = 0; v < 4; ++v) ufv[(size_t)v * nn + i] = u[(size_t)v * nn + i] + dt / m * rfv[(size_t)v * nn + i];
    }
    for (int i = 0; i < nn; ++i)
        if (dt * ds[i] / mass(c, i) > 1.0 && stats) stats[ST_DTX] += 1;
    /* bounds (R6 and Eqs. Bounds_Positivity, Bounds_Barstates) */
    ORC_ROW(ROW_BOUNDS);
    double *rmin = malloc(sizeof(double) * nn), *rmax = malloc(sizeof(double) * nn), *pmin = malloc(sizeof(double) * nn);
    /* combined limiting: the positivity bounds beside the local ones, and
       the indicator per element */
    const int comb = limiting == 3;
    double *rmin2 = malloc(sizeof(double) * nn), *rmax2 = malloc(sizeof(double) * nn);
    double *aind = calloc((size_t)K, sizeof(double));
    if (comb)
        for (int e = 0; e < K; ++e) {
            double pe[NPMAX * NPMAX], q[4];
            for (int n = 0; n < np * np; ++n) { get_u(c, u, e * np * np + n, q); pe[n] = pressure(gm, q); }
            aind[e] = orc_indicator(N, c->xi, pe);
        }
    /* entropy lower bound per node (R21), relaxed: K = eta_min (1 - ETA_RELAX) */
    const int ent = entropy && limiting >= 2;
    double *emin = malloc(sizeof(double) * nn);
    ORC_PARALLEL
    for (int i = 0; i < nn; ++i) {
        double ui[4], uj[4], q[4];
        get_u(c, u, i, ui);
        for (int v = 0; v < 4; ++v) q[v] = ufv[(size_t)v * nn + i];
        double lo, hi, elo;
        if (bounds == 0) {
            /* bar states ubar_(i,j) = (u_i + u_j)/2 - c_ij . (f_j - f_i) / (2 d_ij);
               the node itself is one of them (R6) */
            lo = ui[0]; hi = ui[0];
            elo = ent ? entropy_eta(gm, ui) : 0.0;
            for (int k = c->nb_off[i]; k < c->nb_off[i + 1]; ++k) {
                const orc_nb *b = &c->nb[k];
                node_or_ghost(c, u, gh, b->j, uj);
                double ub[4];
                /* the density bounds need the density alone, the entropy
                   bound the whole state */
                bar_state(gm, ui, uj, b->cx, b->cy, ent ? 4 : 1, ub);
                if (ub[0] < lo) lo = ub[0];
                if (ub[0] > hi) hi = ub[0];
                if (ent) { double eb = entropy_eta(gm, ub); if (eb < elo) elo = eb; }
            }
            if (ent) { double ef = entropy_eta(gm, q); if (ef < elo) elo = ef; }
        } else {
            /* low-order solution of the node and its neighbours (no ghosts) */
            lo = q[0]; hi = q[0];
            elo = ent ? entropy_eta(gm, q) : 0.0;
            for (int k = c->nb_off[i]; k < c->nb_off[i + 1]; ++k) {
                int j = c->nb[k].j;
                if (j < 0) continue;
                double qj[4];
                for (int v = 0; v < 4; ++v) qj[v] = ufv[(size_t)v * nn + j];
                if (qj[0] < lo) lo = qj[0];
                if (qj[0] > hi) hi = qj[0];
                if (ent) { double ej = entropy_eta(gm, qj); if (ej < elo) elo = ej; }
            }
        }
        emin[i] = elo * (1.0 - ETA_RELAX);
        if (limiting >= 2) {
            rmin[i] = lo > beta * q[0] ? lo : beta * q[0];
            rmax[i] = hi;
        } else {
            rmin[i] = beta * q[0];
            rmax[i] = INFINITY;
        }
        if (q[0] < rmin[i]) rmin[i] = q[0];
        if (q[0] > rmax[i]) rmax[i] = q[0];
        rmin2[i] = beta * q[0];
        rmax2[i] = INFINITY;
        if (q[0] < rmin2[i]) rmin2[i] = q[0];
        pmin[i] = beta * pressure(gm, q);
    }
    /* antidiffusive fluxes at interior subcell interfaces: A = F_DG - F_FV in
       the +x (+y) direction, mass-weighted; node a gets -l A, node a+1 +l A */
    int nif = K * 2 * np * N;
    double *A = malloc(sizeof(double) * 4 * nif);
    ORC_PARALLEL
    for (int e = 0; e < K; ++e)
        for (int d = 0; d < 2; ++d)
            for (int r = 0; r < np; ++r)
            {
                double fhr[NPMAX][4];
                ORC_ROW(ROW_VOLUME_FLUX);
                dg_subcell_fluxes_row(c, u, e, d, r, fhr);
                for (int a = 0; a < N; ++a) {
                    int id = ((e * 2 + d) * np + r) * N + a;
                    int gl = d == 0 ? gidx(c, e, a, r) : gidx(c, e, r, a);
                    int gr = d == 0 ? gidx(c, e, a + 1, r) : gidx(c, e, r, a + 1);
                    double *fh = fhr[a], ul[4], ur[4], fl[4], fr[4];
                    /* the low-order subcell flux again (the graph form above
                       carries the same terms: not counted twice) */
                    ORC_ROW(ROW_REFORM);
                    get_u(c, u, gl, ul); get_u(c, u, gr, ur);
                    double cc = c->w[r] * (d == 0 ? c->dy[e] : c->dx[e]) / 4.0;
                    flux_n(gm, ul, d == 0 ? 1.0 : 0.0, d == 1 ? 1.0 : 0.0, fl);
                    flux_n(gm, ur, d == 0 ? 1.0 : 0.0, d == 1 ? 1.0 : 0.0, fr);
                    double lam = lambda_max(gm, ul, ur, d == 0 ? 1.0 : 0.0, d == 1 ? 1.0 : 0.0);
                    for (int v = 0; v < 4; ++v) {
                        double ffv = cc * (fl[v] + fr[v]) - cc * lam * (ur[v] - ul[v]);
                        ORC_ROW(ROW_VOLUME_LIMIT);
                        A[4 * id + v] = c->w[r] * fh[v] - ffv;
                        ORC_ROW(ROW_REFORM);
                    }
                }
            }
    /* R15: an interface whose density antidiffusion changes neither end
       node's density by more than TOL relative is exempt from the density
       limiter (the mortar step below works on bounds relaxed by TOL) */
    ORC_ROW(ROW_VOLUME_LIMIT);
    double *tolr = malloc(sizeof(double) * nn);
    for (int i = 0; i < nn; ++i) tolr[i] = TOL * fabs(ufv[i]);
    char *exempt = malloc(nif);
    ORC_PARALLEL
    for (int e = 0; e < K; ++e)
        for (int d = 0; d < 2; ++d)
            for (int r = 0; r < np; ++r)
                for (int a = 0; a < N; ++a) {
                    int id = ((e * 2 + d) * np + r) * N + a;
                    int gl = d == 0 ? gidx(c, e, a, r) : gidx(c, e, r, a);
                    int gr = d == 0 ? gidx(c, e, a + 1, r) : gidx(c, e, r, a + 1);
                    double Ar = fabs(A[4 * id]);
                    exempt[id] = (dt / mass(c, gl) * Ar <= tolr[gl]) && (dt / mass(c, gr) * Ar <= tolr[gr]);
                }
    /* R7: Zalesak factors for density */
    double *Rp = malloc(sizeof(double) * nn), *Rm = malloc(sizeof(double) * nn);
    double *Rp2 = malloc(sizeof(double) * nn), *Rm2 = malloc(sizeof(double) * nn);
    ORC_PARALLEL
    for (int i = 0; i < nn; ++i) {
        int e = i / (np * np), rr = i % (np * np), a = rr % np, b = rr / np;
        double Pp = 0.0, Pm = 0.0;
        for (int d = 0; d < 2; ++d) {
            int pos = d == 0 ? a : b, row = d == 0 ? b : a;
            if (pos > 0) {
                int id = ((e * 2 + d) * np + row) * N + pos - 1;
                double G = A[4 * id];
                if (!exempt[id]) { Pp += G > 0 ? G : 0; Pm += G < 0 ? G : 0; }
            }
            if (pos < N) {
                int id = ((e * 2 + d) * np + row) * N + pos;
                double G = -A[4 * id];
                if (!exempt[id]) { Pp += G > 0 ? G : 0; Pm += G < 0 ? G : 0; }
            }
        }
        double m = mass(c, i), rfv = ufv[i];
        double Qp = m / dt * (rmax[i] - rfv), Qm = m / dt * (rmin[i] - rfv);
        Rp[i] = (Pp > 0.0) ? (Qp / Pp < 1.0 ? Qp / Pp : 1.0) : 1.0;
        Rm[i] = (Pm < 0.0) ? (Qm / Pm < 1.0 ? Qm / Pm : 1.0) : 1.0;
        if (Rp[i] < 0.0) Rp[i] = 0.0;
        if (Rm[i] < 0.0) Rm[i] = 0.0;
        double Qp2 = m / dt * (rmax2[i] - rfv), Qm2 = m / dt * (rmin2[i] - rfv);
        Rp2[i] = (Pp > 0.0) ? (Qp2 / Pp < 1.0 ? Qp2 / Pp : 1.0) : 1.0;
        Rm2[i] = (Pm < 0.0) ? (Qm2 / Pm < 1.0 ? Qm2 / Pm : 1.0) : 1.0;
        if (Rp2[i] < 0.0) Rp2[i] = 0.0;
        if (Rm2[i] < 0.0) Rm2[i] = 0.0;
    }
    /* R8: per interface, largest factor keeping p >= pmin at both end points
       for the Gamma-scaled single-interface update (Gamma = 2d = 4) */
    const double Gam = 4.0;
    double *ell = malloc(sizeof(double) * nif);
    double *lmin = malloc(sizeof(double) * nn);
    for (int i = 0; i < nn; ++i) lmin[i] = 1.0;
    /* (an element's interfaces touch only its own nodes' lmin) */
    ORC_PARALLEL
    for (int e = 0; e < K; ++e)
        for (int d = 0; d < 2; ++d)
            for (int r = 0; r < np; ++r)
                for (int a = 0; a < N; ++a) {
                    int id = ((e * 2 + d) * np + r) * N + a;
                    int gl = d == 0 ? gidx(c, e, a, r) : gidx(c, e, r, a);
                    int gr = d == 0 ? gidx(c, e, a + 1, r) : gidx(c, e, r, a + 1);
                    double Ar = A[4 * id];
                    /* node gl receives G = -A, node gr receives G = +A */
                    double lr = exempt[id] ? 1.0
                              : (-Ar > 0.0) ? (Rp[gl] < Rm[gr] ? Rp[gl] : Rm[gr]) : (Rm[gl] < Rp[gr] ? Rm[gl] : Rp[gr]);
                    double u0[4], av[4], th_l, th_r;
                    double ml = mass(c, gl), mr = mass(c, gr);
                    for (int v = 0; v < 4; ++v) { u0[v] = ufv[(size_t)v * nn + gl]; av[v] = -Gam * dt / ml * A[4 * id + v]; }
                    th_l = orc_theta(gm, u0, av, pmin[gl], lr);
                    if (ent) th_l = orc_theta_entropy(gm, u0, av, emin[gl], th_l);
                    for (int v = 0; v < 4; ++v) { u0[v] = ufv[(size_t)v * nn + gr]; av[v] = Gam * dt / mr * A[4 * id + v]; }
                    th_r = orc_theta(gm, u0, av, pmin[gr], lr);
                    if (ent) th_r = orc_theta_entropy(gm, u0, av, emin[gr], th_r);
                    double l = th_l < th_r ? th_l : th_r;
                    if (comb) {
                        /* positivity-only factor of the same interface, blended */
                        double lr2 = exempt[id] ? 1.0
                                   : (-Ar > 0.0) ? (Rp2[gl] < Rm2[gr] ? Rp2[gl] : Rm2[gr])
                                                 : (Rm2[gl] < Rp2[gr] ? Rm2[gl] : Rp2[gr]);
                        for (int v = 0; v < 4; ++v) { u0[v] = ufv[(size_t)v * nn + gl]; av[v] = -Gam * dt / ml * A[4 * id + v]; }
                        double t2l = orc_theta(gm, u0, av, pmin[gl], lr2);
                        for (int v = 0; v < 4; ++v) { u0[v] = ufv[(size_t)v * nn + gr]; av[v] = Gam * dt / mr * A[4 * id + v]; }
                        double t2r = orc_theta(gm, u0, av, pmin[gr], lr2);
                        double l2 = t2l < t2r ? t2l : t2r;
                        l = (1.0 - aind[e]) * l2 + aind[e] * l;
                    }
                    if (g_iface_dbg) {
                        double *o = g_iface_dbg + (size_t)id * 8;
                        o[0] = gl; o[1] = gr; o[2] = Ar; o[3] = exempt[id]; o[4] = lr; o[5] = th_l; o[6] = th_r; o[7] = l;
                    }
                    if (g_force_ell >= 0.0) l = g_force_ell;
                    ell[id] = l;
                    if (l < lmin[gl]) lmin[gl] = l;
                    if (l < lmin[gr]) lmin[gr] = l;
                }
    /* volume-corrected state u_vol = u_FV + dt/m sum l G and its residual */
    double *uvol = malloc(sizeof(double) * 4 * nn), *acc = calloc(4 * (size_t)nn, sizeof(double));
    for (int i = 0; i < nn; ++i) {
        int e = i / (np * np), rr = i % (np * np), a = rr % np, b = rr / np;
        double s[4] = {0, 0, 0, 0};
        /* sum over the node's interfaces in a fixed order: x-left, x-right, y-bottom, y-top */
        for (int d = 0; d < 2; ++d) {
            int pos = d == 0 ? a : b, row = d == 0 ? b : a;
            if (pos > 0) { int id = ((e * 2 + d) * np + row) * N + pos - 1; for (int v = 0; v < 4; ++v) s[v] += ell[id] * A[4 * id + v]; }
            if (pos < N) { int id = ((e * 2 + d) * np + row) * N + pos; for (int v = 0; v < 4; ++v) s[v] -= ell[id] * A[4 * id + v]; }
        }
        double m = mass(c, i);
        for (int v = 0; v < 4; ++v) {
            acc[(size_t)v * nn + i] = s[v];
            uvol[(size_t)v * nn + i] = ufv[(size_t)v * nn + i] + dt / m * s[v];
        }
        ORC_ROW(ROW_STATS);
        if (stats) {
            stats[ST_AVOL_M] += m * (1.0 - lmin[i]);
            stats[ST_M] += m;
            if (lmin[i] < 1.0) stats[ST_NVOL] += 1;
        }
        ORC_ROW(ROW_VOLUME_LIMIT);
    }
    if (g_node_dbg)
        for (int i = 0; i < nn; ++i) {
            double *o = g_node_dbg + (size_t)i * 8;
            o[0] = ufv[i]; o[1] = rmin[i]; o[2] = rmax[i]; o[3] = pmin[i]; o[4] = uvol[i]; o[5] = lmin[i]; o[6] = Rp[i]; o[7] = Rm[i];
        }
    /* R9: mortar limiting after the volume correction. Per mortar node, the
       high-order (R5) and low-order (Eq. interfaceflux_local) outward fluxes;
       H = -(F_L2 - F_lo) is the antidiffusive contribution. */
    double *corr = calloc(4 * (size_t)nn, sizeof(double));
    for (int m = 0; m < c->M; ++m) {
        int dir = c->mort[5 * m], L = c->mort[5 * m + 1], low = c->mort[5 * m + 2];
        int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2), sS = sL ^ 1;
        double nxL, nyL; side_normal(sL, &nxL, &nyL);
        double halfL = (dir == 0 ? c->dy[L] : c->dx[L]) / 2.0;
        int gnode[3 * NPMAX];
        double H[3 * NPMAX][4];
        mortar_nodes(c, m, gnode);
        /* low-order sparse fluxes, outward for each side (the graph form
           above carries the same terms) */
        double Flo[3 * NPMAX][4];
        ORC_ROW(ROW_REFORM);
        mortar_low(c, u, m, Flo);
        ORC_ROW(ROW_MORTAR_LIMIT);
        /* high-order outward fluxes from the surface fluxes (signs: +x-direction
           J-weighted fluxes sf; the element on the low side loses it) */
        for (int k = 0; k < np; ++k) {
            double sgn = low ? 1.0 : -1.0;
            for (int v = 0; v < 4; ++v) {
                double FL2 = sgn * c->w[k] * sf[((size_t)(4 * L + sL) * np + k) * 4 + v];
                H[k][v] = -(FL2 - Flo[k][v]);
            }
        }
        for (int p = 0; p < 2; ++p) {
            int es = c->mort[5 * m + 3 + p];
            double sgn = low ? -1.0 : 1.0;
            for (int l = 0; l < np; ++l)
                for (int v = 0; v < 4; ++v) {
                    double FL2 = sgn * c->w[l] * sf[((size_t)(4 * es + sS) * np + l) * 4 + v];
                    H[np + p * np + l][v] = -(FL2 - Flo[np + p * np + l][v]);
                }
        }
        double lS = 1.0, lS2 = 1.0;
        double am = 0.0;
        if (comb) {
            am = aind[L];
            for (int p2 = 0; p2 < 2; ++p2) if (aind[c->mort[5 * m + 3 + p2]] > am) am = aind[c->mort[5 * m + 3 + p2]];
        }
        if (mbad[m]) {
            /* R16: no admissible high-order flux, pure low order */
            for (int q = 0; q < 3 * np; ++q) for (int v = 0; v < 4; ++v) H[q][v] = 0.0;
            lS = 0.0;
        }
        for (int q = 0; q < 3 * np && !mbad[m]; ++q) {
            int i = gnode[q];
            double mi = mass(c, i), ni = (double)c->mcount[i];
            double u0[4], av[4];
            for (int v = 0; v < 4; ++v) { u0[v] = uvol[(size_t)v * nn + i]; av[v] = ni * dt / mi * H[q][v]; }
            double lr = 1.0;
            if (av[0] > 0.0) { double t = (rmax[i] + tolr[i] - u0[0]) / av[0]; if (t < lr) lr = t; }
            else if (av[0] < 0.0) { double t = (rmin[i] - tolr[i] - u0[0]) / av[0]; if (t < lr) lr = t; }
            if (lr < 0.0) lr = 0.0;
            double th = orc_theta(gm, u0, av, pmin[i] - TOL * fabs(pmin[i]), lr);
            if (ent) th = orc_theta_entropy(gm, u0, av, emin[i], th);
            if (th < lS) lS = th;
            if (comb) {
                double lr2 = 1.0;
                if (av[0] < 0.0) { double t = (rmin2[i] - tolr[i] - u0[0]) / av[0]; if (t < lr2) lr2 = t; }
                if (lr2 < 0.0) lr2 = 0.0;
                double th2 = orc_theta(gm, u0, av, pmin[i] - TOL * fabs(pmin[i]), lr2);
                if (th2 < lS2) lS2 = th2;
            }
            if (g_mortar_dbg) {
                double *o = g_mortar_dbg + ((size_t)m * 3 * np + q) * 16;
                o[0] = i; o[1] = lr; o[2] = th;
                for (int v = 0; v < 4; ++v) { o[3 + v] = u0[v]; o[7 + v] = av[v]; }
                o[11] = rmin[i]; o[12] = rmax[i]; o[13] = pmin[i]; o[14] = ni; o[15] = H[q][0];
            }
        }
        if (comb && !mbad[m]) lS = (1.0 - am) * lS2 + am * lS;
        if (g_force_ell >= 0.0) lS = g_force_ell;
        for (int q = 0; q < 3 * np; ++q) {
            int i = gnode[q];
            for (int v = 0; v < 4; ++v) corr[(size_t)v * nn + i] += lS * H[q][v];
        }
        if (g_mortar_ell) g_mortar_ell[m] = lS;
        ORC_ROW(ROW_STATS);
        if (stats) {
            stats[ST_AMORT_L] += 2.0 * halfL * (1.0 - lS);
            stats[ST_L] += 2.0 * halfL;
            if (lS < 1.0) stats[ST_NMORT] += 1;
        }
        ORC_ROW(ROW_MORTAR_LIMIT);
    }
    /* limited residual and stage state; violations (R13) */
    for (int i = 0; i < nn; ++i) {
        ORC_ROW(ROW_STAGE);
        double m = mass(c, i), q[4];
        for (int v = 0; v < 4; ++v) {
            res_out[(size_t)v * nn + i] = rfv[(size_t)v * nn + i] + acc[(size_t)v * nn + i] + corr[(size_t)v * nn + i];
            q[v] = uvol[(size_t)v * nn + i] + dt / m * corr[(size_t)v * nn + i];
            if (utilde) utilde[(size_t)v * nn + i] = q[v];
        }
        ORC_ROW(ROW_STATS);
        if (stats) {
            double p = pressure(gm, q);
            const double *lo_ = comb ? rmin2 : rmin, *hi_ = comb ? rmax2 : rmax;
            if (q[0] < lo_[i] - 1e-13 * fabs(lo_[i]) || q[0] > hi_[i] + 1e-13 * fabs(hi_[i])) stats[ST_VRHO] += 1;
            if (p < pmin[i] - 1e-13 * fabs(pmin[i])) stats[ST_VP] += 1;
            if (ent && !comb && q[0] > 0.0 && entropy_eta(gm, q) < emin[i] / (1.0 - ETA_RELAX) * (1.0 - ETA_VIOL))
                stats[ST_VETA] += 1;
            if (!(q[0] > 0.0) || !(p > 0.0)) stats[ST_NONPOS] += 1;
            if (q[0] < stats[ST_MINRHO]) stats[ST_MINRHO] = q[0];
            if (p < stats[ST_MINP]) stats[ST_MINP] = p;
        }
    }
    free(mbad); free(gh); free(sf); free(rdg); free(rfv); free(ds); free(ufv); free(rmin); free(rmax); free(pmin);
    free(A); free(Rp); free(Rm); free(tolr); free(exempt); free(ell); free(lmin); free(uvol); free(acc); free(corr);
    free(rmin2); free(rmax2); free(aind); free(Rp2); free(Rm2); free(emin);
    return 0;
}

/* threads of the OpenMP build (no effect in the serial build); returns the
   count in use */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void orc_stats_init(double *stats) {
    for (int k = 0; k < NSTAT; ++k) stats[k] = 0.0;
    stats[ST_MINRHO] = INFINITY; stats[ST_MINP] = INFINITY;
}

/* residual per unit mass: rhs = res / m */
int orc_rhs(const orc_ctx *c, const double *u, double time, double dt, int limiting, double beta,
            int bounds, int entropy, double *rhs, double *stats) {
    int rc = orc_stage(c, u, time, dt, limiting, beta, bounds, entropy, rhs, NULL, stats);
    for (int i = 0; i < c->nn; ++i) {
        double m = mass(c, i);
        for (int v = 0; v < 4; ++v) rhs[(size_t)v * c->nn + i] /= m;
    }
    return rc;
}

/* SSP-RK3 (Shu-Osher) steps with dt recomputed from u^n every step (R10).
   dt_hist receives each step's dt. */
int orc_step(const orc_ctx *c, double *u, int nsteps, double *time, double cfl, int dt_rule,
             int limiting, double beta, int bounds, int entropy, double *dt_hist, double *stats) {
    size_t n = 4 * (size_t)c->nn;
    double *u1 = malloc(sizeof(double) * n), *u2 = malloc(sizeof(double) * n), *ut = malloc(sizeof(double) * n);
    double *res = malloc(sizeof(double) * n);
    for (int s = 0; s < nsteps; ++s) {
        double dt = orc_dt(c, u, *time, cfl, dt_rule);
        ORC_CONST(dt);
        if (dt_hist) dt_hist[s] = dt;
        orc_stage(c, u, *time, dt, limiting, beta, bounds, entropy, res, ut, stats);
        ORC_PARALLEL
        for (size_t k = 0; k < n; ++k) u1[k] = ut[k];
        orc_stage(c, u1, *time + dt, dt, limiting, beta, bounds, entropy, res, ut, stats);
        ORC_ROW(ROW_STAGE);
        ORC_PARALLEL
        for (size_t k = 0; k < n; ++k) u2[k] = 0.75 * u[k] + 0.25 * ut[k];
        orc_stage(c, u2, *time + 0.5 * dt, dt, limiting, beta, bounds, entropy, res, ut, stats);
        ORC_ROW(ROW_STAGE);
        ORC_PARALLEL
        for (size_t k = 0; k < n; ++k) u[k] = u[k] / 3.0 + 2.0 / 3.0 * ut[k];
        *time += dt;
    }
    free(u1); free(u2); free(ut); free(res);
    return 0;
}

/* discrete integrals sum_i m_i u_i (conservation) */
void orc_integrals(const orc_ctx *c, const double *u, double *out) {
    for (int v = 0; v < 4; ++v) {
        double s = 0.0;
        for (int i = 0; i < c->nn; ++i) s += mass(c, i) * u[(size_t)v * c->nn + i];
        out[v] = s;
    }
}

/* --- pieces exposed for the pins --------------------------------------- */

/* high-order residual from the subcell fluxes (Eq. fluxdifferencingform) */
void orc_dg_residual_fd(const orc_ctx *c, const double *u, double time, double *res) {
    int np = c->np, N = c->N;
    double *gh = make_ghosts(c, u, time);
    double *sf = surface_fluxes(c, u, gh);
    for (int e = 0; e < c->K; ++e)
        for (int j = 0; j < np; ++j)
            for (int i = 0; i < np; ++i) {
                double fl[4], fr[4], fb[4], ft[4];
                for (int v = 0; v < 4; ++v) {
                    fl[v] = sf[((size_t)(4 * e + 0) * np + j) * 4 + v];
                    fr[v] = sf[((size_t)(4 * e + 1) * np + j) * 4 + v];
                    fb[v] = sf[((size_t)(4 * e + 2) * np + i) * 4 + v];
                    ft[v] = sf[((size_t)(4 * e + 3) * np + i) * 4 + v];
                }
                if (i > 0) dg_subcell_flux(c, u, e, 0, j, i - 1, fl);
                if (i < N) dg_subcell_flux(c, u, e, 0, j, i, fr);
                if (j > 0) dg_subcell_flux(c, u, e, 1, i, j - 1, fb);
                if (j < N) dg_subcell_flux(c, u, e, 1, i, j, ft);
                for (int v = 0; v < 4; ++v)
                    res[(size_t)v * c->nn + gidx(c, e, i, j)] = c->w[j] * (fl[v] - fr[v]) + c->w[i] * (fb[v] - ft[v]);
            }
    free(gh); free(sf);
}

/* low-order residual (mass-weighted) and sum_j 2 d_ij per node */
void orc_fv_residual(const orc_ctx *c, const double *u, double time, double *res, double *dsum) {
    double *gh = make_ghosts(c, u, time);
    fv_residual(c, u, gh, res, dsum);
    free(gh);
}

/* high-order residual (mass-weighted, Eq. evolutionformula) */
void orc_dg_residual(const orc_ctx *c, const double *u, double time, double *res) {
    double *gh = make_ghosts(c, u, time);
    double *sf = surface_fluxes(c, u, gh);
    dg_residual(c, u, sf, res);
    free(gh); free(sf);
}

/* node masses */
void orc_masses(const orc_ctx *c, double *m) { for (int i = 0; i < c->nn; ++i) m[i] = mass(c, i); }

/* Low-order interface fluxes of one interface for the pins, through the same
   weights and pair terms as the stage: the single face carries uA[np][4], the
   other side its `ratio` faces us[ratio np][4] (ratio 1: a conforming face,
   ratio 2: a mortar with the lower small face first); unit face half-length,
   normal +x, the single face on the left. Writes the outward mass-weighted
   fluxes F[(1 + ratio) np][4] (single face first) and the weights
   wt[np][ratio np] in reference units. */
void orc_face_sparse(int N, int ratio, double g, const double *uA, const double *us, double *F, double *wt) {
    double xi[NPMAX], w[NPMAX];
    int np = N + 1;
    orc_lgl(N, xi, w);
    face_overlap_weights(np, w, ratio, wt);
    for (int k = 0; k < 4 * (1 + ratio) * np; ++k) F[k] = 0.0;
    for (int k = 0; k < np; ++k)
        for (int q = 0; q < ratio * np; ++q) {
            double ww = wt[k * ratio * np + q];
            if (ww == 0.0) continue;
            sparse_pair_flux(g, ww, fabs(ww), uA + 4 * k, us + 4 * q, 1.0, 0.0, F + 4 * k, F + 4 * (np + q));
        }
}

/* the 2:1 mortar case of orc_face_sparse (Flo[3np][4]) */
void orc_mortar_sparse(int N, double g, const double *uL, const double *us, double *Flo) {
    double wt[NPMAX * 2 * NPMAX];
    orc_face_sparse(N, 2, g, uL, us, Flo, wt);
}

/* ------------------------------------------------------------------------ */
/* adaptive mesh refinement: indicators, solution transfer (Sec. 2.4,       */
/* Sec. 3); the adaptation plan itself is in oracle/amr.py                  */
/* ------------------------------------------------------------------------ */

/* R27: Loehner-type second-difference indicator of nodal values v[j][i] of
   one element: the largest, over every row and column and every three
   consecutive nodes (a, b, c), of
   |a - 2b + c| / (|c - b| + |b - a| + f (|a| + 2|b| + |c|)), f the noise
   filter (0 if the denominator is 0). */
double orc_lohner(int N, double f, const double *v) {
    int np = N + 1;
    double best = 0.0;
    if (np < 3) return 0.0;
    for (int d = 0; d < 2; ++d)
        for (int r = 0; r < np; ++r)
            for (int k = 1; k < np - 1; ++k) {
                double a, b, c;
                if (d == 0) { a = v[r * np + k - 1]; b = v[r * np + k]; c = v[r * np + k + 1]; }
                else { a = v[(k - 1) * np + r]; b = v[k * np + r]; c = v[(k + 1) * np + r]; }
                double num = fabs(a - 2.0 * b + c);
                double den = fabs(c - b) + fabs(b - a) + f * (fabs(a) + 2.0 * fabs(b) + fabs(c));
                double q = den > 0.0 ? num / den : 0.0;
                if (q > best) best = q;
            }
    return best;
}

/* R26: refinement by interpolation. parent[4][np][np] (variable, j, i) ->
   children[4 children][4][np][np], child c = cx + 2 cy covering
   [cx - 1, cx] x [cy - 1, cy] of the parent's reference square halves:
   u_c(x_i, y_j) = sum_kl phi_k(s_i) phi_l(t_j) u_p(x_k, y_l). */
void orc_refine(int N, const double *parent, double *children) {
    int np = N + 1, nn = np * np;
    double xi[NPMAX], w[NPMAX], D[NPMAX * NPMAX], S[NPMAX * NPMAX], wt[NPMAX * 2 * NPMAX], I[2 * NPMAX * NPMAX],
        P[NPMAX * 2 * NPMAX];
    orc_operators(N, 1, xi, w, D, S, wt, I, P);
    for (int c = 0; c < 4; ++c) {
        int cx = c & 1, cy = c >> 1;
        for (int v = 0; v < 4; ++v)
            for (int j = 0; j < np; ++j)
                for (int i = 0; i < np; ++i) {
                    double acc = 0.0;
                    for (int l = 0; l < np; ++l)
                        for (int k = 0; k < np; ++k)
                            acc += I[(cx * np + i) * np + k] * I[(cy * np + j) * np + l] * parent[(v * np + l) * np + k];
                    children[((c * 4 + v) * np + j) * np + i] = acc;
                }
    }
    (void)nn;
}

/* R26: coarsening by the exact L2 projection of the four children onto the
   parent's polynomials (tensor product of the 1D projections of R5). */
void orc_coarsen(int N, const double *children, double *parent) {
    int np = N + 1;
    double xi[NPMAX], w[NPMAX], D[NPMAX * NPMAX], S[NPMAX * NPMAX], wt[NPMAX * 2 * NPMAX], I[2 * NPMAX * NPMAX],
        P[NPMAX * 2 * NPMAX];
    orc_operators(N, 1, xi, w, D, S, wt, I, P);
    for (int v = 0; v < 4; ++v)
        for (int l = 0; l < np; ++l)
            for (int k = 0; k < np; ++k) {
                double acc = 0.0;
                for (int c = 0; c < 4; ++c) {
                    int cx = c & 1, cy = c >> 1;
                    for (int j = 0; j < np; ++j)
                        for (int i = 0; i < np; ++i)
                            acc += P[k * 2 * np + cx * np + i] * P[l * 2 * np + cy * np + j] *
                                   children[((c * 4 + v) * np + j) * np + i];
                }
                parent[(v * np + l) * np + k] = acc;
            }
}

/* R26: Zhang-Shu scaling of n_el elements' nodal states e[n_el][4][np][np]
   toward the reference state ref[4] (the mean of the parent before
   refinement, or of the coarsened parent): if some node has rho < eps or
   p < eps, theta_rho = min over such nodes of (rho_ref - eps) / (rho_ref -
   rho_i) scales every node, then theta_p, the smallest over the scaled
   nodes of the largest theta in [0, 1] with p(ref + theta (u_i - ref)) >=
   eps (the quadratic of R8 with pmin = eps). One common factor per call
   keeps the sum of the elements' masses. Returns the product of the two
   factors (1 when nothing was scaled). A reference state that is itself
   not admissible is left alone (returns -1). */
double orc_zhang_shu(int N, double g, int n_el, double *e, const double *ref, double eps) {
    int np = N + 1, nn = np * np;
    double pref = (g - 1.0) * (ref[3] - 0.5 * (ref[1] * ref[1] + ref[2] * ref[2]) / ref[0]);
    if (!(ref[0] > eps) || !(pref > eps)) return -1.0;
    double th1 = 1.0;
    for (int q = 0; q < n_el; ++q)
        for (int n = 0; n < nn; ++n) {
            double r = e[(size_t)(q * 4 + 0) * nn + n];
            if (r < eps) { double t = (ref[0] - eps) / (ref[0] - r); if (t < th1) th1 = t; }
        }
    if (th1 < 1.0)
        for (int q = 0; q < n_el; ++q)
            for (int v = 0; v < 4; ++v)
                for (int n = 0; n < nn; ++n) {
                    double *x = &e[(size_t)(q * 4 + v) * nn + n];
                    *x = ref[v] + th1 * (*x - ref[v]);
                }
    double th2 = 1.0;
    for (int q = 0; q < n_el; ++q)
        for (int n = 0; n < nn; ++n) {
            double a[4], u0[4];
            for (int v = 0; v < 4; ++v) { u0[v] = ref[v]; a[v] = e[(size_t)(q * 4 + v) * nn + n] - ref[v]; }
            double t = orc_theta(g, u0, a, eps, 1.0);
            if (t < th2) th2 = t;
        }
    if (th2 < 1.0)
        for (int q = 0; q < n_el; ++q)
            for (int v = 0; v < 4; ++v)
                for (int n = 0; n < nn; ++n) {
                    double *x = &e[(size_t)(q * 4 + v) * nn + n];
                    *x = ref[v] + th2 * (*x - ref[v]);
                }
    return th1 * th2;
}
