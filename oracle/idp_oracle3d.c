/*
 * idp_oracle3d.c -- plain, slow FP64 CPU oracle of the IDP-limited LGL-DGSEM
 * for the 3D Euler equations (d = 3 of Sec. 2, Eq. conservationlaw) on a
 * conforming Cartesian grid of hexahedra (Bolm, Rueda-Ramirez, Kuzmin,
 * Gassner, arXiv 2607.06045).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library. It shares no code with the
 * CUDA path. It is built together with idp_oracle.c, whose LGL operators
 * (orc_operators: nodes, weights, Sbar) and logarithmic mean (orc_logmean,
 * R2) it uses; everything three-dimensional is here.
 *
 * The method is the 2D one of the paper with the third direction added, as
 * Sec. 2 states it for d in {1, 2, 3}:
 *   - the high-order residual of Eq. evolutionformula, a sum over the three
 *     directions of the flux-differencing volume terms with Sbar and the LLF
 *     surface terms, and its subcell fluxes (Eq. fluxdifferencingform);
 *   - the low-order residual in the global graph form of
 *     Eq. LowOrderScheme_globalIndices with the c/d coefficients of Sec. 2.1,
 *     the three directions' subcell neighbours and the face neighbours;
 *   - bar states, density bounds (Eqs. Bounds_Positivity, Bounds_Barstates),
 *     Zalesak density limiting and the pressure factor with Gamma = 2d = 6
 *     (Sec. 2.3);
 *   - the IDP time step (Eq. timestep_restriction) and SSP-RK3.
 * Readings as in idp_oracle.c (R1-R3, R6-R8, R10, R13, R15, R17), with the
 * states u = (rho, rho v1, rho v2, rho v3, rho e) and
 * p = (gamma - 1)(rho e - |m|^2 / (2 rho)); the boundary kinds of R4 without
 * the 2D problem-specific ones (periodic, wall, Dirichlet, outflow).
 *
 * Layout: element e = (ez ny + ey) nx + ex, node g = ((e np + k) np + j) np + i
 * (x index i fastest), state u[5][K np^3].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NP3 9
#define NV 5
#define TOL3 1e-14   /* R15 */

/* from idp_oracle.c */
void orc_operators(int N, int proj, double *xi, double *w, double *D, double *S,
                   double *wt, double *Iint, double *P);
double orc_logmean(double a, double b);

/* Work accounting hooks, as in idp_oracle.c (the op-counting build defines
   them; here they do nothing): ORC_ROW(r) attributes the following
   arithmetic to a step of the hot path, ORC_PURE* make a pure function count
   once per distinct evaluation on solution nodes (ORC_TAG_N identifies a
   state as node g), ORC_SCOPE opens one stage's accounting and ORC_CONST
   marks the time step as a constant of the stages. */
#ifndef ORC_ROWS_DEFINED
enum { ROW_OTHER = 0, ROW_NODE_PREP, ROW_VOLUME_FLUX, ROW_SUBCELL_FV, ROW_FACE_FLUX, ROW_MORTAR_FLUX,
       ROW_LOW_UPDATE, ROW_BOUNDS, ROW_VOLUME_LIMIT, ROW_MORTAR_LIMIT, ROW_STAGE, ROW_DT,
       ROW_REFORM, ROW_STATS, ROW_COUNT };
enum { PF_PRESSURE = 1, PF_VELOCITY, PF_BETA, PF_SOUND, PF_WAVE, PF_FLUX, PF_LOGMEAN, PF_RANOCHA,
       PF_CHANDRASHEKAR, PF_LLF, PF_ETA, PF_BAR };
#endif
#ifndef ORC_ROW
#define ORC_ROW(r) ((void)0)
#define ORC_PURE(...) ((void)0)
#define ORC_PURE_PAIR(...) ((void)0)
#define ORC_PURE2(...) ((void)0)
#define ORC_TAG_N(q, g, n) ((void)0)
#define ORC_SCOPE(u, t) ((void)0)
#define ORC_CONST(x) ((void)0)
#endif

enum { B3_PERIODIC = 0, B3_WALL = 1, B3_DIRICHLET = 2, B3_OUTFLOW = 3 };
enum { S3_AVOL_M = 0, S3_M, S3_NVOL, S3_VRHO, S3_VP, S3_NONPOS, S3_DTX, S3_MINRHO, S3_MINP, S3_N };

typedef struct {
    int j;            /* neighbour node, or -1-q for ghost q */
    int face;         /* 1: across an element face, 0: a subcell neighbour */
    double c[3];      /* c_(i,j) */
} o3_nb;

typedef struct {
    int N, np, nx, ny, nz, K, nn, ng;
    double gamma;
    double xi[NP3], w[NP3], S[NP3][NP3];
    double x0, y0, z0, dx, dy, dz;
    int bc[6];
    double bc_prim[6][NV];
    int *nb_off;
    o3_nb *nb;
    int *g_node;      /* ghost q: the boundary node it mirrors */
    int *g_side;      /* and the side */
} o3_ctx;

#ifdef ORC_COUNTING
static void o3_count_node_prep(const o3_ctx *c, const double *u);
#endif

/* ------------------------------------------------------------------------ */
/* Euler physics in 3D                                                       */
/* ------------------------------------------------------------------------ */

static double pressure3(double g, const double *u) {
    ORC_PURE(PF_PRESSURE, u);
    return (g - 1.0) * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0]);
}

/* velocity v = m / rho */
static void velocity3(const double *u, double *v) {
    ORC_PURE(PF_VELOCITY, u);
    for (int a = 0; a < 3; ++a) v[a] = u[1 + a] / u[0];
}

/* rho / p */
static double beta3(double g, const double *u) {
    ORC_PURE(PF_BETA, u);
    return u[0] / pressure3(g, u);
}

/* speed of sound sqrt(gamma p / rho) */
static double sound3(double g, const double *u) {
    ORC_PURE(PF_SOUND, u);
    return sqrt(g * pressure3(g, u) / u[0]);
}

/* physical flux along axis d (0 x, 1 y, 2 z) */
static void flux3(double g, const double *u, int d, double *f) {
    ORC_PURE(PF_FLUX, u, d);
    double v[3], p = pressure3(g, u);
    velocity3(u, v);
    double vn = v[d];
    f[0] = u[0] * vn;
    for (int a = 0; a < 3; ++a) f[1 + a] = u[1 + a] * vn + (a == d ? p : 0.0);
    f[4] = (u[4] + p) * vn;
}

/* |v_d| + c */
static double wave3(double g, const double *u, int d) {
    ORC_PURE(PF_WAVE, u, d);
    double v[3];
    velocity3(u, v);
    return fabs(v[d]) + sound3(g, u);
}

/* R3: Davis estimate along axis d */
static double lambda3(double g, const double *a, const double *b, int d) {
    double la = wave3(g, a, d), lb = wave3(g, b, d);
    return la > lb ? la : lb;
}

/* LLF flux along axis d, left state first */
void o3_llf(double g, const double *uL, const double *uR, int d, double *f) {
    ORC_PURE2(PF_LLF, uL, uR, d);
    double fL[NV], fR[NV];
    flux3(g, uL, d, fL);
    flux3(g, uR, d, fR);
    double lam = lambda3(g, uL, uR, d);
    for (int v = 0; v < NV; ++v) f[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

/* R1 in 3D: Ranocha's flux along axis d,
   f_rho = {rho}_ln {v_d}, f_m = f_rho {v} + {p} e_d,
   f_E = f_rho (v_L . v_R / 2 + 1 / ((gamma - 1) {rho/p}_ln)) + (p_L v_d,R + p_R v_d,L) / 2 */
void o3_ranocha(double g, const double *uL, const double *uR, int d, double *f) {
    ORC_PURE_PAIR(PF_RANOCHA, uL, uR, d);
    double vL[3], vR[3];
    velocity3(uL, vL);
    velocity3(uR, vR);
    double pL = pressure3(g, uL), pR = pressure3(g, uR);
    double rho_ln = orc_logmean(uL[0], uR[0]);
    double bet_ln = orc_logmean(beta3(g, uL), beta3(g, uR));
    double vdot = vL[0] * vR[0] + vL[1] * vR[1] + vL[2] * vR[2];
    double fr = rho_ln * 0.5 * (vL[d] + vR[d]);
    f[0] = fr;
    for (int a = 0; a < 3; ++a) f[1 + a] = fr * 0.5 * (vL[a] + vR[a]) + (a == d ? 0.5 * (pL + pR) : 0.0);
    f[4] = fr * (0.5 * vdot + 1.0 / ((g - 1.0) * bet_ln)) + 0.5 * (pL * vR[d] + pR * vL[d]);
}

/* Density of the bar state of the pair (i, j) with c_ij along an axis
   (Eq. barstateform): rhobar = (rho_i + rho_j)/2 - c_ij . (f_rho(u_j) -
   f_rho(u_i)) / (2 d_ij), d_ij = |c_ij| lambda_ij (the density bounds need
   the density alone) */
static double bar_rho3(double g, const double *ui, const double *uj, const double *cij) {
    ORC_PURE_PAIR(PF_BAR, ui, uj, cij[0], cij[1], cij[2]);
    int d = cij[0] != 0.0 ? 0 : (cij[1] != 0.0 ? 1 : 2);
    double cn = cij[d], nrm = fabs(cn);
    double dd = nrm * lambda3(g, ui, uj, d);
    double fi[NV], fj[NV];
    flux3(g, ui, d, fi);
    flux3(g, uj, d, fj);
    return 0.5 * (ui[0] + uj[0]) - cn * (fj[0] - fi[0]) / (2.0 * dd);
}

/* R8 with 5 variables: the largest theta <= hi with rho(u0 + theta a) > 0
   and p(u0 + theta a) >= pmin, from g(theta) = (gamma-1)(rho E - |m|^2/2) -
   pmin rho (rho times p - pmin, a quadratic in theta): its smallest
   positive root, aimed 1e-12 inside, verified, halved at most four times. */
double o3_theta(double g, const double *u0, const double *a, double pmin, double hi) {
    if (!(hi > 0.0)) return 0.0;
    double gm1 = g - 1.0;
    double m0 = u0[1] * u0[1] + u0[2] * u0[2] + u0[3] * u0[3];
    double ma = u0[1] * a[1] + u0[2] * a[2] + u0[3] * a[3];
    double aa = a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
    double c0 = gm1 * (u0[0] * u0[4] - 0.5 * m0) - pmin * u0[0];
    double c1 = gm1 * (u0[0] * a[4] + a[0] * u0[4] - ma) - pmin * a[0];
    double c2 = gm1 * (a[0] * a[4] - 0.5 * aa);
    if (!(u0[0] > 0.0) || !(c0 > 0.0)) return 0.0;
    double rho_hi = u0[0] + hi * a[0], g_hi = c0 + hi * (c1 + hi * c2);
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
    for (int it = 0; it < 4; ++it) {
        double v[NV];
        for (int k = 0; k < NV; ++k) v[k] = u0[k] + th * a[k];
        if (v[0] > 0.0 && pressure3(g, v) >= pmin * (1.0 - 1e-13)) return th;
        th *= 0.5;
    }
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* mesh and node graph                                                       */
/* ------------------------------------------------------------------------ */

static int g3(const o3_ctx *c, int e, int i, int j, int k) { return ((e * c->np + k) * c->np + j) * c->np + i; }

static void push3(o3_nb **buf, int *n, int *cap, int j, int d, double cd, int face) {
    if (*n == *cap) { *cap = *cap ? 2 * *cap : 4096; *buf = realloc(*buf, sizeof(o3_nb) * (*cap)); }
    o3_nb *b = &(*buf)[*n];
    b->j = j; b->face = face; b->c[0] = b->c[1] = b->c[2] = 0.0; b->c[d] = cd;
    ++*n;
}

void o3_destroy(o3_ctx *c) {
    if (!c) return;
    free(c->nb_off); free(c->nb); free(c->g_node); free(c->g_side);
    free(c);
}

/* box = {x0, y0, z0, x1, y1, z1}; bc[6] per side; bc_prim[6][5] primitive
   Dirichlet states (rho, v1, v2, v3, p). Opposite sides are both periodic or
   neither. */
o3_ctx *o3_create(int N, double gamma, int nx, int ny, int nz, const double *box, const int32_t *bc,
                  const double *bc_prim, int *err) {
    *err = 0;
    if (N < 1 || N + 1 > NP3 || nx < 1 || ny < 1 || nz < 1) { *err = 1; return NULL; }
    for (int d = 0; d < 3; ++d)
        if ((bc[2 * d] == B3_PERIODIC) != (bc[2 * d + 1] == B3_PERIODIC)) { *err = 1; return NULL; }
    o3_ctx *c = calloc(1, sizeof(o3_ctx));
    c->N = N; c->np = N + 1; c->gamma = gamma; c->nx = nx; c->ny = ny; c->nz = nz;
    int np = N + 1;
    {
        double xi[NP3], w[NP3], D[NP3 * NP3], S[NP3 * NP3], wt[NP3 * 2 * NP3], I[2 * NP3 * NP3], P[NP3 * 2 * NP3];
        orc_operators(N, 1, xi, w, D, S, wt, I, P);
        for (int a = 0; a < np; ++a) { c->xi[a] = xi[a]; c->w[a] = w[a]; }
        for (int a = 0; a < np; ++a) for (int b = 0; b < np; ++b) c->S[a][b] = S[a * np + b];
    }
    c->x0 = box[0]; c->y0 = box[1]; c->z0 = box[2];
    c->dx = (box[3] - box[0]) / nx; c->dy = (box[4] - box[1]) / ny; c->dz = (box[5] - box[2]) / nz;
    for (int s = 0; s < 6; ++s) { c->bc[s] = bc[s]; for (int v = 0; v < NV; ++v) c->bc_prim[s][v] = bc_prim[NV * s + v]; }
    c->K = nx * ny * nz;
    c->nn = c->K * np * np * np;
    /* ghosts: one per boundary face node */
    c->g_node = malloc(sizeof(int) * 6 * np * np * (size_t)(nx * ny + ny * nz + nx * nz) + sizeof(int));
    c->g_side = malloc(sizeof(int) * 6 * np * np * (size_t)(nx * ny + ny * nz + nx * nz) + sizeof(int));
    c->nb_off = malloc(sizeof(int) * (c->nn + 1));
    o3_nb *buf = NULL;
    int cnt = 0, cap = 0;
    double area[3] = {c->dy * c->dz / 4.0, c->dx * c->dz / 4.0, c->dx * c->dy / 4.0};   /* quarter face areas */
    for (int ez = 0; ez < nz; ++ez) for (int ey = 0; ey < ny; ++ey) for (int ex = 0; ex < nx; ++ex) {
        int e = (ez * ny + ey) * nx + ex;
        int ec[3] = {ex, ey, ez}, en[3] = {nx, ny, nz};
        for (int k = 0; k < np; ++k) for (int j = 0; j < np; ++j) for (int i = 0; i < np; ++i) {
            int g = g3(c, e, i, j, k), idx[3] = {i, j, k};
            c->nb_off[g] = cnt;
            for (int d = 0; d < 3; ++d) {
                /* transverse weights of the node along direction d */
                double wt = c->w[idx[(d + 1) % 3]] * c->w[idx[(d + 2) % 3]];
                double cd = wt * area[d] / 2.0;   /* |c_ij| of the subcell and face pairs */
                int pos = idx[d];
                /* subcell neighbours (Sec. 2.1) */
                if (pos > 0) {
                    int q[3] = {i, j, k}; q[d] -= 1;
                    push3(&buf, &cnt, &cap, g3(c, e, q[0], q[1], q[2]), d, -cd, 0);
                }
                if (pos < N) {
                    int q[3] = {i, j, k}; q[d] += 1;
                    push3(&buf, &cnt, &cap, g3(c, e, q[0], q[1], q[2]), d, cd, 0);
                }
                /* face neighbours: the matching node of the element across */
                for (int side = 0; side < 2; ++side) {
                    if ((side == 0 && pos != 0) || (side == 1 && pos != N)) continue;
                    int s = 2 * d + side;
                    int nc[3] = {ec[0], ec[1], ec[2]};
                    nc[d] += side == 0 ? -1 : 1;
                    int out = nc[d] < 0 || nc[d] >= en[d];
                    double cs = side == 0 ? -cd : cd;
                    if (out && bc[s] != B3_PERIODIC) {
                        c->g_node[c->ng] = g; c->g_side[c->ng] = s;
                        push3(&buf, &cnt, &cap, -1 - c->ng, d, cs, 1);
                        c->ng++;
                        continue;
                    }
                    nc[d] = (nc[d] + en[d]) % en[d];
                    int f = (nc[2] * ny + nc[1]) * nx + nc[0];
                    int q[3] = {i, j, k}; q[d] = side == 0 ? N : 0;
                    push3(&buf, &cnt, &cap, g3(c, f, q[0], q[1], q[2]), d, cs, 1);
                }
            }
        }
    }
    c->nb_off[c->nn] = cnt;
    c->nb = buf;
    return c;
}

int o3_n_nodes(const o3_ctx *c) { return c->nn; }

static double mass3(const o3_ctx *c, int g) {
    int np = c->np, i = g % np, j = (g / np) % np, k = (g / (np * np)) % np;
    return c->w[i] * c->w[j] * c->w[k] * c->dx * c->dy * c->dz / 8.0;
}

static void get3(const o3_ctx *c, const double *u, int g, double *q) {
    for (int v = 0; v < NV; ++v) q[v] = u[(size_t)v * c->nn + g];
    ORC_TAG_N(q, g, NV);
}

static void prim_cons3(double g, const double *w, double *q) {
    q[0] = w[0];
    for (int a = 0; a < 3; ++a) q[1 + a] = w[0] * w[1 + a];
    q[4] = w[4] / (g - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

/* R4: the ghost state across boundary side s of the boundary node's state */
static void ghost3(const o3_ctx *c, const double *in, int s, double *q) {
    int kind = c->bc[s], d = s / 2;
    if (kind == B3_WALL) {
        for (int v = 0; v < NV; ++v) q[v] = in[v];
        q[1 + d] = -in[1 + d];
    } else if (kind == B3_DIRICHLET) {
        prim_cons3(c->gamma, c->bc_prim[s], q);
    } else {
        for (int v = 0; v < NV; ++v) q[v] = in[v];
    }
}

static void node_or_ghost3(const o3_ctx *c, const double *u, int j, double *q) {
    if (j >= 0) { get3(c, u, j, q); return; }
    int gq = -1 - j;
    double in[NV];
    get3(c, u, c->g_node[gq], in);
    ghost3(c, in, c->g_side[gq], q);
}

/* ------------------------------------------------------------------------ */
/* residuals                                                                 */
/* ------------------------------------------------------------------------ */

/* mass-weighted high-order residual (Eq. evolutionformula in 3D): per node
   sum over d of (transverse weights) ( -sum_l Sbar_(pos,l) (A_d/4) f*_d(u, u_l)
   + surface LLF terms at the element's faces ) */
static void dg_residual3(const o3_ctx *c, const double *u, double *res) {
    int np = c->np, N = c->N;
    double g = c->gamma;
    double area[3] = {c->dy * c->dz / 4.0, c->dx * c->dz / 4.0, c->dx * c->dy / 4.0};
    for (int e = 0; e < c->K; ++e)
        for (int k = 0; k < np; ++k) for (int j = 0; j < np; ++j) for (int i = 0; i < np; ++i) {
            int gi = g3(c, e, i, j, k), idx[3] = {i, j, k};
            double ui[NV], tot[NV] = {0, 0, 0, 0, 0};
            get3(c, u, gi, ui);
            for (int d = 0; d < 3; ++d) {
                double F[NV] = {0, 0, 0, 0, 0};
                int pos = idx[d];
                for (int l = 0; l < np; ++l) {
                    if (l == pos) continue;   /* Sbar has a zero diagonal */
                    int q[3] = {i, j, k}; q[d] = l;
                    double ul[NV], f[NV];
                    get3(c, u, g3(c, e, q[0], q[1], q[2]), ul);
                    o3_ranocha(g, ui, ul, d, f);
                    for (int v = 0; v < NV; ++v) F[v] -= c->S[pos][l] * area[d] * f[v];
                }
                /* surface terms: the graph holds two entries per direction
                   (pushed low, high, then the face), so at pos 0 or N the
                   face neighbour is the direction's second entry */
                for (int side = 0; side < 2; ++side) {
                    if ((side == 0 && pos != 0) || (side == 1 && pos != N)) continue;
                    double out[NV], f[NV];
                    node_or_ghost3(c, u, c->nb[c->nb_off[gi] + 2 * d + 1].j, out);
                    if (side == 0) { o3_llf(g, out, ui, d, f); for (int v = 0; v < NV; ++v) F[v] += area[d] * f[v]; }
                    else { o3_llf(g, ui, out, d, f); for (int v = 0; v < NV; ++v) F[v] -= area[d] * f[v]; }
                }
                double wt = c->w[idx[(d + 1) % 3]] * c->w[idx[(d + 2) % 3]];
                for (int v = 0; v < NV; ++v) tot[v] += wt * F[v];
            }
            for (int v = 0; v < NV; ++v) res[(size_t)v * c->nn + gi] = tot[v];
        }
}

/* high-order subcell fluxes of one row along d (Eq. fluxdifferencingform):
   fh[l] between nodes l and l+1 = sum_{a <= l} sum_m Sbar_am (A_d/4) f*_d(u_a, u_m);
   the row is fixed by the node (i, j, k) with its d index ignored */
static void dg_subcell_row3(const o3_ctx *c, const double *u, int e, int d, const int *idx, double fh[][NV]) {
    int np = c->np, N = c->N;
    double area[3] = {c->dy * c->dz / 4.0, c->dx * c->dz / 4.0, c->dx * c->dy / 4.0};
    double acc[NV] = {0, 0, 0, 0, 0};
    for (int l = 0; l < N; ++l) {
        int qa[3] = {idx[0], idx[1], idx[2]}; qa[d] = l;
        double ua[NV];
        get3(c, u, g3(c, e, qa[0], qa[1], qa[2]), ua);
        for (int m = 0; m < np; ++m) {
            if (m == l) continue;
            int qm[3] = {idx[0], idx[1], idx[2]}; qm[d] = m;
            double um[NV], f[NV];
            get3(c, u, g3(c, e, qm[0], qm[1], qm[2]), um);
            o3_ranocha(c->gamma, ua, um, d, f);
            for (int v = 0; v < NV; ++v) acc[v] += c->S[l][m] * area[d] * f[v];
        }
        for (int v = 0; v < NV; ++v) fh[l][v] = acc[v];
    }
}

/* low-order residual in the global graph form (Eq. LowOrderScheme_globalIndices):
   sum_j -c_ij . f(u_j) + d_ij (u_j - u_i); dsum = sum_j 2 d_ij */
static void fv_residual3(const o3_ctx *c, const double *u, double *res, double *dsum) {
    double g = c->gamma;
    for (int i = 0; i < c->nn; ++i) {
        double ui[NV], acc[NV] = {0, 0, 0, 0, 0}, s2d = 0.0;
        get3(c, u, i, ui);
        for (int b = c->nb_off[i]; b < c->nb_off[i + 1]; ++b) {
            const o3_nb *nb = &c->nb[b];
            int d = nb->c[0] != 0.0 ? 0 : (nb->c[1] != 0.0 ? 1 : 2);
            ORC_ROW(nb->face ? ROW_FACE_FLUX : ROW_SUBCELL_FV);
            double uj[NV], f[NV];
            node_or_ghost3(c, u, nb->j, uj);
            flux3(g, uj, d, f);
            double dd = fabs(nb->c[d]) * lambda3(g, ui, uj, d);
            for (int v = 0; v < NV; ++v) acc[v] += -nb->c[d] * f[v] + dd * (uj[v] - ui[v]);
            s2d += 2.0 * dd;
        }
        for (int v = 0; v < NV; ++v) res[(size_t)v * c->nn + i] = acc[v];
        if (dsum) dsum[i] = s2d;
    }
}

/* IDP time step (Eq. timestep_restriction): cfl * min_i m_i / sum_j 2 d_ij */
double o3_dt(const o3_ctx *c, const double *u, double cfl) {
    ORC_SCOPE(u, 0.0);
    ORC_ROW(ROW_DT);
    double best = INFINITY;
    for (int i = 0; i < c->nn; ++i) {
        double ui[NV], uj[NV], s2d = 0.0;
        get3(c, u, i, ui);
        for (int b = c->nb_off[i]; b < c->nb_off[i + 1]; ++b) {
            const o3_nb *nb = &c->nb[b];
            int d = nb->c[0] != 0.0 ? 0 : (nb->c[1] != 0.0 ? 1 : 2);
            node_or_ghost3(c, u, nb->j, uj);
            s2d += 2.0 * (fabs(nb->c[d]) * lambda3(c->gamma, ui, uj, d));
        }
        double t = mass3(c, i) / s2d;
        if (t < best) best = t;
    }
    return cfl * best;
}

/* ------------------------------------------------------------------------ */
/* one limited stage (Sec. 2.3 with Gamma = 2d = 6)                          */
/* ------------------------------------------------------------------------ */

static double g_force3 = -1.0;
/* test hook: every factor replaced by v in [0, 1] (v < 0: off) */
void o3_set_force_ell(double v) { g_force3 = v; }
/* test hooks: per node [u_FV (5), rho_min, rho_max, p_min, R+, R-] and per
   interface [left node, right node, exempt, Zalesak factor, theta_left,
   theta_right, factor, A (5)] of the next limited stage */
static double *g_node3 = NULL, *g_iface3 = NULL;
void o3_set_dbg_out(double *node, double *iface) { g_node3 = node; g_iface3 = iface; }

/* interface id of the subcell interface between positions a and a+1 along d
   in the row of node idx of element e */
static int iface3(const o3_ctx *c, int e, int d, const int *idx, int a) {
    int np = c->np, N = c->N;
    int r = idx[(d + 1) % 3] + np * idx[(d + 2) % 3];
    return ((e * 3 + d) * np * np + r) * N + a;
}

int o3_stage(const o3_ctx *c, const double *u, double dt, int limiting, double beta, double *res_out,
             double *utilde, double *stats) {
    int np = c->np, nn = c->nn, K = c->K, N = c->N;
    double gm = c->gamma;
    ORC_SCOPE(u, 0.0);
#ifdef ORC_COUNTING
    o3_count_node_prep(c, u);
#endif
    double *rdg = malloc(sizeof(double) * NV * (size_t)nn);
    if (dt == 0.0 || limiting == 0) {
        dg_residual3(c, u, rdg);
        for (size_t k = 0; k < (size_t)NV * nn; ++k) res_out[k] = rdg[k];
        if (utilde)
            for (int i = 0; i < nn; ++i) for (int v = 0; v < NV; ++v)
                utilde[(size_t)v * nn + i] = u[(size_t)v * nn + i] + dt / mass3(c, i) * rdg[(size_t)v * nn + i];
        free(rdg);
        return 0;
    }
    double *rfv = malloc(sizeof(double) * NV * (size_t)nn), *ds = malloc(sizeof(double) * nn);
    fv_residual3(c, u, rfv, ds);
    double *ufv = malloc(sizeof(double) * NV * (size_t)nn);
    ORC_ROW(ROW_LOW_UPDATE);
    for (int i = 0; i < nn; ++i) {
        double m = mass3(c, i);
        for (int v = 0; v < NV; ++v) ufv[(size_t)v * nn + i] = u[(size_t)v * nn + i] + dt / m * rfv[(size_t)v * nn + i];
        if (dt * ds[i] / m > 1.0 && stats) stats[S3_DTX] += 1;
    }
    /* bounds (R6): bar states of every graph neighbour, the node itself
       included; positivity bounds beta rho_FV, beta p_FV */
    double *rmin = malloc(sizeof(double) * nn), *rmax = malloc(sizeof(double) * nn), *pmin = malloc(sizeof(double) * nn);
    ORC_ROW(ROW_BOUNDS);
    for (int i = 0; i < nn; ++i) {
        double ui[NV], q[NV];
        get3(c, u, i, ui);
        for (int v = 0; v < NV; ++v) q[v] = ufv[(size_t)v * nn + i];
        double lo = ui[0], hi = ui[0];
        for (int b = c->nb_off[i]; b < c->nb_off[i + 1]; ++b) {
            double uj[NV];
            node_or_ghost3(c, u, c->nb[b].j, uj);
            double rb = bar_rho3(gm, ui, uj, c->nb[b].c);
            if (rb < lo) lo = rb;
            if (rb > hi) hi = rb;
        }
        if (limiting >= 2) { rmin[i] = lo > beta * q[0] ? lo : beta * q[0]; rmax[i] = hi; }
        else { rmin[i] = beta * q[0]; rmax[i] = INFINITY; }
        if (q[0] < rmin[i]) rmin[i] = q[0];
        if (q[0] > rmax[i]) rmax[i] = q[0];
        pmin[i] = beta * pressure3(gm, q);
    }
    /* antidiffusive fluxes A = F_DG - F_FV at the interior subcell
       interfaces, mass-weighted; node a gets -l A, node a+1 +l A */
    int nif = K * 3 * np * np * N;
    double *A = malloc(sizeof(double) * NV * (size_t)nif);
    double area[3] = {c->dy * c->dz / 4.0, c->dx * c->dz / 4.0, c->dx * c->dy / 4.0};
    for (int e = 0; e < K; ++e)
        for (int d = 0; d < 3; ++d)
            for (int t2 = 0; t2 < np; ++t2) for (int t1 = 0; t1 < np; ++t1) {
                int idx[3];
                idx[d] = 0; idx[(d + 1) % 3] = t1; idx[(d + 2) % 3] = t2;
                double fh[NP3][NV];
                ORC_ROW(ROW_VOLUME_FLUX);
                dg_subcell_row3(c, u, e, d, idx, fh);
                double wt = c->w[t1] * c->w[t2], cc = wt * area[d] / 2.0;
                for (int a = 0; a < N; ++a) {
                    int ql[3] = {idx[0], idx[1], idx[2]}, qr[3] = {idx[0], idx[1], idx[2]};
                    ql[d] = a; qr[d] = a + 1;
                    double ul[NV], ur[NV], fl[NV], fr[NV];
                    /* the low-order subcell flux again (the graph form above
                       carries the same terms: not counted twice) */
                    ORC_ROW(ROW_REFORM);
                    get3(c, u, g3(c, e, ql[0], ql[1], ql[2]), ul);
                    get3(c, u, g3(c, e, qr[0], qr[1], qr[2]), ur);
                    flux3(gm, ul, d, fl);
                    flux3(gm, ur, d, fr);
                    double lam = lambda3(gm, ul, ur, d);
                    int id = iface3(c, e, d, idx, a);
                    for (int v = 0; v < NV; ++v) {
                        double ffv = cc * (fl[v] + fr[v]) - cc * lam * (ur[v] - ul[v]);
                        ORC_ROW(ROW_VOLUME_LIMIT);
                        A[(size_t)NV * id + v] = wt * fh[a][v] - ffv;
                        ORC_ROW(ROW_REFORM);
                    }
                }
            }
    /* R15 exemption, then Zalesak (R7) */
    ORC_ROW(ROW_VOLUME_LIMIT);
    char *exempt = malloc(nif);
    for (int e = 0; e < K; ++e)
        for (int d = 0; d < 3; ++d)
            for (int t2 = 0; t2 < np; ++t2) for (int t1 = 0; t1 < np; ++t1)
                for (int a = 0; a < N; ++a) {
                    int idx[3]; idx[d] = a; idx[(d + 1) % 3] = t1; idx[(d + 2) % 3] = t2;
                    int gl = g3(c, e, idx[0], idx[1], idx[2]);
                    idx[d] = a + 1;
                    int gr = g3(c, e, idx[0], idx[1], idx[2]);
                    int id = iface3(c, e, d, idx, a);
                    double Ar = fabs(A[(size_t)NV * id]);
                    exempt[id] = (dt / mass3(c, gl) * Ar <= TOL3 * fabs(ufv[gl])) &&
                                 (dt / mass3(c, gr) * Ar <= TOL3 * fabs(ufv[gr]));
                }
    double *Rp = malloc(sizeof(double) * nn), *Rm = malloc(sizeof(double) * nn);
    for (int i = 0; i < nn; ++i) {
        int e = i / (np * np * np), rr = i % (np * np * np);
        int idx[3] = {rr % np, (rr / np) % np, rr / (np * np)};
        double Pp = 0.0, Pm = 0.0;
        for (int d = 0; d < 3; ++d) {
            int pos = idx[d];
            if (pos > 0) {
                double G = A[(size_t)NV * iface3(c, e, d, idx, pos - 1)];
                if (!exempt[iface3(c, e, d, idx, pos - 1)]) { Pp += G > 0 ? G : 0; Pm += G < 0 ? G : 0; }
            }
            if (pos < N) {
                double G = -A[(size_t)NV * iface3(c, e, d, idx, pos)];
                if (!exempt[iface3(c, e, d, idx, pos)]) { Pp += G > 0 ? G : 0; Pm += G < 0 ? G : 0; }
            }
        }
        double m = mass3(c, i), rf = ufv[i];
        double Qp = m / dt * (rmax[i] - rf), Qm = m / dt * (rmin[i] - rf);
        Rp[i] = (Pp > 0.0) ? (Qp / Pp < 1.0 ? Qp / Pp : 1.0) : 1.0;
        Rm[i] = (Pm < 0.0) ? (Qm / Pm < 1.0 ? Qm / Pm : 1.0) : 1.0;
        if (Rp[i] < 0.0) Rp[i] = 0.0;
        if (Rm[i] < 0.0) Rm[i] = 0.0;
    }
    /* R8 with Gamma = 2d = 6: per interface the largest factor keeping both
       end nodes admissible for the Gamma-scaled single-interface update */
    const double Gam = 6.0;
    double *ell = malloc(sizeof(double) * nif), *lmin = malloc(sizeof(double) * nn);
    for (int i = 0; i < nn; ++i) lmin[i] = 1.0;
    for (int e = 0; e < K; ++e)
        for (int d = 0; d < 3; ++d)
            for (int t2 = 0; t2 < np; ++t2) for (int t1 = 0; t1 < np; ++t1)
                for (int a = 0; a < N; ++a) {
                    int idx[3]; idx[d] = a; idx[(d + 1) % 3] = t1; idx[(d + 2) % 3] = t2;
                    int gl = g3(c, e, idx[0], idx[1], idx[2]);
                    idx[d] = a + 1;
                    int gr = g3(c, e, idx[0], idx[1], idx[2]);
                    int id = iface3(c, e, d, idx, a);
                    const double *Ai = &A[(size_t)NV * id];
                    double lr = exempt[id] ? 1.0
                              : (-Ai[0] > 0.0) ? (Rp[gl] < Rm[gr] ? Rp[gl] : Rm[gr]) : (Rm[gl] < Rp[gr] ? Rm[gl] : Rp[gr]);
                    double u0[NV], av[NV];
                    double ml = mass3(c, gl), mr = mass3(c, gr);
                    for (int v = 0; v < NV; ++v) { u0[v] = ufv[(size_t)v * nn + gl]; av[v] = -Gam * dt / ml * Ai[v]; }
                    double thl = o3_theta(gm, u0, av, pmin[gl], lr);
                    for (int v = 0; v < NV; ++v) { u0[v] = ufv[(size_t)v * nn + gr]; av[v] = Gam * dt / mr * Ai[v]; }
                    double thr = o3_theta(gm, u0, av, pmin[gr], lr);
                    double l = thl < thr ? thl : thr;
                    if (g_iface3) {
                        double *o = g_iface3 + (size_t)id * 12;
                        o[0] = gl; o[1] = gr; o[2] = exempt[id]; o[3] = lr; o[4] = thl; o[5] = thr; o[6] = l;
                        for (int v = 0; v < NV; ++v) o[7 + v] = Ai[v];
                    }
                    if (g_force3 >= 0.0) l = g_force3;
                    ell[id] = l;
                    if (l < lmin[gl]) lmin[gl] = l;
                    if (l < lmin[gr]) lmin[gr] = l;
                }
    if (g_node3)
        for (int i = 0; i < nn; ++i) {
            double *o = g_node3 + (size_t)i * 10;
            for (int v = 0; v < NV; ++v) o[v] = ufv[(size_t)v * nn + i];
            o[5] = rmin[i]; o[6] = rmax[i]; o[7] = pmin[i]; o[8] = Rp[i]; o[9] = Rm[i];
        }
    /* limited residual and stage state; violations (R13) */
    for (int i = 0; i < nn; ++i) {
        int e = i / (np * np * np), rr = i % (np * np * np);
        int idx[3] = {rr % np, (rr / np) % np, rr / (np * np)};
        double s[NV] = {0, 0, 0, 0, 0};
        ORC_ROW(ROW_VOLUME_LIMIT);
        /* the node's interfaces in a fixed order: x low, x high, y low, y high, z low, z high */
        for (int d = 0; d < 3; ++d) {
            int pos = idx[d];
            if (pos > 0) { int id = iface3(c, e, d, idx, pos - 1); for (int v = 0; v < NV; ++v) s[v] += ell[id] * A[(size_t)NV * id + v]; }
            if (pos < N) { int id = iface3(c, e, d, idx, pos); for (int v = 0; v < NV; ++v) s[v] -= ell[id] * A[(size_t)NV * id + v]; }
        }
        double m = mass3(c, i), q[NV];
        ORC_ROW(ROW_STAGE);
        for (int v = 0; v < NV; ++v) {
            res_out[(size_t)v * nn + i] = rfv[(size_t)v * nn + i] + s[v];
            q[v] = ufv[(size_t)v * nn + i] + dt / m * s[v];
            if (utilde) utilde[(size_t)v * nn + i] = q[v];
        }
        ORC_ROW(ROW_STATS);
        if (stats) {
            double p = pressure3(gm, q);
            stats[S3_AVOL_M] += m * (1.0 - lmin[i]);
            stats[S3_M] += m;
            if (lmin[i] < 1.0) stats[S3_NVOL] += 1;
            if (q[0] < rmin[i] - 1e-13 * fabs(rmin[i]) || q[0] > rmax[i] + 1e-13 * fabs(rmax[i])) stats[S3_VRHO] += 1;
            if (p < pmin[i] - 1e-13 * fabs(pmin[i])) stats[S3_VP] += 1;
            if (!(q[0] > 0.0) || !(p > 0.0)) stats[S3_NONPOS] += 1;
            if (q[0] < stats[S3_MINRHO]) stats[S3_MINRHO] = q[0];
            if (p < stats[S3_MINP]) stats[S3_MINP] = p;
        }
    }
    free(rdg); free(rfv); free(ds); free(ufv); free(rmin); free(rmax); free(pmin); free(A); free(exempt);
    free(Rp); free(Rm); free(ell); free(lmin);
    return 0;
}

void o3_stats_init(double *stats) {
    for (int k = 0; k < S3_N; ++k) stats[k] = 0.0;
    stats[S3_MINRHO] = INFINITY; stats[S3_MINP] = INFINITY;
}

/* residual per unit mass */
int o3_rhs(const o3_ctx *c, const double *u, double dt, int limiting, double beta, double *rhs, double *stats) {
    int rc = o3_stage(c, u, dt, limiting, beta, rhs, NULL, stats);
    for (int i = 0; i < c->nn; ++i) {
        double m = mass3(c, i);
        for (int v = 0; v < NV; ++v) rhs[(size_t)v * c->nn + i] /= m;
    }
    return rc;
}

/* SSP-RK3 (Shu-Osher) with dt from u^n every step (R10) */
int o3_step(const o3_ctx *c, double *u, int nsteps, double *time, double cfl, int limiting, double beta,
            double *dt_hist, double *stats) {
    size_t n = (size_t)NV * c->nn;
    double *u1 = malloc(sizeof(double) * n), *u2 = malloc(sizeof(double) * n), *ut = malloc(sizeof(double) * n);
    double *res = malloc(sizeof(double) * n);
    for (int s = 0; s < nsteps; ++s) {
        double dt = o3_dt(c, u, cfl);
        ORC_CONST(dt);
        if (dt_hist) dt_hist[s] = dt;
        o3_stage(c, u, dt, limiting, beta, res, ut, stats);
        for (size_t k = 0; k < n; ++k) u1[k] = ut[k];
        o3_stage(c, u1, dt, limiting, beta, res, ut, stats);
        ORC_ROW(ROW_STAGE);
        for (size_t k = 0; k < n; ++k) u2[k] = 0.75 * u[k] + 0.25 * ut[k];
        o3_stage(c, u2, dt, limiting, beta, res, ut, stats);
        ORC_ROW(ROW_STAGE);
        for (size_t k = 0; k < n; ++k) u[k] = u[k] / 3.0 + 2.0 / 3.0 * ut[k];
        *time += dt;
    }
    free(u1); free(u2); free(ut); free(res);
    return 0;
}

void o3_integrals(const o3_ctx *c, const double *u, double *out) {
    for (int v = 0; v < NV; ++v) {
        double s = 0.0;
        for (int i = 0; i < c->nn; ++i) s += mass3(c, i) * u[(size_t)v * c->nn + i];
        out[v] = s;
    }
}

void o3_masses(const o3_ctx *c, double *m) { for (int i = 0; i < c->nn; ++i) m[i] = mass3(c, i); }

/* the two residuals alone (pins) */
void o3_dg_residual(const o3_ctx *c, const double *u, double *res) { dg_residual3(c, u, res); }
void o3_fv_residual(const o3_ctx *c, const double *u, double *res, double *dsum) { fv_residual3(c, u, res, dsum); }
