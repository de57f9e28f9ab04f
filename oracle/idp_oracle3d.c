/*
 * idp_oracle3d.c -- plain, slow FP64 CPU oracle of the IDP-limited LGL-DGSEM
 * for the 3D Euler equations (d = 3 of Sec. 2, Eq. conservationlaw) on
 * 2:1-balanced Cartesian octrees of hexahedra (Bolm, Rueda-Ramirez, Kuzmin,
 * Gassner, arXiv 2607.06045).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library. It shares no code with the
 * CUDA path. It is built together with idp_oracle.c, whose LGL operators
 * (orc_operators: nodes, weights, Sbar) and logarithmic mean (orc_logmean,
 * R2) it uses; everything three-dimensional is here.
 *
 * The mesh is a 2:1-balanced octree of hexahedra (a leaf at level l is one
 * cell of the (nx0 2^l) x (ny0 2^l) x (nz0 2^l) grid over the box); a face
 * between a leaf and four finer ones is a mortar with 2 x 2 small faces. The
 * method is the 2D one of the paper with the third direction added, as
 * Sec. 2 states it for d in {1, 2, 3}:
 *   - the high-order residual of Eq. evolutionformula, a sum over the three
 *     directions of the flux-differencing volume terms with Sbar and the LLF
 *     surface terms, and its subcell fluxes (Eq. fluxdifferencingform);
 *   - the low-order residual in the global graph form of
 *     Eq. LowOrderScheme_globalIndices with the c/d coefficients of Sec. 2.1,
 *     the three directions' subcell neighbours, the face neighbours and, at
 *     mortars, Eq. c_nonconforming with the local weights of App. A taken
 *     as products of the 1D overlap weights along the face's two tangential
 *     directions (reading R32: the overlap of tensor-product subcells);
 *   - the L2 mortar (R5) as the tensor product of the 1D interpolation and
 *     exact L2 projection, and the sparse IDP mortar flux of
 *     Eq. interfaceflux_local with those weights;
 *   - bar states, density bounds (Eqs. Bounds_Positivity, Bounds_Barstates),
 *     Zalesak density limiting and the pressure factor with Gamma = 2d = 6
 *     (Sec. 2.3), and one factor per mortar after the volume correction with
 *     the n_i budget (R9);
 *   - the combined limiting (limiting 3, Sec. 3.5, Eq.
 *     combination_posLim_local): per interface and per mortar the factor
 *     (1 - a) l_positivity + a l_local with a the element's shock indicator
 *     (the largest of the mortar's five elements), the indicator the
 *     modal-energy one of the pressure in the tensor-product Legendre basis
 *     (reading R34);
 *   - the IDP time step (Eq. timestep_restriction) and SSP-RK3.
 * Readings as in idp_oracle.c (R1-R3, R5-R10, R13, R15-R17, R20), with the
 * states u = (rho, rho v1, rho v2, rho v3, rho e) and
 * p = (gamma - 1)(rho e - |m|^2 / (2 rho)); the boundary kinds of R4 without
 * the 2D problem-specific ones (periodic, wall, Dirichlet, outflow).
 *
 * Layout: node g = ((e np + k) np + j) np + i (x index i fastest) of leaf e
 * in the caller's order, state u[5][K np^3]; a uniform grid (o3_create)
 * orders its elements e = (ez ny + ey) nx + ex.
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
enum { F3_CONF = 0, F3_BND = 1, F3_ML = 2, F3_MS = 3 };
enum { S3_AVOL_M = 0, S3_M, S3_NVOL, S3_VRHO, S3_VP, S3_NONPOS, S3_DTX, S3_MINRHO, S3_MINP, S3_AMORT_A, S3_A,
       S3_NMORT, S3_N };

typedef struct {
    int j;            /* neighbour node, or -1-q for ghost q */
    int face;         /* 0 subcell neighbour, 1 across a conforming or boundary face, 2 across a mortar */
    double c[3];      /* c_(i,j) */
} o3_nb;

typedef struct {
    int N, np, K, nn, ng, M;
    double gamma;
    double xi[NP3], w[NP3], S[NP3][NP3];
    double wt[NP3][2 * NP3];    /* 1D local weights (App. A), reference units of the large face */
    double Ii[2 * NP3][NP3];    /* 1D interpolation large -> small-face nodes */
    double P[NP3][2 * NP3];     /* 1D exact L2 projection small -> large */
    int n0[3];
    double box[6];
    int bc[6];
    double bc_prim[6][NV];
    int *lev, *ic;              /* [K], [K][3] */
    double *h;                  /* [K][3] element sides */
    int *ftype, *fnbr, *fpos;   /* [K][6] */
    int *mort;                  /* [M][7]: d, large, large on the low side, small[4] (p = p1 + 2 p2) */
    int *nb_off;
    o3_nb *nb;
    int *g_node, *g_side;       /* ghost q: the boundary node it mirrors, and the side */
    int *mcount;                /* [nn] mortars incident on the node */
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
static int g3v(const o3_ctx *c, int e, const int *idx) { return g3(c, e, idx[0], idx[1], idx[2]); }

/* quarter area of the faces of element e normal to d */
static double qarea(const o3_ctx *c, int e, int d) { return c->h[3 * e + (d + 1) % 3] * c->h[3 * e + (d + 2) % 3] / 4.0; }

static void push3(o3_nb **buf, int *n, int *cap, int j, int d, double cd, int face) {
    if (*n == *cap) { *cap = *cap ? 2 * *cap : 4096; *buf = realloc(*buf, sizeof(o3_nb) * (*cap)); }
    o3_nb *b = &(*buf)[*n];
    b->j = j; b->face = face; b->c[0] = b->c[1] = b->c[2] = 0.0; b->c[d] = cd;
    ++*n;
}

void o3_destroy(o3_ctx *c) {
    if (!c) return;
    free(c->lev); free(c->ic); free(c->h); free(c->ftype); free(c->fnbr); free(c->fpos); free(c->mort);
    free(c->nb_off); free(c->nb); free(c->g_node); free(c->g_side); free(c->mcount);
    free(c);
}

typedef struct { int64_t key; int e; } lk3;
static int cmp_lk3(const void *a, const void *b) {
    int64_t x = ((const lk3 *)a)->key, y = ((const lk3 *)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}
static int64_t key3(int l, int64_t x, int64_t y, int64_t z) { return ((int64_t)l << 57) | (x << 38) | (y << 19) | z; }
static int find3(const lk3 *t, int K, int l, int64_t x, int64_t y, int64_t z) {
    if (l < 0) return -1;
    lk3 q; q.key = key3(l, x, y, z); q.e = -1;
    const lk3 *r = bsearch(&q, t, K, sizeof(lk3), cmp_lk3);
    return r ? r->e : -1;
}

/* element node of face node (a, b) on side s: idx[d] at the side, idx[d+1] = a,
   idx[d+2] = b (tangential axes in cyclic order) */
static void face_idx3(int np, int s, int a, int b, int *idx) {
    int d = s / 2;
    idx[d] = (s & 1) ? np - 1 : 0;
    idx[(d + 1) % 3] = a;
    idx[(d + 2) % 3] = b;
}

/* An octree: nx0 x ny0 x nz0 level-0 cells over box = {x0, y0, z0, x1, y1,
   z1}; leaf e at level level[e] and position (ix, iy, iz)[e] on its level's
   grid. bc[6] per side, bc_prim[6][5] primitive Dirichlet states. err: 1 bad
   arguments, 2 not 2:1 balanced (or a gap). */
o3_ctx *o3_create_leaves(int N, double gamma, int nx0, int ny0, int nz0, const double *box, int K,
                         const int8_t *level, const int32_t *ix, const int32_t *iy, const int32_t *iz,
                         const int32_t *bc, const double *bc_prim, int *err) {
    *err = 0;
    if (N < 1 || N + 1 > NP3 || nx0 < 1 || ny0 < 1 || nz0 < 1 || K < 1) { *err = 1; return NULL; }
    for (int d = 0; d < 3; ++d)
        if ((bc[2 * d] == B3_PERIODIC) != (bc[2 * d + 1] == B3_PERIODIC)) { *err = 1; return NULL; }
    o3_ctx *c = calloc(1, sizeof(o3_ctx));
    c->N = N; c->np = N + 1; c->gamma = gamma; c->K = K;
    int np = N + 1, NR = np * np;
    {
        double xi[NP3], w[NP3], D[NP3 * NP3], S[NP3 * NP3], wt[NP3 * 2 * NP3], I[2 * NP3 * NP3], P[NP3 * 2 * NP3];
        orc_operators(N, 1, xi, w, D, S, wt, I, P);
        for (int a = 0; a < np; ++a) { c->xi[a] = xi[a]; c->w[a] = w[a]; }
        for (int a = 0; a < np; ++a) for (int b = 0; b < np; ++b) c->S[a][b] = S[a * np + b];
        for (int a = 0; a < np; ++a)
            for (int b = 0; b < 2 * np; ++b) { c->wt[a][b] = wt[a * 2 * np + b]; c->P[a][b] = P[a * 2 * np + b]; }
        for (int a = 0; a < 2 * np; ++a) for (int b = 0; b < np; ++b) c->Ii[a][b] = I[a * np + b];
    }
    c->n0[0] = nx0; c->n0[1] = ny0; c->n0[2] = nz0;
    for (int k = 0; k < 6; ++k) c->box[k] = box[k];
    for (int s = 0; s < 6; ++s) { c->bc[s] = bc[s]; for (int v = 0; v < NV; ++v) c->bc_prim[s][v] = bc_prim[NV * s + v]; }
    c->lev = malloc(sizeof(int) * K); c->ic = malloc(sizeof(int) * 3 * K); c->h = malloc(sizeof(double) * 3 * K);
    lk3 *tab = malloc(sizeof(lk3) * K);
    for (int e = 0; e < K; ++e) {
        int l = level[e];
        c->lev[e] = l; c->ic[3 * e] = ix[e]; c->ic[3 * e + 1] = iy[e]; c->ic[3 * e + 2] = iz[e];
        for (int d = 0; d < 3; ++d) c->h[3 * e + d] = (box[3 + d] - box[d]) / ((double)c->n0[d] * (double)(1 << l));
        tab[e].key = key3(l, ix[e], iy[e], iz[e]); tab[e].e = e;
    }
    qsort(tab, K, sizeof(lk3), cmp_lk3);
    c->ftype = malloc(sizeof(int) * 6 * K); c->fnbr = malloc(sizeof(int) * 6 * K); c->fpos = malloc(sizeof(int) * 6 * K);
    c->mort = malloc(sizeof(int) * 7 * 6 * K);
    c->M = 0;
    /* pass 1: conforming, boundary and large-side mortar faces */
    for (int e = 0; e < K && !*err; ++e) {
        int l = c->lev[e];
        for (int s = 0; s < 6; ++s) {
            int d = s / 2, side = s & 1, a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            int64_t nl[3], q[3];
            for (int a = 0; a < 3; ++a) { nl[a] = (int64_t)c->n0[a] << l; q[a] = c->ic[3 * e + a]; }
            q[d] += side ? 1 : -1;
            c->fpos[6 * e + s] = -1;
            if (q[d] < 0 || q[d] >= nl[d]) {
                if (bc[s] != B3_PERIODIC) { c->ftype[6 * e + s] = F3_BND; c->fnbr[6 * e + s] = -1; continue; }
                q[d] = (q[d] + nl[d]) % nl[d];
            }
            int f = find3(tab, K, l, q[0], q[1], q[2]);
            if (f >= 0) { c->ftype[6 * e + s] = F3_CONF; c->fnbr[6 * e + s] = f; continue; }
            if (l > 0 && find3(tab, K, l - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1) >= 0) {
                c->ftype[6 * e + s] = F3_MS; c->fnbr[6 * e + s] = -1; continue;   /* filled in pass 2 */
            }
            /* four finer neighbours across the face */
            int m = c->M, ok = 1;
            int *mr = c->mort + 7 * m;
            mr[0] = d; mr[1] = e; mr[2] = side;   /* large on the low side when its +d side is the face */
            for (int p2 = 0; p2 < 2; ++p2)
                for (int p1 = 0; p1 < 2; ++p1) {
                    int64_t r[3];
                    r[d] = 2 * q[d] + (side ? 0 : 1);
                    r[a1] = 2 * q[a1] + p1;
                    r[a2] = 2 * q[a2] + p2;
                    int sm = find3(tab, K, l + 1, r[0], r[1], r[2]);
                    if (sm < 0) ok = 0;
                    mr[3 + p1 + 2 * p2] = sm;
                }
            if (!ok) { *err = 2; break; }
            c->M++;
            c->ftype[6 * e + s] = F3_ML; c->fnbr[6 * e + s] = m;
        }
    }
    free(tab);
    if (*err) { o3_destroy(c); return NULL; }
    /* pass 2: small-side mortar faces */
    for (int m = 0; m < c->M; ++m) {
        int *mr = c->mort + 7 * m;
        int s_small = 2 * mr[0] + (mr[2] ? 0 : 1);
        for (int p = 0; p < 4; ++p) {
            int e = mr[3 + p];
            c->ftype[6 * e + s_small] = F3_MS; c->fnbr[6 * e + s_small] = m; c->fpos[6 * e + s_small] = p;
        }
    }
    for (int e = 0; e < K; ++e) for (int s = 0; s < 6; ++s)
        if (c->ftype[6 * e + s] == F3_MS && c->fnbr[6 * e + s] < 0) { *err = 2; o3_destroy(c); return NULL; }
    /* global node graph with c_(i,j) (Sec. 2.1, Eq. c_nonconforming) */
    c->nn = K * np * np * np;
    c->nb_off = malloc(sizeof(int) * (c->nn + 1));
    c->mcount = calloc(c->nn, sizeof(int));
    c->g_node = malloc(sizeof(int) * 6 * (size_t)NR * K);
    c->g_side = malloc(sizeof(int) * 6 * (size_t)NR * K);
    o3_nb *buf = NULL;
    int cnt = 0, cap = 0;
    for (int e = 0; e < K; ++e)
        for (int k = 0; k < np; ++k) for (int j = 0; j < np; ++j) for (int i = 0; i < np; ++i) {
            int g = g3(c, e, i, j, k), idx[3] = {i, j, k};
            c->nb_off[g] = cnt;
            for (int d = 0; d < 3; ++d) {
                int a1 = (d + 1) % 3, a2 = (d + 2) % 3, t1 = idx[a1], t2 = idx[a2], pos = idx[d];
                double cd = c->w[t1] * c->w[t2] * qarea(c, e, d) / 2.0;   /* |c_ij| of subcell and conforming pairs */
                /* subcell neighbours (Sec. 2.1) */
                if (pos > 0) { int qq[3] = {i, j, k}; qq[d] -= 1; push3(&buf, &cnt, &cap, g3v(c, e, qq), d, -cd, 0); }
                if (pos < N) { int qq[3] = {i, j, k}; qq[d] += 1; push3(&buf, &cnt, &cap, g3v(c, e, qq), d, cd, 0); }
                for (int side = 0; side < 2; ++side) {
                    if ((side == 0 && pos != 0) || (side == 1 && pos != N)) continue;
                    int s = 2 * d + side, ft = c->ftype[6 * e + s];
                    double sg = side ? 1.0 : -1.0;   /* outward normal along d */
                    if (ft == F3_CONF) {
                        int qq[3] = {i, j, k}; qq[d] = side ? 0 : N;
                        push3(&buf, &cnt, &cap, g3v(c, c->fnbr[6 * e + s], qq), d, sg * cd, 1);
                    } else if (ft == F3_BND) {
                        c->g_node[c->ng] = g; c->g_side[c->ng] = s;
                        push3(&buf, &cnt, &cap, -1 - c->ng, d, sg * cd, 1);
                        c->ng++;
                    } else if (ft == F3_ML) {
                        int m = c->fnbr[6 * e + s];
                        const int *mr = c->mort + 7 * m;
                        double qa = qarea(c, e, d);
                        c->mcount[g]++;
                        for (int p2 = 0; p2 < 2; ++p2) for (int p1 = 0; p1 < 2; ++p1)
                            for (int l2 = 0; l2 < np; ++l2) for (int l1 = 0; l1 < np; ++l1) {
                                double wgt = c->wt[t1][p1 * np + l1] * c->wt[t2][p2 * np + l2];
                                if (wgt == 0.0) continue;
                                int qq[3];
                                face_idx3(np, s ^ 1, l1, l2, qq);
                                push3(&buf, &cnt, &cap, g3v(c, mr[3 + p1 + 2 * p2], qq), d, sg * wgt * qa / 2.0, 2);
                            }
                    } else {
                        int m = c->fnbr[6 * e + s], p = c->fpos[6 * e + s], p1 = p & 1, p2 = p >> 1;
                        const int *mr = c->mort + 7 * m;
                        int L = mr[1];
                        double qa = qarea(c, L, d);
                        c->mcount[g]++;
                        for (int k2 = 0; k2 < np; ++k2) for (int k1 = 0; k1 < np; ++k1) {
                            double wgt = c->wt[k1][p1 * np + t1] * c->wt[k2][p2 * np + t2];
                            if (wgt == 0.0) continue;
                            int qq[3];
                            face_idx3(np, s ^ 1, k1, k2, qq);
                            push3(&buf, &cnt, &cap, g3v(c, L, qq), d, sg * wgt * qa / 2.0, 2);
                        }
                    }
                }
            }
        }
    c->nb_off[c->nn] = cnt;
    c->nb = buf;
    return c;
}

/* a uniform grid: all leaves at level 0, e = (ez ny + ey) nx + ex */
o3_ctx *o3_create(int N, double gamma, int nx, int ny, int nz, const double *box, const int32_t *bc,
                  const double *bc_prim, int *err) {
    if (nx < 1 || ny < 1 || nz < 1) { *err = 1; return NULL; }
    int K = nx * ny * nz;
    int8_t *lev = calloc(K, 1);
    int32_t *ix = malloc(sizeof(int32_t) * K), *iy = malloc(sizeof(int32_t) * K), *iz = malloc(sizeof(int32_t) * K);
    for (int e = 0; e < K; ++e) { ix[e] = e % nx; iy[e] = (e / nx) % ny; iz[e] = e / (nx * ny); }
    o3_ctx *c = o3_create_leaves(N, gamma, nx, ny, nz, box, K, lev, ix, iy, iz, bc, bc_prim, err);
    free(lev); free(ix); free(iy); free(iz);
    return c;
}

int o3_n_nodes(const o3_ctx *c) { return c->nn; }
int o3_n_mortars(const o3_ctx *c) { return c->M; }

static double mass3(const o3_ctx *c, int g) {
    int np = c->np, e = g / (np * np * np), i = g % np, j = (g / np) % np, k = (g / (np * np)) % np;
    return c->w[i] * c->w[j] * c->w[k] * c->h[3 * e] * c->h[3 * e + 1] * c->h[3 * e + 2] / 8.0;
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
/* mortars                                                                   */
/* ------------------------------------------------------------------------ */

/* mortar m: the nodes of its large face (k1 + np k2) and of its small faces
   p (np^2 + p np^2 + l1 + np l2) */
static void mortar_nodes3(const o3_ctx *c, int m, int *gnode) {
    int np = c->np, NR = np * np;
    const int *mr = c->mort + 7 * m;
    int sL = 2 * mr[0] + mr[2], sS = sL ^ 1;
    for (int b = 0; b < np; ++b) for (int a = 0; a < np; ++a) {
        int qq[3];
        face_idx3(np, sL, a, b, qq);
        gnode[a + np * b] = g3v(c, mr[1], qq);
        face_idx3(np, sS, a, b, qq);
        for (int p = 0; p < 4; ++p) gnode[NR + p * NR + a + np * b] = g3v(c, mr[3 + p], qq);
    }
}

/* outward low-order sparse fluxes of Eq. interfaceflux_local at the mortar's
   nodes (mass-weighted), with the weights of reading R32 */
static void mortar_low3(const o3_ctx *c, const double *u, int m, double Flo[][NV]) {
    int np = c->np, NR = np * np;
    double gm = c->gamma;
    const int *mr = c->mort + 7 * m;
    int d = mr[0], low = mr[2];
    double nL = low ? 1.0 : -1.0, qa = qarea(c, mr[1], d);
    int gnode[5 * NP3 * NP3];
    mortar_nodes3(c, m, gnode);
    for (int q = 0; q < 5 * NR; ++q) for (int v = 0; v < NV; ++v) Flo[q][v] = 0.0;
    for (int k2 = 0; k2 < np; ++k2) for (int k1 = 0; k1 < np; ++k1)
        for (int p2 = 0; p2 < 2; ++p2) for (int p1 = 0; p1 < 2; ++p1)
            for (int l2 = 0; l2 < np; ++l2) for (int l1 = 0; l1 < np; ++l1) {
                double wgt = c->wt[k1][p1 * np + l1] * c->wt[k2][p2 * np + l2] * qa;
                if (wgt == 0.0) continue;
                int qi = k1 + np * k2, qj = NR + (p1 + 2 * p2) * NR + l1 + np * l2;
                double ui[NV], uj[NV], fi[NV], fj[NV];
                get3(c, u, gnode[qi], ui); get3(c, u, gnode[qj], uj);
                flux3(gm, ui, d, fi); flux3(gm, uj, d, fj);
                double lam = lambda3(gm, ui, uj, d);
                for (int v = 0; v < NV; ++v) {
                    Flo[qi][v] += 0.5 * (wgt * nL * (fi[v] + fj[v]) - wgt * lam * (uj[v] - ui[v]));
                    Flo[qj][v] += 0.5 * (-wgt * nL * (fi[v] + fj[v]) - wgt * lam * (ui[v] - uj[v]));
                }
            }
}

/* Surface fluxes of every element side, the +d numerical flux times the
   side's quarter area per face node: sf[e][s][a + np b][v]. Mortars: R5 as
   tensor products (interpolate to the small-face nodes, LLF there, exact L2
   projection back); R16: a mortar whose interpolated states are not
   admissible uses its low-order sparse flux and is flagged in mbad. With
   conforming = 0 only the mortar sides are formed (the limited stage takes
   its conforming and boundary faces from the graph, where the LLF flux is
   the low-order face term itself). */
static double *surface_fluxes3(const o3_ctx *c, const double *u, char *mbad, int conforming) {
    int np = c->np, NR = np * np, K = c->K;
    double g = c->gamma;
    double *sf = calloc((size_t)K * 6 * NR * NV, sizeof(double));
    ORC_ROW(ROW_FACE_FLUX);
    for (int e = 0; e < K && conforming; ++e)
        for (int s = 0; s < 6; ++s) {
            int ft = c->ftype[6 * e + s], d = s / 2, side = s & 1;
            if (ft == F3_ML || ft == F3_MS) continue;
            double qa = qarea(c, e, d);
            for (int b = 0; b < np; ++b) for (int a = 0; a < np; ++a) {
                int qq[3];
                face_idx3(np, s, a, b, qq);
                double in[NV], out[NV], f[NV];
                get3(c, u, g3v(c, e, qq), in);
                if (ft == F3_CONF) {
                    int qo[3];
                    face_idx3(np, s ^ 1, a, b, qo);
                    get3(c, u, g3v(c, c->fnbr[6 * e + s], qo), out);
                } else {
                    ghost3(c, in, s, out);
                }
                if (side) o3_llf(g, in, out, d, f); else o3_llf(g, out, in, d, f);
                for (int v = 0; v < NV; ++v) sf[((size_t)(6 * e + s) * NR + a + np * b) * NV + v] = qa * f[v];
            }
        }
    for (int m = 0; m < c->M; ++m) {
        ORC_ROW(ROW_MORTAR_FLUX);
        const int *mr = c->mort + 7 * m;
        int d = mr[0], L = mr[1], low = mr[2], sL = 2 * d + low, sS = sL ^ 1;
        double qaL = qarea(c, L, d), qaS = qaL / 4.0;
        double uL[NP3 * NP3][NV];
        for (int b = 0; b < np; ++b) for (int a = 0; a < np; ++a) {
            int qq[3];
            face_idx3(np, sL, a, b, qq);
            get3(c, u, g3v(c, L, qq), uL[a + np * b]);
        }
        /* interpolated large-side states on each small face */
        double ui[4][NP3 * NP3][NV];
        int bad = 0;
        for (int p = 0; p < 4; ++p)
            for (int l2 = 0; l2 < np; ++l2) for (int l1 = 0; l1 < np; ++l1) {
                double *x = ui[p][l1 + np * l2];
                for (int v = 0; v < NV; ++v) x[v] = 0.0;
                for (int k2 = 0; k2 < np; ++k2) for (int k1 = 0; k1 < np; ++k1) {
                    double wgt = c->Ii[(p & 1) * np + l1][k1] * c->Ii[(p >> 1) * np + l2][k2];
                    for (int v = 0; v < NV; ++v) x[v] += wgt * uL[k1 + np * k2][v];
                }
                if (!(x[0] > 0.0) || !(pressure3(g, x) > 0.0)) bad = 1;
            }
        if (mbad) mbad[m] = (char)bad;
        if (bad) {
            double Flo[5 * NP3 * NP3][NV];
            mortar_low3(c, u, m, Flo);
            for (int b = 0; b < np; ++b) for (int a = 0; a < np; ++a) {
                double wk = c->w[a] * c->w[b];
                for (int v = 0; v < NV; ++v)
                    sf[((size_t)(6 * L + sL) * NR + a + np * b) * NV + v] = (low ? 1.0 : -1.0) * Flo[a + np * b][v] / wk;
                for (int p = 0; p < 4; ++p)
                    for (int v = 0; v < NV; ++v)
                        sf[((size_t)(6 * mr[3 + p] + sS) * NR + a + np * b) * NV + v] =
                            (low ? -1.0 : 1.0) * Flo[NR + p * NR + a + np * b][v] / wk;
            }
            continue;
        }
        double fs[4][NP3 * NP3][NV];
        for (int p = 0; p < 4; ++p)
            for (int b = 0; b < np; ++b) for (int a = 0; a < np; ++a) {
                int qq[3];
                face_idx3(np, sS, a, b, qq);
                double us[NV], f[NV];
                get3(c, u, g3v(c, mr[3 + p], qq), us);
                if (low) o3_llf(g, ui[p][a + np * b], us, d, f); else o3_llf(g, us, ui[p][a + np * b], d, f);
                for (int v = 0; v < NV; ++v) {
                    fs[p][a + np * b][v] = f[v];
                    sf[((size_t)(6 * mr[3 + p] + sS) * NR + a + np * b) * NV + v] = qaS * f[v];
                }
            }
        for (int k2 = 0; k2 < np; ++k2) for (int k1 = 0; k1 < np; ++k1)
            for (int v = 0; v < NV; ++v) {
                double acc = 0.0;
                for (int p = 0; p < 4; ++p)
                    for (int l2 = 0; l2 < np; ++l2) for (int l1 = 0; l1 < np; ++l1)
                        acc += c->P[k1][(p & 1) * np + l1] * c->P[k2][(p >> 1) * np + l2] * fs[p][l1 + np * l2][v];
                sf[((size_t)(6 * L + sL) * NR + k1 + np * k2) * NV + v] = qaL * acc;
            }
    }
    return sf;
}

/* ------------------------------------------------------------------------ */
/* residuals                                                                 */
/* ------------------------------------------------------------------------ */

/* mass-weighted high-order residual (Eq. evolutionformula in 3D): per node
   the sum over d of the transverse weights times ( -sum_l Sbar_(pos,l) (A_d/4)
   f*_d(u, u_l) + the surface terms of the element's faces ) */
static void dg_residual3(const o3_ctx *c, const double *u, const double *sf, double *res) {
    int np = c->np, N = c->N, NR = np * np;
    double g = c->gamma;
    for (int e = 0; e < c->K; ++e)
        for (int k = 0; k < np; ++k) for (int j = 0; j < np; ++j) for (int i = 0; i < np; ++i) {
            int gi = g3(c, e, i, j, k), idx[3] = {i, j, k};
            double ui[NV], tot[NV] = {0, 0, 0, 0, 0};
            get3(c, u, gi, ui);
            for (int d = 0; d < 3; ++d) {
                double F[NV] = {0, 0, 0, 0, 0}, qa = qarea(c, e, d);
                int pos = idx[d], t1 = idx[(d + 1) % 3], t2 = idx[(d + 2) % 3];
                for (int l = 0; l < np; ++l) {
                    if (l == pos) continue;   /* Sbar has a zero diagonal */
                    int q[3] = {i, j, k}; q[d] = l;
                    double ul[NV], f[NV];
                    get3(c, u, g3v(c, e, q), ul);
                    o3_ranocha(g, ui, ul, d, f);
                    for (int v = 0; v < NV; ++v) F[v] -= c->S[pos][l] * qa * f[v];
                }
                int t = t1 + np * t2;
                if (pos == 0) for (int v = 0; v < NV; ++v) F[v] += sf[((size_t)(6 * e + 2 * d) * NR + t) * NV + v];
                if (pos == N) for (int v = 0; v < NV; ++v) F[v] -= sf[((size_t)(6 * e + 2 * d + 1) * NR + t) * NV + v];
                double wt = c->w[t1] * c->w[t2];
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
    double qa = qarea(c, e, d);
    double acc[NV] = {0, 0, 0, 0, 0};
    for (int l = 0; l < N; ++l) {
        int qa_[3] = {idx[0], idx[1], idx[2]}; qa_[d] = l;
        double ua[NV];
        get3(c, u, g3v(c, e, qa_), ua);
        for (int m = 0; m < np; ++m) {
            if (m == l) continue;
            int qm[3] = {idx[0], idx[1], idx[2]}; qm[d] = m;
            double um[NV], f[NV];
            get3(c, u, g3v(c, e, qm), um);
            o3_ranocha(c->gamma, ua, um, d, f);
            for (int v = 0; v < NV; ++v) acc[v] += c->S[l][m] * qa * f[v];
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
            ORC_ROW(nb->face == 2 ? ROW_MORTAR_FLUX : nb->face ? ROW_FACE_FLUX : ROW_SUBCELL_FV);
            double uj[NV], f[NV];
            node_or_ghost3(c, u, nb->j, uj);
            flux3(g, uj, d, f);
            double dd = fabs(nb->c[d]) * lambda3(g, ui, uj, d);
            for (int v = 0; v < NV; ++v) acc[v] += -nb->c[d] * f[v] + dd * (uj[v] - ui[v]);
            s2d += 2.0 * dd;
        }
        ORC_ROW(ROW_SUBCELL_FV);
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

/* ------------------------------------------------------------------------ */
/* shock indicator of the combined limiting (Sec. 3.5, Eq.                   */
/* combination_posLim_local) in 3D: Hennemann et al.'s modal-energy indicator */
/* of the pressure with the tensor-product Legendre modes (reading R34)      */
/* ------------------------------------------------------------------------ */

/* P_k(x) by the three-term recurrence */
static double legendre3(int k, double x) {
    double p0 = 1.0, p1 = x;
    if (k == 0) return p0;
    for (int n = 1; n < k; ++n) {
        double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        p0 = p1; p1 = p2;
    }
    return p1;
}

/* alpha in [0, 1] from the nodal pressures p[(k np + j) np + i] of one
   element: the modal coefficients m = (V^-1 x V^-1 x V^-1) p in the
   orthonormal Legendre tensor basis, V_ik = sqrt((2k+1)/2) P_k(xi_i); e1 the
   energy of the modes with max(k1, k2, k3) = N, e2 of max = N - 1, e0 the
   rest; E = max(e1 / (e0 + e1 + e2), e2 / (e0 + e2)); alpha the logistic map
   1 / (1 + exp(-(s / T)(E - T))), T = 0.5 10^(-1.8 (N+1)^(1/4)),
   s = ln((1 - 1e-4) / 1e-4), snapped to 0 or 1 within 1e-3 of them. */
double o3_indicator(int N, const double *xi, const double *p) {
    int np = N + 1;
    double V[NP3][NP3], Vi[NP3][NP3];
    for (int i = 0; i < np; ++i)
        for (int k = 0; k < np; ++k) { V[i][k] = sqrt((2.0 * k + 1.0) / 2.0) * legendre3(k, xi[i]); Vi[i][k] = i == k; }
    /* Vi = V^-1 by Gauss-Jordan elimination with partial pivoting */
    for (int c = 0; c < np; ++c) {
        int piv = c;
        for (int r = c + 1; r < np; ++r) if (fabs(V[r][c]) > fabs(V[piv][c])) piv = r;
        for (int k = 0; k < np; ++k) {
            double t = V[c][k]; V[c][k] = V[piv][k]; V[piv][k] = t;
            t = Vi[c][k]; Vi[c][k] = Vi[piv][k]; Vi[piv][k] = t;
        }
        double d = V[c][c];
        for (int k = 0; k < np; ++k) { V[c][k] /= d; Vi[c][k] /= d; }
        for (int r = 0; r < np; ++r) {
            if (r == c) continue;
            double f = V[r][c];
            for (int k = 0; k < np; ++k) { V[r][k] -= f * V[c][k]; Vi[r][k] -= f * Vi[c][k]; }
        }
    }
    double a[NP3 * NP3 * NP3], b[NP3 * NP3 * NP3];
    for (int n = 0; n < np * np * np; ++n) a[n] = p[n];
    /* along x, then y, then z */
    for (int k = 0; k < np; ++k) for (int j = 0; j < np; ++j) for (int m = 0; m < np; ++m) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += Vi[m][i] * a[(k * np + j) * np + i];
        b[(k * np + j) * np + m] = s;
    }
    for (int k = 0; k < np; ++k) for (int m = 0; m < np; ++m) for (int i = 0; i < np; ++i) {
        double s = 0.0;
        for (int j = 0; j < np; ++j) s += Vi[m][j] * b[(k * np + j) * np + i];
        a[(k * np + m) * np + i] = s;
    }
    for (int m = 0; m < np; ++m) for (int j = 0; j < np; ++j) for (int i = 0; i < np; ++i) {
        double s = 0.0;
        for (int k = 0; k < np; ++k) s += Vi[m][k] * a[(k * np + j) * np + i];
        b[(m * np + j) * np + i] = s;
    }
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;
    for (int k = 0; k < np; ++k) for (int j = 0; j < np; ++j) for (int i = 0; i < np; ++i) {
        double m2 = b[(k * np + j) * np + i] * b[(k * np + j) * np + i];
        int top = i > j ? i : j;
        if (k > top) top = k;
        if (top == N) e1 += m2;
        else if (top == N - 1) e2 += m2;
        else e0 += m2;
    }
    double E = 0.0;
    if (e0 + e1 + e2 > 0.0) E = e1 / (e0 + e1 + e2);
    if (e0 + e2 > 0.0 && e2 / (e0 + e2) > E) E = e2 / (e0 + e2);
    double T = 0.5 * pow(10.0, -1.8 * pow(N + 1.0, 0.25));
    double sh = log((1.0 - 1e-4) / 1e-4);
    double al = 1.0 / (1.0 + exp(-sh / T * (E - T)));
    if (al < 1e-3) al = 0.0;
    if (al > 1.0 - 1e-3) al = 1.0;
    return al;
}

static double g_force3 = -1.0, g_force_alpha3 = -1.0;
/* test hook: every element's indicator replaced by v in [0, 1] (v < 0: off) */
void o3_set_force_alpha(double v) { g_force_alpha3 = v; }
/* test hook: every factor replaced by v in [0, 1] (v < 0: off) */
void o3_set_force_ell(double v) { g_force3 = v; }
/* test hooks: per node [u_FV (5), rho_min, rho_max, p_min, R+, R-] and per
   interface [left node, right node, exempt, Zalesak factor, theta_left,
   theta_right, factor, A (5)] of the next limited stage */
static double *g_node3 = NULL, *g_iface3 = NULL, *g_mortar3 = NULL, *g_mrec3 = NULL;
void o3_set_dbg_out(double *node, double *iface) { g_node3 = node; g_iface3 = iface; }
/* test hooks: each mortar's factor l_S of the next limited stage and, per
   mortar node (large face, then the small faces p = p1 + 2 p2, each face's
   nodes a + (N+1) b), [node, u_vol (5), n_i dt/m_i H (5), rho_min, rho_max,
   p_min, n_i, H (5)] */
void o3_set_mortar_out(double *ell, double *rec) { g_mortar3 = ell; g_mrec3 = rec; }

/* the mortar table: per mortar [d, large element, large on the low side,
   small elements p = 0..3] */
void o3_mortar_table(const o3_ctx *c, int *out) { for (int k = 0; k < 7 * c->M; ++k) out[k] = c->mort[k]; }

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
    char *mbad = calloc(c->M + 1, 1);
    int high = dt == 0.0 || limiting == 0;
    double *sf = surface_fluxes3(c, u, mbad, high);
    if (high) {
        double *rdg = malloc(sizeof(double) * NV * (size_t)nn);
        ORC_ROW(ROW_VOLUME_FLUX);
        dg_residual3(c, u, sf, rdg);
        ORC_ROW(ROW_STAGE);
        for (size_t k = 0; k < (size_t)NV * nn; ++k) res_out[k] = rdg[k];
        if (utilde)
            for (int i = 0; i < nn; ++i) for (int v = 0; v < NV; ++v)
                utilde[(size_t)v * nn + i] = u[(size_t)v * nn + i] + dt / mass3(c, i) * rdg[(size_t)v * nn + i];
        free(rdg); free(sf); free(mbad);
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
    /* combined limiting (limiting 3): the positivity density bound beside the
       local ones, and the indicator per element from the stage input */
    const int comb = limiting == 3;
    double *rmin2 = malloc(sizeof(double) * nn), *aind = calloc((size_t)K, sizeof(double));
    if (comb)
        for (int e = 0; e < K; ++e) {
            double pe[NP3 * NP3 * NP3], q[NV];
            for (int n = 0; n < np * np * np; ++n) { get3(c, u, e * np * np * np + n, q); pe[n] = pressure3(gm, q); }
            aind[e] = g_force_alpha3 >= 0.0 ? g_force_alpha3 : o3_indicator(N, c->xi, pe);
        }
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
        if (comb) rmin2[i] = beta * q[0] < q[0] ? beta * q[0] : q[0];
        pmin[i] = beta * pressure3(gm, q);
    }
    /* antidiffusive fluxes A = F_DG - F_FV at the interior subcell
       interfaces, mass-weighted; node a gets -l A, node a+1 +l A */
    int nif = K * 3 * np * np * N;
    double *A = malloc(sizeof(double) * NV * (size_t)nif);
    for (int e = 0; e < K; ++e)
        for (int d = 0; d < 3; ++d)
            for (int t2 = 0; t2 < np; ++t2) for (int t1 = 0; t1 < np; ++t1) {
                int idx[3];
                idx[d] = 0; idx[(d + 1) % 3] = t1; idx[(d + 2) % 3] = t2;
                double fh[NP3][NV];
                ORC_ROW(ROW_VOLUME_FLUX);
                dg_subcell_row3(c, u, e, d, idx, fh);
                double wt = c->w[t1] * c->w[t2], cc = wt * qarea(c, e, d) / 2.0;
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
    double *Rp = malloc(sizeof(double) * nn), *Rm = malloc(sizeof(double) * nn), *Rm2 = malloc(sizeof(double) * nn);
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
        /* the positivity bounds alone (no upper density bound: R+ = 1) */
        if (comb) {
            double Qm2 = m / dt * (rmin2[i] - rf);
            Rm2[i] = (Pm < 0.0) ? (Qm2 / Pm < 1.0 ? Qm2 / Pm : 1.0) : 1.0;
            if (Rm2[i] < 0.0) Rm2[i] = 0.0;
        }
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
                    if (comb) {
                        /* the positivity-only factor of the same interface, blended
                           (Eq. combination_posLim_local) */
                        double lr2 = exempt[id] ? 1.0 : (-Ai[0] > 0.0) ? Rm2[gr] : Rm2[gl];
                        for (int v = 0; v < NV; ++v) { u0[v] = ufv[(size_t)v * nn + gl]; av[v] = -Gam * dt / ml * Ai[v]; }
                        double t2l = o3_theta(gm, u0, av, pmin[gl], lr2);
                        for (int v = 0; v < NV; ++v) { u0[v] = ufv[(size_t)v * nn + gr]; av[v] = Gam * dt / mr * Ai[v]; }
                        double t2r = o3_theta(gm, u0, av, pmin[gr], lr2);
                        double l2 = t2l < t2r ? t2l : t2r;
                        l = (1.0 - aind[e]) * l2 + aind[e] * l;
                    }
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
    /* volume-corrected state u_vol = u_FV + dt/m sum l A */
    double *uvol = malloc(sizeof(double) * NV * (size_t)nn), *acc = calloc(NV * (size_t)nn, sizeof(double));
    for (int i = 0; i < nn; ++i) {
        int e = i / (np * np * np), rr = i % (np * np * np);
        int idx[3] = {rr % np, (rr / np) % np, rr / (np * np)};
        double sv[NV] = {0, 0, 0, 0, 0};
        ORC_ROW(ROW_VOLUME_LIMIT);
        /* the node's interfaces in a fixed order: x low, x high, y low, y high, z low, z high */
        for (int d = 0; d < 3; ++d) {
            int pos = idx[d];
            if (pos > 0) { int id = iface3(c, e, d, idx, pos - 1); for (int v = 0; v < NV; ++v) sv[v] += ell[id] * A[(size_t)NV * id + v]; }
            if (pos < N) { int id = iface3(c, e, d, idx, pos); for (int v = 0; v < NV; ++v) sv[v] -= ell[id] * A[(size_t)NV * id + v]; }
        }
        double m = mass3(c, i);
        for (int v = 0; v < NV; ++v) {
            acc[(size_t)v * nn + i] = sv[v];
            uvol[(size_t)v * nn + i] = ufv[(size_t)v * nn + i] + dt / m * sv[v];
        }
        ORC_ROW(ROW_STATS);
        if (stats) {
            stats[S3_AVOL_M] += m * (1.0 - lmin[i]);
            stats[S3_M] += m;
            if (lmin[i] < 1.0) stats[S3_NVOL] += 1;
        }
    }
    /* R9: mortar limiting after the volume correction. Per mortar node the
       high-order (R5) and low-order outward fluxes; H = -(F_L2 - F_lo) is the
       antidiffusive contribution; one factor per mortar with the n_i budget */
    double *corr = calloc(NV * (size_t)nn, sizeof(double));
    int NR = np * np;
    for (int m = 0; m < c->M; ++m) {
        ORC_ROW(ROW_MORTAR_LIMIT);
        const int *mr = c->mort + 7 * m;
        int d = mr[0], L = mr[1], low = mr[2], sL = 2 * d + low, sS = sL ^ 1;
        int gnode[5 * NP3 * NP3];
        double H[5 * NP3 * NP3][NV], Flo[5 * NP3 * NP3][NV];
        mortar_nodes3(c, m, gnode);
        ORC_ROW(ROW_REFORM);
        mortar_low3(c, u, m, Flo);
        ORC_ROW(ROW_MORTAR_LIMIT);
        for (int b = 0; b < np; ++b) for (int a = 0; a < np; ++a) {
            double wk = c->w[a] * c->w[b];
            int t = a + np * b;
            for (int v = 0; v < NV; ++v) {
                double FL2 = (low ? 1.0 : -1.0) * wk * sf[((size_t)(6 * L + sL) * NR + t) * NV + v];
                H[t][v] = -(FL2 - Flo[t][v]);
            }
            for (int p = 0; p < 4; ++p)
                for (int v = 0; v < NV; ++v) {
                    double FL2 = (low ? -1.0 : 1.0) * wk * sf[((size_t)(6 * mr[3 + p] + sS) * NR + t) * NV + v];
                    H[NR + p * NR + t][v] = -(FL2 - Flo[NR + p * NR + t][v]);
                }
        }
        double lS = 1.0, lS2 = 1.0, am = 0.0;
        if (comb) {
            am = aind[L];
            for (int p = 0; p < 4; ++p) if (aind[mr[3 + p]] > am) am = aind[mr[3 + p]];
        }
        if (mbad[m]) {
            /* R16: no admissible high-order flux, pure low order */
            for (int q = 0; q < 5 * NR; ++q) for (int v = 0; v < NV; ++v) H[q][v] = 0.0;
            lS = 0.0;
        }
        for (int q = 0; q < 5 * NR && !mbad[m]; ++q) {
            int i = gnode[q];
            double mi = mass3(c, i), ni = (double)c->mcount[i], tolr = TOL3 * fabs(ufv[i]);
            double u0[NV], av[NV];
            for (int v = 0; v < NV; ++v) { u0[v] = uvol[(size_t)v * nn + i]; av[v] = ni * dt / mi * H[q][v]; }
            /* R15 per mortar slot: a density change below TOL3 |rho_FV| (rounding
               noise of exactly cancelling high- and low-order mortar fluxes) is
               exempt from the density bounds */
            const int exs = fabs(av[0]) <= tolr;
            double lr = 1.0;
            if (!exs && av[0] > 0.0) { double t = (rmax[i] + tolr - u0[0]) / av[0]; if (t < lr) lr = t; }
            else if (!exs && av[0] < 0.0) { double t = (rmin[i] - tolr - u0[0]) / av[0]; if (t < lr) lr = t; }
            if (lr < 0.0) lr = 0.0;
            double th = o3_theta(gm, u0, av, pmin[i] - TOL3 * fabs(pmin[i]), lr);
            if (th < lS) lS = th;
            if (comb) {
                double lr2 = 1.0;
                if (!exs && av[0] < 0.0) { double t = (rmin2[i] - tolr - u0[0]) / av[0]; if (t < lr2) lr2 = t; }
                if (lr2 < 0.0) lr2 = 0.0;
                double th2 = o3_theta(gm, u0, av, pmin[i] - TOL3 * fabs(pmin[i]), lr2);
                if (th2 < lS2) lS2 = th2;
            }
        }
        if (comb && !mbad[m]) lS = (1.0 - am) * lS2 + am * lS;
        for (int q = 0; q < 5 * NR && g_mrec3; ++q) {
            int i = gnode[q];
            double ni = (double)c->mcount[i], *o = g_mrec3 + ((size_t)m * 5 * NR + q) * 20;
            o[0] = i;
            for (int v = 0; v < NV; ++v) {
                o[1 + v] = uvol[(size_t)v * nn + i];
                o[6 + v] = ni * dt / mass3(c, i) * H[q][v];
                o[15 + v] = H[q][v];
            }
            o[11] = rmin[i]; o[12] = rmax[i]; o[13] = pmin[i]; o[14] = ni;
        }
        if (g_force3 >= 0.0) lS = g_force3;
        if (g_mortar3) g_mortar3[m] = lS;
        for (int q = 0; q < 5 * NR; ++q) {
            int i = gnode[q];
            for (int v = 0; v < NV; ++v) corr[(size_t)v * nn + i] += lS * H[q][v];
        }
        ORC_ROW(ROW_STATS);
        if (stats) {
            double area = 4.0 * qarea(c, L, d);
            stats[S3_AMORT_A] += area * (1.0 - lS);
            stats[S3_A] += area;
            if (lS < 1.0) stats[S3_NMORT] += 1;
        }
    }
    /* limited residual and stage state; violations (R13) */
    for (int i = 0; i < nn; ++i) {
        double m = mass3(c, i), q[NV];
        ORC_ROW(ROW_STAGE);
        for (int v = 0; v < NV; ++v) {
            res_out[(size_t)v * nn + i] = rfv[(size_t)v * nn + i] + acc[(size_t)v * nn + i] + corr[(size_t)v * nn + i];
            q[v] = uvol[(size_t)v * nn + i] + dt / m * corr[(size_t)v * nn + i];
            if (utilde) utilde[(size_t)v * nn + i] = q[v];
        }
        ORC_ROW(ROW_STATS);
        if (stats) {
            double p = pressure3(gm, q);
            double lo_ = comb ? rmin2[i] : rmin[i], hi_ = comb ? INFINITY : rmax[i];
            if (q[0] < lo_ - 1e-13 * fabs(lo_) || q[0] > hi_ + 1e-13 * fabs(hi_)) stats[S3_VRHO] += 1;
            if (p < pmin[i] - 1e-13 * fabs(pmin[i])) stats[S3_VP] += 1;
            if (!(q[0] > 0.0) || !(p > 0.0)) stats[S3_NONPOS] += 1;
            if (q[0] < stats[S3_MINRHO]) stats[S3_MINRHO] = q[0];
            if (p < stats[S3_MINP]) stats[S3_MINP] = p;
        }
    }
    free(uvol); free(acc); free(corr); free(sf); free(mbad);
    free(rfv); free(ds); free(ufv); free(rmin); free(rmax); free(pmin); free(A); free(exempt);
    free(Rp); free(Rm); free(ell); free(lmin); free(Rm2); free(rmin2); free(aind);
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
void o3_dg_residual(const o3_ctx *c, const double *u, double *res) {
    double *sf = surface_fluxes3(c, u, NULL, 1);
    dg_residual3(c, u, sf, res);
    free(sf);
}
void o3_fv_residual(const o3_ctx *c, const double *u, double *res, double *dsum) { fv_residual3(c, u, res, dsum); }
