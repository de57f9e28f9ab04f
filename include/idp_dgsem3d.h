/*
 * idp_dgsem3d.h -- C ABI of the 3D IDP-limited LGL-DGSEM (arXiv 2607.06045,
 * Sec. 2 with d = 3) on Cartesian grids and 2:1-balanced octrees of
 * hexahedra, in the same library as idp_dgsem.h (libidpdgsem.so, CUDA,
 * sm_103a).
 *
 * The method per stage: the flux-differencing volume terms of
 * Eq. evolutionformula along x, y and z with Ranocha's two-point flux and
 * LLF faces; the low-order graph-viscosity scheme of
 * Eq. LowOrderScheme_globalIndices; bar-state density bounds and positivity
 * (Eqs. Bounds_Positivity, Bounds_Barstates); Zalesak density limiting and
 * the pressure factor with Gamma = 2d = 6 (Sec. 2.3); the IDP time step
 * (Eq. timestep_restriction) and SSP-RK3 (Sec. 3). FP64 throughout. On an
 * octree a face between a leaf and four finer ones is a mortar with 2 x 2
 * small faces (Sec. 2.2 in 3D): the L2 mortar flux as the tensor product of
 * the 1D interpolation and exact L2 projection, the sparse low-order mortar
 * flux of Eq. interfaceflux_local with products of the 1D overlap weights
 * (App. A), the bar states of its pairs in the density bounds, and one
 * factor per mortar after the volume correction with each node's share
 * scaled by its number of mortars n_i (Sec. 2.3); a mortar whose
 * interpolated states leave the admissible set keeps its low-order flux.
 *
 * State layout (caller-owned device memory): u[5][K][N+1][N+1][N+1] doubles,
 * variables (rho, rho v1, rho v2, rho v3, rho e), then element, then node
 * (k, j, i) with the x index i fastest; on a grid e = (ez ny + ey) nx + ex,
 * on an octree the caller's leaf order. Degrees N = 1..4. Errors: the
 * idp_status codes of idp_dgsem.h.
 */
#ifndef IDP_DGSEM3D_H
#define IDP_DGSEM3D_H

#include <stdint.h>

#include "idp_dgsem.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct idp3d_ctx idp3d_ctx;

/* The grid: nx x ny x nz elements over [x0,x1] x [y0,y1] x [z0,z1]; bc per
 * side (-x, +x, -y, +y, -z, +z) one of IDP_BC_PERIODIC, IDP_BC_WALL
 * (mirrored normal momentum), IDP_BC_DIRICHLET (the primitive state
 * bc_prim[s] = rho, v1, v2, v3, p) or IDP_BC_OUTFLOW (copy); opposite sides
 * are both periodic or neither. */
typedef struct {
    int32_t nx, ny, nz;
    double x0, y0, z0, x1, y1, z1;
    int32_t bc[6];
    double bc_prim[6][5];
} idp3d_grid_desc;

/* limiting: 0 none (the high-order scheme), 1 positivity, 2 local (density
 * bounds from the bar states, with positivity), 3 combined (Sec. 3.5, Eq.
 * combination_posLim_local: per interface and per mortar (1 - a) times the
 * positivity factor plus a times the local one, a the element's shock
 * indicator, the modal energy of the pressure in the tensor Legendre basis;
 * a mortar takes the largest of its five elements'); beta the positivity factor
 * of Eq. Bounds_Positivity (0.1); cfl the factor on the IDP time step;
 * precision 0 FP64 throughout, 1 the FP32 form: node primitives and the
 * two-point, face and subcell fluxes of the element pass in FP32, the bar
 * states, bounds, limiter, sums, stage update, mortars and time step in
 * FP64. */
typedef struct {
    int32_t limiting;
    double beta;
    double cfl;
    int32_t precision;
} idp3d_options;

/* limiting 2, beta 0.1, cfl 0.5, precision 0 */
idp_status idp3d_options_default(idp3d_options *o);

/* Context for one grid and degree N (1..4); *out receives it. IDP_E_ARG for
 * bad arguments (N, sizes, a box of non-positive extent, inconsistent
 * periodic sides, options out of range), IDP_E_CUDA on a CUDA failure. */
idp_status idp3d_create(const idp3d_grid_desc *grid, int32_t N, double gamma, const idp3d_options *opts,
                        idp3d_ctx **out);

/* Context for the leaves of a 2:1-balanced octree over the box of `base`,
 * whose nx, ny, nz give the level-0 grid: leaf e (0 <= e < n_leaves) is cell
 * (ix[e], iy[e], iz[e]) of the (nx 2^l) x (ny 2^l) x (nz 2^l) grid of its
 * level l = level[e] (0..18). Host arrays, read during the call only. The
 * leaves must tile the box, and leaves sharing a face differ by at most one
 * level (across periodic sides too): IDP_E_ARG otherwise, as for the
 * arguments of idp3d_create. */
idp_status idp3d_create_octree(const idp3d_grid_desc *base, int64_t n_leaves, const int8_t *level, const int32_t *ix,
                               const int32_t *iy, const int32_t *iz, int32_t N, double gamma,
                               const idp3d_options *opts, idp3d_ctx **out);

/* n_elems and nodes per element (N+1)^3; either may be NULL. */
idp_status idp3d_layout(const idp3d_ctx *ctx, int64_t *n_elems, int32_t *nodes_per_elem);

/* The last limited stage's factors (after idp3d_rhs or idp3d_step): the
 * combined limiting's shock indicator per element (alpha_host[n_elems]; set
 * by stages with limiting 3 only) and each mortar's factor l_S
 * (mortar_ell_host[n_mortars]); either may be NULL. Synchronises `stream`
 * and the context's stream. */
idp_status idp3d_stage_factors(idp3d_ctx *ctx, double *alpha_host, double *mortar_ell_host, void *stream);

/* the number of mortars and of nodes on mortars; either may be NULL */
idp_status idp3d_mesh_info(const idp3d_ctx *ctx, int64_t *n_mortars, int64_t *n_mortar_nodes);

/* The connectivity idp3d_create_octree builds, on the host only (no device
 * memory, no CUDA call): the number of mortars and mortar nodes, and, where
 * the arrays are not NULL, mortar_info[7 M] (per mortar: direction d, large
 * leaf, 1 if the large leaf is on the low side of the face, the four small
 * leaves p = p1 + 2 p2 by their offsets along (d+1) mod 3 and (d+2) mod 3)
 * and nbr[6 n_leaves] (per leaf side -x, +x, -y, +y, -z, +z: the conforming
 * neighbour, -1 at a boundary, or -2 minus the side's first mortar slot,
 * slot = mortar * 5 (N+1)^2 + face * (N+1)^2, face 0 the large one).
 * Call with NULL arrays for the counts first. IDP_E_ARG as for
 * idp3d_create_octree. */
idp_status idp3d_octree_tables(const idp3d_grid_desc *base, int64_t n_leaves, const int8_t *level, const int32_t *ix,
                               const int32_t *iy, const int32_t *iz, int32_t N, int64_t *n_mortars,
                               int64_t *n_mortar_nodes, int32_t *mortar_info, int32_t *nbr);

/* rhs = the limited residual per unit mass of u for a stage of length dt
 * (dt = 0: the unlimited high-order residual), device arrays in the layout
 * above. Asynchronous on `stream`. */
idp_status idp3d_rhs(idp3d_ctx *ctx, const double *u, double dt, double *rhs, void *stream);

/* *dt_host = cfl * min_i m_i / sum_j 2 d_ij of u (Eq. timestep_restriction).
 * Synchronises `stream`. IDP_E_NUMERIC if u holds a non-admissible state. */
idp_status idp3d_dt(idp3d_ctx *ctx, const double *u, double *dt_host, void *stream);

/* n_steps SSP-RK3 steps of u in place (device array), each with the IDP time
 * step of its u^n; t_host (in/out) the time, dt_last_host (may be NULL) the
 * last step's dt. The step is one CUDA graph per state pointer, launched on
 * `stream` (the context's own stream when NULL). Synchronises. IDP_E_NUMERIC
 * if a stage met a non-admissible input or (with statistics on) a bound
 * violation. */
idp_status idp3d_step(idp3d_ctx *ctx, double *u, int32_t n_steps, double *t_host, double *dt_last_host,
                      void *stream);

/* out_host[5] = sum_i m_i u_i (conservation totals), summed in a fixed order.
 * Synchronises `stream`. */
idp_status idp3d_integrals(idp3d_ctx *ctx, const double *u, double *out_host, void *stream);

/* Statistics of the limited stages since the last call (then reset):
 * mass-weighted mean of 1 - (the node's smallest interface factor), nodes
 * with a factor below one, violations of the density bounds and of the
 * pressure bound (beyond 1e-13 relative), non-admissible results, the
 * smallest density and pressure seen, and the stage count; on octrees the
 * area-weighted mean of 1 - l_S over the mortars, the mortars with l_S < 1
 * and those that kept their low-order flux (counted per stage). */
typedef struct {
    double alpha_mean;
    int64_t n_active, n_viol_density, n_viol_pressure, n_nonpositive, n_stages;
    double min_rho, min_p;
    double alpha_mortar;
    int64_t n_mortar_active, n_mortar_fallback;
} idp3d_stats;

idp_status idp3d_limiter_stats(idp3d_ctx *ctx, idp3d_stats *out, void *stream);

void idp3d_destroy(idp3d_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* IDP_DGSEM3D_H */
