/*
 * idp_dgsem.h -- C ABI of the B300 (sm_103a) implementation of the
 * right-hand side and SSP Runge-Kutta step of the invariant-domain-preserving
 * (IDP) LGL-DGSEM for the 2D compressible Euler equations on 2:1-balanced
 * Cartesian quadtrees with hanging nodes (Bolm, Rueda-Ramirez, Kuzmin,
 * Gassner, arXiv 2607.06045).
 *
 * The problem statement follows the paper: a conservation law on a domain
 * with an initial condition and boundary conditions (Sec. 2, Eq.
 * conservationlaw), a quadtree whose leaves are the elements (Sec. 3.1) and
 * whose face neighbours differ by at most one level (Sec. 2.2), a polynomial
 * degree N and the ratio of specific heats gamma (Sec. 3).
 *
 * Conventions shared by every entry point:
 *  - All functions return an idp_status; none aborts, traps or prints, and no
 *    C++ exception crosses the interface.
 *  - State arrays are caller-owned DEVICE pointers to contiguous FP64 data in
 *    the layout u[4][K][N+1][N+1]: variable (rho, rho v1, rho v2, E), then
 *    element in the caller's leaf order (batched contexts concatenate the
 *    simulations along K), then node j (y) and node i (x, fastest), the local
 *    node ordering of Sec. 2.1. u must be 8-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL: the legacy default
 *    stream). Work is enqueued asynchronously on it; conditions detected on
 *    the device (invalid input state, bound violations) are reported by the
 *    next synchronising call: idp_dgsem_step, idp_dgsem_step_host,
 *    idp_dgsem_sync or idp_dgsem_limiter_stats.
 *  - One context is used by one stream at a time; calls that overlap on the
 *    GPU through the same context race on its scratch buffers.
 */
#ifndef IDP_DGSEM_H
#define IDP_DGSEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IDP_OK = 0,
    IDP_E_ARG = 1,        /* invalid argument (NULL pointer, N out of range, bad option) */
    IDP_E_MESH = 2,       /* leaves overlap, leave a gap, lie outside the grid or are not 2:1 */
    IDP_E_CUDA = 3,       /* a CUDA runtime call failed */
    IDP_E_STATE = 4,      /* input state has rho <= 0, p <= 0 or a non-finite entry */
    IDP_E_DT = 5,         /* no admissible time step (e.g. zero wave speed everywhere) */
    IDP_E_NUMERIC = 6,    /* a limited stage left a bound violated beyond tolerance */
    IDP_E_TIMEOUT = 7,    /* reserved for bounded device waits */
    IDP_E_UNSUPPORTED = 8 /* option combination not built */
} idp_status;

/* Boundary kinds per domain side (Sec. 3.5 describes the double Mach
 * reflection boundaries in words; ghost states are used in the LLF flux and
 * in the bar states):
 *  PERIODIC  the opposite side (both sides of a direction must be periodic);
 *  WALL      reflecting slip wall: ghost = interior state with the normal
 *            momentum mirrored;
 *  DIRICHLET ghost = bc_prim[side] (rho, v1, v2, p);
 *  OUTFLOW   ghost = interior state;
 *  DMR       double Mach reflection: side -x post-shock Dirichlet, +x
 *            outflow, -y post-shock Dirichlet for x < 1/6 and wall
 *            otherwise, +y post-shock for x < 1/6 + (y1 + 20 t)/sqrt(3) and
 *            pre-shock otherwise (states dmr_post and dmr_pre);
 *  JET       high-Mach jet (Sec. 3, astrophysical jet): on side -x the
 *            inflow state dmr_post for |y| <= 0.05 and the ambient state
 *            dmr_pre elsewhere, on side +x the ambient state dmr_pre (both
 *            Dirichlet), outflow on the y sides. */
typedef enum {
    IDP_BC_PERIODIC = 0,
    IDP_BC_WALL = 1,
    IDP_BC_DIRICHLET = 2,
    IDP_BC_OUTFLOW = 3,
    IDP_BC_DMR = 4,
    IDP_BC_JET = 5
} idp_bc;

/* A quadtree mesh: an nx0 x ny0 level-0 grid over [x0,x1] x [y0,y1]; leaf e
 * has level level[e] and integer position (ix[e], iy[e]) on the level-l grid
 * of (nx0 2^l) x (ny0 2^l) cells. All arrays are HOST memory owned by the
 * caller and copied at create time. */
typedef struct {
    int32_t nx0, ny0;
    double x0, y0, x1, y1;
    int32_t n_leaves;
    const int8_t *level;
    const int32_t *ix;
    const int32_t *iy;
    int32_t bc[4];          /* idp_bc for sides -x, +x, -y, +y */
    double bc_prim[4][4];   /* DIRICHLET primitive state per side */
    double dmr_post[4];     /* DMR post-shock primitive state */
    double dmr_pre[4];      /* DMR pre-shock primitive state */
} idp_mesh_desc;

/* Method options (Sec. 2.3 and Sec. 3):
 *  precision  0: all arithmetic FP64; 1: FP32 form -- node primitives, two-
 *             point volume fluxes, subcell and face fluxes in FP32; bounds,
 *             limiter solves, blending, stage update and all sums in FP64.
 *  limiting   0: none (high-order DG); 1: positivity limiting
 *             (Eq. Bounds_Positivity); 2: local limiting -- bar-state density
 *             bounds (Eq. Bounds_Barstates, density part) plus positivity;
 *             3: combined -- per interface and per mortar the factor
 *             (1 - a) l_positivity + a l_local with a the element's shock
 *             indicator (Hennemann et al.'s modal energy indicator of the
 *             pressure; for a mortar the largest of its three elements),
 *             Sec. 3.5 Eq. combination_posLim_local.
 *  bounds     kind of the local bounds (limiting 2 and the local half of 3):
 *             0: bar states of the node and its graph neighbours
 *             (Eq. Bounds_Barstates); 1: the low-order solution of the node
 *             and its neighbours (Eq. Bounds_LowOrder; ghost states are not
 *             neighbours). Kind 1 adds a low-order pre-pass over the elements
 *             and a per-mortar gather to every limited stage.
 *  dt_rule    0: IDP restriction (Eq. timestep_restriction); 1: low-order
 *             CFL estimate (Eq. CFLcondition_lowordermethod).
 *  beta       positivity factor of Eq. Bounds_Positivity (paper: 0.1).
 *  cfl        dt = cfl * (rule's limit).
 *  mortar_projection  0: LGL-weighted adjoint of the interpolation; 1: exact
 *             L2 projection (default) for the high-order mortar flux.
 *  elems_per_block  0: autotune; else elements per thread block.
 *  collect_stats    1: accumulate limiter statistics (idp_limiter_stats).
 *  grid_mode  element-pass grid: 0 chosen by the autotuner (or one block per
 *             element batch when elems_per_block is set), 1 one block per
 *             element batch, 2 persistent (a grid of resident blocks that
 *             loops over the batches).
 *  entropy_bound  1: local limiting also keeps the modified specific entropy
 *             eta = p rho^-gamma / (gamma - 1) at or above the minimum of eta
 *             over the bounds' states (right parts of Eqs. Bounds_Barstates
 *             and Bounds_LowOrder), relaxed by 1e-12 relative; 0: off.
 *  volume_flux  two-point volume flux of the split form: 0 Ranocha's
 *             entropy-conserving, kinetic-energy-preserving flux (Sec. 3);
 *             1 Chandrashekar's (the paper's astrophysical jet).
 *  mortar_low weights of the low-order mortar flux: 0 the sparse local
 *             weights (Eq. local_weights, App. A); 1 the all-to-all weights
 *             (Eq. nonlocal_weight, by the small face's LGL quadrature), the
 *             diffusive baseline the paper starts from. */
typedef struct {
    int32_t precision;
    int32_t limiting;
    int32_t bounds;
    int32_t dt_rule;
    double beta;
    double cfl;
    int32_t mortar_projection;
    int32_t elems_per_block;
    int32_t collect_stats;
    int32_t grid_mode;
    int32_t entropy_bound;
    int32_t volume_flux;
    int32_t mortar_low;
} idp_options;

/* Limiter statistics accumulated over the stages since the previous call of
 * idp_dgsem_limiter_stats (Sec. 3: weighted averages of the limiting factors
 * alpha = 1 - l over elements and over mortars). */
typedef struct {
    double alpha_volume_mean;   /* mass-weighted mean of 1 - min_k l_ik over nodes */
    double alpha_mortar_mean;   /* face-length-weighted mean of alpha_S over mortars */
    int64_t n_stages;
    int64_t n_volume_active;    /* node-stages with alpha > 0 */
    int64_t n_mortar_active;    /* mortar-stages with alpha_S > 0 */
    int64_t n_mortar_fallback;  /* mortar-stages whose interpolated states were inadmissible */
    int64_t n_viol_density;     /* node-stages outside [rho_min, rho_max] beyond 1e-13 relative */
    int64_t n_viol_pressure;    /* node-stages with p < p_min beyond 1e-13 relative */
    int64_t n_nonpositive;      /* node-stages with rho <= 0 or p <= 0 */
    int64_t n_dt_exceed;        /* node-stages with dt sum_j 2 d_ij / m_i > 1 */
    double min_rho, min_p;      /* over limited stage states */
    int64_t n_viol_entropy;     /* node-stages with eta below its bound beyond 1e-11 relative */
} idp_limiter_stats;

typedef struct idp_ctx idp_ctx;

/* Fill *o with the defaults: FP64, local limiting, bar-state bounds, IDP dt,
 * beta 0.1, cfl 0.5, exact L2 projection, autotuned blocks, stats on. */
idp_status idp_options_default(idp_options *o);

/* Build a context for one mesh (the paper's Sec. 2.1-2.3): validates the leaves
 * (IDP_E_MESH when they overlap, leave a gap or are not 2:1 face-balanced),
 * builds the conforming-face, boundary and mortar lists, the LGL operators
 * (nodes, weights, Sbar = 2 Qbar - Bbar), the local mortar weights
 * (Eq. local_weights) and the mortar interpolation/projection, and uploads
 * them to the current CUDA device. 1 <= N <= 7. opts may be NULL (defaults).
 * On success *ctx owns all device tables and scratch; free with
 * idp_dgsem_destroy. */
idp_status idp_dgsem_create(const idp_mesh_desc *mesh, int32_t N, double gamma,
                            const idp_options *opts, idp_ctx **ctx);

/* As idp_dgsem_create for n_sims independent meshes that are advanced
 * together; their elements are concatenated in the given order and every
 * simulation keeps its own time step and time. */
idp_status idp_dgsem_create_batch(const idp_mesh_desc *meshes, int32_t n_sims, int32_t N,
                                  double gamma, const idp_options *opts, idp_ctx **ctx);

/* Sizes: total elements, mortars, simulations; sim_elem_offsets (host,
 * n_sims + 1 entries, may be NULL) receives the first element of each
 * simulation. */
idp_status idp_dgsem_layout(const idp_ctx *ctx, int64_t *n_elems, int64_t *n_mortars,
                            int32_t *n_sims, int64_t *sim_elem_offsets);

/* Element-pass launch configuration in use: elements per thread block, 1 if
 * the grid is persistent (resident blocks looping over element batches) else
 * 0, and the grid size. Before the first rhs/dt/step call of an autotuned
 * context (elems_per_block = 0) all three are 0. Any pointer may be NULL.
 * Host only; no device work. */
idp_status idp_dgsem_launch_config(const idp_ctx *ctx, int32_t *elems_per_block, int32_t *persistent,
                                   int32_t *grid);

/* Right-hand side at time t (Eq. evolutionformula with the limited fluxes of
 * Sec. 2.3). dt == 0: the unlimited high-order DG right-hand side du/dt.
 * dt > 0: the limited forward-Euler increment (u_lim - u)/dt of one
 * FCT stage, u_lim = u_FV + dt/m (sum of limited antidiffusive fluxes),
 * which depends on dt because the limiter bounds do (Sec. 3.2). The same dt
 * is used for every simulation of a batch. u and rhs: device, layout above,
 * must not alias. */
idp_status idp_dgsem_rhs(idp_ctx *ctx, const double *u, double t, double dt, double *rhs,
                         void *stream);

/* Time step of each simulation for state u at time t under the context's
 * dt_rule and cfl; dt_host receives n_sims values (synchronises the stream). */
idp_status idp_dgsem_dt(idp_ctx *ctx, const double *u, const double *t_host, double *dt_host,
                        void *stream);

/* n_steps SSP-RK3 steps (Shu-Osher form, Sec. 3) in place on the device
 * state u. Each step computes its own dt from u^n (dt_rule, cfl). t_host
 * (n_sims values, in/out) holds each simulation's time; dt_last_host (may be
 * NULL) receives the last dt per simulation. Synchronises the stream at the
 * end and returns IDP_E_STATE or IDP_E_NUMERIC if the device flagged an
 * invalid state or a bound violation. */
idp_status idp_dgsem_step(idp_ctx *ctx, double *u, int32_t n_steps, double *t_host,
                          double *dt_last_host, void *stream);

/* As idp_dgsem_step for a HOST state array: copies u_host to the device,
 * steps, and copies the result back (u_host should be page-locked for
 * asynchronous copies). */
idp_status idp_dgsem_step_host(idp_ctx *ctx, double *u_host, int32_t n_steps, double *t_host,
                               double *dt_last_host, void *stream);

/* Discrete integrals sum_i m_i u_i per simulation and variable (the
 * conserved totals of Eq. conservationProperty), out_host[n_sims][4], summed
 * in a fixed order (deterministic). Synchronises the stream. */
idp_status idp_dgsem_integrals(idp_ctx *ctx, const double *u, double *out_host, void *stream);

/* Read and reset the accumulated limiter statistics (synchronises). */
idp_status idp_dgsem_limiter_stats(idp_ctx *ctx, idp_limiter_stats *out, void *stream);

/* Kernel kinds of one SSP-RK3 step, for idp_dgsem_profile_kernels. */
enum {
    IDP_K_DT_INIT = 0,      /* reset of the per-simulation time-step minimum (a
                               standalone time step; a step needs none) */
    IDP_K_MORTAR_FLUX = 1,  /* mortar fluxes (L2 and sparse IDP), bar states */
    IDP_K_DT = 2,           /* IDP time step */
    IDP_K_ELEMENT = 3,      /* element pass: volume, faces, low order, limiting, stage */
    IDP_K_MORTAR_LIMIT = 4, /* one limiting factor per mortar, then the limited
                               mortar corrections and the stage at mortar nodes */
    IDP_K_MORTAR_APPLY = 5, /* (kept for the numbering: no kernel of this kind
                               is launched, the mortar corrections are part of
                               IDP_K_MORTAR_LIMIT) */
    IDP_K_TIME_ADVANCE = 6, /* per-simulation time */
    IDP_K_ELEMENT_LO = 7,   /* low-order pre-pass of the element pass (bounds 1) */
    IDP_K_MORTAR_LOB = 8,   /* low-order bounds across mortars (bounds 1) */
    IDP_K_FACE = 9,         /* conforming-face fluxes of the FP64 element pass (part of it) */
    IDP_K_DT_SPEED = 10,    /* wave speeds of every node for the time step (no face buffer) */
    IDP_K_DT_FILTER = 11,   /* FP64 path with the face buffer: the time step's FP32 pass,
                               which picks the elements whose quotients IDP_K_DT forms
                               in FP64 */
    IDP_NKERNELS = 12
};

/* Measurement support (the paper has no counterpart). mode 1: each step's
 * CUDA-graph launch is bracketed by CUDA events on the step's stream; mode 2:
 * steps are launched kernel by kernel (no graph) with events around the step
 * and around every kernel launch; mode 0: off. In modes 1 and 2
 * idp_dgsem_step synchronises after every step to accumulate the durations.
 * idp_dgsem_profile_read returns the accumulated element-pass milliseconds
 * (mode 2: the element kernel plus, in the FP64 path, the conforming-face
 * kernel that feeds it) and element-kernel launches, and step milliseconds
 * and steps (any pointer may be NULL;
 * reset != 0 clears them). idp_dgsem_profile_kernels writes, for each kernel
 * kind k < IDP_NKERNELS, the accumulated milliseconds ms[k] and launches
 * launches[k] of mode 2 (caller arrays of IDP_NKERNELS entries, either may be
 * NULL; reset != 0 clears them). */
idp_status idp_dgsem_profile(idp_ctx *ctx, int32_t mode);
idp_status idp_dgsem_profile_read(idp_ctx *ctx, double *element_ms, int64_t *element_launches,
                                  double *step_ms, int64_t *steps, int32_t reset);
idp_status idp_dgsem_profile_kernels(idp_ctx *ctx, double *ms, int64_t *launches, int32_t reset);

/* Pipe-throughput probe used for the roofline (no counterpart in the paper):
 * runs short kernels on the current device and stream and writes out[0] FP64
 * TFLOP/s (DFMA, 2 flops each), out[1] FP32 TFLOP/s (FFMA), out[2..4] the
 * cost of one FP64 reciprocal, square root and logarithm as the FP64 flux
 * arithmetic forms them (each plus one add) in DFMA-equivalents.
 * Synchronises. */
idp_status idp_probe_pipes(double *out, void *stream);

/* Test hook (no counterpart in the paper): y[i] = f(x[i]) for i < n with the
 * FP64 routines of the flux arithmetic, f = 1/x (fn 0), sqrt(x) (fn 1) or
 * ln(x) (fn 2); x and y are caller-owned device arrays of n doubles; inputs
 * are meant to be positive, finite and normal. Runs on the given stream and
 * synchronises it. IDP_E_ARG for fn outside 0..2, n < 0 or null pointers with
 * n > 0; IDP_E_CUDA on a CUDA failure. */
idp_status idp_eval_math(int32_t fn, const double *x, double *y, int64_t n, void *stream);

/* Largest element count accepted by idp_integrals_noalloc. */
#define IDP_NOALLOC_MAX_ELEMS (1 << 19)

/* Conservation totals without any device allocation (the paper has no
 * counterpart). For callers that may not call cudaMalloc: one recording a
 * CUDA graph, a framework that forbids allocations after start-up, or a host
 * callback. Computes out[s][v] = sum over the elements e in
 * [sim_elem_offsets[s], sim_elem_offsets[s+1]) of sum_ij (elem_area[e] / 4)
 * w_i w_j u[v][e][j][i], the same totals as idp_dgsem_integrals, with no
 * context. All pointers are caller-owned DEVICE memory: u (layout as above,
 * n_elems elements, degree N), elem_area (n_elems values dx * dy),
 * sim_elem_offsets (n_sims + 1 values; each is clamped to [0, n_elems], so
 * an offset out of range sums fewer elements, never memory beyond this
 * call's partials) and out (4 * n_sims values). The
 * per-element partial sums go to a fixed array of 4 * IDP_NOALLOC_MAX_ELEMS
 * doubles (16 MiB) that the library keeps on every device it is used on
 * until the process exits; n_elems above IDP_NOALLOC_MAX_ELEMS returns
 * IDP_E_ARG. The first call on a device looks up that array's device address
 * (once per device, with the device current): make it before any stream
 * capture. All calls share the array, so calls that overlap on the GPU race;
 * each call overwrites the partials it reads, nothing carries over between
 * calls. Asynchronous on `stream`; calls no allocating routine. */
idp_status idp_integrals_noalloc(const double *u, const double *elem_area, int64_t n_elems, int32_t N,
                                 const int64_t *sim_elem_offsets, int32_t n_sims, double *out,
                                 void *stream);

/* ---- adaptive mesh refinement (Sec. 2.4 and the adaptive runs of Sec. 3) --
 * One adaptation step is: element indicators on the device
 * (idp_dgsem_amr_indicator), the new leaf set on the host (idp_amr_plan),
 * the solution transfer on the device (idp_amr_transfer), then a context for
 * the new mesh (idp_dgsem_create). idp_dgsem_adapt does all of it on the
 * device, in the context. */

/* Indicator kinds and the variable they look at. */
enum { IDP_AMR_HENNEMANN = 0, IDP_AMR_LOHNER = 1, IDP_AMR_MAX = 2 };
enum { IDP_AMR_DENSITY = 0, IDP_AMR_PRESSURE = 1 };

/* indicator         IDP_AMR_HENNEMANN: Hennemann et al.'s modal energy
 *                   indicator in [0, 1] (as for the combined limiting);
 *                   IDP_AMR_LOHNER: the largest second-difference ratio
 *                   |a - 2b + c| / (|c - b| + |b - a| + f (|a| + 2|b| + |c|))
 *                   over consecutive nodes (a, b, c) of every row and column
 *                   (a Loehner-type estimator, f = lohner_filter);
 *                   IDP_AMR_MAX: the larger of the two.
 * variable          IDP_AMR_DENSITY or IDP_AMR_PRESSURE.
 * refine_threshold  a leaf whose indicator exceeds it is refined one level
 *                   (up to max_level);
 * coarsen_threshold four sibling leaves whose indicators are all below it are
 *                   coarsened one level (down to min_level);
 * zs_threshold      the transfer's positivity threshold for density and
 *                   pressure (Zhang-Shu scaling; the paper uses 1e-10). */
typedef struct {
    int32_t indicator;
    int32_t variable;
    double refine_threshold;
    double coarsen_threshold;
    int32_t min_level, max_level;
    double lohner_filter;
    double zs_threshold;
} idp_amr_params;

/* Fills p with the defaults: Hennemann on density, refine above 0.5, coarsen
 * below 0.05, levels 0..3, filter 0.2, threshold 1e-10. */
idp_status idp_amr_params_default(idp_amr_params *p);

/* ind[e] = the indicator of element e of u (device arrays: u in the layout
 * above, ind of n_elems doubles). Asynchronous on `stream`. IDP_E_ARG for
 * null pointers or parameters out of range. */
idp_status idp_dgsem_amr_indicator(idp_ctx *ctx, const double *u, const idp_amr_params *p, double *ind,
                                   void *stream);

/* The adapted leaf set of one mesh (host function, no GPU): from the mesh
 * and its elements' indicators (host array, mesh order) one level of
 * refinement or coarsening per leaf; coarsening needs all four siblings to
 * be leaves marked for it; then 2:1 face balance, refinement winning (a
 * coarser face neighbour two levels apart gives up its coarsening or is
 * refined). New leaves follow the old order: a refined leaf becomes its four
 * children c = cx + 2 cy in place, a coarsened family its parent at its
 * first member's place. Outputs (caller-owned host arrays of `capacity`
 * entries; 4 * n_leaves always suffices): n_new, level/ix/iy of the new
 * leaves, kind (0 copy, 1 child, 2 coarsened parent) and src[4] per new
 * leaf (copy: the old leaf; child: the old parent and the child position;
 * parent: the four old children in child order; unused entries -1).
 * IDP_E_ARG for bad arguments or a capacity too small, IDP_E_MESH for an
 * invalid or unbalanced input mesh. */
idp_status idp_amr_plan(const idp_mesh_desc *mesh, const double *ind, const idp_amr_params *p, int32_t capacity,
                        int32_t *n_new, int8_t *level, int32_t *ix, int32_t *iy, int32_t *kind, int32_t *src);

/* The solution on the adapted mesh (device): u_new (n_new elements) from
 * u_old (n_old elements) of degree N by the plan's kind/src (HOST arrays,
 * copied): copies, children by interpolation of the parent, parents by the
 * exact L2 projection of the four children; then every refined family is
 * scaled toward its parent's mean and every coarsened parent toward its own
 * mean, with one factor per family, until density and pressure reach
 * zs_threshold (Zhang-Shu). *n_scaled (host, may be NULL) receives the
 * number of scaled families. Synchronises `stream`. */
idp_status idp_amr_transfer(int32_t N, double gamma, const double *u_old, int64_t n_old, double *u_new, int64_t n_new,
                            const int32_t *kind, const int32_t *src, double zs_threshold, int64_t *n_scaled,
                            void *stream);

/* One adaptation step on the device (Sec. 2.4), the context kept: the
 * indicator of u_old, the plan (as idp_amr_plan: the same marks, families,
 * 2:1 balance sweeps and leaf order, run as data-parallel sweeps until
 * nothing changes), the transfer (as idp_amr_transfer) into u_new, and the
 * face, mortar, mortar-node and limiting-block tables of the new leaves
 * (the same tables, in the same order, as idp_dgsem_create builds for that
 * mesh), all built in the context's device memory; element and mortar
 * buffers grow with slack when the mesh outgrows them and are never shrunk.
 * u_old (the context's n_elems elements, layout above) and u_new are
 * caller-owned device arrays that must not overlap; u_new holds at least
 * 4 capacity (N+1)^2 doubles and receives the adapted state in its first
 * 4 n_new (N+1)^2, laid out for n_new elements. *n_new (host) receives the
 * new element count; when it exceeds capacity the context is unchanged and
 * the call returns IDP_E_ARG (call again with a larger u_new). *n_scaled (host, may
 * be NULL) as for idp_amr_transfer. After the call the context steps u_new
 * on the new mesh (the step graph is captured again on the next step).
 * Single-mesh contexts only (IDP_E_ARG for a batch or while per-kernel
 * profiling is on); IDP_E_MESH if the tables come out invalid, IDP_E_CUDA
 * on a CUDA failure. Synchronises `stream` and the context's own streams. */
idp_status idp_dgsem_adapt(idp_ctx *ctx, const double *u_old, const idp_amr_params *p, double *u_new,
                           int64_t capacity, int64_t *n_new, int64_t *n_scaled, void *stream);

/* The context's leaves (the mesh it steps, after any idp_dgsem_adapt):
 * level, ix, iy of its n_elems elements in element order, copied to
 * caller-owned host arrays. Synchronous. IDP_E_ARG for null pointers. */
idp_status idp_dgsem_leaves(idp_ctx *ctx, int8_t *level, int32_t *ix, int32_t *iy);

/* Test support (no counterpart in the paper): the context's mesh tables
 * copied to caller-owned host arrays, any of which may be NULL to skip it.
 * sizes[6] (required) = n_elems, n_mortars, mortar nodes, mortar limiting
 * blocks, foreign-mortar entries, the largest foreign count of a block.
 * fnbr [n_elems][4] neighbour per side (x-, x+, y-, y+), ftype [n_elems][4]
 * face kind per side, m_large [n_mortars] and m_small [n_mortars][2] the
 * mortars' elements, m_info [n_mortars] orientation and side bits,
 * mn_node [nodes] the element node (e (N+1)^2 + j (N+1) + i) of each mortar
 * node, mn_slot [nodes][2] its first and second mortar slot (-1 when none),
 * mb_node_off and mb_for_off [blocks + 1] per block offsets into mn_node and
 * mb_foreign [entries] (the foreign mortars of each block, ascending).
 * Synchronous. IDP_E_ARG for a null ctx or sizes. */
idp_status idp_dgsem_mesh_tables(idp_ctx *ctx, int64_t *sizes, int32_t *fnbr, uint8_t *ftype, int32_t *m_large,
                                 int32_t *m_small, int32_t *m_info, int32_t *mn_node, int32_t *mn_slot,
                                 int32_t *mb_node_off, int32_t *mb_for_off, int32_t *mb_foreign);

/* Synchronise the stream and report any device-flagged condition. */
idp_status idp_dgsem_sync(idp_ctx *ctx, void *stream);

void idp_dgsem_destroy(idp_ctx *ctx);

const char *idp_status_str(idp_status s);

/* The CUDA error behind the calling thread's most recent IDP_E_CUDA: the
 * failing step and cudaGetErrorString text ("" if none). Diagnostics only;
 * the string is owned by the library. */
const char *idp_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IDP_DGSEM_H */
