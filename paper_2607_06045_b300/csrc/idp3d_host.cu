// idp3d_host.cu -- host runtime and C ABI of the 3D IDP-limited LGL-DGSEM
// (include/idp_dgsem3d.h): the grid and operators on the device, the
// SSP-RK3 step as one CUDA graph (time step, three limited stages, time
// advance), right-hand sides, time steps, conservation totals and limiter
// statistics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/idp_dgsem3d.h"
#include "idp3d_launch.h"

namespace idp {
void host_lgl_sbar(int N, double *x, double *w, double *S);
}

using namespace idp3;

struct idp3d_ctx {
    int N = 0, NP = 0;
    double gamma = 1.4;
    idp3d_options opt{};
    Grid3 grid{};
    Launchers3 L;
    int grid_el = 1;               // element-kernel blocks
    Ops3 *d_ops = nullptr;
    double *d_buf1 = nullptr, *d_buf2 = nullptr, *d_part = nullptr, *d_tot = nullptr;
    unsigned long long *d_dtmin = nullptr, *d_dtmin2 = nullptr;
    double *d_t = nullptr, *d_dtlast = nullptr;
    unsigned *d_status = nullptr;
    Stats3 *d_stats = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph = nullptr;
    const double *graph_u = nullptr;
    long long n_stages = 0;
    double volume = 0.0;
};

namespace {

constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

size_t nodes_of(const idp3d_ctx *c) { return (size_t)c->grid.K * c->NP * c->NP * c->NP; }

Launchers3 get3(int np) {
    switch (np) {
    case 2: return launchers3_np2();
    case 3: return launchers3_np3();
    case 4: return launchers3_np4();
    default: return launchers3_np5();
    }
}

idp_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? IDP_OK : IDP_E_CUDA; }

void p2c(double g, const double *w, double *q) {
    q[0] = w[0];
    for (int a = 0; a < 3; ++a) q[1 + a] = w[0] * w[1 + a];
    q[4] = w[4] / (g - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

Stage3 stage_args(idp3d_ctx *c, const double *u, const double *un, double *out, int mode, int comb) {
    Stage3 A;
    std::memset(&A, 0, sizeof(A));
    A.u = u; A.un = un; A.out = out;
    A.dtmin = c->d_dtmin; A.cfl = c->opt.cfl;
    A.mode = mode; A.comb = comb;
    A.limiting = c->opt.limiting;
    A.collect = 1;
    A.beta = c->opt.beta; A.gamma = c->gamma;
    A.stats = c->d_stats; A.status = c->d_status;
    return A;
}

int dt_grid(const idp3d_ctx *c) { return (c->grid.K + c->L.epb - 1) / c->L.epb; }

// one SSP-RK3 step of u in place (Shu-Osher): u1 = u~(u), u2 = 3/4 u + 1/4 u~(u1),
// u = 1/3 u + 2/3 u~(u2); dt from u^n
void enqueue_step(idp3d_ctx *c, cudaStream_t st, double *u) {
    c->L.dt(dt_grid(c), st, c->grid, c->d_ops, u, c->gamma, c->d_dtmin, c->d_status);
    Stage3 A = stage_args(c, u, u, c->d_buf1, 1, 0);
    c->L.element(c->grid_el, st, c->grid, c->d_ops, A);
    A = stage_args(c, c->d_buf1, u, c->d_buf2, 1, 1);
    c->L.element(c->grid_el, st, c->grid, c->d_ops, A);
    A = stage_args(c, c->d_buf2, u, u, 1, 2);   // each node reads its own u^n, then writes it
    c->L.element(c->grid_el, st, c->grid, c->d_ops, A);
    k_advance3d<<<1, 32, 0, st>>>(c->d_t, c->d_dtmin, c->opt.cfl, c->d_dtlast);
}

idp_status read_status3(idp3d_ctx *c) {
    unsigned s = 0;
    if (cudaMemcpy(&s, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return IDP_E_CUDA;
    if (s && cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess) return IDP_E_CUDA;
    if (s & S_BAD_INPUT) return IDP_E_STATE;
    if (s & S_VIOLATION) return IDP_E_NUMERIC;
    return IDP_OK;
}

cudaError_t reset_stats3(idp3d_ctx *c, cudaStream_t st) {
    Stats3 z;
    std::memset(&z, 0, sizeof(z));
    z.min_rho_bits = kInfBits;
    z.min_p_bits = kInfBits;
    cudaError_t e = cudaMemcpyAsync(c->d_stats, &z, sizeof(z), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// per-element sums of m u into part[5][K], then one block sums them in a fixed order
__global__ void k_part3(Grid3 G, const Ops3 *ops, const double *u, int NP, double *part) {
    const int NN = NP * NP * NP;
    const size_t KN = (size_t)G.K * NN;
    const double J = G.dx * G.dy * G.dz / 8.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < G.K; e += gridDim.x * blockDim.x) {
        double s[NV] = {0, 0, 0, 0, 0};
        for (int n = 0; n < NN; ++n) {
            const int i = n % NP, j = (n / NP) % NP, k = n / (NP * NP);
            const double m = ops->w[i] * ops->w[j] * ops->w[k] * J;
            for (int v = 0; v < NV; ++v) s[v] += m * u[v * KN + (size_t)e * NN + n];
        }
        for (int v = 0; v < NV; ++v) part[(size_t)v * G.K + e] = s[v];
    }
}

__global__ void __launch_bounds__(1024) k_sum3(const double *part, int K, double *out) {
    __shared__ double sh[1024];
    for (int v = 0; v < NV; ++v) {
        double s = 0.0;
        for (int e = threadIdx.x; e < K; e += 1024) s += part[(size_t)v * K + e];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int h = 512; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[v] = sh[0];
        __syncthreads();
    }
}

}  // namespace

extern "C" {

idp_status idp3d_options_default(idp3d_options *o) {
    if (!o) return IDP_E_ARG;
    o->limiting = 2;
    o->beta = 0.1;
    o->cfl = 0.5;
    return IDP_OK;
}

idp_status idp3d_create(const idp3d_grid_desc *gd, int32_t N, double gamma, const idp3d_options *opts,
                        idp3d_ctx **out) {
    if (!out) return IDP_E_ARG;
    *out = nullptr;
    if (!gd || N < 1 || N > 4 || !(gamma > 1.0)) return IDP_E_ARG;
    if (gd->nx < 1 || gd->ny < 1 || gd->nz < 1 || !(gd->x1 > gd->x0) || !(gd->y1 > gd->y0) || !(gd->z1 > gd->z0))
        return IDP_E_ARG;
    if ((long long)gd->nx * gd->ny * gd->nz > (1LL << 24)) return IDP_E_ARG;
    for (int s = 0; s < 6; ++s)
        if (gd->bc[s] < IDP_BC_PERIODIC || gd->bc[s] > IDP_BC_OUTFLOW) return IDP_E_ARG;
    for (int d = 0; d < 3; ++d)
        if ((gd->bc[2 * d] == IDP_BC_PERIODIC) != (gd->bc[2 * d + 1] == IDP_BC_PERIODIC)) return IDP_E_ARG;
    idp3d_options o;
    idp3d_options_default(&o);
    if (opts) o = *opts;
    if (o.limiting < 0 || o.limiting > 2 || !(o.beta >= 0.0 && o.beta < 1.0) || !(o.cfl > 0.0)) return IDP_E_ARG;
    idp3d_ctx *c = new (std::nothrow) idp3d_ctx();
    if (!c) return IDP_E_ARG;
    c->N = N; c->NP = N + 1; c->gamma = gamma; c->opt = o;
    Grid3 &G = c->grid;
    G.nx = gd->nx; G.ny = gd->ny; G.nz = gd->nz; G.K = gd->nx * gd->ny * gd->nz;
    G.dx = (gd->x1 - gd->x0) / gd->nx; G.dy = (gd->y1 - gd->y0) / gd->ny; G.dz = (gd->z1 - gd->z0) / gd->nz;
    for (int s = 0; s < 6; ++s) {
        G.bc[s] = gd->bc[s];
        p2c(gamma, gd->bc_prim[s], G.bc_cons[s]);
    }
    c->volume = (gd->x1 - gd->x0) * (gd->y1 - gd->y0) * (gd->z1 - gd->z0);
    c->L = get3(c->NP);
    c->grid_el = (G.K + c->L.epb - 1) / c->L.epb;
    Ops3 ops;
    std::memset(&ops, 0, sizeof(ops));
    {
        double x[NPMAX3], w[NPMAX3], S[NPMAX3 * NPMAX3];
        idp::host_lgl_sbar(N, x, w, S);
        for (int i = 0; i <= N; ++i) { ops.xi[i] = x[i]; ops.w[i] = w[i]; ops.iw[i] = 1.0 / w[i]; }
        for (int i = 0; i <= N; ++i) for (int j = 0; j <= N; ++j) ops.S[i][j] = S[i * (N + 1) + j];
    }
    bool ok = true;
    auto chk = [&](cudaError_t e) { if (e != cudaSuccess) ok = false; };
    const size_t kn = nodes_of(c);
    chk(c->L.prepare());
    if (ok) chk(cudaMalloc(&c->d_ops, sizeof(Ops3)));
    if (ok) chk(cudaMemcpy(c->d_ops, &ops, sizeof(Ops3), cudaMemcpyHostToDevice));
    if (ok) chk(cudaMalloc(&c->d_buf1, sizeof(double) * NV * kn));
    if (ok) chk(cudaMalloc(&c->d_buf2, sizeof(double) * NV * kn));
    if (ok) chk(cudaMalloc(&c->d_part, sizeof(double) * NV * (size_t)G.K));
    if (ok) chk(cudaMalloc(&c->d_tot, sizeof(double) * NV));
    if (ok) chk(cudaMalloc(&c->d_dtmin, sizeof(unsigned long long)));
    if (ok) chk(cudaMalloc(&c->d_dtmin2, sizeof(unsigned long long)));
    if (ok) chk(cudaMemcpy(c->d_dtmin, &kInfBits, sizeof(kInfBits), cudaMemcpyHostToDevice));
    if (ok) chk(cudaMalloc(&c->d_t, sizeof(double)));
    if (ok) chk(cudaMalloc(&c->d_dtlast, sizeof(double)));
    if (ok) chk(cudaMalloc(&c->d_status, sizeof(unsigned)));
    if (ok) chk(cudaMemset(c->d_status, 0, sizeof(unsigned)));
    if (ok) chk(cudaMalloc(&c->d_stats, sizeof(Stats3)));
    if (ok) chk(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    if (ok) chk(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    if (ok) chk(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    if (ok) chk(reset_stats3(c, c->stream));
    if (!ok) { idp3d_destroy(c); return IDP_E_CUDA; }
    *out = c;
    return IDP_OK;
}

idp_status idp3d_layout(const idp3d_ctx *c, int64_t *n_elems, int32_t *nodes_per_elem) {
    if (!c) return IDP_E_ARG;
    if (n_elems) *n_elems = c->grid.K;
    if (nodes_per_elem) *nodes_per_elem = c->NP * c->NP * c->NP;
    return IDP_OK;
}

idp_status idp3d_rhs(idp3d_ctx *c, const double *u, double dt, double *rhs, void *stream) {
    if (!c || !u || !rhs || !(dt >= 0.0)) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Stage3 A = stage_args(c, u, u, rhs, 0, 0);
    A.dtmin = nullptr;
    A.dt_host = dt;
    A.collect = 0;
    if (dt == 0.0) A.limiting = 0;   // the unlimited high-order residual
    c->L.element(c->grid_el, st, c->grid, c->d_ops, A);
    return cuda_ok(cudaGetLastError());
}

idp_status idp3d_dt(idp3d_ctx *c, const double *u, double *dt_host, void *stream) {
    if (!c || !u || !dt_host) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long b = kInfBits;
    if (cudaMemcpyAsync(c->d_dtmin2, &kInfBits, sizeof(kInfBits), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return IDP_E_CUDA;
    c->L.dt(dt_grid(c), st, c->grid, c->d_ops, u, c->gamma, c->d_dtmin2, c->d_status);
    if (cudaMemcpyAsync(&b, c->d_dtmin2, sizeof(b), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return IDP_E_CUDA;
    double v;
    std::memcpy(&v, &b, sizeof(v));
    *dt_host = c->opt.cfl * v;
    idp_status r = read_status3(c);
    if (r != IDP_OK) return r;
    return std::isfinite(v) ? IDP_OK : IDP_E_DT;
}

idp_status idp3d_step(idp3d_ctx *c, double *u, int32_t n_steps, double *t_host, double *dt_last_host,
                      void *stream) {
    if (!c || !u || n_steps < 0 || !t_host) return IDP_E_ARG;
    cudaStream_t ust = (cudaStream_t)stream;
    const bool own = ust == nullptr;
    cudaStream_t st = own ? c->stream : ust;
    if (own && (cudaEventRecord(c->ev_in, ust) != cudaSuccess || cudaStreamWaitEvent(st, c->ev_in, 0) != cudaSuccess))
        return IDP_E_CUDA;
    if (cudaMemcpyAsync(c->d_t, t_host, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) return IDP_E_CUDA;
    if (n_steps > 0) {
        if (c->graph == nullptr || c->graph_u != u) {
            if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
            cudaGraph_t g;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return IDP_E_CUDA;
            enqueue_step(c, st, u);
            if (cudaStreamEndCapture(st, &g) != cudaSuccess) return IDP_E_CUDA;
            cudaError_t e = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { c->graph = nullptr; return IDP_E_CUDA; }
            c->graph_u = u;
        }
        for (int k = 0; k < n_steps; ++k)
            if (cudaGraphLaunch(c->graph, st) != cudaSuccess) return IDP_E_CUDA;
        c->n_stages += 3LL * n_steps;
    }
    cudaMemcpyAsync(t_host, c->d_t, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (dt_last_host && n_steps > 0) cudaMemcpyAsync(dt_last_host, c->d_dtlast, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (own) {
        cudaEventRecord(c->ev_out, st);
        cudaStreamWaitEvent(ust, c->ev_out, 0);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return IDP_E_CUDA;
    return read_status3(c);
}

idp_status idp3d_integrals(idp3d_ctx *c, const double *u, double *out_host, void *stream) {
    if (!c || !u || !out_host) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (c->grid.K + 255) / 256;
    k_part3<<<blocks, 256, 0, st>>>(c->grid, c->d_ops, u, c->NP, c->d_part);
    k_sum3<<<1, 1024, 0, st>>>(c->d_part, c->grid.K, c->d_tot);
    if (cudaMemcpyAsync(out_host, c->d_tot, sizeof(double) * NV, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return IDP_E_CUDA;
    return cuda_ok(cudaGetLastError());
}

idp_status idp3d_limiter_stats(idp3d_ctx *c, idp3d_stats *out, void *stream) {
    if (!c || !out) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Stats3 a;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(&a, c->d_stats, sizeof(a), cudaMemcpyDeviceToHost) != cudaSuccess)
        return IDP_E_CUDA;
    std::memset(out, 0, sizeof(*out));
    const double mass = c->volume * (double)c->n_stages;
    out->alpha_mean = mass > 0.0 ? a.alpha_m / mass : 0.0;
    out->n_active = (int64_t)a.n_active;
    out->n_viol_density = (int64_t)a.n_vrho;
    out->n_viol_pressure = (int64_t)a.n_vp;
    out->n_nonpositive = (int64_t)a.n_nonpos;
    out->n_stages = c->n_stages;
    std::memcpy(&out->min_rho, &a.min_rho_bits, sizeof(double));
    std::memcpy(&out->min_p, &a.min_p_bits, sizeof(double));
    c->n_stages = 0;
    if (reset_stats3(c, c->stream) != cudaSuccess) return IDP_E_CUDA;
    return read_status3(c);
}

void idp3d_destroy(idp3d_ctx *c) {
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    void *ptrs[] = {c->d_ops, c->d_buf1, c->d_buf2, c->d_part, c->d_tot, c->d_dtmin, c->d_dtmin2, c->d_t,
                    c->d_dtlast, c->d_status, c->d_stats};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
