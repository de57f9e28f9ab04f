// idp3d_host.cu -- host runtime and C ABI of the 3D IDP-limited LGL-DGSEM
// (include/idp_dgsem3d.h): the octree's connectivity (face neighbours,
// mortars, their slots and nodes) and the operators on the device, the
// SSP-RK3 step as one CUDA graph (mortar fluxes, time step, three limited
// stages with their mortar factors, time advance), right-hand sides, time
// steps, conservation totals and limiter statistics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/idp_dgsem3d.h"
#include "idp3d_launch.h"

namespace idp {
void host_lgl_sbar(int N, double *x, double *w, double *S);
void host_lgl_mortar(int N, double *I, double *P, double *wt);
void host_log_table(LogTab &T);
void host_lgl_indicator(int N, double *Vinv, double *T, double *s);
}

using namespace idp3;

struct idp3d_ctx {
    int N = 0, NP = 0;
    double gamma = 1.4;
    idp3d_options opt{};
    Grid3 grid{};
    Launchers3 L;
    int grid_el = 1, grid_el64 = 1;   // element-kernel blocks: FP32 form, FP64 path
    Ops3 *d_ops = nullptr;
    MOps3 *d_mops = nullptr;
    idp::LogTab *d_lg = nullptr;
    int *d_nbr = nullptr, *d_minfo = nullptr, *d_slot_mn = nullptr, *d_mn_node = nullptr, *d_mn_slot = nullptr;
    int *d_mn_cnt = nullptr, *d_mbad = nullptr;
    signed char *d_lev = nullptr;
    double *d_mslot = nullptr, *d_hand = nullptr, *d_ell = nullptr;
    double *d_buf1 = nullptr, *d_buf2 = nullptr, *d_part = nullptr, *d_tot = nullptr;
    unsigned *d_emin = nullptr;    // FP64 time step: per element, its FP32 pass's minimum
    double *d_ind = nullptr, *d_aind = nullptr;   // combined limiting: indicator operators, per element indicator
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
    A.aind = c->d_aind;
    return A;
}

int dt_grid(const idp3d_ctx *c) { return (c->grid.K + c->L.epb - 1) / c->L.epb; }

bool has_mortars(const idp3d_ctx *c) { return c->grid.mort.M > 0; }

// the time-step kernel of the context's precision
void launch_dt(idp3d_ctx *c, cudaStream_t st, const double *u, unsigned long long *dtmin) {
    if (c->opt.precision == 1) c->L.dt32(dt_grid(c), st, c->grid, c->d_ops, u, c->gamma, dtmin, c->d_status, nullptr);
    else c->L.dt(dt_grid(c), st, c->grid, c->d_ops, u, c->gamma, dtmin, c->d_status, c->d_emin);
}

// one limited stage: the mortar fluxes of its input (unless already formed),
// the element kernel, then the mortar factors and the mortar nodes
void enqueue_stage(idp3d_ctx *c, cudaStream_t st, const Stage3 &A, bool mflux) {
    if (has_mortars(c) && mflux) c->L.mflux(st, c->grid, c->d_mops, A.u, c->gamma);
    if (c->opt.precision == 1) c->L.element32(c->grid_el, st, c->grid, c->d_ops, A);
    else c->L.element(c->grid_el64, st, c->grid, c->d_ops, A);
    if (has_mortars(c)) {
        c->L.mfactor(st, c->grid, A);
        c->L.mapply(st, c->grid, A);
    }
}

// one SSP-RK3 step of u in place (Shu-Osher): u1 = u~(u), u2 = 3/4 u + 1/4 u~(u1),
// u = 1/3 u + 2/3 u~(u2); dt from u^n (its mortar 2 d sums from the first
// stage's mortar fluxes)
void enqueue_step(idp3d_ctx *c, cudaStream_t st, double *u) {
    if (has_mortars(c)) c->L.mflux(st, c->grid, c->d_mops, u, c->gamma);
    launch_dt(c, st, u, c->d_dtmin);
    enqueue_stage(c, st, stage_args(c, u, u, c->d_buf1, 1, 0), false);
    enqueue_stage(c, st, stage_args(c, c->d_buf1, u, c->d_buf2, 1, 1), true);
    // each node reads its own u^n, then writes it
    enqueue_stage(c, st, stage_args(c, c->d_buf2, u, u, 1, 2), true);
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
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < G.K; e += gridDim.x * blockDim.x) {
        double h[3];
        extents3(G, e, h);
        const double J = h[0] * h[1] * h[2] / 8.0;
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

// ---------------------------------------------------------------------------
// octree connectivity
// ---------------------------------------------------------------------------

struct Octree3 {
    std::vector<int> nbr;            // [K][6] (Grid3::nbr)
    std::vector<signed char> lev;    // [K]
    std::vector<int> info;           // [M][7]
    std::vector<int> slot_mn;        // [S]
    std::vector<int> mn_node, mn_cnt;   // [MN]
    std::vector<int> mn_slot;        // [3][MN]
    int M = 0, MN = 0;
};

uint64_t leaf_key(int l, int64_t x, int64_t y, int64_t z) {
    return ((uint64_t)l << 57) | ((uint64_t)x << 38) | ((uint64_t)y << 19) | (uint64_t)z;
}

int node_of_host(int NP, int d, int t, int a) {
    int idx[3];
    idx[d] = a; idx[(d + 1) % 3] = t % NP; idx[(d + 2) % 3] = t / NP;
    return (idx[2] * NP + idx[1]) * NP + idx[0];
}

// Face neighbours (same level), mortars (a leaf whose side faces four finer
// leaves: mortars numbered in the order of their large leaf and side) and
// their slots and nodes. IDP_E_ARG for leaves outside their level's grid,
// duplicates, a gap or overlap, or a level jump above one across a face.
idp_status build_octree3(const idp3d_grid_desc *gd, int64_t K, const int8_t *level, const int32_t *ix,
                         const int32_t *iy, const int32_t *iz, int NP, Octree3 &T) {
    const int64_t n0[3] = {gd->nx, gd->ny, gd->nz};
    std::unordered_map<uint64_t, int> tab;
    tab.reserve((size_t)K * 2);
    int lmax = 0;
    for (int64_t e = 0; e < K; ++e) {
        const int l = level[e];
        if (l < 0 || l > 18) return IDP_E_ARG;
        const int64_t c[3] = {ix[e], iy[e], iz[e]};
        for (int a = 0; a < 3; ++a)
            if (c[a] < 0 || c[a] >= (n0[a] << l)) return IDP_E_ARG;
        if (!tab.emplace(leaf_key(l, c[0], c[1], c[2]), (int)e).second) return IDP_E_ARG;
        lmax = l > lmax ? l : lmax;
    }
    // the leaves' volumes in finest cells add up to the box's (with the face
    // checks below, no gap and no overlap)
    unsigned __int128 vol = 0, box = (unsigned __int128)(n0[0] * n0[1] * n0[2]) << (3 * lmax);
    for (int64_t e = 0; e < K; ++e) vol += (unsigned __int128)1 << (3 * (lmax - level[e]));
    if (vol != box) return IDP_E_ARG;
    auto find = [&](int l, int64_t x, int64_t y, int64_t z) -> int {
        if (l < 0) return -1;
        auto it = tab.find(leaf_key(l, x, y, z));
        return it == tab.end() ? -1 : it->second;
    };
    const int NR = NP * NP, Q = 5 * NR;
    T.nbr.assign((size_t)K * 6, -1);
    T.lev.resize((size_t)K);
    std::vector<char> small((size_t)K * 6, 0);
    for (int64_t e = 0; e < K; ++e) {
        const int l = level[e];
        T.lev[e] = (signed char)l;
        for (int s = 0; s < 6; ++s) {
            const int d = s / 2, side = s & 1, a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            int64_t q[3] = {ix[e], iy[e], iz[e]};
            const int64_t nl = n0[d] << l;
            q[d] += side ? 1 : -1;
            if (q[d] < 0 || q[d] >= nl) {
                if (gd->bc[s] != IDP_BC_PERIODIC) { T.nbr[6 * e + s] = -1; continue; }
                q[d] = (q[d] + nl) % nl;
            }
            const int f = find(l, q[0], q[1], q[2]);
            if (f >= 0) { T.nbr[6 * e + s] = f; continue; }
            if (find(l - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1) >= 0) { small[6 * e + s] = 1; continue; }
            // four finer leaves across the face: a mortar with e as its large leaf
            int sm[4];
            for (int p = 0; p < 4; ++p) {
                int64_t r[3];
                r[d] = 2 * q[d] + (side ? 0 : 1);
                r[a1] = 2 * q[a1] + (p & 1);
                r[a2] = 2 * q[a2] + (p >> 1);
                sm[p] = find(l + 1, r[0], r[1], r[2]);
                if (sm[p] < 0) return IDP_E_ARG;
            }
            const int m = T.M++;
            T.info.insert(T.info.end(), {d, (int)e, side, sm[0], sm[1], sm[2], sm[3]});
            T.nbr[6 * e + s] = -2 - m * Q;
        }
    }
    // the small sides
    for (int m = 0; m < T.M; ++m) {
        const int *inf = &T.info[7 * m];
        const int sS = 2 * inf[0] + (inf[2] ? 0 : 1);
        for (int p = 0; p < 4; ++p) {
            const int e = inf[3 + p];
            if (!small[6 * e + sS]) return IDP_E_ARG;
            small[6 * e + sS] = 2;
            T.nbr[6 * e + sS] = -2 - (m * Q + (1 + p) * NR);
        }
    }
    for (size_t k = 0; k < small.size(); ++k)
        if (small[k] == 1) return IDP_E_ARG;
    // slots and mortar nodes (first appearance in slot order)
    const int NN = NR * NP, N = NP - 1;
    std::unordered_map<int, int> mn_of;
    T.slot_mn.resize((size_t)T.M * Q);
    std::vector<int> slots;   // [MN][3]
    for (int m = 0; m < T.M; ++m) {
        const int *inf = &T.info[7 * m];
        const int d = inf[0], low = inf[2];
        for (int q = 0; q < Q; ++q) {
            const int f = q / NR, t = q - f * NR;
            const int e = f == 0 ? inf[1] : inf[3 + f - 1];
            const int pos = (f == 0) == (low != 0) ? N : 0;
            const int g = e * NN + node_of_host(NP, d, t, pos);
            auto it = mn_of.find(g);
            int mn;
            if (it == mn_of.end()) {
                mn = T.MN++;
                mn_of.emplace(g, mn);
                T.mn_node.push_back(g);
                T.mn_cnt.push_back(0);
                slots.insert(slots.end(), {-1, -1, -1});
            } else {
                mn = it->second;
            }
            if (T.mn_cnt[mn] >= 3) return IDP_E_ARG;   // not reached on a 2:1 octree
            slots[3 * mn + T.mn_cnt[mn]++] = m * Q + q;
            T.slot_mn[(size_t)m * Q + q] = mn;
        }
    }
    T.mn_slot.resize((size_t)3 * T.MN);
    for (int mn = 0; mn < T.MN; ++mn)
        for (int c = 0; c < 3; ++c) T.mn_slot[(size_t)c * T.MN + mn] = slots[3 * mn + c];
    return IDP_OK;
}

// the mortar operators of degree N and their 1D pair lists; false if the
// overlap pattern exceeds the kernels' fixed sizes
bool build_mops3(int N, MOps3 &mo) {
    const int np = N + 1;
    double I[2 * NPMAX3 * NPMAX3], P[NPMAX3 * 2 * NPMAX3], wt[NPMAX3 * 2 * NPMAX3], x[NPMAX3], S[NPMAX3 * NPMAX3];
    std::memset(&mo, 0, sizeof(mo));
    idp::host_lgl_mortar(N, I, P, wt);
    idp::host_lgl_sbar(N, x, mo.w, S);
    for (int r = 0; r < 2 * np; ++r)
        for (int k = 0; k < np; ++k) mo.I[r][k] = I[r * np + k];
    for (int k = 0; k < np; ++k)
        for (int r = 0; r < 2 * np; ++r) { mo.P[k][r] = P[k * 2 * np + r]; mo.wt[k][r] = wt[k * 2 * np + r]; }
    mo.n1 = 0;
    for (int k = 0; k < np; ++k)
        for (int r = 0; r < 2 * np; ++r)
            if (mo.wt[k][r] != 0.0) {
                if (mo.n1 >= 3 * np - 1 || mo.sn[k] >= 2 * np || mo.sn[np + r] >= 2 * np) return false;
                const int p = mo.n1++;
                mo.pk[p] = k; mo.pr[p] = r;
                mo.sp[k][mo.sn[k]++] = p;
                mo.sp[np + r][mo.sn[np + r]++] = p;
            }
    return true;
}

idp_status create3(const idp3d_grid_desc *gd, int64_t K, const int8_t *level, const int32_t *ix, const int32_t *iy,
                   const int32_t *iz, int32_t N, double gamma, const idp3d_options *opts, idp3d_ctx **out) {
    if (N < 1 || N > 4 || !(gamma > 1.0)) return IDP_E_ARG;
    if (!(gd->x1 > gd->x0) || !(gd->y1 > gd->y0) || !(gd->z1 > gd->z0)) return IDP_E_ARG;
    for (int s = 0; s < 6; ++s)
        if (gd->bc[s] < IDP_BC_PERIODIC || gd->bc[s] > IDP_BC_OUTFLOW) return IDP_E_ARG;
    for (int d = 0; d < 3; ++d)
        if ((gd->bc[2 * d] == IDP_BC_PERIODIC) != (gd->bc[2 * d + 1] == IDP_BC_PERIODIC)) return IDP_E_ARG;
    idp3d_options o;
    idp3d_options_default(&o);
    if (opts) o = *opts;
    if (o.limiting < 0 || o.limiting > 3 || !(o.beta >= 0.0 && o.beta < 1.0) || !(o.cfl > 0.0)) return IDP_E_ARG;
    if (o.precision < 0 || o.precision > 1) return IDP_E_ARG;
    Octree3 T;
    idp_status rs = build_octree3(gd, K, level, ix, iy, iz, N + 1, T);
    if (rs != IDP_OK) return rs;
    MOps3 mops;
    if (!build_mops3(N, mops)) return IDP_E_ARG;
    idp3d_ctx *c = new (std::nothrow) idp3d_ctx();
    if (!c) return IDP_E_ARG;
    c->N = N; c->NP = N + 1; c->gamma = gamma; c->opt = o;
    Grid3 &G = c->grid;
    G.nx = gd->nx; G.ny = gd->ny; G.nz = gd->nz; G.K = (int)K;
    G.dx = (gd->x1 - gd->x0) / gd->nx; G.dy = (gd->y1 - gd->y0) / gd->ny; G.dz = (gd->z1 - gd->z0) / gd->nz;
    for (int s = 0; s < 6; ++s) {
        G.bc[s] = gd->bc[s];
        p2c(gamma, gd->bc_prim[s], G.bc_cons[s]);
    }
    c->volume = (gd->x1 - gd->x0) * (gd->y1 - gd->y0) * (gd->z1 - gd->z0);
    c->L = get3(c->NP);
    c->grid_el = (G.K + c->L.epb - 1) / c->L.epb;
    c->grid_el64 = (G.K + c->L.epb64 - 1) / c->L.epb64;
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
    auto upload = [&](auto **dst, const auto *src, size_t n) {
        if (!ok) return;
        chk(cudaMalloc((void **)dst, sizeof(*src) * n));
        if (ok) chk(cudaMemcpy(*dst, src, sizeof(*src) * n, cudaMemcpyHostToDevice));
    };
    const size_t kn = nodes_of(c);
    chk(c->L.prepare());
    upload(&c->d_ops, &ops, 1);
    {
        idp::LogTab lt;
        idp::host_log_table(lt);
        upload(&c->d_lg, &lt, 1);
    }
    G.lg = c->d_lg;
    {
        std::vector<double> ind((size_t)(N + 1) * (N + 1) + 2);
        idp::host_lgl_indicator(N, ind.data(), &ind[(size_t)(N + 1) * (N + 1)], &ind[(size_t)(N + 1) * (N + 1) + 1]);
        upload(&c->d_ind, ind.data(), ind.size());
    }
    G.ind = c->d_ind;
    if (ok) chk(cudaMalloc(&c->d_aind, sizeof(double) * (size_t)K));
    if (ok) chk(cudaMemset(c->d_aind, 0, sizeof(double) * (size_t)K));
    upload(&c->d_nbr, T.nbr.data(), T.nbr.size());
    upload(&c->d_lev, T.lev.data(), T.lev.size());
    G.nbr = c->d_nbr;
    G.lev = c->d_lev;
    Mort3 &MO = G.mort;
    std::memset(&MO, 0, sizeof(MO));
    if (T.M > 0 && ok) {
        const size_t S = (size_t)T.M * 5 * c->NP * c->NP, MN = (size_t)T.MN;
        MO.M = T.M; MO.S = (int)S; MO.MN = T.MN;
        upload(&c->d_mops, &mops, 1);
        upload(&c->d_minfo, T.info.data(), T.info.size());
        upload(&c->d_slot_mn, T.slot_mn.data(), T.slot_mn.size());
        upload(&c->d_mn_node, T.mn_node.data(), T.mn_node.size());
        upload(&c->d_mn_slot, T.mn_slot.data(), T.mn_slot.size());
        upload(&c->d_mn_cnt, T.mn_cnt.data(), T.mn_cnt.size());
        if (ok) chk(cudaMalloc(&c->d_mslot, sizeof(double) * 13 * S));
        if (ok) chk(cudaMalloc(&c->d_hand, sizeof(double) * 15 * MN));
        if (ok) chk(cudaMalloc(&c->d_ell, sizeof(double) * (size_t)T.M));
        if (ok) chk(cudaMalloc(&c->d_mbad, sizeof(int) * (size_t)T.M));
        if (ok) {
            MO.info = c->d_minfo;
            MO.chi = c->d_mslot; MO.clo = c->d_mslot + 5 * S;
            MO.rbmin = c->d_mslot + 10 * S; MO.rbmax = c->d_mslot + 11 * S; MO.dsum = c->d_mslot + 12 * S;
            MO.bad = c->d_mbad; MO.ell = c->d_ell;
            MO.slot_mn = c->d_slot_mn; MO.mn_node = c->d_mn_node; MO.mn_slot = c->d_mn_slot; MO.mn_cnt = c->d_mn_cnt;
            MO.h_uvol = c->d_hand; MO.h_res = c->d_hand + 5 * MN; MO.h_b = c->d_hand + 10 * MN;
        }
    }
    if (ok) chk(cudaMalloc(&c->d_buf1, sizeof(double) * NV * kn));
    if (ok) chk(cudaMalloc(&c->d_buf2, sizeof(double) * NV * kn));
    if (ok && o.precision == 0) chk(cudaMalloc(&c->d_emin, sizeof(unsigned) * (size_t)G.K));
    if (ok) chk(cudaMalloc(&c->d_part, sizeof(double) * NV * (size_t)G.K));
    if (ok) chk(cudaMalloc(&c->d_tot, sizeof(double) * NV));
    // each: the minimum, then the FP32 pass's minimum of the two-pass time step
    if (ok) chk(cudaMalloc(&c->d_dtmin, 2 * sizeof(unsigned long long)));
    if (ok) chk(cudaMalloc(&c->d_dtmin2, 2 * sizeof(unsigned long long)));
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

}  // namespace

extern "C" {

idp_status idp3d_options_default(idp3d_options *o) {
    if (!o) return IDP_E_ARG;
    o->limiting = 2;
    o->beta = 0.1;
    o->cfl = 0.5;
    o->precision = 0;
    return IDP_OK;
}

idp_status idp3d_create(const idp3d_grid_desc *gd, int32_t N, double gamma, const idp3d_options *opts,
                        idp3d_ctx **out) {
    if (!out) return IDP_E_ARG;
    *out = nullptr;
    if (!gd || gd->nx < 1 || gd->ny < 1 || gd->nz < 1) return IDP_E_ARG;
    const long long K = (long long)gd->nx * gd->ny * gd->nz;
    if (K > (1LL << 24)) return IDP_E_ARG;
    // the grid as level-0 leaves, e = (ez ny + ey) nx + ex
    std::vector<int8_t> lev((size_t)K, 0);
    std::vector<int32_t> ix((size_t)K), iy((size_t)K), iz((size_t)K);
    for (long long e = 0; e < K; ++e) {
        ix[e] = (int32_t)(e % gd->nx);
        iy[e] = (int32_t)((e / gd->nx) % gd->ny);
        iz[e] = (int32_t)(e / ((long long)gd->nx * gd->ny));
    }
    return create3(gd, K, lev.data(), ix.data(), iy.data(), iz.data(), N, gamma, opts, out);
}

idp_status idp3d_create_octree(const idp3d_grid_desc *base, int64_t n_leaves, const int8_t *level, const int32_t *ix,
                               const int32_t *iy, const int32_t *iz, int32_t N, double gamma,
                               const idp3d_options *opts, idp3d_ctx **out) {
    if (!out) return IDP_E_ARG;
    *out = nullptr;
    if (!base || !level || !ix || !iy || !iz || n_leaves < 1 || n_leaves > (1LL << 24)) return IDP_E_ARG;
    return create3(base, n_leaves, level, ix, iy, iz, N, gamma, opts, out);
}

idp_status idp3d_layout(const idp3d_ctx *c, int64_t *n_elems, int32_t *nodes_per_elem) {
    if (!c) return IDP_E_ARG;
    if (n_elems) *n_elems = c->grid.K;
    if (nodes_per_elem) *nodes_per_elem = c->NP * c->NP * c->NP;
    return IDP_OK;
}

idp_status idp3d_octree_tables(const idp3d_grid_desc *base, int64_t n_leaves, const int8_t *level, const int32_t *ix,
                               const int32_t *iy, const int32_t *iz, int32_t N, int64_t *n_mortars,
                               int64_t *n_mortar_nodes, int32_t *mortar_info, int32_t *nbr) {
    if (!base || !level || !ix || !iy || !iz || n_leaves < 1 || n_leaves > (1LL << 24) || N < 1 || N > 4)
        return IDP_E_ARG;
    if (base->nx < 1 || base->ny < 1 || base->nz < 1) return IDP_E_ARG;
    for (int d = 0; d < 3; ++d)
        if ((base->bc[2 * d] == IDP_BC_PERIODIC) != (base->bc[2 * d + 1] == IDP_BC_PERIODIC)) return IDP_E_ARG;
    Octree3 T;
    const idp_status rs = build_octree3(base, n_leaves, level, ix, iy, iz, N + 1, T);
    if (rs != IDP_OK) return rs;
    if (n_mortars) *n_mortars = T.M;
    if (n_mortar_nodes) *n_mortar_nodes = T.MN;
    if (mortar_info) std::memcpy(mortar_info, T.info.data(), sizeof(int32_t) * T.info.size());
    if (nbr) std::memcpy(nbr, T.nbr.data(), sizeof(int32_t) * T.nbr.size());
    return IDP_OK;
}

idp_status idp3d_stage_factors(idp3d_ctx *c, double *alpha_host, double *mortar_ell_host, void *stream) {
    if (!c) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) return IDP_E_CUDA;
    if (alpha_host && cudaMemcpy(alpha_host, c->d_aind, sizeof(double) * (size_t)c->grid.K, cudaMemcpyDeviceToHost) != cudaSuccess)
        return IDP_E_CUDA;
    if (mortar_ell_host && c->grid.mort.M > 0 &&
        cudaMemcpy(mortar_ell_host, c->d_ell, sizeof(double) * (size_t)c->grid.mort.M, cudaMemcpyDeviceToHost) != cudaSuccess)
        return IDP_E_CUDA;
    return IDP_OK;
}

idp_status idp3d_mesh_info(const idp3d_ctx *c, int64_t *n_mortars, int64_t *n_mortar_nodes) {
    if (!c) return IDP_E_ARG;
    if (n_mortars) *n_mortars = c->grid.mort.M;
    if (n_mortar_nodes) *n_mortar_nodes = c->grid.mort.MN;
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
    enqueue_stage(c, st, A, true);
    return cuda_ok(cudaGetLastError());
}

idp_status idp3d_dt(idp3d_ctx *c, const double *u, double *dt_host, void *stream) {
    if (!c || !u || !dt_host) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long b = kInfBits;
    if (cudaMemcpyAsync(c->d_dtmin2, &kInfBits, sizeof(kInfBits), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return IDP_E_CUDA;
    if (has_mortars(c)) c->L.mflux(st, c->grid, c->d_mops, u, c->gamma);
    launch_dt(c, st, u, c->d_dtmin2);
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
    out->alpha_mortar = a.mort_area > 0.0 ? a.alpha_mort_a / a.mort_area : 0.0;
    out->n_mortar_active = (int64_t)a.n_mort;
    out->n_mortar_fallback = (int64_t)a.n_mort_fallback;
    c->n_stages = 0;
    if (reset_stats3(c, c->stream) != cudaSuccess) return IDP_E_CUDA;
    return read_status3(c);
}

void idp3d_destroy(idp3d_ctx *c) {
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    void *ptrs[] = {c->d_ops, c->d_buf1, c->d_buf2, c->d_part, c->d_tot, c->d_dtmin, c->d_dtmin2, c->d_t,
                    c->d_dtlast, c->d_status, c->d_stats, c->d_mops, c->d_nbr, c->d_lev, c->d_minfo,
                    c->d_slot_mn, c->d_mn_node, c->d_mn_slot, c->d_mn_cnt, c->d_mbad, c->d_mslot, c->d_hand,
                    c->d_ell, c->d_lg, c->d_emin, c->d_ind, c->d_aind};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
