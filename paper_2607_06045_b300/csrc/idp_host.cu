// idp_host.cu -- host runtime of the IDP LGL-DGSEM library: reference
// operators, quadtree mesh builder and validation, device tables, stage
// sequencing with CUDA graphs, the elements-per-block autotuner and the C ABI
// declared in include/idp_dgsem.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/idp_dgsem.h"
#include "idp_remesh.h"
#include "idp_launch.cuh"

using namespace idp;

// ---------------------------------------------------------------------------
// reference operators (Sec. 2.1, App. A)
// ---------------------------------------------------------------------------
namespace {

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
void legendre_pair(int n, double x, double &pn, double &pnm1) {
    double a = 1.0, b = x;
    if (n == 0) { pn = 1.0; pnm1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
        a = b;
        b = c;
    }
    pn = b;
    pnm1 = a;
}

// LGL nodes: the roots of q = P_{N+1} - P_{N-1}, which vanishes at +-1 and at
// the roots of P_N' (since (2N+1)(x^2-1) P_N' = N(N+1)(P_{N+1} - P_{N-1})),
// found by Newton with q' = (2N+1) P_N; weights 2 / (N (N+1) P_N^2).
void lgl_nodes(int N, double *x, double *w) {
    x[0] = -1.0;
    x[N] = 1.0;
    for (int k = 1; k < N; ++k) {
        double t = -std::cos(M_PI * k / N);
        for (int it = 0; it < 200; ++it) {
            double pNp1, pN, pNm1, tmp;
            legendre_pair(N + 1, t, pNp1, pN);
            legendre_pair(N - 1, t, pNm1, tmp);
            double q = pNp1 - pNm1, dq = (2.0 * N + 1.0) * pN;
            double step = q / dq;
            t -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        x[k] = t;
    }
    for (int k = 0; k <= N; ++k) {
        double pN, pNm1;
        legendre_pair(N, x[k], pN, pNm1);
        w[k] = 2.0 / (N * (N + 1.0) * pN * pN);
    }
}

// Barycentric weights and Lagrange basis values at s.
void bary_weights(int np, const double *x, double *lam) {
    for (int j = 0; j < np; ++j) {
        double p = 1.0;
        for (int k = 0; k < np; ++k)
            if (k != j) p *= (x[j] - x[k]);
        lam[j] = 1.0 / p;
    }
}

void bary_basis(int np, const double *x, const double *lam, double s, double *phi) {
    for (int j = 0; j < np; ++j)
        if (s == x[j]) {
            for (int k = 0; k < np; ++k) phi[k] = k == j ? 1.0 : 0.0;
            return;
        }
    double den = 0.0;
    for (int j = 0; j < np; ++j) den += lam[j] / (s - x[j]);
    for (int j = 0; j < np; ++j) phi[j] = lam[j] / (s - x[j]) / den;
}

// Gauss-Jordan inverse of a small dense matrix (row-major), in place.
bool invert(int n, double *A) {
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0) return false;
        for (int k = 0; k < n; ++k) { std::swap(A[c * n + k], A[p * n + k]); std::swap(I[c * n + k], I[p * n + k]); }
        double d = A[c * n + c];
        for (int k = 0; k < n; ++k) { A[c * n + k] /= d; I[c * n + k] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = A[r * n + c];
            for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
        }
    }
    std::memcpy(A, I.data(), sizeof(double) * n * n);
    return true;
}

// Table of the FP64 logarithm (Tang's method): 1 / F_j and ln F_j as head +
// tail for F_j = 1 + j/128, and ln 2 with a 42-bit head; formed in long double.
void host_log_table_impl(LogTab &T) {
    for (int j = 0; j < kLogTab; ++j) {
        const long double F = 1.0L + (long double)j / kLogTab;
        T.inv[j] = (double)(1.0L / F);
        const long double l = logl(F);
        T.hi[j] = (double)l;
        T.lo[j] = (double)(l - (long double)T.hi[j]);
    }
    const long double ln2 = logl(2.0L);
    double h = (double)ln2;
    uint64_t b;
    std::memcpy(&b, &h, sizeof(b));
    b &= ~((uint64_t(1) << 11) - 1);   // keep 42 significant bits
    std::memcpy(&h, &b, sizeof(b));
    T.ln2_hi = h;
    T.ln2_lo = (double)(ln2 - (long double)h);
}

void build_ops(int N, int proj, int a2a, Ops &o) {
    std::memset(&o, 0, sizeof(o));
    host_log_table_impl(o.lg);
    const int np = N + 1;
    double x[NPMAX], w[NPMAX], lam[NPMAX];
    lgl_nodes(N, x, w);
    bary_weights(np, x, lam);
    for (int i = 0; i < np; ++i) { o.xi[i] = x[i]; o.w[i] = w[i]; o.iw[i] = 1.0 / w[i]; }
    // D_ij = phi_j'(x_i) in barycentric form; Sbar = 2 diag(w) D - B
    for (int i = 0; i < np; ++i) {
        double diag = 0.0;
        double D[NPMAX];
        for (int j = 0; j < np; ++j) {
            if (j == i) continue;
            D[j] = (lam[j] / lam[i]) / (x[i] - x[j]);
            diag -= D[j];
        }
        D[i] = diag;
        for (int j = 0; j < np; ++j) {
            double B = (i == j) ? (i == 0 ? -1.0 : (i == N ? 1.0 : 0.0)) : 0.0;
            o.S[i][j] = 2.0 * w[i] * D[j] - B;
        }
    }
    // local mortar weights: overlap of LGL subcells (App. A); subcells that
    // touch only at a point do not overlap
    double bl[NPMAX + 1], bs[2 * NPMAX + 1];
    bl[0] = -1.0;
    for (int k = 0; k < np; ++k) bl[k + 1] = bl[k] + w[k];
    bs[0] = -1.0;
    for (int e = 0; e < 2; ++e)
        for (int l = 0; l < np; ++l) bs[e * np + l + 1] = (l == 0 ? (e == 0 ? -1.0 : 0.0) : bs[e * np + l]) + 0.5 * w[l];
    for (int k = 0; k < np; ++k)
        for (int e = 0; e < 2; ++e)
            for (int l = 0; l < np; ++l) {
                double lo0 = l == 0 ? (e == 0 ? -1.0 : 0.0) : bs[e * np + l];
                double hi0 = bs[e * np + l + 1];
                double lo = std::max(bl[k], lo0), hi = std::min(bl[k + 1], hi0);
                o.wt[k][e * np + l] = (hi - lo > 1e-12) ? hi - lo : 0.0;
            }
    {
        std::vector<double> V(np * np);
        for (int i = 0; i < np; ++i)
            for (int k = 0; k < np; ++k) {
                double pk, pkm1;
                legendre_pair(k, x[i], pk, pkm1);
                V[i * np + k] = std::sqrt((2.0 * k + 1.0) / 2.0) * pk;
            }
        invert(np, V.data());
        for (int k = 0; k < np; ++k)
            for (int i = 0; i < np; ++i) o.Vinv[k][i] = V[k * np + i];
    }
    o.ind_T = 0.5 * std::pow(10.0, -1.8 * std::pow(N + 1.0, 0.25));
    o.ind_s = std::log((1.0 - 1e-4) / 1e-4);
    // interpolation to the small-face nodes s = (x_l -/+ 1) / 2
    for (int e = 0; e < 2; ++e)
        for (int l = 0; l < np; ++l) {
            double phi[NPMAX];
            bary_basis(np, x, lam, 0.5 * (x[l] + (e == 0 ? -1.0 : 1.0)), phi);
            for (int k = 0; k < np; ++k) o.I[e * np + l][k] = phi[k];
        }
    if (a2a) {
        // all-to-all weights (Eq. nonlocal_weight) by the small face's LGL
        // quadrature: w_l / 2 * phi_k(x_(e,l)) in units of the large face's
        // half length; rounding-level values where nodes meet are zero
        for (int k = 0; k < np; ++k)
            for (int r = 0; r < 2 * np; ++r) {
                const double v = 0.5 * w[r % np] * o.I[r][k];
                o.wt[k][r] = std::fabs(v) < 1e-13 ? 0.0 : v;
            }
    }
    // nonzero weights as pairs (the all-to-all weights can be negative)
    o.npair = 0;
    for (int k = 0; k < np; ++k)
        for (int r = 0; r < 2 * np; ++r)
            if (o.wt[k][r] != 0.0) {
                const int p = o.npair++;
                o.pk[p] = k; o.pr[p] = r;
                o.slot_p[k][o.slot_n[k]++] = p;
                o.slot_p[np + r][o.slot_n[np + r]++] = p;
            }
    if (proj == 0) {
        for (int k = 0; k < np; ++k)
            for (int c = 0; c < 2 * np; ++c) o.P[k][c] = 0.5 * w[c % np] * o.I[c][k] / w[k];
    } else {
        // exact L2 projection: M = (V V^T)^{-1} with V the orthonormal
        // Legendre-Vandermonde matrix; P = M^{-1} B with
        // B_{k,(e,l)} = int_half phi_k psi_l = 1/2 sum_m I_e[m][k] M[m][l]
        std::vector<double> V(np * np), Minv(np * np, 0.0), M(np * np);
        for (int i = 0; i < np; ++i)
            for (int n = 0; n < np; ++n) {
                double pn, pm;
                legendre_pair(n, x[i], pn, pm);
                V[i * np + n] = std::sqrt((2.0 * n + 1.0) / 2.0) * pn;
            }
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                double s = 0.0;
                for (int n = 0; n < np; ++n) s += V[i * np + n] * V[j * np + n];
                Minv[i * np + j] = s;
            }
        M = Minv;
        invert(np, M.data());
        for (int k = 0; k < np; ++k)
            for (int e = 0; e < 2; ++e)
                for (int l = 0; l < np; ++l) {
                    double acc = 0.0;
                    for (int j = 0; j < np; ++j) {
                        double Bjl = 0.0;
                        for (int m = 0; m < np; ++m) Bjl += 0.5 * o.I[e * np + m][j] * M[m * np + l];
                        acc += Minv[k * np + j] * Bjl;
                    }
                    o.P[k][e * np + l] = acc;
                }
    }
}

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------

struct HostMesh {
    std::vector<Geo> geom;
    std::vector<int32_t> sim;
    std::vector<int4> fnbr;
    std::vector<uchar4> ftype;
    std::vector<int32_t> m_large, m_info;
    std::vector<int2> m_small;
    std::vector<SimInfo> siminfo;
    std::vector<long long> sim_off;
};

inline uint64_t leaf_key(int l, int64_t x, int64_t y) { return ((uint64_t)l << 58) | ((uint64_t)x << 29) | (uint64_t)y; }

void prim_to_cons(double g, const double *p, double *q) {
    q[0] = p[0];
    q[1] = p[0] * p[1];
    q[2] = p[0] * p[2];
    q[3] = p[3] / (g - 1.0) + 0.5 * p[0] * (p[1] * p[1] + p[2] * p[2]);
}

idp_status build_mesh(const idp_mesh_desc &d, double gamma, int simid, HostMesh &H) {
    if (d.nx0 < 1 || d.ny0 < 1 || d.n_leaves < 1 || !d.level || !d.ix || !d.iy) return IDP_E_ARG;
    if (!(d.x1 > d.x0) || !(d.y1 > d.y0)) return IDP_E_ARG;
    for (int s = 0; s < 4; ++s)
        if (d.bc[s] < IDP_BC_PERIODIC || d.bc[s] > IDP_BC_JET) return IDP_E_ARG;
    if ((d.bc[0] == IDP_BC_PERIODIC) != (d.bc[1] == IDP_BC_PERIODIC)) return IDP_E_ARG;
    if ((d.bc[2] == IDP_BC_PERIODIC) != (d.bc[3] == IDP_BC_PERIODIC)) return IDP_E_ARG;
    const int K = d.n_leaves, base = (int)H.geom.size(), mbase = (int)H.m_large.size();
    int Lmax = 0;
    for (int e = 0; e < K; ++e) {
        int l = d.level[e];
        if (l < 0 || l > 24) return IDP_E_MESH;
        Lmax = std::max(Lmax, l);
    }
    if (((int64_t)d.nx0 << Lmax) >= (1LL << 28) || ((int64_t)d.ny0 << Lmax) >= (1LL << 28)) return IDP_E_ARG;
    std::unordered_map<uint64_t, int> tab;
    tab.reserve((size_t)K * 2);
    unsigned __int128 area = 0;
    for (int e = 0; e < K; ++e) {
        int l = d.level[e];
        int64_t nx = (int64_t)d.nx0 << l, ny = (int64_t)d.ny0 << l;
        if (d.ix[e] < 0 || d.iy[e] < 0 || d.ix[e] >= nx || d.iy[e] >= ny) return IDP_E_MESH;
        if (!tab.emplace(leaf_key(l, d.ix[e], d.iy[e]), e).second) return IDP_E_MESH;   // duplicate
        area += (unsigned __int128)1 << (2 * (Lmax - l));
    }
    if (area != ((unsigned __int128)d.nx0 * d.ny0) << (2 * Lmax)) return IDP_E_MESH;   // gap or overlap
    for (int e = 0; e < K; ++e) {   // no leaf may contain another
        int64_t x = d.ix[e], y = d.iy[e];
        for (int l = d.level[e] - 1; l >= 0; --l) {
            x >>= 1; y >>= 1;
            if (tab.count(leaf_key(l, x, y))) return IDP_E_MESH;
        }
    }
    auto find = [&](int l, int64_t x, int64_t y) {
        auto it = tab.find(leaf_key(l, x, y));
        return it == tab.end() ? -1 : it->second;
    };
    for (int e = 0; e < K; ++e) {
        int l = d.level[e];
        double dx = (d.x1 - d.x0) / ((double)d.nx0 * (double)(1LL << l));
        double dy = (d.y1 - d.y0) / ((double)d.ny0 * (double)(1LL << l));
        Geo g;
        g.x = d.x0 + d.ix[e] * dx; g.y = d.y0 + d.iy[e] * dy; g.z = dx; g.w = dy;
        H.geom.push_back(g);
        H.sim.push_back(simid);
        H.fnbr.push_back(make_int4(-1, -1, -1, -1));
        H.ftype.push_back(make_uchar4(FT_BND, FT_BND, FT_BND, FT_BND));
    }
    std::vector<char> pending((size_t)K * 4, 0);
    for (int e = 0; e < K; ++e) {
        int l = d.level[e];
        int64_t nxl = (int64_t)d.nx0 << l, nyl = (int64_t)d.ny0 << l;
        for (int s = 0; s < 4; ++s) {
            int64_t qx = d.ix[e] + (s == 0 ? -1 : (s == 1 ? 1 : 0));
            int64_t qy = d.iy[e] + (s == 2 ? -1 : (s == 3 ? 1 : 0));
            bool outside = qx < 0 || qx >= nxl || qy < 0 || qy >= nyl;
            int kind = FT_BND, nb = -1;
            if (!outside || d.bc[s] == IDP_BC_PERIODIC) {
                qx = (qx + nxl) % nxl;
                qy = (qy + nyl) % nyl;
                int f = find(l, qx, qy);
                if (f >= 0) { kind = FT_CONF; nb = base + f; }
                else if (l > 0 && find(l - 1, qx >> 1, qy >> 1) >= 0) { pending[(size_t)e * 4 + s] = 1; continue; }
                else {
                    int64_t ax, ay, bx, by;
                    if (s < 2) { ax = bx = 2 * qx + (s == 0 ? 1 : 0); ay = 2 * qy; by = 2 * qy + 1; }
                    else { ay = by = 2 * qy + (s == 2 ? 1 : 0); ax = 2 * qx; bx = 2 * qx + 1; }
                    int a = find(l + 1, ax, ay), b = find(l + 1, bx, by);
                    if (a < 0 || b < 0) return IDP_E_MESH;   // not 2:1 balanced
                    int m = (int)H.m_large.size();
                    int low = (s == 1 || s == 3) ? 1 : 0;
                    H.m_large.push_back(base + e);
                    H.m_small.push_back(make_int2(base + a, base + b));
                    H.m_info.push_back((s >> 1) | (low << 1));
                    kind = FT_MLARGE;
                    nb = m;
                }
            }
            int4 &n4 = H.fnbr[base + e];
            uchar4 &t4 = H.ftype[base + e];
            (s == 0 ? n4.x : s == 1 ? n4.y : s == 2 ? n4.z : n4.w) = nb;
            (s == 0 ? t4.x : s == 1 ? t4.y : s == 2 ? t4.z : t4.w) = (unsigned char)kind;
        }
    }
    for (int m = mbase; m < (int)H.m_large.size(); ++m) {
        int dir = H.m_info[m] & 1, low = (H.m_info[m] >> 1) & 1;
        int s_small = dir == 0 ? (low ? 0 : 1) : (low ? 2 : 3);
        for (int p = 0; p < 2; ++p) {
            int es = p == 0 ? H.m_small[m].x : H.m_small[m].y;
            if (!pending[(size_t)(es - base) * 4 + s_small]) return IDP_E_MESH;
            pending[(size_t)(es - base) * 4 + s_small] = 0;
            int4 &n4 = H.fnbr[es];
            uchar4 &t4 = H.ftype[es];
            (s_small == 0 ? n4.x : s_small == 1 ? n4.y : s_small == 2 ? n4.z : n4.w) = m;
            (s_small == 0 ? t4.x : s_small == 1 ? t4.y : s_small == 2 ? t4.z : t4.w) =
                (unsigned char)(p == 0 ? FT_MSLO : FT_MSHI);
        }
    }
    for (size_t k = 0; k < pending.size(); ++k)
        if (pending[k]) return IDP_E_MESH;
    SimInfo si;
    std::memset(&si, 0, sizeof(si));
    for (int s = 0; s < 4; ++s) {
        si.bc[s] = d.bc[s];
        prim_to_cons(gamma, d.bc_prim[s], si.bc_cons[s]);
    }
    prim_to_cons(gamma, d.dmr_post, si.dmr_post);
    prim_to_cons(gamma, d.dmr_pre, si.dmr_pre);
    si.y1 = d.y1;
    H.siminfo.push_back(si);
    return IDP_OK;
}

template <typename T>
cudaError_t upload(T **dptr, const std::vector<T> &h) {
    *dptr = nullptr;
    if (h.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)dptr, sizeof(T) * h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dptr, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

Launchers get_launchers(int np) {
    switch (np) {
    case 2: return launchers_np2();
    case 3: return launchers_np3();
    case 4: return launchers_np4();
    case 5: return launchers_np5();
    case 6: return launchers_np6();
    case 7: return launchers_np7();
    default: return launchers_np8();
    }
}

std::mutex g_tune_mu;
thread_local char g_last_error[256] = "";

// Record the first failing CUDA call of an entry point (diagnostics only).
cudaError_t note(cudaError_t e, const char *what) {
    if (e != cudaSuccess) std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    return e;
}
std::map<long long, std::pair<int, int>> g_tune_cache;   // key -> (epb, persistent)

}  // namespace

namespace idp {
// table of the FP64 logarithm (used by the probes and the test hook)
// Global node of slot q of mortar m (large face first, then the lower and
// upper small faces).
static long long mortar_slot_node(int NP, int m, int q, const std::vector<int32_t> &m_large,
                                  const std::vector<int2> &m_small, const std::vector<int32_t> &m_info) {
    const int NN = NP * NP, dir = m_info[m] & 1, low = (m_info[m] >> 1) & 1;
    const int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2), sS = sL ^ 1;
    int e, s, t;
    if (q < NP) { e = m_large[m]; s = sL; t = q; }
    else { e = ((q - NP) / NP == 0) ? m_small[m].x : m_small[m].y; s = sS; t = (q - NP) % NP; }
    const int i = s == 0 ? 0 : (s == 1 ? NP - 1 : t), j = s == 2 ? 0 : (s == 3 ? NP - 1 : t);
    return (long long)e * NN + j * NP + i;
}

// The unique mortar nodes with their (first, second or -1) slot, and the
// blocks of the mortar limiting kernel: block b owns mortars [b W, b W + W)
// and the nodes whose first slot is one of theirs, listed in slot order; a
// node's second mortar in a later block is one of the block's foreign
// mortars (sorted, unique), whose factor the block forms too. A node on more
// than two mortars is an invalid mesh.
idp_status host_mortar_tables(int NP, int W, int K, int M, const std::vector<int32_t> &m_large,
                              const std::vector<int2> &m_small, const std::vector<int32_t> &m_info,
                              std::vector<int32_t> &mn_node, std::vector<int2> &mn_slot,
                              std::vector<int32_t> &mb_node_off, std::vector<int32_t> &mb_for_off,
                              std::vector<int32_t> &mb_foreign, int &fmax) {
    const int Q = 3 * NP;
    std::vector<int> first((size_t)K * NP * NP, -1), second((size_t)K * NP * NP, -1);
    for (int m = 0; m < M; ++m)
        for (int q = 0; q < Q; ++q) {
            const long long g = mortar_slot_node(NP, m, q, m_large, m_small, m_info);
            const int sl = m * Q + q;
            if (first[g] < 0) first[g] = sl;
            else if (second[g] < 0) second[g] = sl;
            else return IDP_E_MESH;
        }
    const int nb = M > 0 ? (M + W - 1) / W : 0;
    fmax = 0;
    mn_node.clear(); mn_slot.clear(); mb_foreign.clear();
    mb_node_off.assign(1, 0); mb_for_off.assign(1, 0);
    for (int b = 0; b < nb; ++b) {
        std::vector<int32_t> fore;
        for (int m = b * W; m < std::min(M, b * W + W); ++m)
            for (int q = 0; q < Q; ++q) {
                const int sl = m * Q + q;
                const long long g = mortar_slot_node(NP, m, q, m_large, m_small, m_info);
                if (first[g] != sl) continue;
                mn_node.push_back((int32_t)g);
                mn_slot.push_back(make_int2(sl, second[g]));
                if (second[g] >= 0 && (second[g] / Q) / W != b) fore.push_back(second[g] / Q);
            }
        mb_node_off.push_back((int32_t)mn_node.size());
        std::sort(fore.begin(), fore.end());
        fore.erase(std::unique(fore.begin(), fore.end()), fore.end());
        for (int32_t m : fore) mb_foreign.push_back(m);
        mb_for_off.push_back((int32_t)mb_foreign.size());
        fmax = std::max(fmax, (int)fore.size());
    }
    if (mb_foreign.empty()) mb_foreign.push_back(0);
    return IDP_OK;
}

void host_log_table(LogTab &T) { host_log_table_impl(T); }

// LGL quadrature weights for degree N (used by the allocation-free integrals)
void host_lgl_weights(int N, double *w) {
    double x[NPMAX];
    lgl_nodes(N, x, w);
}

// the 1D mortar operators of degree N (the 3D contexts take their tensor
// products): interpolation I[2(N+1)][N+1] to the two half-faces' nodes, the
// exact L2 projection P[N+1][2(N+1)] back and the local overlap weights
// wt[N+1][2(N+1)] (App. A), row-major, as the 2D contexts build them
void host_lgl_mortar(int N, double *I, double *P, double *wt) {
    Ops o;
    build_ops(N, 1, 0, o);
    const int np = N + 1;
    for (int r = 0; r < 2 * np; ++r)
        for (int k = 0; k < np; ++k) I[r * np + k] = o.I[r][k];
    for (int k = 0; k < np; ++k)
        for (int r = 0; r < 2 * np; ++r) { P[k * 2 * np + r] = o.P[k][r]; wt[k * 2 * np + r] = o.wt[k][r]; }
}

// the shock indicator's operators of degree N (the 3D contexts take their
// tensor products): the inverse of V_ik = sqrt((2k+1)/2) P_k(xi_i) (row-major,
// (N+1)^2), the threshold T and the sharpness s, as the 2D contexts build them
void host_lgl_indicator(int N, double *Vinv, double *T, double *s) {
    Ops o;
    build_ops(N, 1, 0, o);
    const int np = N + 1;
    for (int k = 0; k < np; ++k)
        for (int i = 0; i < np; ++i) Vinv[k * np + i] = o.Vinv[k][i];
    *T = o.ind_T;
    *s = o.ind_s;
}

// LGL nodes and weights and Sbar (row-major, (N+1)^2) for degree N (the 3D
// contexts), the operators the 2D contexts use
void host_lgl_sbar(int N, double *x, double *w, double *S) {
    Ops o;
    build_ops(N, 1, 0, o);
    const int np = N + 1;
    for (int i = 0; i < np; ++i) { x[i] = o.xi[i]; w[i] = o.w[i]; }
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) S[i * np + j] = o.S[i][j];
}
}  // namespace idp

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct idp_ctx {
    int N = 0, NP = 0, n_sims = 0;
    double gamma = 1.4;
    idp_options opt;
    int num_sms = 0;
    long long K = 0, M = 0;
    int n_mnodes = 0;
    std::vector<long long> sim_off;
    Launchers L;
    MeshDev mesh;
    SlotsDev slots;
    Ops *d_ops = nullptr;
    Geo *d_geom = nullptr;
    GeoC *d_geoc = nullptr;
    int32_t *d_sim = nullptr, *d_mlarge = nullptr, *d_minfo = nullptr, *d_mnnode = nullptr;
    int32_t *d_mbnode = nullptr, *d_mbfor = nullptr, *d_mbforeign = nullptr;
    int mb_fmax = 0, mb_blocks = 0;
    int4 *d_fnbr = nullptr;
    uchar4 *d_ftype = nullptr;
    int2 *d_msmall = nullptr, *d_mnslot = nullptr;
    SimInfo *d_siminfo = nullptr;
    void *d_slot_block = nullptr;
    double *d_buf1 = nullptr, *d_buf2 = nullptr, *d_hostbuf = nullptr;
    unsigned long long *d_dtmin = nullptr;
    double *d_tsim = nullptr, *d_dtlast = nullptr;
    unsigned *d_status = nullptr;
    StatsAcc *d_stats = nullptr;
    double *d_part = nullptr, *d_intout = nullptr;
    long long *d_off = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // a second stream for work that runs beside the main one (the mortar
    // fluxes beside the face or wave-speed kernel), forked and joined by events
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int epb = 0, persistent = 0, bps = 1;
    bool tuned = false;
    cudaGraphExec_t graph = nullptr;
    const double *graph_u = nullptr;
    bool graph_stale = false;   // the mesh changed since the capture
    long long n_stages = 0;
    double total_area = 0.0;   // sum of element areas (all simulations)
    double *d_aind = nullptr;  // per element: shock indicator of the stage (combined limiting)
    double total_mortar_len = 0.0;   // sum of the large faces' lengths over the mortars
    // statistics across adaptations: the normalisers of the stages on earlier
    // meshes since the last read, and the stage count when the mesh changed
    double stats_mass_prior = 0.0, stats_mlen_prior = 0.0;
    long long stats_stages_prior = 0;
    // local-limiting variants: extended element kernel, low-order bounds
    int ext = 0;               // entropy bound or low-order bounds in use
    int lob = 0;               // low-order bounds (pre-pass + mortar gather each stage)
    int ent_bar = 0;           // entropy bound with bar-state bounds (mortar bar-state entropies)
    double *d_lofv = nullptr;  // [2][K (N+1)^2] pre-pass output
    int facebuf = 0;           // FP64 default kernel: conforming faces from k_face
    double *d_fbuf = nullptr;  // k_face output: [6][2 K (N+1)] doubles + [2 K (N+1)] floats
    void *d_lam = nullptr;     // wave speeds of every node for the time step (no face buffer)
    unsigned *d_emin = nullptr;   // with the face buffer: per element, the FP32 pass's time-step minimum
    // adaptation on the device (single-mesh contexts): the leaves' level and
    // indices, the level-0 grid, the transfer's operators, the buffer sizes
    // in elements and mortars, and a scratch area that only grows
    int8_t *d_lev = nullptr;
    int32_t *d_ix = nullptr, *d_iy = nullptr;
    RemeshMesh rmesh = {};
    Ops *d_ops_amr = nullptr;
    long long capK = 0, capM = 0, cap_nodes = 0, cap_blocks = 0, cap_foreign = 0;
    void *d_rm = nullptr;
    size_t rm_bytes = 0;
    // optional timing: 1 step spans around the graph launches; 2 steps
    // launched without the graph, with element-pass events
    int prof = 0;
    cudaEvent_t pev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double prof_step_ms = 0.0;
    long long prof_steps = 0;
    // mode 2: events around every kernel launch of a step, by kind
    static constexpr int kMaxKev = 32;
    cudaEvent_t kev[kMaxKev][2] = {};
    int kev_kind[kMaxKev] = {};
    int kev_n = 0;
    double kms[IDP_NKERNELS] = {};
    long long kcnt[IDP_NKERNELS] = {};
};

namespace {

size_t KN(const idp_ctx *c) { return (size_t)c->K * c->NP * c->NP; }

int element_grid(const idp_ctx *c, int epb, int persistent, int bps) {
    long long blocks = (c->K + epb - 1) / epb;
    if (persistent) blocks = std::min<long long>(blocks, (long long)c->num_sms * std::max(bps, 1));
    return (int)std::max<long long>(blocks, 1);
}

StageArgs base_args(idp_ctx *c) {
    StageArgs A;
    std::memset(&A, 0, sizeof(A));
    A.limiting = c->opt.limiting;
    A.collect = c->opt.collect_stats;
    A.dtmin = c->d_dtmin;
    A.cfl = c->opt.cfl;
    A.t_sim = c->d_tsim;
    A.beta = c->opt.beta;
    A.gas = make_gas(c->gamma, &c->d_ops->lg);
    A.ops = c->d_ops;
    A.status = c->d_status;
    A.stats = c->d_stats;
    A.aind = c->d_aind;
    A.entropy = c->opt.entropy_bound;
    A.lob = c->lob;
    A.pass = 0;
    A.lofv = c->d_lofv;
    A.fbuf = c->d_fbuf;
    A.vflux = c->opt.volume_flux;
    return A;
}

// Profiling mode 2: CUDA events before and after a launch, by kernel kind
// (kt_begin returns the event slot, or -1 when not profiling).
int kt_begin(idp_ctx *c, cudaStream_t st, int kind) {
    if (c->prof != 2 || c->kev_n >= idp_ctx::kMaxKev) return -1;
    const int k = c->kev_n++;
    c->kev_kind[k] = kind;
    cudaEventRecord(c->kev[k][0], st);
    return k;
}
void kt_end(idp_ctx *c, cudaStream_t st, int k) {
    if (k >= 0) cudaEventRecord(c->kev[k][1], st);
}
// after the step's stream has synchronised
cudaError_t kt_collect(idp_ctx *c) {
    for (int k = 0; k < c->kev_n; ++k) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, c->kev[k][0], c->kev[k][1]);
        if (e != cudaSuccess) return e;
        c->kms[c->kev_kind[k]] += ms;
        c->kcnt[c->kev_kind[k]] += 1;
    }
    c->kev_n = 0;
    return cudaSuccess;
}

// one stage: mortar fluxes (unless already current), element pass, mortar
// limiting
// The mortar fluxes may run on the second stream beside the main stream's
// next kernel that does not read them, except when kernels are timed one by
// one (their events would then measure overlapping work).
static bool can_fork(const idp_ctx *c) { return c->prof != 2 && c->st2 != nullptr; }

static cudaStream_t fork_to_second(idp_ctx *c, cudaStream_t st) {
    cudaEventRecord(c->ev_fork, st);
    cudaStreamWaitEvent(c->st2, c->ev_fork, 0);
    return c->st2;
}

void enqueue_stage(idp_ctx *c, cudaStream_t st, const StageArgs &A, bool need_mortar_flux, bool need_face) {
    const int gm = (int)((c->M + MORTARS_PER_BLOCK - 1) / MORTARS_PER_BLOCK);
    bool dgmode = (A.mode == 0 && A.dt == 0.0) || A.limiting == 0;
    // FP64 path: the mortar fluxes beside the conforming-face kernel, both on
    // the stage's input state; joined before the element pass
    const bool fork = can_fork(c) && c->M > 0 && need_mortar_flux && c->facebuf && need_face && !(c->lob && !dgmode);
    if (c->M > 0 && need_mortar_flux) {
        cudaStream_t sm = fork ? fork_to_second(c, st) : st;
        int k = kt_begin(c, sm, IDP_K_MORTAR_FLUX);
        c->L.mortar_flux(c->opt.precision, c->ent_bar, c->opt.mortar_low, gm, sm, c->mesh, c->slots, A.u, A.gas, c->d_ops);
        kt_end(c, sm, k);
        if (fork) cudaEventRecord(c->ev_join, sm);
    }
    const int grid = element_grid(c, c->epb, c->persistent, c->bps);
    if (c->lob && !dgmode) {
        // low-order bounds (Eq. Bounds_LowOrder): u_FV of every node first,
        // then the ranges across the mortars
        StageArgs P = A;
        P.pass = 1;
        int k = kt_begin(c, st, IDP_K_ELEMENT_LO);
        c->L.element(c->opt.precision, c->ext, c->epb, grid, st, c->mesh, c->slots, P);
        kt_end(c, st, k);
        if (c->M > 0) {
            k = kt_begin(c, st, IDP_K_MORTAR_LOB);
            c->L.mortar_lob(st, c->mesh, c->slots, c->d_ops, c->d_lofv, c->opt.entropy_bound, c->num_sms);
            kt_end(c, st, k);
        }
    }
    int k;
    if (c->facebuf && need_face) {
        k = kt_begin(c, st, IDP_K_FACE);
        c->L.face(st, c->mesh, A.u, A.gas, c->d_ops, c->d_fbuf, c->num_sms);
        kt_end(c, st, k);
    }
    if (fork) cudaStreamWaitEvent(st, c->ev_join, 0);
    k = kt_begin(c, st, IDP_K_ELEMENT);
    c->L.element(c->opt.precision, c->ext, c->epb, grid, st, c->mesh, c->slots, A);
    kt_end(c, st, k);
    if (c->M > 0 && !dgmode) {
        k = kt_begin(c, st, IDP_K_MORTAR_LIMIT);
        c->L.mortar_limit(gm, st, c->mesh, c->slots, A);
        kt_end(c, st, k);
    }
}

// The per-simulation time-step minimum is +inf between calls: the context
// starts so, a step's k_time_advance resets it after use, and every other
// caller that forms a time step (reset = true) resets it first and restores
// it after reading it (dt_restore), so a step needs no reset launch.
void enqueue_dt(idp_ctx *c, cudaStream_t st, const double *u, bool mortar_flux, bool reset) {
    int k;
    if (reset) {
        k = kt_begin(c, st, IDP_K_DT_INIT);
        k_dt_init<<<(2 * c->n_sims + 255) / 256, 256, 0, st>>>(c->d_dtmin, c->n_sims);
        kt_end(c, st, k);
    }
    // the mortar fluxes of u^n beside the face or wave-speed kernel; the time
    // step joins them before it reads the mortars' 2d sums
    const bool fork = can_fork(c) && c->M > 0 && mortar_flux && c->opt.dt_rule == 0;
    if (c->M > 0 && mortar_flux && c->opt.dt_rule == 0) {
        const int gm = (int)((c->M + MORTARS_PER_BLOCK - 1) / MORTARS_PER_BLOCK);
        cudaStream_t sm = fork ? fork_to_second(c, st) : st;
        k = kt_begin(c, sm, IDP_K_MORTAR_FLUX);
        c->L.mortar_flux(c->opt.precision, c->ent_bar, c->opt.mortar_low, gm, sm, c->mesh, c->slots, u, make_gas(c->gamma, &c->d_ops->lg),
                         c->d_ops);
        kt_end(c, sm, k);
        if (fork) cudaEventRecord(c->ev_join, sm);
    }
    // FP64 path: the conforming faces of u^n first; the time step reads their
    // wave speeds and stage 1 of a step their fluxes
    const bool faces = c->facebuf && c->opt.dt_rule == 0;
    if (faces) {
        k = kt_begin(c, st, IDP_K_FACE);
        c->L.face(st, c->mesh, u, make_gas(c->gamma, &c->d_ops->lg), c->d_ops, c->d_fbuf, c->num_sms);
        kt_end(c, st, k);
    }
    int g = (int)std::max<long long>(1, std::min<long long>(((long long)KN(c) + 255) / 256, (long long)c->num_sms * 16));
    // without the face buffer: every node's wave speeds first (beside the
    // mortar fluxes), which the time step reads for its own and its
    // conforming neighbours' nodes
    void *lam = faces ? nullptr : c->d_lam;
    if (lam) {
        k = kt_begin(c, st, IDP_K_DT_SPEED);
        c->L.dt_speed(c->opt.precision, st, c->mesh, u, make_gas(c->gamma, &c->d_ops->lg), c->d_status, lam, c->num_sms);
        kt_end(c, st, k);
    }
    if (fork) cudaStreamWaitEvent(st, c->ev_join, 0);   // the mortars' 2d sums
    const Gas gas = make_gas(c->gamma, &c->d_ops->lg);
    if (faces && c->d_emin) {
        // FP64 path: the FP32 pass over every node, then the FP64 quotients
        // of the elements within its margin (the same minimum as one FP64
        // pass over every node)
        k = kt_begin(c, st, IDP_K_DT_FILTER);
        c->L.dt(0, g, st, c->mesh, c->slots, u, gas, c->opt.dt_rule, c->d_ops, c->d_tsim, c->d_dtmin, c->d_status,
                c->d_fbuf, nullptr, 1, c->d_emin);
        kt_end(c, st, k);
        k = kt_begin(c, st, IDP_K_DT);
        c->L.dt(0, g, st, c->mesh, c->slots, u, gas, c->opt.dt_rule, c->d_ops, c->d_tsim, c->d_dtmin, c->d_status,
                c->d_fbuf, nullptr, 2, c->d_emin);
        kt_end(c, st, k);
    } else {
        k = kt_begin(c, st, IDP_K_DT);
        c->L.dt(c->opt.precision, g, st, c->mesh, c->slots, u, gas, c->opt.dt_rule, c->d_ops, c->d_tsim, c->d_dtmin,
                c->d_status, faces ? c->d_fbuf : nullptr, lam, 0, nullptr);
        kt_end(c, st, k);
    }
}

// one SSP-RK3 step on u (in place), using the ctx stage buffers
static void dt_restore(idp_ctx *c, cudaStream_t st) {
    k_dt_init<<<(2 * c->n_sims + 255) / 256, 256, 0, st>>>(c->d_dtmin, c->n_sims);
}

void enqueue_step(idp_ctx *c, cudaStream_t st, double *u) {
    enqueue_dt(c, st, u, true, false);
    StageArgs A = base_args(c);
    A.mode = 1;
    A.un = u;
    // stage 1: u1 = ut(u)
    A.u = u; A.out = c->d_buf1; A.comb = 0; A.tstage = 0.0;
    enqueue_stage(c, st, A, c->opt.dt_rule != 0, c->opt.dt_rule != 0);   // mortars and faces of u^n are current
    // stage 2: u2 = 3/4 u + 1/4 ut(u1)
    A.u = c->d_buf1; A.out = c->d_buf2; A.comb = 1; A.tstage = 1.0;
    enqueue_stage(c, st, A, true, true);
    // stage 3: u3 = u/3 + 2/3 ut(u2), in place
    A.u = c->d_buf2; A.out = u; A.comb = 2; A.tstage = 0.5;
    enqueue_stage(c, st, A, true, true);
    const int k = kt_begin(c, st, IDP_K_TIME_ADVANCE);
    k_time_advance<<<(c->n_sims + 255) / 256, 256, 0, st>>>(c->d_tsim, c->d_dtmin, c->opt.cfl, c->d_dtlast,
                                                           c->n_sims);
    kt_end(c, st, k);
}

idp_status check_cuda(cudaError_t e) { return note(e, "launch") == cudaSuccess ? IDP_OK : IDP_E_CUDA; }

// Choose elements per block and grid mode by timing the element pass on the
// given state, output to a scratch buffer: as a right-hand side (rhs calls)
// or as an SSP-RK3 stage with its stage combination and the time step
// already in d_dtmin (step calls; the right-hand-side epilogue divides by the
// node mass and so weighs the FP64 pipe differently). Cached per degree,
// precision, kernel, mode, SM count and mesh-size bucket.
idp_status autotune(idp_ctx *c, const double *u, cudaStream_t st, double dt, int step_mode) {
    if (c->tuned) return IDP_OK;
    long long bucket = 0;
    for (long long k = c->K; k > 1; k >>= 1) ++bucket;
    long long key = ((long long)c->NP << 48) | ((long long)c->opt.precision << 40) | ((long long)c->ext << 39) |
                    ((long long)(step_mode != 0) << 38) |
                    ((long long)c->opt.grid_mode << 36) | ((long long)c->num_sms << 16) | bucket;
    if (c->opt.elems_per_block > 0) {
        int bps = 1;
        if (c->L.element_prepare(c->opt.precision, c->ext, c->opt.elems_per_block, &bps) != cudaSuccess || bps < 1)
            return IDP_E_ARG;
        c->epb = c->opt.elems_per_block; c->bps = bps; c->persistent = c->opt.grid_mode == 2 ? 1 : 0;
        c->tuned = true;
        return IDP_OK;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            int bps = 1;
            if (c->L.element_prepare(c->opt.precision, c->ext, it->second.first, &bps) == cudaSuccess) {
                c->epb = it->second.first; c->persistent = it->second.second; c->bps = bps; c->tuned = true;
                return IDP_OK;
            }
        }
    }
    StageArgs A = base_args(c);
    A.mode = 0; A.u = u; A.out = c->d_buf1; A.dt = dt; A.t = 0.0; A.collect = 0;
    if (step_mode) { A.mode = 1; A.un = u; A.comb = 2; A.tstage = 0.5; }
    if (c->facebuf) c->L.face(st, c->mesh, u, A.gas, c->d_ops, c->d_fbuf, c->num_sms);   // faces of u, once
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // every candidate is timed in two interleaved rounds and keeps its
    // faster round: one round alone picked configurations up to 7% slower
    // (clock ramp and run-to-run spread are of the order of the differences)
    float cand_ms[kNumEpb][2];
    int cand_bps[kNumEpb];
    for (int ci = 0; ci < kNumEpb; ++ci) {
        cand_ms[ci][0] = cand_ms[ci][1] = -1.0f;   // < 0: not a candidate
        int epb = kEpbChoices[ci], bps = 0;
        cand_bps[ci] = 0;
        if (c->L.element_prepare(c->opt.precision, c->ext, epb, &bps) != cudaSuccess || bps < 1) { cudaGetLastError(); continue; }
        if ((long long)epb > 4 * c->K && epb > 1) continue;
        cand_bps[ci] = bps;
        for (int pers = 0; pers < 2; ++pers) {
            if ((c->opt.grid_mode == 1 && pers == 1) || (c->opt.grid_mode == 2 && pers == 0)) continue;
            c->L.element(c->opt.precision, c->ext, epb, element_grid(c, epb, pers, bps), st, c->mesh, c->slots,
                         A);                                                     // warm-up
            if (cudaGetLastError() != cudaSuccess) continue;                     // not launchable
            cand_ms[ci][pers] = 1e30f;
        }
    }
    for (int round = 0; round < 2; ++round)
        for (int ci = 0; ci < kNumEpb; ++ci)
            for (int pers = 0; pers < 2; ++pers) {
                if (cand_ms[ci][pers] < 0.0f) continue;
                const int epb = kEpbChoices[ci], grid = element_grid(c, epb, pers, cand_bps[ci]);
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3; ++r) c->L.element(c->opt.precision, c->ext, epb, grid, st, c->mesh, c->slots, A);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return IDP_E_CUDA; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                cand_ms[ci][pers] = std::min(cand_ms[ci][pers], ms);
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    float best = 1e30f;
    int best_epb = 0, best_pers = 0, best_bps = 1;
    for (int ci = 0; ci < kNumEpb; ++ci)
        for (int pers = 0; pers < 2; ++pers)
            if (cand_ms[ci][pers] >= 0.0f && cand_ms[ci][pers] < best) {
                best = cand_ms[ci][pers]; best_epb = kEpbChoices[ci]; best_pers = pers; best_bps = cand_bps[ci];
            }
    if (!best_epb) return IDP_E_CUDA;
    c->epb = best_epb; c->persistent = best_pers; c->bps = best_bps; c->tuned = true;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {best_epb, best_pers};
    return check_cuda(cudaGetLastError());
}

// Device-flagged conditions are reported once: the word is cleared after reading.
idp_status read_status(idp_ctx *c) {
    unsigned st = 0;
    if (cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return IDP_E_CUDA;
    if (st && cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess) return IDP_E_CUDA;
    if (st & ST_BAD_INPUT) return IDP_E_STATE;
    if (st & ST_VIOLATION) return IDP_E_NUMERIC;
    return IDP_OK;
}

void reset_stats(idp_ctx *c, cudaStream_t st) {
    StatsAcc z;
    std::memset(&z, 0, sizeof(z));
    z.min_rho_bits = 0x7FF0000000000000ull;
    z.min_p_bits = 0x7FF0000000000000ull;
    cudaMemcpyAsync(c->d_stats, &z, sizeof(z), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
}

// The mortar slots (index m * 3(N+1) + q) as one block of device memory with
// room for Mcap mortars; the sub-arrays hold the current M mortars' slots,
// S = M 3(N+1) apart for the [4][S] ones. Zeroed.
cudaError_t alloc_slots(idp_ctx *c, long long Mcap) {
    const int Q = 3 * c->NP;
    if (c->d_slot_block) { cudaFree(c->d_slot_block); c->d_slot_block = nullptr; }
    const size_t S = (size_t)c->M * Q, MM = (size_t)std::max<long long>(Mcap, 1),
                 SS = std::max<size_t>((size_t)Mcap * Q, 1);
    size_t bytes = sizeof(double) * (SS * (4 + 4 + 3 + 4 + 4 + 6 + 5)) + sizeof(float) * SS + sizeof(int32_t) * MM +
                   sizeof(double) * MM + 22 * 256;   // 21 sub-arrays, each padded to 256 B
    cudaError_t e = cudaMalloc(&c->d_slot_block, bytes);
    if (e == cudaSuccess) e = cudaMemset(c->d_slot_block, 0, bytes);
    if (e != cudaSuccess) return e;
    char *p = (char *)c->d_slot_block;
    auto take = [&](size_t nb) { char *r = p; p += (nb + 255) & ~size_t(255); return (void *)r; };
    SlotsDev &sl = c->slots;
    sl.S = (int)S;
    sl.chi = (double *)take(sizeof(double) * 4 * SS);
    sl.clo = (double *)take(sizeof(double) * 4 * SS);
    sl.rbmin = (double *)take(sizeof(double) * SS);
    sl.rbmax = (double *)take(sizeof(double) * SS);
    sl.dsum = (double *)take(sizeof(double) * SS);
    sl.uvol = (double *)take(sizeof(double) * 4 * SS);
    sl.un = (double *)take(sizeof(double) * 4 * SS);
    sl.rmin = (double *)take(sizeof(double) * SS);
    sl.rmax = (double *)take(sizeof(double) * SS);
    sl.pmin = (double *)take(sizeof(double) * SS);
    sl.tol = (double *)take(sizeof(double) * SS);
    sl.mass = (double *)take(sizeof(double) * SS);
    sl.rfv = (double *)take(sizeof(double) * SS);
    sl.nmort = (float *)take(sizeof(float) * SS);
    sl.bad = (int32_t *)take(sizeof(int32_t) * MM);
    sl.ell = (double *)take(sizeof(double) * MM);
    sl.lnK = (double *)take(sizeof(double) * SS);
    sl.sbmin = (double *)take(sizeof(double) * SS);
    sl.lbmin = (double *)take(sizeof(double) * SS);
    sl.lbmax = (double *)take(sizeof(double) * SS);
    sl.lsmin = (double *)take(sizeof(double) * SS);
    if ((size_t)(p - (char *)c->d_slot_block) > bytes) return cudaErrorMemoryAllocation;
    return cudaSuccess;
}

idp_status create_impl(const idp_mesh_desc *meshes, int n_sims, int N, double gamma, const idp_options *opts,
                       idp_ctx **out) {
    if (!out) return IDP_E_ARG;
    *out = nullptr;
    if (!meshes || n_sims < 1 || N < 1 || N > NPMAX - 1 || !(gamma > 1.0)) return IDP_E_ARG;
    idp_options o;
    idp_options_default(&o);
    if (opts) o = *opts;
    if (o.precision < 0 || o.precision > 1 || o.limiting < 0 || o.limiting > 3 || o.dt_rule < 0 || o.dt_rule > 1 ||
        !(o.beta >= 0.0 && o.beta < 1.0) || !(o.cfl > 0.0) || o.mortar_projection < 0 || o.mortar_projection > 1)
        return IDP_E_ARG;
    if (o.bounds < 0 || o.bounds > 1 || o.entropy_bound < 0 || o.entropy_bound > 1 || o.volume_flux < 0 ||
        o.volume_flux > 1 || o.mortar_low < 0 || o.mortar_low > 1)
        return IDP_E_ARG;
    if (o.elems_per_block != 0 && o.elems_per_block != 1 && o.elems_per_block != 2 && o.elems_per_block != 4 &&
        o.elems_per_block != 8 && o.elems_per_block != 16)
        return IDP_E_ARG;
    if (o.grid_mode < 0 || o.grid_mode > 2) return IDP_E_ARG;
    HostMesh H;
    H.sim_off.push_back(0);
    std::vector<int8_t> all_lev;
    std::vector<int32_t> all_ix, all_iy;
    for (int s = 0; s < n_sims; ++s) {
        idp_status r = build_mesh(meshes[s], gamma, s, H);
        if (r != IDP_OK) return r;
        H.sim_off.push_back((long long)H.geom.size());
        all_lev.insert(all_lev.end(), meshes[s].level, meshes[s].level + meshes[s].n_leaves);
        all_ix.insert(all_ix.end(), meshes[s].ix, meshes[s].ix + meshes[s].n_leaves);
        all_iy.insert(all_iy.end(), meshes[s].iy, meshes[s].iy + meshes[s].n_leaves);
    }
    idp_ctx *c = new (std::nothrow) idp_ctx();
    if (!c) return IDP_E_ARG;
    c->N = N; c->NP = N + 1; c->n_sims = n_sims; c->gamma = gamma; c->opt = o;
    // the variants act only in local limiting (and its half of the combined mode)
    c->lob = o.limiting >= 2 && o.bounds == 1;
    c->ext = (o.limiting >= 2 && (o.bounds == 1 || o.entropy_bound == 1)) || o.volume_flux == 1;
    c->ent_bar = o.limiting >= 2 && o.entropy_bound == 1 && o.bounds == 0;
    c->facebuf = o.precision == 0 && !c->ext;
    c->K = (long long)H.geom.size(); c->M = (long long)H.m_large.size();
    c->sim_off = H.sim_off;
    for (const Geo &g : H.geom) c->total_area += g.z * g.w;
    for (size_t m = 0; m < H.m_large.size(); ++m) {
        const Geo &g = H.geom[H.m_large[m]];
        c->total_mortar_len += (H.m_info[m] & 1) == 0 ? g.w : g.z;
    }
    c->L = get_launchers(c->NP);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) { note(ce, "device query"); delete c; return IDP_E_CUDA; }
    Ops ops;
    build_ops(N, o.mortar_projection, o.mortar_low, ops);
    // unique mortar nodes and the blocks of the mortar limiting kernel
    const int NP = c->NP, NN = NP * NP, Q = 3 * NP;
    std::vector<int32_t> mn_node;
    std::vector<int2> mn_slot;
    std::vector<int32_t> mb_node_off(1, 0), mb_for_off(1, 0), mb_foreign;
    {
        idp_status r = host_mortar_tables(c->NP, c->L.mortar_w, (int)c->K, (int)c->M, H.m_large, H.m_small, H.m_info,
                                          mn_node, mn_slot, mb_node_off, mb_for_off, mb_foreign, c->mb_fmax);
        if (r != IDP_OK) { delete c; return r; }
        c->n_mnodes = (int)mn_node.size();
        c->mb_blocks = (int)mb_node_off.size() - 1;
    }
    bool ok = true;
    int step_no = 0;
    auto chk = [&](cudaError_t e) { ++step_no; if (e != cudaSuccess) { ok = false; char w[32]; std::snprintf(w, 32, "create step %d", step_no); note(e, w); } };
    chk(cudaMalloc(&c->d_ops, sizeof(Ops)));
    if (ok) chk(cudaMemcpy(c->d_ops, &ops, sizeof(Ops), cudaMemcpyHostToDevice));
    if (ok) chk(upload(&c->d_geom, H.geom));
    {
        std::vector<GeoC> gcv(H.geom.size());
        for (size_t e = 0; e < H.geom.size(); ++e) {
            const Geo &g = H.geom[e];
            GeoC &q = gcv[e];
            std::memset(&q, 0, sizeof(q));
            q.iA4 = 4.0 / (g.z * g.w); q.A4 = 0.25 * (g.z * g.w);
            q.hx = 0.5 * g.z; q.hy = 0.5 * g.w; q.qx = 0.25 * g.z; q.qy = 0.25 * g.w;
            q.hxf = (float)q.hx; q.hyf = (float)q.hy; q.qxf = (float)q.qx; q.qyf = (float)q.qy; q.A4f = (float)q.A4;
        }
        if (ok) chk(upload(&c->d_geoc, gcv));
    }
    if (ok) chk(upload(&c->d_sim, H.sim));
    if (ok) chk(upload(&c->d_fnbr, H.fnbr));
    if (ok) chk(upload(&c->d_ftype, H.ftype));
    if (ok) chk(upload(&c->d_mlarge, H.m_large));
    if (ok) chk(upload(&c->d_msmall, H.m_small));
    if (ok) chk(upload(&c->d_minfo, H.m_info));
    if (ok) chk(upload(&c->d_siminfo, H.siminfo));
    if (ok) chk(upload(&c->d_mnnode, mn_node));
    if (ok) chk(upload(&c->d_mnslot, mn_slot));
    if (ok) chk(upload(&c->d_mbnode, mb_node_off));
    if (ok) chk(upload(&c->d_mbfor, mb_for_off));
    if (ok) chk(upload(&c->d_mbforeign, mb_foreign));
    if (ok) chk(upload(&c->d_lev, all_lev));
    if (ok) chk(upload(&c->d_ix, all_ix));
    if (ok) chk(upload(&c->d_iy, all_iy));
    c->rmesh.nx0 = meshes[0].nx0; c->rmesh.ny0 = meshes[0].ny0;
    c->rmesh.x0 = meshes[0].x0; c->rmesh.y0 = meshes[0].y0; c->rmesh.x1 = meshes[0].x1; c->rmesh.y1 = meshes[0].y1;
    for (int s = 0; s < 4; ++s) c->rmesh.bc[s] = meshes[0].bc[s];
    c->capK = c->K; c->capM = c->M;
    c->cap_nodes = (long long)mn_node.size(); c->cap_blocks = (long long)mb_node_off.size();
    c->cap_foreign = (long long)mb_foreign.size();
    // slots: one block of device memory
    if (ok) chk(alloc_slots(c, c->M));
    const size_t kn = KN(c);
    if (ok) chk(cudaMalloc(&c->d_buf1, sizeof(double) * 4 * kn));
    if (ok) chk(cudaMalloc(&c->d_buf2, sizeof(double) * 4 * kn));
    // the time-step minimum per simulation, then the FP32 pass's minimum of
    // the two-pass time step (k_dt)
    if (ok) chk(cudaMalloc(&c->d_dtmin, sizeof(unsigned long long) * 2 * n_sims));
    if (ok) {
        const std::vector<unsigned long long> inf(2 * n_sims, 0x7FF0000000000000ull);   // +inf: no step formed yet
        chk(cudaMemcpy(c->d_dtmin, inf.data(), sizeof(unsigned long long) * 2 * n_sims, cudaMemcpyHostToDevice));
    }
    if (ok) chk(cudaMalloc(&c->d_tsim, sizeof(double) * n_sims));
    if (ok) chk(cudaMalloc(&c->d_dtlast, sizeof(double) * n_sims));
    if (ok) chk(cudaMalloc(&c->d_status, sizeof(unsigned)));
    if (ok) chk(cudaMemset(c->d_status, 0, sizeof(unsigned)));
    if (ok) chk(cudaMalloc(&c->d_stats, sizeof(StatsAcc)));
    if (ok) chk(cudaMalloc(&c->d_part, sizeof(double) * 4 * (size_t)c->K));
    if (ok) chk(cudaMalloc(&c->d_aind, sizeof(double) * (size_t)c->K));
    if (ok) chk(cudaMemset(c->d_aind, 0, sizeof(double) * (size_t)c->K));
    if (ok && c->facebuf) {
        const size_t F = (size_t)2 * c->K * c->NP;
        chk(cudaMalloc(&c->d_fbuf, sizeof(double) * 6 * F + sizeof(float) * F));
    }
    if (ok && (!c->facebuf || o.dt_rule != 0))
        chk(cudaMalloc(&c->d_lam, (o.precision ? sizeof(float) : sizeof(double)) * 2 * kn));
    if (ok && c->facebuf && o.dt_rule == 0) chk(cudaMalloc(&c->d_emin, sizeof(unsigned) * (size_t)c->K));
    if (ok && c->lob) chk(cudaMalloc(&c->d_lofv, sizeof(double) * 2 * kn));
    if (ok && c->lob) chk(cudaMemset(c->d_lofv, 0, sizeof(double) * 2 * kn));
    if (ok) chk(cudaMalloc(&c->d_intout, sizeof(double) * 4 * n_sims));
    if (ok) chk(upload(&c->d_off, c->sim_off));
    if (ok) chk(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    if (ok) chk(cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking));
    if (ok) chk(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    if (ok) chk(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    if (ok) chk(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    if (ok) chk(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    if (!ok) { idp_dgsem_destroy(c); return IDP_E_CUDA; }
    MeshDev &md = c->mesh;
    md.K = (int)c->K; md.M = (int)c->M; md.n_sims = n_sims; md.n_mnodes = c->n_mnodes;
    md.geom = c->d_geom; md.geoc = c->d_geoc; md.sim = c->d_sim; md.fnbr = c->d_fnbr; md.ftype = c->d_ftype;
    md.m_large = c->d_mlarge; md.m_small = c->d_msmall; md.m_info = c->d_minfo; md.siminfo = c->d_siminfo;
    md.mn_node = c->d_mnnode; md.mn_slot = c->d_mnslot;
    md.mb_node_off = c->d_mbnode; md.mb_for_off = c->d_mbfor; md.mb_foreign = c->d_mbforeign;
    md.mb_fmax = c->mb_fmax; md.mb_blocks = c->mb_blocks;
    reset_stats(c, c->stream);
    std::vector<double> tz(n_sims, 0.0);
    cudaMemcpy(c->d_tsim, tz.data(), sizeof(double) * n_sims, cudaMemcpyHostToDevice);
    if (note(cudaDeviceSynchronize(), "create sync") != cudaSuccess) { idp_dgsem_destroy(c); return IDP_E_CUDA; }
    *out = c;
    return IDP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {
// (re)allocate *p for n elements of T when it holds fewer than cap
template <typename T>
cudaError_t ensure(T **p, long long n, long long cap) {
    if (n <= cap && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<long long>(n, 1));
}
}  // namespace

extern "C" {

const char *idp_last_cuda_error(void) { return g_last_error; }

const char *idp_status_str(idp_status s) {
    switch (s) {
    case IDP_OK: return "ok";
    case IDP_E_ARG: return "invalid argument";
    case IDP_E_MESH: return "invalid mesh (overlap, gap, out of range or not 2:1 balanced)";
    case IDP_E_CUDA: return "CUDA runtime error";
    case IDP_E_STATE: return "invalid state (rho <= 0, p <= 0 or non-finite)";
    case IDP_E_DT: return "no admissible time step";
    case IDP_E_NUMERIC: return "bound violation after limiting";
    case IDP_E_TIMEOUT: return "device wait timed out";
    case IDP_E_UNSUPPORTED: return "option not supported";
    }
    return "unknown status";
}

idp_status idp_options_default(idp_options *o) {
    if (!o) return IDP_E_ARG;
    std::memset(o, 0, sizeof(*o));
    o->precision = 0;
    o->limiting = 2;
    o->bounds = 0;
    o->dt_rule = 0;
    o->beta = 0.1;
    o->cfl = 0.5;
    o->mortar_projection = 1;
    o->elems_per_block = 0;
    o->collect_stats = 1;
    return IDP_OK;
}

idp_status idp_dgsem_create(const idp_mesh_desc *mesh, int32_t N, double gamma, const idp_options *opts,
                            idp_ctx **ctx) {
    try {
        return create_impl(mesh, 1, N, gamma, opts, ctx);
    } catch (...) {
        return IDP_E_ARG;
    }
}

idp_status idp_dgsem_create_batch(const idp_mesh_desc *meshes, int32_t n_sims, int32_t N, double gamma,
                                  const idp_options *opts, idp_ctx **ctx) {
    try {
        return create_impl(meshes, n_sims, N, gamma, opts, ctx);
    } catch (...) {
        return IDP_E_ARG;
    }
}

idp_status idp_dgsem_layout(const idp_ctx *c, int64_t *n_elems, int64_t *n_mortars, int32_t *n_sims,
                            int64_t *sim_elem_offsets) {
    if (!c) return IDP_E_ARG;
    if (n_elems) *n_elems = c->K;
    if (n_mortars) *n_mortars = c->M;
    if (n_sims) *n_sims = c->n_sims;
    if (sim_elem_offsets)
        for (int s = 0; s <= c->n_sims; ++s) sim_elem_offsets[s] = c->sim_off[s];
    return IDP_OK;
}

idp_status idp_dgsem_launch_config(const idp_ctx *c, int32_t *elems_per_block, int32_t *persistent,
                                   int32_t *grid) {
    if (!c) return IDP_E_ARG;
    const bool t = c->tuned;
    if (elems_per_block) *elems_per_block = t ? c->epb : 0;
    if (persistent) *persistent = t ? c->persistent : 0;
    if (grid) *grid = t ? element_grid(c, c->epb, c->persistent, c->bps) : 0;
    return IDP_OK;
}

idp_status idp_dgsem_rhs(idp_ctx *c, const double *u, double t, double dt, double *rhs, void *stream) {
    if (!c || !u || !rhs || u == rhs || !(dt >= 0.0) || !std::isfinite(dt)) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    idp_status r = autotune(c, u, st, dt, 0);
    if (r != IDP_OK) return r;
    StageArgs A = base_args(c);
    A.mode = 0; A.u = u; A.out = rhs; A.dt = dt; A.t = t;
    enqueue_stage(c, st, A, true, true);
    if (dt > 0.0 && c->opt.limiting > 0) c->n_stages += 1;
    return check_cuda(cudaGetLastError());
}

idp_status idp_dgsem_dt(idp_ctx *c, const double *u, const double *t_host, double *dt_host, void *stream) {
    if (!c || !u || !dt_host) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> tz(c->n_sims, 0.0);
    if (t_host) for (int s = 0; s < c->n_sims; ++s) tz[s] = t_host[s];
    if (cudaMemcpyAsync(c->d_tsim, tz.data(), sizeof(double) * c->n_sims, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return IDP_E_CUDA;
    enqueue_dt(c, st, u, true, true);
    std::vector<unsigned long long> b(c->n_sims);
    if (cudaMemcpyAsync(b.data(), c->d_dtmin, sizeof(unsigned long long) * c->n_sims, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return IDP_E_CUDA;
    dt_restore(c, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return IDP_E_CUDA;
    for (int s = 0; s < c->n_sims; ++s) {
        double v;
        std::memcpy(&v, &b[s], sizeof(double));
        if (!(v > 0.0) || !std::isfinite(v)) return IDP_E_DT;
        dt_host[s] = c->opt.cfl * v;
    }
    return read_status(c);
}

idp_status idp_dgsem_step(idp_ctx *c, double *u, int32_t n_steps, double *t_host, double *dt_last_host,
                          void *stream) {
    if (!c || !u || n_steps < 0 || !t_host) return IDP_E_ARG;
    cudaStream_t ust = (cudaStream_t)stream;
    // steps run on the caller's stream; the legacy default stream cannot be
    // captured into a graph, so then the context's own stream is used,
    // ordered after the caller's
    const bool own = ust == nullptr;
    cudaStream_t st = own ? c->stream : ust;
    if (own && (cudaEventRecord(c->ev_in, ust) != cudaSuccess || cudaStreamWaitEvent(st, c->ev_in, 0) != cudaSuccess))
        return IDP_E_CUDA;
    if (cudaMemcpyAsync(c->d_tsim, t_host, sizeof(double) * c->n_sims, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return IDP_E_CUDA;
    if (!c->tuned) {
        // tune on u with its own IDP step
        enqueue_dt(c, st, u, true, true);
        std::vector<unsigned long long> b(c->n_sims);
        cudaMemcpyAsync(b.data(), c->d_dtmin, sizeof(unsigned long long) * c->n_sims, cudaMemcpyDeviceToHost, st);
        dt_restore(c, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return IDP_E_CUDA;
        double v;
        std::memcpy(&v, &b[0], sizeof(double));
        idp_status r = autotune(c, u, st, std::isfinite(v) ? c->opt.cfl * v : 0.0, 1);
        if (r != IDP_OK) return r;
    }
    if (n_steps > 0 && c->prof == 2) {
        for (int k = 0; k < n_steps; ++k) {
            cudaEventRecord(c->pev[6], st);
            enqueue_step(c, st, u);
            cudaEventRecord(c->pev[7], st);
            if (note(cudaStreamSynchronize(st), "step") != cudaSuccess) return IDP_E_CUDA;
            if (note(kt_collect(c), "profile") != cudaSuccess) return IDP_E_CUDA;
            float ms = 0.f;
            if (note(cudaEventElapsedTime(&ms, c->pev[6], c->pev[7]), "profile") != cudaSuccess) return IDP_E_CUDA;
            c->prof_step_ms += ms;
            c->prof_steps += 1;
        }
        c->n_stages += 3LL * n_steps;
    } else if (n_steps > 0) {
        if (c->graph == nullptr || c->graph_u != u || c->graph_stale) {
            // re-captured when u or the mesh changes; the executable graph is
            // updated in place when the new capture has its shape
            cudaGraph_t g;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return IDP_E_CUDA;
            enqueue_step(c, st, u);
            if (cudaStreamEndCapture(st, &g) != cudaSuccess) return IDP_E_CUDA;
            bool updated = false;
            if (c->graph) {
                cudaGraphExecUpdateResultInfo info;
                updated = cudaGraphExecUpdate(c->graph, g, &info) == cudaSuccess;
                if (!updated) {
                    cudaGetLastError();   // the failed update is not an error of the step
                    cudaGraphExecDestroy(c->graph);
                    c->graph = nullptr;
                }
            }
            cudaError_t e = updated ? cudaSuccess : cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { c->graph = nullptr; return IDP_E_CUDA; }
            c->graph_u = u;
            c->graph_stale = false;
        }
        for (int k = 0; k < n_steps; ++k) {
            if (c->prof) cudaEventRecord(c->pev[6], st);
            if (note(cudaGraphLaunch(c->graph, st), "graph launch") != cudaSuccess) return IDP_E_CUDA;
            if (c->prof) {
                cudaEventRecord(c->pev[7], st);
                if (note(cudaStreamSynchronize(st), "step") != cudaSuccess) return IDP_E_CUDA;
                float ms = 0.f;
                if (note(cudaEventElapsedTime(&ms, c->pev[6], c->pev[7]), "profile") != cudaSuccess) return IDP_E_CUDA;
                c->prof_step_ms += ms;
                c->prof_steps += 1;
            }
        }
        c->n_stages += 3LL * n_steps;
    }
    cudaMemcpyAsync(t_host, c->d_tsim, sizeof(double) * c->n_sims, cudaMemcpyDeviceToHost, st);
    if (dt_last_host && n_steps > 0)
        cudaMemcpyAsync(dt_last_host, c->d_dtlast, sizeof(double) * c->n_sims, cudaMemcpyDeviceToHost, st);
    if (own) {
        cudaEventRecord(c->ev_out, st);
        cudaStreamWaitEvent(ust, c->ev_out, 0);
    }
    if (note(cudaStreamSynchronize(st), "step sync") != cudaSuccess) return IDP_E_CUDA;
    return read_status(c);
}

idp_status idp_dgsem_step_host(idp_ctx *c, double *u_host, int32_t n_steps, double *t_host, double *dt_last_host,
                               void *stream) {
    if (!c || !u_host) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = sizeof(double) * 4 * KN(c);
    // sized for the element capacity, which adaptation may fill
    if (!c->d_hostbuf &&
        cudaMalloc(&c->d_hostbuf, sizeof(double) * 4 * (size_t)c->capK * c->NP * c->NP) != cudaSuccess)
        return IDP_E_CUDA;
    if (cudaMemcpyAsync(c->d_hostbuf, u_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return IDP_E_CUDA;
    idp_status r = idp_dgsem_step(c, c->d_hostbuf, n_steps, t_host, dt_last_host, stream);
    if (r != IDP_OK && r != IDP_E_NUMERIC) return r;
    if (cudaMemcpyAsync(u_host, c->d_hostbuf, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return IDP_E_CUDA;
    return r;
}

idp_status idp_dgsem_integrals(idp_ctx *c, const double *u, double *out_host, void *stream) {
    if (!c || !u || !out_host) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int g = (int)std::max<long long>(1, std::min<long long>((c->K + 255) / 256, (long long)c->num_sms * 8));
    c->L.integrals(g, st, c->mesh, u, c->d_ops, c->d_part);
    k_sum_segments<<<c->n_sims, 256, 0, st>>>(c->d_part, (int)c->K, c->d_off, c->d_intout);
    if (cudaMemcpyAsync(out_host, c->d_intout, sizeof(double) * 4 * c->n_sims, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return IDP_E_CUDA;
    return IDP_OK;
}

idp_status idp_dgsem_limiter_stats(idp_ctx *c, idp_limiter_stats *out, void *stream) {
    if (!c || !out) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    StatsAcc a;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(&a, c->d_stats, sizeof(a), cudaMemcpyDeviceToHost) != cudaSuccess)
        return IDP_E_CUDA;
    std::memset(out, 0, sizeof(*out));
    // every limited stage visits every node once: the mass sum is the mesh
    // area times the number of limited stages (summed over the meshes the
    // stages ran on, when the context adapted in between)
    const double mass = c->stats_mass_prior + c->total_area * (double)(c->n_stages - c->stats_stages_prior);
    out->alpha_volume_mean = mass > 0 ? a.alpha_vol_m / mass : 0.0;
    // every limited stage limits every mortar once: the length sum is the
    // total mortar length times the number of limited stages
    const double mlen = c->stats_mlen_prior + c->total_mortar_len * (double)(c->n_stages - c->stats_stages_prior);
    out->alpha_mortar_mean = mlen > 0 ? a.alpha_mort_len / mlen : 0.0;
    out->n_stages = c->n_stages;
    out->n_volume_active = (int64_t)a.n_vol;
    out->n_mortar_active = (int64_t)a.n_mort;
    out->n_mortar_fallback = (int64_t)a.n_fallback;
    out->n_viol_density = (int64_t)a.n_vrho;
    out->n_viol_pressure = (int64_t)a.n_vp;
    out->n_nonpositive = (int64_t)a.n_nonpos;
    out->n_dt_exceed = (int64_t)a.n_dtx;
    out->n_viol_entropy = (int64_t)a.n_veta;
    std::memcpy(&out->min_rho, &a.min_rho_bits, sizeof(double));
    std::memcpy(&out->min_p, &a.min_p_bits, sizeof(double));
    c->n_stages = 0;
    c->stats_mass_prior = c->stats_mlen_prior = 0.0;
    c->stats_stages_prior = 0;
    reset_stats(c, c->stream);
    return read_status(c);
}

idp_status idp_dgsem_profile(idp_ctx *c, int32_t mode) {
    if (!c || mode < 0 || mode > 2) return IDP_E_ARG;
    if (mode && !c->pev[0]) {
        for (int k = 0; k < 8; ++k)
            if (note(cudaEventCreate(&c->pev[k]), "profile events") != cudaSuccess) return IDP_E_CUDA;
        for (int k = 0; k < idp_ctx::kMaxKev; ++k)
            for (int b = 0; b < 2; ++b)
                if (note(cudaEventCreate(&c->kev[k][b]), "profile events") != cudaSuccess) return IDP_E_CUDA;
    }
    c->kev_n = 0;
    c->prof = mode;
    return IDP_OK;
}

idp_status idp_dgsem_profile_read(idp_ctx *c, double *element_ms, int64_t *element_launches, double *step_ms,
                                  int64_t *steps, int32_t reset) {
    if (!c) return IDP_E_ARG;
    if (element_ms) *element_ms = c->kms[IDP_K_ELEMENT] + c->kms[IDP_K_FACE];
    if (element_launches) *element_launches = c->kcnt[IDP_K_ELEMENT];
    if (step_ms) *step_ms = c->prof_step_ms;
    if (steps) *steps = c->prof_steps;
    if (reset) {
        for (int k = 0; k < IDP_NKERNELS; ++k) { c->kms[k] = 0.0; c->kcnt[k] = 0; }
        c->prof_step_ms = 0.0; c->prof_steps = 0;
    }
    return IDP_OK;
}

idp_status idp_dgsem_profile_kernels(idp_ctx *c, double *ms, int64_t *launches, int32_t reset) {
    if (!c) return IDP_E_ARG;
    for (int k = 0; k < IDP_NKERNELS; ++k) {
        if (ms) ms[k] = c->kms[k];
        if (launches) launches[k] = c->kcnt[k];
        if (reset) { c->kms[k] = 0.0; c->kcnt[k] = 0; }
    }
    return IDP_OK;
}

idp_status idp_dgsem_sync(idp_ctx *c, void *stream) {
    if (!c) return IDP_E_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
        return IDP_E_CUDA;
    return read_status(c);
}

// ---- adaptive mesh refinement -------------------------------------------

idp_status idp_amr_params_default(idp_amr_params *p) {
    if (!p) return IDP_E_ARG;
    std::memset(p, 0, sizeof(*p));
    p->indicator = IDP_AMR_HENNEMANN;
    p->variable = IDP_AMR_DENSITY;
    p->refine_threshold = 0.5;
    p->coarsen_threshold = 0.05;
    p->min_level = 0;
    p->max_level = 3;
    p->lohner_filter = 0.2;
    p->zs_threshold = 1e-10;
    return IDP_OK;
}

static bool amr_params_ok(const idp_amr_params *p) {
    return p && p->indicator >= IDP_AMR_HENNEMANN && p->indicator <= IDP_AMR_MAX && p->variable >= 0 &&
           p->variable <= 1 && p->min_level >= 0 && p->max_level >= p->min_level && p->max_level <= 24 &&
           p->lohner_filter >= 0.0 && p->zs_threshold >= 0.0;
}

idp_status idp_dgsem_amr_indicator(idp_ctx *c, const double *u, const idp_amr_params *p, double *ind, void *stream) {
    if (!c || !u || !ind || !amr_params_ok(p)) return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    c->L.amr_indicator(st, u, (int)c->K, c->d_ops, c->gamma - 1.0, p->indicator, p->variable, p->lohner_filter, ind,
                       c->num_sms);
    return check_cuda(cudaGetLastError());
}

// The adaptation plan (host): marks, complete families for coarsening, 2:1
// face balance with refinement winning, new leaves in the old order.
idp_status idp_amr_plan(const idp_mesh_desc *mesh, const double *ind, const idp_amr_params *p, int32_t capacity,
                        int32_t *n_new, int8_t *level, int32_t *ix, int32_t *iy, int32_t *kind, int32_t *src) {
    if (!mesh || !ind || !amr_params_ok(p) || !n_new || !level || !ix || !iy || !kind || !src || capacity < 0)
        return IDP_E_ARG;
    {   // the input must be a valid balanced quadtree
        HostMesh H;
        idp_status r = build_mesh(*mesh, 1.4, 0, H);
        if (r != IDP_OK) return r;
    }
    const idp_mesh_desc &d = *mesh;
    const int K = d.n_leaves;
    std::unordered_map<uint64_t, int> key;
    key.reserve((size_t)K * 2);
    for (int e = 0; e < K; ++e) key.emplace(leaf_key(d.level[e], d.ix[e], d.iy[e]), e);
    auto find = [&](int l, int64_t x, int64_t y) {
        if (l < 0) return -1;
        auto it = key.find(leaf_key(l, x, y));
        return it == key.end() ? -1 : it->second;
    };
    std::vector<int> mark(K, 0);
    for (int e = 0; e < K; ++e) {
        if (ind[e] > p->refine_threshold && d.level[e] < p->max_level) mark[e] = 1;
        else if (ind[e] < p->coarsen_threshold && d.level[e] > p->min_level) mark[e] = -1;
    }
    auto family = [&](int e, int f[4]) {
        const int l = d.level[e];
        const int64_t px = d.ix[e] >> 1, py = d.iy[e] >> 1;
        for (int c = 0; c < 4; ++c) f[c] = find(l, 2 * px + (c & 1), 2 * py + (c >> 1));
    };
    for (int e = 0; e < K; ++e) {
        if (mark[e] != -1) continue;
        int f[4];
        family(e, f);
        bool ok = true;
        for (int c = 0; c < 4; ++c) ok = ok && f[c] >= 0 && mark[f[c]] == -1;
        if (!ok)
            for (int c = 0; c < 4; ++c)
                if (f[c] >= 0 && mark[f[c]] == -1) mark[f[c]] = 0;
    }
    const bool perx = d.bc[0] == IDP_BC_PERIODIC, pery = d.bc[2] == IDP_BC_PERIODIC;
    auto neighbours = [&](int e, int s, int out[2]) {
        const int l = d.level[e];
        const int64_t nx = (int64_t)d.nx0 << l, ny = (int64_t)d.ny0 << l;
        int64_t qx = d.ix[e] + (s == 0 ? -1 : (s == 1 ? 1 : 0));
        int64_t qy = d.iy[e] + (s == 2 ? -1 : (s == 3 ? 1 : 0));
        if (qx < 0 || qx >= nx) { if (!perx) return 0; qx = (qx + nx) % nx; }
        if (qy < 0 || qy >= ny) { if (!pery) return 0; qy = (qy + ny) % ny; }
        int f = find(l, qx, qy);
        if (f >= 0) { out[0] = f; return 1; }
        f = find(l - 1, qx >> 1, qy >> 1);
        if (l > 0 && f >= 0) { out[0] = f; return 1; }
        if (s < 2) {
            const int cx = s == 0 ? 1 : 0;
            out[0] = find(l + 1, 2 * qx + cx, 2 * qy);
            out[1] = find(l + 1, 2 * qx + cx, 2 * qy + 1);
        } else {
            const int cy = s == 2 ? 1 : 0;
            out[0] = find(l + 1, 2 * qx, 2 * qy + cy);
            out[1] = find(l + 1, 2 * qx + 1, 2 * qy + cy);
        }
        return 2;
    };
    for (bool changed = true; changed;) {
        changed = false;
        for (int e = 0; e < K; ++e) {
            int fe = d.level[e] + mark[e];
            for (int s = 0; s < 4; ++s) {
                int nb[2];
                const int cnt = neighbours(e, s, nb);
                for (int t = 0; t < cnt; ++t) {
                    const int f = nb[t];
                    if (f < 0) return IDP_E_MESH;
                    if (d.level[f] + mark[f] - fe >= 2) {
                        if (mark[e] == -1) {
                            int fam[4];
                            family(e, fam);
                            for (int c = 0; c < 4; ++c)
                                if (fam[c] >= 0) mark[fam[c]] = 0;
                        } else {
                            mark[e] = 1;
                        }
                        fe = d.level[e] + mark[e];
                        changed = true;
                    }
                }
            }
        }
    }
    int n = 0;
    auto emit = [&](int l, int64_t x, int64_t y, int k, int s0, int s1, int s2, int s3) {
        if (n < capacity) {
            level[n] = (int8_t)l; ix[n] = (int32_t)x; iy[n] = (int32_t)y; kind[n] = k;
            src[4 * n] = s0; src[4 * n + 1] = s1; src[4 * n + 2] = s2; src[4 * n + 3] = s3;
        }
        ++n;
    };
    for (int e = 0; e < K; ++e) {
        const int l = d.level[e];
        const int64_t x = d.ix[e], y = d.iy[e];
        if (mark[e] == 1) {
            for (int c = 0; c < 4; ++c) emit(l + 1, 2 * x + (c & 1), 2 * y + (c >> 1), 1, e, c, -1, -1);
        } else if (mark[e] == -1) {
            int f[4];
            family(e, f);
            if (std::min(std::min(f[0], f[1]), std::min(f[2], f[3])) == e) emit(l - 1, x >> 1, y >> 1, 2, f[0], f[1], f[2], f[3]);
        } else {
            emit(l, x, y, 0, e, -1, -1, -1);
        }
    }
    *n_new = n;
    return n <= capacity ? IDP_OK : IDP_E_ARG;
}

idp_status idp_amr_transfer(int32_t N, double gamma, const double *u_old, int64_t n_old, double *u_new, int64_t n_new,
                            const int32_t *kind, const int32_t *src, double zs_threshold, int64_t *n_scaled,
                            void *stream) {
    if (N < 1 || N > NPMAX - 1 || !(gamma > 1.0) || !u_old || !u_new || n_old < 1 || n_new < 1 || !kind || !src ||
        !(zs_threshold >= 0.0) || n_old > INT32_MAX || n_new > INT32_MAX)
        return IDP_E_ARG;
    // families for the Zhang-Shu scaling, and an argument check of the plan
    std::vector<int4> fam;
    for (int64_t e = 0; e < n_new;) {
        const int k = kind[e];
        const int32_t *s = src + 4 * e;
        if (k == 0) {
            if (s[0] < 0 || s[0] >= n_old) return IDP_E_ARG;
            ++e;
        } else if (k == 1) {
            if (e + 4 > n_new) return IDP_E_ARG;
            for (int c = 0; c < 4; ++c)
                if (kind[e + c] != 1 || src[4 * (e + c)] != s[0] || src[4 * (e + c) + 1] != c || s[0] < 0 || s[0] >= n_old)
                    return IDP_E_ARG;
            fam.push_back(make_int4((int)e, 4, 0, s[0]));
            e += 4;
        } else if (k == 2) {
            for (int c = 0; c < 4; ++c)
                if (s[c] < 0 || s[c] >= n_old) return IDP_E_ARG;
            fam.push_back(make_int4((int)e, 1, 1, (int)e));
            ++e;
        } else {
            return IDP_E_ARG;
        }
    }
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return IDP_E_CUDA;
    Ops ops;
    build_ops(N, 1, 0, ops);
    Launchers L = get_launchers(N + 1);
    cudaStream_t st = (cudaStream_t)stream;
    Ops *d_ops = nullptr;
    int *d_kind = nullptr;
    int4 *d_src = nullptr, *d_fam = nullptr;
    unsigned long long *d_cnt = nullptr;
    idp_status rc = IDP_OK;
    std::vector<int4> src4((size_t)n_new);
    for (int64_t e = 0; e < n_new; ++e) src4[e] = make_int4(src[4 * e], src[4 * e + 1], src[4 * e + 2], src[4 * e + 3]);
    auto ok = [&](cudaError_t e, const char *w) { if (e != cudaSuccess && rc == IDP_OK) { note(e, w); rc = IDP_E_CUDA; } return rc == IDP_OK; };
    if (ok(cudaMalloc(&d_ops, sizeof(Ops)), "amr alloc") && ok(cudaMalloc(&d_kind, sizeof(int) * n_new), "amr alloc") &&
        ok(cudaMalloc(&d_src, sizeof(int4) * n_new), "amr alloc") &&
        ok(cudaMalloc(&d_fam, sizeof(int4) * std::max<size_t>(fam.size(), 1)), "amr alloc") &&
        ok(cudaMalloc(&d_cnt, sizeof(unsigned long long)), "amr alloc") &&
        ok(cudaMemcpyAsync(d_ops, &ops, sizeof(Ops), cudaMemcpyHostToDevice, st), "amr copy") &&
        ok(cudaMemcpyAsync(d_kind, kind, sizeof(int) * n_new, cudaMemcpyHostToDevice, st), "amr copy") &&
        ok(cudaMemcpyAsync(d_src, src4.data(), sizeof(int4) * n_new, cudaMemcpyHostToDevice, st), "amr copy") &&
        (fam.empty() || ok(cudaMemcpyAsync(d_fam, fam.data(), sizeof(int4) * fam.size(), cudaMemcpyHostToDevice, st), "amr copy")) &&
        ok(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st), "amr copy")) {
        L.amr_transfer(st, u_old, (int)n_old, u_new, (int)n_new, d_kind, d_src, d_ops, sms);
        L.amr_zs(st, u_new, (int)n_new, u_old, (int)n_old, d_fam, (int)fam.size(), d_ops, gamma - 1.0, zs_threshold, d_cnt);
        unsigned long long cnt = 0;
        if (ok(cudaGetLastError(), "amr launch") && ok(cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st), "amr copy") &&
            ok(cudaStreamSynchronize(st), "amr sync") && n_scaled)
            *n_scaled = (int64_t)cnt;
    }
    cudaFree(d_ops); cudaFree(d_kind); cudaFree(d_src); cudaFree(d_fam); cudaFree(d_cnt);
    return rc;
}

// ---- adaptation on the device --------------------------------------------

idp_status idp_dgsem_adapt(idp_ctx *c, const double *u_old, const idp_amr_params *p, double *u_new,
                           int64_t capacity, int64_t *n_new, int64_t *n_scaled, void *stream) {
    if (!c || !u_old || !u_new || !amr_params_ok(p) || capacity < 1 || !n_new) return IDP_E_ARG;
    if (c->n_sims != 1 || c->prof == 2) return IDP_E_ARG;
    // leaf indices of the finest level must fit the 28-bit leaf keys (as at create)
    if (((int64_t)c->rmesh.nx0 << p->max_level) >= (1LL << 28) || ((int64_t)c->rmesh.ny0 << p->max_level) >= (1LL << 28))
        return IDP_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = (int)c->K, NP = c->NP, NN = NP * NP, Q = 3 * NP, W = c->L.mortar_w;
    // scratch: the indicator, the plan and its leaves (at most 4 K), then the
    // mesh builders' tables; it only grows
    const long long K4 = 4LL * K;
    const int Kb = (int)std::min<long long>(K4, std::max<long long>(capacity, 1));
    const size_t plan_ints = remesh_plan_scratch_ints(K);
    auto pad = [](size_t nb) { return (nb + 255) & ~size_t(255); };
    const size_t head = pad(sizeof(double) * K) + pad(sizeof(int) * plan_ints) + pad((size_t)Kb) +
                        3 * pad(sizeof(int) * (size_t)Kb) + 2 * pad(sizeof(int4) * (size_t)Kb) +
                        pad(sizeof(unsigned long long) + 2 * sizeof(double));
    // a 2:1 balanced mesh has at most one mortar per leaf (each mortar has
    // two small sides, each leaf at most two small sides)
    const size_t need = head + std::max(remesh_build_scratch_bytes(Kb, NP), remesh_nodes_scratch_bytes(Kb, NP, Kb, W));
    if (need > c->rm_bytes) {
        if (c->d_rm) cudaFree(c->d_rm);
        c->d_rm = nullptr;
        c->rm_bytes = 0;
        if (note(cudaMalloc(&c->d_rm, need), "adapt scratch") != cudaSuccess) return IDP_E_CUDA;
        c->rm_bytes = need;
    }
    char *q = (char *)c->d_rm;
    auto take = [&](size_t nb) { char *r = q; q += pad(nb); return (void *)r; };
    double *ind = (double *)take(sizeof(double) * K);
    int *plan_s = (int *)take(sizeof(int) * plan_ints);
    int8_t *nlev = (int8_t *)take((size_t)Kb);
    int *nix = (int *)take(sizeof(int) * Kb), *niy = (int *)take(sizeof(int) * Kb), *kind = (int *)take(sizeof(int) * Kb);
    int4 *src = (int4 *)take(sizeof(int4) * Kb), *fam = (int4 *)take(sizeof(int4) * Kb);
    unsigned long long *d_cnt = (unsigned long long *)take(sizeof(unsigned long long) + 2 * sizeof(double));
    void *build_s = (void *)q;
    // the context's streams are idle before its tables change
    if (note(cudaStreamSynchronize(c->stream), "adapt sync") != cudaSuccess ||
        note(cudaStreamSynchronize(c->st2), "adapt sync") != cudaSuccess)
        return IDP_E_CUDA;
    // indicator and plan on the current mesh
    c->L.amr_indicator(st, u_old, K, c->d_ops, c->gamma - 1.0, p->indicator, p->variable, p->lohner_filter, ind,
                       c->num_sms);
    PlanIn pin = {K, ind, c->d_lev, c->d_ix, c->d_iy, c->d_fnbr, c->d_ftype, c->d_mlarge, c->d_msmall,
                  p->refine_threshold, p->coarsen_threshold, p->min_level, p->max_level};
    PlanOut pout = {Kb, nlev, nix, niy, kind, src, fam};
    int Kn = 0, nfam = 0, iters = 0;
    if (note(remesh_plan(pin, pout, plan_s, st, c->num_sms, &Kn, &nfam, &iters), "adapt plan") != cudaSuccess)
        return IDP_E_CUDA;
    if (iters < 0) return IDP_E_MESH;
    *n_new = Kn;
    if (Kn > capacity) return IDP_E_ARG;   // the caller's state buffer is too small: *n_new says how large
    // transfer (interpolation, exact L2 projection, Zhang-Shu scaling)
    if (!c->d_ops_amr) {
        Ops oa;
        build_ops(c->N, 1, 0, oa);
        if (note(cudaMalloc(&c->d_ops_amr, sizeof(Ops)), "adapt ops") != cudaSuccess ||
            note(cudaMemcpy(c->d_ops_amr, &oa, sizeof(Ops), cudaMemcpyHostToDevice), "adapt ops") != cudaSuccess)
            return IDP_E_CUDA;
    }
    cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
    c->L.amr_transfer(st, u_old, K, u_new, Kn, kind, src, c->d_ops_amr, c->num_sms);
    c->L.amr_zs(st, u_new, Kn, u_old, K, fam, nfam, c->d_ops_amr, c->gamma - 1.0, p->zs_threshold, d_cnt);
    if (note(cudaStreamSynchronize(st), "adapt transfer") != cudaSuccess) return IDP_E_CUDA;
    // element buffers, grown with slack when the mesh outgrows them (their
    // contents are rebuilt or per stage)
    cudaError_t ce = cudaSuccess;
    auto chk = [&](cudaError_t e) { if (ce == cudaSuccess && e != cudaSuccess) ce = e; };
    const long long oK = c->capK, nK = Kn > oK ? std::max<long long>(Kn, oK + oK / 4) : oK;
    if (nK > oK) {
        chk(ensure(&c->d_geom, nK, 0));
        chk(ensure(&c->d_geoc, nK, 0));
        chk(ensure(&c->d_sim, nK, 0));
        chk(ensure(&c->d_fnbr, nK, 0));
        chk(ensure(&c->d_ftype, nK, 0));
        chk(ensure(&c->d_aind, nK, 0));
        chk(ensure(&c->d_part, 4 * nK, 0));
        chk(ensure(&c->d_buf1, 4 * nK * NN, 0));
        chk(ensure(&c->d_buf2, 4 * nK * NN, 0));
        chk(ensure(&c->d_lev, nK, 0));
        chk(ensure(&c->d_ix, nK, 0));
        chk(ensure(&c->d_iy, nK, 0));
        if (c->d_fbuf) {
            const long long F = 2 * nK * NP;
            cudaFree(c->d_fbuf);
            c->d_fbuf = nullptr;
            chk(cudaMalloc(&c->d_fbuf, sizeof(double) * 6 * F + sizeof(float) * F));
        }
        if (c->d_lam) {
            cudaFree(c->d_lam);
            c->d_lam = nullptr;
            chk(cudaMalloc(&c->d_lam, (c->opt.precision ? sizeof(float) : sizeof(double)) * 2 * (size_t)nK * NN));
        }
        if (c->d_emin) chk(ensure(&c->d_emin, nK, 0));
        if (c->d_lofv) chk(ensure(&c->d_lofv, 2 * nK * NN, 0));
        if (c->d_hostbuf) { cudaFree(c->d_hostbuf); c->d_hostbuf = nullptr; }
        if (ce != cudaSuccess) { note(ce, "adapt alloc"); return IDP_E_CUDA; }
        c->capK = nK;
    }
    // the new leaves become the context's
    chk(cudaMemcpyAsync(c->d_lev, nlev, (size_t)Kn, cudaMemcpyDeviceToDevice, st));
    chk(cudaMemcpyAsync(c->d_ix, nix, sizeof(int) * Kn, cudaMemcpyDeviceToDevice, st));
    chk(cudaMemcpyAsync(c->d_iy, niy, sizeof(int) * Kn, cudaMemcpyDeviceToDevice, st));
    chk(cudaMemsetAsync(c->d_aind, 0, sizeof(double) * Kn, st));
    if (c->d_lofv) chk(cudaMemsetAsync(c->d_lofv, 0, sizeof(double) * 2 * (size_t)Kn * NN, st));
    if (ce != cudaSuccess) { note(ce, "adapt copy"); return IDP_E_CUDA; }
    // faces and mortars: the first pass counts the mortars and writes them
    // when the buffers hold them, else they grow and a second pass writes
    BuildIn bin = {c->rmesh, Kn, c->d_lev, c->d_ix, c->d_iy};
    BuildOut bout = {c->d_geom, c->d_geoc, c->d_sim, c->d_fnbr, c->d_ftype, c->d_mlarge, c->d_msmall, c->d_minfo,
                     (int)(c->d_mlarge ? c->capM : 0)};
    int Mn = 0, err = 0;
    if (note(remesh_build_faces(bin, bout, build_s, st, c->num_sms, &Mn, &err), "adapt faces") != cudaSuccess)
        return IDP_E_CUDA;
    if (err) return IDP_E_MESH;
    if (Mn > bout.capM) {
        const long long nM = std::max<long long>(Mn, c->capM + c->capM / 4);
        chk(ensure(&c->d_mlarge, nM, 0));
        chk(ensure(&c->d_msmall, nM, 0));
        chk(ensure(&c->d_minfo, nM, 0));
        c->capM = nM;
        // the slot block is sized for capM mortars
        chk(alloc_slots(c, nM));
        if (ce != cudaSuccess) { note(ce, "adapt alloc"); return IDP_E_CUDA; }
        bout.m_large = c->d_mlarge; bout.m_small = c->d_msmall; bout.m_info = c->d_minfo; bout.capM = (int)nM;
        if (note(remesh_build_faces(bin, bout, build_s, st, c->num_sms, &Mn, &err), "adapt faces") != cudaSuccess)
            return IDP_E_CUDA;
        if (err) return IDP_E_MESH;
    }
    // mortar nodes and the mortar limiting blocks: at most Q nodes per
    // mortar, one foreign entry per node
    const long long need_nodes = std::max<long long>((long long)Mn * Q, 1), need_blocks = (Mn + W - 1) / W + 1;
    if (need_nodes > c->cap_nodes || !c->d_mnnode || !c->d_mnslot) {
        const long long n = std::max<long long>(need_nodes, c->cap_nodes + c->cap_nodes / 4);
        chk(ensure(&c->d_mnnode, n, 0));
        chk(ensure(&c->d_mnslot, n, 0));
        c->cap_nodes = n;
    }
    if (need_blocks > c->cap_blocks || !c->d_mbnode || !c->d_mbfor) {
        const long long n = std::max<long long>(need_blocks, c->cap_blocks + c->cap_blocks / 4);
        chk(ensure(&c->d_mbnode, n, 0));
        chk(ensure(&c->d_mbfor, n, 0));
        c->cap_blocks = n;
    }
    if (need_nodes + 1 > c->cap_foreign || !c->d_mbforeign) {
        const long long n = std::max<long long>(need_nodes + 1, c->cap_foreign + c->cap_foreign / 4);
        chk(ensure(&c->d_mbforeign, n, 0));
        c->cap_foreign = n;
    }
    if (ce != cudaSuccess) { note(ce, "adapt alloc"); return IDP_E_CUDA; }
    NodesIn nin = {NP, Kn, Mn, W, c->d_mlarge, c->d_msmall, c->d_minfo};
    NodesOut nout = {c->d_mnnode, c->d_mnslot, c->d_mbnode, c->d_mbfor, c->d_mbforeign, (int)c->cap_nodes,
                     (int)c->cap_foreign, (int)c->cap_blocks};
    int nmn = 0, nblk = 0, fmax = 0;
    if (note(remesh_build_mortar_nodes(nin, nout, build_s, st, c->num_sms, &nmn, &nblk, &fmax, &err), "adapt nodes") !=
        cudaSuccess)
        return IDP_E_CUDA;
    if (err) return IDP_E_MESH;
    // sizes and the totals of the adapted mesh (host arithmetic as at create)
    c->K = Kn;
    c->M = Mn;
    c->slots.S = Mn * Q;
    c->n_mnodes = nmn;
    c->mb_blocks = nblk;
    c->mb_fmax = fmax;
    c->sim_off = {0, (long long)Kn};
    chk(cudaMemcpyAsync(c->d_off, c->sim_off.data(), sizeof(long long) * 2, cudaMemcpyHostToDevice, st));
    // statistics so far are normalised with the old mesh's totals
    c->stats_mass_prior += c->total_area * (double)(c->n_stages - c->stats_stages_prior);
    c->stats_mlen_prior += c->total_mortar_len * (double)(c->n_stages - c->stats_stages_prior);
    c->stats_stages_prior = c->n_stages;
    double *d_tot = (double *)(d_cnt + 1);
    remesh_totals(c->rmesh, c->d_lev, Kn, c->d_mlarge, c->d_minfo, Mn, d_tot, st);
    MeshDev &md = c->mesh;
    md.K = Kn; md.M = Mn; md.n_mnodes = nmn;
    md.geom = c->d_geom; md.geoc = c->d_geoc; md.sim = c->d_sim; md.fnbr = c->d_fnbr; md.ftype = c->d_ftype;
    md.m_large = c->d_mlarge; md.m_small = c->d_msmall; md.m_info = c->d_minfo;
    md.mn_node = c->d_mnnode; md.mn_slot = c->d_mnslot;
    md.mb_node_off = c->d_mbnode; md.mb_for_off = c->d_mbfor; md.mb_foreign = c->d_mbforeign;
    md.mb_fmax = fmax; md.mb_blocks = nblk;
    // the step graph is captured again for the new mesh
    c->graph_stale = true;
    unsigned long long cnt = 0;
    double tot[2] = {0.0, 0.0};
    if (note(cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st), "adapt count") != cudaSuccess ||
        note(cudaMemcpyAsync(tot, d_tot, sizeof(tot), cudaMemcpyDeviceToHost, st), "adapt totals") != cudaSuccess ||
        note(cudaStreamSynchronize(st), "adapt sync") != cudaSuccess)
        return IDP_E_CUDA;
    c->total_area = tot[0];
    c->total_mortar_len = tot[1];
    if (n_scaled) *n_scaled = (int64_t)cnt;
    return check_cuda(cudaGetLastError());
}

idp_status idp_dgsem_leaves(idp_ctx *c, int8_t *level, int32_t *ix, int32_t *iy) {
    if (!c || !level || !ix || !iy) return IDP_E_ARG;
    const size_t K = (size_t)c->K;
    if (cudaMemcpy(level, c->d_lev, K, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ix, c->d_ix, sizeof(int32_t) * K, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(iy, c->d_iy, sizeof(int32_t) * K, cudaMemcpyDeviceToHost) != cudaSuccess)
        return IDP_E_CUDA;
    return IDP_OK;
}

// Device tables of the context's mesh, copied to host arrays (test support):
// fnbr/ftype [K][4], m_large [M], m_small [M][2], m_info [M], mn_node and
// mn_slot [n_mnodes] (the slot pair as two ints), mb_node_off and mb_for_off
// [mb_blocks + 1], mb_foreign [mb_for_off[mb_blocks]]; sizes[6] = K, M,
// n_mnodes, mb_blocks, foreign count, mb_fmax. With null arrays only sizes.
idp_status idp_dgsem_mesh_tables(idp_ctx *c, int64_t *sizes, int32_t *fnbr, uint8_t *ftype, int32_t *m_large,
                                 int32_t *m_small, int32_t *m_info, int32_t *mn_node, int32_t *mn_slot,
                                 int32_t *mb_node_off, int32_t *mb_for_off, int32_t *mb_foreign) {
    if (!c || !sizes) return IDP_E_ARG;
    int32_t nfore = 0;
    if (c->mb_blocks > 0 &&
        cudaMemcpy(&nfore, c->d_mbfor + c->mb_blocks, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return IDP_E_CUDA;
    sizes[0] = c->K; sizes[1] = c->M; sizes[2] = c->n_mnodes; sizes[3] = c->mb_blocks; sizes[4] = nfore;
    sizes[5] = c->mb_fmax;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *h, const void *d, size_t b) { if (h && b && e == cudaSuccess) e = cudaMemcpy(h, d, b, cudaMemcpyDeviceToHost); };
    cp(fnbr, c->d_fnbr, sizeof(int4) * c->K);
    cp(ftype, c->d_ftype, sizeof(uchar4) * c->K);
    cp(m_large, c->d_mlarge, sizeof(int32_t) * c->M);
    cp(m_small, c->d_msmall, sizeof(int2) * c->M);
    cp(m_info, c->d_minfo, sizeof(int32_t) * c->M);
    cp(mn_node, c->d_mnnode, sizeof(int32_t) * c->n_mnodes);
    cp(mn_slot, c->d_mnslot, sizeof(int2) * c->n_mnodes);
    if (c->mb_blocks > 0) {
        cp(mb_node_off, c->d_mbnode, sizeof(int32_t) * (c->mb_blocks + 1));
        cp(mb_for_off, c->d_mbfor, sizeof(int32_t) * (c->mb_blocks + 1));
        cp(mb_foreign, c->d_mbforeign, sizeof(int32_t) * nfore);
    }
    return e == cudaSuccess ? IDP_OK : IDP_E_CUDA;
}

void idp_dgsem_destroy(idp_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    void *ptrs[] = {c->d_lev, c->d_ix, c->d_iy, c->d_ops_amr, c->d_rm, c->d_fbuf, c->d_lam, c->d_emin, c->d_lofv, c->d_aind, c->d_ops, c->d_geom, c->d_geoc, c->d_sim, c->d_mlarge, c->d_minfo, c->d_mnnode, c->d_fnbr, c->d_ftype,
                    c->d_mbnode, c->d_mbfor, c->d_mbforeign,
                    c->d_msmall, c->d_mnslot, c->d_siminfo, c->d_slot_block, c->d_buf1, c->d_buf2, c->d_hostbuf,
                    c->d_dtmin, c->d_tsim, c->d_dtlast, c->d_status, c->d_stats, c->d_part, c->d_intout, c->d_off};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    for (int k = 0; k < 8; ++k)
        if (c->pev[k]) cudaEventDestroy(c->pev[k]);
    for (int k = 0; k < idp_ctx::kMaxKev; ++k)
        for (int b = 0; b < 2; ++b)
            if (c->kev[k][b]) cudaEventDestroy(c->kev[k][b]);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->st2) cudaStreamDestroy(c->st2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
}

}  // extern "C"
