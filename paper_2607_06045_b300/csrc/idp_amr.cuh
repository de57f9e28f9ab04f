// idp_amr.cuh -- device kernels of one adaptive-mesh-refinement step
// (arXiv 2607.06045, Sec. 2.4): element indicators, the solution transfer to
// the adapted mesh (interpolation for refinement, exact L2 projection for
// coarsening) and the Zhang-Shu scaling of the transferred families.
#pragma once

#include "idp_device.cuh"

namespace idp {

// Hennemann et al.'s modal energy indicator of nodal values v[j][i] (the
// same definition as the combined limiting's): modal coefficients in the
// orthonormal Legendre basis, energy fractions of the two highest mode
// shells, logistic map, snapped to 0 or 1 within 1e-3.
template <int NP>
__device__ __forceinline__ double hennemann_indicator(const double *v, const Ops *ops) {
    constexpr int N = NP - 1;
    double T[NP][NP];   // T[k][j] = sum_i Vinv[k][i] v[j][i]
    for (int k = 0; k < NP; ++k)
        for (int j = 0; j < NP; ++j) {
            double acc = 0.0;
            for (int i = 0; i < NP; ++i) acc += ops->Vinv[k][i] * v[j * NP + i];
            T[k][j] = acc;
        }
    double en[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < NP; ++k)
        for (int l = 0; l < NP; ++l) {
            double m = 0.0;
            for (int j = 0; j < NP; ++j) m += T[k][j] * ops->Vinv[l][j];
            const int top = k > l ? k : l;
            en[top == N ? 1 : (top == N - 1 ? 2 : 0)] += m * m;
        }
    double E = 0.0;
    const double t0 = en[0] + en[1] + en[2], t1 = en[0] + en[2];
    if (t0 > 0.0) E = en[1] / t0;
    if (t1 > 0.0 && en[2] / t1 > E) E = en[2] / t1;
    const double Tt = ops->ind_T, sh = ops->ind_s;
    double a = 1.0 / (1.0 + exp(-sh / Tt * (E - Tt)));
    if (a < 1e-3) a = 0.0;
    if (a > 1.0 - 1e-3) a = 1.0;
    return a;
}

// Loehner-type estimator (reading R27): the largest second-difference ratio
// over consecutive nodes (a, b, c) of every row and column.
template <int NP>
__device__ __forceinline__ double lohner_indicator(const double *v, double f) {
    double best = 0.0;
    for (int d = 0; d < 2; ++d)
        for (int r = 0; r < NP; ++r)
            for (int k = 1; k < NP - 1; ++k) {
                const double a = d == 0 ? v[r * NP + k - 1] : v[(k - 1) * NP + r];
                const double b = d == 0 ? v[r * NP + k] : v[k * NP + r];
                const double c = d == 0 ? v[r * NP + k + 1] : v[(k + 1) * NP + r];
                const double num = fabs(a - 2.0 * b + c);
                const double den = fabs(c - b) + fabs(b - a) + f * (fabs(a) + 2.0 * fabs(b) + fabs(c));
                const double q = den > 0.0 ? num / den : 0.0;
                best = q > best ? q : best;
            }
    return best;
}

// One thread per element: kind 0 Hennemann, 1 Loehner, 2 the larger; var 0
// density, 1 pressure.
template <int NP>
__global__ void __launch_bounds__(128) k_amr_indicator(const double *__restrict__ u, int K, const Ops *ops, double gm1,
                                                       int kind, int var, double filt, double *ind) {
    constexpr int NN = NP * NP;
    const size_t KN = (size_t)K * NN;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        double v[NN];
        for (int n = 0; n < NN; ++n) {
            const size_t g = (size_t)e * NN + n;
            const double r = u[g];
            v[n] = var == 0 ? r : gm1 * (u[3 * KN + g] - 0.5 * (u[KN + g] * u[KN + g] + u[2 * KN + g] * u[2 * KN + g]) / r);
        }
        double a = 0.0;
        if (kind != 1) a = hennemann_indicator<NP>(v, ops);
        if (kind != 0) { const double b = lohner_indicator<NP>(v, filt); a = b > a ? b : a; }
        ind[e] = a;
    }
}

// One thread per node of the adapted mesh: kind 0 copy of src.x; kind 1
// child src.y (c = cx + 2 cy) of the old parent src.x by tensor
// interpolation; kind 2 the exact L2 projection of the four old children
// src.x..w (child order) onto the parent (tensor product of the 1D
// projections).
template <int NP>
__global__ void __launch_bounds__(256) k_amr_transfer(const double *__restrict__ uo, int Ko, double *__restrict__ un,
                                                      int Kn, const int *__restrict__ kind, const int4 *__restrict__ src,
                                                      const Ops *ops) {
    constexpr int NN = NP * NP;
    const size_t KNo = (size_t)Ko * NN, KNn = (size_t)Kn * NN;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < KNn; k += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(k / NN), n = (int)(k - (size_t)e * NN), i = n % NP, j = n / NP;
        const int kd = kind[e];
        const int4 s = src[e];
        for (int v = 0; v < 4; ++v) {
            double acc = 0.0;
            if (kd == 0) {
                acc = uo[v * KNo + (size_t)s.x * NN + n];
            } else if (kd == 1) {
                const int cx = s.y & 1, cy = s.y >> 1;
                const double *p = uo + v * KNo + (size_t)s.x * NN;
                for (int l = 0; l < NP; ++l)
                    for (int kk = 0; kk < NP; ++kk)
                        acc += ops->I[cx * NP + i][kk] * ops->I[cy * NP + j][l] * p[l * NP + kk];
            } else {
                const int ch[4] = {s.x, s.y, s.z, s.w};
                for (int c = 0; c < 4; ++c) {
                    const int cx = c & 1, cy = c >> 1;
                    const double *q = uo + v * KNo + (size_t)ch[c] * NN;
                    for (int jj = 0; jj < NP; ++jj)
                        for (int ii = 0; ii < NP; ++ii)
                            acc += ops->P[i][cx * NP + ii] * ops->P[j][cy * NP + jj] * q[jj * NP + ii];
                }
            }
            un[v * KNn + k] = acc;
        }
    }
}

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
// minimum of non-negative doubles (their bits order like their values)
__device__ __forceinline__ double warp_min_nn(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long c = __shfl_xor_sync(0xffffffffu, b, o);
        b = c < b ? c : b;
    }
    return __longlong_as_double((long long)b);
}

// Zhang-Shu scaling (reading R26), one warp per family fam = (first new
// element, element count, reference: 0 an old element / 1 a new element,
// its index): reference state = the LGL mean of that element; theta_rho from
// the nodes with rho < eps, then theta_p (the largest factor keeping
// p >= eps, R8's solve) on the scaled states; one factor per family.
template <int NP>
__global__ void __launch_bounds__(128) k_amr_zs(double *__restrict__ un, int Kn, const double *__restrict__ uo, int Ko,
                                                const int4 *__restrict__ fam, int nfam, const Ops *ops, double gm1,
                                                double eps, unsigned long long *nscaled) {
    constexpr int NN = NP * NP;
    const size_t KNo = (size_t)Ko * NN, KNn = (size_t)Kn * NN;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (f >= nfam) return;   // uniform per warp
    const int4 F = fam[f];
    const double *rs = F.z == 0 ? uo : un;
    const size_t rK = F.z == 0 ? KNo : KNn;
    double ref[4];
    for (int v = 0; v < 4; ++v) {
        double acc = 0.0;
        for (int n = lane; n < NN; n += 32)
            acc += ops->w[n / NP] * ops->w[n % NP] * rs[v * rK + (size_t)F.w * NN + n];
        ref[v] = warp_sum(acc) * 0.25;
    }
    const double pref = gm1 * (ref[3] - 0.5 * (ref[1] * ref[1] + ref[2] * ref[2]) / ref[0]);
    if (!(ref[0] > eps) || !(pref > eps)) return;   // no admissible reference: left alone
    const int cnt = F.y * NN;
    double th1 = 1.0;
    for (int q = lane; q < cnt; q += 32) {
        const double r = un[(size_t)F.x * NN + q];
        if (r < eps) { const double t = (ref[0] - eps) / (ref[0] - r); th1 = t < th1 ? t : th1; }
    }
    th1 = warp_min_nn(th1);
    if (th1 < 1.0)
        for (int q = lane; q < cnt; q += 32)
            for (int v = 0; v < 4; ++v) {
                double &x = un[v * KNn + (size_t)F.x * NN + q];
                x = ref[v] + th1 * (x - ref[v]);
            }
    __syncwarp();
    const double c0 = g_zero(gm1, ref, eps);
    double th2 = 1.0;
    for (int q = lane; q < cnt; q += 32) {
        double a[4];
        for (int v = 0; v < 4; ++v) a[v] = un[v * KNn + (size_t)F.x * NN + q] - ref[v];
        const double t = theta_max(gm1, ref, a, gm1, eps, c0, 1.0);
        th2 = t < th2 ? t : th2;
    }
    th2 = warp_min_nn(th2);
    if (th2 < 1.0)
        for (int q = lane; q < cnt; q += 32)
            for (int v = 0; v < 4; ++v) {
                double &x = un[v * KNn + (size_t)F.x * NN + q];
                x = ref[v] + th2 * (x - ref[v]);
            }
    if (lane == 0 && th1 * th2 < 1.0) atomicAdd(nscaled, 1ull);
}

}  // namespace idp
