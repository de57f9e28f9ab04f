// idp_variants.cuh -- device functions of the limiter and flux variants
// (arXiv 2607.06045): Chandrashekar's volume flux (the paper's astrophysical
// jet) and the entropy bound of local limiting (Eq. Bounds_Barstates, right
// part). Only the extended element kernel and the mortar kernels use them.
#pragma once

#include "idp_device.cuh"

namespace idp {

// Chandrashekar's entropy-conserving, kinetic-energy-preserving two-point
// flux along axis d (reading R23; the paper's astrophysical jet), with
// beta = rho / p: f_rho = {rho}_ln {v_n}, f_m = f_rho {v} + ({rho}/{beta}) n,
// f_E = f_rho (1 / ((gamma-1) {beta}_ln) - {|v|^2} / 2) + f_m . {v}.
template <typename FT>
__device__ __forceinline__ void chandrashekar(const Prim<FT> &a, const Prim<FT> &b, int d, FT ginv1, FT f[4]) {
    FT rho_ln, ibeta;
    log_means<FT>(a, b, rho_ln, ibeta);
    FT v1m = FT(0.5) * (a.v1 + b.v1), v2m = FT(0.5) * (a.v2 + b.v2);
    FT fr = rho_ln * (d == 0 ? v1m : v2m);
    FT ph;
    if constexpr (sizeof(FT) == 8) ph = (a.rho + b.rho) * fast_rcp(a.beta + b.beta);
    else ph = (a.rho + b.rho) / (a.beta + b.beta);
    FT v2a = FT(0.5) * ((a.v1 * a.v1 + a.v2 * a.v2) + (b.v1 * b.v1 + b.v2 * b.v2));
    f[0] = fr;
    f[1] = fr * v1m + (d == 0 ? ph : FT(0));
    f[2] = fr * v2m + (d == 1 ? ph : FT(0));
    f[3] = fr * (ibeta * ginv1 - FT(0.5) * v2a) + f[1] * v1m + f[2] * v2m;
}

// x > 0, finite and normal (the domain of fast_log)
__device__ __forceinline__ bool dnormpos(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0x0010000000000000LL && b < 0x7ff0000000000000LL;
}

// s = ln p - gamma ln rho of a conserved state (FP64); -inf where rho or p is
// not positive (no entropy bound from that state).
__device__ __forceinline__ double entropy_s(const Gas &G, double r, double m1, double m2, double E) {
    if (!dnormpos(r)) return -INFINITY;
    const double ri = fast_rcp(r);
    const double p = G.gm1 * (E - 0.5 * (m1 * (m1 * ri) + m2 * (m2 * ri)));
    if (!dnormpos(p)) return -INFINITY;
    return fast_log(p, G.lg) - G.g * fast_log(r, G.lg);
}

// s of the bar state ubar = (ua + ub)/2 - sgn (fb - fa) i2l (Sec. 2.2) of a
// graph edge along axis d, from both states and their physical fluxes along
// that axis; in the flux type (FP32 in the FP32 form, whose bounds only need
// to stay below the low-order state's, which is in FP64).
template <typename FT>
__device__ __forceinline__ double bar_entropy(const Gas &G, const FT ua[4], const FT fa[4], const FT ub[4],
                                              const FT fb[4], FT sgn_i2l) {
    FT q[4];
    for (int v = 0; v < 4; ++v) q[v] = FT(0.5) * (ua[v] + ub[v]) - sgn_i2l * (fb[v] - fa[v]);
    if constexpr (sizeof(FT) == 8) {
        return entropy_s(G, q[0], q[1], q[2], q[3]);
    } else {
        if (!(q[0] > 0.0f)) return -INFINITY;
        const float p = G.gm1f * (q[3] - 0.5f * (q[1] * q[1] + q[2] * q[2]) / q[0]);
        if (!(p > 0.0f) || !(p < 3e38f)) return -INFINITY;
        return (double)(logf(p) - G.gf * logf(q[0]));
    }
}

// Psi(v) = rho e(v) - K rho(v)^gamma, K = exp(lnK), with
// rho e = E - |m|^2 / (2 rho): Psi >= 0 iff eta(v) >= K (rho > 0). Psi is
// concave in v (rho e is concave and K rho^gamma convex). Also returns
// dPsi/dtheta along a.
__device__ __forceinline__ double entropy_psi(const Gas &G, const double v[4], const double a[4], double lnK,
                                              double &dpsi) {
    const double ri = fast_rcp(v[0]);
    const double v1 = v[1] * ri, v2 = v[2] * ri;
    const double re = v[3] - 0.5 * (v[1] * v1 + v[2] * v2);
    const double kr = exp(lnK + G.g * fast_log(v[0], G.lg));
    dpsi = a[3] - (v1 * a[1] + v2 * a[2]) + 0.5 * (v1 * v1 + v2 * v2) * a[0] - G.g * (kr * ri) * a[0];
    return re - kr;
}

// Reading R21: largest theta in [0, hi] with eta(u0 + theta a) >= K, with a
// margin: the target is Psi >= delta, delta = 1e-14 (|E_0| + K rho_0^gamma),
// well above the rounding of Psi, so that the decision and the root do not
// depend on it. {Psi >= delta} is convex, so the admissible thetas are an
// interval [0, theta*]; the caller guarantees rho > 0 on [0, hi] (hi is the
// pressure factor). theta* by Newton's method on Psi - delta from hi: Psi is
// concave, so the iterates decrease monotonically to the root. Verified
// against Psi >= 0, halved at most four times (a safeguard).
__device__ __forceinline__ double theta_entropy(const Gas &G, const double u0[4], const double a[4], double lnK,
                                                double hi) {
    if (!dpos(hi) || !dnormpos(u0[0])) return 0.0;
    double v[4], dp;
    // the margin is a scale, not a decision: K rho_0^gamma in FP32 (FP64 only
    // outside the FP32 range)
    float kr0 = expf(d2f(lnK) + G.gf * logf(d2f(u0[0])));
    const double krd = (kr0 < 3e38f) ? f2d(kr0) : exp(lnK + G.g * fast_log(u0[0], G.lg));
    const double delta = 1e-14 * (fabs(u0[3]) + krd);
    for (int k = 0; k < 4; ++k) v[k] = u0[k] + hi * a[k];
    if (dnormpos(v[0]) && !dlt(entropy_psi(G, v, a, lnK, dp), delta)) return hi;
    if (dlt(entropy_psi(G, u0, a, lnK, dp), delta)) return 0.0;
    double th = hi;
    for (int it = 0; it < 40; ++it) {
        for (int k = 0; k < 4; ++k) v[k] = u0[k] + th * a[k];
        if (!dnormpos(v[0])) { th *= 0.5; continue; }
        const double ps = entropy_psi(G, v, a, lnK, dp) - delta;
        if (!dneg(ps) || !dneg(dp)) break;   // at the target by rounding, or no descent
        const double nt = th - ps / dp;
        if (!(nt < th)) break;
        if (!dpos(nt)) { th *= 0.5; continue; }
        const bool done = th - nt <= 1e-15 * th;
        th = nt;
        if (done) break;
    }
    for (int it = 0; it < 4; ++it) {
        for (int k = 0; k < 4; ++k) v[k] = u0[k] + th * a[k];
        if (dnormpos(v[0]) && !dneg(entropy_psi(G, v, a, lnK, dp))) return th;
        th *= 0.5;
    }
    return 0.0;
}

}  // namespace idp
