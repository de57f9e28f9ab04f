"""Pins of the oracle's point fluxes against textbook facts.

- Euler flux written out here from the conservation law (Sec. 2, Eq.
  conservationlaw with the ideal-gas pressure) as the consistency target.
- Ranocha's volume flux (R1): consistency, symmetry, exact Tadmor entropy
  conservation (w_R - w_L) . f* = psi_R - psi_L with the textbook entropy
  variables, and the kinetic-energy-preserving momentum form.
- Logarithmic mean (R2): against a 50-digit mpmath evaluation.
- LLF flux: consistency and conservation under swapping sides.
- R8 admissible-factor solve: maximal and feasible, by brute force.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle

G = 1.4


def euler_flux(u, n, g=G):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (g - 1) * (E - 0.5 * rho * (v1 * v1 + v2 * v2))
    vn = v1 * n[0] + v2 * n[1]
    return np.array([rho * vn, m1 * vn + p * n[0], m2 * vn + p * n[1], (E + p) * vn])


def rand_state(rng, g=G):
    rho = rng.uniform(0.1, 10)
    v = rng.uniform(-2, 2, 2)
    p = rng.uniform(0.1, 10)
    return np.array([rho, rho * v[0], rho * v[1], p / (g - 1) + 0.5 * rho * (v @ v)])


def entropy_vars(u, g=G):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (g - 1) * (E - 0.5 * rho * (v1 * v1 + v2 * v2))
    s = math.log(p) - g * math.log(rho)
    return np.array([(g - s) / (g - 1) - rho * (v1 * v1 + v2 * v2) / (2 * p), rho * v1 / p, rho * v2 / p, -rho / p])


def test_logmean_high_precision():
    rng = np.random.default_rng(1)
    mpmath.mp.dps = 50
    worst = 0.0
    for k in range(4000):
        a = 10 ** rng.uniform(-8, 3)
        b = a * (1 + 10 ** rng.uniform(-16, 1) * rng.choice([-1, 1])) if k % 2 else 10 ** rng.uniform(-8, 3)
        if b <= 0:
            continue
        A, B = mpmath.mpf(a), mpmath.mpf(b)
        ref = A if A == B else (A - B) / (mpmath.log(A) - mpmath.log(B))
        worst = max(worst, abs(float((mpmath.mpf(oracle.logmean(a, b)) - ref) / ref)))
    assert worst < 1e-14, worst
    assert oracle.logmean(2.0, 2.0) == 2.0


@pytest.mark.parametrize("d", [0, 1])
def test_ranocha_consistent_symmetric(d):
    rng = np.random.default_rng(2 + d)
    n = (1.0, 0.0) if d == 0 else (0.0, 1.0)
    for _ in range(200):
        a, b = rand_state(rng), rand_state(rng)
        np.testing.assert_allclose(oracle.ranocha(a, a, d), euler_flux(a, n), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(oracle.ranocha(a, b, d), oracle.ranocha(b, a, d), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1])
def test_ranocha_entropy_conservative(d):
    rng = np.random.default_rng(5 + d)
    for _ in range(500):
        a, b = rand_state(rng), rand_state(rng)
        f = oracle.ranocha(a, b, d)
        psi = lambda u: u[1 + d]   # rho v_n
        lhs = (entropy_vars(b) - entropy_vars(a)) @ f
        rhs = psi(b) - psi(a)
        scale = np.abs(entropy_vars(b) - entropy_vars(a)) @ np.abs(f) + abs(psi(a)) + abs(psi(b))
        assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


def test_ranocha_kep_momentum():
    rng = np.random.default_rng(9)
    for _ in range(100):
        a, b = rand_state(rng), rand_state(rng)
        f = oracle.ranocha(a, b, 0)
        pa = (G - 1) * (a[3] - 0.5 * (a[1] ** 2 + a[2] ** 2) / a[0])
        pb = (G - 1) * (b[3] - 0.5 * (b[1] ** 2 + b[2] ** 2) / b[0])
        v1m = 0.5 * (a[1] / a[0] + b[1] / b[0])
        v2m = 0.5 * (a[2] / a[0] + b[2] / b[0])
        np.testing.assert_allclose(f[1], f[0] * v1m + 0.5 * (pa + pb), rtol=1e-13)
        np.testing.assert_allclose(f[2], f[0] * v2m, rtol=1e-13, atol=1e-14)


def test_llf_consistent_conservative():
    rng = np.random.default_rng(3)
    for _ in range(200):
        a, b = rand_state(rng), rand_state(rng)
        th = rng.uniform(0, 2 * np.pi)
        n = (math.cos(th), math.sin(th))
        np.testing.assert_allclose(oracle.llf(a, a, n), euler_flux(a, n), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(oracle.llf(a, b, n), -oracle.llf(b, a, (-n[0], -n[1])), rtol=1e-13, atol=1e-13)


def _p(u):
    return (G - 1) * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / u[0])


def test_theta_is_maximal_and_feasible():
    rng = np.random.default_rng(11)
    grid = np.linspace(0, 1, 100001)
    n_root = 0
    for _ in range(300):
        u0 = rand_state(rng)
        a = rng.normal(0, 1, 4) * np.array([u0[0], abs(u0[1]) + 1, abs(u0[2]) + 1, u0[3]]) * rng.uniform(0.5, 5)
        pmin = 0.1 * _p(u0)
        hi = rng.uniform(0.2, 1.0)
        th = oracle.theta(u0, a, pmin, hi)
        assert 0 <= th <= hi
        v = u0 + th * a
        assert v[0] > 0 and _p(v) >= pmin * (1 - 1e-12)
        # brute force: every grid theta up to th is feasible, and if th < hi
        # the first grid point beyond th + 1e-9 relative is infeasible
        ts = grid[grid <= th] if th > 0 else np.array([0.0])
        V = u0[None, :] + ts[:, None] * a[None, :]
        P = (G - 1) * (V[:, 3] - 0.5 * (V[:, 1] ** 2 + V[:, 2] ** 2) / V[:, 0])
        assert (V[:, 0] > 0).all() and (P >= pmin * (1 - 1e-12)).all()
        if th < hi:
            n_root += 1
            t2 = min(hi, th * (1 + 1e-8) + 1e-12)
            w = u0 + t2 * a
            assert not (w[0] > 0 and _p(w) >= pmin), (th, t2)
    assert n_root > 30
