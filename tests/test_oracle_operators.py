"""Pins of the oracle's reference operators against the paper and closed forms.

- LGL weights: the values printed in App. A (N = 3, 4, 5).
- LGL nodes: roots of P_N' from numpy's Legendre class (an independent routine).
- SBP property Qbar + Qbar^T = Bbar and skew-symmetry of Sbar (Sec. 2.1).
- D exact on monomials of degree <= N (closed form k x^(k-1)).
- Local mortar weights: the tables printed in App. A; their row and column
  sums (Eq. sum_local_omega); a brute-force overlap integral.
- Mortar interpolation exact for polynomials of degree <= N; projection
  conservative and constant-preserving.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden


@pytest.mark.parametrize("row", read_golden("lgl_weights.txt"))
def test_lgl_weights_match_paper(row):
    N, w_paper = int(row[0]), np.array(row[1:])
    _, w = oracle.lgl(N)
    np.testing.assert_allclose(w, w_paper, rtol=0, atol=2e-16)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
def test_lgl_nodes_are_roots_of_dPN(N):
    x, w = oracle.lgl(N)
    assert x[0] == -1.0 and x[-1] == 1.0
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()
    if N > 1:
        assert np.abs(dP(x[1:-1])).max() < 1e-13
    assert abs(w.sum() - 2.0) < 1e-14
    # LGL quadrature is exact for degree 2N-1
    for k in range(2 * N):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs((w * x ** k).sum() - exact) < 1e-14


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7])
def test_sbp_and_skew(N):
    xi, w, D, S, *_ = oracle.operators(N)
    Q = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1)); B[0, 0] = -1; B[N, N] = 1
    np.testing.assert_allclose(Q + Q.T, B, atol=1e-14)
    np.testing.assert_allclose(S, -S.T, atol=2e-14)
    np.testing.assert_allclose(S.sum(axis=1), -np.diag(B), atol=2e-14)
    for k in range(N + 1):
        exact = k * xi ** (k - 1) if k > 0 else 0 * xi
        np.testing.assert_allclose(D @ xi ** k, exact, atol=1e-12)


@pytest.mark.parametrize("N,fname", [(3, "local_weights_N3.txt"), (4, "local_weights_N4.txt"),
                                     (5, "local_weights_N5.txt")])
def test_local_weights_match_paper(N, fname):
    table = np.array(read_golden(fname))
    *_, wt, _, _ = oracle.operators(N)
    np.testing.assert_allclose(wt, table, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_local_weight_sums_and_overlap(N):
    xi, w, _, _, wt, _, _ = oracle.operators(N)
    # Eq. sum_local_omega: rows give the large-side weights, columns the
    # halved small-side weights
    np.testing.assert_allclose(wt.sum(axis=1), w, atol=1e-15)
    np.testing.assert_allclose(wt.sum(axis=0), np.concatenate([w, w]) / 2, atol=1e-15)
    # brute force: integrate psi_i psi_j on a fine midpoint grid
    n = 200000
    s = -1 + (np.arange(n) + 0.5) * (2.0 / n)
    edges = np.concatenate([[-1.0], -1 + np.cumsum(w)])
    big = np.searchsorted(edges, s, side="right") - 1
    hw = np.concatenate([w, w]) / 2
    sedges = np.concatenate([[-1.0], -1 + np.cumsum(hw)])
    small = np.searchsorted(sedges, s, side="right") - 1
    brute = np.zeros_like(wt)
    np.add.at(brute, (big, small), 2.0 / n)
    np.testing.assert_allclose(wt, brute, atol=5e-5)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 7])
@pytest.mark.parametrize("proj", [0, 1])
def test_mortar_interpolation_projection(N, proj):
    xi, w, _, _, _, I, P = oracle.operators(N, proj)
    np_ = N + 1
    s = np.concatenate([(xi - 1) / 2, (xi + 1) / 2])
    for k in range(np_):
        np.testing.assert_allclose(I @ xi ** k, s ** k, atol=1e-13)
    # constants are preserved and the projection conserves the integral
    np.testing.assert_allclose(P.sum(axis=1), np.ones(np_), atol=1e-13)
    np.testing.assert_allclose(w @ P, np.concatenate([w, w]) / 2, atol=1e-14)
    if proj == 1:
        # exact L2 projection reproduces global polynomials of degree <= N
        for k in range(np_):
            np.testing.assert_allclose(P @ s ** k, xi ** k, atol=1e-12)
