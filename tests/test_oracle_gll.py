"""Pins for the oracle's GLL nodes, weights and derivative matrix (Section 3, Eq. 3).

Values come from textbook closed forms and from quadrature exactness, not
from the oracle itself.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import sem_oracle as so

S5, S37 = 1 / math.sqrt(5), math.sqrt(3 / 7)
CLOSED = {
    1: ([-1, 1], [1, 1]),
    2: ([-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1, -S5, S5, 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1, -S37, 0, S37, 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("N", sorted(CLOSED))
def test_closed_forms(N):
    xi, w = so.gll_nodes_weights(N)
    np.testing.assert_allclose(xi, CLOSED[N][0], atol=1e-15)
    np.testing.assert_allclose(w, CLOSED[N][1], rtol=1e-14)


@pytest.mark.parametrize("N", range(1, 16))
def test_quadrature_exactness(N):
    xi, w = so.gll_nodes_weights(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):  # exact through degree 2N-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, xi ** k) - exact) < 1e-13, k
    # and not for degree 2N (GLL loses exactness there)
    assert abs(np.dot(w, xi ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-9


@pytest.mark.parametrize("N", range(1, 16))
def test_symmetry_and_roots(N):
    xi, w = so.gll_nodes_weights(N)
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-15)
    np.testing.assert_allclose(w, w[::-1], rtol=1e-14)
    assert np.all(np.diff(xi) > 0)
    if N >= 2:
        # interior nodes are the roots of L_N' (numpy's Legendre series as the check)
        dcoef = npleg.legder([0] * N + [1])
        np.testing.assert_allclose(npleg.legval(xi[1:-1], dcoef), 0, atol=1e-11 * N * N)


@pytest.mark.parametrize("N", range(1, 14))
def test_derivative_matrix(N):
    xi, _ = so.gll_nodes_weights(N)
    D = so.lagrange_derivative_matrix(xi)
    np.testing.assert_allclose(D.sum(axis=1), 0, atol=1e-12 * N * N)
    for k in range(0, N + 1):  # D xi^k = k xi^(k-1) for polynomials of degree <= N
        want = k * xi ** (k - 1) if k else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** k, want, atol=2e-13 * N ** 3)
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-12 * N * N
    assert abs(D[N, N] - N * (N + 1) / 4) < 1e-12 * N * N
    np.testing.assert_allclose(np.diag(D)[1:N], 0, atol=1e-12 * N * N)
    # closed form off the diagonal: L_N(xi_i) / (L_N(xi_j) (xi_i - xi_j))
    L = npleg.legval(xi, [0] * N + [1])
    for i in range(N + 1):
        for j in range(N + 1):
            if i != j:
                assert abs(D[i, j] - L[i] / (L[j] * (xi[i] - xi[j]))) < 1e-11 * N * N
