"""Pins for the oracle's gather-scatter (Eq. 5, Section 4.3), weighted inner
product and Jacobi-preconditioned CG (Algorithm 1), and the right-hand side."""
import math

import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh


def _prob(n, N, jitter=0.1, seed=0):
    m = BoxMesh(n, n, n, jitter=jitter, seed=seed)
    return so.SemProblem(N, m.vert_xyz, m.elem_verts)


def test_dssum_is_qqt():
    prob = _prob(2, 3, 0.2)
    rng = np.random.default_rng(0)
    w = rng.standard_normal(prob.n)
    n_glob = prob.num.n_glob
    Q = np.zeros((prob.n, n_glob))
    Q[np.arange(prob.n), prob.glo_num] = 1.0
    np.testing.assert_allclose(so.dssum(w, prob.glo_num), Q @ (Q.T @ w), rtol=1e-14, atol=1e-14)
    masked = so.dssum(w, prob.glo_num, prob.mask)
    assert np.all(masked[prob.mask != 0] == 0)
    np.testing.assert_array_equal(masked[prob.mask == 0], so.dssum(w, prob.glo_num)[prob.mask == 0])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_dssum_left_to_right_order(dtype):
    # three copies of one global node: (big + 1) - big depends on the order
    glo = np.array([0, 1, 0, 0, 1])
    big = dtype(2.0 ** 60)
    w = np.array([big, 3, 1, -big, 4], dtype=dtype)
    out = so.dssum(w, glo, dtype=dtype)
    want0 = (big + dtype(1)) + (-big)  # ascending local index: w0 + w2 + w3
    assert want0 == 0 and out.dtype == dtype
    np.testing.assert_array_equal(out, np.array([want0, 7, want0, want0, 7], dtype=dtype))


def test_glsc3_counts_shared_nodes_once():
    prob = _prob(3, 4, 0.1)
    rng = np.random.default_rng(1)
    a_g, b_g = rng.standard_normal((2, prob.num.n_glob))
    a, b = so.scatter_local(a_g, prob.glo_num), so.scatter_local(b_g, prob.glo_num)
    assert abs(so.glsc3(a, b, prob.c) - np.dot(a_g, b_g)) < 1e-11 * np.abs(a_g * b_g).sum()


def test_cg_matches_dense_solve():
    prob = _prob(2, 3, 0.2)
    K = so.assembled_stiffness_dense(prob)
    free = np.ones(prob.num.n_glob, dtype=bool)
    free[prob.glo_num[prob.mask != 0]] = False
    b = prob.rhs()
    b_glob = np.zeros(prob.num.n_glob)
    b_glob[prob.glo_num] = b.ravel()
    x_glob = np.zeros(prob.num.n_glob)
    x_glob[free] = np.linalg.solve(K[np.ix_(free, free)], b_glob[free])
    for precond in (False, True):
        res = so.pcg(prob, b, rtol=1e-13, precond=precond)
        assert res.converged
        np.testing.assert_allclose(res.x.ravel(), x_glob[prob.glo_num], atol=1e-11 * np.abs(x_glob).max())


def test_cg_iterations_monotone_in_rtol():
    prob = _prob(3, 5, 0.15)
    b = prob.rhs()
    its = [so.pcg(prob, b, rtol=t).iterations for t in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10)]
    assert all(x <= y for x, y in zip(its, its[1:])) and its[0] < its[-1]
    # Jacobi preconditioning: fewer iterations than plain CG at the same tolerance
    assert so.pcg(prob, b, rtol=1e-8).iterations <= so.pcg(prob, b, rtol=1e-8, precond=False).iterations


def test_rhs_integrates_f():
    # sum of B f over all local points is the quadrature of f = 3 pi^2 sin sin sin
    # over the unit cube: 3 pi^2 (2/pi)^3 = 24/pi (spectrally accurate at N = 7).
    prob = _prob(4, 7, 0.1)
    x = prob.coords()
    f = 3 * math.pi ** 2 * np.prod(np.sin(math.pi * x), axis=-1)
    assert abs((prob.B * f).sum() - 24 / math.pi) < 1e-8


@pytest.mark.slow
def test_spectral_convergence():
    # max nodal error to sin(pi x) sin(pi y) sin(pi z) falls geometrically in N
    errs = []
    for N in range(2, 9):
        prob = _prob(2, N, 0.1, seed=0)
        res = so.pcg(prob, prob.rhs(), rtol=1e-13)
        errs.append(np.abs(res.x - prob.exact_solution()).max())
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1]), errs
    rate = np.exp(np.polyfit(np.arange(2, 9), np.log(errs), 1)[0])
    assert rate < 0.25, (rate, errs)
    assert errs[-1] < 1e-6
