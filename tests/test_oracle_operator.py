"""Pins for the oracle's local operator A_L = D^T G D (Eq. 4, Section 3.1) and the
assembled operator QQ^T A_L (Eq. 5), against closed forms, invariants and a
brute-force dense stiffness matrix."""
import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh


def _prob(n, N, jitter, seed=7, dirichlet=None):
    m = BoxMesh(n, n, n, jitter=jitter, seed=seed)
    return so.SemProblem(N, m.vert_xyz, m.elem_verts, dirichlet)


@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_kronecker_sum_on_box_element(N):
    # undeformed cube of side h: A_L = (h/2) (K1 x W x W + W x K1 x W + W x W x K1), K1 = D^T W D
    h = 0.5
    xi, w = so.gll_nodes_weights(N)
    D = so.lagrange_derivative_matrix(xi)
    X = np.zeros((1, 8, 3))
    for v, (a, b, c) in enumerate(so._CORNER):
        X[0, v] = h * np.array([a, b, c], dtype=float)
    G, _ = so.geometric_factors(X, xi, w)
    W = np.diag(w)
    K1 = D.T @ W @ D
    A = (h / 2) * (np.kron(K1, np.kron(W, W)) + np.kron(W, np.kron(K1, W)) + np.kron(W, np.kron(W, K1)))
    Np = N + 1
    cols = []
    for q in range(Np ** 3):
        e = np.zeros(Np ** 3)
        e[q] = 1.0
        cols.append(so.ax_local(e.reshape(1, Np, Np, Np), G, D).ravel())
    np.testing.assert_allclose(np.array(cols).T, A, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("N,jitter", [(2, 0.2), (3, 0.2), (7, 0.15)])
def test_matches_brute_force_dense(N, jitter):
    prob = _prob(2, N, jitter)
    K = so.assembled_stiffness_dense(prob)
    assert np.allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    rng = np.random.default_rng(1)
    n_glob = prob.num.n_glob
    V = rng.standard_normal((n_glob, 4 if N == 7 else n_glob))
    if N != 7:
        V = np.eye(n_glob)
    for col in range(V.shape[1]):
        v = V[:, col]
        w_loc = prob.ax(so.scatter_local(v, prob.glo_num).reshape(prob.shape()), assemble=False)
        got = so.gather_global(w_loc, prob.glo_num, n_glob)
        np.testing.assert_allclose(got, K @ v, atol=1e-11 * np.abs(K).max() * max(1.0, np.abs(v).max()))
    # and the dense K's diagonal is the oracle's Jacobi diagonal
    d_loc = prob.jacobi_diagonal().ravel()
    d_glob = np.zeros(n_glob)
    d_glob[prob.glo_num] = d_loc
    np.testing.assert_allclose(d_glob, np.diag(K), rtol=1e-12)


def test_constants_in_kernel_and_spd():
    prob = _prob(2, 3, 0.2)
    K = so.assembled_stiffness_dense(prob)
    ones = np.ones(prob.num.n_glob)
    assert np.abs(K @ ones).max() < 1e-12 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-12 * ev.max()  # PSD
    # masked operator (Dirichlet rows/cols removed) is SPD
    free = np.ones(prob.num.n_glob, dtype=bool)
    free[prob.glo_num[prob.mask != 0]] = False
    evm = np.linalg.eigvalsh(K[np.ix_(free, free)])
    assert evm.min() > 1e-6 * evm.max()


@pytest.mark.parametrize("N", [3, 7])
def test_assembled_invariants(N):
    prob = _prob(3, N, 0.15)
    rng = np.random.default_rng(2)
    n_glob = prob.num.n_glob
    # A 1 = 0 for the unmasked assembled operator
    one = np.ones(prob.shape())
    a1 = so.dssum(prob.ax_local(one), prob.glo_num)
    scale = np.abs(prob.G).max() * np.abs(prob.D).max() ** 2
    assert np.abs(a1).max() < 1e-12 * scale
    # symmetry u^T A v = v^T A u on continuous fields (weights c count shared nodes once)
    u = so.scatter_local(rng.standard_normal(n_glob), prob.glo_num).reshape(prob.shape())
    v = so.scatter_local(rng.standard_normal(n_glob), prob.glo_num).reshape(prob.shape())
    c = prob.c.reshape(prob.shape())
    unmasked = lambda f: so.dssum(prob.ax_local(f), prob.glo_num)
    uav = so.glsc3(u, unmasked(v), c)
    vau = so.glsc3(v, unmasked(u), c)
    assert abs(uav - vau) < 1e-12 * abs(uav)
    # the masked operator is symmetric on fields that vanish on the Dirichlet nodes
    keep = (prob.mask == 0).reshape(prob.shape())
    um, vm = u * keep, v * keep
    uav = so.glsc3(um, prob.ax(vm), c)
    vau = so.glsc3(vm, prob.ax(um), c)
    assert abs(uav - vau) < 1e-12 * abs(uav)
    assert so.glsc3(um, prob.ax(um), c) > 0


@pytest.mark.parametrize("N", [3, 5, 7])
def test_linear_patch_test(N):
    # x is in the discrete space and harmonic: the masked assembled A x vanishes
    # (GLL quadrature is exact for these integrands when N >= 3).
    prob = _prob(3, N, 0.15)
    x = prob.coords()
    for comp in range(3):
        r = prob.ax(x[..., comp])
        assert np.abs(r).max() < 1e-12 * np.abs(prob.ax_local(x[..., comp])).max()
