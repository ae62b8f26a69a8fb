"""Pins for the oracle's trilinear geometry, G^e and B (Eq. 4; Section 4.2: six
geometric factors per point; Section 5.1: linearly deformed hexahedra)."""
import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh


def _unit_cube_vertices(h=1.0, origin=(0.0, 0.0, 0.0)):
    X = np.zeros((1, 8, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                X[0, a + 2 * b + 4 * c] = np.array(origin) + h * np.array([a, b, c], dtype=float)
    return X


@pytest.mark.parametrize("N", [1, 3, 7])
def test_undeformed_box(N):
    h = 0.37
    xi, w = so.gll_nodes_weights(N)
    X = _unit_cube_vertices(h, (0.3, -1.2, 2.0))
    J = so.jacobian(X, xi)
    np.testing.assert_allclose(J, np.broadcast_to((h / 2) * np.eye(3), J.shape), atol=1e-15)
    G, B = so.geometric_factors(X, xi, w)
    W3 = so.weights3(w)
    for m, diag in enumerate([1, 0, 0, 1, 0, 1]):
        np.testing.assert_allclose(G[0, m], diag * W3 * (h / 2), atol=1e-15)
    np.testing.assert_allclose(B[0], W3 * (h / 2) ** 3, rtol=1e-14)


def _random_hex(rng, jitter=0.2):
    X = _unit_cube_vertices(1.0)
    return X + jitter * (rng.random(X.shape) - 0.5)


def test_translation_rotation_scaling():
    rng = np.random.default_rng(3)
    xi, w = so.gll_nodes_weights(5)
    X = _random_hex(rng)
    G0, B0 = so.geometric_factors(X, xi, w)
    G1, B1 = so.geometric_factors(X + np.array([5.0, -3.0, 0.25]), xi, w)
    np.testing.assert_allclose(G1, G0, rtol=1e-12, atol=1e-14)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    G2, B2 = so.geometric_factors(X @ Q.T, xi, w)
    np.testing.assert_allclose(G2, G0, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(B2, B0, rtol=1e-12)
    s = 2.5  # stiffness of a 3D element scales linearly with its size, mass with size^3
    G3, B3 = so.geometric_factors(s * X, xi, w)
    np.testing.assert_allclose(G3, s * G0, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(B3, s ** 3 * B0, rtol=1e-12)


def test_affine_element_constant_jacobian():
    rng = np.random.default_rng(5)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    X = _unit_cube_vertices(1.0) @ A.T  # parallelepiped x = A * corner
    xi, w = so.gll_nodes_weights(4)
    J = so.jacobian(X, xi)
    np.testing.assert_allclose(J, np.broadcast_to(A / 2, J.shape), atol=1e-14)
    x = so.coordinates(X, xi)
    for v, (a, b, c) in enumerate(so._CORNER):
        np.testing.assert_allclose(x[0, c * 4, b * 4, a * 4], X[0, v], atol=1e-15)


@pytest.mark.parametrize("N", [2, 5, 7])
def test_mass_sums_to_volume(N):
    # det J of a trilinear map has degree <= 2 in each reference variable, so GLL
    # quadrature integrates it exactly for N >= 2: the masses sum to the volume.
    m = BoxMesh(3, 4, 2, jitter=0.15, seed=11)
    xi, w = so.gll_nodes_weights(N)
    _, B = so.geometric_factors(so.element_vertices(m.vert_xyz, m.elem_verts), xi, w)
    assert abs(B.sum() - 1.0) < 1e-13


def test_inverted_element_raises():
    xi, w = so.gll_nodes_weights(3)
    X = _unit_cube_vertices(1.0)
    X[0, [0, 1]] = X[0, [1, 0]]  # swap two vertices: the map folds over
    with pytest.raises(so.MeshError):
        so.geometric_factors(X, xi, w)
