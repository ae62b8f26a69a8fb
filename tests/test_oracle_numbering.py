"""Pins for the oracle's global numbering, multiplicity and Dirichlet mask
(Section 3.1: Q and the local representation; Section 4.3, Eq. 9: number of
element-boundary points; Algorithm 1: the weight vector c)."""
import itertools
import os

import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out[key] = np.array([int(v) for v in vals], dtype=np.int64)
    return out


def test_hand_derived_2x1x1():
    g = _read_golden("numbering_2x1x1_N2.txt")
    m = BoxMesh(2, 1, 1)
    num = so.number_nodes(2, m.elem_verts)
    np.testing.assert_array_equal(num.glo_num, g["glo_num"])
    assert num.n_glob == 45
    unmasked = np.unique(num.glo_num[num.mask == 0])
    np.testing.assert_array_equal(unmasked, g["unmasked"])


@pytest.mark.parametrize("n,N", [(1, 1), (2, 3), (3, 2), (4, 7)])
def test_box_counts(n, N):
    m = BoxMesh(n, n, n, jitter=0.1, seed=0)
    num = so.number_nodes(N, m.elem_verts)
    E, Np = n ** 3, N + 1
    assert num.n_glob == (n * N + 1) ** 3
    assert len(np.unique(num.glo_num[num.mask == 0])) == max(n * N - 1, 0) ** 3
    # Eq. 9: local points with some index in {0, N} number E((N+1)^3 - (N-1)^3)
    loc = num.glo_num.reshape(E, Np, Np, Np)
    k, j, i = np.meshgrid(np.arange(Np), np.arange(Np), np.arange(Np), indexing="ij")
    on_bdry = (i % N == 0) | (j % N == 0) | (k % N == 0)
    assert int(on_bdry.sum()) * E == E * (Np ** 3 - (N - 1) ** 3)
    # element-interior points are never shared
    assert np.all(num.mult[loc[:, ~on_bdry]] == 1)
    # multiplicity histogram of a box: interior faces 2, edges 4, vertices 8
    mult_local = num.mult[num.glo_num]
    assert set(np.unique(num.mult)) <= {1, 2, 4, 8}
    if n >= 2:
        interior_vertex_nodes = (n - 1) ** 3
        assert int((num.mult == 8).sum()) == interior_vertex_nodes
    assert abs(np.sum(1.0 / mult_local) - num.n_glob) < 1e-9


def test_first_occurrence_order():
    m = BoxMesh(3, 2, 2)
    num = so.number_nodes(3, m.elem_verts)
    first = np.maximum.accumulate(num.glo_num)
    # ids appear for the first time in increasing order 0, 1, 2, ...
    new = np.r_[True, first[1:] > first[:-1]]
    np.testing.assert_array_equal(num.glo_num[new], np.arange(num.n_glob))
    assert np.all(np.diff(first) <= 1)


# the 24 rotations of the reference cube as signed permutation matrices with det +1
ROTATIONS = [np.array(P) * s for P in itertools.permutations(np.eye(3, dtype=int))
             for s in itertools.product((1, -1), repeat=3)
             if round(np.linalg.det(np.array(P) * np.array(s))) == 1]


def _reorient(elem_verts, rng):
    """Relabel each element's local vertices by a random rotation of the reference cube."""
    out = elem_verts.copy()
    for e in range(elem_verts.shape[0]):
        R = ROTATIONS[rng.integers(len(ROTATIONS))]
        for v, (a, b, c) in enumerate(so._CORNER):
            s = R.T @ np.array([2 * a - 1, 2 * b - 1, 2 * c - 1])
            a0, b0, c0 = ((s + 1) // 2).tolist()
            out[e, v] = elem_verts[e, a0 + 2 * b0 + 4 * c0]
    return out


@pytest.mark.parametrize("N", [2, 4, 5])
def test_numbering_matches_coincident_points(N):
    # Brute force: two local nodes share a global id iff their physical points coincide,
    # with every element given a random local orientation.
    rng = np.random.default_rng(N)
    m = BoxMesh(3, 2, 3, jitter=0.2, seed=5)
    ev = _reorient(m.elem_verts, rng)
    num = so.number_nodes(N, ev)
    xi, _ = so.gll_nodes_weights(N)
    x = so.coordinates(so.element_vertices(m.vert_xyz, ev), xi).reshape(-1, 3)
    keys = np.round(x * 2 ** 30).astype(np.int64)
    _, pos_class = np.unique(keys, axis=0, return_inverse=True)
    pos_class = pos_class.ravel()
    assert num.n_glob == pos_class.max() + 1 == (3 * N + 1) * (2 * N + 1) * (3 * N + 1)
    # same partition: glo -> class is a function and a bijection
    pairs = np.unique(np.stack([num.glo_num, pos_class], axis=1), axis=0)
    assert pairs.shape[0] == num.n_glob
    # Dirichlet mask = points on the box surface
    on_surface = (np.abs(x - 0.5) > 0.5 - 1e-12).any(axis=1)
    np.testing.assert_array_equal(num.mask.astype(bool), on_surface)


def test_dirichlet_vertex_flags():
    m = BoxMesh(2, 2, 2)
    flags = np.zeros(m.num_vertices, dtype=np.uint8)
    flags[m.vert_xyz[:, 2] == 0.0] = 1  # only the bottom face is Dirichlet
    num = so.number_nodes(3, m.elem_verts, flags)
    xi, _ = so.gll_nodes_weights(3)
    x = so.coordinates(so.element_vertices(m.vert_xyz, m.elem_verts), xi).reshape(-1, 3)
    np.testing.assert_array_equal(num.mask.astype(bool), np.abs(x[:, 2]) < 1e-14)


def test_repeated_vertex_rejected():
    ev = BoxMesh(1, 1, 1).elem_verts.copy()
    ev[0, 3] = ev[0, 0]
    with pytest.raises(so.MeshError):
        so.number_nodes(2, ev)
