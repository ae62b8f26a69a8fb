"""The pins must catch plausible mistakes: each test plants one mistake in a
copy of an oracle step (on the CPU) and checks that the independent pin
(brute-force dense stiffness, left-to-right dssum order) rejects it."""
import numpy as np

from oracle import sem_oracle as so
from synthetic import BoxMesh


def _brute_force_gap(ax_fn, N=3):
    m = BoxMesh(2, 2, 2, jitter=0.2, seed=7)
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    K = so.assembled_stiffness_dense(prob)
    v = np.random.default_rng(0).standard_normal(prob.num.n_glob)
    w = ax_fn(so.scatter_local(v, prob.glo_num).reshape(prob.shape()), prob.G, prob.D)
    got = so.gather_global(w, prob.glo_num, prob.num.n_glob)
    return np.abs(got - K @ v).max() / np.abs(K @ v).max()


def test_correct_oracle_passes():
    assert _brute_force_gap(so.ax_local) < 1e-12


def test_transposed_D_caught():
    assert _brute_force_gap(lambda u, G, D: so.ax_local(u, G, D.T)) > 1e-3


def test_dropped_cross_term_caught():
    def ax(u, G, D):
        G2 = G.copy()
        G2[:, 1] = 0.0  # forget G12
        return so.ax_local(u, G2, D)
    assert _brute_force_gap(ax) > 1e-3


def test_swapped_factor_order_caught():
    def ax(u, G, D):  # G13 and G23 swapped (wrong index bookkeeping)
        return so.ax_local(u, G[:, [0, 1, 4, 3, 2, 5]], D)
    assert _brute_force_gap(ax) > 1e-3


def test_wrong_inverse_orientation_caught():
    # G built as J^-T J^-1 instead of J^-1 J^-T
    m = BoxMesh(2, 2, 2, jitter=0.2, seed=7)
    prob = so.SemProblem(3, m.vert_xyz, m.elem_verts)
    J = so.jacobian(prob.X, prob.xi)
    Jinv = np.linalg.inv(J)
    M = np.swapaxes(Jinv, -1, -2) @ Jinv
    Gf = M * (so.weights3(prob.w)[None] * np.linalg.det(J))[..., None, None]
    Gbad = np.stack([Gf[..., 0, 0], Gf[..., 0, 1], Gf[..., 0, 2], Gf[..., 1, 1], Gf[..., 1, 2], Gf[..., 2, 2]], 1)
    assert _brute_force_gap(lambda u, G, D: so.ax_local(u, Gbad, D)) > 1e-3


def test_reversed_dssum_order_caught():
    glo = np.array([0, 0, 0])
    big = 2.0 ** 60
    w = np.array([1.0, big, -big])
    right_to_left = (w[2] + w[1]) + w[0]  # = 1
    assert right_to_left == 1.0 and so.dssum(w, glo)[0] == 0.0
