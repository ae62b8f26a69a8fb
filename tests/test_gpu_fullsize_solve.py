"""Full-size solves checked with the oracle's arithmetic: on the 32^3, N = 7 mesh of the
Ax-throughput workload (16,777,216 local points), the right-hand side is the oracle's (Eq. 2 by
GLL quadrature, assembled and masked), the GPU solves to rtol 1e-10 with each solver the
benchmark times, and the true residual b - A x of every solution is formed by the oracle
(element-by-element A_L, QQ^T by explicit sums, <r, r, c>). The gate is Algorithm 1's stopping
test applied to the true residual: sqrt(<r,r,c>/<b,b,c>) <= 1e-10 (1 + 1e-3).

The oracle's set-up at this size (numbering by dictionary over 16.8M points) takes a minute or
two of host time; it is built once for the module."""
import math

import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh

pytestmark = pytest.mark.gpu

NEL, N, JITTER, SEED = 32, 7, 0.15, 1
RTOL = 1e-10


@pytest.fixture(scope="module")
def problem():
    import torch
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    torch.cuda.set_device(0)
    m = BoxMesh(NEL, NEL, NEL, jitter=JITTER, seed=SEED)
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    mesh = sem_mod.Mesh(N, m.vert_xyz, m.elem_verts,
                        flags=sem_mod.SEM_MESH_F64_STORED | sem_mod.SEM_MESH_F64X_STORED)
    yield sem_mod, prob, b, mesh
    mesh.close()


def _oracle_true_rel(prob, b, x):
    r = b - prob.ax(x.reshape(prob.shape()))
    return math.sqrt(so.glsc3(r, r, prob.c) / so.glsc3(b, b, prob.c))


SOLVERS = {
    "fp64-cg": dict(variant=0),
    "mixed-reliable-otf": dict(mixed=2, variant=0, inner_variant=1, inner_rtol=0.1),
    "double-float-cg": dict(variant=0, f64_arith=1),
    "double-float-otf-cg": dict(variant=1, f64_arith=1),
}


@pytest.mark.parametrize("name", list(SOLVERS))
def test_full_size_solve_meets_the_oracle_true_residual(problem, name):
    import torch
    sem, prob, b, mesh = problem
    bd = torch.tensor(b.ravel(), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(bd)
    res = sem.sem_cg_solve(mesh.handle, bd, x, sem.sem_cg_default_opts(rtol=RTOL, **SOLVERS[name]))
    assert res["status"] == sem.SEM_OK, res
    rel = _oracle_true_rel(prob, b, x.cpu().numpy())
    assert rel <= RTOL * (1 + 1e-3), (name, rel, res)


def test_full_size_batched_solves_meet_the_oracle_true_residual(problem):
    """The batched solver on the full-size mesh (two right-hand sides on one mesh, so the
    table holds 2 x 8192 element groups, 2 x 4096 update chunks)."""
    import torch
    sem, prob, b, mesh = problem
    bd = torch.tensor(b.ravel(), dtype=torch.float64, device="cuda")
    b2 = 2.0 * b
    bd2 = torch.tensor(b2.ravel(), dtype=torch.float64, device="cuda")
    xs = [torch.zeros_like(bd), torch.zeros_like(bd)]
    res = sem.sem_cg_solve_batch([mesh, mesh], [bd, bd2], xs,
                                 sem.sem_cg_default_opts(rtol=RTOL, mixed=2, variant=0, inner_variant=1,
                                                         inner_rtol=0.1, check_every=25))
    for r, rhs, x in zip(res, (b, b2), xs):
        assert r["status"] == sem.SEM_OK, r
        assert _oracle_true_rel(prob, rhs, x.cpu().numpy()) <= RTOL * (1 + 1e-3)
