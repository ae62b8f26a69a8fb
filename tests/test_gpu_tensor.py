"""GPU tests of the FP32 on-the-fly operator whose line contractions run on the tensor cores
(mma.sync m16n8k8 with TF32 operands split into high and low parts, N = 7; block shape
choice 3 of the tuner): A_L element by element and assembled against the FP64 oracle within
the FP32 bound (2e-6 relative 2-norm), the fused CG mode inside a mixed solve against the
oracle's true residual, and the tuner timing it beside the CUDA-core shapes."""
import math

import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh, local_field

pytestmark = pytest.mark.gpu

N = 7


@pytest.fixture(scope="module")
def sem():
    import torch
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    torch.cuda.set_device(0)
    yield sem_mod
    sem_mod.sem_autotune_clear()


@pytest.mark.parametrize("shape", [(5, 4, 3), (1, 1, 1), (9, 7, 6)], ids=["5x4x3", "one-element", "9x7x6"])
def test_tensor_core_operator_matches_the_oracle(sem, shape):
    import torch
    m = BoxMesh(*shape, jitter=0.15, seed=7)
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=0)
    u = local_field(mesh.n, seed=31)
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    w_tc, w_cc = torch.empty_like(ud), torch.empty_like(ud)
    sem.sem_autotune_set(N, sem.SEM_F32, sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE)
    sem.sem_ax(mesh.handle, sem.SEM_AX_OTF, sem.SEM_F32, ud, w_tc, assemble=False)
    sem.sem_autotune_set(N, sem.SEM_F32, sem.SEM_AX_OTF, 0)
    sem.sem_ax(mesh.handle, sem.SEM_AX_OTF, sem.SEM_F32, ud, w_cc, assemble=False)
    want = prob.ax_local(ud.double().cpu().numpy()).ravel()
    got = w_tc.double().cpu().numpy()
    assert np.linalg.norm(got - want) <= 2e-6 * np.linalg.norm(want)
    # element by element too (each element's contractions are separate tiles)
    P = (N + 1) ** 3
    err = np.linalg.norm((got - want).reshape(-1, P), axis=1) / np.linalg.norm(want.reshape(-1, P), axis=1)
    assert err.max() <= 2e-6, err.max()
    cc = w_cc.double().cpu().numpy()
    assert np.linalg.norm(got - cc) <= 2e-6 * np.linalg.norm(want)
    # assembled (QQ^T and the mask after the tensor-core A_L)
    sem.sem_autotune_set(N, sem.SEM_F32, sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE)
    sem.sem_ax(mesh.handle, sem.SEM_AX_OTF, sem.SEM_F32, ud, w_tc, assemble=True)
    want_a = prob.ax(ud.double().cpu().numpy()).ravel()
    assert np.linalg.norm(w_tc.double().cpu().numpy() - want_a) <= 2e-6 * np.linalg.norm(want_a)
    sem.sem_autotune_clear()
    mesh.close()


def test_tensor_core_cg_mode_in_a_mixed_solve(sem):
    import torch
    m = BoxMesh(4, 4, 4, jitter=0.1, seed=0)
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=sem.SEM_MESH_F64_STORED)
    bd = torch.tensor(b.ravel(), device="cuda")
    sem.sem_autotune_set(N, sem.SEM_F32, sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE)
    for graph in (1, 0):
        x = torch.zeros_like(bd)
        res = sem.sem_cg_solve(mesh.handle, bd, x, sem.sem_cg_default_opts(rtol=1e-10, mixed=2, inner_variant=1,
                                                                           inner_rtol=0.1, use_graph=graph))
        assert res["status"] == sem.SEM_OK, res
        r = b - prob.ax(x.cpu().numpy().reshape(prob.shape()))
        assert math.sqrt(so.glsc3(r, r, prob.c) / so.glsc3(b, b, prob.c)) <= 1e-10 * (1 + 1e-3)
    sem.sem_autotune_clear()
    mesh.close()


def test_tuner_times_the_tensor_core_candidate(sem):
    m = BoxMesh(6, 6, 6, jitter=0.1, seed=3)
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=sem.SEM_MESH_F32_STORED)
    rep = sem.sem_autotune(mesh.handle, sem.SEM_F32, reps=3)
    shapes = [(c["variant"], c["shape"]) for c in rep["candidates"]]
    assert (sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE) in shapes, shapes
    assert all(c["ms"] > 0 for c in rep["candidates"])
    sem.sem_autotune_clear()
    with pytest.raises(sem.SemError):
        sem.sem_autotune_set(5, sem.SEM_F32, sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE)  # compiled for N = 7 only
    mesh.close()
