"""Failure detection on the GPU without a fault: the bounded waits that guard every TMA copy
give up after their time limit and report SEM_ERR_TIMEOUT (the copy is never issued, so
nothing arrives), the CUDA context stays usable, and the same wait completes when the copy
is issued; likewise the bounded grid barrier of the persistent small-mesh CG kernel (a block
that never arrives)."""
import numpy as np
import pytest

from synthetic import BoxMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem():
    import torch
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    torch.cuda.set_device(0)
    return sem_mod


def test_bounded_wait_completes_when_the_copy_arrives(sem):
    st, ms = sem.sem_probe_bounded_wait(1_000_000_000, 1)
    assert st == sem.SEM_OK and ms < 100.0, (st, ms)


@pytest.mark.parametrize("limit_ms", [5, 50])
def test_bounded_wait_times_out_and_the_context_survives(sem, limit_ms):
    import torch
    st, ms = sem.sem_probe_bounded_wait(limit_ms * 1_000_000, 0)
    assert st == sem.SEM_ERR_TIMEOUT
    assert limit_ms * 0.99 <= ms <= limit_ms + 500.0, ms
    # the context still works: an operator application and a reduction afterwards
    m = BoxMesh(2, 2, 2, jitter=0.1, seed=3)
    mesh = sem.Mesh(3, m.vert_xyz, m.elem_verts)
    u = torch.ones(mesh.n, dtype=torch.float64, device="cuda")
    w = torch.empty_like(u)
    sem.sem_ax(mesh.handle, sem.SEM_AX_STORED, sem.SEM_F64, u, w, assemble=False)
    assert float(torch.linalg.norm(w)) / np.sqrt(mesh.n) < 1e-12  # A_L 1 = 0 element by element
    st2, _ = sem.sem_probe_bounded_wait(1_000_000_000, 1)
    assert st2 == sem.SEM_OK
    mesh.close()


def test_launch_count_matches_the_kernels_run(sem):
    """sem_launch_count (the benchmark's gpu_launches) counts every kernel the library runs: one
    for A_L, one more for the assembly; three per CG iteration, replayed from a graph or not."""
    import torch
    m = BoxMesh(3, 2, 2, jitter=0.1, seed=4)
    mesh = sem.Mesh(4, m.vert_xyz, m.elem_verts)
    u = torch.rand(mesh.n, dtype=torch.float64, device="cuda")
    w = torch.empty_like(u)
    c0 = sem.sem_launch_count()
    sem.sem_ax(mesh.handle, sem.SEM_AX_STORED, sem.SEM_F64, u, w, assemble=False)
    c1 = sem.sem_launch_count()
    sem.sem_ax(mesh.handle, sem.SEM_AX_STORED, sem.SEM_F64, u, w, assemble=True)
    c2 = sem.sem_launch_count()
    assert (c1 - c0, c2 - c1) == (1, 2)
    b = torch.empty_like(u)
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, b)
    # three launches per iteration, replayed from a graph or not; with use_graph = 2, stored
    # factors and a mesh of fewer elements than SMs the persistent kernel runs the 5 iterations
    # in one launch
    for variant, graph, want in ((sem.SEM_AX_OTF, 0, 15), (sem.SEM_AX_STORED, 1, 15), (sem.SEM_AX_STORED, 2, 1),
                                 (sem.SEM_AX_OTF, 2, 15)):
        x = torch.zeros_like(b)
        cg = sem.sem_cg_create(mesh.handle, sem.sem_cg_default_opts(rtol=0.0, max_iter=1 << 20, use_graph=graph,
                                                                    variant=variant))
        sem.sem_cg_start(cg, b, x)
        c3 = sem.sem_launch_count()
        sem.sem_cg_iterate(cg, 5)
        q = sem.sem_cg_query(cg)
        assert q["iters"] == 5 and sem.sem_launch_count() - c3 == want, (variant, graph)
        sem.sem_cg_destroy(cg)
    mesh.close()


def test_grid_barrier_completes_when_every_block_arrives(sem):
    st, ms = sem.sem_probe_grid_barrier(0)
    assert st == sem.SEM_OK and ms < 100.0, (st, ms)


def test_grid_barrier_times_out_and_the_context_survives(sem):
    """The persistent small-mesh CG kernel meets at bounded grid barriers: a block that never
    arrives makes the others give up after the limit (1 s) with SEM_ERR_TIMEOUT; then a
    persistent solve runs normally on the same context."""
    import torch
    from oracle import sem_oracle as so
    st, ms = sem.sem_probe_grid_barrier(1)
    assert st == sem.SEM_ERR_TIMEOUT
    assert 990.0 <= ms <= 3000.0, ms
    m = BoxMesh(2, 2, 2, jitter=0.1, seed=3)
    prob = so.SemProblem(5, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    mesh = sem.Mesh(5, m.vert_xyz, m.elem_verts)
    bd = torch.tensor(b.ravel(), device="cuda")
    x = torch.zeros_like(bd)
    res = sem.sem_cg_solve(mesh.handle, bd, x, sem.sem_cg_default_opts(rtol=1e-10, use_graph=2))
    assert res["status"] == sem.SEM_OK
    r = b - prob.ax(x.cpu().numpy().reshape(prob.shape()))
    assert np.sqrt(so.glsc3(r, r, prob.c) / so.glsc3(b, b, prob.c)) <= 1e-10 * (1 + 1e-3)
    mesh.close()
