"""GPU conjugate gradient (Algorithm 1 with Jacobi z = M^-1 r) against the FP64 oracle.

Several iterates are correct (the reductions add in another order), so the gate is:
the oracle-recomputed true residual of the GPU solution meets rtol (1 + 1e-3); the
iteration count is within 2% of the oracle's; the error to the manufactured solution
sin(pi x) sin(pi y) sin(pi z) matches the oracle's to 3 significant digits."""
import math

import numpy as np
import pytest

from oracle import sem_oracle as so
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


@pytest.fixture(scope="module")
def c1(sem):
    """4x4x4 mesh on [0,1]^3, interior jitter 0.1h (seed 0), N = 7, sine RHS, rtol 1e-10."""
    m = BoxMesh(4, 4, 4, jitter=0.1, seed=0)
    prob = so.SemProblem(7, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    ref = so.pcg(prob, b, rtol=1e-10)
    mesh = sem.Mesh(7, m.vert_xyz, m.elem_verts, flags=3)
    return m, prob, b, ref, mesh


def _true_rel(prob, b, x):
    x = x.reshape(prob.shape())
    r = b - prob.ax(x)
    return math.sqrt(so.glsc3(r, r, prob.c) / so.glsc3(b, b, prob.c))


def _solve(sem, mesh, prob, opts):
    import torch
    b = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, b)
    x = torch.zeros_like(b)
    res = sem.sem_cg_solve(mesh.handle, b, x, opts)
    return res, x.cpu().numpy()


@pytest.mark.parametrize("variant,use_graph,check_every,f64_arith", [(0, 1, 50, 0), (1, 1, 17, 0), (0, 0, 1, 0),
                                                                     (0, 1, 50, 1), (1, 1, 50, 1), (0, 2, 50, 0),
                                                                     (0, 2, 7, 0)],
                         ids=["stored-graph", "otf-graph", "stored-eager", "stored-doublefloat", "otf-doublefloat",
                              "stored-persistent", "stored-persistent-short-runs"])
def test_cg_fp64_matches_oracle(sem, c1, variant, use_graph, check_every, f64_arith):
    m, prob, b, ref, mesh = c1
    opts = sem.sem_cg_default_opts(rtol=1e-10, variant=variant, use_graph=use_graph, check_every=check_every,
                                   f64_arith=f64_arith)
    res, x = _solve(sem, mesh, prob, opts)
    assert res["status"] == sem.SEM_OK, res
    assert abs(res["iters"] - ref.iterations) <= max(1, 0.02 * ref.iterations), (res["iters"], ref.iterations)
    assert _true_rel(prob, b, x) <= 1e-10 * (1 + 1e-3)
    e_gpu = np.abs(x - prob.exact_solution().ravel()).max()
    e_ref = np.abs(ref.x - prob.exact_solution()).max()
    assert abs(e_gpu - e_ref) <= 5e-4 * e_ref, (e_gpu, e_ref)


@pytest.mark.parametrize("inner_variant,f64_arith", [(1, 0), (0, 0), (1, 1)],
                         ids=["inner-otf", "inner-stored", "inner-otf-outer-doublefloat"])
def test_cg_mixed_precision(sem, c1, inner_variant, f64_arith):
    m, prob, b, ref, mesh = c1
    opts = sem.sem_cg_default_opts(rtol=1e-10, mixed=1, inner_variant=inner_variant, inner_rtol=1e-4,
                                   f64_arith=f64_arith)
    res, x = _solve(sem, mesh, prob, opts)
    assert res["status"] == sem.SEM_OK, res
    assert res["outer_iters"] >= 2
    assert _true_rel(prob, b, x) <= 1e-10 * (1 + 1e-3)
    e_gpu = np.abs(x - prob.exact_solution().ravel()).max()
    e_ref = np.abs(ref.x - prob.exact_solution()).max()
    assert abs(e_gpu - e_ref) <= 5e-4 * e_ref + 1e-11, (e_gpu, e_ref)


@pytest.mark.parametrize("inner_variant,graph", [(1, 1), (0, 0)], ids=["inner-otf-graph", "inner-stored-eager"])
def test_cg_mixed_reliable_updates(sem, c1, inner_variant, graph):
    """mixed = 2: the FP32 CG keeps its direction across residual replacements, so it needs
    about as many iterations as FP64 CG (restarted refinement needs far more)."""
    m, prob, b, ref, mesh = c1
    opts = sem.sem_cg_default_opts(rtol=1e-10, mixed=2, inner_variant=inner_variant, inner_rtol=0.1,
                                   use_graph=graph, check_every=7)
    res, x = _solve(sem, mesh, prob, opts)
    assert res["status"] == sem.SEM_OK, res
    assert res["outer_iters"] >= 5  # residual replacements
    assert _true_rel(prob, b, x) <= 1e-10 * (1 + 1e-3)
    assert res["iters"] <= 1.3 * ref.iterations, (res["iters"], ref.iterations)
    e_gpu = np.abs(x - prob.exact_solution().ravel()).max()
    e_ref = np.abs(ref.x - prob.exact_solution()).max()
    assert abs(e_gpu - e_ref) <= 5e-4 * e_ref + 1e-11, (e_gpu, e_ref)


def test_cg_small_mesh_runs_persistent(sem, c1):
    """Config 1 (64 elements, fewer than the SMs) with stored FP64 factors and use_graph = 2 runs
    the persistent kernel: a whole run of check_every iterations is one launch; the oracle gates
    hold (the parametrized test above) and the launch count shows the path taken."""
    import torch
    m, prob, b, ref, mesh = c1
    bd = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, bd)
    x = torch.zeros_like(bd)
    c0 = sem.sem_launch_count()
    res = sem.sem_cg_solve(mesh.handle, bd, x, sem.sem_cg_default_opts(rtol=1e-10, check_every=50, use_graph=2))
    launches = sem.sem_launch_count() - c0
    assert res["status"] == sem.SEM_OK
    assert launches <= 20, launches  # set-up kernels + one persistent launch per 50 iterations
    assert _true_rel(prob, b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-3)


def test_cg_stateful_and_limits(sem, c1):
    import torch
    m, prob, b, ref, mesh = c1
    bd = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, bd)
    x = torch.zeros_like(bd)
    cg = sem.sem_cg_create(mesh.handle, sem.sem_cg_default_opts(rtol=1e-10, check_every=10))
    sem.sem_cg_start(cg, bd, x)
    sem.sem_cg_iterate(cg, 10)
    q = sem.sem_cg_query(cg)
    assert q["iters"] == 10 and q["status"] == sem.SEM_ERR_BUSY
    # the residual history matches the oracle's to rounding in the first iterations
    assert abs(q["rel_res"] - ref.history[10]) <= 1e-8 * ref.history[10]
    for _ in range(100):
        sem.sem_cg_iterate(cg, 10)
        q = sem.sem_cg_query(cg)
        if q["status"] != sem.SEM_ERR_BUSY:
            break
    assert q["status"] == sem.SEM_OK and q["iters"] == pytest.approx(ref.iterations, abs=max(1, 0.02 * ref.iterations))
    sem.sem_cg_iterate(cg, 10)  # no-ops after convergence
    assert sem.sem_cg_query(cg)["iters"] == q["iters"]
    sem.sem_cg_destroy(cg)
    # iteration limit
    x.zero_()
    res = sem.sem_cg_solve(mesh.handle, bd, x, sem.sem_cg_default_opts(max_iter=7, check_every=3))
    assert res["status"] == sem.SEM_ERR_NOT_CONVERGED and res["iters"] == 7
    # zero right-hand side with x0 = 0: converged before the first iteration
    x.zero_()
    res = sem.sem_cg_solve(mesh.handle, torch.zeros_like(bd), x, sem.sem_cg_default_opts())
    assert res["status"] == sem.SEM_OK and res["iters"] == 0
    # a non-finite right-hand side is reported as a breakdown, not a hang
    bad = bd.clone()
    bad[5] = float("nan")
    x.zero_()
    res = sem.sem_cg_solve(mesh.handle, bad, x, sem.sem_cg_default_opts())
    assert res["status"] == sem.SEM_ERR_BREAKDOWN


@pytest.mark.parametrize("mixed", [0, 1], ids=["fp64", "mixed"])
def test_cg_single_element(sem, mixed):
    """Degenerate mesh: one element (every boundary face Dirichlet, (N-1)^3 unknowns), so each
    kernel's grid is a single partial element group."""
    m = BoxMesh(1, 1, 1)
    prob = so.SemProblem(7, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    ref = so.pcg(prob, b, rtol=1e-10)
    mesh = sem.Mesh(7, m.vert_xyz, m.elem_verts, flags=3)
    res, x = _solve(sem, mesh, prob, sem.sem_cg_default_opts(rtol=1e-10, mixed=mixed, inner_variant=sem.SEM_AX_OTF))
    mesh.close()
    assert res["status"] == sem.SEM_OK, res
    assert _true_rel(prob, b, x) <= 1e-10 * (1 + 1e-3)
    if not mixed:
        assert abs(res["iters"] - ref.iterations) <= max(1, 0.02 * ref.iterations), (res["iters"], ref.iterations)


@pytest.mark.parametrize("graph", [1, 0], ids=["graph", "eager"])
def test_cg_deferred_update_split_runs(sem, c1, graph):
    """The double-float CG makes each x update one iteration late, in the operator's prologue,
    and adds the pending one when a run of iterations ends. Runs of 4 + 3 + 5 iterations give
    the x of one run of 12 bit for bit, the residual follows the oracle's history, and runs
    after convergence change nothing."""
    import torch
    m, prob, b, ref, mesh = c1
    bd = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, bd)
    opts = sem.sem_cg_default_opts(rtol=1e-10, f64_arith=1, use_graph=graph, check_every=5)

    def run(chunks):
        x = torch.zeros_like(bd)
        cg = sem.sem_cg_create(mesh.handle, opts)
        sem.sem_cg_start(cg, bd, x)
        for k in chunks:
            sem.sem_cg_iterate(cg, k)
        q = sem.sem_cg_query(cg)
        return cg, x, q

    cg_a, xa, qa = run([12])
    cg_b, xb, qb = run([4, 3, 5])
    assert qa["iters"] == qb["iters"] == 12
    np.testing.assert_array_equal(xa.cpu().numpy(), xb.cpu().numpy())
    assert abs(qa["rel_res"] - ref.history[12]) <= 1e-8 * ref.history[12]
    # the returned x is the 12th iterate: its true residual is the recurrence's
    assert abs(_true_rel(prob, b, xa.cpu().numpy()) - qa["rel_res"]) <= 1e-6 * qa["rel_res"]
    sem.sem_cg_destroy(cg_b)
    for _ in range(100):
        sem.sem_cg_iterate(cg_a, 25)
        q = sem.sem_cg_query(cg_a)
        if q["status"] != sem.SEM_ERR_BUSY:
            break
    assert q["status"] == sem.SEM_OK and q["rel_res"] <= 1e-10
    # the flushed x carries the last update: its true residual is the recurrence's (the
    # double-float operator's own error, about 1e-14 of |A||x|, is far below 1e-12 here)
    assert abs(_true_rel(prob, b, xa.cpu().numpy()) - q["rel_res"]) <= 1e-12
    done = xa.cpu().numpy()
    sem.sem_cg_iterate(cg_a, 7)
    assert sem.sem_cg_query(cg_a)["iters"] == q["iters"]
    np.testing.assert_array_equal(xa.cpu().numpy(), done)
    sem.sem_cg_destroy(cg_a)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 8, 10, 11])
def test_cg_fused_prologue_every_order(sem, N):
    """The FP32 CG (reliable updates; TMA-staged prologue inputs for even N + 1, plain loads for
    odd) and the double-float CG (fused prologue for every order) on a ragged jittered mesh:
    the oracle's true residual of each solution meets rtol."""
    m = BoxMesh(3, 2, 2, jitter=0.1, seed=N)
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=sem.SEM_MESH_F64_STORED | sem.SEM_MESH_F32_STORED)
    for opts in (sem.sem_cg_default_opts(rtol=1e-10, mixed=2, inner_variant=sem.SEM_AX_OTF, inner_rtol=0.1),
                 sem.sem_cg_default_opts(rtol=1e-10, mixed=2, inner_variant=sem.SEM_AX_STORED, inner_rtol=0.1,
                                         use_graph=0),
                 sem.sem_cg_default_opts(rtol=1e-9, f64_arith=1)):
        res, x = _solve(sem, mesh, prob, opts)
        assert res["status"] == sem.SEM_OK, (N, res)
        assert _true_rel(prob, b, x) <= opts.rtol * (1 + 1e-3), N
    mesh.close()


@pytest.fixture(scope="module")
def c1_plain(c1):
    """The oracle's unpreconditioned CG (Algorithm 1 exactly as the paper states it) on config 1."""
    m, prob, b, ref, mesh = c1
    return so.pcg(prob, b, rtol=1e-10, precond=False)


@pytest.mark.parametrize("kw", [dict(), dict(variant=1, use_graph=0), dict(f64_arith=1),
                                dict(mixed=2, inner_rtol=0.1), dict(mixed=2, inner_rtol=0.1, inner_variant=0, use_graph=0)],
                         ids=["fp64-stored", "fp64-otf-eager", "double-float", "mixed-otf", "mixed-stored-eager"])
def test_cg_unpreconditioned(sem, c1, c1_plain, kw):
    """precond = 0: z = r (no M^-1 read; the FP32 operator's prologue copies three vectors
    instead of four). Same gate as the preconditioned solves against the oracle's plain CG."""
    m, prob, b, ref, mesh = c1
    res, x = _solve(sem, mesh, prob, sem.sem_cg_default_opts(rtol=1e-10, precond=0, **kw))
    assert res["status"] == sem.SEM_OK, res
    assert _true_rel(prob, b, x) <= 1e-10 * (1 + 1e-3)
    if not kw.get("mixed"):
        assert abs(res["iters"] - c1_plain.iterations) <= max(1, 0.02 * c1_plain.iterations), \
            (res["iters"], c1_plain.iterations)
    err = np.abs(x.reshape(prob.shape()) - prob.exact_solution()).max()
    err_ref = np.abs(c1_plain.x - prob.exact_solution()).max()
    assert abs(err - err_ref) <= 5e-4 * err_ref + (1e-11 if kw.get("mixed") else 0.0), (err, err_ref)


def test_cg_partial_dirichlet_and_otf_scale(sem):
    """Dirichlet nodes only on the bottom and top faces (vertex flags; the side faces keep the
    natural boundary condition), solved with stored factors, with the one-word-per-point
    on-the-fly variant (SEM_AX_OTF_SCALE), in double-float and in mixed precision; each
    solution meets the oracle's true residual, FP64 iterations within 2% of the oracle's."""
    import torch
    m = BoxMesh(3, 3, 2, jitter=0.1, seed=9)
    flags = ((m.vert_xyz[:, 2] < 1e-12) | (m.vert_xyz[:, 2] > 1 - 1e-12)).astype(np.uint8)
    N = 5
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts, dirichlet_vertex_flags=flags)
    b = prob.rhs()
    ref = so.pcg(prob, b, rtol=1e-10)
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, dirichlet_vertex_flags=flags,
                    flags=sem.SEM_MESH_F64_STORED | sem.SEM_MESH_OTF_SCALE)
    assert np.array_equal(sem.sem_mesh_get_glo_num(mesh.handle), prob.glo_num)
    for kw in (dict(), dict(variant=sem.SEM_AX_OTF_SCALE), dict(f64_arith=1),
               dict(mixed=2, inner_variant=sem.SEM_AX_OTF_SCALE, inner_rtol=0.1)):
        bd = torch.tensor(b.ravel(), device="cuda")
        x = torch.zeros_like(bd)
        res = sem.sem_cg_solve(mesh.handle, bd, x, sem.sem_cg_default_opts(rtol=1e-10, **kw))
        assert res["status"] == sem.SEM_OK, (kw, res)
        assert _true_rel(prob, b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-3), kw
        if not kw.get("mixed"):
            assert abs(res["iters"] - ref.iterations) <= max(1, 0.02 * ref.iterations), (kw, res["iters"], ref.iterations)
    mesh.close()
