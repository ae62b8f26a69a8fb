"""GPU tests of the batched mixed-precision solves (sem_cg_solve_batch and the server's batch):
many small problems of different orders and sizes advance together in shared launches over a
device-side table. Each problem's x is bit-identical to the x of the same problem solved
alone through the same path (its partial sums are fixed by the problem, not by the mix), and
meets the oracle's true residual."""
import math
import time

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


# (elements per direction, order, wave numbers): orders with odd and even points per direction,
# a single element, ragged boxes
PROBLEMS = [((3, 3, 3), 5, (1, 1, 1)), ((4, 3, 2), 7, (2, 1, 3)), ((2, 2, 2), 9, (1, 2, 1)),
            ((5, 4, 3), 3, (3, 3, 1)), ((3, 2, 4), 7, (1, 3, 2)), ((2, 3, 2), 5, (2, 2, 2)),
            ((1, 1, 1), 7, (1, 1, 1)), ((4, 4, 4), 4, (1, 2, 3)), ((2, 2, 3), 1, (1, 1, 1)),
            ((3, 3, 2), 10, (2, 3, 1)), ((6, 5, 4), 5, (1, 1, 2))]


def _opts(sem, mixed, rtol=1e-9):
    return sem.sem_cg_default_opts(rtol=rtol, mixed=mixed, variant=sem.SEM_AX_OTF, inner_variant=sem.SEM_AX_OTF,
                                   inner_rtol=1e-4 if mixed == 1 else 0.1, check_every=13)


def _problem(sem, q):
    import torch
    d, N, sine = PROBLEMS[q]
    m = BoxMesh(*d, jitter=0.1, seed=90 + q)
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=0)
    b = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, *sine, sem.SEM_F64, b)
    return m, mesh, b


def _true_rel(N, m, sine, x):
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    b = prob.rhs(*sine)
    r = b - prob.ax(x.reshape(prob.shape()))
    return math.sqrt(so.glsc3(r, r, prob.c) / so.glsc3(b, b, prob.c))


@pytest.mark.parametrize("mixed", [2, 1], ids=["reliable-updates", "restarted"])
def test_batch_alone_equals_in_the_mix_and_meets_the_oracle(sem, mixed):
    import torch
    opts = _opts(sem, mixed)
    probs = [_problem(sem, q) for q in range(len(PROBLEMS))]
    xs = [torch.zeros_like(b) for _, _, b in probs]
    res = sem.sem_cg_solve_batch([p[1] for p in probs], [p[2] for p in probs], xs, opts)
    for q, ((m, mesh, b), x, r) in enumerate(zip(probs, xs, res)):
        d, N, sine = PROBLEMS[q]
        assert r["status"] == sem.SEM_OK, (q, r)
        assert r["outer_iters"] >= 2
        assert _true_rel(N, m, sine, x.cpu().numpy()) <= opts.rtol * (1 + 1e-3), q
        # the same problem alone through the batched path: the same x, bit for bit
        x1 = torch.zeros_like(b)
        r1 = sem.sem_cg_solve_batch([mesh], [b], [x1], opts)[0]
        assert r1["iters"] == r["iters"] and r1["outer_iters"] == r["outer_iters"], (q, r1, r)
        np.testing.assert_array_equal(x1.cpu().numpy(), x.cpu().numpy())
    # the order of the problems in the call does not matter either
    rev = list(reversed(range(len(probs))))
    xr = [torch.zeros_like(probs[q][2]) for q in rev]
    sem.sem_cg_solve_batch([probs[q][1] for q in rev], [probs[q][2] for q in rev], xr, opts)
    for k, q in enumerate(rev):
        np.testing.assert_array_equal(xr[k].cpu().numpy(), xs[q].cpu().numpy())
    for _, mesh, _ in probs:
        mesh.close()


def test_batch_iterations_match_the_single_mesh_solver(sem):
    """The batched FP32 iteration is the single-mesh one (same steps; only the split of the
    reductions differs): iteration counts agree within 2%, and the round length does not change
    the result."""
    import torch
    m, mesh, b = _problem(sem, 1)
    opts = _opts(sem, 2, rtol=1e-10)
    x = torch.zeros_like(b)
    r_single = sem.sem_cg_solve(mesh.handle, b, x, opts)
    xb = torch.zeros_like(b)
    r_batch = sem.sem_cg_solve_batch([mesh], [b], [xb], opts)[0]
    assert r_single["status"] == r_batch["status"] == sem.SEM_OK
    assert abs(r_batch["iters"] - r_single["iters"]) <= max(2, 0.02 * r_single["iters"]), (r_batch, r_single)
    xc = torch.zeros_like(b)
    opts.check_every = 1
    sem.sem_cg_solve_batch([mesh], [b], [xc], opts)
    np.testing.assert_array_equal(xc.cpu().numpy(), xb.cpu().numpy())
    mesh.close()


def test_batch_limits_and_errors(sem):
    import torch
    m, mesh, b = _problem(sem, 0)
    x = torch.zeros_like(b)
    with pytest.raises(sem.SemError) as e:  # FP64 CG is not batched
        sem.sem_cg_solve_batch([mesh], [b], [x], sem.sem_cg_default_opts(mixed=0))
    assert e.value.status == sem.SEM_ERR_ARG
    with pytest.raises(sem.SemError) as e:  # the stored-factor inner operator is not batched
        sem.sem_cg_solve_batch([mesh], [b], [x], sem.sem_cg_default_opts(mixed=2, inner_variant=sem.SEM_AX_STORED))
    assert e.value.status == sem.SEM_ERR_ARG
    with pytest.raises(sem.SemError) as e:  # one x for two problems
        sem.sem_cg_solve_batch([mesh, mesh], [b, b], [x, x], _opts(sem, 2))
    assert e.value.status == sem.SEM_ERR_ARG
    # the iteration limit ends a problem alone; the others converge
    m2, mesh2, b2 = _problem(sem, 5)
    x2 = torch.zeros_like(b2)
    o = _opts(sem, 2)
    o.max_iter = 5
    res = sem.sem_cg_solve_batch([mesh, mesh2], [b, b2], [x, x2], o, raise_on=())
    assert all(r["status"] == sem.SEM_ERR_NOT_CONVERGED for r in res)
    # one mesh may serve two problems with different right-hand sides
    b3 = torch.empty_like(b)
    sem.sem_rhs_sine(mesh.handle, 2, 1, 1, sem.SEM_F64, b3)
    xa, xb = torch.zeros_like(b), torch.zeros_like(b)
    res = sem.sem_cg_solve_batch([mesh, mesh], [b, b3], [xa, xb], _opts(sem, 2))
    assert all(r["status"] == sem.SEM_OK for r in res)
    d, N, _ = PROBLEMS[0]
    assert _true_rel(N, m, (2, 1, 1), xb.cpu().numpy()) <= 1e-9 * (1 + 1e-3)
    mesh.close()
    mesh2.close()


def _drain(sem, srv, tickets, timeout=300):
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t not in results:
                r = sem.sem_server_poll(srv, t)
                if r is not None:
                    results[t] = r
        time.sleep(0.002)
    assert len(results) == len(tickets), "server did not finish in time"
    return results


def test_server_batches_small_requests_identically_alone_and_in_the_mix(sem):
    """Twelve small requests submitted at once run in the server's batch together (at least
    eight at the same time); each result is bit-identical to the same request submitted alone,
    and a large request in the same stream takes its own stream."""
    opts = _opts(sem, 2, rtol=1e-8)
    reqs = [PROBLEMS[q % len(PROBLEMS)] for q in range(12)]
    meshes = [BoxMesh(*d, jitter=0.1, seed=300 + q) for q, (d, _, _) in enumerate(reqs)]
    srv = sem.sem_server_create(16 << 30, 12, batch_max_points=1 << 21, batch_round_iters=10)
    tickets = [sem.sem_server_submit(srv, N, m.vert_xyz, m.elem_verts, sine, opts)
               for m, (_, N, sine) in zip(meshes, reqs)]
    big = BoxMesh(14, 14, 14, jitter=0.1, seed=399)  # N = 7: 1.4M points > the 1M batch limit below
    results = _drain(sem, srv, tickets)
    stats = sem.sem_server_batch_stats(srv)
    sem.sem_server_destroy(srv)
    assert stats["max_batch"] >= 8, stats
    for m, (d, N, sine), t in zip(meshes, reqs, tickets):
        res, x = results[t]
        assert res["status"] == sem.SEM_OK and res["batched"] == 1, res
        alone = sem.sem_server_create(4 << 30, 1, batch_max_points=1 << 21, batch_round_iters=7)
        ta = sem.sem_server_submit(alone, N, m.vert_xyz, m.elem_verts, sine, opts)
        ra, xa = _drain(sem, alone, [ta])[ta]
        sem.sem_server_destroy(alone)
        assert ra["batched"] == 1 and ra["cg"]["iters"] == res["cg"]["iters"]
        np.testing.assert_array_equal(xa, x)
    m, (d, N, sine) = meshes[0], reqs[0]
    assert _true_rel(N, m, sine, results[tickets[0]][1]) <= 1e-8 * (1 + 1e-3)
    # a request above the batch limit is solved on its own stream
    srv = sem.sem_server_create(16 << 30, 2, batch_max_points=1 << 20)
    t = sem.sem_server_submit(srv, 7, big.vert_xyz, big.elem_verts, (1, 1, 1), opts)
    res, _ = _drain(sem, srv, [t])[t]
    sem.sem_server_destroy(srv)
    assert res["status"] == sem.SEM_OK and res["batched"] == 0
