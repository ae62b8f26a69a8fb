"""GPU tests of the solve server: requests of different sizes and orders run concurrently
give the same solution as each request solved alone (bit for bit: same launches and
fixed-order reductions), a request with an invalid mesh fails alone, and admission
respects the device-memory budget."""
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


REQS = [((3, 3, 3), 5, (1, 1, 1)), ((4, 3, 2), 7, (2, 1, 3)), ((2, 2, 2), 9, (1, 2, 1)), ((5, 4, 3), 3, (3, 3, 1)),
        ((3, 2, 4), 7, (1, 3, 2)), ((2, 3, 2), 5, (2, 2, 2))]


def _opts(sem, mixed=1):
    return sem.sem_cg_default_opts(rtol=1e-8, mixed=mixed, variant=sem.SEM_AX_OTF, inner_variant=sem.SEM_AX_OTF,
                                   inner_rtol=1e-5 if mixed == 1 else 0.1, check_every=20)


def _solo(sem, m, N, sine, opts, batched=False):
    """The request solved alone by the path the server took: the batched solver for requests
    the server batched, sem_cg_solve for the others."""
    import torch
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=0)
    b = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, *sine, sem.SEM_F64, b)
    x = torch.zeros_like(b)
    if batched:
        res = sem.sem_cg_solve_batch([mesh], [b], [x], opts)[0]
    else:
        res = sem.sem_cg_solve(mesh.handle, b, x, opts)
    out = x.cpu().numpy()
    mesh.close()
    return res, out


def _drain(sem, srv, tickets):
    import time
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < 300:
        for t in tickets:
            if t not in results:
                r = sem.sem_server_poll(srv, t)
                if r is not None:
                    results[t] = r
        time.sleep(0.005)
    assert len(results) == len(tickets), "server did not finish in time"
    return results


@pytest.mark.parametrize("mixed,batch", [(1, 0), (2, 0), (2, 1 << 21)],
                         ids=["restarted-streams", "reliable-updates-streams", "reliable-updates-batched"])
def test_results_alone_equal_results_in_the_mix(sem, mixed, batch):
    opts = _opts(sem, mixed)
    meshes = [BoxMesh(*d, jitter=0.1, seed=40 + q) for q, (d, _, _) in enumerate(REQS)]
    srv = sem.sem_server_create(8 << 30, 4, batch_max_points=batch)
    tickets = [sem.sem_server_submit(srv, N, m.vert_xyz, m.elem_verts, sine, opts)
               for m, (_, N, sine) in zip(meshes, REQS)]
    results = _drain(sem, srv, tickets)
    sem.sem_server_destroy(srv)
    for m, (d, N, sine), t in zip(meshes, REQS, tickets):
        res, x = results[t]
        assert res["status"] == sem.SEM_OK, res
        assert res["latency_ms"] >= res["setup_ms"] > 0
        assert res["batched"] == int(batch > 0), res
        solo, x_solo = _solo(sem, m, N, sine, opts, batched=batch > 0)
        assert solo["status"] == sem.SEM_OK and solo["iters"] == res["cg"]["iters"]
        np.testing.assert_array_equal(x, x_solo)  # identical alone and in the mix
    # and one of them against the FP64 oracle's true residual
    m, (d, N, sine) = meshes[0], REQS[0]
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    b = prob.rhs(*sine)
    r = b - prob.ax(results[tickets[0]][1].reshape(prob.shape()))
    assert np.sqrt(so.glsc3(r, r, prob.c) / so.glsc3(b, b, prob.c)) <= 1e-8 * (1 + 1e-3)


def test_bad_request_fails_alone_and_budget(sem):
    opts = _opts(sem)
    good = BoxMesh(3, 2, 2, jitter=0.1, seed=7)
    bad = BoxMesh(2, 2, 2)
    ev = bad.elem_verts.copy()
    ev[3, [0, 1]] = ev[3, [1, 0]]  # element 3 folded inside out: det J < 0
    srv = sem.sem_server_create(1 << 30, 2)
    t_good = sem.sem_server_submit(srv, 5, good.vert_xyz, good.elem_verts, (1, 1, 1), opts)
    t_bad = sem.sem_server_submit(srv, 5, bad.vert_xyz, ev, (1, 1, 1), opts)
    t_good2 = sem.sem_server_submit(srv, 7, good.vert_xyz, good.elem_verts, (2, 1, 1), opts)
    results = _drain(sem, srv, [t_good, t_bad, t_good2])
    assert results[t_bad][0]["status"] == sem.SEM_ERR_MESH
    assert results[t_good][0]["status"] == sem.SEM_OK and results[t_good2][0]["status"] == sem.SEM_OK
    big = BoxMesh(40, 40, 40)  # N = 9: 64M points, far beyond a 1 GB budget
    with pytest.raises(sem.SemError) as e:
        sem.sem_server_submit(srv, 9, big.vert_xyz, big.elem_verts, (1, 1, 1), opts)
    assert e.value.status == sem.SEM_ERR_ARG
    assert sem.sem_server_stats(srv)["active"] == 0
    sem.sem_server_destroy(srv)


def test_prebuilt_mesh_requests(sem):
    """sem_server_submit_mesh: a mesh built by the caller (with stored factors) and a host
    right-hand side from the oracle give, in the mix with ordinary requests, the same x as
    sem_cg_solve on an identical mesh; the server takes the mesh over, and prebuilt meshes
    still queued when the server is destroyed are released with it."""
    import torch
    cases = [((3, 3, 2), 7, 0, sem.SEM_MESH_F64_STORED), ((2, 3, 3), 5, 2, sem.SEM_MESH_F32_STORED),
             ((4, 2, 2), 9, 0, sem.SEM_MESH_F64X_STORED)]
    srv = sem.sem_server_create(8 << 30, 3)
    tickets, want = [], []
    for q, (d, N, mixed, flags) in enumerate(cases):
        m = BoxMesh(*d, jitter=0.1, seed=70 + q)
        opts = sem.sem_cg_default_opts(rtol=1e-9, mixed=mixed, variant=sem.SEM_AX_STORED if mixed == 0 else sem.SEM_AX_OTF,
                                       inner_variant=sem.SEM_AX_STORED, inner_rtol=0.1, check_every=10,
                                       f64_arith=int(flags == sem.SEM_MESH_F64X_STORED))
        b = so.SemProblem(N, m.vert_xyz, m.elem_verts).rhs(1 + q, 2, 1).ravel()
        solo_mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=flags)
        bd = torch.tensor(b, device="cuda")
        x = torch.zeros_like(bd)
        res = sem.sem_cg_solve(solo_mesh.handle, bd, x, opts)
        assert res["status"] == sem.SEM_OK, res
        want.append((res, x.cpu().numpy(), N, m, b))
        solo_mesh.close()
        mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=flags)
        assert sem.sem_mesh_info(mesh.handle) == (mesh.n, mesh.info["n_glob"], mesh.info["n_seg"])
        with pytest.raises(sem.SemError):
            sem.sem_server_submit_mesh(srv, mesh, b[:-1], opts)  # wrong size: the caller keeps the mesh
        assert mesh.handle is not None
        tickets.append(sem.sem_server_submit_mesh(srv, mesh, b, opts))
        assert mesh.handle is None
        tickets.append(sem.sem_server_submit(srv, 5, m.vert_xyz, m.elem_verts, (1, 1, 1), _opts(sem, 2)))
    results = _drain(sem, srv, tickets)
    sem.sem_server_destroy(srv)
    for (res, x_solo, N, m, b), t in zip(want, tickets[0::2]):
        got, x = results[t]
        assert got["status"] == sem.SEM_OK and got["cg"]["iters"] == res["iters"], (got, res)
        np.testing.assert_array_equal(x, x_solo)
    res, x_solo, N, m, b = want[0]
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    bb = b.reshape(prob.shape())
    r = bb - prob.ax(x_solo.reshape(prob.shape()))
    assert np.sqrt(so.glsc3(r, r, prob.c) / so.glsc3(bb, bb, prob.c)) <= 1e-9 * (1 + 1e-3)
    # a server destroyed with prebuilt meshes still queued releases them
    srv = sem.sem_server_create(8 << 30, 1)
    m = BoxMesh(3, 3, 3, jitter=0.1, seed=80)
    b = so.SemProblem(5, m.vert_xyz, m.elem_verts).rhs(1, 1, 1).ravel()
    for _ in range(4):
        sem.sem_server_submit_mesh(srv, sem.Mesh(5, m.vert_xyz, m.elem_verts, flags=0), b, _opts(sem, 2))
    sem.sem_server_destroy(srv)
    torch.cuda.synchronize()
