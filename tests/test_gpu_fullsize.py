"""Full-size GPU checks on the 32^3, N = 7 mesh (16,777,216 local points: the Ax-throughput
workload) in the launch configuration the benchmark uses: a grid of resident blocks striding
over element groups, with the next group's factor copy in flight.

- A_L of every variant and precision on 64 sampled elements against the FP64 oracle, element
  by element (Eq. 4 with the factors of Section 4.2 / Section 5.1);
- gather-scatter (Eq. 5, Algorithm 1 step 7) bit-exact on sampled segments against the
  left-to-right sum of their copies;
- CG mode (Algorithm 1 with the fused prologue and reductions, as timed by the benchmark):
  its iterates equal those of a CG driven step by step through the plain operator and dot
  product of the library, and its recurrence residual equals the true residual b - A x."""
import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh, global_field, local_field

pytestmark = pytest.mark.gpu

NEL, N, JITTER, SEED = 32, 7, 0.15, 1
P = (N + 1) ** 3


@pytest.fixture(scope="module")
def full():
    import torch
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    torch.cuda.set_device(0)
    m = BoxMesh(NEL, NEL, NEL, jitter=JITTER, seed=SEED)
    mesh = sem_mod.Mesh(N, m.vert_xyz, m.elem_verts, flags=15)  # every stored-factor form
    yield sem_mod, m, mesh
    mesh.close()


VARIANTS = [(0, 0, 1e-12), (1, 0, 1e-12), (3, 0, 1e-12), (0, 2, 1e-12), (0, 1, 2e-6), (1, 1, 2e-6), (3, 1, 2e-6)]
VIDS = ["stored-f64", "otf-f64", "otfscale-f64", "stored-f64x", "stored-f32", "otf-f32", "otfscale-f32"]


@pytest.mark.parametrize("variant,prec,tol", VARIANTS, ids=VIDS)
def test_ax_sampled_elements(full, variant, prec, tol):
    import torch
    sem, m, mesh = full
    u = local_field(mesh.n, seed=SEED + 17)
    ud = torch.tensor(u, dtype=torch.float32 if prec == 1 else torch.float64, device="cuda")
    wd = torch.empty_like(ud)
    sem.sem_ax(mesh.handle, variant, prec, ud, wd, assemble=False)
    rng = np.random.default_rng(5 + variant + 10 * prec)
    els = np.sort(rng.choice(m.num_elements, size=64, replace=False))
    els[0], els[-1] = 0, m.num_elements - 1  # first and last element groups of the grid stride
    xi, wq = so.gll_nodes_weights(N)
    D = so.lagrange_derivative_matrix(xi)
    G, _ = so.geometric_factors(so.element_vertices(m.vert_xyz, m.elem_verts[els]), xi, wq)
    want = so.ax_local(u.reshape(-1, P)[els].reshape(len(els), N + 1, N + 1, N + 1), G, D).reshape(len(els), P)
    got = wd.double().cpu().numpy().reshape(-1, P)[els]
    err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert err.max() <= tol, (err.max(), els[np.argmax(err)])


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_dssum_sampled_segments(full, prec):
    import torch
    sem, m, mesh = full
    off, idx, msk = sem.sem_mesh_get_segments(mesh.handle)
    dt = torch.float32 if prec == 1 else torch.float64
    u = torch.tensor(local_field(mesh.n, seed=SEED + 23), dtype=dt, device="cuda")
    before = u.cpu().numpy()
    sem.sem_dssum(mesh.handle, prec, u, apply_mask=True)
    after = u.cpu().numpy()
    rng = np.random.default_rng(11 + prec)
    segs = np.concatenate([[0, len(msk) - 1], rng.choice(len(msk), size=20000, replace=False)])
    for g in segs:
        copies = idx[off[g]:off[g + 1]]
        s = before[copies[0]]
        for c in copies[1:]:
            s = s + before[c]  # left to right, in the vector's precision
        want = 0.0 if msk[g] else s
        assert np.all(after[copies] == want), g
    # element-interior points are untouched
    interior = np.ones(mesh.n, dtype=bool)
    interior[idx] = False
    assert np.array_equal(after[interior], before[interior])


def _driven_cg(sem, mesh, b, x, k, f64x):
    """k Jacobi-PCG iterations (Algorithm 1 with z = M^-1 r) driven step by step through the
    library's plain calls: assembled A (sem_ax), <a, b, c> (sem_glsc3), M^-1 (sem_jacobi)."""
    import torch
    prec = 2 if f64x else 0
    minv = torch.empty_like(b)
    sem.sem_jacobi(mesh.handle, 0, minv)
    w = torch.empty_like(b)
    dot = torch.empty(1, dtype=torch.float64, device="cuda")

    def glsc3(a, c):
        sem.sem_glsc3(mesh.handle, 0, a, c, dot)
        return float(dot.item())

    sem.sem_ax(mesh.handle, 0, prec, x, w, assemble=True)
    r = b - w
    z = minv * r
    p = z.clone()
    rho = glsc3(r, z)
    for _ in range(k):
        sem.sem_ax(mesh.handle, 0, prec, p, w, assemble=True)
        alpha = rho / glsc3(p, w)
        x += alpha * p
        r -= alpha * w
        z = minv * r
        rho_new = glsc3(r, z)
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, float(np.sqrt(glsc3(r, r) / glsc3(b, b)))


@pytest.mark.parametrize("f64x", [0, 1], ids=["f64", "f64x"])
def test_cg_mode_iterates(full, f64x):
    import torch
    sem, m, mesh = full
    info = mesh.info
    u_glob = torch.tensor(global_field(info["n_glob"], SEED, start=m.draws_used), dtype=torch.float64, device="cuda")
    x0 = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
    sem.sem_scatter(mesh.handle, 0, u_glob, x0)
    b = torch.empty_like(x0)
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, 0, b)
    k = 6
    # the benchmark's configuration: eager kernels, scalars checked every iteration
    x = x0.clone()
    cg = sem.sem_cg_create(mesh.handle, sem.sem_cg_default_opts(rtol=0.0, max_iter=1 << 30, use_graph=0,
                                                                check_every=1, f64_arith=f64x))
    sem.sem_cg_start(cg, b, x)
    sem.sem_cg_iterate_timed(cg, k)
    q = sem.sem_cg_query(cg)
    sem.sem_cg_destroy(cg)
    assert q["iters"] == k and q["status"] == sem.SEM_ERR_BUSY, q
    xr, rel_driven = _driven_cg(sem, mesh, b, x0.clone(), k, f64x)
    diff = float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr - x0))
    assert diff <= 1e-9, diff
    assert abs(q["rel_res"] - rel_driven) <= 1e-8 * rel_driven, (q["rel_res"], rel_driven)
    # recurrence residual against the true residual of the returned x (FP64 operator)
    w = torch.empty_like(b)
    sem.sem_ax(mesh.handle, 0, 0, x, w, assemble=True)
    r = b - w
    dot = torch.empty(1, dtype=torch.float64, device="cuda")
    sem.sem_glsc3(mesh.handle, 0, r, r, dot)
    rr = float(dot.item())
    sem.sem_glsc3(mesh.handle, 0, b, b, dot)
    true_rel = float(np.sqrt(rr / float(dot.item())))
    assert abs(true_rel - q["rel_res"]) <= 1e-6 * q["rel_res"], (true_rel, q["rel_res"])


@pytest.mark.parametrize("mixed", [1, 2], ids=["restarted", "reliable-updates"])
def test_mixed_solve_full_size(full, mixed):
    """FP32 on-the-fly CG (fused prologue, TMA-staged inputs, deferred x updates) inside FP64
    refinement on the full-size mesh: the solution's true residual b - A x, formed with the
    FP64 operator and the FP64 weighted dot, meets rtol."""
    import torch
    sem, m, mesh = full
    b = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, 0, b)
    x = torch.zeros_like(b)
    opts = sem.sem_cg_default_opts(rtol=1e-10, mixed=mixed, variant=sem.SEM_AX_STORED, inner_variant=sem.SEM_AX_OTF,
                                   inner_rtol=0.1 if mixed == 2 else 1e-5)
    res = sem.sem_cg_solve(mesh.handle, b, x, opts)
    assert res["status"] == sem.SEM_OK, res
    w = torch.empty_like(b)
    sem.sem_ax(mesh.handle, 0, 0, x, w, assemble=True)
    r = b - w
    dot = torch.empty(1, dtype=torch.float64, device="cuda")
    sem.sem_glsc3(mesh.handle, 0, r, r, dot)
    rr = float(dot.item())
    sem.sem_glsc3(mesh.handle, 0, b, b, dot)
    assert np.sqrt(rr / float(dot.item())) <= 1e-10 * (1 + 1e-3)
