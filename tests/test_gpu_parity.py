"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same
seeded inputs. Gates: numbering, segments, mask and gather-scatter bit-exact; FP64 Ax
within 1e-12 relative 2-norm, FP32 Ax within 2e-6 of the FP64 oracle; geometry,
Jacobi diagonal, RHS and dot products to FP64 rounding.

Passages: Section 3 Eqs. 3-5 (basis, A_L = D^T G D, QQ^T), Section 4.2 (six factors per
point), Section 4.3 Eq. 9 (element-boundary points), Section 5.1 (on-the-fly factors),
Algorithm 1 (mask, weighted inner product)."""
import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh, global_field, local_field

pytestmark = pytest.mark.gpu

FLAGS_ALL = 15  # SEM_MESH_F64_STORED | SEM_MESH_F32_STORED | SEM_MESH_OTF_SCALE | SEM_MESH_F64X_STORED


@pytest.fixture(scope="module")
def sem():
    import torch
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    torch.cuda.set_device(0)
    return sem_mod


_CACHE = {}


def _case(sem, dims, N, jitter, seed):
    """(oracle problem, library mesh) for a jittered box; cached per module run."""
    key = (dims, N, jitter, seed)
    if key not in _CACHE:
        m = BoxMesh(*dims, jitter=jitter, seed=seed)
        prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
        mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=FLAGS_ALL)
        _CACHE[key] = (m, prob, mesh)
    return _CACHE[key]


def _t(x, prec):
    import torch
    return torch.tensor(np.ascontiguousarray(x).ravel(), dtype=torch.float32 if prec == 1 else torch.float64,
                        device="cuda")


def _h(t):
    return t.double().cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [((4, 4, 4), 7, 0.1, 0), ((5, 3, 1), 7, 0.15, 2), ((3, 2, 2), 1, 0.1, 3), ((3, 3, 2), 2, 0.1, 4),
         ((2, 3, 3), 3, 0.15, 5), ((3, 2, 3), 4, 0.1, 6), ((2, 2, 3), 5, 0.1, 7), ((2, 2, 2), 6, 0.1, 8),
         ((3, 1, 2), 8, 0.1, 9), ((2, 2, 1), 9, 0.1, 10), ((1, 2, 2), 10, 0.1, 11), ((2, 1, 2), 11, 0.1, 12),
         ((1, 1, 1), 7, 0.0, 13)]  # the last: a single element, a grid of one partial element group
IDS = [f"{d[0]}x{d[1]}x{d[2]}-N{N}" for d, N, _, _ in CASES]


@pytest.mark.parametrize("dims,N,jitter,seed", CASES, ids=IDS)
def test_numbering_segments_mask(sem, dims, N, jitter, seed):
    m, prob, mesh = _case(sem, dims, N, jitter, seed)
    info = mesh.info
    assert info["n_glob"] == prob.num.n_glob
    assert info["n_gs"] == prob.E * ((N + 1) ** 3 - (N - 1) ** 3)  # Eq. 9
    np.testing.assert_array_equal(sem.sem_mesh_get_glo_num(mesh.handle), prob.glo_num)
    np.testing.assert_array_equal(sem.sem_mesh_get_mask(mesh.handle), prob.mask)
    # segments: global nodes with copies on element boundaries, ascending id, copies ascending
    Np = N + 1
    k, j, i = np.meshgrid(np.arange(Np), np.arange(Np), np.arange(Np), indexing="ij")
    bd = np.tile(((i % N == 0) | (j % N == 0) | (k % N == 0)).ravel(), prob.E)
    loc = np.flatnonzero(bd)
    order = np.lexsort((loc, prob.glo_num[loc]))
    want_idx = loc[order]
    gl = prob.glo_num[want_idx]
    starts = np.flatnonzero(np.r_[True, gl[1:] != gl[:-1]])
    off, idx, smask = sem.sem_mesh_get_segments(mesh.handle)
    np.testing.assert_array_equal(idx, want_idx)
    np.testing.assert_array_equal(off, np.r_[starts, gl.size])
    np.testing.assert_array_equal(smask, prob.mask[want_idx[starts]])


@pytest.mark.parametrize("dims,N,jitter,seed", CASES[:4] + CASES[-1:], ids=IDS[:4] + IDS[-1:])
def test_geometry(sem, dims, N, jitter, seed):
    import torch
    m, prob, mesh = _case(sem, dims, N, jitter, seed)
    P = (N + 1) ** 3
    G = torch.empty(prob.E * 6 * P, dtype=torch.float64, device="cuda")
    B = torch.empty(prob.E * P, dtype=torch.float64, device="cuda")
    sem.sem_mesh_geometry(mesh.handle, sem.SEM_F64, G, B)
    Gw = prob.G.reshape(prob.E, 6, P)
    np.testing.assert_allclose(_h(G).reshape(prob.E, 6, P), Gw, rtol=0, atol=1e-14 * np.abs(Gw).max())
    np.testing.assert_allclose(_h(B), prob.B.ravel(), rtol=1e-13)
    G32 = torch.empty(prob.E * 6 * P, dtype=torch.float32, device="cuda")
    sem.sem_mesh_geometry(mesh.handle, sem.SEM_F32, G32, None)
    np.testing.assert_allclose(_h(G32).reshape(prob.E, 6, P), Gw, rtol=0, atol=1e-7 * np.abs(Gw).max())
    xyz = torch.empty(3 * prob.n, dtype=torch.float64, device="cuda")
    sem.sem_mesh_coords(mesh.handle, xyz)
    want = prob.coords().reshape(-1, 3).T.ravel()
    np.testing.assert_allclose(_h(xyz), want, rtol=0, atol=4e-15)


VARIANTS = [(0, 0, 1e-12), (1, 0, 1e-12), (0, 1, 2e-6), (1, 1, 2e-6), (0, 2, 1e-12), (1, 2, 1e-12), (3, 0, 1e-12),
            (3, 1, 2e-6)]  # (variant, prec, tol)
VIDS = ["stored-f64", "otf-f64", "stored-f32", "otf-f32", "stored-f64x", "otf-f64x", "otfscale-f64", "otfscale-f32"]


@pytest.mark.parametrize("variant,prec,tol", VARIANTS, ids=VIDS)
@pytest.mark.parametrize("dims,N,jitter,seed", CASES, ids=IDS)
def test_ax_local(sem, dims, N, jitter, seed, variant, prec, tol):
    m, prob, mesh = _case(sem, dims, N, jitter, seed)
    u = local_field(prob.n, seed=seed + 100)  # discontinuous: tests A_L element by element
    want = prob.ax_local(u).ravel()  # the FP64 oracle on the unrounded input
    ud = _t(u, prec)
    wd = ud.new_empty(ud.shape)
    sem.sem_ax(mesh.handle, variant, prec, ud, wd, assemble=False)
    err = _rel(_h(wd), want)
    assert err <= tol, err


@pytest.mark.parametrize("dims,N,jitter,seed", CASES[:3] + CASES[-1:], ids=IDS[:3] + IDS[-1:])
def test_ax_f64x_from_fp64_factors(sem, dims, N, jitter, seed):
    """SEM_F64X on a mesh without float-pair factors: the kernel splits the FP64 factors."""
    m = BoxMesh(*dims, jitter=jitter, seed=seed)
    prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=1)
    u = local_field(prob.n, seed=seed + 300)
    ud = _t(u, 0)
    wd = ud.new_empty(ud.shape)
    sem.sem_ax(mesh.handle, 0, 2, ud, wd, assemble=False)
    mesh.close()
    assert _rel(_h(wd), prob.ax_local(u).ravel()) <= 1e-12


@pytest.mark.parametrize("variant,prec,tol", VARIANTS, ids=VIDS)
@pytest.mark.parametrize("dims,N,jitter,seed", CASES[:3] + CASES[6:7], ids=IDS[:3] + IDS[6:7])
def test_ax_assembled(sem, dims, N, jitter, seed, variant, prec, tol):
    m, prob, mesh = _case(sem, dims, N, jitter, seed)
    u = so.scatter_local(global_field(prob.num.n_glob, seed=seed + 200), prob.glo_num)
    want = prob.ax(u).ravel()
    ud = _t(u, prec)
    wd = ud.new_empty(ud.shape)
    sem.sem_ax(mesh.handle, variant, prec, ud, wd, assemble=True)
    got = _h(wd)
    assert _rel(got, want) <= tol
    assert np.all(got[prob.mask != 0] == 0)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("apply_mask", [0, 1])
@pytest.mark.parametrize("dims,N,jitter,seed", CASES[:2] + CASES[8:9], ids=IDS[:2] + IDS[8:9])
def test_dssum_bit_exact(sem, dims, N, jitter, seed, prec, apply_mask):
    m, prob, mesh = _case(sem, dims, N, jitter, seed)
    dt = np.float64 if prec == 0 else np.float32
    w = local_field(prob.n, seed=seed + 300, lo=-1e3, hi=1e3).astype(dt)
    want = so.dssum(w, prob.glo_num, prob.mask if apply_mask else None, dtype=dt)
    wd = _t(w, prec)
    sem.sem_dssum(mesh.handle, prec, wd, apply_mask)
    got = wd.cpu().numpy()
    assert got.dtype == dt
    np.testing.assert_array_equal(got.view(np.uint64 if prec == 0 else np.uint32),
                                  want.view(np.uint64 if prec == 0 else np.uint32))


@pytest.mark.parametrize("dims,N,jitter,seed", CASES[:2], ids=IDS[:2])
def test_glsc3_jacobi_rhs_scatter(sem, dims, N, jitter, seed):
    import torch
    m, prob, mesh = _case(sem, dims, N, jitter, seed)
    a, b = local_field(prob.n, seed=1), local_field(prob.n, seed=2)
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    sem.sem_glsc3(mesh.handle, sem.SEM_F64, _t(a, 0), _t(b, 0), res)
    want = so.glsc3(a, b, prob.c)
    assert abs(res.item() - want) <= 1e-13 * np.sum(np.abs(a * b * prob.c))
    minv = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    sem.sem_jacobi(mesh.handle, sem.SEM_F64, minv)
    np.testing.assert_allclose(_h(minv), prob.jacobi_inverse().ravel(), rtol=1e-13, atol=0)
    rhs = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 2, 3, sem.SEM_F64, rhs)
    want = prob.rhs(1, 2, 3).ravel()
    np.testing.assert_allclose(_h(rhs), want, rtol=0, atol=1e-13 * np.abs(want).max())
    ug = global_field(prob.num.n_glob, seed=4)
    ul = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    sem.sem_scatter(mesh.handle, sem.SEM_F64, _t(ug, 0), ul)
    np.testing.assert_array_equal(_h(ul), so.scatter_local(ug, prob.glo_num))


def test_invalid_inputs(sem):
    import torch
    m = BoxMesh(2, 1, 1)
    X = m.vert_xyz.copy()
    ev = m.elem_verts.copy()
    ev[0, [0, 1]] = ev[0, [1, 0]]  # fold element 0 inside out: det J < 0
    with pytest.raises(sem.SemError) as e:
        sem.Mesh(3, X, ev)
    assert e.value.status == sem.SEM_ERR_MESH
    mesh = sem.Mesh(3, X, m.elem_verts, flags=sem.SEM_MESH_F64_STORED)
    u = torch.zeros(mesh.n, dtype=torch.float32, device="cuda")
    w = torch.zeros_like(u)
    with pytest.raises(sem.SemError) as e:  # FP32 stored factors were not requested
        sem.sem_ax(mesh.handle, sem.SEM_AX_STORED, sem.SEM_F32, u, w)
    assert e.value.status == sem.SEM_ERR_ARG
    u64, w64 = torch.zeros(mesh.n, dtype=torch.float64, device="cuda"), torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:  # double-float arithmetic has no stored-scale variant
        sem.sem_ax(mesh.handle, sem.SEM_AX_OTF_SCALE, sem.SEM_F64X, u64, w64)
    assert e.value.status in (sem.SEM_ERR_UNSUPPORTED, sem.SEM_ERR_ARG)
    u64 = torch.zeros(mesh.n + 1, dtype=torch.float64, device="cuda")
    lib = sem.load_library()
    st = lib.sem_ax(mesh.handle, 0, 0, u64.data_ptr() + 8, u64.data_ptr(), 0, None)  # misaligned
    assert st == sem.SEM_ERR_ARG
    mesh.close()
