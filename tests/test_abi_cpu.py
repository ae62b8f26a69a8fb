"""CPU-side checks of the C ABI: the library builds and loads, exports every symbol
include/sem.h declares, and its host mesh builder (Section 3.1's numbering Q, the
Dirichlet mask of Algorithm 1 step 7) matches the oracle bit for bit."""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh
from tests.test_oracle_numbering import _reorient

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def sem():
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    return sem_mod


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "sem.h")).read()
    return set(re.findall(r"^\s*(?:sem_status|uint64_t|const char\*)\s+(sem_\w+)\s*\(", text, flags=re.M))


def test_exports_every_declared_symbol(sem):
    declared = _header_symbols()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", sem.LIB_PATH], capture_output=True, text=True, check=True)
    exported = {line.split()[-1] for line in out.stdout.splitlines() if " T " in line}
    assert declared <= exported, declared - exported
    assert declared == set(sem.EXPORTS)


@pytest.mark.parametrize("n,N,jitter", [((1, 1, 1), 1, 0.0), ((2, 1, 1), 2, 0.0), ((3, 2, 2), 3, 0.2),
                                         ((4, 4, 4), 7, 0.1), ((2, 3, 2), 11, 0.1)])
def test_host_numbering_matches_oracle(sem, n, N, jitter):
    m = BoxMesh(*n, jitter=jitter, seed=3)
    glo, mask, n_glob = sem.sem_mesh_numbering(N, m.num_vertices, m.elem_verts)
    num = so.number_nodes(N, m.elem_verts)
    assert n_glob == num.n_glob
    np.testing.assert_array_equal(glo, num.glo_num)
    np.testing.assert_array_equal(mask, num.mask)


@pytest.mark.parametrize("N", [2, 3, 6])
def test_host_numbering_reoriented_elements(sem, N):
    m = BoxMesh(3, 3, 2, jitter=0.2, seed=9)
    ev = _reorient(m.elem_verts, np.random.default_rng(100 + N))
    glo, mask, n_glob = sem.sem_mesh_numbering(N, m.num_vertices, ev)
    num = so.number_nodes(N, ev)
    np.testing.assert_array_equal(glo, num.glo_num)
    np.testing.assert_array_equal(mask, num.mask)


def test_host_numbering_dirichlet_flags(sem):
    m = BoxMesh(2, 2, 3)
    flags = (m.vert_xyz[:, 0] == 0.0).astype(np.uint8) | (m.vert_xyz[:, 2] == 1.0).astype(np.uint8)
    glo, mask, _ = sem.sem_mesh_numbering(4, m.num_vertices, m.elem_verts, flags)
    num = so.number_nodes(4, m.elem_verts, flags)
    np.testing.assert_array_equal(glo, num.glo_num)
    np.testing.assert_array_equal(mask, num.mask)


def test_host_numbering_full_size_properties(sem):
    # the 32^3, N = 7 Ax-throughput mesh: counts and first-occurrence order (Eq. 9)
    m = BoxMesh(32, 32, 32, jitter=0.15, seed=1)
    glo, mask, n_glob = sem.sem_mesh_numbering(7, m.num_vertices, m.elem_verts)
    assert n_glob == 225 ** 3
    first = np.maximum.accumulate(glo)
    assert first[0] == 0 and np.all(np.diff(first) <= 1) and first[-1] == n_glob - 1
    mult = np.bincount(glo, minlength=n_glob)
    assert int((mult == 8).sum()) == 31 ** 3 and set(np.unique(mult)) == {1, 2, 4, 8}
    assert int((mult == 1).sum()) == 32 ** 3 * 6 ** 3 + 6 * 32 ** 2 * 6 ** 2 + 12 * 32 * 6 + 8
    assert len(np.unique(glo[mask == 0])) == 223 ** 3


def test_host_errors(sem):
    m = BoxMesh(1, 1, 1)
    ev = m.elem_verts.copy()
    ev[0, 1] = ev[0, 0]
    with pytest.raises(sem.SemError) as e:
        sem.sem_mesh_numbering(3, m.num_vertices, ev)
    assert e.value.status == sem.SEM_ERR_MESH
    ev = m.elem_verts.copy()
    ev[0, 2] = 99
    with pytest.raises(sem.SemError) as e:
        sem.sem_mesh_numbering(3, m.num_vertices, ev)
    assert e.value.status == sem.SEM_ERR_MESH
    for N in (0, 12):
        with pytest.raises(sem.SemError) as e:
            sem.sem_mesh_numbering(N, m.num_vertices, m.elem_verts)
        assert e.value.status == sem.SEM_ERR_UNSUPPORTED
    # empty mesh
    with pytest.raises(sem.SemError) as e:
        sem.sem_mesh_numbering(3, m.num_vertices, np.empty((0, 8), dtype=np.int64))
    assert e.value.status == sem.SEM_ERR_ARG
    # largest size: E (N+1)^3 must stay below 2^31 (checked before any vertex is read)
    lib = sem.load_library()
    E_max = (1 << 31) // 12 ** 3
    ev_big = np.zeros((E_max + 1, 8), dtype=np.int64)
    glo, msk, ng = np.empty(1, dtype=np.int64), np.empty(1, dtype=np.uint8), sem.C.c_int64()
    st = lib.sem_mesh_numbering(11, 8, E_max + 1, ev_big.ctypes.data, None, glo.ctypes.data, msk.ctypes.data,
                                sem.C.byref(ng))
    assert st == sem.SEM_ERR_ARG
    # three hexahedra on one face: not a manifold mesh
    ev3 = np.concatenate([m.elem_verts, m.elem_verts[:, [0, 1, 2, 3, 4, 5, 6, 7]] + 0], axis=0)
    with pytest.raises(sem.SemError):
        sem.sem_mesh_numbering(2, m.num_vertices, np.concatenate([ev3, m.elem_verts]))


def _golden_hashes():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "numbering_hashes.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, N, n_glob, hg, hm = line.split()
            out[(int(n), int(N))] = (int(n_glob), hg, hm)
    return out


@pytest.mark.parametrize("n,N", [(32, 7), (20, 3), (9, 11)])
def test_host_numbering_full_size_hash(sem, n, N):
    # the oracle's numbering of these full-size meshes, pinned by SHA-256
    # (tests/golden/make_numbering_hashes.py, which calls only the oracle)
    import hashlib
    n_glob, hg, hm = _golden_hashes()[(n, N)]
    m = BoxMesh(n, n, n, jitter=0.15, seed=1)
    glo, mask, ng = sem.sem_mesh_numbering(N, m.num_vertices, m.elem_verts)
    assert ng == n_glob
    assert hashlib.sha256(glo.astype("<i8").tobytes()).hexdigest() == hg
    assert hashlib.sha256(mask.tobytes()).hexdigest() == hm


def test_null_handles_are_argument_errors(sem):
    """Calls with a null handle or output pointer return SEM_ERR_ARG (and touch no device)."""
    lib = sem.load_library()
    a = sem.C.c_int64()
    assert lib.sem_mesh_info(None, sem.C.byref(a), None, None) == sem.SEM_ERR_ARG
    opts = sem.sem_cg_default_opts()
    t = sem.C.c_uint64()
    b = np.zeros(4)
    assert lib.sem_server_submit_mesh(None, None, b.ctypes.data, sem.C.byref(opts), sem.C.byref(t)) == sem.SEM_ERR_ARG
    assert lib.sem_mesh_destroy(None) == sem.SEM_OK
    assert lib.sem_server_destroy(None) == sem.SEM_OK
    assert "null" in lib.sem_last_error().decode()


def test_probe_argument_errors(sem):
    """The bounded-wait self-test validates its arguments before touching a device."""
    lib = sem.load_library()
    ms = sem.C.c_double()
    assert lib.sem_probe_bounded_wait(10, 0, sem.C.byref(ms), None) == sem.SEM_ERR_ARG  # below 1 ms
    assert lib.sem_probe_bounded_wait(3_000_000_000, 0, sem.C.byref(ms), None) == sem.SEM_ERR_ARG
    assert lib.sem_probe_bounded_wait(20_000_000, 0, None, None) == sem.SEM_ERR_ARG


def test_tuner_table_rules(sem):
    """sem_autotune_set validates on the host: shape 1 is not offered for double-float or the
    per-point-scale variant, shape 3 only where the tensor-core operator is compiled (FP32 on
    the fly, N = 7); double-float takes the stored and on-the-fly variants."""
    lib = sem.load_library()
    try:
        assert lib.sem_autotune_set(7, sem.SEM_F64X, sem.SEM_AX_OTF, 0) == sem.SEM_OK
        assert lib.sem_autotune_set(7, sem.SEM_F64X, sem.SEM_AX_STORED, 0) == sem.SEM_OK
        assert lib.sem_autotune_set(7, sem.SEM_F64X, sem.SEM_AX_OTF, 1) == sem.SEM_ERR_ARG
        assert lib.sem_autotune_set(7, sem.SEM_F32, sem.SEM_AX_OTF_SCALE, 1) == sem.SEM_ERR_ARG
        assert lib.sem_autotune_set(7, sem.SEM_F32, sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE) == sem.SEM_OK
        assert lib.sem_autotune_set(5, sem.SEM_F32, sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE) == sem.SEM_ERR_ARG
        assert lib.sem_autotune_set(7, sem.SEM_F64, sem.SEM_AX_STORED, sem.SEM_TENSOR_SHAPE) == sem.SEM_ERR_ARG
        assert lib.sem_autotune_set(0, sem.SEM_F64, sem.SEM_AX_STORED, 0) == sem.SEM_ERR_UNSUPPORTED
        assert lib.sem_autotune_set(7, sem.SEM_F64, 9, 0) == sem.SEM_ERR_ARG
    finally:
        assert lib.sem_autotune_clear() == sem.SEM_OK


def test_batch_and_server_config_argument_errors(sem):
    """The batched solver and the server configuration check their arguments on the host,
    before any device call."""
    lib = sem.load_library()
    opts = sem.sem_cg_default_opts(mixed=2, inner_rtol=0.1)
    res = (sem.CgResult * 2)()
    ptrs = (sem.C.c_void_p * 2)(None, None)
    assert lib.sem_cg_solve_batch(0, ptrs, ptrs, ptrs, sem.C.byref(opts), res, None) == sem.SEM_ERR_ARG
    assert lib.sem_cg_solve_batch(257, ptrs, ptrs, ptrs, sem.C.byref(opts), res, None) == sem.SEM_ERR_ARG
    assert lib.sem_cg_solve_batch(1, None, ptrs, ptrs, sem.C.byref(opts), res, None) == sem.SEM_ERR_ARG
    assert lib.sem_cg_solve_batch(1, ptrs, ptrs, ptrs, sem.C.byref(opts), res, None) == sem.SEM_ERR_ARG  # null mesh
    cfg = sem.sem_server_default_config(1 << 30, 4)
    assert cfg.batch_max_points == 2097152 and cfg.batch_round_iters == 20 and cfg.size_priorities == 1
    out = sem.C.c_void_p()
    for field, value in (("max_slots", 0), ("max_slots", 257), ("hbm_budget_bytes", 0), ("batch_max_solves", 0),
                         ("batch_max_solves", 257), ("batch_round_iters", 0), ("batch_max_points", -1)):
        bad = sem.sem_server_default_config(1 << 30, 4)
        setattr(bad, field, value)
        assert lib.sem_server_create_config(sem.C.byref(bad), sem.C.byref(out)) == sem.SEM_ERR_ARG, field
        assert out.value is None
