"""sem_glsc3_noalloc: the weighted inner product for callers that cannot let the library
allocate device memory (programs that own all device memory through their own pool, or loops
that cannot take cudaMalloc's device-wide synchronisation). Its scratch is a static device
array, so it is checked against sem_glsc3 (the allocating entry point) and against the
oracle's <a, b, c> on two calls in a row, on meshes whose point counts give one block (fewer
points than one chunk), a ragged last chunk, and many chunks; and its size limit is checked.
Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

from synthetic import BoxMesh, local_field

pytestmark = pytest.mark.gpu

MAX_POINTS = 4096 * 8192
CHUNK = 8192


@pytest.fixture(scope="module")
def sem():
    import torch
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    torch.cuda.set_device(0)
    return sem_mod


# (nx, ny, nz, N): 5,832 points (one block, which is also the last); 61,440 points (8
# chunks, the last one short); 658,560 points (81 chunks, the last one short)
MESHES = [(3, 3, 3, 5), (6, 5, 4, 7), (16, 12, 10, 6)]


@pytest.mark.parametrize("shape", MESHES, ids=["one_block", "ragged", "many_chunks"])
@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_noalloc_matches_glsc3_and_oracle_twice(sem, prec, shape):
    import torch
    from oracle import sem_oracle as so
    nx, ny, nz, N = shape
    m = BoxMesh(nx, ny, nz, jitter=0.1, seed=4)
    mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=0)
    assert mesh.n % CHUNK != 0 and (mesh.n < CHUNK) == (shape == MESHES[0])
    dt = torch.float64 if prec == 0 else torch.float32
    a = torch.tensor(local_field(mesh.n, seed=21), dtype=dt, device="cuda")
    b = torch.tensor(local_field(mesh.n, seed=22), dtype=dt, device="cuda")
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    sem.sem_glsc3(mesh.handle, prec, a, b, ref)
    c = so.number_nodes(N, m.elem_verts).c()
    want = so.glsc3(a.double().cpu().numpy(), b.double().cpu().numpy(), c)
    lib = sem.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    scale = float(torch.sum(torch.abs(a.double() * b.double())))
    for call in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.sem_glsc3_noalloc(mesh.handle, prec, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == sem.SEM_OK, lib.sem_last_error()
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= 1e-13 * scale, (call, out.item(), ref.item())
        assert abs(out.item() - want) <= 1e-13 * scale, (call, out.item(), want)
    mesh.close()


def test_noalloc_rejects_meshes_beyond_its_scratch(sem):
    import torch
    m = BoxMesh(27, 27, 27)  # N = 11: 19,683 x 1728 = 34,012,224 local points > 33,554,432
    mesh = sem.Mesh(11, m.vert_xyz, m.elem_verts, flags=0)
    assert mesh.n > MAX_POINTS
    a = torch.zeros(mesh.n, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        sem.sem_glsc3_noalloc(mesh.handle, sem.SEM_F32, a, a, out)
    assert e.value.status == sem.SEM_ERR_ARG and "at most 33554432" in str(e.value)
    mesh.close()
