"""Autotuning of the local operator: every candidate the tuner can choose (stored or
on-the-fly factors, both block shapes) must give the oracle's A_L (Eq. 4), and the tuned
SEM_AX_AUTO variant too; tables are keyed by the GPU model."""
import os

import numpy as np
import pytest

from oracle import sem_oracle as so
from synthetic import BoxMesh, local_field

pytestmark = pytest.mark.gpu

CASES = [((3, 2, 3), 2), ((3, 3, 2), 3), ((2, 3, 2), 5), ((3, 2, 2), 7), ((2, 2, 3), 9), ((2, 1, 2), 11)]


@pytest.fixture(scope="module")
def sem():
    import torch
    from paper_2108_12188_gb300 import build_lib, sem as sem_mod
    build_lib.build()
    sem_mod.load_library()
    torch.cuda.set_device(0)
    return sem_mod


def _check_all(sem, tmp_path, force_shape):
    import torch
    for dims, N in CASES:
        m = BoxMesh(*dims, jitter=0.12, seed=N)
        prob = so.SemProblem(N, m.vert_xyz, m.elem_verts)
        mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=7)
        u = local_field(prob.n, seed=N + 5)
        want = prob.ax_local(u).ravel()
        for prec, tol in ((sem.SEM_F64, 1e-12), (sem.SEM_F32, 2e-6)):
            rep = sem.sem_autotune(mesh.handle, prec, reps=2)
            assert len(rep["candidates"]) >= 2 and 0 <= rep["best"] < len(rep["candidates"])
            if force_shape is not None:
                path = tmp_path / "tune.txt"
                sem.sem_autotune_save(path)
                lines = path.read_text().splitlines()
                out = [lines[0]] + [" ".join(l.split()[:3] + [str(force_shape), str(force_shape), "0"]
                                             + l.split()[6:]) for l in lines[1:]]
                path.write_text("\n".join(out) + "\n")
                sem.sem_autotune_load(path)
            dt = torch.float64 if prec == sem.SEM_F64 else torch.float32
            ud = torch.tensor(u, dtype=dt, device="cuda")
            for variant in (sem.SEM_AX_STORED, sem.SEM_AX_OTF, sem.SEM_AX_OTF_SCALE, sem.SEM_AX_AUTO):
                wd = torch.empty_like(ud)
                sem.sem_ax(mesh.handle, variant, prec, ud, wd, assemble=False)
                err = np.linalg.norm(wd.double().cpu().numpy() - want) / np.linalg.norm(want)
                assert err <= tol, (N, prec, variant, force_shape, err)
        mesh.close()


@pytest.mark.parametrize("force_shape", [None, 0, 1], ids=["tuned", "shape0", "shape1"])
def test_every_candidate_matches_oracle(sem, tmp_path, force_shape):
    _check_all(sem, tmp_path, force_shape)


def test_table_from_another_gpu_is_refused(sem, tmp_path):
    path = tmp_path / "other.txt"
    path.write_text("sem-autotune 2 Some_Other_GPU\n0 7 0 0 0 0 1.0 2.0 3.0\n")
    with pytest.raises(sem.SemError) as e:
        sem.sem_autotune_load(path)
    assert e.value.status == sem.SEM_ERR_ARG
    path.write_text("not a table\n")
    with pytest.raises(sem.SemError):
        sem.sem_autotune_load(path)
