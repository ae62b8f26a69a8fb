"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only input generation: a counter-based random stream, the
vertex coordinates and connectivity of jittered box meshes, and random fields
drawn per node. It contains none of the spectral-element arithmetic (no GLL
points, no geometric factors, no operator), so both the CPU oracle and the CUDA
path may use it without sharing any of the method.

Workload shapes follow Section 6 of the paper: cubic domains meshed with
E = 128 ... 32768 hexahedra, linearly deformed (Section 5.1 restricts the
on-the-fly variant to linearly deformed hexahedra), here produced by jittering
the interior vertices of a uniform box mesh.

Random stream: SplitMix64. Draw k (k = 0, 1, 2, ...) of the stream with seed s
is mix(s + (k + 1) * 0x9E3779B97F4A7C15) where mix is the SplitMix64 output
function (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014). A uniform double in [0, 1) is (x >> 11) * 2**-53.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from draws start .. start+count-1."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class BoxMesh:
    """A jittered nx*ny*nz hexahedral mesh of the box [0,Lx]x[0,Ly]x[0,Lz].

    vert_xyz   : float64 [num_vertices, 3]; vertex id = ix + (nx+1)*(iy + (ny+1)*iz)
    elem_verts : int64 [E, 8]; element id = ex + nx*(ey + ny*ez); local vertex
                 a + 2b + 4c sits at (ex+a, ey+b, ez+c) (tensor order, a along x).
    Interior vertices are moved by U(-jitter*h, jitter*h) per coordinate
    (h the cell size along that axis); boundary vertices stay on the box faces.
    The draws are taken in ascending vertex id, x then y then z, interior
    vertices only, from draw 0 of stream `seed`.  `draws_used` is the number of
    draws consumed, so follow-up fields can continue the same stream.
    """

    def __init__(self, nx: int, ny: int, nz: int, jitter: float = 0.0, seed: int = 0,
                 lengths=(1.0, 1.0, 1.0)):
        if min(nx, ny, nz) < 1:
            raise ValueError("box mesh needs at least one element per direction")
        self.nx, self.ny, self.nz = nx, ny, nz
        self.jitter, self.seed = float(jitter), int(seed)
        Lx, Ly, Lz = (float(v) for v in lengths)
        hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
        iz, iy, ix = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
        xyz = np.stack([ix * hx, iy * hy, iz * hz], axis=1).astype(np.float64)
        interior = (ix > 0) & (ix < nx) & (iy > 0) & (iy < ny) & (iz > 0) & (iz < nz)
        n_int = int(interior.sum())
        self.draws_used = 0
        if self.jitter != 0.0 and n_int > 0:
            r = uniform01(self.seed, 0, 3 * n_int).reshape(n_int, 3)
            h = np.array([hx, hy, hz])
            xyz[interior] += (2.0 * r - 1.0) * self.jitter * h
            self.draws_used = 3 * n_int
        self.vert_xyz = np.ascontiguousarray(xyz)
        ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
        ev = np.empty((ex.size, 8), dtype=np.int64)
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    ev[:, a + 2 * b + 4 * c] = (ex + a) + (nx + 1) * ((ey + b) + (ny + 1) * (ez + c))
        self.elem_verts = np.ascontiguousarray(ev)

    @property
    def num_elements(self) -> int:
        return self.elem_verts.shape[0]

    @property
    def num_vertices(self) -> int:
        return self.vert_xyz.shape[0]


def global_field(n_glob: int, seed: int, start: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """One U(lo, hi) value per global node, in global-id order, from draw `start` on."""
    return lo + (hi - lo) * uniform01(seed, start, n_glob)


def local_field(n_local: int, seed: int, start: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """One U(lo, hi) value per local (replicated) node: a discontinuous field."""
    return lo + (hi - lo) * uniform01(seed, start, n_local)


def n_for_points(Np: int, target_points: int = 16_777_216) -> int:
    """Elements per direction so that n^3 * Np^3 is close to target_points."""
    return int(round((target_points / Np ** 3) ** (1.0 / 3.0)))
