"""Thin ctypes binding of libsem (include/sem.h): same names, argument marshalling only.

Every computation happens in the library's CUDA kernels. Device buffers are torch
CUDA tensors (contiguous, of the precision the call names); the stream defaults to
torch's current stream. A missing or unloadable library raises immediately: there
is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsem.so")

SEM_OK, SEM_ERR_ARG, SEM_ERR_MESH, SEM_ERR_OOM, SEM_ERR_CUDA = 0, 1, 2, 3, 4
SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN, SEM_ERR_TIMEOUT, SEM_ERR_BUSY, SEM_ERR_UNSUPPORTED = 5, 6, 7, 8, 9
SEM_F64, SEM_F32, SEM_F64X = 0, 1, 2
SEM_AX_STORED, SEM_AX_OTF, SEM_AX_AUTO, SEM_AX_OTF_SCALE = 0, 1, 2, 3
SEM_MESH_F64_STORED, SEM_MESH_F32_STORED, SEM_MESH_OTF_SCALE, SEM_MESH_F64X_STORED = 1, 2, 4, 8
SEM_MAX_N = 11

# every symbol include/sem.h declares (checked by the tests)
EXPORTS = [
    "sem_mesh_create", "sem_mesh_numbering", "sem_mesh_destroy", "sem_mesh_get_info", "sem_mesh_get_glo_num", "sem_mesh_get_mask",
    "sem_mesh_get_segments", "sem_mesh_coords", "sem_mesh_geometry", "sem_scatter", "sem_ax", "sem_dssum",
    "sem_glsc3", "sem_glsc3_noalloc", "sem_jacobi", "sem_rhs_sine", "sem_cg_default_opts", "sem_cg_solve", "sem_cg_create",
    "sem_cg_start", "sem_cg_iterate", "sem_cg_iterate_timed", "sem_cg_query", "sem_cg_destroy", "sem_launch_count", "sem_last_error",
    "sem_status_string", "sem_server_create", "sem_server_submit", "sem_server_poll", "sem_server_stats",
    "sem_server_destroy", "sem_autotune", "sem_autotune_save", "sem_autotune_load", "sem_mesh_info",
    "sem_server_submit_mesh", "sem_probe_bounded_wait", "sem_cg_solve_batch", "sem_server_default_config",
    "sem_server_create_config", "sem_server_batch_stats", "sem_autotune_set", "sem_autotune_clear", "sem_probe_grid_barrier",
]


class SemError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class MeshInfo(C.Structure):
    _fields_ = [("N", C.c_int), ("Np", C.c_int), ("E", C.c_int64), ("n_local", C.c_int64),
                ("n_glob", C.c_int64), ("n_seg", C.c_int64), ("n_gs", C.c_int64), ("flags", C.c_uint),
                ("device", C.c_int), ("device_bytes", C.c_size_t)]


class CgOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int), ("precond", C.c_int), ("variant", C.c_int),
                ("mixed", C.c_int), ("inner_variant", C.c_int), ("inner_rtol", C.c_double),
                ("max_outer", C.c_int), ("check_every", C.c_int), ("use_graph", C.c_int), ("f64_arith", C.c_int)]


class CgResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_iters", C.c_int), ("rel_res", C.c_double), ("time_ms", C.c_double),
                ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneEntry(C.Structure):
    _fields_ = [("variant", C.c_int), ("shape", C.c_int), ("elements_per_block", C.c_int), ("ms", C.c_double)]


class TuneReport(C.Structure):
    _fields_ = [("N", C.c_int), ("prec", C.c_int), ("n_candidates", C.c_int), ("candidates", TuneEntry * 6),
                ("best", C.c_int)]

    def as_dict(self):
        cands = [{f: getattr(self.candidates[q], f) for f, _ in TuneEntry._fields_} for q in range(self.n_candidates)]
        return {"N": self.N, "prec": self.prec, "candidates": cands, "best": self.best}


class Request(C.Structure):
    _fields_ = [("N", C.c_int), ("num_vertices", C.c_int64), ("vert_xyz_host", C.c_void_p), ("E", C.c_int64),
                ("elem_verts_host", C.c_void_p), ("dirichlet_vertex_flags_host", C.c_void_p),
                ("sine", C.c_int * 3), ("opts", CgOpts)]


class ServerResult(C.Structure):
    _fields_ = [("status", C.c_int), ("n_local", C.c_int64), ("cg", CgResult), ("queue_ms", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("latency_ms", C.c_double),
                ("batched", C.c_int)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "cg"}
        d["cg"] = self.cg.as_dict()
        return d


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int), ("batch_max_points", C.c_int64),
                ("batch_max_solves", C.c_int), ("batch_round_iters", C.c_int), ("size_priorities", C.c_int)]


_lib = None
_VP, _I, _I64, _D, _U = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint


def load_library(path: str | None = None):
    """Loads libsem.so (built in-tree by build_lib); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libsem.so not found at {path}: build it first (python -m paper_2108_12188_gb300.build_lib)")
    lib = C.CDLL(path)
    sig = {
        "sem_mesh_create": [_I, _I64, _VP, _I64, _VP, _VP, _U, _VP, C.POINTER(_VP)],
        "sem_mesh_destroy": [_VP],
        "sem_mesh_numbering": [_I, _I64, _I64, _VP, _VP, _VP, _VP, C.POINTER(_I64)],
        "sem_mesh_get_info": [_VP, C.POINTER(MeshInfo)],
        "sem_mesh_info": [_VP, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)],
        "sem_probe_bounded_wait": [_I64, C.c_int, C.POINTER(C.c_double), _VP],
        "sem_probe_grid_barrier": [C.c_int, C.POINTER(C.c_double), _VP],
        "sem_mesh_get_glo_num": [_VP, _VP],
        "sem_mesh_get_mask": [_VP, _VP],
        "sem_mesh_get_segments": [_VP, _VP, _VP, _VP],
        "sem_mesh_coords": [_VP, _VP, _VP],
        "sem_mesh_geometry": [_VP, _I, _VP, _VP, _VP],
        "sem_scatter": [_VP, _I, _VP, _VP, _VP],
        "sem_ax": [_VP, _I, _I, _VP, _VP, _I, _VP],
        "sem_dssum": [_VP, _I, _VP, _I, _VP],
        "sem_glsc3": [_VP, _I, _VP, _VP, _VP, _VP],
        "sem_glsc3_noalloc": [_VP, _I, _VP, _VP, _VP, _VP],
        "sem_jacobi": [_VP, _I, _VP, _VP],
        "sem_rhs_sine": [_VP, _I, _I, _I, _I, _VP, _VP],
        "sem_cg_default_opts": [C.POINTER(CgOpts)],
        "sem_cg_solve": [_VP, _VP, _VP, C.POINTER(CgOpts), C.POINTER(CgResult), _VP],
        "sem_cg_create": [_VP, C.POINTER(CgOpts), C.POINTER(_VP)],
        "sem_cg_start": [_VP, _VP, _VP, _VP],
        "sem_cg_iterate": [_VP, _I, _VP],
        "sem_cg_query": [_VP, C.POINTER(CgResult), _VP],
        "sem_cg_iterate_timed": [_VP, _I, C.POINTER(_D), C.POINTER(_D), _VP],
        "sem_cg_destroy": [_VP],
        "sem_server_create": [C.c_size_t, _I, C.POINTER(_VP)],
        "sem_server_default_config": [C.c_size_t, _I, C.POINTER(ServerConfig)],
        "sem_server_create_config": [C.POINTER(ServerConfig), C.POINTER(_VP)],
        "sem_cg_solve_batch": [_I, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), C.POINTER(CgOpts),
                               C.POINTER(CgResult), _VP],
        "sem_server_submit": [_VP, C.POINTER(Request), C.POINTER(C.c_uint64)],
        "sem_server_submit_mesh": [_VP, _VP, _VP, C.POINTER(CgOpts), C.POINTER(C.c_uint64)],
        "sem_server_poll": [_VP, C.c_uint64, _VP, _I64, C.POINTER(ServerResult)],
        "sem_server_stats": [_VP, C.POINTER(_I), C.POINTER(_I), C.POINTER(C.c_size_t)],
        "sem_server_batch_stats": [_VP, C.POINTER(_I64), C.POINTER(_I), C.POINTER(_D)],
        "sem_server_destroy": [_VP],
        "sem_autotune": [_VP, _I, _I, C.POINTER(TuneReport), _VP],
        "sem_autotune_save": [C.c_char_p],
        "sem_autotune_load": [C.c_char_p],
        "sem_autotune_set": [_I, _I, _I, _I],
        "sem_autotune_clear": [],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = _I
    lib.sem_launch_count.argtypes, lib.sem_launch_count.restype = [], C.c_uint64
    lib.sem_last_error.argtypes, lib.sem_last_error.restype = [], C.c_char_p
    lib.sem_status_string.argtypes, lib.sem_status_string.restype = [_I], C.c_char_p
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = {0: "SEM_OK", 1: "SEM_ERR_ARG", 2: "SEM_ERR_MESH", 3: "SEM_ERR_OOM", 4: "SEM_ERR_CUDA",
             5: "SEM_ERR_NOT_CONVERGED", 6: "SEM_ERR_BREAKDOWN", 7: "SEM_ERR_TIMEOUT", 8: "SEM_ERR_BUSY",
             9: "SEM_ERR_UNSUPPORTED"}
    return names.get(s, str(s))


def _check(status: int, ok=(SEM_OK,)):
    if status not in ok:
        raise SemError(status, load_library().sem_last_error().decode())
    return status


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor, after checking dtype and size."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _torch_dtype(prec):
    import torch
    return torch.float32 if prec == SEM_F32 else torch.float64


# ---------------------------------------------------------------------------
# mesh
# ---------------------------------------------------------------------------

def sem_mesh_create(N, vert_xyz, elem_verts, dirichlet_vertex_flags=None, flags=SEM_MESH_F64_STORED, stream=None):
    lib = load_library()
    vx = np.ascontiguousarray(vert_xyz, dtype=np.float64)
    ev = np.ascontiguousarray(elem_verts, dtype=np.int64)
    if vx.ndim != 2 or vx.shape[1] != 3 or ev.ndim != 2 or ev.shape[1] != 8:
        raise ValueError("vert_xyz must be [nv, 3] and elem_verts [E, 8]")
    df = None if dirichlet_vertex_flags is None else np.ascontiguousarray(dirichlet_vertex_flags, dtype=np.uint8)
    out = _VP()
    _check(lib.sem_mesh_create(int(N), vx.shape[0], vx.ctypes.data, ev.shape[0], ev.ctypes.data,
                               None if df is None else df.ctypes.data, int(flags), _stream(stream), C.byref(out)))
    return out


def sem_mesh_numbering(N, num_vertices, elem_verts, dirichlet_vertex_flags=None):
    """Host-only numbering: returns (glo_num int64 [n], mask uint8 [n], n_glob)."""
    lib = load_library()
    ev = np.ascontiguousarray(elem_verts, dtype=np.int64)
    n = ev.shape[0] * (int(N) + 1) ** 3
    glo = np.empty(n, dtype=np.int64)
    msk = np.empty(n, dtype=np.uint8)
    df = None if dirichlet_vertex_flags is None else np.ascontiguousarray(dirichlet_vertex_flags, dtype=np.uint8)
    ng = C.c_int64()
    _check(lib.sem_mesh_numbering(int(N), int(num_vertices), ev.shape[0], ev.ctypes.data,
                                  None if df is None else df.ctypes.data, glo.ctypes.data, msk.ctypes.data,
                                  C.byref(ng)))
    return glo, msk, int(ng.value)


def sem_mesh_destroy(mesh):
    _check(load_library().sem_mesh_destroy(mesh))


def sem_mesh_get_info(mesh) -> dict:
    info = MeshInfo()
    _check(load_library().sem_mesh_get_info(mesh, C.byref(info)))
    return {f: getattr(info, f) for f, _ in MeshInfo._fields_}


def sem_mesh_info(mesh) -> tuple:
    """(n_local, n_glob, n_shared_seg) of a mesh."""
    a, b, c = _I64(), _I64(), _I64()
    _check(load_library().sem_mesh_info(mesh, C.byref(a), C.byref(b), C.byref(c)))
    return int(a.value), int(b.value), int(c.value)


def sem_probe_bounded_wait(limit_ns, issue_copy, stream=None):
    """(status, kernel ms) of the bounded-wait self-test; SEM_ERR_TIMEOUT is a result here."""
    ms = C.c_double()
    st = _check(load_library().sem_probe_bounded_wait(int(limit_ns), int(issue_copy), C.byref(ms), _stream(stream)),
                ok=(SEM_OK, SEM_ERR_TIMEOUT))
    return st, float(ms.value)


def sem_probe_grid_barrier(skip_one, stream=None):
    """(status, kernel ms) of the grid-barrier self-test; SEM_ERR_TIMEOUT is a result here."""
    ms = C.c_double()
    st = _check(load_library().sem_probe_grid_barrier(int(skip_one), C.byref(ms), _stream(stream)),
                ok=(SEM_OK, SEM_ERR_TIMEOUT))
    return st, float(ms.value)


def sem_mesh_get_glo_num(mesh) -> np.ndarray:
    n = sem_mesh_get_info(mesh)["n_local"]
    out = np.empty(n, dtype=np.int64)
    _check(load_library().sem_mesh_get_glo_num(mesh, out.ctypes.data))
    return out


def sem_mesh_get_mask(mesh) -> np.ndarray:
    n = sem_mesh_get_info(mesh)["n_local"]
    out = np.empty(n, dtype=np.uint8)
    _check(load_library().sem_mesh_get_mask(mesh, out.ctypes.data))
    return out


def sem_mesh_get_segments(mesh):
    info = sem_mesh_get_info(mesh)
    off = np.empty(info["n_seg"] + 1, dtype=np.int32)
    idx = np.empty(info["n_gs"], dtype=np.int32)
    msk = np.empty(info["n_seg"], dtype=np.uint8)
    _check(load_library().sem_mesh_get_segments(mesh, off.ctypes.data, idx.ctypes.data, msk.ctypes.data))
    return off, idx, msk


def sem_mesh_coords(mesh, xyz, stream=None):
    import torch
    n = sem_mesh_get_info(mesh)["n_local"]
    _check(load_library().sem_mesh_coords(mesh, _dev(xyz, torch.float64, 3 * n, "xyz"), _stream(stream)))


def sem_mesh_geometry(mesh, prec, G=None, B=None, stream=None):
    info = sem_mesh_get_info(mesh)
    P = info["Np"] ** 3
    dt = _torch_dtype(prec)
    _check(load_library().sem_mesh_geometry(mesh, prec, _dev(G, dt, info["E"] * 6 * P, "G"),
                                            _dev(B, dt, info["E"] * P, "B"), _stream(stream)))


def sem_scatter(mesh, prec, u_glob, u_local, stream=None):
    info = sem_mesh_get_info(mesh)
    dt = _torch_dtype(prec)
    _check(load_library().sem_scatter(mesh, prec, _dev(u_glob, dt, info["n_glob"], "u_glob"),
                                      _dev(u_local, dt, info["n_local"], "u_local"), _stream(stream)))


def sem_ax(mesh, variant, prec, u, w, assemble=True, stream=None, n_local=None):
    n = n_local if n_local is not None else sem_mesh_get_info(mesh)["n_local"]
    dt = _torch_dtype(prec)
    _check(load_library().sem_ax(mesh, variant, prec, _dev(u, dt, n, "u"), _dev(w, dt, n, "w"), int(bool(assemble)),
                                 _stream(stream)))


def sem_dssum(mesh, prec, u, apply_mask=True, stream=None):
    n = sem_mesh_get_info(mesh)["n_local"]
    _check(load_library().sem_dssum(mesh, prec, _dev(u, _torch_dtype(prec), n, "u"), int(bool(apply_mask)),
                                    _stream(stream)))


def sem_glsc3(mesh, prec, a, b, result, stream=None):
    import torch
    n = sem_mesh_get_info(mesh)["n_local"]
    dt = _torch_dtype(prec)
    _check(load_library().sem_glsc3(mesh, prec, _dev(a, dt, n, "a"), _dev(b, dt, n, "b"),
                                    _dev(result, torch.float64, 1, "result"), _stream(stream)))


def sem_glsc3_noalloc(mesh, prec, a, b, result, stream=None):
    """<a, b, c> without any device allocation (static scratch; see include/sem.h)."""
    import torch
    n = sem_mesh_get_info(mesh)["n_local"]
    dt = _torch_dtype(prec)
    _check(load_library().sem_glsc3_noalloc(mesh, prec, _dev(a, dt, n, "a"), _dev(b, dt, n, "b"),
                                            _dev(result, torch.float64, 1, "result"), _stream(stream)))


def sem_jacobi(mesh, prec, minv, stream=None):
    n = sem_mesh_get_info(mesh)["n_local"]
    _check(load_library().sem_jacobi(mesh, prec, _dev(minv, _torch_dtype(prec), n, "minv"), _stream(stream)))


def sem_rhs_sine(mesh, a, b, c, prec, rhs, stream=None):
    n = sem_mesh_get_info(mesh)["n_local"]
    _check(load_library().sem_rhs_sine(mesh, int(a), int(b), int(c), prec, _dev(rhs, _torch_dtype(prec), n, "rhs"),
                                       _stream(stream)))


# ---------------------------------------------------------------------------
# conjugate gradient
# ---------------------------------------------------------------------------

def sem_cg_default_opts(**overrides) -> CgOpts:
    o = CgOpts()
    _check(load_library().sem_cg_default_opts(C.byref(o)))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def sem_cg_solve(mesh, b, x, opts=None, stream=None, raise_on=(SEM_ERR_ARG, SEM_ERR_MESH, SEM_ERR_OOM,
                                                            SEM_ERR_CUDA, SEM_ERR_UNSUPPORTED)) -> dict:
    """Runs sem_cg_solve; returns the result as a dict (its 'status' tells convergence)."""
    import torch
    n = sem_mesh_get_info(mesh)["n_local"]
    opts = opts or sem_cg_default_opts()
    res = CgResult()
    st = load_library().sem_cg_solve(mesh, _dev(b, torch.float64, n, "b"), _dev(x, torch.float64, n, "x"),
                                     C.byref(opts), C.byref(res), _stream(stream))
    if st in raise_on:
        _check(st)
    return res.as_dict()


def sem_cg_solve_batch(meshes, bs, xs, opts=None, stream=None,
                       raise_on=(SEM_ERR_ARG, SEM_ERR_MESH, SEM_ERR_OOM, SEM_ERR_CUDA, SEM_ERR_UNSUPPORTED)) -> list:
    """Solves the problems (meshes[i], bs[i], xs[i]) together (see include/sem.h); returns one
    result dict per problem."""
    import torch
    k = len(meshes)
    if not (len(bs) == len(xs) == k):
        raise ValueError("meshes, bs and xs must have the same length")
    hm = (_VP * k)(*[m.handle if isinstance(m, Mesh) else m for m in meshes])
    ns = [sem_mesh_get_info(hm[q])["n_local"] for q in range(k)]
    hb = (_VP * k)(*[_dev(bs[q], torch.float64, ns[q], "b") for q in range(k)])
    hx = (_VP * k)(*[_dev(xs[q], torch.float64, ns[q], "x") for q in range(k)])
    res = (CgResult * k)()
    o = opts or sem_cg_default_opts(mixed=2, inner_rtol=0.1)
    st = load_library().sem_cg_solve_batch(k, hm, hb, hx, C.byref(o), res, _stream(stream))
    if st in raise_on:
        _check(st)
    return [res[q].as_dict() for q in range(k)]


def sem_cg_create(mesh, opts=None):
    out = _VP()
    _check(load_library().sem_cg_create(mesh, C.byref(opts or sem_cg_default_opts()), C.byref(out)))
    return out


def sem_cg_start(cg, b, x, stream=None):
    import torch
    _check(load_library().sem_cg_start(cg, _dev(b, torch.float64, None, "b"), _dev(x, torch.float64, None, "x"),
                                       _stream(stream)))


def sem_cg_iterate(cg, k, stream=None):
    _check(load_library().sem_cg_iterate(cg, int(k), _stream(stream)))


def sem_cg_iterate_timed(cg, k, stream=None):
    """Runs k instrumented iterations; returns (total_ms, [ax_ms, gather_scatter_ms, update_ms])."""
    total = C.c_double()
    per = (C.c_double * 3)()
    _check(load_library().sem_cg_iterate_timed(cg, int(k), C.byref(total), per, _stream(stream)))
    return total.value, [per[0], per[1], per[2]]


def sem_cg_query(cg, stream=None) -> dict:
    res = CgResult()
    _check(load_library().sem_cg_query(cg, C.byref(res), _stream(stream)))
    return res.as_dict()


def sem_cg_destroy(cg):
    _check(load_library().sem_cg_destroy(cg))


# ---------------------------------------------------------------------------
# solve server
# ---------------------------------------------------------------------------

def sem_server_default_config(hbm_budget_bytes: int, max_slots: int, **overrides) -> ServerConfig:
    cfg = ServerConfig()
    _check(load_library().sem_server_default_config(int(hbm_budget_bytes), int(max_slots), C.byref(cfg)))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def sem_server_create(hbm_budget_bytes: int, max_slots: int, **config):
    """A server with the default configuration, or with the given sem_server_config fields
    (batch_max_points, batch_max_solves, batch_round_iters) changed."""
    out = _VP()
    if config:
        cfg = sem_server_default_config(hbm_budget_bytes, max_slots, **config)
        _check(load_library().sem_server_create_config(C.byref(cfg), C.byref(out)))
    else:
        _check(load_library().sem_server_create(int(hbm_budget_bytes), int(max_slots), C.byref(out)))
    return out


def sem_server_submit(server, N, vert_xyz, elem_verts, sine=(1, 1, 1), opts=None, dirichlet_vertex_flags=None):
    vx = np.ascontiguousarray(vert_xyz, dtype=np.float64)
    ev = np.ascontiguousarray(elem_verts, dtype=np.int64)
    df = None if dirichlet_vertex_flags is None else np.ascontiguousarray(dirichlet_vertex_flags, dtype=np.uint8)
    req = Request(int(N), vx.shape[0], vx.ctypes.data, ev.shape[0], ev.ctypes.data,
                  None if df is None else df.ctypes.data, (C.c_int * 3)(*sine), opts or sem_cg_default_opts())
    ticket = C.c_uint64()
    _check(load_library().sem_server_submit(server, C.byref(req), C.byref(ticket)))  # copies the arrays
    return int(ticket.value)


def sem_server_submit_mesh(server, mesh, b_host, opts=None):
    """Queues a solve from x = 0 on a prebuilt mesh (a Mesh, which gives up its handle, or a
    raw handle) with the FP64 host right-hand side b_host (copied). The server destroys the mesh."""
    handle = mesh.handle if isinstance(mesh, Mesh) else mesh
    b = np.ascontiguousarray(b_host, dtype=np.float64)
    n, _, _ = sem_mesh_info(handle)
    if b.size != n:
        raise SemError(SEM_ERR_ARG, f"b has {b.size} values, the mesh {n} points")
    o = opts or sem_cg_default_opts()
    ticket = C.c_uint64()
    _check(load_library().sem_server_submit_mesh(server, handle, b.ctypes.data, C.byref(o), C.byref(ticket)))
    if isinstance(mesh, Mesh):
        mesh.handle = None  # now the server's
    return int(ticket.value)


def sem_server_poll(server, ticket, want_x=True):
    """None while busy; else (result dict, x as numpy array or None)."""
    lib = load_library()
    res = ServerResult()
    st = lib.sem_server_poll(server, C.c_uint64(ticket), None, 0, C.byref(res))
    if st == SEM_ERR_BUSY:
        return None
    _check(st)
    x = None
    if want_x:
        x = np.empty(res.n_local, dtype=np.float64)
        _check(lib.sem_server_poll(server, C.c_uint64(ticket), x.ctypes.data, x.size, C.byref(res)))
    return res.as_dict(), x


def sem_server_stats(server):
    q, a, b = _I(), _I(), C.c_size_t()
    _check(load_library().sem_server_stats(server, C.byref(q), C.byref(a), C.byref(b)))
    return {"queued": q.value, "active": a.value, "bytes_in_use": b.value}


def sem_server_batch_stats(server):
    r, m, a = _I64(), _I(), _D()
    _check(load_library().sem_server_batch_stats(server, C.byref(r), C.byref(m), C.byref(a)))
    return {"rounds": int(r.value), "max_batch": int(m.value), "mean_batch": float(a.value)}


def sem_server_destroy(server):
    _check(load_library().sem_server_destroy(server))


def sem_autotune(mesh, prec, reps=10, stream=None) -> dict:
    rep = TuneReport()
    _check(load_library().sem_autotune(mesh, int(prec), int(reps), C.byref(rep), _stream(stream)))
    return rep.as_dict()


def sem_autotune_set(N, prec, variant, shape):
    _check(load_library().sem_autotune_set(int(N), int(prec), int(variant), int(shape)))


def sem_autotune_clear():
    _check(load_library().sem_autotune_clear())


SEM_TENSOR_SHAPE = 3


def sem_autotune_save(path):
    _check(load_library().sem_autotune_save(str(path).encode()))


def sem_autotune_load(path):
    _check(load_library().sem_autotune_load(str(path).encode()))


def sem_launch_count() -> int:
    return int(load_library().sem_launch_count())


def sem_status_string(s: int) -> str:
    return load_library().sem_status_string(int(s)).decode()


class Mesh:
    """Owns a sem_mesh handle; frees it on close() or garbage collection."""

    def __init__(self, N, vert_xyz, elem_verts, dirichlet_vertex_flags=None, flags=SEM_MESH_F64_STORED, stream=None):
        self.handle = sem_mesh_create(N, vert_xyz, elem_verts, dirichlet_vertex_flags, flags, stream)
        self.info = sem_mesh_get_info(self.handle)
        self.n = self.info["n_local"]

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            sem_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
