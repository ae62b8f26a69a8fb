"""Benchmark of the spectral-element hot path on GB300.

Workload: the Ax-throughput configuration - a 32 x 32 x 32 box of hexahedra on [0,1]^3,
interior vertices jittered by U(-0.15h, 0.15h) (seed 1), order N = 7, 16,777,216 local
points. One step = one Jacobi-preconditioned CG iteration (Algorithm 1) on the device:
the local operator A_L with FP64 stored geometric factors and the fused p = z + beta p
prologue, the gather-scatter QQ^T with the Dirichlet mask and <p, w, c>, and the fused
x / r / z update with <r, z, c> and <r, r, c>. Every step moves more than L2 (1.1 GB).
value = local points per step / device time per step (GDOF/s), aggregated over ranks.

Also reported: the local operator alone for FP64/FP32 x stored/on-the-fly factors (with
L2 flushed between timed calls) with its error against the FP64 oracle on sampled
elements; the end-to-end rate through sem_cg_solve with pinned host buffers; the oracle
on the host cores (cpu_baseline); SM clocks during the timed region. Two legs cover the rest
of the metric (rank 0; --no-legs skips them): solve_c3, the 64^3 full solve to 1e-10 by FP64
CG, by FP32 CG with FP64 reliable updates and by double-float CG (seconds, iterations, true
residual, error to the manufactured solution); serve_c5, 1000 served solve requests at one
arrival rate (p50/p99 latency, solves/s), with the server's batch of small requests.

python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--no-legs]
python bench.py --workload solve|serve|sweep   (the full solve, serving and order-sweep studies)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ax GDOF/s & %roofline (FP64/FP32); CG time to 1e-10; served p50/p99 latency"
WORKLOAD = ("32x32x32 hexahedra on [0,1]^3, interior vertices jittered +-0.15h (seed 1), N=7, "
            "16,777,216 local points; step = one Jacobi-PCG iteration, FP64 stored geometric factors")
NEL, NORD, JITTER, SEED = 32, 7, 0.15, 1
HBM_FALLBACK_GBS = 6800.0
# FP64 / FP32 FMA issue rates of a GB300 SM (2 and 128 per clock; the FP64 rate was
# measured at 1.91 FMA/clk/SM with an FMA-chain probe) x 152 SMs x 2070 MHz x 2 flop.
SMS, CLK_MHZ = 152, 2070.0
PEAK_FP64_TFLOPS = SMS * 2 * 2 * CLK_MHZ * 1e6 / 1e12      # 1.259
PEAK_FP32_TFLOPS = SMS * 128 * 2 * CLK_MHZ * 1e6 / 1e12    # 80.5


def flops_eq11(N: int) -> int:
    """Eq. 11: flops of A_L per local point, 12(N+1) + 15."""
    return 12 * (N + 1) + 15


def ax_bytes_per_point(variant: str, prec: str, N: int) -> float:
    """Algorithmic bytes of one A_L application per local point (u read, w written, factors)."""
    word = 8 if prec == "f64" else 4
    P = (N + 1) ** 3
    if variant == "stored":
        return word * (1 + 1 + 6)
    if variant == "otfscale":  # u, w and the per-point scale w/det J, plus the coefficients
        return word * (1 + 1 + 1) + word * 21 / P
    return word * (1 + 1) + word * 21 / P  # 21 trilinear coefficients per element


def cg_bytes_per_point(N: int) -> float:
    """Algorithmic bytes per local point of one fused Jacobi-PCG iteration (FP64, stored):
    Ax kernel z, p in, p, w out, G (10 words); gather-scatter 2 n_gs/n words of w and p at
    one copy per segment; update x, p, r, w, M^-1 in, x, r, z out (8 words) + 1 byte of
    multiplicity."""
    Np = N + 1
    ngs_frac = (Np ** 3 - (N - 1) ** 3) / Np ** 3
    return 8 * (10 + 2 * ngs_frac + 8) + 1


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


KERNEL_SOURCES = ("k_ax.cuh", "k_common.cuh", "k_tma.cuh", "k_df.cuh")  # every source the local operator is built from


def kernel_digest() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2108_12188_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        digest = kernel_digest()
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and parts[0] == kernel_key and parts[1] == digest:
                    return float(parts[2])
    except OSError:
        pass
    return None


# ---------------------------------------------------------------------------
# ranks: one process per GPU (torchrun); every rank runs its own replica
# ---------------------------------------------------------------------------

class Ranks:
    """Rank bookkeeping for N independent replicas: barrier and max/sum over ranks of host
    scalars. `backend` is nccl on GPUs (scalars travel on the rank's GPU) or gloo (CPU)."""

    def __init__(self, backend: str):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = torch.device("cuda", self.local_rank) if backend == "nccl" else torch.device("cpu")
        if self.world > 1 and not dist.is_initialized():
            kw = {"device_id": self.device} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def _reduce(self, v: float, op) -> float:
        if self.world == 1:
            return float(v)
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.MAX)

    def sum(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.SUM)

    def close(self):
        if self.world > 1 and self.dist.is_initialized():
            self.dist.destroy_process_group()


def whole_job_rate(local_units: float, local_ms: float, ranks: Ranks) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling)."""
    return ranks.sum(local_units) / (ranks.max(local_ms) * 1e-3)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples (every 20 ms) taken while the timed region runs.

    The sampler is started and its first line awaited before the region begins; samples
    are kept if their host timestamp falls inside [start, stop] of the region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.samples = []  # (host time, fields)
        self.t0 = self.t1 = None

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except OSError:
            self.proc = None
            self.t0 = time.time()
            return self
        first = threading.Event()

        def reader():
            for ln in self.proc.stdout:
                if ln.strip():
                    self.samples.append((time.time(), [x.strip() for x in ln.split(",")]))
                    first.set()

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        first.wait(timeout=10)
        self.t0 = time.time()
        return self

    def __exit__(self, *exc):
        self.t1 = time.time()
        if self.proc is not None:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for t, f in self.samples:
            if self.t0 is None or t < self.t0 or t > self.t1 + 0.03:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(self.REASONS, f[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

def oracle_cg_sample(nel: int = 12, budget_s: float = 10.0) -> dict:
    """Oracle Jacobi-PCG iterations on an nel^3 sub-box of the workload (same order, jitter,
    seed); returns local points per second of CG iterations (setup excluded)."""
    from oracle import sem_oracle as so
    from synthetic import BoxMesh
    m = BoxMesh(nel, nel, nel, jitter=JITTER, seed=SEED)
    prob = so.SemProblem(NORD, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    t0 = time.perf_counter()
    so.pcg(prob, b, rtol=0.0, max_iter=1)
    t1 = time.perf_counter()
    per_iter_guess = max(t1 - t0, 1e-3)
    iters = max(2, min(2000, int(budget_s / per_iter_guess)))
    t2 = time.perf_counter()
    so.pcg(prob, b, rtol=0.0, max_iter=1 + iters)
    t3 = time.perf_counter()
    dt = ((t3 - t2) - (t1 - t0)) / iters
    return {"n_local": prob.n, "iters": iters, "s_per_iter": dt, "gdof_s": prob.n / dt / 1e9,
            "sample": f"{nel}^3 elements of the same jittered box (N={NORD}, {prob.n} local points), "
                      f"{iters} oracle Jacobi-PCG iterations"}


def oracle_small_solve() -> dict:
    """The oracle's Jacobi-PCG solve of the small workload (4^3 hexahedra, jitter 0.1h,
    seed 0, N = 7, sine right-hand side, rtol 1e-10), timed whole (set-up excluded)."""
    from oracle import sem_oracle as so
    from synthetic import BoxMesh
    m = BoxMesh(4, 4, 4, jitter=0.1, seed=0)
    prob = so.SemProblem(NORD, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    t0 = time.perf_counter()
    ref = so.pcg(prob, b, rtol=1e-10)
    return {"seconds": time.perf_counter() - t0, "iterations": ref.iterations}


def _oracle_procs(count: int, budget_s: float) -> list:
    """Runs oracle_cg_sample in `count` fresh single-threaded processes at the same time (no
    CUDA state inherited); returns their results."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench; print('RESULT ' + json.dumps(bench.oracle_cg_sample(budget_s=%r)))" % budget_s)
    procs = [subprocess.Popen([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for _ in range(count)]
    out = []
    for p in procs:
        so_, se_ = p.communicate(timeout=900)
        res = [json.loads(ln[7:]) for ln in so_.splitlines() if ln.startswith("RESULT ")]
        if not res:
            raise RuntimeError("cpu baseline failed: " + se_[-2000:])
        out.append(res[0])
    return out


def run_cpu_baseline(budget_s: float = 10.0) -> dict:
    """The oracle on the host cores: one process alone, then one process per core at once
    (the oracle is single-threaded; each process times its own sample); and the oracle's
    whole solve of the small 4^3 workload, single-threaded."""
    single = _oracle_procs(1, budget_s)[0]
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = "import json, bench; print('RESULT ' + json.dumps(bench.oracle_small_solve()))"
    pr = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    c1 = [json.loads(ln[7:]) for ln in pr.stdout.splitlines() if ln.startswith("RESULT ")]
    cores = max(1, min(os.cpu_count() or 1, 72))
    many = _oracle_procs(cores, budget_s) if cores > 1 else [single]
    total = sum(r["gdof_s"] for r in many)
    return {"value": total, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
            "sample": f"{single['sample']}; one such sample per core, {cores} single-threaded processes at once",
            "single_core_value": single["gdof_s"], "s_per_iter_single_core": single["s_per_iter"],
            "solve_4cube_n7": c1[0] if c1 else None}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import sem_oracle as so
    from synthetic import BoxMesh, global_field
    nel = 12
    m = BoxMesh(nel, nel, nel, jitter=JITTER, seed=SEED)
    prob = so.SemProblem(NORD, m.vert_xyz, m.elem_verts)
    b = prob.rhs()
    # one step = one oracle Jacobi-PCG iteration on the 12^3 sample of the workload
    shape = prob.shape()
    c = prob.c.reshape(shape)
    Minv = prob.jacobi_inverse()
    x = so.scatter_local(global_field(prob.num.n_glob, SEED), prob.glo_num).reshape(shape)
    r = b - prob.ax(x)
    z = Minv * r
    p = z.copy()
    rho = so.glsc3(r, z, c)

    def step():
        nonlocal x, r, z, p, rho
        w = prob.ax(p)
        alpha = rho / so.glsc3(p, w, c)
        x = x + alpha * p
        r = r - alpha * w
        z = Minv * r
        rho_new = so.glsc3(r, z, c)
        so.glsc3(r, r, c)
        p = z + (rho_new / rho) * p
        rho = rho_new

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    val = prob.n / dt / 1e9
    sample = f"{nel}^3 elements of the same jittered box (N={NORD}, {prob.n} local points), one iteration per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GDOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample": sample},
        "cpu_baseline": {"value": val, "unit": "GDOF/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def flush_l2(buf):
    buf.add_(1.0)  # writes more bytes than L2 holds


def time_ax(sem, mesh, variant, prec, u, w, flush_buf, reps, warmup, assemble):
    import torch
    for _ in range(warmup):
        sem.sem_ax(mesh.handle, variant, prec, u, w, assemble=assemble, n_local=mesh.n)
    times = []
    s = torch.cuda.current_stream()
    for _ in range(reps):
        flush_l2(flush_buf)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        sem.sem_ax(mesh.handle, variant, prec, u, w, assemble=assemble, n_local=mesh.n)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times), min(times), max(times)


def ax_error_vs_oracle(sem, mesh, m, variant, prec, n_sample=48):
    """Relative 2-norm error of A_L against the FP64 oracle on sampled elements (local input)."""
    import numpy as np
    import torch
    from oracle import sem_oracle as so
    from synthetic import local_field
    P = (NORD + 1) ** 3
    u = local_field(mesh.n, seed=SEED + 17)
    dt = torch.float32 if prec == 1 else torch.float64
    ud = torch.tensor(u, dtype=dt, device="cuda")
    wd = torch.empty_like(ud)
    sem.sem_ax(mesh.handle, variant, prec, ud, wd, assemble=False, n_local=mesh.n)
    rng = np.random.default_rng(5)
    els = np.sort(rng.choice(m.num_elements, size=n_sample, replace=False))
    xi, wq = so.gll_nodes_weights(NORD)
    D = so.lagrange_derivative_matrix(xi)
    X = so.element_vertices(m.vert_xyz, m.elem_verts[els])
    G, _ = so.geometric_factors(X, xi, wq)
    ue = u.reshape(-1, P)[els].reshape(n_sample, NORD + 1, NORD + 1, NORD + 1)
    want = so.ax_local(ue, G, D).ravel()
    got = wd.double().cpu().numpy().reshape(-1, P)[els].ravel()
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def run_gpu(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    ranks = Ranks("nccl")

    def barrier():
        ranks.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return ranks.max(v)

    from paper_2108_12188_gb300 import build_lib, sem
    from synthetic import BoxMesh, global_field
    build_lib.build()
    sem.load_library()
    hbm_gbs, peak_src = measured_peaks()

    m = BoxMesh(NEL, NEL, NEL, jitter=JITTER, seed=SEED)
    mesh = sem.Mesh(NORD, m.vert_xyz, m.elem_verts,
                    flags=sem.SEM_MESH_F64_STORED | sem.SEM_MESH_F32_STORED | sem.SEM_MESH_OTF_SCALE
                    | sem.SEM_MESH_F64X_STORED)
    n = mesh.n
    info = mesh.info
    u_glob = torch.tensor(global_field(info["n_glob"], SEED, start=m.draws_used), dtype=torch.float64, device="cuda")
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    sem.sem_scatter(mesh.handle, sem.SEM_F64, u_glob, x0)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, b)
    x = x0.clone()

    # ---- timed region: K device-resident CG iterations
    opts = sem.sem_cg_default_opts(rtol=0.0, max_iter=1 << 30, use_graph=0, check_every=1)
    cg = sem.sem_cg_create(mesh.handle, opts)
    sem.sem_cg_start(cg, b, x)
    sem.sem_cg_iterate_timed(cg, args.warmup)
    barrier()
    l0 = sem.sem_launch_count()
    with ClockSampler(local_rank) as clk:
        total_ms, kernel_ms = sem.sem_cg_iterate_timed(cg, args.steps)
        barrier()
    launches = sem.sem_launch_count() - l0
    q = sem.sem_cg_query(cg)
    if q["status"] != sem.SEM_ERR_BUSY or q["iters"] != args.warmup + args.steps:
        raise RuntimeError(f"CG stopped early during the benchmark: {q}")
    sem.sem_cg_destroy(cg)
    value = whole_job_rate(n * args.steps, total_ms, ranks) / 1e9
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / args.steps

    # the same step with the double-float FP64 operator (sem_cg_opts.f64_arith = 1)
    x_df = x0.clone()
    cg_df = sem.sem_cg_create(mesh.handle, sem.sem_cg_default_opts(rtol=0.0, max_iter=1 << 30, use_graph=0,
                                                                   check_every=1, f64_arith=1))
    sem.sem_cg_start(cg_df, b, x_df)
    sem.sem_cg_iterate_timed(cg_df, args.warmup)
    df_total, df_kernels = sem.sem_cg_iterate_timed(cg_df, args.steps)
    sem.sem_cg_destroy(cg_df)
    del x_df
    step_f64x = {"ms_per_step": df_total / args.steps, "gdof_s": n / (df_total / args.steps * 1e-3) / 1e9,
                 "per_kernel_ms": {"ax": df_kernels[0], "gather_scatter": df_kernels[1], "update": df_kernels[2]},
                 # fused CG prologue: p, r, M^-1, x in and x, p out besides the plain operator's u/w/G
                 "ax_hbm_frac": (ax_bytes_per_point("stored", "f64", NORD) * n + 40 * n) / (df_kernels[0] * 1e-3)
                 / 1e9 / hbm_gbs}

    # roofline of the dominant kernel (the local operator, FP64 stored, CG mode)
    ax_ms = kernel_ms[0]
    ax_flops = flops_eq11(NORD) * n
    ax_bytes = ax_bytes_per_point("stored", "f64", NORD) * n + 8 * 2 * n  # + p = z + beta p prologue
    achieved_tf = ax_flops / (ax_ms * 1e-3) / 1e12
    traffic = ncu_traffic("ax_f64_stored_cg")
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / PEAK_FP64_TFLOPS, "traffic": traffic,
                "kernel": "k_ax<8,double,stored,CG>", "kernel_ms": ax_ms,
                "hbm_achieved_gbs": ax_bytes / (ax_ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm_gbs,
                "hbm_frac": ax_bytes / (ax_ms * 1e-3) / 1e9 / hbm_gbs,
                "peak_source": f"FP64 FMA issue rate (2/clk/SM) x 152 SMs x 2070 MHz, derived (nominal); HBM {peak_src}",
                "fp64_probe_fma_per_clk_per_sm": [1.6, 1.9],  # FMA-chain probe on GB300 (measured range)
                "fp64_pipe_active_ncu": 0.845,  # ncu FP64-pipe utilisation of this kernel (profiles/)
                "per_kernel_ms": {"ax": kernel_ms[0], "gather_scatter": kernel_ms[1], "update": kernel_ms[2]},
                "step_bytes_algorithmic": cg_bytes_per_point(NORD) * n,
                "step_hbm_frac": cg_bytes_per_point(NORD) * n / (ms_step * 1e-3) / 1e9 / hbm_gbs}

    # ---- the local operator alone, per variant (rank 0 reports), each FP32 variant at the block
    # shape the tuner picks on this mesh (what SEM_AX_AUTO runs); FP64 keeps its default shapes
    ax = {}
    tune32 = sem.sem_autotune(mesh.handle, sem.SEM_F32)
    otf32_shape = min((c for c in tune32["candidates"] if c["variant"] == sem.SEM_AX_OTF
                       and c["shape"] != sem.SEM_TENSOR_SHAPE), key=lambda c: c["ms"])["shape"]
    sem.sem_autotune_set(NORD, sem.SEM_F32, sem.SEM_AX_OTF, otf32_shape)
    ax["f32_tune"] = [{"variant": c["variant"], "shape": c["shape"], "elements_per_block": c["elements_per_block"],
                       "ms": c["ms"]} for c in tune32["candidates"]]
    flush = torch.zeros(96 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 384 MB > L2
    for vname, variant, pname, prec in (("stored", sem.SEM_AX_STORED, "f64", sem.SEM_F64),
                                        ("stored", sem.SEM_AX_STORED, "f64x", sem.SEM_F64X),
                                        ("stored", sem.SEM_AX_STORED, "f32", sem.SEM_F32),
                                        ("otf", sem.SEM_AX_OTF, "f64", sem.SEM_F64),
                                        ("otf", sem.SEM_AX_OTF, "f64x", sem.SEM_F64X),
                                        ("otf", sem.SEM_AX_OTF, "f32", sem.SEM_F32),
                                        ("otf_tc", sem.SEM_AX_OTF, "f32", sem.SEM_F32),
                                        ("otfscale", sem.SEM_AX_OTF_SCALE, "f64", sem.SEM_F64),
                                        ("otfscale", sem.SEM_AX_OTF_SCALE, "f32", sem.SEM_F32)):
        dt = torch.float32 if prec == sem.SEM_F32 else torch.float64
        u = x0.to(dt)
        w = torch.empty_like(u)
        if vname == "otf_tc":  # the line contractions on the tensor cores (block shape choice 3)
            sem.sem_autotune_set(NORD, sem.SEM_F32, sem.SEM_AX_OTF, sem.SEM_TENSOR_SHAPE)
        med, lo, hi = time_ax(sem, mesh, variant, prec, u, w, flush, reps=10, warmup=2, assemble=False)
        med_a, _, _ = time_ax(sem, mesh, variant, prec, u, w, flush, reps=5, warmup=1, assemble=True)
        byt = ax_bytes_per_point("otf" if vname == "otf_tc" else vname, "f32" if pname == "f32" else "f64", NORD) * n
        fl = flops_eq11(NORD) * n
        if pname == "f64x":  # FP64 data, FP32-pipe arithmetic: report against the HBM roof
            t_roof = byt / (hbm_gbs * 1e9)
        else:
            peak_tf = PEAK_FP64_TFLOPS if pname == "f64" else PEAK_FP32_TFLOPS
            t_roof = max(byt / (hbm_gbs * 1e9), fl / (peak_tf * 1e12))
        err = ax_error_vs_oracle(sem, mesh, m, variant, prec) if rank == 0 else None
        if vname == "otf_tc":
            sem.sem_autotune_set(NORD, sem.SEM_F32, sem.SEM_AX_OTF, otf32_shape)
        ax[f"{pname}_{vname}"] = {
            "ms": med, "ms_min": lo, "ms_max": hi, "gdof_s": n / (med * 1e-3) / 1e9,
            "gflop_s_eq11": fl / (med * 1e-3) / 1e9, "hbm_gbs": byt / (med * 1e-3) / 1e9,
            "hbm_frac": byt / (med * 1e-3) / 1e9 / hbm_gbs,
            "roofline_frac_eq11": t_roof / (med * 1e-3),
            "assembled_ms": med_a, "assembled_gdof_s": n / (med_a * 1e-3) / 1e9,
            "rel_err_vs_fp64_oracle": err}
    del flush

    # ---- end to end through the public API with pinned host buffers
    bh = b.cpu().pin_memory()
    xh = x0.cpu().pin_memory()
    xo = torch.empty(n, dtype=torch.float64).pin_memory()
    bd = torch.empty_like(b)
    xd = torch.empty_like(b)
    e2e_iters = min(args.steps, 50)
    e_opts = sem.sem_cg_default_opts(rtol=0.0, max_iter=e2e_iters, check_every=e2e_iters, use_graph=1)
    s = torch.cuda.current_stream()

    def e2e_step():
        bd.copy_(bh, non_blocking=True)
        xd.copy_(xh, non_blocking=True)
        res = sem.sem_cg_solve(mesh.handle, bd, xd, e_opts)
        xo.copy_(xd, non_blocking=True)
        return res

    e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_reps = 2
    e0.record(s)
    for _ in range(e2e_reps):
        res = e2e_step()
    e1.record(s)
    e1.synchronize()
    barrier()
    e2e_local_ms = e0.elapsed_time(e1) / e2e_reps
    e2e_rate = whole_job_rate(n * e2e_iters, e2e_local_ms, ranks)
    e2e_ms = max_over_ranks(e2e_local_ms)
    if res["iters"] != e2e_iters:
        raise RuntimeError(f"end-to-end solve ran {res['iters']} iterations, expected {e2e_iters}")
    e2e = {"value": e2e_rate / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8,
           "step": f"sem_cg_solve of {e2e_iters} Jacobi-PCG iterations from pinned host b and x0 to host x "
                   "(work-vector allocation, r0 = b - A x0 and CUDA-graph capture included)",
           "ms_per_step": e2e_ms}

    # ---- small solve: 4^3 mesh (+-0.1h, seed 0), N = 7, sine RHS, Jacobi-CG from zero to 1e-10
    m1 = BoxMesh(4, 4, 4, jitter=0.1, seed=0)
    mesh1 = sem.Mesh(NORD, m1.vert_xyz, m1.elem_verts, flags=sem.SEM_MESH_F64_STORED)
    b1 = torch.empty(mesh1.n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh1.handle, 1, 1, 1, sem.SEM_F64, b1)
    x1 = torch.zeros_like(b1)
    cg_c1 = {}
    for name, o in (("fp64", sem.sem_cg_default_opts(rtol=1e-10)),
                    ("fp64_persistent", sem.sem_cg_default_opts(rtol=1e-10, use_graph=2)),
                    ("f64x", sem.sem_cg_default_opts(rtol=1e-10, f64_arith=1)),
                    ("mixed_otf", sem.sem_cg_default_opts(rtol=1e-10, mixed=1, inner_rtol=1e-5)),
                    ("mixed_reliable", sem.sem_cg_default_opts(rtol=1e-10, mixed=2, inner_rtol=0.1))):
        times = []
        for _ in range(3):  # first solve builds the Jacobi diagonal and the graphs
            x1.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            r1 = sem.sem_cg_solve(mesh1.handle, b1, x1, o)
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        cg_c1[name] = {"ms": min(times[1:]), "iterations": r1["iters"], "outer": r1["outer_iters"],
                       "rel_res": r1["rel_res"], "status": sem.sem_status_string(r1["status"])}
    mesh1.close()

    # ---- the solve and serving legs of the metric (rank 0; replicas run the step above only)
    legs = {}
    if rank == 0 and not args.no_legs:
        mesh.close()  # the 32^3 mesh's factors are not needed any more
        legs["solve_c3"] = solve_leg(sem)
        torch.cuda.empty_cache()
        with ClockSampler(local_rank) as clk_s:
            serve = serve_stream(sem, args.leg_requests, args.leg_rate, 0, args.slots, 2097152)
        serve["clocks"] = clk_s.summary()
        serve["workload"] = ("solve requests: n^3 box, n~U{8..40}, N~U{5,7,9}, jitter 0.1h, sine RHS a,b,c~U{1,2,3}, "
                             "rtol 1e-8 FP32 CG with FP64 reliable updates, Poisson arrivals, 100 GB admission "
                             "budget, requests of at most 2,097,152 local points batched")
        legs["serve_c5"] = serve

    if rank == 0:
        cpu = run_cpu_baseline()
        out = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mesh": f"{NEL}^3 jittered box", "N": NORD, "n_local": n,
                       "n_glob": info["n_glob"], "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (about 1.1 GB of algorithmic traffic per step)",
                       "gflop_s_eq11": flops_eq11(NORD) * n / (ms_step * 1e-3) / 1e9},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "ax": ax, "cg_4cube_n7": cg_c1, "step_f64x": step_f64x, **legs,
        }
        print(json.dumps(out))
    mesh.close()
    ranks.close()


def solve_metrics(sem, mesh, b, x, xyz):
    """True relative residual sqrt(<r,r,c>/<b,b,c>) with r = b - A x (FP64 operator) and the
    max nodal error to sin(pi x) sin(pi y) sin(pi z)."""
    import torch
    w = torch.empty_like(x)
    variant = sem.SEM_AX_STORED if mesh.info["flags"] & sem.SEM_MESH_F64_STORED else sem.SEM_AX_OTF
    sem.sem_ax(mesh.handle, variant, sem.SEM_F64, x, w, assemble=True, n_local=mesh.n)
    r = b - w
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    bb = torch.zeros(1, dtype=torch.float64, device="cuda")
    sem.sem_glsc3(mesh.handle, sem.SEM_F64, r, r, rr)
    sem.sem_glsc3(mesh.handle, sem.SEM_F64, b, b, bb)
    n = mesh.n
    exact = torch.sin(math.pi * xyz[:n]) * torch.sin(math.pi * xyz[n:2 * n]) * torch.sin(math.pi * xyz[2 * n:])
    return math.sqrt(rr.item() / bb.item()), float(torch.max(torch.abs(x - exact)))


def solve_leg(sem, nel: int = 64, solvers=("fp64_cg", "mixed_reliable", "f64x_cg"), inner_rtol: float = 1e-5) -> dict:
    """Full-solve configuration: nel^3 hexahedra (+-0.15h, seed 2), N = 7 (64^3: 134,217,728
    local points), manufactured sine right-hand side, each solver to the relative residual 1e-10:
      fp64_cg         FP64 Jacobi-CG, stored FP64 factors;
      mixed_reliable  FP32 Jacobi-CG with on-the-fly factors and FP64 reliable updates (the
                      true FP64 residual replaces the FP32 one after each 10x reduction);
      f64x_cg         Jacobi-CG with the double-float operator, restarts from the FP64 residual;
      mixed_otf       FP32 inner CG to inner_rtol with restarted FP64 refinement.
    Per solver: device seconds (CUDA events around sem_cg_solve), iterations, the true residual
    b - A x (FP64 operator) and the max nodal error to sin(pi x) sin(pi y) sin(pi z)."""
    import torch
    from synthetic import BoxMesh
    t0 = time.perf_counter()
    m = BoxMesh(nel, nel, nel, jitter=JITTER, seed=2)
    mesh = sem.Mesh(NORD, m.vert_xyz, m.elem_verts, flags=sem.SEM_MESH_F64_STORED | sem.SEM_MESH_F64X_STORED)
    setup_s = time.perf_counter() - t0
    n = mesh.n
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, b)
    xyz = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    sem.sem_mesh_coords(mesh.handle, xyz)
    x = torch.zeros_like(b)
    mj = torch.empty_like(b)
    sem.sem_jacobi(mesh.handle, sem.SEM_F64, mj)  # builds the Jacobi diagonal once (set-up)
    del mj
    for prec in (sem.SEM_F64, sem.SEM_F32):  # block shapes of this order (set-up); used by every variant
        sem.sem_autotune(mesh.handle, prec, reps=5)
    configs = {
        "fp64_cg": sem.sem_cg_default_opts(rtol=1e-10, variant=sem.SEM_AX_STORED, check_every=50),
        "f64x_cg": sem.sem_cg_default_opts(rtol=1e-10, variant=sem.SEM_AX_STORED, check_every=50, f64_arith=1),
        "mixed_otf": sem.sem_cg_default_opts(rtol=1e-10, mixed=1, variant=sem.SEM_AX_STORED,
                                             inner_variant=sem.SEM_AX_OTF, inner_rtol=inner_rtol, check_every=50),
        "mixed_reliable": sem.sem_cg_default_opts(rtol=1e-10, mixed=2, variant=sem.SEM_AX_STORED,
                                                  inner_variant=sem.SEM_AX_OTF, inner_rtol=0.1, check_every=50),
    }
    runs = {}
    for name in solvers:
        x.zero_()
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            res = sem.sem_cg_solve(mesh.handle, b, x, configs[name])
            e1.record()
            e1.synchronize()
        rel, err = solve_metrics(sem, mesh, b, x, xyz)
        runs[name] = {"seconds": e0.elapsed_time(e1) / 1e3, "host_seconds": res["time_ms"] / 1e3,
                      "iterations": res["iters"], "outer_iterations": res["outer_iters"],
                      "status": sem.sem_status_string(res["status"]), "solver_rel_res": res["rel_res"],
                      "true_rel_res": rel, "max_err_vs_sine": err, "clocks": clk.summary()}
    mesh.close()
    out = {"workload": f"{nel}^3 hexahedra on [0,1]^3, jitter +-0.15h (seed 2), N={NORD}, {n} local points, "
                       "sine right-hand side, rtol 1e-10", "n_local": n, "mesh_setup_s": setup_s, **runs}
    if "fp64_cg" in runs and "mixed_reliable" in runs:
        out["speedup_mixed_reliable_vs_fp64"] = runs["fp64_cg"]["seconds"] / runs["mixed_reliable"]["seconds"]
    return out


def run_solve(args):
    """The full-solve configuration alone, with every solver (see solve_leg)."""
    import torch
    from paper_2108_12188_gb300 import build_lib, sem
    build_lib.build()
    sem.load_library()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    leg = solve_leg(sem, args.nel, ("fp64_cg", "f64x_cg", "mixed_otf", "mixed_reliable"), args.inner_rtol)
    print(json.dumps({"metric": "CG time to 1e-10 (s)", "value": leg["mixed_reliable"]["seconds"], "unit": "s",
                      "higher_is_better": False, "n_gpus": 1, "dtype": "f64 (outer) / f32 (inner)",
                      "data": "synthetic", "config": {"workload": leg["workload"], "inner_rtol": args.inner_rtol},
                      **leg}))


def serve_stream(sem, requests: int, rate: float, seed: int, slots: int, batch_points: int, round_iters: int = 20,
                 priorities: int = 1):
    """One request stream through a fresh server: `requests` Poisson-solve requests with Poisson
    arrivals at `rate` per second (seeded), each an n^3 box with n ~ U{8..40}, N ~ U{5,7,9},
    jitter 0.1h, sine right-hand side with a, b, c ~ U{1,2,3}, rtol 1e-8, FP32 CG with FP64
    reliable updates; 100 GB admission budget. Requests of at most batch_points local points run
    in the server's batch (0: none). Latency = submit -> solution in host memory."""
    import numpy as np
    from synthetic import BoxMesh, splitmix64
    opts = sem.sem_cg_default_opts(rtol=1e-8, mixed=2, variant=sem.SEM_AX_OTF, inner_variant=sem.SEM_AX_OTF,
                                   inner_rtol=0.1, check_every=25)
    budget = 100 * 10 ** 9
    R = requests
    draws = splitmix64(1000 + seed, 0, 6 * R)
    srv = sem.sem_server_create(budget, slots, batch_max_points=int(batch_points), batch_round_iters=round_iters,
                                size_priorities=int(priorities))
    rng_t = np.random.default_rng(2000 + seed)
    arrivals = np.cumsum(rng_t.exponential(1.0 / rate, size=R))
    tickets, done, pending = [], {}, set()
    t0 = time.perf_counter()
    q = 0
    while len(done) < R:
        now = time.perf_counter() - t0
        while q < R and arrivals[q] <= now:
            d = draws[6 * q: 6 * q + 6]
            nel = 8 + int(d[0] % 33)
            N = (5, 7, 9)[int(d[1] % 3)]
            sine = tuple(1 + int(v % 3) for v in d[2:5])
            mesh = BoxMesh(nel, nel, nel, jitter=0.1, seed=int(d[5] % (1 << 31)))
            t = sem.sem_server_submit(srv, N, mesh.vert_xyz, mesh.elem_verts, sine, opts)
            tickets.append(t)
            pending.add(t)
            q += 1
        for t in list(pending):
            r = sem.sem_server_poll(srv, t, want_x=False)
            if r is not None:
                sem.sem_server_poll(srv, t, want_x=True)  # take the solution, release the ticket
                done[t] = r[0]
                pending.discard(t)
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    bstats = sem.sem_server_batch_stats(srv)
    sem.sem_server_destroy(srv)
    lat = np.array([done[t]["latency_ms"] for t in tickets])
    bat = np.array([done[t]["batched"] for t in tickets], dtype=bool)
    ok = sum(1 for t in tickets if done[t]["status"] == sem.SEM_OK)
    pts = sum(done[t]["n_local"] for t in tickets)
    out = {"arrival_rate_per_s": rate, "requests": R, "ok": ok, "batch_max_points": int(batch_points),
           "size_priorities": int(priorities),
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "solves_per_s": R / wall, "wall_s": wall,
           "mean_queue_ms": float(np.mean([done[t]["queue_ms"] for t in tickets])),
           "mean_setup_ms": float(np.mean([done[t]["setup_ms"] for t in tickets])),
           "mean_solve_ms": float(np.mean([done[t]["solve_ms"] for t in tickets])),
           "local_points": int(pts), "batched_requests": int(bat.sum()), "batch": bstats}
    if bat.any():
        out["batched_p50_ms"] = float(np.percentile(lat[bat], 50))
        out["batched_p99_ms"] = float(np.percentile(lat[bat], 99))
    if (~bat).any():
        out["unbatched_p50_ms"] = float(np.percentile(lat[~bat], 50))
        out["unbatched_p99_ms"] = float(np.percentile(lat[~bat], 99))
    return out


def run_serve(args):
    """Serving configuration (see serve_stream) at each arrival rate of --rates, with the
    server's batch (--batch-points local points at most per batched request) and without it
    (0). Reports p50/p99 latency and solves/s per rate and setting."""
    import torch
    from paper_2108_12188_gb300 import build_lib, sem
    build_lib.build()
    sem.load_library()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rates = [float(r) for r in args.rates.split(",")]
    settings = [int(b) for b in args.batch_points.split(",")]
    prios = [int(p) for p in args.priorities.split(",")]
    runs = []
    for pr in prios:
        for bp in settings:
            for ri, lam in enumerate(rates):
                runs.append(serve_stream(sem, args.requests, lam, ri, args.slots, bp, priorities=pr))
                print(json.dumps({"rate": lam, "batch_points": bp, "priorities": pr, "p50_ms": runs[-1]["p50_ms"],
                                  "p99_ms": runs[-1]["p99_ms"], "solves_per_s": runs[-1]["solves_per_s"]}),
                      file=sys.stderr)
    main = runs[0]
    print(json.dumps({
        "metric": "served p50/p99 latency (ms)", "value": main["p50_ms"], "unit": "ms", "higher_is_better": False,
        "n_gpus": 1, "dtype": "f64 (outer) / f32 (inner)", "data": "synthetic",
        "config": {"workload": "solve requests: n^3 box, n~U{8..40}, N~U{5,7,9}, jitter 0.1h, sine RHS a,b,c~U{1,2,3}, "
                               "rtol 1e-8 FP32 CG with FP64 reliable updates, Poisson arrivals, 100 GB admission budget",
                   "requests_per_rate": args.requests, "slots": args.slots, "batch_points": settings,
                   "size_priorities": prios},
        "p99_ms": main["p99_ms"], "runs": runs}))


def oracle_ax_rate(N: int, nel: int = 8, reps: int = 3) -> dict:
    """The oracle's local operator A_L (FP64, stored factors, element by element) on one host
    core, on a bounded sample: nel^3 elements of the sweep's jittered box at order N."""
    import numpy as np
    from oracle import sem_oracle as so
    from synthetic import BoxMesh
    m = BoxMesh(nel, nel, nel, jitter=0.1, seed=100 + N)
    xi, wq = so.gll_nodes_weights(N)
    D = so.lagrange_derivative_matrix(xi)
    G, _ = so.geometric_factors(so.element_vertices(m.vert_xyz, m.elem_verts), xi, wq)
    u = np.random.default_rng(N).uniform(-1.0, 1.0, (nel ** 3, N + 1, N + 1, N + 1))
    so.ax_local(u, G, D)
    t0 = time.perf_counter()
    for _ in range(reps):
        so.ax_local(u, G, D)
    dt = (time.perf_counter() - t0) / reps
    pts = nel ** 3 * (N + 1) ** 3
    return {"gdof_s": pts / dt / 1e9, "cores": 1, "kind": "oracle",
            "sample": f"{nel}^3 elements at N={N} ({pts} local points), A_L only, {reps} repetitions"}


def run_sweep(args):
    """Polynomial-order sweep: N in {3,5,7,9,11}, E = n^3 with n = round(cbrt(16.8M / (N+1)^3)),
    interior jitter +-0.1h; per N the autotuner picks block shape and stored versus on-the-fly
    factors for FP64 and FP32, then A_L (tuned) and the CG solve to 1e-10 are timed: FP64
    Jacobi-CG and FP32 CG with FP64 reliable updates, CG iterations replayed as CUDA graphs."""
    import torch
    from paper_2108_12188_gb300 import build_lib, sem
    from synthetic import BoxMesh, n_for_points
    build_lib.build()
    sem.load_library()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    flush = torch.zeros(96 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rows = []
    for N in (3, 5, 7, 9, 11):
        nel = n_for_points(N + 1)
        m = BoxMesh(nel, nel, nel, jitter=0.1, seed=100 + N)
        mesh = sem.Mesh(N, m.vert_xyz, m.elem_verts, flags=sem.SEM_MESH_F64_STORED | sem.SEM_MESH_F32_STORED)
        n = mesh.n
        row = {"N": N, "elements": nel ** 3, "n_local": n, "flops_per_point_eq11": flops_eq11(N)}
        for pname, prec in (("f64", sem.SEM_F64), ("f32", sem.SEM_F32)):
            rep = sem.sem_autotune(mesh.handle, prec, reps=10)
            best = rep["candidates"][rep["best"]]
            dt = torch.float64 if prec == sem.SEM_F64 else torch.float32
            u = torch.rand(n, dtype=dt, device="cuda")
            w = torch.empty_like(u)
            med, _, _ = time_ax(sem, mesh, sem.SEM_AX_AUTO, prec, u, w, flush, reps=10, warmup=2, assemble=False)
            row[pname] = {"tuner": rep["candidates"], "chosen": best, "ax_ms": med, "ax_gdof_s": n / (med * 1e-3) / 1e9,
                          "ax_gflop_s_eq11": flops_eq11(N) * n / (med * 1e-3) / 1e9}
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        sem.sem_rhs_sine(mesh.handle, 1, 1, 1, sem.SEM_F64, b)
        x = torch.zeros_like(b)
        for name, o in (("cg_fp64", sem.sem_cg_default_opts(rtol=1e-10, variant=sem.SEM_AX_AUTO)),
                        ("cg_mixed", sem.sem_cg_default_opts(rtol=1e-10, mixed=2, variant=sem.SEM_AX_AUTO,
                                                             inner_variant=sem.SEM_AX_AUTO, inner_rtol=0.1))):
            x.zero_()
            sem.sem_cg_solve(mesh.handle, b, x, sem.sem_cg_default_opts(rtol=1e-2))  # warm-up: graphs, Jacobi
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            res = sem.sem_cg_solve(mesh.handle, b, x, o)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            row[name] = {"ms": ms, "iterations": res["iters"], "outer": res["outer_iters"],
                         "ms_per_iteration": ms / max(res["iters"], 1), "rel_res": res["rel_res"],
                         "status": sem.sem_status_string(res["status"])}
        row["cpu_baseline_ax"] = oracle_ax_rate(N)
        rows.append(row)
        mesh.close()
        print(json.dumps({"N": N, "done": True}), file=sys.stderr)
    print(json.dumps({"metric": "Ax GDOF/s per polynomial order (tuned)", "value": rows[2]["f32"]["ax_gdof_s"],
                      "unit": "GDOF/s", "higher_is_better": True, "n_gpus": 1, "dtype": "f64/f32", "data": "synthetic",
                      "config": {"workload": "N in {3,5,7,9,11}, n^3 elements with n = round(cbrt(16.8M/(N+1)^3)), "
                                             "jitter 0.1h, autotuned, CG as CUDA graphs"},
                      "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sem", choices=["sem", "reference"])
    ap.add_argument("--workload", default="ax", choices=["ax", "solve", "serve", "sweep"],
                    help="ax: the Ax-throughput line (default); solve: the 64^3 full-solve comparison; "
                         "serve: the request-stream latency measurement")
    ap.add_argument("--requests", type=int, default=1000, help="requests per arrival rate (serve)")
    ap.add_argument("--rates", default="1,2,4", help="arrival rates in requests/s (serve)")
    ap.add_argument("--slots", type=int, default=16, help="worker threads of the server (serve)")
    ap.add_argument("--batch-points", default="2097152,0",
                    help="server batch limits in local points to compare, 0 = no batch (serve)")
    ap.add_argument("--priorities", default="1", help="size-ordered stream priorities to compare, 1 on / 0 off (serve)")
    ap.add_argument("--nel", type=int, default=64, help="elements per direction of the solve workload")
    ap.add_argument("--no-legs", action="store_true", help="ax: skip the full-solve and serving legs")
    ap.add_argument("--leg-requests", type=int, default=1000, help="ax: requests of the serving leg")
    ap.add_argument("--leg-rate", type=float, default=4.0, help="ax: arrival rate of the serving leg (1/s)")
    ap.add_argument("--inner-rtol", type=float, default=1e-5)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "solve":
        run_solve(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
