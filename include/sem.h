/*
 * sem.h - C ABI of the GB300 spectral-element Poisson library (libsem.so).
 *
 * The library evaluates the matrix-free spectral-element (SEM) Laplace
 * operator and runs conjugate gradient on it, following Karp et al., "A
 * High-Fidelity Flow Solver for Unstructured Meshes on FPGAs" (HPC Asia
 * 2022): Section 3 (Eqs. 1-5), Section 3.2 (Algorithm 1) and Section 5.1
 * (geometric factors recomputed on the fly, "rematerialisation").
 *
 * Problem (Eqs. 1-2, read as -lap(u) = f with u = 0 on the Dirichlet part of
 * the boundary): E trilinear hexahedra, order N (Np = N + 1 Gauss-Lobatto-
 * Legendre points per direction), P = Np^3 points per element.
 *
 * Conventions shared by every call:
 *  - Every call returns a sem_status and never aborts; sem_last_error() gives
 *    a thread-local message for the last non-OK status of the calling thread.
 *  - Vectors live on the "local" (replicated) layout of Section 3.1,
 *    u_L = Q u: n = E * P entries indexed ((e * Np + k) * Np + j) * Np + i,
 *    i fastest (i along xi, j along eta, k along gamma). FP64 vectors are
 *    double*, FP32 vectors float* (sem_prec says which).
 *  - Pointers named *_dev are device pointers owned by the caller (for
 *    example torch tensor data_ptr()); they must be 16-byte aligned and hold
 *    n elements of the stated precision. The library never frees caller
 *    memory and keeps no reference to it after the call returns.
 *  - Pointers named *_host are host pointers read or written synchronously.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls marked
 *    "async" only enqueue work on `stream` and do not synchronise the host.
 *  - A mesh is used on the CUDA device that was current when it was
 *    created; calls made with another device current return SEM_ERR_ARG.
 *  - Calls on one mesh from several host threads must be serialised by the
 *    caller; different meshes are independent.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SEM_OK = 0,
  SEM_ERR_ARG = 1,           /* invalid argument (null pointer, size, precision not prepared, ...) */
  SEM_ERR_MESH = 2,          /* invalid mesh: bad vertex id, repeated vertex, det J <= 0, non-manifold face */
  SEM_ERR_OOM = 3,           /* device or host allocation failed */
  SEM_ERR_CUDA = 4,          /* a CUDA runtime call failed; the message names it */
  SEM_ERR_NOT_CONVERGED = 5, /* CG stopped at max_iter; the result holds the last iterate */
  SEM_ERR_BREAKDOWN = 6,     /* CG breakdown: <p, A p, c> <= 0 or a non-finite scalar */
  SEM_ERR_TIMEOUT = 7,       /* a bounded wait ran out */
  SEM_ERR_BUSY = 8,          /* resource temporarily unavailable (admission refused / not done yet) */
  SEM_ERR_UNSUPPORTED = 9    /* e.g. polynomial order outside [1, SEM_MAX_N] */
} sem_status;

/* SEM_F64: FP64 data and FP64 arithmetic. SEM_F32: FP32 data and arithmetic.
 * SEM_F64X: FP64 data (double* vectors, FP64 stored factors); the local operator runs in
 * double-float arithmetic (pairs of floats with error-free products and sums, about 47
 * significant bits) on the FP32 pipes, which GB300 issues 64 times faster than FP64. Only
 * sem_ax (and the CG options' f64_arith) use it: with SEM_AX_STORED on the float-pair factors of
 * SEM_MESH_F64X_STORED if the mesh has them, else the FP64 ones; with SEM_AX_OTF on factors
 * rebuilt from the element's trilinear coefficients (the per-column polynomial coefficients
 * in FP64, every point in double-float); SEM_AX_OTF_SCALE gives SEM_ERR_UNSUPPORTED. Every
 * other call treats SEM_F64X like SEM_F64. Values below 2^-126 in magnitude are flushed to
 * zero inside it. */
typedef enum { SEM_F64 = 0, SEM_F32 = 1, SEM_F64X = 2 } sem_prec;

/* Variants of the local operator A_L (Section 5.1):
 * STORED reads the six geometric factors per point from device memory;
 * OTF recomputes them per point from 21 per-element trilinear-map coefficients;
 * OTF_SCALE recomputes them too but reads one word per point, w_i w_j w_k / det J, so the
 *   per-point division is not repeated (the rematerialisation of Section 5.1 with an I/O
 *   cost of one word per point); needs SEM_MESH_OTF_SCALE;
 * AUTO uses the variant and block shape sem_autotune found fastest for this order and
 * precision (before tuning: STORED if the mesh holds the factors, else OTF). */
typedef enum { SEM_AX_STORED = 0, SEM_AX_OTF = 1, SEM_AX_AUTO = 2, SEM_AX_OTF_SCALE = 3 } sem_ax_variant;

#define SEM_MAX_N 11 /* polynomial orders 1..11 are compiled in */

/* Flags for sem_mesh_create: which stored-factor arrays to keep on the device.
 * The per-element coefficients for the OTF variant are always kept (FP64 and FP32). */
#define SEM_MESH_F64_STORED 1u /* G in FP64: 48 bytes per local point */
#define SEM_MESH_F32_STORED 2u /* G in FP32: 24 bytes per local point */
#define SEM_MESH_OTF_SCALE 4u  /* w_i w_j w_k / det J per point, FP64 and FP32: 12 bytes per local point */
#define SEM_MESH_F64X_STORED 8u /* G as float pairs (high, low: 48 significant bits) for SEM_F64X: 48 bytes
                                 * per local point; without it SEM_F64X splits the FP64 factors itself */

typedef struct sem_mesh_s* sem_mesh;
typedef struct sem_cg_s* sem_cg;

typedef struct {
  int N;           /* polynomial order */
  int Np;          /* N + 1 */
  int64_t E;       /* elements */
  int64_t n_local; /* E * Np^3 local (replicated) points */
  int64_t n_glob;  /* distinct global nodes */
  int64_t n_seg;   /* gather-scatter segments (global nodes on element boundaries) */
  int64_t n_gs;    /* local points on element boundaries: E((N+1)^3 - (N-1)^3), Eq. 9 */
  unsigned flags;  /* SEM_MESH_* flags the mesh was created with */
  int device;      /* CUDA device ordinal */
  size_t device_bytes; /* device memory held by the mesh */
} sem_mesh_info_t;

/* Create a mesh (Section 3: E hexahedra, GLL points of order N).
 *  vert_xyz_host    [num_vertices][3] FP64 vertex coordinates.
 *  elem_verts_host  [E][8] vertex ids; local vertex a + 2b + 4c (a, b, c in
 *                   {0,1}) sits at reference corner (2a-1, 2b-1, 2c-1), a along
 *                   xi, b along eta, c along gamma. The map must be orientation
 *                   preserving (det J > 0 at every GLL point) or SEM_ERR_MESH.
 *  dirichlet_vertex_flags_host  NULL: every boundary face (a face owned by one
 *                   element) is Dirichlet. Otherwise [num_vertices] bytes; a
 *                   boundary face is Dirichlet iff its four vertices are flagged.
 * Global numbering (Section 3.1's Q): two local points are one global node iff
 * they sit on the same vertex, edge or face at the same position; global ids
 * follow the first occurrence in the local order. The call validates the mesh
 * on the host, builds numbering, gather-scatter segments and mask, copies the
 * per-element data to the device, computes geometric factors (kernel) and
 * synchronises `stream`. The host arrays are copied; the caller keeps them.
 * Limits: 1 <= N <= SEM_MAX_N, E >= 1, E * (N+1)^3 < 2^31. */
sem_status sem_mesh_create(int N, int64_t num_vertices, const double* vert_xyz_host, int64_t E,
                           const int64_t* elem_verts_host, const uint8_t* dirichlet_vertex_flags_host,
                           unsigned flags, void* stream, sem_mesh* out);
/* Releases the mesh. Waits for the streams the mesh was used on (not the whole device),
 * then frees its memory stream-ordered; those streams must still exist. NULL is a no-op. */
sem_status sem_mesh_destroy(sem_mesh mesh);
/* Host-only: the numbering and mask sem_mesh_create would build (Section 3.1's Q), without
 * touching a GPU. glo_num_host [E*(N+1)^3] int64, mask_host [E*(N+1)^3] uint8 (either may be
 * NULL), n_glob_host receives the number of global nodes. Same validation as sem_mesh_create
 * except for the geometry (det J) check, which needs the device. */
sem_status sem_mesh_numbering(int N, int64_t num_vertices, int64_t E, const int64_t* elem_verts_host,
                              const uint8_t* dirichlet_vertex_flags_host, int64_t* glo_num_host, uint8_t* mask_host,
                              int64_t* n_glob_host);

sem_status sem_mesh_get_info(sem_mesh mesh, sem_mesh_info_t* info_host);
/* The three sizes of the mesh: local points E (N+1)^3, distinct global nodes, and
 * gather-scatter segments (global nodes with copies on element boundaries). Any pointer may
 * be NULL. */
sem_status sem_mesh_info(sem_mesh mesh, int64_t* n_local, int64_t* n_glob, int64_t* n_shared_seg);

/* Test hooks: copy the numbering (int64 [n_local]), the Dirichlet mask (uint8
 * [n_local], 1 = zeroed) and the gather-scatter segments to host buffers.
 * Segments: global nodes on element boundaries in ascending global id;
 * seg_off [n_seg + 1] int32 offsets into seg_idx [n_gs] int32 local indices
 * (ascending within a segment); seg_mask [n_seg] uint8. They are rebuilt from the
 * device's gather-scatter plan (segments grouped by copy count), so they show exactly
 * what the gather-scatter kernels use. Any pointer may be NULL. */
sem_status sem_mesh_get_glo_num(sem_mesh mesh, int64_t* glo_num_host);
sem_status sem_mesh_get_mask(sem_mesh mesh, uint8_t* mask_host);
sem_status sem_mesh_get_segments(sem_mesh mesh, int32_t* seg_off_host, int32_t* seg_idx_host,
                                 uint8_t* seg_mask_host);

/* Self-test of the bounded waits that guard every TMA copy of the library (failure
 * detection without a GPU fault): one block prepares an mbarrier for a 16-byte copy and waits
 * for it with a limit of limit_ns nanoseconds (1 ms .. 2 s, else SEM_ERR_ARG). issue_copy = 1
 * issues the copy: the wait completes, SEM_OK. issue_copy = 0 issues nothing: the wait gives
 * up after the limit and the call returns SEM_ERR_TIMEOUT, the status a CG solve reports when
 * a copy of the local operator does not arrive; the context stays usable. Synchronises
 * `stream`; *elapsed_ms_host receives the kernel's duration. */
sem_status sem_probe_bounded_wait(int64_t limit_ns, int issue_copy, double* elapsed_ms_host, void* stream);
/* Self-test of the bounded grid barrier of the persistent small-mesh CG kernel: a cooperative
 * launch of a few blocks meets at one barrier. skip_one = 0: all arrive, SEM_OK. skip_one = 1: one
 * block never arrives, the others give up after the barrier's limit (1 s) and the call returns
 * SEM_ERR_TIMEOUT, the status a solve reports when a barrier runs out; no fault, the context
 * stays usable. Synchronises `stream`; *elapsed_ms_host receives the kernel's duration. */
sem_status sem_probe_grid_barrier(int skip_one, double* elapsed_ms_host, void* stream);

/* Physical coordinates of the local points (trilinear map, Section 5.1):
 * xyz_dev [3][n_local] FP64 (all x, then all y, then all z). Async. */
sem_status sem_mesh_coords(sem_mesh mesh, double* xyz_dev, void* stream);

/* The six geometric factors G = w_i w_j w_k |det J| J^-1 J^-T of Eq. 4
 * (Section 4.2), G_dev [E][6][P] in the order G11, G12, G13, G22, G23, G33,
 * and the mass B = w_i w_j w_k |det J| in B_dev [E][P] (either may be NULL).
 * Computed from the element coefficients in FP64 (prec F64) or FP64 rounded
 * to FP32 (prec F32). Async. */
sem_status sem_mesh_geometry(sem_mesh mesh, sem_prec prec, void* G_dev, void* B_dev, void* stream);

/* Q (Section 3.1): u_local[i] = u_glob[glo_num[i]]; u_glob_dev has n_glob entries. Async. */
sem_status sem_scatter(sem_mesh mesh, sem_prec prec, const void* u_glob_dev, void* u_local_dev, void* stream);

/* Ax (Section 3.1): w = A_L u (Eq. 4, element by element); with assemble != 0
 * also the gather-scatter QQ^T and the Dirichlet mask (Algorithm 1 steps 6-7).
 * u and w must not overlap. STORED needs the factors of that precision
 * (SEM_MESH_F64_STORED / SEM_MESH_F32_STORED) else SEM_ERR_ARG. Async. */
sem_status sem_ax(sem_mesh mesh, sem_ax_variant variant, sem_prec prec, const void* u_dev, void* w_dev,
                  int assemble, void* stream);

/* Gather-scatter QQ^T in place (Eq. 5, Section 4.3): every local copy of a
 * global node receives the sum of all copies, added left to right in
 * ascending local index (so the result is bit-reproducible); with
 * apply_mask != 0 Dirichlet copies are then set to 0. Async. */
sem_status sem_dssum(sem_mesh mesh, sem_prec prec, void* u_dev, int apply_mask, void* stream);

/* Weighted inner product <a, b, c> = sum_i a_i b_i c_i with c_i = 1 /
 * multiplicity (Algorithm 1), accumulated in FP64; writes one double to
 * result_dev. Deterministic for a given mesh. Async. */
sem_status sem_glsc3(sem_mesh mesh, sem_prec prec, const void* a_dev, const void* b_dev, double* result_dev,
                     void* stream);

/* Allocation-free variant of sem_glsc3 (no counterpart in the paper). Some callers cannot
 * let a library allocate device memory: programs that own every device buffer through their
 * own pool, or loops that cannot take the device-wide synchronisation of cudaMalloc/cudaFree.
 * This call computes the same <a, b, c> as sem_glsc3 (FP64 accumulation; it may differ from
 * sem_glsc3 in the last bits because blocks split the sum differently) without allocating
 * anything: its block partials and completion counter live in a static device array of
 * 33,024 bytes that every GPU loading the library holds until the process exits. Limits and
 * rules: n_local <= 33,554,432 (4096 blocks x 8192 points), else SEM_ERR_ARG; all calls share
 * the array, so calls that overlap on the GPU (other streams or host threads) race and give
 * wrong results; the counter is cleared on `stream` before each launch; the first call on
 * each device looks up the array's device address and must come before any stream capture
 * is started; that address is kept for the life of the process, so the call must not be used
 * after cudaDeviceReset. Async. */
sem_status sem_glsc3_noalloc(sem_mesh mesh, sem_prec prec, const void* a_dev, const void* b_dev, double* result_dev,
                             void* stream);

/* Jacobi preconditioner: minv_dev = 1 / diag(QQ^T A_L) on unmasked points, 0 on
 * Dirichlet points (exact diagonal of the assembled operator). Async. */
sem_status sem_jacobi(sem_mesh mesh, sem_prec prec, void* minv_dev, void* stream);

/* Right-hand side for the manufactured solution u = sin(a pi x) sin(b pi y)
 * sin(c pi z): rhs = mask(QQ^T (B f)) with f = (a^2+b^2+c^2) pi^2 u evaluated
 * at the mapped GLL points (Eq. 2's right side by GLL quadrature). Async. */
sem_status sem_rhs_sine(sem_mesh mesh, int a, int b, int c, sem_prec prec, void* rhs_dev, void* stream);

/* ---- Autotuning of the local operator ----
 * sem_autotune times every candidate implementation of A_L on this mesh (stored, on-the-fly
 * or on-the-fly with per-point scale where available, times two block shapes: elements per
 * thread block; the per-point-scale variant has one shape; for FP32 on the fly at N = 7 also
 * shape 3, the line contractions on the tensor cores: mma.sync TF32 with split operands;
 * for SEM_F64X stored and on the fly, one shape each) with CUDA events over `reps` launches each, and records the fastest for the mesh's order
 * and the precision, process-wide; SEM_AX_AUTO then uses it, and explicit variants use the
 * faster block shape. Synchronises `stream`. sem_autotune_save / sem_autotune_load write and
 * read the table as text, keyed by the GPU name (a table from another GPU model is refused
 * with SEM_ERR_ARG). The paper has no tuner (its kernels are fixed FPGA pipelines). */
typedef struct {
  int variant;            /* sem_ax_variant */
  int shape;              /* block shape choice 0 / 1, or 3 (tensor cores) */
  int elements_per_block;
  double ms;              /* mean time of one A_L application */
} sem_tune_entry;

typedef struct {
  int N;
  int prec;
  int n_candidates;
  sem_tune_entry candidates[6];
  int best;               /* index into candidates */
} sem_tune_report;

sem_status sem_autotune(sem_mesh mesh, sem_prec prec, int reps, sem_tune_report* report_host, void* stream);
/* Sets the block shape choice of one variant for an order and precision by hand (shape 0 or
 * 1, or 3 = the FP32 on-the-fly operator with its line contractions on the tensor cores, where
 * compiled: N = 7); SEM_AX_AUTO keeps its choice (or the variant given, if the order and
 * precision were never tuned). sem_autotune_clear forgets every tuning result. */
sem_status sem_autotune_set(int N, sem_prec prec, sem_ax_variant variant, int shape);
sem_status sem_autotune_clear(void);
sem_status sem_autotune_save(const char* path);
sem_status sem_autotune_load(const char* path);

/* ---- Conjugate gradient (Algorithm 1 + Jacobi z = M^-1 r) ---- */

typedef struct {
  double rtol;        /* stop when sqrt(<r,r,c> / <b,b,c>) <= rtol (checked after the r update) */
  int max_iter;       /* FP64 CG: iteration limit; mixed: limit on inner iterations in total */
  int precond;        /* 0: none, 1: Jacobi */
  int variant;        /* sem_ax_variant of the FP64 operator (SEM_AX_AUTO allowed) */
  int mixed;          /* 0: FP64 CG; 1: FP32 inner CG + FP64 iterative refinement (inner CG restarted at
                       * each refinement step); 2: the same with reliable updates: the FP32 CG keeps its
                       * search direction and its residual is replaced by the true FP64 residual each
                       * time it has dropped by inner_rtol (0.1 is typical) */
  int inner_variant;  /* sem_ax_variant of the FP32 inner operator (mixed; SEM_AX_AUTO allowed) */
  double inner_rtol;  /* relative tolerance of each inner solve (mixed = 1) or reduction between
                       * residual replacements (mixed = 2) */
  int max_outer;      /* refinement steps (mixed = 1) or residual replacements (mixed = 2) limit */
  int check_every;    /* iterations between host reads of the device convergence flag (>= 1) */
  int use_graph;      /* 1: replay check_every iterations as one captured CUDA graph; 2: as 1, except that FP64
                       * CG with stored factors on a mesh with fewer elements than the GPU has SMs runs
                       * check_every iterations in one persistent cooperative kernel (bounded grid
                       * barriers, SEM_ERR_TIMEOUT if one runs out); 0: launch every kernel */
  int f64_arith;      /* FP64 operator arithmetic: 0 native FP64, 1 double-float (SEM_F64X; stored or otf) */
} sem_cg_opts;

typedef struct {
  int iters;       /* operator applications inside the CG loop(s) */
  int outer_iters; /* refinement steps (mixed), else 0 */
  double rel_res;  /* final sqrt(<r,r,c> / <b,b,c>) as tracked by the solver */
  double time_ms;  /* wall time of the solve on the host clock */
  int status;      /* sem_status of the solve */
} sem_cg_result;

/* Fill opts with defaults: rtol 1e-10, max_iter 100000, Jacobi, STORED FP64,
 * not mixed, inner OTF with inner_rtol 1e-5, max_outer 50, check_every 50, graph on,
 * native FP64 operator arithmetic. */
sem_status sem_cg_default_opts(sem_cg_opts* opts_host);

/* Solve A x = b to rtol. b_dev, x_dev: FP64 [n_local]; x_dev holds x0 on entry
 * and the solution on return (also on NOT_CONVERGED / BREAKDOWN). b must be
 * assembled and masked (e.g. from sem_rhs_sine). The solve ends when the true residual
 * b - A x meets rtol: FP64 CG restarts from x once its recursively updated residual
 * converges (so the reported iterations include any restart), and the refinement loop
 * recomputes b - A x in FP64 every outer step. Blocks the host until done. Work vectors
 * are allocated on the first call and kept with the mesh for later solves (freed by
 * sem_mesh_destroy). */
sem_status sem_cg_solve(sem_mesh mesh, const double* b_dev, double* x_dev, const sem_cg_opts* opts,
                        sem_cg_result* result_host, void* stream);

/* Stateful FP64 CG for step-wise use (benchmarks, servers):
 *  sem_cg_create   allocates work vectors and device scalars (FP64, non-mixed opts only);
 *  sem_cg_start    r = b - A x0, z, rho; async;
 *  sem_cg_iterate  enqueues k iterations (a captured graph when opts.use_graph);
 *                  iterations after convergence are no-ops; async; when they have run,
 *                  x_dev holds the iterate of the last one (with opts.f64_arith the
 *                  operator makes each x update one iteration late, and the call ends
 *                  with the pending one);
 *  sem_cg_query    synchronises `stream` and reports iterations, residual, status;
 *  sem_cg_destroy  frees the handle. x_dev passed to sem_cg_start is updated in place
 *  and must stay valid until the last sem_cg_iterate has completed. */
sem_status sem_cg_create(sem_mesh mesh, const sem_cg_opts* opts, sem_cg* out);
sem_status sem_cg_start(sem_cg cg, const double* b_dev, double* x_dev, void* stream);
sem_status sem_cg_iterate(sem_cg cg, int k, void* stream);
sem_status sem_cg_query(sem_cg cg, sem_cg_result* result_host, void* stream);
/* Instrumented variant of sem_cg_iterate for measurement: runs k iterations eagerly
 * (no graph) with CUDA events recorded on `stream` before the first kernel and after
 * each of the three kernels of every iteration (local operator, gather-scatter, vector
 * update); synchronises `stream` and returns the elapsed time of the k iterations in
 * total_ms_host and the mean duration of each kernel in kernel_ms_host[3]. With
 * opts.f64_arith the last update interval also holds the pending x update (see
 * sem_cg_iterate), so the total covers all the work of the k iterations. */
sem_status sem_cg_iterate_timed(sem_cg cg, int k, double* total_ms_host, double* kernel_ms_host, void* stream);

sem_status sem_cg_destroy(sem_cg cg); /* waits for the streams the handle was used on */

/* Solves `count` independent problems A_i x_i = b_i (1 <= count <= 256) together by mixed
 * precision (opts->mixed = 1 or 2, as in sem_cg_solve; opts->inner_variant SEM_AX_OTF or
 * SEM_AX_AUTO, which here means SEM_AX_OTF): the FP32 inner CG iterations of all problems run in
 * shared launches over a device-side table of the problems (one operator launch per polynomial
 * order present, one gather-scatter and one vector-update launch per iteration, replayed as a
 * CUDA graph of opts->check_every iterations), and the FP64 refinement steps (residual b - A x
 * with the FP64 operator of opts->variant, x += d) are launched per problem between those runs.
 * Algorithm 1 with z = M^-1 r; the batching itself has no counterpart in the paper. Every
 * problem's arithmetic is fixed by the problem alone (partial sums per fixed part of its mesh,
 * combined in a fixed order), so each x is bit-identical to the x this call gives for the same
 * problem alone or in any other mix. It may differ in the last bits from sem_cg_solve's x, whose
 * reductions are split differently. meshes[i]: meshes of the current device (one mesh may serve
 * several problems); b_dev[i], x_dev[i]: FP64 [n_local of meshes[i]], x_dev[i] holds x0 on entry
 * and the solution on return, no two x_dev alike; results_host[count] receives each problem's
 * result (iterations are inner FP32 iterations, outer_iters the refinement steps). Blocks until
 * every problem has finished; returns SEM_OK if all converged, else the status of the first
 * problem that did not (results_host says which). Work space is allocated stream-ordered on
 * `stream` and freed before the call returns. */
sem_status sem_cg_solve_batch(int count, const sem_mesh* meshes, const double* const* b_dev, double* const* x_dev,
                              const sem_cg_opts* opts, sem_cg_result* results_host, void* stream);

/* ---- Solve server (continuous batching of Poisson solves) ----
 * Requests are queued on submit and admitted first in, first out when the device memory the
 * request needs (estimated from E, N and its options) fits in the budget and a worker thread is
 * free; the worker builds the request's mesh and right-hand side on its own CUDA stream. Then:
 *  - small mixed-precision requests (n_local <= batch_max_points, mixed = 1 or 2, on-the-fly
 *    inner operator) join the batch: one engine thread advances all of them together in shared
 *    launches over a device-side table of the admitted solves (as sem_cg_solve_batch does),
 *    admitting new ones and retiring finished ones between rounds of batch_round_iters
 *    iterations; the worker is free again as soon as it has handed the solve over;
 *  - every other request is solved by the worker with sem_cg_solve on its own stream, so these
 *    solves overlap with each other and with the batch on the GPU.
 * When a solve ends, x is copied to host memory and the request's device memory is released,
 * so new requests enter as earlier ones finish. A request's result does not depend on the other
 * requests: each takes the same path alone and in any mix, and both paths reduce in a fixed
 * order per request. A failing request (invalid mesh, non-convergence) reports its status alone.
 * The server uses the device current at sem_server_create. The paper has no server; this serves
 * its solver (Algorithm 1). */
typedef struct sem_server_s* sem_server;

typedef struct {
  int N;                                      /* polynomial order */
  int64_t num_vertices;
  const double* vert_xyz_host;                /* [num_vertices][3], copied at submit */
  int64_t E;
  const int64_t* elem_verts_host;             /* [E][8], as in sem_mesh_create, copied at submit */
  const uint8_t* dirichlet_vertex_flags_host; /* NULL or [num_vertices], copied at submit */
  int sine[3];                                /* right-hand side of sem_rhs_sine with wave numbers (a, b, c) */
  sem_cg_opts opts;                           /* solver options (mixed precision, tolerance, ...) */
} sem_request;

typedef struct {
  int status;         /* sem_status of the request; SEM_ERR_BUSY while queued or running */
  int64_t n_local;    /* length of the solution vector */
  sem_cg_result cg;   /* solver result */
  double queue_ms;    /* submit -> admitted */
  double setup_ms;    /* mesh, right-hand side */
  double solve_ms;    /* CG and copy of x to host memory */
  double latency_ms;  /* submit -> solution available in host memory */
  int batched;        /* 1 if the request was solved in the batch */
} sem_server_result;

typedef struct {
  size_t hbm_budget_bytes;  /* device memory the admitted requests may hold together */
  int max_slots;            /* worker threads (1..256): concurrent set-ups and non-batched solves */
  int64_t batch_max_points; /* requests with at most this many local points join the batch; 0: no batch */
  int batch_max_solves;     /* solves in the batch at once (1..256) */
  int batch_round_iters;    /* batched FP32 iterations between admissions and refinement steps (>= 1) */
  int size_priorities;      /* 1: each request's stream gets a CUDA stream priority by its size, the
                             * smaller the higher (the batch the highest), so short solves are served
                             * first on a busy GPU; 0: default priority for all */
} sem_server_config;

/* Defaults: the given budget and slots, batch_max_points 2,097,152, batch_max_solves 64,
 * batch_round_iters 20, size_priorities 1. */
sem_status sem_server_default_config(size_t hbm_budget_bytes, int max_slots, sem_server_config* cfg_host);
sem_status sem_server_create_config(const sem_server_config* cfg, sem_server* out);
/* sem_server_create_config with sem_server_default_config(hbm_budget_bytes, max_slots). */
sem_status sem_server_create(size_t hbm_budget_bytes, int max_slots, sem_server* out);
/* Copies the request and queues it; never waits for the GPU. SEM_ERR_ARG if the request alone
 * needs more than the budget. */
sem_status sem_server_submit(sem_server server, const sem_request* request, uint64_t* ticket);
/* Queues a solve of A x = b on a mesh the caller has built (sem_mesh_create on the server's
 * device), from x = 0, with the options `opts`. b_host: [n_local] FP64 right-hand side
 * (assembled and masked), copied at submit. On SEM_OK the mesh belongs to the server, which
 * destroys it after the solve; the streams the mesh was used on are synchronised here, so the
 * caller may release them afterwards. On any other status the caller keeps the mesh. */
sem_status sem_server_submit_mesh(sem_server server, sem_mesh mesh, const double* b_host, const sem_cg_opts* opts,
                                  uint64_t* ticket);
/* SEM_ERR_BUSY (res->status too) while the request is queued or running. When done: SEM_OK and
 * res filled; if x_host is not NULL and x_capacity >= res->n_local, x is copied into it and the
 * ticket is released (later polls of it return SEM_ERR_ARG). */
sem_status sem_server_poll(sem_server server, uint64_t ticket, double* x_host, int64_t x_capacity,
                           sem_server_result* res);
/* queued: waiting for admission; active: admitted and not finished (set-up, batch or solve);
 * bytes_in_use: their estimated device memory. Any pointer may be NULL. */
sem_status sem_server_stats(sem_server server, int* queued, int* active, size_t* bytes_in_use);
/* Counters of the batch engine: rounds run, the most solves in one round, and the mean number
 * of solves per round. Any pointer may be NULL. */
sem_status sem_server_batch_stats(sem_server server, int64_t* rounds, int* max_batch, double* mean_batch);
/* Drops queued requests, waits for the running ones, frees the server. */
sem_status sem_server_destroy(sem_server server);

/* Number of kernel launches the library enqueued since load (all entry points). */
uint64_t sem_launch_count(void);

const char* sem_last_error(void);
const char* sem_status_string(sem_status s);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
