// Internal declarations shared by the host (C++) and device (CUDA) parts of libsem.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <exception>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sem.h"

namespace sem {

constexpr int kMaxNp = SEM_MAX_N + 1;  // 12 points per direction at most

// Sets the thread-local error message and returns `s`.
sem_status fail(sem_status s, const std::string& msg);

// Runs the body of a C entry point; a C++ exception (a failed host allocation, a thread that
// cannot be started) becomes a status instead of crossing the C boundary.
template <typename F>
sem_status guarded(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(SEM_ERR_OOM, "host memory allocation failed");
  } catch (const std::exception& e) {
    return fail(SEM_ERR_CUDA, std::string("host error: ") + e.what());
  } catch (...) {
    return fail(SEM_ERR_CUDA, "unknown host error");
  }
}
sem_status cuda_fail(cudaError_t e, const char* what);
// Counts kernel launches (sem_launch_count); launches made while this thread captures a CUDA
// graph (set_capturing(true)) are not counted, the graph's launch counts them.
void count_launch(int k = 1);
void set_capturing(bool on);

}  // namespace sem

struct sem_mesh_s;

namespace sem {

// Checks shared by the C entry points (api.cpp): a mesh of the current device, a non-null
// 16-byte aligned device pointer. note_stream records a stream the mesh's memory is used on,
// so that sem_mesh_destroy waits for it before the memory is released.
sem_status check_mesh(sem_mesh_s* m);
sem_status check_ptr(const void* p, const char* name);
void note_stream(sem_mesh_s* m, cudaStream_t s);

#define SEM_TRY_STATUS(expr)              \
  do {                                    \
    const sem_status _st = (expr);        \
    if (_st != SEM_OK) return _st;        \
  } while (0)

#define SEM_CUDA_TRY(expr)                                    \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::sem::cuda_fail(_e, #expr); \
  } while (0)

// ---- host GLL tables (gll.cpp) ----
struct GllTable {
  double xi[kMaxNp], w[kMaxNp], D[kMaxNp * kMaxNp];  // D[i*Np + j] = l_j'(xi_i)
};
const GllTable& gll_table(int N);  // N in [1, SEM_MAX_N]

// ---- host topology builder (topology.cpp) ----
// Allocator whose resize() leaves new elements uninitialised: the builder writes every
// element from its worker threads, so the pages are first touched in parallel.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <typename U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <typename T>
using HostVec = std::vector<T, NoInitAlloc<T>>;

struct Topology {
  int N = 0, Np = 0;
  int64_t E = 0, n = 0, n_glob = 0;
  HostVec<int32_t> glo;      // [n] (n < 2^31)
  HostVec<uint8_t> mask;     // [n]
  HostVec<uint8_t> mult;     // [n] multiplicity of the node's global id (<= 255)
  HostVec<int32_t> seg_off;  // [n_seg + 1]
  HostVec<int32_t> seg_idx;  // [n_gs]
  HostVec<uint8_t> seg_mask; // [n_seg]
};
sem_status build_topology(int N, int64_t num_vertices, int64_t E, const int64_t* elem_verts,
                          const uint8_t* dirichlet_flags, Topology& out);

// Host arrays of the gather-scatter plan (see GsPlan below): the segments of T grouped by
// copy count, each class in ascending segment order.
struct GsHost {
  HostVec<int32_t> rec[4];  // fixed-width records, widths 1, 2, 4, 8, padded with -1
  HostVec<uint8_t> msk[4];
  HostVec<int32_t> xoff, xidx;  // segments with more than 8 copies
  HostVec<uint8_t> xmsk;
};
void build_gs_host(const Topology& T, GsHost& out);

// ---- device-side CG scalars ----
struct CgScalars {
  double rho, alpha, beta, pw, rz, rr, bb, rtol2;
  int iter, max_iter, done, status;  // status: 0 running, SEM_OK converged, else sem_status
  unsigned int ticket[5];            // last-block-done counters (reset by the last block)
};

// Element stride (in elements of the factor type) of the mesh's stored-factor arrays: the six
// P-point arrays of an element, padded so that every element block starts and ends on a
// 16-byte boundary (bulk TMA copies need both). FP64 blocks (48 P bytes) need no padding.
inline int64_t factor_stride(int Np, bool fp32) {
  const int64_t s = 6LL * Np * Np * Np;
  return fp32 ? (s + 3) / 4 * 4 : s;
}

// ---- reduction scratch ----
constexpr int kRedMax = 8192;  // upper bound of blocks of any reducing launch

// Device gather-scatter plan (k_gs.cu). The segments (global nodes with copies on element
// boundaries) are grouped by copy count: class c holds the segments with at most kGsWidth[c]
// copies as fixed-width records of copy indices (ascending local index, padded with -1),
// in ascending segment order, so one vector load gives all copies of a segment; segments
// with more copies keep CSR lists. Every class has a Dirichlet flag per segment.
constexpr int kGsClasses = 4;
constexpr int kGsWidth[kGsClasses] = {1, 2, 4, 8};
struct GsPlan {
  int64_t n[kGsClasses] = {0, 0, 0, 0};
  const int32_t* rec[kGsClasses] = {nullptr, nullptr, nullptr, nullptr};
  const uint8_t* msk[kGsClasses] = {nullptr, nullptr, nullptr, nullptr};
  int64_t nx = 0;
  const int32_t* xoff = nullptr;  // [nx + 1]
  const int32_t* xidx = nullptr;
  const uint8_t* xmsk = nullptr;
  int64_t total() const { return n[0] + n[1] + n[2] + n[3] + nx; }
};

// ---- CG layout of the operator's output (k_common.cuh cg_pos) ----
// In CG mode the FP64-data local operators (FP64, double-float) write w element by element with
// the element's boundary points (any of i, j, k in {0, N}) first and its interior points after
// them, each part in the (k, j, i) order of the local layout. The gather-scatter then finds the
// copies of neighbouring segments next to each other (copies on the i = 0 and i = N faces of
// consecutive rows are adjacent instead of a row apart, in the same DRAM sector), and the vector
// update reads w through the same map. Every other vector keeps the local layout.
struct CgMap {
  const int* perm = nullptr;      // [P]: position in the CG layout of local point loc
  int P = 0;
  unsigned long long magic = 0;   // UINT64_MAX / P + 1: idx / P = umulhi64(idx, magic) for idx < 2^31
};

// ---- batched CG over a table of solves (k_batch.cu, batch.cpp) ----
// Several independent FP32 CG solves (the inner iteration of mixed-precision refinement,
// on-the-fly factors, fused prologue) advance together: each batched kernel strides over the
// work items of every solve in a device-side table. Every work item covers a fixed part of
// one solve (an element group, a chunk of segments, a chunk of points) and writes its partial
// sums to that solve's own arrays; per-solve counters let the item that finishes a solve's
// last part form its scalars in a fixed order. A solve's arithmetic therefore does not depend
// on which other solves share the table, nor on the launch shapes.
constexpr int kBatchMax = 256;        // solves in one table
constexpr int kBatchThreads = 256;    // threads of the gather-scatter, update and flush kernels
constexpr int kBatchGsSeg = 512;      // segments per gather-scatter work item
constexpr int kBatchChunk = 4096;     // points per update / flush work item

struct BatchSolve {
  int NP;                  // points per direction
  int64_t E, n;
  const float* coef;       // [E][24] FP32 trilinear coefficients
  float *x, *p, *r, *w;    // inner CG vectors (x: the correction d)
  const float* minv;       // Jacobi inverse or null
  const uint8_t* mult;
  const double* ctab;
  GsPlan gs;
  CgScalars* st;           // inner CG scalars
  double* ax_part;         // [ax_cnt] partial <p, w> of each element group
  double* up_part;         // [2 up_cnt] partial <r, z, c>, <r, r, c> of each chunk
  int* err;
  int64_t ax_beg, ax_cnt;  // element groups: first item in the work list of its order, count
  int64_t gs_beg;          // first gather-scatter item in the table's list
  int64_t gs_at[6];        // local gather-scatter item where the classes of width 2, 4, 8, 1 and the
                           // CSR lists start; gs_at[5] = the solve's gather-scatter items
  int64_t up_beg, up_cnt;  // update / flush items (chunks of kBatchChunk points)
};
struct BatchOrder {
  int s_lo, s_hi;  // solves of this order occupy table entries [s_lo, s_hi)
  int64_t items;   // element groups of those solves
};
struct BatchTable {
  int count;
  int64_t gs_items, up_items;
  BatchOrder order[kMaxNp + 1];  // indexed by points per direction
  BatchSolve s[kBatchMax];
};

}  // namespace sem

// The mesh object behind the opaque handle.
struct sem_mesh_s {
  int N = 0, Np = 0, device = 0;
  unsigned flags = 0;
  int64_t E = 0, n = 0, n_glob = 0, n_seg = 0, n_gs = 0;
  sem::HostVec<int32_t> glo;   // host copy for the test hooks
  sem::HostVec<uint8_t> mask;  // host copy
  // device arrays
  double* coef64 = nullptr;   // [E][24] trilinear coefficients a0..a7 (x, y, z)
  float* coef32 = nullptr;    // [E][24] rounded to FP32
  double* G64 = nullptr;      // [E][6][P] or null
  float* G32 = nullptr;       // [E][factor_stride] (the [6][P] block, padded to 16 bytes) or null
  float* Gx = nullptr;        // [E][6][P] float pairs (high, low) of G for SEM_F64X, or null
  double* scale64 = nullptr;  // [n] w_i w_j w_k / det J (SEM_MESH_OTF_SCALE) or null
  float* scale32 = nullptr;
  int32_t* gs_rec[sem::kGsClasses] = {};  // gather-scatter plan (views in gs)
  uint8_t* gs_msk[sem::kGsClasses] = {};
  int32_t* gs_xoff = nullptr;
  int32_t* gs_xidx = nullptr;
  int64_t gs_xidx_count = 0;
  uint8_t* gs_xmsk = nullptr;
  sem::GsPlan gs;
  // the gather-scatter plan with copy indices in the CG layout (built with the first CG handle)
  int32_t* gs_cg_rec[sem::kGsClasses] = {};
  int32_t* gs_cg_xidx = nullptr;
  int* cg_perm = nullptr;     // [P]
  sem::GsPlan gs_cg;
  sem::CgMap cg_map;
  uint8_t* mult = nullptr;    // [n]
  double* minv64 = nullptr;   // lazily built Jacobi inverse
  float* minv32 = nullptr;
  double* ctab = nullptr;     // [256] exact reciprocals 1/m (weights c = 1/multiplicity)
  double* partials = nullptr; // reduction scratch [kRedMax] for sem_glsc3
  unsigned int* ticket = nullptr;
  int* dev_err = nullptr;     // device error word written by kernels whose bounded waits ran out
  size_t device_bytes = 0;
  // Stream-ordered memory: everything is allocated with cudaMallocAsync and released with
  // cudaFreeAsync on `home` (a private non-blocking stream) after the streams the mesh was used
  // on have drained, so destroying a mesh never waits for unrelated work on the device.
  cudaStream_t home = nullptr;
  std::vector<cudaStream_t> used;
  // work space of sem_cg_solve, kept between solves (freed with the mesh)
  sem_cg solve_cg64 = nullptr;      // FP64 CG handle
  sem_cg solve_cg32 = nullptr;      // FP32 inner CG handle (mixed precision)
  double* ir_w64 = nullptr;         // refinement: A x, residual (FP64), residual and correction (FP32)
  double* ir_r64 = nullptr;
  float* ir_r32 = nullptr;
  float* ir_d32 = nullptr;
  sem::CgScalars* ir_st = nullptr;
  double* ir_part = nullptr;
};

namespace sem {

// ---- kernel launchers (CUDA translation units) ----
struct AxLaunch {
  int64_t E;
  const void* u;      // input (plain mode)
  void* w;            // output
  const void* G;      // stored factors or null
  bool g_pairs;       // SEM_F64X: G holds float pairs (high, low) instead of FP64 values
  const void* coef;   // trilinear coefficients (otf)
  const void* scale;  // per-point w/det J (otf with stored scale)
  // CG mode (p = z + beta p prologue, <p, w> partials in the epilogue)
  const void* z;
  void* p;
  // fused CG prologue (FP32 and double-float operators, fused_cg): x += alpha p, the update
  // deferred from the previous iteration, and z = M^-1 r (minv null: no preconditioner)
  const void* r;
  const void* minv;
  void* x;
  CgScalars* st;
  double* partials;   // [gridDim.x] interior partial dots
  int* grid_out;      // receives gridDim.x used
  int* err;           // device error word (bounded waits that ran out write SEM_ERR_TIMEOUT)
  int shape;          // block shape: 0 default elements per block (the alternative if it is smaller and the
                      // mesh has fewer element groups than SMs), 1 the alternative, 2 the default always
};
sem_status launch_ax_f64_lo(int N, sem_ax_variant v, bool cg_mode, const AxLaunch& a, cudaStream_t s);  // N+1 <= 7
sem_status launch_ax_f64_hi(int N, sem_ax_variant v, bool cg_mode, const AxLaunch& a, cudaStream_t s);  // N+1 >= 8
sem_status launch_ax_f32_lo(int N, sem_ax_variant v, bool cg_mode, const AxLaunch& a, cudaStream_t s);
sem_status launch_ax_f32_hi(int N, sem_ax_variant v, bool cg_mode, const AxLaunch& a, cudaStream_t s);
inline sem_status launch_ax_f64(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  return N + 1 <= 7 ? launch_ax_f64_lo(N, v, cg, a, s) : launch_ax_f64_hi(N, v, cg, a, s);
}
inline sem_status launch_ax_f32(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  return N + 1 <= 7 ? launch_ax_f32_lo(N, v, cg, a, s) : launch_ax_f32_hi(N, v, cg, a, s);
}
// elements per block of shape choice 0 / 1 for N + 1 points per direction (host side)
int ax_elements_per_block(int N, int shape);
// Block shape choice kTensorShape: the FP32 on-the-fly operator with its line contractions on
// the tensor cores (k_ax_tc.cu), where compiled (ax_tensor_available); one element per block.
constexpr int kTensorShape = 3;
bool ax_tensor_available(int N, sem_prec prec, sem_ax_variant v);
sem_status launch_ax_tc(int N, bool cg_mode, const AxLaunch& a, cudaStream_t s);
sem_status launch_ax_f64x(int N, sem_ax_variant v, bool cg_mode, const AxLaunch& a, cudaStream_t s);
sem_status launch_ax_f64x_hi(int N, bool cg_mode, const AxLaunch& a, cudaStream_t s);      // stored, N + 1 >= 8
sem_status launch_ax_f64x_otf_lo(int N, bool cg_mode, const AxLaunch& a, cudaStream_t s);  // on the fly, N + 1 <= 7
sem_status launch_ax_f64x_otf_hi(int N, bool cg_mode, const AxLaunch& a, cudaStream_t s);  // on the fly, N + 1 >= 8
// The local operator of a mesh (api.cpp): resolves SEM_AX_AUTO and the block shape, fills the
// mesh's data pointers into `a` and launches the kernel of the precision.
sem_status launch_ax_any(sem_mesh_s* m, sem_prec prec, sem_ax_variant v, bool cg, AxLaunch a, cudaStream_t s);
// Builds the mesh's Jacobi inverse (FP64 and FP32) once; synchronises `s` when it builds it.
sem_status ensure_jacobi(sem_mesh_s* m, cudaStream_t s);
// element type of a precision's data: FP64 for SEM_F64 and SEM_F64X
inline sem_prec data_prec(sem_prec p) { return p == SEM_F32 ? SEM_F32 : SEM_F64; }

// Persistent FP64 CG for small meshes (k_cg_small.cu): `iters` iterations (fewer if the solve
// ends) in one cooperative launch of at most max_blocks blocks (one per SM), stored FP64 factors,
// w in the local layout with the plan gs. part: 3 x kRedMax doubles; bar: two words, zero at launch.
struct SmallCgLaunch {
  int64_t E = 0, n = 0;
  const double* G = nullptr;
  double *x = nullptr, *p = nullptr, *r = nullptr, *z = nullptr, *w = nullptr;
  const double* minv = nullptr;
  const uint8_t* mult = nullptr;
  const double* ctab = nullptr;
  GsPlan gs;
  CgScalars* st = nullptr;
  double* part = nullptr;
  unsigned* bar = nullptr;
  int* err = nullptr;
  int iters = 0;
  int max_blocks = 0;
};
sem_status launch_cg_small(int N, const SmallCgLaunch& a, cudaStream_t s);
// Self-test of the grid barrier: `blocks` blocks (all resident) meet at one barrier; block
// skip_block (-1: none) never arrives, so the others' bounded waits run out. status: -1 on entry,
// then SEM_OK or SEM_ERR_TIMEOUT.
sem_status launch_probe_barrier(unsigned* bar, int blocks, int skip_block, int* status, cudaStream_t s);

// element geometry (k_mesh.cu)
sem_status launch_coefficients(int64_t E, const double* X, double* coef64, float* coef32, cudaStream_t s);
// G64 / G32 (either may be null) are written with element strides gs64 / gs32.
sem_status launch_geometry(int N, int64_t E, const double* coef64, double* G64, float* G32, double* B64,
                           float* B32, int* bad_flag, int64_t gs64, int64_t gs32, cudaStream_t s,
                           double* S64 = nullptr, float* S32 = nullptr, float* GX = nullptr);
sem_status launch_coords(int N, int64_t E, const double* coef64, double* xyz, int64_t n, cudaStream_t s);
sem_status launch_local_diag(int N, int64_t E, const double* coef64, double* d, cudaStream_t s);
sem_status launch_rhs_local(int N, int64_t E, const double* coef64, int a, int b, int c, double* out,
                            cudaStream_t s);
sem_status launch_scatter(sem_prec prec, int64_t n, const int32_t* glo, const void* ug, void* ul, cudaStream_t s);
sem_status launch_invert(int64_t n, const double* d, double* m64, float* m32, cudaStream_t s);
sem_status launch_cast(int64_t n, const double* in, float* out, cudaStream_t s);

// gather-scatter (k_gs.cu)
sem_status launch_dssum(sem_prec prec, const GsPlan& g, void* u, int apply_mask, cudaStream_t s);
// CG variant: with p, also the boundary part of <p, w, c> (the operator added the interior
// part), and the last block combines the partials and sets alpha (or a breakdown status);
// with p == nullptr the operator's partials hold the whole product (whole_dot) and block 0
// sums them and sets alpha before its share of the segments.
inline bool whole_dot(sem_prec) { return true; }  // every CG-mode operator forms the whole <p, w>
// The CG layout (CgMap) is used for FP64 data (FP64 and double-float operators): their w does not
// fit in L2 and the gather-scatter is bound by DRAM sectors. FP32 CG keeps the local layout (its
// w stays in L2, and reading w through the map costs the FP32 update more than it saves).
inline bool cg_layout(sem_prec prec) { return prec != SEM_F32; }
// The same operators take the fused CG prologue (AxLaunch::r, minv, x): the update kernel
// then skips x and z, and after the last iteration launch_cg_flush adds the pending alpha p.
inline bool fused_cg(sem_prec prec) { return prec != SEM_F64; }
sem_status launch_dssum_cg(sem_prec prec, const GsPlan& g, void* w, const void* p, CgScalars* st,
                           const double* ax_partials, int ax_blocks, double* partials, cudaStream_t s);
// Batched kernels (k_batch.cu) over the device table `t` (host copy `h` gives the orders present
// and is read on the host only). One CG iteration: an operator launch per order present, then
// the gather-scatter and the update; the flush ends a run of iterations. launch_batch_status copies
// every solve's scalars to out[0 .. count).
int batch_ax_elements_per_group(int NP);
sem_status launch_batch_ax(int NP, const BatchTable* t, cudaStream_t s);
sem_status launch_batch_gs(const BatchTable* t, cudaStream_t s);
sem_status launch_batch_update(const BatchTable* t, cudaStream_t s);
sem_status launch_batch_flush(const BatchTable* t, cudaStream_t s);
sem_status launch_batch_status(const BatchTable* t, int count, CgScalars* out, cudaStream_t s);
// Jacobi: assembled diagonal inverted (0 on Dirichlet nodes) on every element-boundary copy.
sem_status launch_dssum_invert(const GsPlan& g, const double* d, double* m64, float* m32, cudaStream_t s);

// CG vector kernels (k_cg.cu)
sem_status launch_glsc3(sem_prec prec, int64_t n, const void* a, const void* b, const uint8_t* mult,
                        const double* ctab, double* partials, unsigned int* ticket, double* result, cudaStream_t s);
sem_status launch_cg_init(sem_prec prec, int64_t n, const void* b, const void* ax0, void* r, void* z, void* p,
                          const void* minv, const uint8_t* mult, const double* ctab, CgScalars* st, double* partials,
                          cudaStream_t s);
// fused (fused_cg): x and z are left to the operator's CG prologue (see AxLaunch::r). w is read
// in the CG layout through `map`.
sem_status launch_cg_update(sem_prec prec, bool fused, int64_t n, void* x, const void* p, void* r, const void* w,
                            void* z, const void* minv, const uint8_t* mult, const double* ctab, CgScalars* st,
                            double* partials, const CgMap& map, cudaStream_t s);
// perm[loc] = cg_pos of local point loc for N + 1 = NP points per direction (P entries).
sem_status launch_cg_perm(int NP, int* perm, cudaStream_t s);
// out[q] = the CG-layout position of local index in[q] (negative entries, record padding, copied).
sem_status launch_map_indices(int64_t count, const int32_t* in, int32_t* out, const CgMap& map, cudaStream_t s);
// x += alpha p if an update is pending (alpha != 0), then alpha = 0 (fused CG, at the end of
// a run of iterations)
sem_status launch_cg_flush(sem_prec prec, int64_t n, void* x, const void* p, CgScalars* st, cudaStream_t s);
// Iterative refinement (FP64 outer loop around an FP32 inner solve):
// r64 = b - w64, r32 = (float) r64, <r,r,c> and <b,b,c> into st (done when converged).
sem_status launch_ir_residual(int64_t n, const double* b, const double* w, double* r64, float* r32,
                              const uint8_t* mult, const double* ctab, CgScalars* st, double* partials,
                              cudaStream_t s);
// x64 += (double) d32
sem_status launch_ir_correct(int64_t n, double* x, const float* d, cudaStream_t s);
// Residual replacement of the FP32 CG (reliable updates): r = rnew, z = M^-1 r, new rho and
// beta = rho_new / rho, p kept; partials needs 2 x gridDim doubles.
sem_status launch_cg_replace(int64_t n, const float* rnew, float* r, float* z, const float* minv, const uint8_t* mult,
                             const double* ctab, CgScalars* st, double* partials, cudaStream_t s);

}  // namespace sem

namespace sem {

// ---- batched mixed-precision solves (batch.cpp) ----
// One solve of the batch engine: A x = b on mesh m (FP64 b and x, device), refined in FP64
// around an FP32 inner CG whose iterations run in the shared batched launches. The engine
// owns the work space it allocates for the job; the caller keeps m, b and x.
struct BatchJob {
  sem_mesh m = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  sem_cg_opts o{};
  void* user = nullptr;      // the caller's tag
  // result (valid once the engine reports the job done)
  sem_cg_result res{};
  // engine state
  int state = 0;
  int total_inner = 0, outer = 0, before = 0;
  int64_t groups = 0, chunks = 0;
  float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *w32 = nullptr, *d32 = nullptr, *rr32 = nullptr;
  double *w64 = nullptr, *r64 = nullptr;
  CgScalars *ist = nullptr, *ost = nullptr;
  double *ax_part = nullptr, *up_part = nullptr, *init_part = nullptr, *opart = nullptr;
  CgScalars ost_h{};  // the last refinement residual's scalars
};

class BatchEngine {
 public:
  BatchEngine() = default;
  BatchEngine(const BatchEngine&) = delete;
  BatchEngine& operator=(const BatchEngine&) = delete;
  ~BatchEngine();
  // All work is enqueued on `s` (which must outlive the engine).
  sem_status init(cudaStream_t s);
  // Checks the job's options (mixed 1 or 2), builds the mesh's Jacobi inverse if needed,
  // allocates the job's work space on the engine's stream and queues the job.
  sem_status add(BatchJob* j);
  // One round: the FP64 refinement steps that are due, then `iters` batched FP32 CG iterations
  // of every job whose inner solve runs, then their statuses (synchronises the stream).
  // Finished jobs move to the done list.
  sem_status round(int iters);
  std::vector<BatchJob*> take_done();
  // Frees the job's work space (stream-ordered on the engine's stream).
  void release(BatchJob* j);
  size_t running() const { return jobs_.size(); }

 private:
  sem_status residual(BatchJob* j, CgScalars* host_out);
  sem_status start_inner(BatchJob* j);
  void finish(BatchJob* j, int status);
  sem_status upload_table();
  sem_status iterate(int iters);
  cudaStream_t s_ = nullptr;
  cudaStream_t cap_ = nullptr;  // private stream for graph capture
  BatchTable* tab_d_ = nullptr;
  BatchTable* tab_h_ = nullptr;  // pinned
  CgScalars* stat_d_ = nullptr;
  CgScalars* stat_h_ = nullptr;  // pinned [kBatchMax]
  CgScalars* ost_pin_ = nullptr; // pinned [kBatchMax]: refinement residual scalars
  std::vector<BatchJob*> jobs_;   // not finished
  std::vector<BatchJob*> table_;  // jobs in the device table, in table order
  std::vector<BatchJob*> done_;
  bool dirty_ = true;
  struct Graph {
    unsigned orders;
    int iters;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs_;
};

}  // namespace sem
