// C ABI of libsem: mesh lifecycle, operator entry points and the conjugate-gradient
// drivers (Algorithm 1 with Jacobi, FP64; and FP32-inner / FP64-outer iterative refinement).
#include <atomic>
#include <chrono>
#include <cmath>
#include <algorithm>
#include <cstring>
#include <cstdio>
#include <fstream>
#include <memory>
#include <mutex>
#include <sstream>

#include "sem_internal.h"

namespace sem {

namespace {
thread_local std::string t_last_error;
thread_local bool t_capturing = false;
std::atomic<uint64_t> g_launches{0};
}  // namespace

sem_status fail(sem_status s, const std::string& msg) {
  t_last_error = msg;
  return s;
}

sem_status cuda_fail(cudaError_t e, const char* what) {
  t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return SEM_ERR_OOM;
  return SEM_ERR_CUDA;
}

void count_launch(int k) {
  if (!t_capturing) g_launches.fetch_add(static_cast<uint64_t>(k), std::memory_order_relaxed);
}

void set_capturing(bool on) { t_capturing = on; }

void note_stream(sem_mesh m, cudaStream_t s) {
  for (cudaStream_t u : m->used)
    if (u == s) return;
  m->used.push_back(s);
}

sem_status check_mesh(sem_mesh m) {
  if (!m) return fail(SEM_ERR_ARG, "null mesh");
  int dev = -1;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != m->device) return fail(SEM_ERR_ARG, "the mesh belongs to another CUDA device than the current one");
  return SEM_OK;
}

sem_status check_ptr(const void* p, const char* name) {
  if (!p) return fail(SEM_ERR_ARG, std::string(name) + " is null");
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return fail(SEM_ERR_ARG, std::string(name) + " is not 16-byte aligned");
  return SEM_OK;
}

namespace {

// Stream-ordered allocation on `s` (the memory is usable on `s` at once and on other streams
// once `s` has been synchronised).
template <typename T>
sem_status dmalloc(T** p, size_t count, size_t* acc, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) count = 1;
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA,
                "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  if (acc) *acc += bytes;
  return SEM_OK;
}

template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

#define SEM_TRY(expr)                 \
  do {                                \
    sem_status _s = (expr);           \
    if (_s != SEM_OK) return _s;      \
  } while (0)

sem_status check_prec(int prec) {
  if (prec != SEM_F64 && prec != SEM_F32 && prec != SEM_F64X)
    return fail(SEM_ERR_ARG, "precision must be SEM_F64, SEM_F32 or SEM_F64X");
  return SEM_OK;
}

void cg_free(sem_cg c);

// Waits for the streams the mesh was used on, then returns its memory on the private stream.
void free_mesh(sem_mesh m) {
  for (cudaStream_t u : m->used) cudaStreamSynchronize(u);
  if (m->solve_cg64) cg_free(m->solve_cg64);
  if (m->solve_cg32) cg_free(m->solve_cg32);
  m->solve_cg64 = m->solve_cg32 = nullptr;
  cudaStream_t h = m->home;
  dfree(m->ir_w64, h);
  dfree(m->ir_r64, h);
  dfree(m->ir_r32, h);
  dfree(m->ir_d32, h);
  dfree(m->ir_st, h);
  dfree(m->ir_part, h);
  dfree(m->coef64, h);
  dfree(m->coef32, h);
  dfree(m->G64, h);
  dfree(m->G32, h);
  dfree(m->Gx, h);
  dfree(m->scale64, h);
  dfree(m->scale32, h);
  for (int c = 0; c < kGsClasses; ++c) {
    dfree(m->gs_rec[c], h);
    dfree(m->gs_msk[c], h);
  }
  dfree(m->gs_xoff, h);
  dfree(m->gs_xidx, h);
  for (int c = 0; c < kGsClasses; ++c) dfree(m->gs_cg_rec[c], h);
  dfree(m->gs_cg_xidx, h);
  dfree(m->cg_perm, h);
  dfree(m->gs_xmsk, h);
  dfree(m->mult, h);
  dfree(m->minv64, h);
  dfree(m->minv32, h);
  dfree(m->ctab, h);
  dfree(m->partials, h);
  dfree(m->ticket, h);
  dfree(m->dev_err, h);
  if (h) {
    cudaStreamSynchronize(h);
    cudaStreamDestroy(h);
  }
  m->home = nullptr;
  m->used.clear();
}

// Process-wide tuning results per precision (F64, F32, F64X) and order: the best variant and,
// for each variant, its faster block shape.
struct TuneSlot {
  bool valid = false;
  sem_ax_variant best = SEM_AX_STORED;
  int shape[3] = {0, 0, 0};  // per variant slot: STORED, OTF, OTF_SCALE
  double ms[3] = {0, 0, 0};
};
inline int vslot(sem_ax_variant v) { return v == SEM_AX_OTF_SCALE ? 2 : static_cast<int>(v); }
std::mutex g_tune_mu;
TuneSlot g_tune[3][SEM_MAX_N + 1];

// Stored factors the local operator of precision `prec` reads: FP32 for SEM_F32; for SEM_F64X the
// float pairs if the mesh has them, else the FP64 factors (split in the kernel); FP64 otherwise.
const void* stored_factors(sem_mesh m, sem_prec prec, bool* pairs) {
  *pairs = false;
  if (prec == SEM_F32) return m->G32;
  if (prec == SEM_F64X && m->Gx) {
    *pairs = true;
    return m->Gx;
  }
  return m->G64;
}
bool has_factors(sem_mesh m, sem_prec prec) {
  bool pairs;
  return stored_factors(m, prec, &pairs) != nullptr;
}
bool has_scales(sem_mesh m) { return m->scale64 != nullptr; }

// Resolves SEM_AX_AUTO and picks the tuned block shape.
void resolve_variant(sem_mesh m, sem_prec prec, sem_ax_variant v, sem_ax_variant* out_v, int* out_shape) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const TuneSlot& t = g_tune[prec][m->N];
  sem_ax_variant r = v;
  if (v == SEM_AX_AUTO) {
    if (t.valid && (t.best == SEM_AX_OTF || (t.best == SEM_AX_STORED && has_factors(m, prec)) ||
                    (t.best == SEM_AX_OTF_SCALE && has_scales(m))))
      r = t.best;
    else
      r = has_factors(m, prec) ? SEM_AX_STORED : SEM_AX_OTF;
    if (prec == SEM_F64X && r == SEM_AX_OTF_SCALE) r = has_factors(m, prec) ? SEM_AX_STORED : SEM_AX_OTF;
  }
  *out_v = r;
  *out_shape = t.valid ? t.shape[vslot(r)] : 0;
}

}  // namespace

sem_status launch_ax_any(sem_mesh m, sem_prec prec, sem_ax_variant v, bool cg, AxLaunch a, cudaStream_t s) {
  resolve_variant(m, prec, v, &v, &a.shape);
  a.E = m->E;
  a.err = m->dev_err;
  const bool fp64_data = prec != SEM_F32;
  a.coef = fp64_data ? static_cast<const void*>(m->coef64) : static_cast<const void*>(m->coef32);
  a.G = stored_factors(m, prec, &a.g_pairs);
  a.scale = fp64_data ? static_cast<const void*>(m->scale64) : static_cast<const void*>(m->scale32);
  if (v == SEM_AX_STORED && !a.G)
    return fail(SEM_ERR_ARG, "stored factors of this precision were not requested at mesh creation");
  if (v == SEM_AX_OTF_SCALE && !a.scale)
    return fail(SEM_ERR_ARG, "per-point scales were not requested at mesh creation (SEM_MESH_OTF_SCALE)");
  if (prec == SEM_F64X) return launch_ax_f64x(m->N, v, cg, a, s);
  if (a.shape == kTensorShape && ax_tensor_available(m->N, prec, v)) return launch_ax_tc(m->N, cg, a, s);
  return prec == SEM_F64 ? launch_ax_f64(m->N, v, cg, a, s) : launch_ax_f32(m->N, v, cg, a, s);
}

// Jacobi inverse diagonal, built once per mesh in FP64 (and rounded to FP32).
sem_status ensure_jacobi(sem_mesh m, cudaStream_t s) {
  if (m->minv64) return SEM_OK;
  note_stream(m, s);
  double* d = nullptr;
  SEM_TRY(dmalloc(&d, m->n, nullptr, s));
  sem_status st = SEM_OK;
  size_t bytes = 0;
  if ((st = dmalloc(&m->minv64, m->n, &bytes, s)) == SEM_OK && (st = dmalloc(&m->minv32, m->n, &bytes, s)) == SEM_OK &&
      (st = launch_local_diag(m->N, m->E, m->coef64, d, s)) == SEM_OK &&
      (st = launch_invert(m->n, d, m->minv64, m->minv32, s)) == SEM_OK &&
      (st = launch_dssum_invert(m->gs, d, m->minv64, m->minv32, s)) == SEM_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize (Jacobi set-up)");
  }
  dfree(d, s);
  if (st != SEM_OK) {
    dfree(m->minv64, s);
    dfree(m->minv32, s);
    cudaStreamSynchronize(s);
    return st;
  }
  m->device_bytes += bytes;
  return SEM_OK;
}

// The CG layout of the operator's output (CgMap) and the gather-scatter plan in it, built once
// per mesh on its first CG handle: the plan's copy indices mapped on the device.
sem_status ensure_cg_layout(sem_mesh m, cudaStream_t s) {
  if (m->cg_perm) return SEM_OK;
  note_stream(m, s);
  const int P = m->Np * m->Np * m->Np;
  size_t bytes = 0;
  sem_status st = dmalloc(&m->cg_perm, static_cast<size_t>(P), &bytes, s);
  if (st == SEM_OK) st = launch_cg_perm(m->Np, m->cg_perm, s);
  CgMap map;
  map.perm = m->cg_perm;
  map.P = P;
  map.magic = ~0ull / static_cast<unsigned long long>(P) + 1ull;
  GsPlan g = m->gs;
  for (int c = 0; c < kGsClasses && st == SEM_OK; ++c) {
    const int64_t cnt = m->gs.n[c] * kGsWidth[c];
    if (cnt == 0) continue;
    if ((st = dmalloc(&m->gs_cg_rec[c], static_cast<size_t>(cnt), &bytes, s)) == SEM_OK)
      st = launch_map_indices(cnt, m->gs_rec[c], m->gs_cg_rec[c], map, s);
    g.rec[c] = m->gs_cg_rec[c];
  }
  if (st == SEM_OK && m->gs_xidx_count > 0) {
    if ((st = dmalloc(&m->gs_cg_xidx, static_cast<size_t>(m->gs_xidx_count), &bytes, s)) == SEM_OK)
      st = launch_map_indices(m->gs_xidx_count, m->gs_xidx, m->gs_cg_xidx, map, s);
    g.xidx = m->gs_cg_xidx;
  }
  if (st == SEM_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize (CG layout)");
  }
  if (st != SEM_OK) {
    for (int c = 0; c < kGsClasses; ++c) dfree(m->gs_cg_rec[c], s);
    dfree(m->gs_cg_xidx, s);
    dfree(m->cg_perm, s);
    cudaStreamSynchronize(s);
    return st;
  }
  m->gs_cg = g;
  m->cg_map = map;
  m->device_bytes += bytes;
  return SEM_OK;
}

}  // namespace sem

using namespace sem;

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------

extern "C" sem_status sem_mesh_create(int N, int64_t nv, const double* vert_xyz, int64_t E, const int64_t* elem_verts,
                                      const uint8_t* dflags, unsigned flags, void* stream, sem_mesh* out) {
  return guarded([&]() -> sem_status {
    if (!out) return fail(SEM_ERR_ARG, "out is null");
    *out = nullptr;
    if (!vert_xyz || !elem_verts) return fail(SEM_ERR_ARG, "vert_xyz and elem_verts must be given");
    if (flags & ~(SEM_MESH_F64_STORED | SEM_MESH_F32_STORED | SEM_MESH_OTF_SCALE | SEM_MESH_F64X_STORED))
      return fail(SEM_ERR_ARG, "unknown mesh flags");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Topology T;
    SEM_TRY(build_topology(N, nv, E, elem_verts, dflags, T));
    for (int64_t v = 0; v < nv; ++v)
      for (int c = 0; c < 3; ++c)
        if (!std::isfinite(vert_xyz[3 * v + c])) return fail(SEM_ERR_MESH, "non-finite vertex coordinate");

    auto m = std::make_unique<sem_mesh_s>();
    SEM_CUDA_TRY(cudaGetDevice(&m->device));
    m->N = N;
    m->Np = N + 1;
    m->flags = flags;
    m->E = E;
    m->n = T.n;
    m->n_glob = T.n_glob;
    m->n_seg = static_cast<int64_t>(T.seg_mask.size());
    m->n_gs = static_cast<int64_t>(T.seg_idx.size());
    const int64_t P = static_cast<int64_t>(m->Np) * m->Np * m->Np;

    std::vector<double> X(static_cast<size_t>(E) * 24);
    for (int64_t e = 0; e < E; ++e)
      for (int v = 0; v < 8; ++v)
        for (int c = 0; c < 3; ++c) X[e * 24 + v * 3 + c] = vert_xyz[3 * elem_verts[e * 8 + v] + c];
    std::vector<double> ctab(256, 0.0);
    for (int k = 1; k < 256; ++k) ctab[k] = 1.0 / k;

    double* Xd = nullptr;
    int* bad = nullptr;
    SEM_CUDA_TRY(cudaStreamCreateWithFlags(&m->home, cudaStreamNonBlocking));
    m->used.push_back(s);
    auto cleanup = [&](sem_status st) {
      dfree(Xd, s);
      dfree(bad, s);
      if (st != SEM_OK) free_mesh(m.get());
      return st;
    };
    size_t& acc = m->device_bytes;
    sem_status st = SEM_OK;
  #define SEM_STEP(expr)               \
    do {                               \
      st = (expr);                     \
      if (st != SEM_OK) return cleanup(st); \
    } while (0)
  #define SEM_CSTEP(expr)                                  \
    do {                                                   \
      cudaError_t _e = (expr);                             \
      if (_e != cudaSuccess) return cleanup(cuda_fail(_e, #expr)); \
    } while (0)
    SEM_STEP(dmalloc(&Xd, X.size(), nullptr, s));
    SEM_STEP(dmalloc(&bad, 1, nullptr, s));
    SEM_STEP(dmalloc(&m->coef64, static_cast<size_t>(E) * 24, &acc, s));
    SEM_STEP(dmalloc(&m->coef32, static_cast<size_t>(E) * 24, &acc, s));
    if (flags & SEM_MESH_F64_STORED) SEM_STEP(dmalloc(&m->G64, static_cast<size_t>(E * 6 * P), &acc, s));
    if (flags & SEM_MESH_F64X_STORED) SEM_STEP(dmalloc(&m->Gx, static_cast<size_t>(2 * E * 6 * P), &acc, s));
    if (flags & SEM_MESH_F32_STORED)
      SEM_STEP(dmalloc(&m->G32, static_cast<size_t>(E * factor_stride(m->Np, true)), &acc, s));
    if (flags & SEM_MESH_OTF_SCALE) {
      SEM_STEP(dmalloc(&m->scale64, static_cast<size_t>(E * P), &acc, s));
      SEM_STEP(dmalloc(&m->scale32, static_cast<size_t>(E * P), &acc, s));
    }
    GsHost H;
    build_gs_host(T, H);
    for (int c = 0; c < kGsClasses; ++c) {
      SEM_STEP(dmalloc(&m->gs_rec[c], H.rec[c].size(), &acc, s));
      SEM_STEP(dmalloc(&m->gs_msk[c], H.msk[c].size(), &acc, s));
    }
    SEM_STEP(dmalloc(&m->gs_xoff, H.xoff.size(), &acc, s));
    SEM_STEP(dmalloc(&m->gs_xidx, H.xidx.size(), &acc, s));
    m->gs_xidx_count = static_cast<int64_t>(H.xidx.size());
    SEM_STEP(dmalloc(&m->gs_xmsk, H.xmsk.size(), &acc, s));
    SEM_STEP(dmalloc(&m->mult, T.mult.size(), &acc, s));
    SEM_STEP(dmalloc(&m->ctab, 256, &acc, s));
    SEM_STEP(dmalloc(&m->partials, kRedMax, &acc, s));
    SEM_STEP(dmalloc(&m->ticket, 1, &acc, s));
    SEM_STEP(dmalloc(&m->dev_err, 1, &acc, s));
    SEM_CSTEP(cudaMemsetAsync(m->dev_err, 0, sizeof(int), s));
    SEM_CSTEP(cudaMemcpyAsync(Xd, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    for (int c = 0; c < kGsClasses; ++c) {
      m->gs.n[c] = static_cast<int64_t>(H.msk[c].size());
      m->gs.rec[c] = m->gs_rec[c];
      m->gs.msk[c] = m->gs_msk[c];
      if (!H.msk[c].empty()) {
        SEM_CSTEP(cudaMemcpyAsync(m->gs_rec[c], H.rec[c].data(), H.rec[c].size() * 4, cudaMemcpyHostToDevice, s));
        SEM_CSTEP(cudaMemcpyAsync(m->gs_msk[c], H.msk[c].data(), H.msk[c].size(), cudaMemcpyHostToDevice, s));
      }
    }
    m->gs.nx = static_cast<int64_t>(H.xmsk.size());
    m->gs.xoff = m->gs_xoff;
    m->gs.xidx = m->gs_xidx;
    m->gs.xmsk = m->gs_xmsk;
    SEM_CSTEP(cudaMemcpyAsync(m->gs_xoff, H.xoff.data(), H.xoff.size() * 4, cudaMemcpyHostToDevice, s));
    if (!H.xmsk.empty()) {
      SEM_CSTEP(cudaMemcpyAsync(m->gs_xidx, H.xidx.data(), H.xidx.size() * 4, cudaMemcpyHostToDevice, s));
      SEM_CSTEP(cudaMemcpyAsync(m->gs_xmsk, H.xmsk.data(), H.xmsk.size(), cudaMemcpyHostToDevice, s));
    }
    SEM_CSTEP(cudaMemcpyAsync(m->mult, T.mult.data(), T.mult.size(), cudaMemcpyHostToDevice, s));
    SEM_CSTEP(cudaMemcpyAsync(m->ctab, ctab.data(), 256 * sizeof(double), cudaMemcpyHostToDevice, s));
    SEM_CSTEP(cudaMemsetAsync(m->ticket, 0, sizeof(unsigned int), s));
    SEM_CSTEP(cudaMemsetAsync(bad, 0, sizeof(int), s));
    SEM_STEP(launch_coefficients(E, Xd, m->coef64, m->coef32, s));
    // geometric factors (and the det J > 0 check at every GLL point)
    SEM_STEP(launch_geometry(N, E, m->coef64, m->G64, m->G32, nullptr, nullptr, bad, factor_stride(m->Np, false),
                             factor_stride(m->Np, true), s, m->scale64, m->scale32, m->Gx));
    int bad_h = 0;
    SEM_CSTEP(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CSTEP(cudaStreamSynchronize(s));
    if (bad_h) return cleanup(fail(SEM_ERR_MESH, "det J <= 0 (inverted or degenerate element)"));
  #undef SEM_STEP
  #undef SEM_CSTEP
    cleanup(SEM_OK);
    m->glo = std::move(T.glo);
    m->mask = std::move(T.mask);
    *out = m.release();
    return SEM_OK;
  });
}

extern "C" sem_status sem_mesh_numbering(int N, int64_t nv, int64_t E, const int64_t* elem_verts,
                                         const uint8_t* dflags, int64_t* glo_out, uint8_t* mask_out,
                                         int64_t* n_glob_out) {
  return guarded([&]() -> sem_status {
    Topology T;
    SEM_TRY(build_topology(N, nv, E, elem_verts, dflags, T));
    if (glo_out)
      for (size_t i = 0; i < T.glo.size(); ++i) glo_out[i] = T.glo[i];
    if (mask_out) std::memcpy(mask_out, T.mask.data(), T.mask.size());
    if (n_glob_out) *n_glob_out = T.n_glob;
    return SEM_OK;
  });
}

extern "C" sem_status sem_mesh_destroy(sem_mesh m) {
  return guarded([&]() -> sem_status {
    if (!m) return SEM_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != m->device) cudaSetDevice(m->device);
    free_mesh(m);
    if (cur != m->device) cudaSetDevice(cur);
    delete m;
    return SEM_OK;
  });
}

extern "C" sem_status sem_mesh_info(sem_mesh m, int64_t* n_local, int64_t* n_glob, int64_t* n_shared_seg) {
  return guarded([&]() -> sem_status {
    if (!m) return fail(SEM_ERR_ARG, "null mesh");
    if (n_local) *n_local = m->n;
    if (n_glob) *n_glob = m->n_glob;
    if (n_shared_seg) *n_shared_seg = m->n_seg;
    return SEM_OK;
  });
}

extern "C" sem_status sem_mesh_get_info(sem_mesh m, sem_mesh_info_t* info) {
  return guarded([&]() -> sem_status {
    if (!m || !info) return fail(SEM_ERR_ARG, "null argument");
    info->N = m->N;
    info->Np = m->Np;
    info->E = m->E;
    info->n_local = m->n;
    info->n_glob = m->n_glob;
    info->n_seg = m->n_seg;
    info->n_gs = m->n_gs;
    info->flags = m->flags;
    info->device = m->device;
    info->device_bytes = m->device_bytes;
    return SEM_OK;
  });
}

extern "C" sem_status sem_mesh_get_glo_num(sem_mesh m, int64_t* out) {
  return guarded([&]() -> sem_status {
    if (!m || !out) return fail(SEM_ERR_ARG, "null argument");
    for (size_t i = 0; i < m->glo.size(); ++i) out[i] = m->glo[i];
    return SEM_OK;
  });
}

extern "C" sem_status sem_mesh_get_mask(sem_mesh m, uint8_t* out) {
  return guarded([&]() -> sem_status {
    if (!m || !out) return fail(SEM_ERR_ARG, "null argument");
    std::memcpy(out, m->mask.data(), m->mask.size());
    return SEM_OK;
  });
}

// Rebuilt from the device plan: every segment's copies (records without padding, CSR lists)
// with its flag, segments in ascending order of their first copy (= ascending global id).
extern "C" sem_status sem_mesh_get_segments(sem_mesh m, int32_t* off, int32_t* idx, uint8_t* smask) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    static constexpr int kW[kGsClasses] = {1, 2, 4, 8};
    struct Seg {
      int32_t first;
      int cls;
      int64_t at;
    };
    std::vector<int32_t> rec[kGsClasses], xoff(m->gs.nx + 1), xidx;
    std::vector<uint8_t> msk[kGsClasses], xmsk(m->gs.nx);
    std::vector<Seg> segs;
    segs.reserve(static_cast<size_t>(m->n_seg));
    for (int c = 0; c < kGsClasses; ++c) {
      rec[c].resize(m->gs.n[c] * kW[c]);
      msk[c].resize(m->gs.n[c]);
      if (m->gs.n[c] == 0) continue;
      SEM_CUDA_TRY(cudaMemcpy(rec[c].data(), m->gs_rec[c], rec[c].size() * 4, cudaMemcpyDeviceToHost));
      SEM_CUDA_TRY(cudaMemcpy(msk[c].data(), m->gs_msk[c], msk[c].size(), cudaMemcpyDeviceToHost));
      for (int64_t q = 0; q < m->gs.n[c]; ++q) segs.push_back({rec[c][q * kW[c]], c, q});
    }
    SEM_CUDA_TRY(cudaMemcpy(xoff.data(), m->gs_xoff, xoff.size() * 4, cudaMemcpyDeviceToHost));
    if (m->gs.nx > 0) {
      xidx.resize(xoff.back());
      SEM_CUDA_TRY(cudaMemcpy(xidx.data(), m->gs_xidx, xidx.size() * 4, cudaMemcpyDeviceToHost));
      SEM_CUDA_TRY(cudaMemcpy(xmsk.data(), m->gs_xmsk, xmsk.size(), cudaMemcpyDeviceToHost));
      for (int64_t q = 0; q < m->gs.nx; ++q) segs.push_back({xidx[xoff[q]], kGsClasses, q});
    }
    std::sort(segs.begin(), segs.end(), [](const Seg& a, const Seg& b) { return a.first < b.first; });
    int64_t o = 0;
    for (size_t k = 0; k < segs.size(); ++k) {
      const Seg& g = segs[k];
      if (off) off[k] = static_cast<int32_t>(o);
      if (g.cls < kGsClasses) {
        if (smask) smask[k] = msk[g.cls][g.at];
        for (int q = 0; q < kW[g.cls]; ++q) {
          const int32_t v = rec[g.cls][g.at * kW[g.cls] + q];
          if (v < 0) break;
          if (idx) idx[o] = v;
          ++o;
        }
      } else {
        if (smask) smask[k] = xmsk[g.at];
        for (int32_t q = xoff[g.at]; q < xoff[g.at + 1]; ++q) {
          if (idx) idx[o] = xidx[q];
          ++o;
        }
      }
    }
    if (off) off[segs.size()] = static_cast<int32_t>(o);
    return SEM_OK;
  });
}

extern "C" sem_status sem_mesh_coords(sem_mesh m, double* xyz, void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_ptr(xyz, "xyz_dev"));
    note_stream(m, static_cast<cudaStream_t>(stream));
    return launch_coords(m->N, m->E, m->coef64, xyz, m->n, static_cast<cudaStream_t>(stream));
  });
}

extern "C" sem_status sem_mesh_geometry(sem_mesh m, sem_prec prec, void* G, void* B, void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    if (G) SEM_TRY(check_ptr(G, "G_dev"));
    if (B) SEM_TRY(check_ptr(B, "B_dev"));
    if (!G && !B) return SEM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    note_stream(m, s);
    int* bad = nullptr;
    SEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&bad), sizeof(int), s));
    const bool f64 = prec != SEM_F32;
    sem_status st = launch_geometry(m->N, m->E, m->coef64, f64 ? static_cast<double*>(G) : nullptr,
                                    prec == SEM_F32 ? static_cast<float*>(G) : nullptr,
                                    f64 ? static_cast<double*>(B) : nullptr,
                                    prec == SEM_F32 ? static_cast<float*>(B) : nullptr, bad, 6LL * m->Np * m->Np * m->Np,
                                    6LL * m->Np * m->Np * m->Np, s);
    cudaFreeAsync(bad, s);
    return st;
  });
}

extern "C" sem_status sem_scatter(sem_mesh m, sem_prec prec, const void* ug, void* ul, void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    SEM_TRY(check_ptr(ug, "u_glob_dev"));
    SEM_TRY(check_ptr(ul, "u_local_dev"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    note_stream(m, s);
    const HostVec<int32_t>& g32 = m->glo;
    int32_t* gd = nullptr;
    SEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&gd), g32.size() * 4, s));
    sem_status st = SEM_OK;
    cudaError_t e = cudaMemcpyAsync(gd, g32.data(), g32.size() * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync (numbering)");
    if (st == SEM_OK) st = launch_scatter(data_prec(prec), m->n, gd, ug, ul, s);
    // the host copy must outlive the transfer
    e = cudaStreamSynchronize(s);
    if (st == SEM_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    cudaFreeAsync(gd, s);
    return st;
  });
}

extern "C" sem_status sem_ax(sem_mesh m, sem_ax_variant v, sem_prec prec, const void* u, void* w, int assemble,
                             void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    if (v < SEM_AX_STORED || v > SEM_AX_OTF_SCALE) return fail(SEM_ERR_ARG, "unknown Ax variant");
    SEM_TRY(check_ptr(u, "u_dev"));
    SEM_TRY(check_ptr(w, "w_dev"));
    if (u == w) return fail(SEM_ERR_ARG, "u and w must not overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    note_stream(m, s);
    AxLaunch a{};
    a.u = u;
    a.w = w;
    SEM_TRY(launch_ax_any(m, prec, v, false, a, s));
    if (assemble) SEM_TRY(launch_dssum(data_prec(prec), m->gs, w, 1, s));
    return SEM_OK;
  });
}

extern "C" sem_status sem_dssum(sem_mesh m, sem_prec prec, void* u, int apply_mask, void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    SEM_TRY(check_ptr(u, "u_dev"));
    note_stream(m, static_cast<cudaStream_t>(stream));
    return launch_dssum(data_prec(prec), m->gs, u, apply_mask,
                        static_cast<cudaStream_t>(stream));
  });
}

extern "C" sem_status sem_glsc3(sem_mesh m, sem_prec prec, const void* a, const void* b, double* result,
                                void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    SEM_TRY(check_ptr(a, "a_dev"));
    SEM_TRY(check_ptr(b, "b_dev"));
    if (!result) return fail(SEM_ERR_ARG, "result_dev is null");
    note_stream(m, static_cast<cudaStream_t>(stream));
    return launch_glsc3(data_prec(prec), m->n, a, b, m->mult, m->ctab, m->partials, m->ticket, result,
                        static_cast<cudaStream_t>(stream));
  });
}

extern "C" sem_status sem_jacobi(sem_mesh m, sem_prec prec, void* minv, void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    SEM_TRY(check_ptr(minv, "minv_dev"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    note_stream(m, s);
    SEM_TRY(ensure_jacobi(m, s));
    const bool f32 = prec == SEM_F32;
    const size_t bytes = m->n * (f32 ? sizeof(float) : sizeof(double));
    SEM_CUDA_TRY(cudaMemcpyAsync(minv, f32 ? static_cast<void*>(m->minv32) : static_cast<void*>(m->minv64),
                                 bytes, cudaMemcpyDeviceToDevice, s));
    return SEM_OK;
  });
}

extern "C" sem_status sem_rhs_sine(sem_mesh m, int a, int b, int c, sem_prec prec, void* rhs, void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    SEM_TRY(check_ptr(rhs, "rhs_dev"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    note_stream(m, s);
    double* tmp = static_cast<double*>(rhs);
    if (prec == SEM_F32) SEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&tmp), m->n * sizeof(double), s));
    sem_status st = launch_rhs_local(m->N, m->E, m->coef64, a, b, c, tmp, s);
    if (st == SEM_OK) st = launch_dssum(SEM_F64, m->gs, tmp, 1, s);
    if (prec == SEM_F32) {
      if (st == SEM_OK) st = launch_cast(m->n, tmp, static_cast<float*>(rhs), s);
      cudaFreeAsync(tmp, s);
    }
    return st;
  });
}

// ---------------------------------------------------------------------------
// conjugate gradient
// ---------------------------------------------------------------------------

struct sem_cg_s {
  sem_mesh m = nullptr;
  sem_prec prec = SEM_F64;
  sem_ax_variant variant = SEM_AX_STORED;
  int precond = 1, max_iter = 0, use_graph = 1;
  double rtol = 0;
  void *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr;
  void* x = nullptr;
  const void* b = nullptr;
  CgScalars* st = nullptr;
  CgScalars st_host{};  // host mirror of the device scalars (pageable: no device-wide synchronisation)
  double *ax_part = nullptr, *gs_part = nullptr, *upd_part = nullptr, *init_part = nullptr;
  int ax_blocks = 0;
  cudaStream_t cap = nullptr;     // private stream: allocation, graph capture, release
  unsigned* bar = nullptr;        // grid barrier words of the persistent small-mesh kernel
  std::vector<cudaStream_t> used; // streams the solver's work was enqueued on
  cudaGraphExec_t exec = nullptr;
  int exec_k = 0;
  void* exec_x = nullptr;
};

namespace sem {
namespace {

const void* minv_of(sem_cg c) {
  if (!c->precond) return nullptr;
  return c->prec == SEM_F32 ? static_cast<const void*>(c->m->minv32) : static_cast<const void*>(c->m->minv64);
}

void cg_note(sem_cg c, cudaStream_t s) {
  for (cudaStream_t u : c->used)
    if (u == s) return;
  c->used.push_back(s);
}

// Waits for the streams the solver was used on, then releases its memory on its own stream.
void cg_free(sem_cg c) {
  for (cudaStream_t u : c->used) cudaStreamSynchronize(u);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  cudaStream_t h = c->cap;
  for (void* q : {c->r, c->z, c->p, c->w})
    if (q) cudaFreeAsync(q, h);
  dfree(c->ax_part, h);
  dfree(c->gs_part, h);
  dfree(c->upd_part, h);
  dfree(c->init_part, h);
  dfree(c->st, h);
  dfree(c->bar, h);
  if (h) {
    cudaStreamSynchronize(h);
    cudaStreamDestroy(h);
  }
  delete c;
}

sem_status cg_alloc(sem_mesh m, sem_prec prec, sem_ax_variant v, int precond, double rtol, int max_iter, int use_graph,
                    sem_cg* out) {
  *out = nullptr;
  if (v == SEM_AX_STORED && !has_factors(m, prec))
    return fail(SEM_ERR_ARG, "stored factors of this precision were not requested at mesh creation");
  if (prec == SEM_F64X && v == SEM_AX_OTF_SCALE)
    return fail(SEM_ERR_UNSUPPORTED, "double-float FP64 arithmetic runs the stored and on-the-fly variants");
  if (v == SEM_AX_OTF_SCALE && !has_scales(m))
    return fail(SEM_ERR_ARG, "per-point scales were not requested at mesh creation (SEM_MESH_OTF_SCALE)");
  if (cg_layout(prec)) SEM_TRY(ensure_cg_layout(m, m->home));
  sem_cg c = new sem_cg_s();
  c->m = m;
  c->prec = prec;
  c->variant = v;
  c->precond = precond;
  c->rtol = rtol;
  c->max_iter = max_iter;
  c->use_graph = use_graph;
  const size_t es = prec == SEM_F32 ? sizeof(float) : sizeof(double);
  sem_status st = SEM_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaStreamCreate");
  }
  for (void** q : {&c->r, &c->z, &c->p, &c->w}) {
    e = cudaMallocAsync(q, m->n * es, c->cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *q = nullptr;
      st = fail(SEM_ERR_OOM, "cudaMallocAsync of CG work vectors failed");
      break;
    }
  }
  if (st == SEM_OK) st = dmalloc(&c->ax_part, kRedMax, nullptr, c->cap);
  if (st == SEM_OK) st = dmalloc(&c->gs_part, kRedMax, nullptr, c->cap);
  if (st == SEM_OK) st = dmalloc(&c->upd_part, 2 * kRedMax, nullptr, c->cap);
  if (st == SEM_OK) st = dmalloc(&c->init_part, 3 * kRedMax, nullptr, c->cap);
  if (st == SEM_OK) st = dmalloc(&c->st, 1, nullptr, c->cap);
  if (st == SEM_OK) st = dmalloc(&c->bar, 2, nullptr, c->cap);
  if (st == SEM_OK && (e = cudaStreamSynchronize(c->cap)) != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
  if (st != SEM_OK) {
    cg_free(c);
    return st;
  }
  *out = c;
  return SEM_OK;
}

// The solver handle kept on the mesh for sem_cg_solve: reused while the variant,
// preconditioner and graph setting are unchanged (rtol and max_iter are per solve).
sem_status cached_cg(sem_mesh m, sem_prec prec, sem_ax_variant v, int precond, int use_graph, double rtol,
                     int max_iter, sem_cg* out) {
  sem_cg& slot = prec == SEM_F32 ? m->solve_cg32 : m->solve_cg64;
  if (slot && (slot->prec != prec || slot->variant != v || slot->precond != precond || slot->use_graph != use_graph)) {
    cg_free(slot);
    slot = nullptr;
  }
  if (!slot) SEM_TRY(cg_alloc(m, prec, v, precond, rtol, max_iter, use_graph, &slot));
  slot->rtol = rtol;
  slot->max_iter = max_iter;
  *out = slot;
  return SEM_OK;
}

// Host-side state reset + r0 = b - A x0, z0, rho0 (device).
sem_status cg_start(sem_cg c, const void* b, void* x, bool x0_is_zero, cudaStream_t s) {
  sem_mesh m = c->m;
  if (c->precond) SEM_TRY(ensure_jacobi(m, s));
  CgScalars init{};
  init.rtol2 = c->rtol * c->rtol;
  init.max_iter = c->max_iter;
  cg_note(c, s);
  note_stream(m, s);
  c->st_host = init;
  SEM_CUDA_TRY(cudaMemcpyAsync(c->st, &c->st_host, sizeof(CgScalars), cudaMemcpyHostToDevice, s));
  c->b = b;
  c->x = x;
  const void* ax0 = nullptr;
  if (!x0_is_zero) {
    AxLaunch a{};
    a.u = x;
    a.w = c->w;
    // The residual of a (re)start is formed with the native FP64 operator also when the
    // iterations run in double-float arithmetic: a restart after the recursive residual has
    // converged then replaces it by the true residual b - A x, and the solve corrects the
    // double-float operator's own rounding (about 1e-14 of |A| |x|) instead of stalling on it.
    sem_prec rp = c->prec;
    sem_ax_variant rv = c->variant;
    if (rp == SEM_F64X) {
      rp = SEM_F64;
      if (rv == SEM_AX_STORED && !m->G64) rv = SEM_AX_OTF;
    }
    SEM_TRY(launch_ax_any(m, rp, rv, false, a, s));
    SEM_TRY(launch_dssum(data_prec(c->prec), m->gs, c->w, 1, s));
    ax0 = c->w;
  }
  SEM_TRY(launch_cg_init(data_prec(c->prec), m->n, b, ax0, c->r, c->z, c->p, minv_of(c), m->mult, m->ctab, c->st, c->init_part,
                         s));
  // the host struct is reused by query: make sure the copy above has been consumed
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  return SEM_OK;
}

// The operator's CG-mode launch: p = z + beta p (fused_cg: also the deferred x += alpha p,
// with z = M^-1 r formed from r), w = A_L p, partials of <p, w>.
AxLaunch cg_ax_launch(sem_cg c) {
  AxLaunch a{};
  a.w = c->w;
  a.z = c->z;
  a.p = c->p;
  if (fused_cg(c->prec)) {
    a.r = c->r;
    a.minv = minv_of(c);
    a.x = c->x;
  }
  a.st = c->st;
  a.partials = c->ax_part;
  a.grid_out = &c->ax_blocks;
  return a;
}

// QQ^T and the mask on w (FP64 data: in the CG layout); every CG-mode operator formed the whole
// <p, w>.
sem_status cg_enqueue_gs(sem_cg c, cudaStream_t s) {
  return launch_dssum_cg(data_prec(c->prec), cg_layout(c->prec) ? c->m->gs_cg : c->m->gs, c->w,
                         whole_dot(c->prec) ? nullptr : c->p, c->st, c->ax_part, c->ax_blocks, c->gs_part, s);
}

sem_status cg_enqueue_update(sem_cg c, cudaStream_t s) {
  return launch_cg_update(data_prec(c->prec), fused_cg(c->prec), c->m->n, c->x, c->p, c->r, c->w, c->z, minv_of(c),
                          c->m->mult, c->m->ctab, c->st, c->upd_part, c->m->cg_map, s);
}

// fused_cg: the x update of the last iteration run (a no-op if there is none)
sem_status cg_enqueue_flush(sem_cg c, cudaStream_t s) {
  if (!fused_cg(c->prec)) return SEM_OK;
  return launch_cg_flush(data_prec(c->prec), c->m->n, c->x, c->p, c->st, s);
}

// One iteration of Algorithm 1: [p = z + beta p; w = A_L p; <p,w> partials] -> [QQ^T, mask,
// (boundary <p,w>), alpha] -> [r, z (and x) updates, <r,z,c>, <r,r,c>, beta, stop test].
sem_status cg_enqueue_iteration(sem_cg c, cudaStream_t s) {
  SEM_TRY(launch_ax_any(c->m, c->prec, c->variant, true, cg_ax_launch(c), s));
  SEM_TRY(cg_enqueue_gs(c, s));
  return cg_enqueue_update(c, s);
}

int host_sm_count() {
  static const int n = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
  }();
  return n;
}

// use_graph = 2: FP64 CG with stored factors on a mesh with fewer elements than the device has
// SMs runs in the persistent kernel (k_cg_small.cu), a run of iterations per launch.
bool small_path(sem_cg c) {
  if (c->use_graph != 2 || c->prec != SEM_F64 || !c->m->G64 || c->m->E >= host_sm_count()) return false;
  sem_ax_variant v;
  int shape;
  resolve_variant(c->m, SEM_F64, c->variant, &v, &shape);
  return v == SEM_AX_STORED;
}

sem_status cg_iterate_small(sem_cg c, int k, cudaStream_t s) {
  sem_mesh m = c->m;
  SEM_CUDA_TRY(cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), s));
  SmallCgLaunch a;
  a.E = m->E;
  a.n = m->n;
  a.G = m->G64;
  a.x = static_cast<double*>(c->x);
  a.p = static_cast<double*>(c->p);
  a.r = static_cast<double*>(c->r);
  a.z = static_cast<double*>(c->z);
  a.w = static_cast<double*>(c->w);
  a.minv = static_cast<const double*>(minv_of(c));
  a.mult = m->mult;
  a.ctab = m->ctab;
  a.gs = m->gs;
  a.st = c->st;
  a.part = c->init_part;
  a.bar = c->bar;
  a.err = m->dev_err;
  a.iters = k;
  a.max_blocks = host_sm_count();
  return launch_cg_small(m->N, a, s);
}

sem_status cg_iterate(sem_cg c, int k, cudaStream_t s) {
  if (k <= 0) return SEM_OK;
  cg_note(c, s);
  note_stream(c->m, s);
  if (small_path(c)) return cg_iterate_small(c, k, s);
  if (!c->use_graph) {
    for (int q = 0; q < k; ++q) SEM_TRY(cg_enqueue_iteration(c, s));
    return cg_enqueue_flush(c, s);
  }
  if (!c->exec || c->exec_k != k || c->exec_x != c->x) {
    if (c->exec) {
      cudaGraphExecDestroy(c->exec);
      c->exec = nullptr;
    }
    SEM_CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    t_capturing = true;
    sem_status st = SEM_OK;
    for (int q = 0; q < k && st == SEM_OK; ++q) st = cg_enqueue_iteration(c, c->cap);
    if (st == SEM_OK) st = cg_enqueue_flush(c, c->cap);
    t_capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (st != SEM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    c->exec_k = k;
    c->exec_x = c->x;
  }
  SEM_CUDA_TRY(cudaGraphLaunch(c->exec, s));
  count_launch(3 * k + (fused_cg(c->prec) ? 1 : 0));
  return SEM_OK;
}

sem_status cg_query(sem_cg c, sem_cg_result* res, cudaStream_t s) {
  cg_note(c, s);
  SEM_CUDA_TRY(cudaMemcpyAsync(&c->st_host, c->st, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  const CgScalars& h = c->st_host;
  if (res) {
    res->iters = h.iter;
    res->outer_iters = 0;
    res->rel_res = h.bb > 0 ? std::sqrt(h.rr / h.bb) : std::sqrt(h.rr);
    res->status = h.done ? h.status : SEM_ERR_BUSY;
  }
  return SEM_OK;
}

sem_status check_opts(const sem_cg_opts* o) {
  if (!o) return fail(SEM_ERR_ARG, "opts is null");
  if (!(o->rtol >= 0) || o->max_iter < 0 || o->check_every < 1 || (o->precond != 0 && o->precond != 1) ||
      (o->variant < SEM_AX_STORED || o->variant > SEM_AX_OTF_SCALE) ||
      (o->inner_variant < SEM_AX_STORED || o->inner_variant > SEM_AX_OTF_SCALE) ||
      (o->f64_arith != 0 && o->f64_arith != 1) || o->use_graph < 0 || o->use_graph > 2)
    return fail(SEM_ERR_ARG, "invalid CG options");
  if (o->mixed < 0 || o->mixed > 2) return fail(SEM_ERR_ARG, "mixed must be 0, 1 or 2");
  if (o->mixed && (!(o->inner_rtol > 0 && o->inner_rtol < 1) || o->max_outer < 1))
    return fail(SEM_ERR_ARG, "mixed precision needs 0 < inner_rtol < 1 and max_outer >= 1");
  return SEM_OK;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Runs a started solver until its device flag says done; polls every check_every iterations.
sem_status cg_run(sem_cg c, int check_every, sem_cg_result* r, cudaStream_t s) {
  for (;;) {
    SEM_TRY(cg_iterate(c, check_every, s));
    SEM_TRY(cg_query(c, r, s));
    if (r->status != SEM_ERR_BUSY) return SEM_OK;
  }
}

// FP32 inner CG (on-the-fly or stored factors) inside FP64 iterative refinement:
//   r = b - A x (FP64 operator, FP64 dots); stop if ||r||_c / ||b||_c <= rtol;
//   solve A d = r in FP32 to inner_rtol; x += d.
// mixed = 1 restarts the FP32 CG from d = 0 after each refinement step. mixed = 2 keeps it
// going (reliable updates, i.e. residual replacement as in van der Vorst and Ye, 2000): each
// time its residual has dropped by inner_rtol, x += d (FP64), d = 0, the true residual
// b - A x is formed in FP64 and replaces the FP32 residual, and the FP32 CG continues along
// its current search direction, so the Krylov process is not restarted.
sem_status solve_mixed(sem_mesh m, const double* b, double* x, const sem_cg_opts* o, sem_cg_result* res,
                       cudaStream_t s) {
  sem_cg inner = nullptr;
  SEM_TRY(cached_cg(m, SEM_F32, static_cast<sem_ax_variant>(o->inner_variant), o->precond, o->use_graph,
                    o->inner_rtol, o->max_iter, &inner));
  if (!m->ir_part) {
    sem_status a = SEM_OK;
    note_stream(m, s);
    if ((a = dmalloc(&m->ir_w64, m->n, nullptr, s)) != SEM_OK || (a = dmalloc(&m->ir_r64, m->n, nullptr, s)) != SEM_OK ||
        (a = dmalloc(&m->ir_r32, m->n, nullptr, s)) != SEM_OK || (a = dmalloc(&m->ir_d32, m->n, nullptr, s)) != SEM_OK ||
        (a = dmalloc(&m->ir_st, 1, nullptr, s)) != SEM_OK ||
        (a = dmalloc(&m->ir_part, 2 * kRedMax, nullptr, s)) != SEM_OK) {
      dfree(m->ir_w64, s);
      dfree(m->ir_r64, s);
      dfree(m->ir_r32, s);
      dfree(m->ir_d32, s);
      dfree(m->ir_st, s);
      dfree(m->ir_part, s);
      return a;
    }
  }
  double* w64 = m->ir_w64;
  double* r64 = m->ir_r64;
  float* r32 = m->ir_r32;
  float* d32 = m->ir_d32;
  CgScalars* ost = m->ir_st;
  double* opart = m->ir_part;
  sem_status st = SEM_OK;
  CgScalars oinit{};
  oinit.rtol2 = o->rtol * o->rtol;
  int total_inner = 0, outer = 0;
  res->status = SEM_ERR_NOT_CONVERGED;
  for (;;) {
    // FP64 residual
    AxLaunch a{};
    a.u = x;
    a.w = w64;
    if ((st = launch_ax_any(m, o->f64_arith ? SEM_F64X : SEM_F64, static_cast<sem_ax_variant>(o->variant), false, a,
                            s)) != SEM_OK)
      break;
    if ((st = launch_dssum(SEM_F64, m->gs, w64, 1, s)) != SEM_OK) break;
    cudaError_t e = cudaMemcpyAsync(ost, &oinit, sizeof(CgScalars), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaMemcpyAsync"); break; }
    if ((st = launch_ir_residual(m->n, b, w64, r64, r32, m->mult, m->ctab, ost, opart, s)) != SEM_OK) break;
    CgScalars oh{};
    e = cudaMemcpyAsync(&oh, ost, sizeof(CgScalars), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = cuda_fail(e, "reading the refinement residual"); break; }
    res->rel_res = oh.bb > 0 ? std::sqrt(oh.rr / oh.bb) : std::sqrt(oh.rr);
    if (oh.done) {
      res->status = oh.status;
      break;
    }
    if (outer >= o->max_outer || total_inner >= o->max_iter) {
      res->status = SEM_ERR_NOT_CONVERGED;
      break;
    }
    const bool replace = o->mixed == 2 && outer > 0;
    if (replace) {  // reliable update: the true residual replaces the FP32 one, p is kept
      if ((st = launch_cg_replace(m->n, r32, static_cast<float*>(inner->r), static_cast<float*>(inner->z),
                                  static_cast<const float*>(minv_of(inner)), m->mult, m->ctab, inner->st,
                                  inner->init_part, s)) != SEM_OK)
        break;
    } else {  // FP32 inner solve from d = 0
      inner->max_iter = o->max_iter - total_inner;
      if ((e = cudaMemsetAsync(d32, 0, m->n * sizeof(float), s)) != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
      if ((st = cg_start(inner, r32, d32, true, s)) != SEM_OK) break;
    }
    const int before = o->mixed == 2 ? total_inner : 0;  // mixed = 2: the count continues across replacements
    sem_cg_result ir{};
    if ((st = cg_run(inner, o->check_every, &ir, s)) != SEM_OK) break;
    const int steps = ir.iters - before;
    total_inner = o->mixed == 2 ? ir.iters : total_inner + ir.iters;
    ++outer;
    if (ir.status == SEM_ERR_BREAKDOWN && steps == 0) {
      res->status = SEM_ERR_BREAKDOWN;
      break;
    }
    if ((st = launch_ir_correct(m->n, x, d32, s)) != SEM_OK) break;
    if (o->mixed == 2 && (e = cudaMemsetAsync(d32, 0, m->n * sizeof(float), s)) != cudaSuccess) {
      st = cuda_fail(e, "memset");
      break;
    }
  }
  res->iters = total_inner;
  res->outer_iters = outer;
  return st;
}

}  // namespace
}  // namespace sem

extern "C" sem_status sem_cg_default_opts(sem_cg_opts* o) {
  return guarded([&]() -> sem_status {
    if (!o) return fail(SEM_ERR_ARG, "opts is null");
    o->rtol = 1e-10;
    o->max_iter = 100000;
    o->precond = 1;
    o->variant = SEM_AX_STORED;
    o->mixed = 0;
    o->inner_variant = SEM_AX_OTF;
    o->inner_rtol = 1e-5;
    o->max_outer = 50;
    o->check_every = 50;
    o->use_graph = 1;
    o->f64_arith = 0;
    return SEM_OK;
  });
}

extern "C" sem_status sem_cg_create(sem_mesh m, const sem_cg_opts* o, sem_cg* out) {
  return guarded([&]() -> sem_status {
    if (!out) return fail(SEM_ERR_ARG, "out is null");
    *out = nullptr;
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_opts(o));
    if (o->mixed) return fail(SEM_ERR_ARG, "the stateful CG handle runs FP64 CG only (mixed=0)");
    return cg_alloc(m, o->f64_arith ? SEM_F64X : SEM_F64, static_cast<sem_ax_variant>(o->variant), o->precond, o->rtol,
                    o->max_iter, o->use_graph, out);
  });
}

extern "C" sem_status sem_cg_start(sem_cg c, const double* b, double* x, void* stream) {
  return guarded([&]() -> sem_status {
    if (!c) return fail(SEM_ERR_ARG, "null CG handle");
    SEM_TRY(check_mesh(c->m));
    SEM_TRY(check_ptr(b, "b_dev"));
    SEM_TRY(check_ptr(x, "x_dev"));
    return cg_start(c, b, x, false, static_cast<cudaStream_t>(stream));
  });
}

extern "C" sem_status sem_cg_iterate(sem_cg c, int k, void* stream) {
  return guarded([&]() -> sem_status {
    if (!c) return fail(SEM_ERR_ARG, "null CG handle");
    if (!c->x) return fail(SEM_ERR_ARG, "sem_cg_start has not been called");
    return cg_iterate(c, k, static_cast<cudaStream_t>(stream));
  });
}

extern "C" sem_status sem_cg_iterate_timed(sem_cg c, int k, double* total_ms, double* kernel_ms, void* stream) {
  return guarded([&]() -> sem_status {
    if (!c || !total_ms || !kernel_ms) return fail(SEM_ERR_ARG, "null argument");
    if (!c->x) return fail(SEM_ERR_ARG, "sem_cg_start has not been called");
    if (k < 1) return fail(SEM_ERR_ARG, "k must be >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    sem_mesh m = c->m;
    cg_note(c, s);
    note_stream(m, s);
    std::vector<cudaEvent_t> ev(3 * static_cast<size_t>(k) + 1, nullptr);
    auto destroy = [&] {
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    };
    for (auto& e : ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) {
        destroy();
        return cuda_fail(r, "cudaEventCreate");
      }
    }
    sem_status st = SEM_OK;
    cudaEventRecord(ev[0], s);
    for (int q = 0; q < k && st == SEM_OK; ++q) {
      st = launch_ax_any(m, c->prec, c->variant, true, cg_ax_launch(c), s);
      cudaEventRecord(ev[3 * q + 1], s);
      if (st == SEM_OK) st = cg_enqueue_gs(c, s);
      cudaEventRecord(ev[3 * q + 2], s);
      if (st == SEM_OK) st = cg_enqueue_update(c, s);
      if (st == SEM_OK && q == k - 1) st = cg_enqueue_flush(c, s);  // inside the timed region
      cudaEventRecord(ev[3 * q + 3], s);
    }
    cudaError_t r = cudaStreamSynchronize(s);
    if (st == SEM_OK && r != cudaSuccess) st = cuda_fail(r, "cudaStreamSynchronize");
    if (st == SEM_OK) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[0], ev[3 * k]);
      *total_ms = t;
      for (int j = 0; j < 3; ++j) kernel_ms[j] = 0.0;
      for (int q = 0; q < k; ++q)
        for (int j = 0; j < 3; ++j) {
          cudaEventElapsedTime(&t, ev[3 * q + j], ev[3 * q + j + 1]);
          kernel_ms[j] += t / k;
        }
    }
    destroy();
    return st;
  });
}

extern "C" sem_status sem_cg_query(sem_cg c, sem_cg_result* res, void* stream) {
  return guarded([&]() -> sem_status {
    if (!c || !res) return fail(SEM_ERR_ARG, "null argument");
    res->time_ms = 0;
    return cg_query(c, res, static_cast<cudaStream_t>(stream));
  });
}

extern "C" sem_status sem_cg_destroy(sem_cg c) {
  return guarded([&]() -> sem_status {
    if (!c) return SEM_OK;
    cg_free(c);  // waits only for the streams this solver was used on
    return SEM_OK;
  });
}

extern "C" sem_status sem_cg_solve(sem_mesh m, const double* b, double* x, const sem_cg_opts* o, sem_cg_result* res,
                                   void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_opts(o));
    SEM_TRY(check_ptr(b, "b_dev"));
    SEM_TRY(check_ptr(x, "x_dev"));
    if (!res) return fail(SEM_ERR_ARG, "result is null");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double t0 = now_ms();
    *res = sem_cg_result{};
    sem_status st;
    if (o->mixed) {
      st = solve_mixed(m, b, x, o, res, s);
    } else {
      // Algorithm 1; when the recursively updated residual meets rtol, CG restarts from x:
      // the restart recomputes r = b - A x, so the solve ends only when the true residual meets
      // rtol (long runs let the recursive residual drift away from b - A x).
      sem_cg c = nullptr;
      SEM_TRY(cached_cg(m, o->f64_arith ? SEM_F64X : SEM_F64, static_cast<sem_ax_variant>(o->variant), o->precond,
                        o->use_graph, o->rtol, o->max_iter, &c));
      st = cg_start(c, b, x, false, s);
      int total = 0;
      for (int restart = 0; st == SEM_OK; ++restart) {
        sem_cg_result r{};
        st = cg_query(c, &r, s);
        if (st != SEM_OK) break;
        if (r.status != SEM_ERR_BUSY) {  // decided at the (re)start: true residual small, or limit
          res->status = r.status;
          res->rel_res = r.rel_res;
          break;
        }
        st = cg_run(c, o->check_every, &r, s);
        if (st != SEM_OK) break;
        total += r.iters;
        res->status = r.status;
        res->rel_res = r.rel_res;
        if (r.status != SEM_OK || restart >= 20) break;
        c->max_iter = o->max_iter - total;
        st = cg_start(c, b, x, false, s);
      }
      res->iters = total;
      cudaStreamSynchronize(s);
    }
    res->time_ms = now_ms() - t0;
    if (st != SEM_OK) {
      res->status = st;
      return st;
    }
    if (res->status == SEM_ERR_NOT_CONVERGED) return fail(SEM_ERR_NOT_CONVERGED, "CG reached max_iter");
    if (res->status == SEM_ERR_BREAKDOWN) return fail(SEM_ERR_BREAKDOWN, "CG breakdown (<p,Ap,c> <= 0 or non-finite)");
    return static_cast<sem_status>(res->status);
  });
}

extern "C" uint64_t sem_launch_count(void) { return g_launches.load(); }

extern "C" const char* sem_last_error(void) { return t_last_error.c_str(); }

extern "C" const char* sem_status_string(sem_status s) {
  switch (s) {
    case SEM_OK: return "SEM_OK";
    case SEM_ERR_ARG: return "SEM_ERR_ARG";
    case SEM_ERR_MESH: return "SEM_ERR_MESH";
    case SEM_ERR_OOM: return "SEM_ERR_OOM";
    case SEM_ERR_CUDA: return "SEM_ERR_CUDA";
    case SEM_ERR_NOT_CONVERGED: return "SEM_ERR_NOT_CONVERGED";
    case SEM_ERR_BREAKDOWN: return "SEM_ERR_BREAKDOWN";
    case SEM_ERR_TIMEOUT: return "SEM_ERR_TIMEOUT";
    case SEM_ERR_BUSY: return "SEM_ERR_BUSY";
    case SEM_ERR_UNSUPPORTED: return "SEM_ERR_UNSUPPORTED";
  }
  return "unknown";
}

// ---------------------------------------------------------------------------
// autotuning
// ---------------------------------------------------------------------------

namespace {
std::string device_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p{};
  cudaGetDeviceProperties(&p, dev);
  std::string n = p.name;
  for (char& ch : n)
    if (ch == ' ') ch = '_';
  return n;
}
}  // namespace

extern "C" sem_status sem_autotune(sem_mesh m, sem_prec prec, int reps, sem_tune_report* rep, void* stream) {
  return guarded([&]() -> sem_status {
    SEM_TRY(check_mesh(m));
    SEM_TRY(check_prec(prec));
    if (!rep || reps < 1) return fail(SEM_ERR_ARG, "need a report and reps >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    note_stream(m, s);
    const size_t es = prec == SEM_F32 ? sizeof(float) : sizeof(double);
    void *u = nullptr, *w = nullptr;
    SEM_CUDA_TRY(cudaMallocAsync(&u, m->n * es, s));
    cudaError_t e = cudaMallocAsync(&w, m->n * es, s);
    if (e != cudaSuccess) {
      cudaFreeAsync(u, s);
      return cuda_fail(e, "cudaMallocAsync");
    }
    cudaMemsetAsync(u, 0, m->n * es, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    *rep = sem_tune_report{};
    rep->N = m->N;
    rep->prec = prec;
    sem_status st = SEM_OK;
    for (const sem_ax_variant v : {SEM_AX_STORED, SEM_AX_OTF, SEM_AX_OTF_SCALE}) {
      if (st != SEM_OK) break;
      if (v == SEM_AX_STORED && !has_factors(m, prec)) continue;
      if (v == SEM_AX_OTF_SCALE && prec == SEM_F64X) continue;
      if (v == SEM_AX_OTF_SCALE && !has_scales(m)) continue;
      for (int shape : {0, 1, kTensorShape}) {
        if (st != SEM_OK) break;
        if (shape == 1 && (prec == SEM_F64X || v == SEM_AX_OTF_SCALE ||
                           ax_elements_per_block(m->N, 1) == ax_elements_per_block(m->N, 0)))
          continue;
        if (shape == kTensorShape && !ax_tensor_available(m->N, prec, v)) continue;
        AxLaunch a{};
        a.u = u;
        a.w = w;
        a.E = m->E;
        a.err = m->dev_err;
        a.shape = shape == 0 ? 2 : shape;  // the tuner times each shape as it is
        a.coef = prec == SEM_F32 ? static_cast<const void*>(m->coef32) : static_cast<const void*>(m->coef64);
        a.G = stored_factors(m, prec, &a.g_pairs);
        a.scale = prec == SEM_F32 ? static_cast<const void*>(m->scale32) : static_cast<const void*>(m->scale64);
        auto launch = [&] {
          if (prec == SEM_F64X) return launch_ax_f64x(m->N, v, false, a, s);
          if (shape == kTensorShape) return launch_ax_tc(m->N, false, a, s);
          return prec == SEM_F64 ? launch_ax_f64(m->N, v, false, a, s) : launch_ax_f32(m->N, v, false, a, s);
        };
        for (int q = 0; q < 2 && st == SEM_OK; ++q) st = launch();
        cudaEventRecord(e0, s);
        for (int q = 0; q < reps && st == SEM_OK; ++q) st = launch();
        cudaEventRecord(e1, s);
        if (st != SEM_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        sem_tune_entry& c = rep->candidates[rep->n_candidates++];
        c.variant = v;
        c.shape = shape;
        c.elements_per_block = prec == SEM_F64X ? 0 : shape == kTensorShape ? 1 : ax_elements_per_block(m->N, shape);
        c.ms = ms / reps;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(u, s);
    cudaFreeAsync(w, s);
    cudaStreamSynchronize(s);
    if (st != SEM_OK) return st;
    if (rep->n_candidates == 0) return fail(SEM_ERR_ARG, "no candidate implementation for this precision");
    TuneSlot t;
    t.valid = true;
    double best = 1e300;
    double best_v[3] = {1e300, 1e300, 1e300};
    for (int q = 0; q < rep->n_candidates; ++q) {
      const sem_tune_entry& c = rep->candidates[q];
      const int slot = vslot(static_cast<sem_ax_variant>(c.variant));
      if (c.ms < best_v[slot]) {
        best_v[slot] = c.ms;
        t.shape[slot] = c.shape;
        t.ms[slot] = c.ms;
      }
      if (c.ms < best) {
        best = c.ms;
        rep->best = q;
        t.best = static_cast<sem_ax_variant>(c.variant);
      }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[prec][m->N] = t;
    return SEM_OK;
  });
}

extern "C" sem_status sem_autotune_set(int N, sem_prec prec, sem_ax_variant variant, int shape) {
  return guarded([&]() -> sem_status {
    if (N < 1 || N > SEM_MAX_N) return fail(SEM_ERR_UNSUPPORTED, "polynomial order out of range");
    SEM_TRY(check_prec(prec));
    if (variant != SEM_AX_STORED && variant != SEM_AX_OTF && variant != SEM_AX_OTF_SCALE)
      return fail(SEM_ERR_ARG, "variant must be SEM_AX_STORED, SEM_AX_OTF or SEM_AX_OTF_SCALE");
    const bool ok = shape == 0 || (shape == 1 && variant != SEM_AX_OTF_SCALE && prec != SEM_F64X) ||
                    (shape == kTensorShape && ax_tensor_available(N, prec, variant));
    if (!ok) return fail(SEM_ERR_ARG, "block shape choice not available for this order, precision and variant");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    TuneSlot& t = g_tune[prec][N];
    if (!t.valid) {
      t = TuneSlot{};
      t.valid = true;
      t.best = variant;
    }
    t.shape[vslot(variant)] = shape;
    return SEM_OK;
  });
}

extern "C" sem_status sem_autotune_clear(void) {
  return guarded([&]() -> sem_status {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto& row : g_tune)
      for (TuneSlot& t : row) t = TuneSlot{};
    return SEM_OK;
  });
}

extern "C" sem_status sem_autotune_save(const char* path) {
  return guarded([&]() -> sem_status {
    if (!path) return fail(SEM_ERR_ARG, "null path");
    std::ofstream f(path);
    if (!f) return fail(SEM_ERR_ARG, std::string("cannot write ") + path);
    f << "sem-autotune 2 " << device_name() << "\n";
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (int p = 0; p < 3; ++p)
      for (int N = 1; N <= SEM_MAX_N; ++N) {
        const TuneSlot& t = g_tune[p][N];
        if (t.valid)
          f << p << " " << N << " " << t.best << " " << t.shape[0] << " " << t.shape[1] << " " << t.shape[2] << " "
            << t.ms[0] << " " << t.ms[1] << " " << t.ms[2] << "\n";
      }
    return f ? SEM_OK : fail(SEM_ERR_ARG, "write failed");
  });
}

extern "C" sem_status sem_autotune_load(const char* path) {
  return guarded([&]() -> sem_status {
    if (!path) return fail(SEM_ERR_ARG, "null path");
    std::ifstream f(path);
    if (!f) return fail(SEM_ERR_ARG, std::string("cannot read ") + path);
    std::string magic, gpu;
    int version = 0;
    f >> magic >> version >> gpu;
    if (magic != "sem-autotune" || version != 2) return fail(SEM_ERR_ARG, "not a tuning table");
    if (gpu != device_name()) return fail(SEM_ERR_ARG, "tuning table was made on " + gpu);
    int p, N, best, s0, s1, s2;
    double m0, m1, m2;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    while (f >> p >> N >> best >> s0 >> s1 >> s2 >> m0 >> m1 >> m2) {
      if (p < 0 || p > 2 || N < 1 || N > SEM_MAX_N || !(best == 0 || best == 1 || best == 3) || s0 < 0 || s0 > 1 ||
          !(s1 == 0 || s1 == 1 || (s1 == kTensorShape && ax_tensor_available(N, static_cast<sem_prec>(p), SEM_AX_OTF))) ||
          s2 != 0)
        return fail(SEM_ERR_ARG, "corrupt tuning table");
      TuneSlot& t = g_tune[p][N];
      t.valid = true;
      t.best = static_cast<sem_ax_variant>(best);
      t.shape[0] = s0;
      t.shape[1] = s1;
      t.shape[2] = s2;
      t.ms[0] = m0;
      t.ms[1] = m1;
      t.ms[2] = m2;
    }
    return SEM_OK;
  });
}
