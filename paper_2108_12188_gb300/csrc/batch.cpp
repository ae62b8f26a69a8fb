// Batched mixed-precision solves: many small Poisson solves advance together. Each job is the
// refinement of sem_cg_solve's mixed modes (FP64 residual b - A x, x += d, FP64 dots; FP32
// Jacobi-CG with on-the-fly factors for the correction d, restarted for mixed = 1, continued
// with residual replacement for mixed = 2), but the FP32 iterations of all jobs whose inner
// solve is running are shared launches over a device-side table (k_batch.cu): per iteration,
// one operator launch per polynomial order present, one gather-scatter and one update launch,
// replayed as a CUDA graph that depends only on the orders present, so jobs join and leave
// between rounds without a new capture. The refinement steps (a few per job) are launched per
// job between rounds.
//
// Per-job arithmetic is fixed by the job alone (see k_batch.cu), so a job's x is bit-identical
// whatever else is in the batch and however the rounds fall. The paper motivates lower
// precision (Section 8) and gives the solver (Algorithm 1); the batching is this library's.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "sem_internal.h"

namespace sem {

namespace {

enum : int { kResidual = 0, kDecide = 1, kInner = 2, kDone = 3 };

template <typename T>
sem_status balloc(T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA, "cudaMallocAsync of batch work space failed");
  }
  return SEM_OK;
}

template <typename T>
void bfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

}  // namespace

BatchEngine::~BatchEngine() {
  for (Graph& g : graphs_) cudaGraphExecDestroy(g.exec);
  if (s_) {
    if (tab_d_) cudaFreeAsync(tab_d_, s_);
    if (stat_d_) cudaFreeAsync(stat_d_, s_);
    cudaStreamSynchronize(s_);
  }
  if (tab_h_) cudaFreeHost(tab_h_);
  if (stat_h_) cudaFreeHost(stat_h_);
  if (ost_pin_) cudaFreeHost(ost_pin_);
  if (cap_) cudaStreamDestroy(cap_);
}

sem_status BatchEngine::init(cudaStream_t s) {
  s_ = s;
  SEM_CUDA_TRY(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
  SEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&tab_d_), sizeof(BatchTable), s_));
  SEM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&stat_d_), kBatchMax * sizeof(CgScalars), s_));
  SEM_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&tab_h_), sizeof(BatchTable)));
  SEM_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&stat_h_), kBatchMax * sizeof(CgScalars)));
  SEM_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&ost_pin_), kBatchMax * sizeof(CgScalars)));
  std::memset(static_cast<void*>(tab_h_), 0, sizeof(BatchTable));
  return SEM_OK;
}

sem_status BatchEngine::add(BatchJob* j) {
  const sem_cg_opts& o = j->o;
  if (!(o.rtol >= 0) || o.max_iter < 0 || o.max_outer < 1 || !(o.inner_rtol > 0 && o.inner_rtol < 1) ||
      (o.precond != 0 && o.precond != 1) || o.variant < SEM_AX_STORED || o.variant > SEM_AX_OTF_SCALE ||
      (o.f64_arith != 0 && o.f64_arith != 1))
    return fail(SEM_ERR_ARG, "invalid CG options");
  if (o.mixed != 1 && o.mixed != 2) return fail(SEM_ERR_ARG, "batched solves run mixed precision (mixed = 1 or 2)");
  if (o.inner_variant != SEM_AX_OTF && o.inner_variant != SEM_AX_AUTO)
    return fail(SEM_ERR_ARG, "batched solves run the on-the-fly FP32 inner operator");
  if (jobs_.size() >= static_cast<size_t>(kBatchMax)) return fail(SEM_ERR_BUSY, "the batch is full");
  sem_mesh m = j->m;
  note_stream(m, s_);
  if (o.precond) SEM_TRY_STATUS(ensure_jacobi(m, s_));
  const int64_t n = m->n;
  const int epb = batch_ax_elements_per_group(m->Np);
  if (epb <= 0) return fail(SEM_ERR_UNSUPPORTED, "polynomial order not compiled in");
  j->groups = (m->E + epb - 1) / epb;
  j->chunks = (n + kBatchChunk - 1) / kBatchChunk;
  sem_status st = SEM_OK;
  auto step = [&](sem_status r) {
    if (st == SEM_OK) st = r;
  };
  for (float** v : {&j->r32, &j->z32, &j->p32, &j->w32, &j->d32, &j->rr32}) step(balloc(v, n, s_));
  step(balloc(&j->w64, n, s_));
  step(balloc(&j->r64, n, s_));
  step(balloc(&j->ist, 1, s_));
  step(balloc(&j->ost, 1, s_));
  step(balloc(&j->ax_part, j->groups, s_));
  step(balloc(&j->up_part, 2 * j->chunks, s_));
  step(balloc(&j->init_part, 3 * kRedMax, s_));
  step(balloc(&j->opart, 2 * kRedMax, s_));
  if (st != SEM_OK) {
    release(j);
    return st;
  }
  j->state = kResidual;
  j->total_inner = j->outer = j->before = 0;
  j->res = sem_cg_result{};
  j->res.status = SEM_ERR_BUSY;
  jobs_.push_back(j);
  return SEM_OK;
}

void BatchEngine::release(BatchJob* j) {
  for (float** v : {&j->r32, &j->z32, &j->p32, &j->w32, &j->d32, &j->rr32}) bfree(*v, s_);
  bfree(j->w64, s_);
  bfree(j->r64, s_);
  bfree(j->ist, s_);
  bfree(j->ost, s_);
  bfree(j->ax_part, s_);
  bfree(j->up_part, s_);
  bfree(j->init_part, s_);
  bfree(j->opart, s_);
}

// FP64 residual of the refinement: r = b - A x (FP64 operator, QQ^T, mask), its FP32 copy,
// <r, r, c> and <b, b, c>; the scalars are copied to the job's host mirror.
sem_status BatchEngine::residual(BatchJob* j, CgScalars* host_out) {
  sem_mesh m = j->m;
  AxLaunch a{};
  a.u = j->x;
  a.w = j->w64;
  SEM_TRY_STATUS(launch_ax_any(m, j->o.f64_arith ? SEM_F64X : SEM_F64, static_cast<sem_ax_variant>(j->o.variant), false,
                               a, s_));
  SEM_TRY_STATUS(launch_dssum(SEM_F64, m->gs, j->w64, 1, s_));
  CgScalars init{};
  init.rtol2 = j->o.rtol * j->o.rtol;
  SEM_CUDA_TRY(cudaMemcpyAsync(j->ost, &init, sizeof(CgScalars), cudaMemcpyHostToDevice, s_));
  SEM_TRY_STATUS(launch_ir_residual(m->n, j->b, j->w64, j->r64, j->rr32, m->mult, m->ctab, j->ost, j->opart, s_));
  SEM_CUDA_TRY(cudaMemcpyAsync(host_out, j->ost, sizeof(CgScalars), cudaMemcpyDeviceToHost, s_));
  return SEM_OK;
}

// The refinement decision after a residual: converged, out of steps, or the next inner solve
// (restarted from d = 0, or continued with the true residual replacing the FP32 one).
sem_status BatchEngine::start_inner(BatchJob* j) {
  sem_mesh m = j->m;
  const sem_cg_opts& o = j->o;
  const CgScalars& h = j->ost_h;
  j->res.rel_res = h.bb > 0 ? std::sqrt(h.rr / h.bb) : std::sqrt(h.rr);
  if (h.done) {
    finish(j, h.status);
    return SEM_OK;
  }
  if (j->outer >= o.max_outer || j->total_inner >= o.max_iter) {
    finish(j, SEM_ERR_NOT_CONVERGED);
    return SEM_OK;
  }
  const float* minv = o.precond ? m->minv32 : nullptr;
  if (o.mixed == 2 && j->outer > 0) {
    SEM_TRY_STATUS(launch_cg_replace(m->n, j->rr32, j->r32, j->z32, minv, m->mult, m->ctab, j->ist, j->init_part, s_));
  } else {
    CgScalars init{};
    init.rtol2 = o.inner_rtol * o.inner_rtol;
    init.max_iter = o.max_iter - j->total_inner;
    SEM_CUDA_TRY(cudaMemcpyAsync(j->ist, &init, sizeof(CgScalars), cudaMemcpyHostToDevice, s_));
    SEM_CUDA_TRY(cudaMemsetAsync(j->d32, 0, m->n * sizeof(float), s_));
    SEM_TRY_STATUS(launch_cg_init(SEM_F32, m->n, j->rr32, nullptr, j->r32, j->z32, j->p32, minv, m->mult, m->ctab,
                                  j->ist, j->init_part, s_));
  }
  j->before = o.mixed == 2 ? j->total_inner : 0;
  j->state = kInner;
  dirty_ = true;
  return SEM_OK;
}

void BatchEngine::finish(BatchJob* j, int status) {
  j->state = kDone;
  j->res.iters = j->total_inner;
  j->res.outer_iters = j->outer;
  j->res.status = status;
  jobs_.erase(std::find(jobs_.begin(), jobs_.end(), j));
  done_.push_back(j);
  dirty_ = true;
}

// The table of the jobs whose inner solve runs, grouped by order (entries of one order are
// contiguous, in job order), with every job's work-item ranges.
sem_status BatchEngine::upload_table() {
  table_.clear();
  for (int np = 2; np <= kMaxNp; ++np)
    for (BatchJob* j : jobs_)
      if (j->state == kInner && j->m->Np == np) table_.push_back(j);
  BatchTable& t = *tab_h_;
  t.count = static_cast<int>(table_.size());
  for (BatchOrder& o : t.order) o = BatchOrder{0, 0, 0};
  int64_t gs = 0, up = 0;
  for (int q = 0; q < t.count; ++q) {
    BatchJob* j = table_[q];
    sem_mesh m = j->m;
    BatchSolve& d = t.s[q];
    d = BatchSolve{};
    d.NP = m->Np;
    d.E = m->E;
    d.n = m->n;
    d.coef = m->coef32;
    d.x = j->d32;
    d.p = j->p32;
    d.r = j->r32;
    d.w = j->w32;
    d.minv = j->o.precond ? m->minv32 : nullptr;
    d.mult = m->mult;
    d.ctab = m->ctab;
    d.gs = m->gs;
    d.st = j->ist;
    d.ax_part = j->ax_part;
    d.up_part = j->up_part;
    d.err = m->dev_err;
    BatchOrder& o = t.order[m->Np];
    if (o.s_hi == 0 && o.items == 0) o.s_lo = q;
    o.s_hi = q + 1;
    d.ax_beg = o.items;
    d.ax_cnt = j->groups;
    o.items += j->groups;
    // gather-scatter items: classes of width 2, 4, 8, 1, then the CSR lists
    const int64_t cls[5] = {m->gs.n[1], m->gs.n[2], m->gs.n[3], m->gs.n[0], m->gs.nx};
    d.gs_at[0] = 0;
    for (int c = 0; c < 5; ++c) d.gs_at[c + 1] = d.gs_at[c] + (cls[c] + kBatchGsSeg - 1) / kBatchGsSeg;
    if (d.gs_at[5] == 0) d.gs_at[5] = 1;  // one empty item, so that alpha is still formed
    d.gs_beg = gs;
    gs += d.gs_at[5];
    d.up_beg = up;
    d.up_cnt = j->chunks;
    up += j->chunks;
  }
  t.gs_items = gs;
  t.up_items = up;
  const size_t bytes = offsetof(BatchTable, s) + sizeof(BatchSolve) * static_cast<size_t>(t.count > 0 ? t.count : 1);
  SEM_CUDA_TRY(cudaMemcpyAsync(tab_d_, tab_h_, bytes, cudaMemcpyHostToDevice, s_));
  dirty_ = false;
  return SEM_OK;
}

// `iters` batched iterations and the flush, as a CUDA graph keyed by the orders present.
sem_status BatchEngine::iterate(int iters) {
  unsigned orders = 0;
  for (BatchJob* j : table_) orders |= 1u << j->m->Np;
  int norders = 0;
  for (int np = 2; np <= kMaxNp; ++np) norders += (orders >> np) & 1u;
  Graph* g = nullptr;
  for (Graph& c : graphs_)
    if (c.orders == orders && c.iters == iters) g = &c;
  if (!g) {
    SEM_CUDA_TRY(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    sem_status st = SEM_OK;
    for (int it = 0; it < iters && st == SEM_OK; ++it) {
      for (int np = 2; np <= kMaxNp && st == SEM_OK; ++np)
        if ((orders >> np) & 1u) st = launch_batch_ax(np, tab_d_, cap_);
      if (st == SEM_OK) st = launch_batch_gs(tab_d_, cap_);
      if (st == SEM_OK) st = launch_batch_update(tab_d_, cap_);
    }
    if (st == SEM_OK) st = launch_batch_flush(tab_d_, cap_);
    set_capturing(false);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap_, &graph);
    if (st != SEM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture (batch)");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
    graphs_.push_back(Graph{orders, iters, exec});
    g = &graphs_.back();
  }
  SEM_CUDA_TRY(cudaGraphLaunch(g->exec, s_));
  count_launch(iters * (norders + 2) + 1);
  return SEM_OK;
}

sem_status BatchEngine::round(int iters) {
  if (iters < 1) return fail(SEM_ERR_ARG, "a round needs at least one iteration");
  // residuals that are due (new jobs, and jobs whose inner solve ended last round)
  std::vector<BatchJob*> due;
  for (BatchJob* j : jobs_)
    if (j->state == kResidual) {
      SEM_TRY_STATUS(residual(j, &ost_pin_[due.size()]));
      j->state = kDecide;
      due.push_back(j);
    }
  if (!due.empty()) {
    SEM_CUDA_TRY(cudaStreamSynchronize(s_));
    for (size_t q = 0; q < due.size(); ++q) due[q]->ost_h = ost_pin_[q];
  }
  const std::vector<BatchJob*> snapshot = jobs_;
  for (BatchJob* j : snapshot)
    if (j->state == kDecide) SEM_TRY_STATUS(start_inner(j));
  bool inner = false;
  for (BatchJob* j : jobs_) inner = inner || j->state == kInner;
  if (!inner) return SEM_OK;
  if (dirty_) SEM_TRY_STATUS(upload_table());
  SEM_TRY_STATUS(iterate(iters));
  SEM_TRY_STATUS(launch_batch_status(tab_d_, static_cast<int>(table_.size()), stat_d_, s_));
  SEM_CUDA_TRY(cudaMemcpyAsync(stat_h_, stat_d_, table_.size() * sizeof(CgScalars), cudaMemcpyDeviceToHost, s_));
  SEM_CUDA_TRY(cudaStreamSynchronize(s_));
  for (size_t q = 0; q < table_.size(); ++q) {
    BatchJob* j = table_[q];
    const CgScalars& h = stat_h_[q];
    if (!h.done) continue;
    const int steps = h.iter - j->before;
    j->total_inner = j->o.mixed == 2 ? h.iter : j->total_inner + h.iter;
    ++j->outer;
    if (h.status == SEM_ERR_BREAKDOWN && steps == 0) {
      finish(j, SEM_ERR_BREAKDOWN);
      continue;
    }
    sem_mesh m = j->m;
    SEM_TRY_STATUS(launch_ir_correct(m->n, j->x, j->d32, s_));
    if (j->o.mixed == 2) SEM_CUDA_TRY(cudaMemsetAsync(j->d32, 0, m->n * sizeof(float), s_));
    j->state = kResidual;
    dirty_ = true;
  }
  return SEM_OK;
}

std::vector<BatchJob*> BatchEngine::take_done() {
  std::vector<BatchJob*> d;
  d.swap(done_);
  return d;
}

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_cg_solve_batch(int count, const sem_mesh* meshes, const double* const* b_dev,
                                         double* const* x_dev, const sem_cg_opts* opts, sem_cg_result* results,
                                         void* stream) {
  return guarded([&]() -> sem_status {
    if (count < 1 || count > kBatchMax) return fail(SEM_ERR_ARG, "count must be in [1, 256]");
    if (!meshes || !b_dev || !x_dev || !opts || !results) return fail(SEM_ERR_ARG, "null argument");
    if (opts->check_every < 1) return fail(SEM_ERR_ARG, "invalid CG options");
    for (int q = 0; q < count; ++q) {
      SEM_TRY_STATUS(check_mesh(meshes[q]));
      SEM_TRY_STATUS(check_ptr(b_dev[q], "b_dev[i]"));
      SEM_TRY_STATUS(check_ptr(x_dev[q], "x_dev[i]"));
      for (int r = 0; r < q; ++r)
        if (x_dev[r] == x_dev[q]) return fail(SEM_ERR_ARG, "two problems share one x_dev");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchEngine eng;
    SEM_TRY_STATUS(eng.init(s));
    std::vector<BatchJob> jobs(static_cast<size_t>(count));
    sem_status st = SEM_OK;
    int added = 0;
    for (int q = 0; q < count && st == SEM_OK; ++q) {
      jobs[q].m = meshes[q];
      jobs[q].b = b_dev[q];
      jobs[q].x = x_dev[q];
      jobs[q].o = *opts;
      st = eng.add(&jobs[q]);
      if (st == SEM_OK) ++added;
    }
    int finished = 0;
    while (st == SEM_OK && finished < added) {
      st = eng.round(opts->check_every);
      finished += static_cast<int>(eng.take_done().size());
    }
    for (int q = 0; q < added; ++q) eng.release(&jobs[q]);
    cudaStreamSynchronize(s);
    if (st != SEM_OK) return st;
    sem_status first = SEM_OK;
    for (int q = 0; q < count; ++q) {
      results[q] = jobs[q].res;
      if (first == SEM_OK && results[q].status != SEM_OK) first = static_cast<sem_status>(results[q].status);
    }
    if (first != SEM_OK) return fail(first, "at least one batched solve did not converge");
    return SEM_OK;
  });
}
