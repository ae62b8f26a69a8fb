// Solve server: admits Poisson solve requests of different sizes and orders by a device
// memory budget and runs the admitted ones concurrently; requests that arrive while others
// run are admitted as memory frees up (continuous batching).
//
// A request carries its mesh (vertices, connectivity, order), the wave numbers of the
// manufactured right-hand side and CG options (or a mesh the caller built and a host
// right-hand side). A worker thread builds the mesh and the right-hand side on its own
// non-blocking stream. Small mixed-precision requests are then handed to the batch engine
// thread, which advances all of them together in shared launches over a device-side table of
// the admitted solves (BatchEngine, batch.cpp), taking new ones in and retiring finished ones
// between rounds; the worker is free again at once. Other requests are solved by their worker
// with sem_cg_solve on the worker's stream. Every device allocation is stream-ordered, so one
// request's set-up or teardown never waits for the others' kernels. A request that fails (bad
// mesh, non-convergence) fails alone.
//
// Results do not depend on what else runs: a request takes the same path alone and in a mix
// (the path depends on its size and options only), and on both paths its launches and
// reductions are fixed by the request itself (fixed grids or per-request work items,
// fixed-order sums, no atomics on values).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "sem_internal.h"

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  sem_mesh mesh = nullptr;       // prebuilt mesh (sem_server_submit_mesh), owned by the server
  std::vector<double> b_host;    // its right-hand side
  int N = 0;
  std::vector<double> vxyz;
  std::vector<int64_t> ev;
  std::vector<uint8_t> dflags;
  int sine[3] = {1, 1, 1};
  sem_cg_opts opts{};
  size_t est_bytes = 0;
  int64_t n_local = 0;
  bool batched = false;
  // results
  bool done = false;
  sem_server_result res{};
  std::vector<double> x;
  double t_submit = 0, t_start = 0;
  ~Request() {  // a prebuilt mesh still queued when the server is destroyed
    if (mesh) sem_mesh_destroy(mesh);
  }
};

}  // namespace

struct sem_server_s {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int max_slots = 1, active = 0;
  int64_t batch_max_points = 0;
  int batch_max_solves = 1, batch_round_iters = 1;
  bool size_priorities = true;
  int prio_least = 0, prio_greatest = 0;  // the device's CUDA stream priority range
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<std::thread> workers;
  // batch engine thread and the solves handed to it (set up, not yet in the engine)
  std::thread engine;
  bool engine_stop = false;
  std::deque<sem::BatchJob*> batch_in;
  std::condition_variable batch_cv;
  int64_t batch_rounds = 0, batch_solve_rounds = 0;  // rounds run; sum over rounds of the solves in them
  int batch_max = 0;                                 // most solves in one round
};

namespace {

// Device bytes of one request: mesh (coefficients, segments, multiplicities), stored factors
// if the options need them, Jacobi inverse (FP64 + FP32), right-hand side and solution,
// FP64 CG or refinement work vectors plus the FP32 inner CG.
size_t estimate_bytes(int64_t E, int N, const sem_cg_opts& o) {
  const size_t Np = static_cast<size_t>(N) + 1;
  const size_t n = static_cast<size_t>(E) * Np * Np * Np;
  size_t b = static_cast<size_t>(E) * 24 * 12 + 5 * n + 12 * n + 16 * n;
  const bool f64_stored = o.variant == SEM_AX_STORED;
  const bool f32_stored = o.mixed && o.inner_variant == SEM_AX_STORED;
  if (f64_stored) b += 48 * n;
  if (f32_stored) b += 24 * n;
  b += o.mixed ? (16 * n + 8 * n + 16 * n) : 32 * n;
  return b + (8u << 20);
}

// CUDA stream priority of a request's work: with size priorities, the fewer local points the
// higher the priority (the batch engine's stream takes the highest), one level per factor 2
// above 2^21 points, so that the GPU's block scheduler serves short solves first; otherwise
// the default priority.
int request_priority(const sem_server_s* srv, int64_t n_local) {
  if (!srv->size_priorities || srv->prio_greatest == srv->prio_least) return srv->prio_least;
  int level = 0;
  for (int64_t t = int64_t(1) << 21; t < n_local && level < 62; t <<= 1) ++level;
  const int p = srv->prio_greatest + 1 + level;  // greatest is the numerically lowest
  return p < srv->prio_least ? p : srv->prio_least;
}

void run_request(sem_server srv, Request* r) {
  cudaSetDevice(srv->device);
  sem_server_result& res = r->res;
  cudaStream_t s = nullptr;
  sem_mesh mesh = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  sem_status st = SEM_OK;
  const double t0 = now_ms();
  if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, request_priority(srv, r->n_local)) != cudaSuccess)
    st = SEM_ERR_CUDA;
  unsigned flags = 0;
  if (r->opts.variant == SEM_AX_STORED) flags |= r->opts.f64_arith ? SEM_MESH_F64X_STORED : SEM_MESH_F64_STORED;
  if (r->opts.mixed && r->opts.inner_variant == SEM_AX_STORED) flags |= SEM_MESH_F32_STORED;
  if (r->mesh) {  // prebuilt mesh: now the server's
    mesh = r->mesh;
    r->mesh = nullptr;
  } else if (st == SEM_OK) {
    st = sem_mesh_create(r->N, static_cast<int64_t>(r->vxyz.size() / 3), r->vxyz.data(),
                         static_cast<int64_t>(r->ev.size() / 8), r->ev.data(),
                         r->dflags.empty() ? nullptr : r->dflags.data(), flags, s, &mesh);
  }
  sem_mesh_info_t info{};
  if (st == SEM_OK) st = sem_mesh_get_info(mesh, &info);
  if (st == SEM_OK && cudaMallocAsync(reinterpret_cast<void**>(&b), info.n_local * sizeof(double), s) != cudaSuccess)
    st = SEM_ERR_OOM;
  if (st == SEM_OK && cudaMallocAsync(reinterpret_cast<void**>(&x), info.n_local * sizeof(double), s) != cudaSuccess)
    st = SEM_ERR_OOM;
  if (st == SEM_OK) {
    if (r->b_host.empty()) {
      st = sem_rhs_sine(mesh, r->sine[0], r->sine[1], r->sine[2], SEM_F64, b, s);
    } else if (cudaMemcpyAsync(b, r->b_host.data(), r->b_host.size() * sizeof(double), cudaMemcpyHostToDevice, s) !=
               cudaSuccess) {
      st = SEM_ERR_CUDA;
    }
  }
  if (st == SEM_OK && cudaMemsetAsync(x, 0, info.n_local * sizeof(double), s) != cudaSuccess) st = SEM_ERR_CUDA;
  const double t1 = now_ms();
  if (st == SEM_OK && r->batched) {  // hand the solve over to the batch engine
    if (cudaStreamSynchronize(s) != cudaSuccess) st = SEM_ERR_CUDA;
    if (st == SEM_OK) {
      mesh->used.clear();  // this stream has drained and goes away; the engine records its own
      auto* j = new sem::BatchJob();
      j->m = mesh;
      j->b = b;
      j->x = x;
      j->o = r->opts;
      j->user = r;
      cudaStreamDestroy(s);
      std::lock_guard<std::mutex> lock(srv->mu);
      res.setup_ms = t1 - t0;
      srv->batch_in.push_back(j);
      srv->batch_cv.notify_all();
      return;
    }
  }
  sem_cg_result cg{};
  if (st == SEM_OK) {
    sem_status solve = sem_cg_solve(mesh, b, x, &r->opts, &cg, s);
    if (solve == SEM_ERR_ARG || solve == SEM_ERR_OOM || solve == SEM_ERR_CUDA || solve == SEM_ERR_UNSUPPORTED)
      st = solve;
  }
  std::vector<double> xh;
  if (st == SEM_OK) {
    try {
      xh.resize(static_cast<size_t>(info.n_local));
    } catch (const std::bad_alloc&) {
      st = SEM_ERR_OOM;
    }
  }
  if (st == SEM_OK && (cudaMemcpyAsync(xh.data(), x, xh.size() * sizeof(double), cudaMemcpyDeviceToHost, s) !=
                           cudaSuccess ||
                       cudaStreamSynchronize(s) != cudaSuccess))
    st = SEM_ERR_CUDA;
  const double t2 = now_ms();
  if (b) cudaFreeAsync(b, s);
  if (x) cudaFreeAsync(x, s);
  if (mesh) sem_mesh_destroy(mesh);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  std::lock_guard<std::mutex> lock(srv->mu);
  res.status = st == SEM_OK ? cg.status : st;
  res.n_local = info.n_local;
  res.cg = cg;
  res.queue_ms = r->t_start - r->t_submit;
  res.setup_ms = t1 - t0;
  res.solve_ms = t2 - t1;
  res.latency_ms = t2 - r->t_submit;
  res.batched = 0;
  r->x = std::move(xh);
  r->done = true;
  srv->in_use -= r->est_bytes;
  --srv->active;
  srv->cv.notify_all();
}

// A batched solve has ended (or failed to start): x to host memory, release, report.
void finish_batched(sem_server srv, sem::BatchEngine* eng, sem::BatchJob* j, cudaStream_t es, sem_status st,
                    double t_handover) {
  Request* r = static_cast<Request*>(j->user);
  const int64_t n = j->m->n;
  std::vector<double> xh;
  if (st == SEM_OK) {
    try {
      xh.resize(static_cast<size_t>(n));
    } catch (const std::bad_alloc&) {
      st = SEM_ERR_OOM;
    }
  }
  if (st == SEM_OK && (cudaMemcpyAsync(xh.data(), j->x, xh.size() * sizeof(double), cudaMemcpyDeviceToHost, es) !=
                           cudaSuccess ||
                       cudaStreamSynchronize(es) != cudaSuccess))
    st = SEM_ERR_CUDA;
  const double t2 = now_ms();
  if (eng) eng->release(j);
  cudaFreeAsync(const_cast<double*>(j->b), es);
  cudaFreeAsync(j->x, es);
  sem_mesh_destroy(j->m);
  const sem_cg_result cg = j->res;
  delete j;
  std::lock_guard<std::mutex> lock(srv->mu);
  sem_server_result& res = r->res;
  res.status = st == SEM_OK ? cg.status : st;
  res.n_local = n;
  res.cg = cg;
  res.cg.time_ms = t2 - t_handover;
  res.queue_ms = r->t_start - r->t_submit;
  res.solve_ms = t2 - t_handover;
  res.latency_ms = t2 - r->t_submit;
  res.batched = 1;
  r->x = std::move(xh);
  r->done = true;
  srv->in_use -= r->est_bytes;
  --srv->active;
  srv->cv.notify_all();
}

// The batch engine thread: takes handed-over solves into the engine (up to batch_max_solves at
// once), runs rounds while any solve is running, and reports the solves that end.
void engine_loop(sem_server srv) {
  cudaSetDevice(srv->device);
  cudaStream_t es = nullptr;
  sem::BatchEngine eng;
  const int prio = srv->size_priorities ? srv->prio_greatest : srv->prio_least;
  sem_status est =
      cudaStreamCreateWithPriority(&es, cudaStreamNonBlocking, prio) == cudaSuccess ? SEM_OK : SEM_ERR_CUDA;
  if (est == SEM_OK) est = eng.init(es);
  std::unordered_map<sem::BatchJob*, double> handed;  // hand-over times
  for (;;) {
    std::vector<sem::BatchJob*> incoming;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      if (eng.running() == 0)
        srv->batch_cv.wait(lock, [&] { return srv->engine_stop || !srv->batch_in.empty(); });
      if (srv->engine_stop && srv->batch_in.empty() && eng.running() == 0) break;
      while (!srv->batch_in.empty() &&
             eng.running() + incoming.size() < static_cast<size_t>(srv->batch_max_solves)) {
        incoming.push_back(srv->batch_in.front());
        srv->batch_in.pop_front();
      }
    }
    const double t = now_ms();
    for (sem::BatchJob* j : incoming) {
      handed[j] = t;
      sem_status a = est == SEM_OK ? eng.add(j) : est;
      if (a != SEM_OK) {
        finish_batched(srv, nullptr, j, es, a, t);
        handed.erase(j);
      }
    }
    if (eng.running() > 0) {
      const int in_round = static_cast<int>(eng.running());
      sem_status rs = eng.round(srv->batch_round_iters);
      if (rs != SEM_OK) est = rs;  // the device state of the batch is unknown: fail what runs
      std::lock_guard<std::mutex> lock(srv->mu);
      ++srv->batch_rounds;
      srv->batch_solve_rounds += in_round;
      if (in_round > srv->batch_max) srv->batch_max = in_round;
    }
    for (sem::BatchJob* j : eng.take_done()) {
      finish_batched(srv, &eng, j, es, SEM_OK, handed[j]);
      handed.erase(j);
    }
    if (est != SEM_OK && eng.running() > 0) {
      for (auto& hj : handed) finish_batched(srv, &eng, hj.first, es, est, hj.second);
      handed.clear();
      break;  // later hand-overs fail at once (below)
    }
  }
  // only after a failure of the engine: report what is still handed over
  for (;;) {
    sem::BatchJob* j = nullptr;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->batch_cv.wait(lock, [&] { return srv->engine_stop || !srv->batch_in.empty(); });
      if (srv->batch_in.empty()) break;
      j = srv->batch_in.front();
      srv->batch_in.pop_front();
    }
    finish_batched(srv, nullptr, j, es, est == SEM_OK ? SEM_ERR_CUDA : est, now_ms());
  }
  if (es) {
    cudaStreamSynchronize(es);
  }
}

void worker_loop(sem_server srv) {
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->cv.wait(lock, [&] {
        if (srv->stop) return true;
        if (srv->queue.empty()) return false;
        const Request* h = srv->queue.front();
        // first in, first admitted: the head waits until its memory fits (or the device is idle)
        return srv->active == 0 || srv->in_use + h->est_bytes <= srv->budget;
      });
      if (srv->stop) return;
      r = srv->queue.front();
      srv->queue.pop_front();
      srv->in_use += r->est_bytes;
      ++srv->active;
      r->t_start = now_ms();
    }
    run_request(srv, r);
  }
}

}  // namespace

using sem::fail;
using sem::guarded;

namespace {

// The path a request takes: the batch for small mixed-precision solves with the on-the-fly
// inner operator (the batched kernels' operator), its worker's own stream otherwise.
bool routes_to_batch(const sem_server_s* srv, int64_t n_local, const sem_cg_opts& o) {
  return srv->batch_max_points > 0 && n_local <= srv->batch_max_points && (o.mixed == 1 || o.mixed == 2) &&
         (o.inner_variant == SEM_AX_OTF || o.inner_variant == SEM_AX_AUTO);
}

}  // namespace

extern "C" sem_status sem_server_default_config(size_t hbm_budget_bytes, int max_slots, sem_server_config* cfg) {
  return guarded([&]() -> sem_status {
    if (!cfg) return fail(SEM_ERR_ARG, "cfg is null");
    cfg->hbm_budget_bytes = hbm_budget_bytes;
    cfg->max_slots = max_slots;
    cfg->batch_max_points = 2097152;
    cfg->batch_max_solves = 64;
    cfg->batch_round_iters = 20;
    cfg->size_priorities = 1;
    return SEM_OK;
  });
}

extern "C" sem_status sem_server_create_config(const sem_server_config* cfg, sem_server* out) {
  return guarded([&]() -> sem_status {
    if (!out || !cfg) return fail(SEM_ERR_ARG, "null argument");
    *out = nullptr;
    if (cfg->max_slots < 1 || cfg->max_slots > 256 || cfg->hbm_budget_bytes == 0)
      return fail(SEM_ERR_ARG, "need 1 <= max_slots <= 256 and a non-zero budget");
    if (cfg->batch_max_points < 0 || cfg->batch_max_solves < 1 || cfg->batch_max_solves > sem::kBatchMax ||
        cfg->batch_round_iters < 1)
      return fail(SEM_ERR_ARG, "need batch_max_points >= 0, 1 <= batch_max_solves <= 256, batch_round_iters >= 1");
    auto srv = std::make_unique<sem_server_s>();
    SEM_CUDA_TRY(cudaGetDevice(&srv->device));
    // keep freed stream-ordered memory in the pool between requests (this process only)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, srv->device) == cudaSuccess) {
      uint64_t keep = cfg->hbm_budget_bytes;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    srv->budget = cfg->hbm_budget_bytes;
    srv->max_slots = cfg->max_slots;
    srv->batch_max_points = cfg->batch_max_points;
    srv->batch_max_solves = cfg->batch_max_solves;
    srv->batch_round_iters = cfg->batch_round_iters;
    srv->size_priorities = cfg->size_priorities != 0;
    SEM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&srv->prio_least, &srv->prio_greatest));
    try {
      srv->engine = std::thread(engine_loop, srv.get());
      for (int q = 0; q < cfg->max_slots; ++q) srv->workers.emplace_back(worker_loop, srv.get());
    } catch (const std::exception&) {  // a thread could not be started: stop the ones that did
      {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        srv->engine_stop = true;
      }
      srv->cv.notify_all();
      srv->batch_cv.notify_all();
      for (auto& t : srv->workers) t.join();
      if (srv->engine.joinable()) srv->engine.join();
      return fail(SEM_ERR_OOM, "could not start the server's threads");
    }
    *out = srv.release();
    return SEM_OK;
  });
}

extern "C" sem_status sem_server_create(size_t hbm_budget_bytes, int max_slots, sem_server* out) {
  sem_server_config cfg{};
  const sem_status st = sem_server_default_config(hbm_budget_bytes, max_slots, &cfg);
  if (st != SEM_OK) return st;
  return sem_server_create_config(&cfg, out);
}

extern "C" sem_status sem_server_submit(sem_server srv, const sem_request* req, uint64_t* ticket) {
  return guarded([&]() -> sem_status {
    if (!srv || !req || !ticket) return fail(SEM_ERR_ARG, "null argument");
    if (req->N < 1 || req->N > SEM_MAX_N) return fail(SEM_ERR_UNSUPPORTED, "polynomial order out of range");
    if (req->E < 1 || req->num_vertices < 8 || !req->vert_xyz_host || !req->elem_verts_host)
      return fail(SEM_ERR_ARG, "request needs vertices and elements");
    auto r = std::make_unique<Request>();
    r->N = req->N;
    r->vxyz.assign(req->vert_xyz_host, req->vert_xyz_host + 3 * req->num_vertices);
    r->ev.assign(req->elem_verts_host, req->elem_verts_host + 8 * req->E);
    if (req->dirichlet_vertex_flags_host)
      r->dflags.assign(req->dirichlet_vertex_flags_host, req->dirichlet_vertex_flags_host + req->num_vertices);
    std::memcpy(r->sine, req->sine, sizeof(r->sine));
    r->opts = req->opts;
    const size_t Np = static_cast<size_t>(req->N) + 1;
    r->n_local = static_cast<int64_t>(static_cast<size_t>(req->E) * Np * Np * Np);
    r->est_bytes = estimate_bytes(req->E, req->N, req->opts);
    r->batched = routes_to_batch(srv, r->n_local, r->opts);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (r->est_bytes > srv->budget) return fail(SEM_ERR_ARG, "request needs more device memory than the budget");
    r->t_submit = now_ms();
    r->ticket = srv->next_ticket++;
    r->res.status = SEM_ERR_BUSY;
    *ticket = r->ticket;
    srv->queue.push_back(r.get());
    srv->all.emplace(r->ticket, std::move(r));
    srv->cv.notify_all();
    return SEM_OK;
  });
}

extern "C" sem_status sem_server_submit_mesh(sem_server srv, sem_mesh mesh, const double* b_host,
                                              const sem_cg_opts* opts, uint64_t* ticket) {
  return guarded([&]() -> sem_status {
    if (!srv || !mesh || !b_host || !opts || !ticket) return fail(SEM_ERR_ARG, "null argument");
    if (mesh->device != srv->device) return fail(SEM_ERR_ARG, "the mesh lives on another device than the server");
    auto r = std::make_unique<Request>();
    r->N = mesh->N;
    r->n_local = mesh->n;
    r->b_host.assign(b_host, b_host + mesh->n);
    r->opts = *opts;
    // the mesh's memory plus the solver's: b, x, the Jacobi inverse (FP64 and FP32) and the
    // CG work vectors (FP64 CG, or FP32 CG with the FP64 refinement buffers)
    const size_t n = static_cast<size_t>(mesh->n);
    r->est_bytes = mesh->device_bytes + 16 * n + 12 * n + (opts->mixed ? 40 * n : 32 * n) + (8u << 20);
    r->batched = routes_to_batch(srv, r->n_local, r->opts);
    if (r->est_bytes > srv->budget) return fail(SEM_ERR_ARG, "request needs more device memory than the budget");
    // the caller's streams may go away: finish their work on the mesh now (without the lock)
    for (cudaStream_t u : mesh->used) SEM_CUDA_TRY(cudaStreamSynchronize(u));
    mesh->used.clear();
    std::lock_guard<std::mutex> lock(srv->mu);
    r->mesh = mesh;
    r->t_submit = now_ms();
    r->ticket = srv->next_ticket++;
    r->res.status = SEM_ERR_BUSY;
    *ticket = r->ticket;
    srv->queue.push_back(r.get());
    srv->all.emplace(r->ticket, std::move(r));
    srv->cv.notify_all();
    return SEM_OK;
  });
}

extern "C" sem_status sem_server_poll(sem_server srv, uint64_t ticket, double* x_host, int64_t x_capacity,
                                      sem_server_result* res) {
  return guarded([&]() -> sem_status {
    if (!srv || !res) return fail(SEM_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) return fail(SEM_ERR_ARG, "unknown or released ticket");
    Request* r = it->second.get();
    if (!r->done) {
      *res = sem_server_result{};
      res->status = SEM_ERR_BUSY;
      res->n_local = r->n_local;
      return SEM_ERR_BUSY;
    }
    *res = r->res;
    if (x_host) {
      if (x_capacity < static_cast<int64_t>(r->x.size())) return fail(SEM_ERR_ARG, "x_host is too small");
      std::memcpy(x_host, r->x.data(), r->x.size() * sizeof(double));
      srv->all.erase(it);  // released once its solution has been taken
    }
    return SEM_OK;
  });
}

extern "C" sem_status sem_server_stats(sem_server srv, int* queued, int* active, size_t* bytes_in_use) {
  return guarded([&]() -> sem_status {
    if (!srv) return fail(SEM_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lock(srv->mu);
    if (queued) *queued = static_cast<int>(srv->queue.size());
    if (active) *active = srv->active;
    if (bytes_in_use) *bytes_in_use = srv->in_use;
    return SEM_OK;
  });
}

extern "C" sem_status sem_server_batch_stats(sem_server srv, int64_t* rounds, int* max_batch, double* mean_batch) {
  return guarded([&]() -> sem_status {
    if (!srv) return fail(SEM_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lock(srv->mu);
    if (rounds) *rounds = srv->batch_rounds;
    if (max_batch) *max_batch = srv->batch_max;
    if (mean_batch)
      *mean_batch = srv->batch_rounds ? static_cast<double>(srv->batch_solve_rounds) / srv->batch_rounds : 0.0;
    return SEM_OK;
  });
}

extern "C" sem_status sem_server_destroy(sem_server srv) {
  return guarded([&]() -> sem_status {
    if (!srv) return SEM_OK;
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->stop = true;
      srv->queue.clear();  // queued requests are dropped; running ones finish
    }
    srv->cv.notify_all();
    for (auto& t : srv->workers) t.join();
    {  // every hand-over has happened: the engine finishes the batch and stops
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->engine_stop = true;
    }
    srv->batch_cv.notify_all();
    if (srv->engine.joinable()) srv->engine.join();
    delete srv;
    return SEM_OK;
  });
}
