// Persistent FP64 Jacobi-PCG for small meshes (Algorithm 1 with z = M^-1 r): one cooperative
// launch runs a whole run of iterations, each iteration being three phases separated by grid
// barriers instead of three kernel launches:
//   A  local operator, stored factors: p = z + beta p, w = A_L p (Eq. 4), block partials of <p, w>
//   B  gather-scatter QQ^T and the Dirichlet mask on w (Eq. 5, Algorithm 1 step 7)
//   C  x += alpha p, r -= alpha w, z = M^-1 r, block partials of <r, z, c> and <r, r, c>
// After each barrier every block adds the partials in the same fixed order, so all blocks hold
// the same alpha, beta and stopping decision without a host round trip (deterministic).
//
// A small mesh has fewer elements than the GPU has SMs, so phase A gives each element a block of
// its own and splits every line contraction between two threads (each forms half of the line's
// outputs from the whole even/odd-split line): 2 (N+1)^2 threads per element, four warps at
// N = 7, so that one element keeps all four FP64 units of its SM busy.
//
// Grid barriers are bounded waits: a block that waits longer than kBarrierLimitNs (1 s of the
// global timer) gives up, records SEM_ERR_TIMEOUT and leaves; the others then give up at their
// next barrier, so the kernel always ends. A cooperative launch guarantees that all blocks are
// resident, so in normal operation no wait comes near the limit.
#include <type_traits>

#include "k_ax.cuh"
#include "k_gs.cuh"

namespace sem {
namespace {

constexpr uint64_t kBarrierLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier over the launch's blocks: bar[0] counts arrivals, bar[1] is the generation the
// last arrival advances. `gen` is the generation this block saw before the barrier. Returns false
// (in every thread of the block) if the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen, bool* sok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    const unsigned g = gen;
    __threadfence();
    const unsigned a = atomicAdd(&bar[0], 1u);
    if (a == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], g + 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (ld_acquire(&bar[1]) == g) {
        if (global_ns() - t0 > kBarrierLimitNs) {
          ok = false;
          break;
        }
      }
    }
    __threadfence();
    gen = g + 1u;
    *sok = ok;
  }
  __syncthreads();
  return *sok;
}

// Fixed-order sum of part[0 .. count) in every thread of the block (the same value in every block).
__device__ __forceinline__ double all_sum(const double* part, int count, double* sh, double* bcast) {
  const double s = sum_partials(part, count, 1, 0, sh);
  if (threadIdx.x == 0) *bcast = s;
  __syncthreads();
  const double v = *bcast;
  __syncthreads();
  return v;
}

// Half of the outputs of a line contraction out = M in (even/odd split, see EoMat): half h of the
// pairs (i, N - i), i < H, and for odd NP the middle output in half 1. store(index, value).
template <int NP, typename F>
__device__ __forceinline__ void eo_half(const EoMat<NP, double>& M, const double (&in)[NP], int h, F&& store) {
  constexpr int H = NP / 2, N = NP - 1, H2 = (H + 1) / 2;
  double e[H > 0 ? H : 1], o[H > 0 ? H : 1];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    e[l] = in[l] + in[N - l];
    o[l] = in[l] - in[N - l];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    if ((i < H2) != (h == 0)) continue;
    double a = M.E[i][0] * e[0], b = M.O[i][0] * o[0];
#pragma unroll
    for (int l = 1; l < H; ++l) {
      a += M.E[i][l] * e[l];
      b += M.O[i][l] * o[l];
    }
    if constexpr (NP % 2 == 1) a += M.E[i][H] * in[H];
    store(i, a + b);
    store(N - i, b - a);
  }
  if constexpr (NP % 2 == 1) {
    if (h == 1 || H == 0) {
      double c = 0.0;
#pragma unroll
      for (int l = 0; l < H; ++l) c += M.O[H][l] * o[l];
      store(H, c);
    }
  }
}

template <int NP>
struct SmallCg {
  static constexpr int kLines = NP * NP;
  static constexpr int kThreads = (2 * kLines + 31) / 32 * 32 < 128 ? 128 : (2 * kLines + 31) / 32 * 32;
};

template <int NP>
__global__ void __launch_bounds__(SmallCg<NP>::kThreads, 1)
    k_cg_small(const __grid_constant__ GllParam<NP, double> tab, int64_t E, int64_t n, const double* __restrict__ G,
               double* __restrict__ x, double* __restrict__ p, double* __restrict__ r, double* __restrict__ z,
               double* __restrict__ w, const double* __restrict__ minv, const uint8_t* __restrict__ mult,
               const double* __restrict__ ctab, const GsPlan gs, CgScalars* __restrict__ st,
               double* __restrict__ part, unsigned* __restrict__ bar, int* __restrict__ err, int max_iters) {
  constexpr int NP2 = NP * NP, P = NP2 * NP, SZ = Stage<NP>::kSize, T = SmallCg<NP>::kThreads;
  constexpr int K2 = (NP + 1) / 2;
  __shared__ double sA[SZ], sR[SZ], sS[SZ], sT[SZ];
  __shared__ double sRed[T / 32];
  __shared__ double sB;
  __shared__ bool sOk;
  // every block reads the scalars before any block can change them (the first change comes
  // after the first barrier, which every block reaches after this point)
  if (st->done) return;
  double rho = st->rho, beta = st->beta, bb = st->bb, rtol2 = st->rtol2;
  int iter = st->iter;
  const int max_iter = st->max_iter;
  unsigned gen = ld_acquire(&bar[1]);
  const int G_ = gridDim.x;
  double* part_pw = part;
  double* part_rz = part + G_;
  double* part_rr = part + 2 * G_;
  const int tid = threadIdx.x;
  const int t = tid >> 1, h = tid & 1;                 // line t, half h (tid < 2 NP^2)
  const int la = t % NP, lb = t / NP;                  // line coordinates
  const bool line_thread = tid < 2 * NP2;
  const int64_t gtid = static_cast<int64_t>(blockIdx.x) * T + tid, gstride = static_cast<int64_t>(G_) * T;
  constexpr int kRunning = -1;  // no decision yet (SEM_OK is 0)
  int status = kRunning;
  double alpha = 0.0, pw = 0.0, rz = 0.0, rr = 0.0;
  for (int it = 0; it < max_iters; ++it) {
    // ---- phase A: p = z + beta p, w = A_L p, <p, w>
    double dot = 0.0;
    for (int64_t e = blockIdx.x; e < E; e += G_) {
      const int64_t eb = e * P;
      // column (la, lb), half h of its k range
      if (line_thread) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          if ((k < K2) != (h == 0)) continue;
          const int64_t q = eb + k * NP2 + t;
          const double v = z[q] + beta * p[q];
          p[q] = v;
          sA[Stage<NP>::at(la, lb, k)] = v;
        }
      }
      __syncthreads();
      // forward contractions: i-row (j, k) = (la, lb) -> R; j-line (i, k) = (la, lb) -> S;
      // k-column (i, j) = (la, lb) -> T
      if (line_thread) {
        double in[NP];
#pragma unroll
        for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(l, la, lb)];
        eo_half<NP>(tab.Df, in, h, [&](int l, double v) { sR[Stage<NP>::at(l, la, lb)] = v; });
#pragma unroll
        for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(la, l, lb)];
        eo_half<NP>(tab.Df, in, h, [&](int l, double v) { sS[Stage<NP>::at(la, l, lb)] = v; });
#pragma unroll
        for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(la, lb, l)];
        eo_half<NP>(tab.Df, in, h, [&](int l, double v) { sT[Stage<NP>::at(la, lb, l)] = v; });
      }
      __syncthreads();
      // geometric factors on the column (la, lb), half h of k
      if (line_thread) {
        const double* g = G + e * 6 * P + t;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          if ((k < K2) != (h == 0)) continue;
          const int at = Stage<NP>::at(la, lb, k);
          const double ur = sR[at], us = sS[at], ut = sT[at];
          const double* gk = g + k * NP2;
          const double g11 = gk[0], g12 = gk[P], g13 = gk[2 * P], g22 = gk[3 * P], g23 = gk[4 * P], g33 = gk[5 * P];
          sR[at] = g11 * ur + g12 * us + g13 * ut;
          sS[at] = g12 * ur + g22 * us + g23 * ut;
          sT[at] = g13 * ur + g23 * us + g33 * ut;
        }
      }
      __syncthreads();
      // transposed contractions in place: the two threads of a line (lanes 2t, 2t + 1 of one
      // warp) read it whole before either writes, and lines of one direction are disjoint. Every
      // thread of the block reaches each warp synchronisation (also threads without a line,
      // which a warp may hold when 2 (N+1)^2 is not a multiple of 32).
      {
        double in[NP];
        if (line_thread) {
#pragma unroll
          for (int l = 0; l < NP; ++l) in[l] = sR[Stage<NP>::at(l, la, lb)];
        }
        __syncwarp();
        if (line_thread) {
          eo_half<NP>(tab.Dt, in, h, [&](int l, double v) { sR[Stage<NP>::at(l, la, lb)] = v; });
#pragma unroll
          for (int l = 0; l < NP; ++l) in[l] = sS[Stage<NP>::at(la, l, lb)];
        }
        __syncwarp();
        if (line_thread) {
          eo_half<NP>(tab.Dt, in, h, [&](int l, double v) { sS[Stage<NP>::at(la, l, lb)] = v; });
#pragma unroll
          for (int l = 0; l < NP; ++l) in[l] = sT[Stage<NP>::at(la, lb, l)];
        }
        __syncwarp();
        if (line_thread) eo_half<NP>(tab.Dt, in, h, [&](int l, double v) { sT[Stage<NP>::at(la, lb, l)] = v; });
      }
      __syncthreads();
      if (line_thread) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          if ((k < K2) != (h == 0)) continue;
          const int at = Stage<NP>::at(la, lb, k);
          const double v = sR[at] + sS[at] + sT[at];
          const int64_t q = eb + k * NP2 + t;
          w[q] = v;
          dot = fma(sA[at], v, dot);
        }
      }
      // the next element's column loads write sA only after this barrier, by which every thread
      // has read sA and sR, sS, sT of this element
      __syncthreads();
    }
    {
      const double s = block_sum(dot, sRed);
      if (tid == 0) part_pw[blockIdx.x] = s;
    }
    if (!grid_barrier(bar, gen, &sOk)) {
      status = SEM_ERR_TIMEOUT;
      break;
    }
    pw = all_sum(part_pw, G_, sRed, &sB);
    if (!(pw > 0.0) || !isfinite(pw)) {
      status = SEM_ERR_BREAKDOWN;
      alpha = 0.0;
      break;
    }
    alpha = rho / pw;
    // ---- phase B: QQ^T and the mask on w
    auto gs_class = [&](auto width, int c) {
      constexpr int W = decltype(width)::value;
      for (int64_t s = gtid; s < gs.n[c]; s += gstride) {
        int ix[W];
        double v[W];
        load_rec<W>(gs.rec[c], s, ix);
        seg_load<W>(w, ix, v);
        seg_store<W>(w, ix, gs.msk[c][s] ? 0.0 : seg_add<W>(ix, v));
      }
    };
    gs_class(std::integral_constant<int, 2>{}, 1);
    gs_class(std::integral_constant<int, 4>{}, 2);
    gs_class(std::integral_constant<int, 8>{}, 3);
    gs_class(std::integral_constant<int, 1>{}, 0);
    for (int64_t xq = gtid; xq < gs.nx; xq += gstride) {
      const int o0 = gs.xoff[xq], o1 = gs.xoff[xq + 1];
      double s = w[gs.xidx[o0]];
      for (int o = o0 + 1; o < o1; ++o) s += w[gs.xidx[o]];
      if (gs.xmsk[xq]) s = 0.0;
      for (int o = o0; o < o1; ++o) w[gs.xidx[o]] = s;
    }
    if (!grid_barrier(bar, gen, &sOk)) {
      status = SEM_ERR_TIMEOUT;
      break;
    }
    // ---- phase C: x, r, z updates and the two dots
    double drz = 0.0, drr = 0.0;
    for (int64_t i = gtid; i < n; i += gstride) {
      x[i] += alpha * p[i];
      const double ri = r[i] - alpha * w[i];
      const double zi = minv ? minv[i] * ri : ri;
      r[i] = ri;
      z[i] = zi;
      const unsigned m = mult[i];
      const double c = m == 1u ? 1.0 : __ldg(ctab + m);
      drz = fma(ri, c * zi, drz);
      drr = fma(ri, c * ri, drr);
    }
    {
      const double a = block_sum(drz, sRed);
      const double b = block_sum(drr, sRed);
      if (tid == 0) {
        part_rz[blockIdx.x] = a;
        part_rr[blockIdx.x] = b;
      }
    }
    if (!grid_barrier(bar, gen, &sOk)) {
      status = SEM_ERR_TIMEOUT;
      break;
    }
    rz = all_sum(part_rz, G_, sRed, &sB);
    rr = all_sum(part_rr, G_, sRed, &sB);
    ++iter;
    if (!isfinite(rz) || !isfinite(rr)) {
      status = SEM_ERR_BREAKDOWN;
      break;
    }
    if (rr <= rtol2 * bb) {
      status = SEM_OK;
      break;
    }
    if (iter >= max_iter) {
      status = SEM_ERR_NOT_CONVERGED;
      break;
    }
    beta = rz / rho;
    rho = rz;
  }
  // every block took the same decisions; block 0 publishes them
  if (blockIdx.x == 0 && tid == 0) {
    st->iter = iter;
    st->rho = rho;
    st->beta = beta;
    st->alpha = 0.0;  // x is up to date (no deferred update in this solver)
    st->pw = pw;
    st->rz = rz;
    st->rr = rr;
    if (status != kRunning) {
      st->status = status;
      st->done = 1;
    }
  }
  if (status == SEM_ERR_TIMEOUT && tid == 0) {  // whichever block gave up, the solve reports it
    atomicExch(err, static_cast<int>(SEM_ERR_TIMEOUT));
    atomicExch(&st->status, static_cast<int>(SEM_ERR_TIMEOUT));
    atomicExch(&st->done, 1);
  }
}

template <int NP>
sem_status launch_small_np(int N, const SmallCgLaunch& a, cudaStream_t s) {
  constexpr int T = SmallCg<NP>::kThreads;
  static const int cap = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_small<NP>, T, 0);
    return per_sm > 0 ? sms : 0;  // one block per SM (all resident: cooperative launch)
  }();
  if (cap <= 0) return fail(SEM_ERR_UNSUPPORTED, "the persistent CG kernel does not fit on an SM");
  int grid = cap < a.max_blocks ? cap : a.max_blocks;
  if (grid > kRedMax) grid = kRedMax;
  const GllParam<NP, double> tab = make_gll_param<NP, double>(N);
  int64_t E = a.E, n = a.n;
  const double* G = a.G;
  double *x = a.x, *p = a.p, *r = a.r, *z = a.z, *w = a.w;
  const double* minv = a.minv;
  const uint8_t* mult = a.mult;
  const double* ctab = a.ctab;
  GsPlan gs = a.gs;
  CgScalars* st = a.st;
  double* part = a.part;
  unsigned* bar = a.bar;
  int* err = a.err;
  int iters = a.iters;
  void* args[] = {const_cast<GllParam<NP, double>*>(&tab), &E, &n, &G, &x, &p, &r, &z, &w, &minv, &mult, &ctab,
                  &gs, &st, &part, &bar, &err, &iters};
  SEM_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_cg_small<NP>), dim3(grid), dim3(T), args, 0, s));
  count_launch();
  return SEM_OK;
}

template <int LO, int HI>
sem_status launch_small_range(int N, const SmallCgLaunch& a, cudaStream_t s) {
  if constexpr (LO > HI) {
    return fail(SEM_ERR_UNSUPPORTED, "polynomial order not compiled in");
  } else {
    if (N + 1 == LO) return launch_small_np<LO>(N, a, s);
    return launch_small_range<LO + 1, HI>(N, a, s);
  }
}

}  // namespace

sem_status launch_cg_small(int N, const SmallCgLaunch& a, cudaStream_t s) {
  return launch_small_range<2, kMaxNp>(N, a, s);
}

// ---- self-test of the grid barrier's bounded wait ----
namespace {

__global__ void k_probe_barrier(unsigned* bar, int skip_block, int* status) {
  __shared__ bool ok;
  unsigned gen = ld_acquire(&bar[1]);
  if (static_cast<int>(blockIdx.x) == skip_block) return;  // this block never arrives
  const bool done = grid_barrier(bar, gen, &ok);
  if (threadIdx.x == 0) atomicMax(status, done ? static_cast<int>(SEM_OK) : static_cast<int>(SEM_ERR_TIMEOUT));
}

}  // namespace

sem_status launch_probe_barrier(unsigned* bar, int blocks, int skip_block, int* status, cudaStream_t s) {
  void* args[] = {&bar, &skip_block, &status};
  SEM_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_probe_barrier), dim3(blocks), dim3(32), args, 0, s));
  count_launch();
  return SEM_OK;
}

}  // namespace sem
