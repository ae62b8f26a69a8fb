// Gather-scatter QQ^T with the Dirichlet mask (Eq. 5; Section 4.3; Algorithm 1 step 7).
//
// Segments are the global nodes that have copies on element boundaries (n_gs copies in
// all, Eq. 9); the copies of a segment are added in ascending local index. One thread owns
// one segment at a time: it reads the segment's copy indices (one vector load from the
// fixed-width record of its class, see GsPlan), loads the copies, sums them left to right,
// replaces the sum by 0 if the node is Dirichlet, and writes the result to every copy. No
// atomics, and the floating-point result does not depend on the launch shape or on the
// order in which segments are visited.
#include <type_traits>

#include "k_common.cuh"
#include "k_gs.cuh"

namespace sem {
namespace {

constexpr int kThreads = 256;

// Up to eight 256-thread blocks per SM, grid-stride beyond. More blocks than are resident at
// once: the gathers are latency-bound, and sizing the grid to the resident blocks (as the
// vector kernels are) made the gather-scatter 5-8% slower.
int seg_grid(int64_t n_seg) {
  static const int cap = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 8 * (sms > 0 ? sms : 1);
  }();
  const int64_t b = (n_seg + kThreads - 1) / kThreads;
  return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

// Visits the segments of fixed-width class c (records of width W): f(ix, masked).
template <int W, typename F>
__device__ __forceinline__ void for_class(const GsPlan& g, int c, int64_t t0, int64_t stride, F&& f) {
  for (int64_t t = t0; t < g.n[c]; t += stride) {
    const int64_t s = g.n[c] - 1 - t;  // last segments first: their copies were written last
    int ix[W];
    load_rec<W>(g.rec[c], s, ix);
    f(ix, g.msk[c][s] != 0);
  }
}

// In-place gather-scatter of class c, two segments per thread at a time (both records, then
// the copies of both, are loaded before anything is added or stored: segments never share
// copies). value(masked, sum, pf) gives what is written to the copies; pf is pv at the
// segment's first copy, loaded with the copies (0 if pv is null).
template <int W, typename T, typename F>
__device__ __forceinline__ void gs_class(const GsPlan& g, int c, int64_t t0, int64_t stride, T* __restrict__ u,
                                         const T* __restrict__ pv, F&& value) {
  const int64_t n = g.n[c];
  int64_t t = t0;
  for (; t + stride < n; t += 2 * stride) {
    const int64_t s0 = n - 1 - t, s1 = s0 - stride;  // last segments first: their copies were written last
    int a[W], b[W];
    load_rec<W>(g.rec[c], s0, a);
    load_rec<W>(g.rec[c], s1, b);
    const bool ma = g.msk[c][s0] != 0, mb = g.msk[c][s1] != 0;
    T va[W], vb[W];
    seg_load<W>(u, a, va);
    seg_load<W>(u, b, vb);
    const T pa = pv ? pv[a[0]] : T(0), pb = pv ? pv[b[0]] : T(0);
    const T ra = value(ma, seg_add<W>(a, va), pa);
    const T rb = value(mb, seg_add<W>(b, vb), pb);
    seg_store<W>(u, a, ra);
    seg_store<W>(u, b, rb);
  }
  if (t < n) {
    const int64_t s0 = n - 1 - t;
    int a[W];
    load_rec<W>(g.rec[c], s0, a);
    T va[W];
    seg_load<W>(u, a, va);
    const T pa = pv ? pv[a[0]] : T(0);
    seg_store<W>(u, a, value(g.msk[c][s0] != 0, seg_add<W>(a, va), pa));
  }
}

template <typename T>
__global__ void k_dssum(const GsPlan g, T* __restrict__ u, int apply_mask) {
  const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  auto value = [&](bool masked, T sum, T) { return (apply_mask && masked) ? T(0) : sum; };
  gs_class<2>(g, 1, t0, stride, u, static_cast<const T*>(nullptr), value);
  gs_class<4>(g, 2, t0, stride, u, static_cast<const T*>(nullptr), value);
  gs_class<8>(g, 3, t0, stride, u, static_cast<const T*>(nullptr), value);
  gs_class<1>(g, 0, t0, stride, u, static_cast<const T*>(nullptr), value);
  for (int64_t x = t0; x < g.nx; x += stride) {
    const int o0 = g.xoff[x], o1 = g.xoff[x + 1];
    T s = u[g.xidx[o0]];
    for (int o = o0 + 1; o < o1; ++o) s += u[g.xidx[o]];
    if (apply_mask && g.xmsk[x]) s = T(0);
    for (int o = o0; o < o1; ++o) u[g.xidx[o]] = s;
  }
}

// CG step 7. DOT: also the boundary part of <p, w, c>: after the sum, all copies of a
// segment hold the same w and the same p, and their weights c = 1/multiplicity add up to
// one, so the segment contributes p * w once; the last block adds the operator's partials and
// its own, forms <p, w, c> and alpha = rho / <p, w, c> (Algorithm 1 step 8). Without DOT the
// operator has already formed the whole product over the unassembled w (sum over local points
// of p_i (A_L p)_i equals <p, QQ^T A_L p, c> because p has one value per global node and is 0
// on Dirichlet nodes): block 0 sums the operator's partials (complete at this launch) in a
// fixed order and forms alpha before its share of the segments, and no block reduces anything
// else (no ticket, no last block).
template <typename T, bool DOT>
__global__ void __launch_bounds__(kThreads, 4) k_dssum_cg(const GsPlan g, T* __restrict__ w, const T* __restrict__ p, CgScalars* __restrict__ st,
                           const double* __restrict__ ax_partials, int ax_blocks, double* __restrict__ partials) {
  __shared__ double sRed[kThreads / 32];
  if (st->done) return;
  if constexpr (!DOT) {
    if (blockIdx.x == 0) {
      const double pw = sum_partials(ax_partials, ax_blocks, 1, 0, sRed);
      if (threadIdx.x == 0) {
        st->pw = pw;
        if (!(pw > 0.0) || !isfinite(pw)) {
          st->status = SEM_ERR_BREAKDOWN;
          st->done = 1;
          st->alpha = 0.0;  // x is not advanced along this p (fused CG: nothing left to flush)
        } else {
          st->alpha = st->rho / pw;
        }
      }
    }
  }
  const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  DotAcc<T> dot;
  const T* pv = DOT ? p : nullptr;
  auto value = [&](bool masked, T sum, T pf) {
    const T s = masked ? T(0) : sum;
    if constexpr (DOT) dot.add(pf, s);
    return s;
  };
  gs_class<2>(g, 1, t0, stride, w, pv, value);
  gs_class<4>(g, 2, t0, stride, w, pv, value);
  gs_class<8>(g, 3, t0, stride, w, pv, value);
  gs_class<1>(g, 0, t0, stride, w, pv, value);
  for (int64_t x = t0; x < g.nx; x += stride) {
    const int o0 = g.xoff[x], o1 = g.xoff[x + 1];
    const int first = g.xidx[o0];
    T s = w[first];
    for (int o = o0 + 1; o < o1; ++o) s += w[g.xidx[o]];
    if (g.xmsk[x]) s = T(0);
    for (int o = o0; o < o1; ++o) w[g.xidx[o]] = s;
    if constexpr (DOT) dot.add(p[first], s);
  }
  if constexpr (DOT) {  // without DOT block 0 has formed alpha: nothing to reduce here
    const double v[1] = {block_sum(dot.value(), sRed)};
    if (publish_partials<1>(v, partials, &st->ticket[0])) {
      const double a = sum_partials(ax_partials, ax_blocks, 1, 0, sRed);
      const double b = sum_partials(partials, gridDim.x, 1, 0, sRed);
      if (threadIdx.x == 0) {
        const double pw = a + b;
        st->pw = pw;
        if (!(pw > 0.0) || !isfinite(pw)) {
          st->status = SEM_ERR_BREAKDOWN;
          st->done = 1;
          st->alpha = 0.0;  // x is not advanced along this p (fused CG: nothing left to flush)
        } else {
          st->alpha = st->rho / pw;
        }
      }
    }
  }
}

// Jacobi: out = 1 / (sum of the local diagonals of a segment), or 0 if Dirichlet.
__global__ void k_dssum_invert(const GsPlan g, const double* __restrict__ d, double* __restrict__ m64,
                               float* __restrict__ m32) {
  const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  auto body = [&](const auto& ix, bool masked) {
    constexpr int W = std::extent<std::remove_reference_t<decltype(ix)>>::value;
    const double v = masked ? 0.0 : 1.0 / seg_sum<W>(d, ix);
    if (m64) seg_store<W>(m64, ix, v);
    if (m32) seg_store<W>(m32, ix, static_cast<float>(v));
  };
  for_class<2>(g, 1, t0, stride, body);
  for_class<4>(g, 2, t0, stride, body);
  for_class<8>(g, 3, t0, stride, body);
  for_class<1>(g, 0, t0, stride, body);
  for (int64_t x = t0; x < g.nx; x += stride) {
    const int o0 = g.xoff[x], o1 = g.xoff[x + 1];
    double s = d[g.xidx[o0]];
    for (int o = o0 + 1; o < o1; ++o) s += d[g.xidx[o]];
    const double v = g.xmsk[x] ? 0.0 : 1.0 / s;
    for (int o = o0; o < o1; ++o) {
      if (m64) m64[g.xidx[o]] = v;
      if (m32) m32[g.xidx[o]] = static_cast<float>(v);
    }
  }
}

}  // namespace

sem_status launch_dssum(sem_prec prec, const GsPlan& g, void* u, int apply_mask, cudaStream_t s) {
  if (g.total() == 0) return SEM_OK;
  const int grid = seg_grid(g.total());
  if (prec == SEM_F64)
    k_dssum<double><<<grid, kThreads, 0, s>>>(g, static_cast<double*>(u), apply_mask);
  else
    k_dssum<float><<<grid, kThreads, 0, s>>>(g, static_cast<float*>(u), apply_mask);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_dssum_cg(sem_prec prec, const GsPlan& g, void* w, const void* p, CgScalars* st,
                           const double* ax_partials, int ax_blocks, double* partials, cudaStream_t s) {
  const int grid = seg_grid(g.total());
  if (prec == SEM_F64) {
    if (p)
      k_dssum_cg<double, true><<<grid, kThreads, 0, s>>>(g, static_cast<double*>(w), static_cast<const double*>(p),
                                                         st, ax_partials, ax_blocks, partials);
    else
      k_dssum_cg<double, false><<<grid, kThreads, 0, s>>>(g, static_cast<double*>(w), nullptr, st, ax_partials,
                                                          ax_blocks, partials);
  } else {
    if (p)
      k_dssum_cg<float, true><<<grid, kThreads, 0, s>>>(g, static_cast<float*>(w), static_cast<const float*>(p), st,
                                                        ax_partials, ax_blocks, partials);
    else
      k_dssum_cg<float, false><<<grid, kThreads, 0, s>>>(g, static_cast<float*>(w), nullptr, st, ax_partials,
                                                         ax_blocks, partials);
  }
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_dssum_invert(const GsPlan& g, const double* d, double* m64, float* m32, cudaStream_t s) {
  if (g.total() == 0) return SEM_OK;
  k_dssum_invert<<<seg_grid(g.total()), kThreads, 0, s>>>(g, d, m64, m32);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
