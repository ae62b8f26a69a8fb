// Gather-scatter QQ^T with the Dirichlet mask (Eq. 5; Section 4.3; Algorithm 1 step 7).
//
// Segments are the global nodes that have copies on element boundaries (n_gs copies in
// all, Eq. 9), in ascending global id; the copies of a segment are listed in ascending
// local index. One thread owns one segment: it sums the copies left to right, replaces
// the sum by 0 if the node is Dirichlet, and writes the result to every copy. No atomics,
// and the floating-point result does not depend on the launch shape.
#include "k_common.cuh"

namespace sem {
namespace {

constexpr int kThreads = 256;

int seg_grid(int64_t n_seg) {
  const int64_t b = (n_seg + kThreads - 1) / kThreads;
  const int64_t cap = 152 * 8;  // eight 256-thread blocks per SM; grid-stride beyond
  return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename T>
__global__ void k_dssum(int64_t n_seg, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                        const uint8_t* __restrict__ smask, T* __restrict__ u, int apply_mask) {
  for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < n_seg;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int o0 = off[g], o1 = off[g + 1];
    T s = u[idx[o0]];
    for (int o = o0 + 1; o < o1; ++o) s += u[idx[o]];
    if (apply_mask && smask[g]) s = T(0);
    for (int o = o0; o < o1; ++o) u[idx[o]] = s;
  }
}

// CG step 7 + the boundary part of <p, w, c>: after the sum, all copies of a segment hold
// the same w and the same p, and their weights c = 1/multiplicity add up to one, so the
// segment contributes p * w once. The last block adds the Ax kernel's element-interior
// partials, forms <p, w, c> and alpha = rho / <p, w, c> (Algorithm 1 step 8).
template <typename T>
__global__ void k_dssum_cg(int64_t n_seg, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                           const uint8_t* __restrict__ smask, T* __restrict__ w, const T* __restrict__ p,
                           CgScalars* __restrict__ st, const double* __restrict__ ax_partials, int ax_blocks,
                           double* __restrict__ partials) {
  __shared__ double sRed[kThreads / 32];
  if (st->done) return;
  DotAcc<T> dot;
  for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < n_seg;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int o0 = off[g], o1 = off[g + 1];
    const int first = idx[o0];
    T s = w[first];
    for (int o = o0 + 1; o < o1; ++o) s += w[idx[o]];
    if (smask[g]) s = T(0);
    for (int o = o0; o < o1; ++o) w[idx[o]] = s;
    dot.add(p[first], s);
  }
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
      } else {
        st->alpha = st->rho / pw;
      }
    }
  }
}

// Jacobi: out = 1 / (sum of the local diagonals of a segment), or 0 if Dirichlet.
__global__ void k_dssum_invert(int64_t n_seg, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                               const uint8_t* __restrict__ smask, const double* __restrict__ d,
                               double* __restrict__ m64, float* __restrict__ m32) {
  for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < n_seg;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int o0 = off[g], o1 = off[g + 1];
    double s = d[idx[o0]];
    for (int o = o0 + 1; o < o1; ++o) s += d[idx[o]];
    const double v = smask[g] ? 0.0 : 1.0 / s;
    for (int o = o0; o < o1; ++o) {
      if (m64) m64[idx[o]] = v;
      if (m32) m32[idx[o]] = static_cast<float>(v);
    }
  }
}

}  // namespace

sem_status launch_dssum(sem_prec prec, int64_t n_seg, const int32_t* off, const int32_t* idx, const uint8_t* smask,
                        void* u, int apply_mask, cudaStream_t s) {
  if (n_seg == 0) return SEM_OK;
  if (prec == SEM_F64)
    k_dssum<double><<<seg_grid(n_seg), kThreads, 0, s>>>(n_seg, off, idx, smask, static_cast<double*>(u), apply_mask);
  else
    k_dssum<float><<<seg_grid(n_seg), kThreads, 0, s>>>(n_seg, off, idx, smask, static_cast<float*>(u), apply_mask);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_dssum_cg(sem_prec prec, int64_t n_seg, const int32_t* off, const int32_t* idx,
                           const uint8_t* smask, void* w, const void* p, CgScalars* st, const double* ax_partials,
                           int ax_blocks, double* partials, cudaStream_t s) {
  const int grid = seg_grid(n_seg);
  if (prec == SEM_F64)
    k_dssum_cg<double><<<grid, kThreads, 0, s>>>(n_seg, off, idx, smask, static_cast<double*>(w),
                                                 static_cast<const double*>(p), st, ax_partials, ax_blocks, partials);
  else
    k_dssum_cg<float><<<grid, kThreads, 0, s>>>(n_seg, off, idx, smask, static_cast<float*>(w),
                                                static_cast<const float*>(p), st, ax_partials, ax_blocks, partials);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_dssum_invert(int64_t n_seg, const int32_t* off, const int32_t* idx, const uint8_t* smask,
                               const double* d, double* m64, float* m32, cudaStream_t s) {
  if (n_seg == 0) return SEM_OK;
  k_dssum_invert<<<seg_grid(n_seg), kThreads, 0, s>>>(n_seg, off, idx, smask, d, m64, m32);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
