// Device helpers shared by the kernels of libsem.
#pragma once

#include <cuda_runtime.h>

#include "sem_internal.h"

namespace sem {

// GLL nodes, weights and derivative matrix of one order, passed by value as a
// __grid_constant__ kernel parameter (it lives in the constant bank, so fixed indices
// become constant operands and no per-module symbol upload is needed).
template <int NP, typename T>
struct GllParam {
  T D[NP * NP];  // D[a*NP + b] = l_b'(xi_a)
  T xi[NP];
  T w[NP];
};

template <int NP, typename T>
inline GllParam<NP, T> make_gll_param(int N) {
  const GllTable& t = gll_table(N);
  GllParam<NP, T> g;
  for (int a = 0; a < NP * NP; ++a) g.D[a] = static_cast<T>(t.D[a]);
  for (int a = 0; a < NP; ++a) {
    g.xi[a] = static_cast<T>(t.xi[a]);
    g.w[a] = static_cast<T>(t.w[a]);
  }
  return g;
}

// Sum of `v` over the block in a fixed order (warp shuffle tree, then warps in order);
// the result is valid in thread 0. `sh` needs blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < static_cast<int>((blockDim.x + 31) >> 5); ++q) s += sh[q];
  return s;
}

// Each block stores its partial(s); the block that arrives last (ticket) returns true
// in every thread and may then read all partials. The ticket is reset for the next use.
template <int K>
__device__ __forceinline__ bool publish_partials(const double (&v)[K], double* partials, unsigned int* ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) partials[K * blockIdx.x + q] = v[q];
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
    if (last) *ticket = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Fixed-order sum of partials[q*K + c] over q in [0, count); valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* partials, int count, int K, int c, double* sh) {
  double s = 0.0;
  for (int q = threadIdx.x; q < count; q += blockDim.x) s += __ldcg(partials + q * K + c);
  return block_sum(s, sh);
}

__host__ __device__ constexpr int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace sem

namespace sem {

// Per-thread accumulator of dot products.
// FP64 data: plain FP64 fused multiply-adds.
// FP32 data: each product is formed exactly as a pair of floats (p = x*y, e = fma(x, y, -p))
// and added to a compensated pair (Knuth's two-sum on the high parts, errors gathered in the
// low part), a 48-bit accumulation that keeps the FP64 pipe free; value() returns it in FP64
// and the block and grid sums then continue in FP64.
template <typename T>
struct DotAcc;

template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  // round-to-nearest intrinsics: the compiler must not fuse or reorder these steps
  __device__ __forceinline__ void add(float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, e));
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

}  // namespace sem
