// Gather-scatter helpers shared by the single-mesh kernels (k_gs.cu) and the batched ones
// (k_batch.cu): reading a segment's copy indices from its fixed-width record (GsPlan), loading
// its copies, adding them in record order (ascending local index) and storing the sum.
#pragma once

#include "k_common.cuh"

namespace sem {

// Copy indices of segment s of a class of width W (padding entries are -1).
template <int W>
__device__ __forceinline__ void load_rec(const int32_t* __restrict__ rec, int64_t s, int (&ix)[W]) {
  if constexpr (W == 1) {
    ix[0] = __ldg(rec + s);
  } else if constexpr (W == 2) {
    const int2 v = __ldg(reinterpret_cast<const int2*>(rec) + s);
    ix[0] = v.x;
    ix[1] = v.y;
  } else {
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(rec) + s * (W / 4) + q);
      ix[4 * q] = v.x;
      ix[4 * q + 1] = v.y;
      ix[4 * q + 2] = v.z;
      ix[4 * q + 3] = v.w;
    }
  }
}

// Sum of the copies in record order (ascending local index), padding skipped; the loads
// are issued before the additions.
template <int W, typename T>
__device__ __forceinline__ T seg_sum(const T* __restrict__ u, const int (&ix)[W]) {
  T v[W];
#pragma unroll
  for (int q = 0; q < W; ++q) v[q] = (q == 0 || ix[q] >= 0) ? u[ix[q]] : T(0);
  T s = v[0];
#pragma unroll
  for (int q = 1; q < W; ++q)
    if (ix[q] >= 0) s += v[q];
  return s;
}

template <int W, typename T>
__device__ __forceinline__ void seg_store(T* __restrict__ u, const int (&ix)[W], T s) {
#pragma unroll
  for (int q = 0; q < W; ++q)
    if (q == 0 || ix[q] >= 0) u[ix[q]] = s;
}

// Copies of a segment in record order (padding entries read as 0, never added).
template <int W, typename T>
__device__ __forceinline__ void seg_load(const T* __restrict__ u, const int (&ix)[W], T (&v)[W]) {
#pragma unroll
  for (int q = 0; q < W; ++q) v[q] = (q == 0 || ix[q] >= 0) ? u[ix[q]] : T(0);
}

template <int W, typename T>
__device__ __forceinline__ T seg_add(const int (&ix)[W], const T (&v)[W]) {
  T s = v[0];
#pragma unroll
  for (int q = 1; q < W; ++q)
    if (ix[q] >= 0) s += v[q];
  return s;
}

}  // namespace sem
