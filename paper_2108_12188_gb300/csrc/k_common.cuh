// Device helpers shared by the kernels of libsem.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "sem_internal.h"

namespace sem {

// GLL nodes, weights and derivative matrix of one order, passed by value as a
// __grid_constant__ kernel parameter (it lives in the constant bank, so fixed indices
// become constant operands and no per-module symbol upload is needed).
//
// A matrix M with M(N-i, N-l) = -M(i, l) (D and D^T: the GLL nodes are symmetric, so
// l_{N-b}'(xi_{N-a}) = -l_b'(xi_a)) is kept in its even/odd split (Kopriva's form): with
// H = NP/2, e_l = u_l + u_{N-l} and o_l = u_l - u_{N-l} (l < H),
//   A_i = sum_l E(i,l) e_l [+ M(i,m) u_m],  B_i = sum_l O(i,l) o_l   (i < H),
//   (M u)_i = A_i + B_i,  (M u)_{N-i} = B_i - A_i,  [(M u)_m = sum_l M(m,l) o_l],
// E(i,l) = (M(i,l) + M(i,N-l)) / 2, O(i,l) = (M(i,l) - M(i,N-l)) / 2; the bracketed terms
// exist for odd NP only (middle index m = H, where M(m,m) = 0). E carries M(i,m) as its last
// column and O carries M(m,l) as its last row. A line of NP values then costs 2 H^2 + 4 H
// (+ 2 H) operations instead of NP^2.
// FP32: the H x H blocks of E and O interleaved, (E(i,l), O(i,l)) as one float2, so that
// eo_apply forms A_i and B_i together with the two-wide FP32 multiply-add of sm_100 and
// later (one instruction for both sums, the same roundings as two scalar ones).
template <int NP, typename T>
struct EoPairs {};
template <int NP>
struct EoPairs<NP, float> {
  float2 EO[NP / 2 > 0 ? NP / 2 : 1][NP / 2 > 0 ? NP / 2 : 1];
};

template <int NP, typename T>
struct EoMat : EoPairs<NP, T> {
  static constexpr int H = NP / 2, HC = (NP + 1) / 2;
  T E[H][HC];
  T O[HC][H];
};

template <int NP, typename T>
struct GllParam {
  T D[NP * NP];  // D[a*NP + b] = l_b'(xi_a)
  T xi[NP];
  T w[NP];
  EoMat<NP, T> Df;  // split of D
  EoMat<NP, T> Dt;  // split of D^T
};

// Even/odd split of the NP x NP matrix M(i, l) = m(i, l) (FP64 on the host).
template <int NP, typename T, typename F>
inline EoMat<NP, T> make_eo(F m) {
  constexpr int H = NP / 2, N = NP - 1;
  EoMat<NP, T> r{};
  for (int i = 0; i < H; ++i) {
    for (int l = 0; l < H; ++l) {
      r.E[i][l] = static_cast<T>(0.5 * (m(i, l) + m(i, N - l)));
      r.O[i][l] = static_cast<T>(0.5 * (m(i, l) - m(i, N - l)));
    }
    if (NP % 2) r.E[i][(NP + 1) / 2 - 1] = static_cast<T>(m(i, H));
  }
  if constexpr (std::is_same_v<T, float>)
    for (int i = 0; i < H; ++i)
      for (int l = 0; l < H; ++l) r.EO[i][l] = make_float2(r.E[i][l], r.O[i][l]);
  if (NP % 2)
    for (int l = 0; l < H; ++l) r.O[(NP + 1) / 2 - 1][l] = static_cast<T>(m(H, l));
  return r;
}

template <int NP, typename T>
inline GllParam<NP, T> make_gll_param(int N) {
  const GllTable& t = gll_table(N);
  GllParam<NP, T> g;
  for (int a = 0; a < NP * NP; ++a) g.D[a] = static_cast<T>(t.D[a]);
  for (int a = 0; a < NP; ++a) {
    g.xi[a] = static_cast<T>(t.xi[a]);
    g.w[a] = static_cast<T>(t.w[a]);
  }
  g.Df = make_eo<NP, T>([&](int i, int l) { return t.D[i * NP + l]; });
  g.Dt = make_eo<NP, T>([&](int i, int l) { return t.D[l * NP + i]; });
  return g;
}

// out = M in through the even/odd split (see EoMat); `in` and `out` may not alias.
template <int NP, typename T>
__device__ __forceinline__ void eo_apply(const EoMat<NP, T>& M, const T (&in)[NP], T (&out)[NP]) {
  constexpr int H = NP / 2, N = NP - 1;
  T e[H], o[H];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    e[l] = in[l] + in[N - l];
    o[l] = in[l] - in[N - l];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T a, b;
    if constexpr (std::is_same_v<T, float>) {  // both sums in one two-wide multiply-add per l
      float2 ab = __fmul2_rn(M.EO[i][0], make_float2(e[0], o[0]));
#pragma unroll
      for (int l = 1; l < H; ++l) ab = __ffma2_rn(M.EO[i][l], make_float2(e[l], o[l]), ab);
      a = ab.x;
      b = ab.y;
    } else {
      a = M.E[i][0] * e[0];
      b = M.O[i][0] * o[0];
#pragma unroll
      for (int l = 1; l < H; ++l) {
        a += M.E[i][l] * e[l];
        b += M.O[i][l] * o[l];
      }
    }
    if constexpr (NP % 2 == 1) a += M.E[i][H] * in[H];
    out[i] = a + b;
    out[N - i] = b - a;
  }
  if constexpr (NP % 2 == 1) {
    T c = M.O[H][0] * o[0];
#pragma unroll
    for (int l = 1; l < H; ++l) c += M.O[H][l] * o[l];
    out[H] = c;
  }
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

// Blocks of kernel K (with `threads` threads and no dynamic shared memory) that are resident
// on the device at once: SMs x blocks per SM, computed on first use. Grid-stride kernels are
// launched with at most this many blocks, so that all of them run in one wave.
template <auto K>
int resident_blocks(int threads) {
  static const int cap = [threads] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K, threads, 0);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }();
  return cap;
}

__host__ __device__ constexpr int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

// Position of point (i, j, k) of an element in the CG layout (see CgMap): with MB = 4 NP - 4
// boundary points per interior k-plane and NB = NP^3 - (NP - 2)^3 boundary points per element,
// the k = 0 plane, then for 0 < k < N its row j = 0, the ends i = 0 and i = N of rows 0 < j < N,
// its row j = N, then the k = N plane, and after the NB boundary points the interior ones.
__host__ __device__ __forceinline__ int cg_pos(int NP, int i, int j, int k) {
  const int N = NP - 1, NP2 = NP * NP, MB = 4 * NP - 4;
  if (k == 0) return j * NP + i;
  if (k == N) return NP2 + (N - 1) * MB + j * NP + i;
  const int base = NP2 + (k - 1) * MB;
  if (j == 0) return base + i;
  if (j == N) return base + NP + 2 * (NP - 2) + i;
  if (i == 0) return base + NP + 2 * (j - 1);
  if (i == N) return base + NP + 2 * (j - 1) + 1;
  const int NB = 2 * NP2 + (NP - 2) * MB;
  return NB + ((k - 1) * (NP - 2) + (j - 1)) * (NP - 2) + (i - 1);
}

// The CG-layout position of local index idx (idx < 2^31).
__device__ __forceinline__ int64_t cg_at(const CgMap& m, int64_t idx) {
  const unsigned long long e = __umul64hi(static_cast<unsigned long long>(idx), m.magic);
  const int loc = static_cast<int>(idx - static_cast<int64_t>(e) * m.P);
  return static_cast<int64_t>(e) * m.P + __ldg(m.perm + loc);
}

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
  __device__ __forceinline__ void add_sum(double v) { s += v; }
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
  // adds a partial sum formed elsewhere (Knuth's two-sum; its error goes to the low part)
  __device__ __forceinline__ void add_sum(float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, t);
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

}  // namespace sem
