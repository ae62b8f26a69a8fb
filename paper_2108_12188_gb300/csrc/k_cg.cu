// Conjugate-gradient vector kernels (Algorithm 1 with z = M^-1 r for the Jacobi
// preconditioner). Steps 9-11 are fused into one pass (Section 5.1's loop fusion):
//   x += alpha p;  r -= alpha w;  z = M^-1 r;  partials of <r, z, c> and <r, r, c>,
// and the last block to finish forms rho, beta, the iteration count and the stopping
// decision on the device, so the host never waits inside an iteration. With the FP32 and
// double-float operators the x update (one iteration late) and z = M^-1 r move into the
// operator's prologue (fused update kernel; k_cg_flush adds the last pending x update).
//
// Weights c = 1 / multiplicity come from a per-point multiplicity byte and a 256-entry
// table of exact reciprocals (interior points have multiplicity 1). Dot products are
// accumulated per thread and combined in FP64 in a fixed order, so they are bitwise
// reproducible for a given mesh and launch. In the FP64 update the two dots run in
// double-float arithmetic on the FP32 pipes (k_df.cuh): GB300's FP64 pipe, 1/64 of the FP32
// rate, would otherwise bound the kernel above its HBM time.
#include "k_common.cuh"
#include "k_df.cuh"

namespace sem {
namespace {

constexpr int kThreads = 256;

// One thread per kThreads-th of the points at most, and no more blocks than are resident at
// once (cap = resident_blocks of the kernel): grid-stride beyond.
int vec_grid(int64_t n, int cap) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

__device__ __forceinline__ double weight(const uint8_t* __restrict__ mult, const double* __restrict__ ctab, int64_t i) {
  const unsigned m = mult[i];
  return m == 1u ? 1.0 : __ldg(ctab + m);
}

// c_i in the vector's type: the FP64 table for FP64 data, its FP32 rounding for FP32 data
// (exact for multiplicities that are powers of two, as on box meshes).
template <typename T>
__device__ __forceinline__ T weight_t(const uint8_t* __restrict__ mult, const double* __restrict__ ctab, int64_t i) {
  const unsigned m = mult[i];
  return m == 1u ? T(1) : static_cast<T>(__ldg(ctab + m));
}

template <typename T>
__global__ void k_glsc3(int64_t n, const T* __restrict__ a, const T* __restrict__ b, const uint8_t* __restrict__ mult,
                        const double* __restrict__ ctab, double* __restrict__ partials, unsigned int* ticket,
                        double* __restrict__ result) {
  __shared__ double sRed[kThreads / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    acc += static_cast<double>(a[i]) * static_cast<double>(b[i]) * weight(mult, ctab, i);
  const double v[1] = {block_sum(acc, sRed)};
  if (publish_partials<1>(v, partials, ticket)) {
    const double s = sum_partials(partials, gridDim.x, 1, 0, sRed);
    if (threadIdx.x == 0) *result = s;
  }
}

// r = b - A x0 (A x0 assembled and masked; null for x0 = 0), z = M^-1 r, p = 0;
// rho = <r,z,c>, <r,r,c>, <b,b,c>.
template <typename T>
__global__ void k_cg_init(int64_t n, const T* __restrict__ b, const T* __restrict__ ax0, T* __restrict__ r,
                          T* __restrict__ z, T* __restrict__ p, const T* __restrict__ minv,
                          const uint8_t* __restrict__ mult, const double* __restrict__ ctab, CgScalars* st,
                          double* __restrict__ partials) {
  __shared__ double sRed[kThreads / 32];
  DotAcc<T> rz, rr, bb;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const T bi = b[i];
    const T ri = ax0 ? bi - ax0[i] : bi;  // ax0 == nullptr: x0 = 0
    const T zi = minv ? minv[i] * ri : ri;
    r[i] = ri;
    z[i] = zi;
    p[i] = T(0);
    const T c = weight_t<T>(mult, ctab, i);
    rz.add(ri, c * zi);
    rr.add(ri, c * ri);
    bb.add(bi, c * bi);
  }
  const double v[3] = {block_sum(rz.value(), sRed), block_sum(rr.value(), sRed), block_sum(bb.value(), sRed)};
  if (publish_partials<3>(v, partials, &st->ticket[2])) {
    const double srz = sum_partials(partials, gridDim.x, 3, 0, sRed);
    const double srr = sum_partials(partials, gridDim.x, 3, 1, sRed);
    const double sbb = sum_partials(partials, gridDim.x, 3, 2, sRed);
    if (threadIdx.x == 0) {
      st->rho = srz;
      st->rz = srz;
      st->rr = srr;
      st->bb = sbb;
      st->beta = 0.0;
      st->alpha = 0.0;
      st->iter = 0;
      if (!isfinite(srz) || !isfinite(srr) || !isfinite(sbb)) {
        st->status = SEM_ERR_BREAKDOWN;
        st->done = 1;
      } else if (srr <= st->rtol2 * sbb) {
        st->status = SEM_OK;
        st->done = 1;
      } else if (st->max_iter <= 0) {
        st->status = SEM_ERR_NOT_CONVERGED;
        st->done = 1;
      } else {
        st->status = 0;
        st->done = 0;
      }
    }
  }
}

// Vector of 16 bytes of T (two doubles, four floats) and the matching multiplicity bytes.
template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
  using type = double2;
  using mtype = uchar2;
  static constexpr int V = 2;
};
template <>
struct Vec16<float> {
  using type = float4;
  using mtype = uchar4;
  static constexpr int V = 4;
};

// Algorithm 1 steps 9-13 with z = M^-1 r. Each thread takes 16 bytes of every vector per
// step (vector loads and stores; FUSED: two steps at a time with all their loads issued
// first); the last n mod (16 / sizeof(T)) points are done singly. FP64 w, written by the
// operator in the CG layout and assembled there by the gather-scatter, is read through `map`.
// FUSED: the operator's CG prologue makes x += alpha p (one iteration later) and recomputes
// z = M^-1 r, so this kernel leaves x alone and stores no z (z is formed for the dots only).
template <typename T, bool FUSED>
__global__ void k_cg_update(int64_t n, T* __restrict__ x, const T* __restrict__ p, T* __restrict__ r,
                            const T* __restrict__ w, T* __restrict__ z, const T* __restrict__ minv,
                            const uint8_t* __restrict__ mult, const double* __restrict__ ctab, CgScalars* st,
                            double* __restrict__ partials, const CgMap map) {
  __shared__ double sRed[kThreads / 32];
  if (st->done) return;
  using VT = typename Vec16<T>::type;
  using MT = typename Vec16<T>::mtype;
  constexpr int V = Vec16<T>::V;
  const T alpha = static_cast<T>(st->alpha);
  const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t nv = n / V;
  struct Pack {
    VT x, r, p, w, m;
    MT c;
  };
  auto load = [&](int64_t q, Pack& k) {
    k.r = reinterpret_cast<const VT*>(r)[q];
    if constexpr (sizeof(T) == 4) {
      k.w = reinterpret_cast<const VT*>(w)[q];
    } else {  // w of the V points q V .. q V + V - 1, read in the CG layout
      T* ws = reinterpret_cast<T*>(&k.w);
      const int64_t i0 = q * V;
      unsigned long long e = __umul64hi(static_cast<unsigned long long>(i0), map.magic);
      int loc = static_cast<int>(i0 - static_cast<int64_t>(e) * map.P);
#pragma unroll
      for (int l = 0; l < V; ++l) {
        ws[l] = w[static_cast<int64_t>(e) * map.P + __ldg(map.perm + loc)];
        if (++loc == map.P) {
          loc = 0;
          ++e;
        }
      }
    }
    k.m = minv ? reinterpret_cast<const VT*>(minv)[q] : VT{};
    k.c = reinterpret_cast<const MT*>(mult)[q];
    if constexpr (!FUSED) {
      k.x = reinterpret_cast<const VT*>(x)[q];
      k.p = reinterpret_cast<const VT*>(p)[q];
    } else {
      k.x = VT{};
      k.p = VT{};
    }
  };
  // point(x, p, r, w, z, minv, multiplicity) on every lane of step q, then the stores
  auto finish = [&](int64_t q, Pack& k, auto&& point) {
    VT zv;
    T* xs = reinterpret_cast<T*>(&k.x);
    T* rs = reinterpret_cast<T*>(&k.r);
    T* zs = reinterpret_cast<T*>(&zv);
    const T* ps = reinterpret_cast<const T*>(&k.p);
    const T* ws = reinterpret_cast<const T*>(&k.w);
    const T* ms = reinterpret_cast<const T*>(&k.m);
    const unsigned char* cs = reinterpret_cast<const unsigned char*>(&k.c);
#pragma unroll
    for (int l = 0; l < V; ++l) point(xs[l], ps[l], rs[l], ws[l], zs[l], ms[l], cs[l]);
    reinterpret_cast<VT*>(r)[q] = k.r;
    if constexpr (!FUSED) {
      reinterpret_cast<VT*>(x)[q] = k.x;
      reinterpret_cast<VT*>(z)[q] = zv;
    }
  };
  auto sweep = [&](auto&& point) {
    int64_t q = t0;
    // two steps at a time where the fewer vectors leave the registers for it (fused)
    for (; FUSED && q + stride < nv; q += 2 * stride) {
      Pack a, b;
      load(q, a);
      load(q + stride, b);
      finish(q, a, point);
      finish(q + stride, b, point);
    }
    for (; q < nv; q += stride) {
      Pack a;
      load(q, a);
      finish(q, a, point);
    }
    for (int64_t i = nv * V + t0; i < n; i += stride) {
      T xi = FUSED ? T(0) : x[i], ri = r[i], zi;
      point(xi, FUSED ? T(0) : p[i], ri, w[sizeof(T) == 4 ? i : cg_at(map, i)], zi, minv ? minv[i] : T(0), mult[i]);
      r[i] = ri;
      if constexpr (!FUSED) {
        x[i] = xi;
        z[i] = zi;
      }
    }
  };
  double v[2];
  if constexpr (sizeof(T) == 8) {
    // x, r, z: three FP64 operations per point. <r, z, c> and <r, r, c>: r and z as float
    // pairs (integer split), c as a float pair from a shared table, (c r) an error-free
    // product, then rz += (c r) z and rr += (c r) r in double-float.
    __shared__ df2 sC[256];
    for (int m = threadIdx.x; m < 256; m += blockDim.x) sC[m] = m == 1 ? df2{1.f, 0.f} : df_from_double(ctab[m]);
    __syncthreads();
    df2 rz{0.f, 0.f}, rr{0.f, 0.f};
    sweep([&](T& xi, T pi, T& ri, T wi, T& zi, T mi, unsigned m) {
      if constexpr (!FUSED) xi += alpha * pi;
      ri = ri - alpha * wi;
      zi = minv ? mi * ri : ri;
      const df2 r2 = df_from_double(ri), z2 = df_from_double(zi), c2 = sC[m];
      float ch, cl;
      df_prod(c2.h, c2.l, r2.h, r2.l, ch, cl);
      df_fma_acc(rz, ch, cl, z2.h, z2.l);
      df_fma_acc(rr, ch, cl, r2.h, r2.l);
    });
    v[0] = block_sum(static_cast<double>(rz.h) + static_cast<double>(rz.l), sRed);
    v[1] = block_sum(static_cast<double>(rr.h) + static_cast<double>(rr.l), sRed);
  } else {
    DotAcc<T> rz, rr;
    sweep([&](T& xi, T pi, T& ri, T wi, T& zi, T mi, unsigned m) {
      if constexpr (!FUSED) xi += alpha * pi;
      ri = ri - alpha * wi;
      zi = minv ? mi * ri : ri;
      const T c = m == 1u ? T(1) : static_cast<T>(__ldg(ctab + m));
      rz.add(ri, c * zi);
      rr.add(ri, c * ri);
    });
    v[0] = block_sum(rz.value(), sRed);
    v[1] = block_sum(rr.value(), sRed);
  }
  if (publish_partials<2>(v, partials, &st->ticket[1])) {
    const double srz = sum_partials(partials, gridDim.x, 2, 0, sRed);
    const double srr = sum_partials(partials, gridDim.x, 2, 1, sRed);
    if (threadIdx.x == 0) {
      const int it = st->iter + 1;
      st->iter = it;
      st->rz = srz;
      st->rr = srr;
      if (!isfinite(srz) || !isfinite(srr)) {
        st->status = SEM_ERR_BREAKDOWN;
        st->done = 1;
      } else if (srr <= st->rtol2 * st->bb) {
        st->status = SEM_OK;
        st->done = 1;
      } else if (it >= st->max_iter) {
        st->status = SEM_ERR_NOT_CONVERGED;
        st->done = 1;
      } else {
        st->beta = srz / st->rho;
        st->rho = srz;
      }
    }
  }
}

}  // namespace

sem_status launch_glsc3(sem_prec prec, int64_t n, const void* a, const void* b, const uint8_t* mult,
                        const double* ctab, double* partials, unsigned int* ticket, double* result, cudaStream_t s) {
  const int grid = vec_grid(n, prec == SEM_F64 ? resident_blocks<k_glsc3<double>>(kThreads)
                                               : resident_blocks<k_glsc3<float>>(kThreads));
  if (prec == SEM_F64)
    k_glsc3<double><<<grid, kThreads, 0, s>>>(n, static_cast<const double*>(a), static_cast<const double*>(b), mult,
                                              ctab, partials, ticket, result);
  else
    k_glsc3<float><<<grid, kThreads, 0, s>>>(n, static_cast<const float*>(a), static_cast<const float*>(b), mult,
                                             ctab, partials, ticket, result);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_cg_init(sem_prec prec, int64_t n, const void* b, const void* ax0, void* r, void* z, void* p,
                          const void* minv, const uint8_t* mult, const double* ctab, CgScalars* st, double* partials,
                          cudaStream_t s) {
  const int grid = vec_grid(n, prec == SEM_F64 ? resident_blocks<k_cg_init<double>>(kThreads)
                                               : resident_blocks<k_cg_init<float>>(kThreads));
  if (prec == SEM_F64)
    k_cg_init<double><<<grid, kThreads, 0, s>>>(n, static_cast<const double*>(b), static_cast<const double*>(ax0),
                                                static_cast<double*>(r), static_cast<double*>(z),
                                                static_cast<double*>(p), static_cast<const double*>(minv), mult, ctab,
                                                st, partials);
  else
    k_cg_init<float><<<grid, kThreads, 0, s>>>(n, static_cast<const float*>(b), static_cast<const float*>(ax0),
                                               static_cast<float*>(r), static_cast<float*>(z), static_cast<float*>(p),
                                               static_cast<const float*>(minv), mult, ctab, st, partials);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_cg_update(sem_prec prec, bool fused, int64_t n, void* x, const void* p, void* r, const void* w,
                            void* z, const void* minv, const uint8_t* mult, const double* ctab, CgScalars* st,
                            double* partials, const CgMap& map, cudaStream_t s) {
  const int grid = vec_grid(n, prec != SEM_F64 ? resident_blocks<k_cg_update<float, true>>(kThreads)
                               : fused         ? resident_blocks<k_cg_update<double, true>>(kThreads)
                                               : resident_blocks<k_cg_update<double, false>>(kThreads));
  if (prec == SEM_F64) {
    auto* xd = static_cast<double*>(x);
    auto* pd = static_cast<const double*>(p);
    auto* rd = static_cast<double*>(r);
    auto* wd = static_cast<const double*>(w);
    auto* zd = static_cast<double*>(z);
    auto* md = static_cast<const double*>(minv);
    if (fused)
      k_cg_update<double, true><<<grid, kThreads, 0, s>>>(n, xd, pd, rd, wd, zd, md, mult, ctab, st, partials, map);
    else
      k_cg_update<double, false><<<grid, kThreads, 0, s>>>(n, xd, pd, rd, wd, zd, md, mult, ctab, st, partials, map);
  } else {
    if (!fused) return fail(SEM_ERR_UNSUPPORTED, "the FP32 CG update runs with the fused operator prologue only");
    k_cg_update<float, true><<<grid, kThreads, 0, s>>>(n, static_cast<float*>(x), static_cast<const float*>(p),
                                                       static_cast<float*>(r), static_cast<const float*>(w),
                                                       static_cast<float*>(z), static_cast<const float*>(minv), mult,
                                                       ctab, st, partials, map);
  }
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

namespace {

// x += alpha p: the update that the fused CG prologue defers to the next iteration, made
// when the iterations stop. The last block sets alpha to 0, so that a later prologue (more
// iterations on the same state) adds nothing twice; alpha == 0 means nothing is pending.
template <typename T>
__global__ void k_cg_flush(int64_t n, T* __restrict__ x, const T* __restrict__ p, CgScalars* st) {
  const double a64 = st->alpha;  // every block reads alpha before the last one clears it
  if (a64 == 0.0) return;
  const T a = static_cast<T>(a64);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] += a * p[i];
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(&st->ticket[4], 1u);
    last = (t == gridDim.x - 1);
    if (last) {
      st->ticket[4] = 0u;
      st->alpha = 0.0;
    }
  }
}

}  // namespace

sem_status launch_cg_flush(sem_prec prec, int64_t n, void* x, const void* p, CgScalars* st, cudaStream_t s) {
  const int grid = vec_grid(n, prec == SEM_F64 ? resident_blocks<k_cg_flush<double>>(kThreads)
                                               : resident_blocks<k_cg_flush<float>>(kThreads));
  if (prec == SEM_F64)
    k_cg_flush<double><<<grid, kThreads, 0, s>>>(n, static_cast<double*>(x), static_cast<const double*>(p), st);
  else
    k_cg_flush<float><<<grid, kThreads, 0, s>>>(n, static_cast<float*>(x), static_cast<const float*>(p), st);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem

namespace sem {
namespace {

__global__ void k_ir_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ w,
                              double* __restrict__ r64, float* __restrict__ r32, const uint8_t* __restrict__ mult,
                              const double* __restrict__ ctab, CgScalars* st, double* __restrict__ partials) {
  __shared__ double sRed[kThreads / 32];
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double bi = b[i], ri = bi - w[i];
    r64[i] = ri;
    r32[i] = static_cast<float>(ri);
    const double c = weight(mult, ctab, i);
    rr += c * ri * ri;
    bb += c * bi * bi;
  }
  const double v[2] = {block_sum(rr, sRed), block_sum(bb, sRed)};
  if (publish_partials<2>(v, partials, &st->ticket[3])) {
    const double srr = sum_partials(partials, gridDim.x, 2, 0, sRed);
    const double sbb = sum_partials(partials, gridDim.x, 2, 1, sRed);
    if (threadIdx.x == 0) {
      st->rr = srr;
      st->bb = sbb;
      if (!isfinite(srr) || !isfinite(sbb)) {
        st->status = SEM_ERR_BREAKDOWN;
        st->done = 1;
      } else if (srr <= st->rtol2 * sbb) {
        st->status = SEM_OK;
        st->done = 1;
      }
    }
  }
}

// Residual replacement in the FP32 CG of the reliable-update solver: r = rnew (the FP32 copy
// of the true FP64 residual), z = M^-1 r, rho' = <r, z, c>. The search direction p is kept; the
// next direction update uses beta = rho' / rho, rho being the last accepted <r, z, c> (the
// update kernel leaves it in place when it stops), and <r, r, c> becomes the reference of the
// relative stopping test. The iteration count continues.
__global__ void k_cg_replace(int64_t n, const float* __restrict__ rnew, float* __restrict__ r, float* __restrict__ z,
                             const float* __restrict__ minv, const uint8_t* __restrict__ mult,
                             const double* __restrict__ ctab, CgScalars* st, double* __restrict__ partials) {
  __shared__ double sRed[kThreads / 32];
  DotAcc<float> rz, rr;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float ri = rnew[i];
    const float zi = minv ? minv[i] * ri : ri;
    r[i] = ri;
    z[i] = zi;
    const float c = weight_t<float>(mult, ctab, i);
    rz.add(ri, c * zi);
    rr.add(ri, c * ri);
  }
  const double v[2] = {block_sum(rz.value(), sRed), block_sum(rr.value(), sRed)};
  if (publish_partials<2>(v, partials, &st->ticket[2])) {
    const double srz = sum_partials(partials, gridDim.x, 2, 0, sRed);
    const double srr = sum_partials(partials, gridDim.x, 2, 1, sRed);
    if (threadIdx.x == 0) {
      if (!isfinite(srz) || !isfinite(srr) || !(st->rho > 0.0)) {
        st->status = SEM_ERR_BREAKDOWN;
        st->done = 1;
      } else {
        st->beta = srz / st->rho;
        st->rho = srz;
        st->rz = srz;
        st->rr = srr;
        st->bb = srr;
        st->status = 0;
        st->done = srr > 0.0 ? 0 : 1;
        if (st->done) st->status = SEM_OK;
      }
    }
  }
}

__global__ void k_ir_correct(int64_t n, double* __restrict__ x, const float* __restrict__ d) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] += static_cast<double>(d[i]);
}

}  // namespace

sem_status launch_ir_residual(int64_t n, const double* b, const double* w, double* r64, float* r32,
                              const uint8_t* mult, const double* ctab, CgScalars* st, double* partials,
                              cudaStream_t s) {
  k_ir_residual<<<vec_grid(n, resident_blocks<k_ir_residual>(kThreads)), kThreads, 0, s>>>(n, b, w, r64, r32, mult, ctab, st, partials);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_cg_replace(int64_t n, const float* rnew, float* r, float* z, const float* minv, const uint8_t* mult,
                             const double* ctab, CgScalars* st, double* partials, cudaStream_t s) {
  k_cg_replace<<<vec_grid(n, resident_blocks<k_cg_replace>(kThreads)), kThreads, 0, s>>>(n, rnew, r, z, minv, mult, ctab, st, partials);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_ir_correct(int64_t n, double* x, const float* d, cudaStream_t s) {
  k_ir_correct<<<vec_grid(n, resident_blocks<k_ir_correct>(kThreads)), kThreads, 0, s>>>(n, x, d);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

namespace {

__global__ void k_cg_perm(int NP, int* __restrict__ perm) {
  const int P = NP * NP * NP;
  for (int loc = blockIdx.x * blockDim.x + threadIdx.x; loc < P; loc += gridDim.x * blockDim.x)
    perm[loc] = cg_pos(NP, loc % NP, (loc / NP) % NP, loc / (NP * NP));
}

__global__ void k_map_indices(int64_t count, const int32_t* __restrict__ in, int32_t* __restrict__ out, const CgMap map) {
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < count;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t v = in[q];
    out[q] = v < 0 ? v : static_cast<int32_t>(cg_at(map, v));
  }
}

}  // namespace

sem_status launch_cg_perm(int NP, int* perm, cudaStream_t s) {
  const int P = NP * NP * NP;
  k_cg_perm<<<(P + kThreads - 1) / kThreads, kThreads, 0, s>>>(NP, perm);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_map_indices(int64_t count, const int32_t* in, int32_t* out, const CgMap& map, cudaStream_t s) {
  if (count <= 0) return SEM_OK;
  k_map_indices<<<vec_grid(count, resident_blocks<k_map_indices>(kThreads)), kThreads, 0, s>>>(count, in, out, map);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
