// Local SEM operator w = A_L u = D^T G D u (Eq. 4, Section 3.1), one element per NP x NP
// thread tile, EPB elements per block, grid-stride over element groups.
//
//   forward:   ur = sum_l D_il u(l,j,k), us = sum_l D_jl u(i,l,k), ut = sum_l D_kl u(i,j,l)
//   geometry:  (vr, vs, vt) = G (ur, us, ut), G read from memory (STORED) or rebuilt from
//              the element's trilinear coefficients (OTF, Section 5.1's rematerialisation)
//   transpose: w = sum_l D_li vr(l,j,k) + sum_l D_lj vs(i,l,k) + sum_l D_lk vt(i,j,l)
// Each contraction runs on whole lines of NP values held in registers, through the even/odd
// split of D and D^T (EoMat), which needs about 3/4 of the multiply-adds of the plain sums;
// the split matrices are kernel parameters, so they are constant-bank operands.
// STORED: the six factor arrays of an element are one contiguous block; a bulk TMA copy
// brings the next element group's blocks into shared memory while the current group runs
// its transposed contractions (bounded mbarrier waits; a timeout sets SEM_ERR_TIMEOUT).
//
// OTF geometry without forming G: with g_b = dx/dxi_b (columns of J) and the cofactor
// rows c_0 = g_1 x g_2, c_1 = g_2 x g_0, c_2 = g_0 x g_1 (c_b = det J * row b of J^-1),
//   G v = (w_i w_j w_k / det J) C (C^T v),  C^T v = sum_b c_b v_b,
// which costs 21 multiply-adds instead of building six factors and applying them.
//
// CG mode (Algorithm 1, steps 5-6 fused, Section 5.1): the prologue forms p = z + beta p
// and stores it, the epilogue stores w (FP64 in the CG layout, cg_pos: boundary points first)
// and adds p.w over every point into a per-block partial of <p, w, c> (the sum over the local
// points of p_i (A_L p)_i is <p, QQ^T A_L p, c>, p having one value per global node and 0 on
// Dirichlet nodes), so the gather-scatter reads no p. FP64 adds the interior points' products
// with FP64 multiply-adds and the boundary points' in double-float arithmetic on the FP32
// pipes, which the FP64-pipe-bound kernel leaves idle. The FP32 prologue also takes the
// previous iteration's x update and z = M^-1 r (phase 0 below).
#pragma once

#include <type_traits>

#include "k_common.cuh"
#include "k_df.cuh"
#include "k_tma.cuh"

namespace sem {

// Elements per block: the default shape and the alternative the tuner also tries (block shape
// choice 0 / 1). Both keep the two staging buffers of a block within 48 KB of shared memory.
template <int NP>
__host__ __device__ constexpr int ax_epb() {
  return NP <= 2 ? 32 : NP == 3 ? 16 : NP == 4 ? 8 : NP == 5 ? 5 : NP <= 7 ? (NP == 6 ? 4 : 3) : NP <= 9 ? 2 : 1;
}
template <int NP>
__host__ __device__ constexpr int ax_epb_alt() {
  return NP == 2 ? 16 : NP == 3 ? 8 : NP == 4 ? 4 : NP <= 6 ? 2 : NP <= 9 ? 1 : NP <= 11 ? 2 : 1;
}
template <int NP>
__host__ __device__ constexpr int ax_epb_of(int choice) {
  return choice == 0 ? ax_epb<NP>() : ax_epb_alt<NP>();
}

template <typename T>
struct Vec3 {
  T x, y, z;
};
template <typename T>
__device__ __forceinline__ Vec3<T> cross(const Vec3<T>& a, const Vec3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ T dot3(const Vec3<T>& a, const Vec3<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T>
__device__ __forceinline__ T div_fast(T a, T b) {
  return a / b;
}
template <>
__device__ __forceinline__ float div_fast<float>(float a, float b) {
  return __fdividef(a, b);
}

// On-the-fly geometry along one k-column (i, j) of an element (Section 5.1's rematerialised
// factors). The trilinear map x = a0 + a1 xi + a2 eta + a3 gam + a4 xi eta + a5 xi gam
// + a6 eta gam + a7 xi eta gam has the Jacobian columns
//   g0 = dx/dxi = P0 + gam Q0,  g1 = dx/deta = P1 + gam Q1,  g2 = dx/dgam (constant along k),
// so the cofactor rows c0 = g1 x g2, c1 = g2 x g0, c2 = g0 x g1 (c_b = det J times row b of
// J^-1) and det J = g0 . c0 are polynomials in gam of degree 1, 1, 2 and 2. Their coefficients
// are formed once per column; each point then costs 14 multiply-adds for C and det J, and
//   G v = (w_i w_j w_k / det J) C (C^T v)
// 21 more, instead of forming G.
template <typename T>
struct OtfColumn {
  Vec3<T> c0a, c0b, c1a, c1b, c2a, c2b, c2c;
  T da, db, dc;

  __device__ __forceinline__ void init(const T* __restrict__ a, T xi, T eta) {
    const Vec3<T> a1{a[3], a[4], a[5]}, a2{a[6], a[7], a[8]}, a3{a[9], a[10], a[11]};
    const Vec3<T> a4{a[12], a[13], a[14]}, a5{a[15], a[16], a[17]}, a6{a[18], a[19], a[20]};
    const Vec3<T> a7{a[21], a[22], a[23]};
    const Vec3<T> g2{a3.x + a5.x * xi + a6.x * eta + a7.x * xi * eta, a3.y + a5.y * xi + a6.y * eta + a7.y * xi * eta,
                     a3.z + a5.z * xi + a6.z * eta + a7.z * xi * eta};
    const Vec3<T> P0{a1.x + a4.x * eta, a1.y + a4.y * eta, a1.z + a4.z * eta};
    const Vec3<T> Q0{a5.x + a7.x * eta, a5.y + a7.y * eta, a5.z + a7.z * eta};
    const Vec3<T> P1{a2.x + a4.x * xi, a2.y + a4.y * xi, a2.z + a4.z * xi};
    const Vec3<T> Q1{a6.x + a7.x * xi, a6.y + a7.y * xi, a6.z + a7.z * xi};
    c0a = cross(P1, g2);
    c0b = cross(Q1, g2);
    c1a = cross(g2, P0);
    c1b = cross(g2, Q0);
    c2a = cross(P0, P1);
    const Vec3<T> u = cross(P0, Q1), v = cross(Q0, P1);
    c2b = {u.x + v.x, u.y + v.y, u.z + v.z};
    c2c = cross(Q0, Q1);
    da = dot3(P0, c0a);
    db = dot3(Q0, c0a) + dot3(P0, c0b);
    dc = dot3(Q0, c0b);
  }
  __device__ __forceinline__ T det(T gam) const { return da + gam * (db + gam * dc); }
  // (vr, vs, vt) = sc C (C^T (ur, us, ut)) at gam; sc = w_i w_j w_k / det J
  __device__ __forceinline__ void apply(T gam, T sc, T& ur, T& us, T& ut) const {
    const Vec3<T> c0{c0a.x + gam * c0b.x, c0a.y + gam * c0b.y, c0a.z + gam * c0b.z};
    const Vec3<T> c1{c1a.x + gam * c1b.x, c1a.y + gam * c1b.y, c1a.z + gam * c1b.z};
    const Vec3<T> c2{c2a.x + gam * (c2b.x + gam * c2c.x), c2a.y + gam * (c2b.y + gam * c2c.y),
                     c2a.z + gam * (c2b.z + gam * c2c.z)};
    const Vec3<T> q{sc * (c0.x * ur + c1.x * us + c2.x * ut), sc * (c0.y * ur + c1.y * us + c2.y * ut),
                    sc * (c0.z * ur + c1.z * us + c2.z * ut)};
    ur = dot3(c0, q);
    us = dot3(c1, q);
    ut = dot3(c2, q);
  }
};

// Phase 3 of the FP32 on-the-fly operator on one column, one point per step:
// (rR, rS, rT) <- (w_i w_j w_k / det J) C (C^T (rR, rS, rT)) (GEO 1), or with the stored word
// per point instead of w_i w_j w_k / det J (GEO 2, scale[base + k NP^2]). The nine cofactor
// entries and det J are evaluated two at a time in the lanes of the two-wide FP32 multiply-add
// of sm_100 and later, paired by component: (c0_x, c0_y), (c0_z, c1_z), (c1_x, c1_y) (linear in
// gam) and (c2_x, c2_y), (c2_z, det J) (quadratic), so no coefficient is duplicated; every
// lane performs the operations of OtfColumn in the same order.
template <int NP, int GEO>
__device__ __forceinline__ void otf_lanes(const GllParam<NP, float>& tab, const OtfColumn<float>& geo, float wij,
                                          bool valid, const float* __restrict__ scale, int64_t base,
                                          float (&rR)[NP], float (&rS)[NP], float (&rT)[NP]) {
  constexpr int NP2 = NP * NP;
  const float2 la[3] = {make_float2(geo.c0a.x, geo.c0a.y), make_float2(geo.c0a.z, geo.c1a.z),
                        make_float2(geo.c1a.x, geo.c1a.y)};
  const float2 lb[3] = {make_float2(geo.c0b.x, geo.c0b.y), make_float2(geo.c0b.z, geo.c1b.z),
                        make_float2(geo.c1b.x, geo.c1b.y)};
  const float2 qa[2] = {make_float2(geo.c2a.x, geo.c2a.y), make_float2(geo.c2a.z, geo.da)};
  const float2 qb[2] = {make_float2(geo.c2b.x, geo.c2b.y), make_float2(geo.c2b.z, geo.db)};
  const float2 qc[2] = {make_float2(geo.c2c.x, geo.c2c.y), make_float2(geo.c2c.z, geo.dc)};
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float gam = tab.xi[k];
    const float2 g2 = make_float2(gam, gam);
    float2 l[3], q[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) l[a] = __ffma2_rn(g2, lb[a], la[a]);
#pragma unroll
    for (int a = 0; a < 2; ++a) q[a] = __ffma2_rn(g2, __ffma2_rn(g2, qc[a], qb[a]), qa[a]);
    const Vec3<float> c0{l[0].x, l[0].y, l[1].x}, c1{l[2].x, l[2].y, l[1].y}, c2{q[0].x, q[0].y, q[1].x};
    float sc = 0.f;
    if (valid) {
      if constexpr (GEO == 2)
        sc = scale[base + k * NP2];
      else
        sc = div_fast(wij * tab.w[k], q[1].y);
    }
    const float ur = rR[k], us = rS[k], ut = rT[k];
    const Vec3<float> qv{sc * (c0.x * ur + c1.x * us + c2.x * ut), sc * (c0.y * ur + c1.y * us + c2.y * ut),
                         sc * (c0.z * ur + c1.z * us + c2.z * ut)};
    rR[k] = dot3(c0, qv);
    rS[k] = dot3(c1, qv);
    rT[k] = dot3(c2, qv);
  }
}

// Element stride of the stored factors (the mesh pads each element's [6][P] block to 16 bytes).
template <int NP, typename T>
__host__ __device__ constexpr int ax_gstride() {
  return sizeof(T) == 8 ? 6 * NP * NP * NP : (6 * NP * NP * NP + 3) / 4 * 4;
}

// Staging buffer of one element in shared memory: position of point (i, j, k). For NP = 8
// every k-plane has one row of padding and the position inside a row is XOR-swizzled by
// (j >> 1) | ((k & 1) << 2); then the three access patterns of k_ax (a thread per i-row, a
// thread per j-line, a thread per k-column, 32 consecutive threads covering four rows, lines
// or columns) touch every shared-memory bank equally often, for FP64 and FP32 data.
template <int NP>
struct Stage {
  static constexpr int kPlane = NP == 8 ? 72 : NP * NP;
  static constexpr int kSize = NP * kPlane;
  __device__ static __forceinline__ int at(int i, int j, int k) {
    if constexpr (NP == 8)
      return k * kPlane + j * NP + (i ^ ((j >> 1) | ((k & 1) << 2)));
    else
      return k * kPlane + j * NP + i;
  }
};

// FP32 CG mode with the fused prologue takes the group's p, r, M^-1 and x by TMA bulk copies
// (one per element and array: P floats, a multiple of 16 bytes when NP is even).
template <int NP, typename T, bool CG>
__host__ __device__ constexpr bool ax_tma_in() {
  return CG && sizeof(T) == 4 && (NP * NP * NP) % 4 == 0;
}

// Dynamic shared memory of k_ax: [factors of the element group (STORED only, TMA target)]
// [staging buffers A, B] [p, r, M^-1, x of the group (ax_tma_in only, TMA target)]
// [two mbarriers].
template <int NP, typename T, int GEO, bool CG, int EPB>
__host__ __device__ constexpr size_t ax_smem_bytes() {
  return (GEO != 0 ? 0 : static_cast<size_t>(EPB) * ax_gstride<NP, T>() * sizeof(T)) +
         2 * static_cast<size_t>(EPB) * Stage<NP>::kSize * sizeof(T) +
         (ax_tma_in<NP, T, CG>() ? 4 * static_cast<size_t>(EPB) * NP * NP * NP * sizeof(T) : 0) + 32;
}

// GEO: 0 stored factors, 1 factors recomputed from the element coefficients, 2 recomputed
// with the per-point scale w_i w_j w_k / det J read from memory (one word per point, the
// division moved out of the kernel: Section 5.1's rematerialisation with I/O cost n).
//
// Work of a group of EPB elements; thread t of an element takes i-row (j, k) = (t % NP, t / NP),
// j-line (i, k) = (t % NP, t / NP) and k-column (i, j) = (t % NP, t / NP), each a line of NP
// values that it contracts with D or D^T in registers (even/odd split, see EoMat):
//   0  column of u (or of p = z + beta p) -> registers and buffer A. FP32 CG mode also makes
//      the previous iteration's x update here, x += alpha p (alpha is 0 when none is
//      pending), and forms z = M^-1 r from r and M^-1 instead of reading a stored z: the
//      update kernel then neither reads nor writes x and writes no z (12 of its 33 bytes
//      per point), and this kernel, bound by instruction issue, absorbs the extra loads;
//      for even NP they arrive by TMA bulk copies of the group's p, r, M^-1 and x, issued
//      during the previous group's phases 1-5 (ax_tma_in)
//   1  i-rows of A -> ur into B;               column -> ut (registers)
//   2  j-lines of A -> us, in place in A
//   3  column: (vr, vs, vt) = G (ur, us, ut); vr, vs in place in B, A; vt in registers
//   4  i-rows of B -> D^T vr in place;  j-lines of A -> D^T vs in place;  column -> D^T vt
//   5  column: w = the three sums; stored (CG mode: p.w added, see kWholeDot)
// with a block barrier between phases. Every thread reads and writes only its own line in
// the in-place phases.
template <int NP, typename T, int GEO, bool CG, int EPB>
__global__ void __launch_bounds__(NP * NP * EPB)
    k_ax(const __grid_constant__ GllParam<NP, T> tab, int64_t E, const T* __restrict__ u, T* __restrict__ w,
         const T* __restrict__ G, const T* __restrict__ coef, const T* __restrict__ scale, const T* __restrict__ z,
         T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ minv, T* __restrict__ x,
         CgScalars* __restrict__ st, double* __restrict__ partials, int* __restrict__ err) {
  constexpr bool OTF = GEO != 0;
  // CG mode: FP32 adds p.w over every point as FP32 column sums; FP64 adds the interior
  // points with FP64 multiply-adds and the boundary points in double-float arithmetic
  constexpr bool kWholeDot = sizeof(T) == 4;
  constexpr bool kFused = sizeof(T) == 4;  // the fused CG prologue of phase 0
  constexpr int NP2 = NP * NP, P = NP2 * NP, GS = ax_gstride<NP, T>(), SZ = Stage<NP>::kSize;
  constexpr size_t kG = OTF ? 0 : static_cast<size_t>(EPB) * GS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr bool kTmaIn = ax_tma_in<NP, T, CG>();
  constexpr size_t kIn = kTmaIn ? 4 * static_cast<size_t>(EPB) * P : 0;
  T* sG = reinterpret_cast<T*>(smem_raw);
  T* sA0 = sG + kG;
  T* sB0 = sA0 + EPB * SZ;
  T* sIn = sB0 + EPB * SZ;  // [4][EPB][P]: p, r, M^-1, x (kTmaIn)
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      smem_raw + ((reinterpret_cast<uintptr_t>(sIn + kIn) - reinterpret_cast<uintptr_t>(smem_raw) + 7) &
                  ~uintptr_t(7)));
  uint64_t* bar_in = bar + 1;
  __shared__ double sRed[32];

  T beta = T(0), alpha = T(0);
  if constexpr (CG) {
    if (st->done) return;  // uniform over the grid: set by an earlier launch
    beta = static_cast<T>(st->beta);
    alpha = static_cast<T>(st->alpha);
  }
  const int64_t n_groups = (E + EPB - 1) / EPB;
  constexpr unsigned kElemBytes = static_cast<unsigned>(GS * sizeof(T));
  static_assert(OTF || kElemBytes % 16 == 0, "factor blocks must be whole 16-byte units");
  if constexpr (!OTF) {
    if (threadIdx.x == 0) {  // factors of the first group
      mbar_init(bar, 1);
      const int64_t e0 = static_cast<int64_t>(blockIdx.x) * EPB;
      const int cnt = static_cast<int>(E - e0 < EPB ? E - e0 : EPB);
      fence_proxy_async();
      mbar_expect_tx(bar, kElemBytes * cnt);
      for (int q = 0; q < cnt; ++q) tma_load_1d(sG + q * GS, G + (e0 + q) * GS, kElemBytes, bar);
    }
  }
  // kTmaIn: the copies need 16-byte aligned vectors (the library's own are); else plain loads
  const bool tma_in =
      kTmaIn && ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(x) |
                  reinterpret_cast<uintptr_t>(minv)) & 15u) == 0;
  constexpr unsigned kInBytes = static_cast<unsigned>(P * sizeof(T));
  auto issue_in = [&](int64_t e0, int cnt) {  // thread 0: the group's p, r, M^-1, x
    fence_proxy_async();
    mbar_expect_tx(bar_in, kInBytes * static_cast<unsigned>(cnt) * (minv ? 4u : 3u));
    for (int q = 0; q < cnt; ++q) {
      const int64_t off = (e0 + q) * P;
      tma_load_1d(sIn + (0 * EPB + q) * P, p + off, kInBytes, bar_in);
      tma_load_1d(sIn + (1 * EPB + q) * P, r + off, kInBytes, bar_in);
      if (minv) tma_load_1d(sIn + (2 * EPB + q) * P, minv + off, kInBytes, bar_in);
      tma_load_1d(sIn + (3 * EPB + q) * P, x + off, kInBytes, bar_in);
    }
  };
  if constexpr (kTmaIn) {
    if (tma_in && threadIdx.x == 0) {  // inputs of the first group
      mbar_init(bar_in, 1);
      const int64_t e0 = static_cast<int64_t>(blockIdx.x) * EPB;
      issue_in(e0, static_cast<int>(E - e0 < EPB ? E - e0 : EPB));
    }
  }
  const int slot = threadIdx.x / NP2, tid = threadIdx.x % NP2;
  const int i = tid % NP, j = tid / NP;  // column (i, j); i-row (j, k) = (i, j); j-line (i, k) = (i, j)
  T* sA = sA0 + slot * SZ;
  T* sB = sB0 + slot * SZ;
  DotAcc<T> dot;
  df2 bdot{0.f, 0.f};  // FP64 CG mode: boundary points' part of <p, w>
  unsigned parity = 0, parity_in = 0;
  bool in_pend = tma_in;  // an input copy is in flight (uniform over the block)
  __syncthreads();

  for (int64_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int64_t e = grp * EPB + slot;
    const bool valid = e < E;
    const int64_t base = e * P + tid;
    // phase 0: the column of the input
    T rU[NP];
    if constexpr (CG && kFused) {
      // every load of the column first, so that they are all in flight together (kTmaIn: the
      // group's copies in shared memory)
      T po[NP], rq[NP], xq[NP], mq[NP];
      bool from_smem = false;
      if constexpr (kTmaIn) {
        if (tma_in) {
          const bool ok = mbar_wait_bounded(bar_in, parity_in);
          parity_in ^= 1u;
          in_pend = false;
          if (__syncthreads_or(!ok)) {  // the copies did not arrive: report and leave together
            if (threadIdx.x == 0) {  // first let this block's copies in flight land (bounded)
              mbar_wait_bounded(bar_in, parity_in ^ 1u);
              if constexpr (!OTF) mbar_wait_bounded(bar, parity);  // this group's factors
              atomicExch(err, static_cast<int>(SEM_ERR_TIMEOUT));
              st->status = SEM_ERR_TIMEOUT;
              st->done = 1;
            }
            return;
          }
          from_smem = true;
        }
      }
      if (from_smem) {
        const T* sp = sIn + slot * P + tid;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          po[k] = valid ? sp[0 * EPB * P + k * NP2] : T(0);
          rq[k] = valid ? sp[1 * EPB * P + k * NP2] : T(0);
          mq[k] = valid && minv ? sp[2 * EPB * P + k * NP2] : T(1);
          xq[k] = valid ? sp[3 * EPB * P + k * NP2] : T(0);
        }
      } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const int64_t q = base + k * NP2;
          po[k] = valid ? p[q] : T(0);
          rq[k] = valid ? r[q] : T(0);
          xq[k] = valid ? x[q] : T(0);
          mq[k] = valid && minv ? minv[q] : T(1);
        }
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int64_t q = base + k * NP2;
        const T zq = minv ? mq[k] * rq[k] : rq[k];
        const T val = zq + beta * po[k];
        if (valid) {
          x[q] = xq[k] + alpha * po[k];
          p[q] = val;
        }
        rU[k] = val;
        sA[Stage<NP>::at(i, j, k)] = val;
      }
    } else {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        T val = T(0);
        if (valid) {
          if constexpr (CG) {
            val = z[base + k * NP2] + beta * p[base + k * NP2];
            p[base + k * NP2] = val;
          } else {
            val = u[base + k * NP2];
          }
        }
        rU[k] = val;
        sA[Stage<NP>::at(i, j, k)] = val;
      }
    }
    __syncthreads();
    if constexpr (kTmaIn) {  // the input copies are consumed: the next group's, during phases 1-5
      in_pend = tma_in && grp + gridDim.x < n_groups;
      if (in_pend && threadIdx.x == 0) {
        const int64_t e0 = (grp + gridDim.x) * EPB;
        issue_in(e0, static_cast<int>(E - e0 < EPB ? E - e0 : EPB));
      }
    }

    // phase 1: i-row (j, k) = (i, j) of A -> ur into B; the column -> ut
    T rT[NP];
    {
      T in[NP], out[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(l, i, j)];
      eo_apply<NP, T>(tab.Df, in, out);
#pragma unroll
      for (int l = 0; l < NP; ++l) sB[Stage<NP>::at(l, i, j)] = out[l];
      eo_apply<NP, T>(tab.Df, rU, rT);
    }
    __syncthreads();
    // phase 2: j-line (i, k) = (i, j) of A -> us, in place
    {
      T in[NP], out[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(i, l, j)];
      eo_apply<NP, T>(tab.Df, in, out);
#pragma unroll
      for (int l = 0; l < NP; ++l) sA[Stage<NP>::at(i, l, j)] = out[l];
    }
    if constexpr (!OTF) {
      const bool ok = mbar_wait_bounded(bar, parity);  // this group's factors
      parity ^= 1u;
      if (__syncthreads_or(!ok)) {  // the factor copy did not arrive: report and leave together
        if (threadIdx.x == 0) {  // first let this block's copies in flight land (bounded)
          mbar_wait_bounded(bar, parity ^ 1u);
          if (in_pend) mbar_wait_bounded(bar_in, parity_in);
          atomicExch(err, static_cast<int>(SEM_ERR_TIMEOUT));
          if constexpr (CG) {
            st->status = SEM_ERR_TIMEOUT;
            st->done = 1;
          }
        }
        return;
      }
    } else {
      __syncthreads();
    }

    // phase 3: (vr, vs, vt) = G (ur, us, ut) on the column
    // OTF: the column's cofactor polynomials (a0, the centroid, is not needed)
    OtfColumn<T> geo{};
    T wij = T(0);
    if constexpr (OTF) {
      if (valid) {
        geo.init(coef + e * 24, tab.xi[i], tab.xi[j]);
        wij = tab.w[i] * tab.w[j];
      }
    }
    // (all loads first, then the arithmetic, then the stores: the compiler cannot move a load
    // of the staging buffers above a store to them)
    T rR[NP], rS[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int at = Stage<NP>::at(i, j, k);
      rR[k] = sB[at];
      rS[k] = sA[at];
    }
    constexpr bool kLanes = OTF && std::is_same_v<T, float>;  // FP32: otf_lanes does the column
    if constexpr (kLanes) otf_lanes<NP, GEO>(tab, geo, wij, valid, scale, base, rR, rS, rT);
#pragma unroll
    for (int k = kLanes ? NP : 0; k < NP; ++k) {
      const T ur = rR[k], us = rS[k], ut = rT[k];
      T vr, vs, vt;
      if constexpr (OTF) {
        const T gam = tab.xi[k];
        T sc;
        if constexpr (GEO == 2) {
          sc = valid ? scale[base + k * NP2] : T(0);
        } else {
          sc = valid ? div_fast(wij * tab.w[k], geo.det(gam)) : T(0);
        }
        vr = ur;
        vs = us;
        vt = ut;
        geo.apply(gam, sc, vr, vs, vt);
      } else {
        const T* gp = sG + slot * GS + k * NP2 + tid;
        const T g11 = gp[0 * P], g12 = gp[1 * P], g13 = gp[2 * P], g22 = gp[3 * P], g23 = gp[4 * P],
                g33 = gp[5 * P];
        vr = g11 * ur + g12 * us + g13 * ut;
        vs = g12 * ur + g22 * us + g23 * ut;
        vt = g13 * ur + g23 * us + g33 * ut;
      }
      rR[k] = vr;
      rS[k] = vs;
      rT[k] = vt;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int at = Stage<NP>::at(i, j, k);
      sB[at] = rR[k];
      sA[at] = rS[k];
    }
    __syncthreads();  // the factors are consumed
    if constexpr (!OTF) {
      if (threadIdx.x == 0 && grp + gridDim.x < n_groups) {  // next group's factors, during phases 4-2
        const int64_t e0 = (grp + gridDim.x) * EPB;
        const int cnt = static_cast<int>(E - e0 < EPB ? E - e0 : EPB);
        fence_proxy_async();
        mbar_expect_tx(bar, kElemBytes * cnt);
        for (int q = 0; q < cnt; ++q) tma_load_1d(sG + q * GS, G + (e0 + q) * GS, kElemBytes, bar);
      }
    }

    // phase 4: D^T on i-rows of B and j-lines of A (in place) and on the column
    T rW[NP];
    {
      T inR[NP], inS[NP], outR[NP], outS[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        inR[l] = sB[Stage<NP>::at(l, i, j)];
        inS[l] = sA[Stage<NP>::at(i, l, j)];
      }
      eo_apply<NP, T>(tab.Dt, inR, outR);
      eo_apply<NP, T>(tab.Dt, inS, outS);
      eo_apply<NP, T>(tab.Dt, rT, rW);
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        sB[Stage<NP>::at(l, i, j)] = outR[l];
        sA[Stage<NP>::at(i, l, j)] = outS[l];
      }
    }
    __syncthreads();

    // phase 5: w on the column (FP32 CG mode: the column's part of <p, w> as one multiply-add
    // chain, added to the compensated block sum once per column)
    T col = T(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int at = Stage<NP>::at(i, j, k);
      const T acc = sB[at] + sA[at] + rW[k];
      if constexpr (CG) {
        if (valid) w[kWholeDot ? base + k * NP2 : e * P + cg_pos(NP, i, j, k)] = acc;  // FP64: CG layout
        if constexpr (kWholeDot) {
          col = fma(rU[k], acc, col);
        } else {
          const bool interior = i > 0 && i < NP - 1 && j > 0 && j < NP - 1 && k > 0 && k < NP - 1;
          if (valid && interior) {
            dot.add(rU[k], acc);
          } else if (valid) {
            const df2 a = df_from_double(rU[k]), b = df_from_double(acc);
            df_fma_acc(bdot, a.h, a.l, b.h, b.l);
          }
        }
      } else {
        if (valid) w[base + k * NP2] = acc;
      }
    }
    if constexpr (CG && kWholeDot) {
      if (valid) dot.add_sum(col);
    }
    __syncthreads();  // the staging buffers are free for the next group
  }
  if constexpr (CG) {
    const double s = block_sum(dot.value() + (static_cast<double>(bdot.h) + static_cast<double>(bdot.l)), sRed);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

template <int NP, typename T, int GEO, bool CG, int EPB>
int ax_max_blocks() {
  // resident blocks per SM x SMs; computed once (thread-safe static initialisation)
  static const int cached = [] {
    constexpr size_t smem = ax_smem_bytes<NP, T, GEO, CG, EPB>();
    cudaFuncSetAttribute(k_ax<NP, T, GEO, CG, EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax<NP, T, GEO, CG, EPB>, NP * NP * EPB, smem);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }();
  return cached;
}

template <int NP, typename T, int GEO, bool CG, int EPB>
sem_status launch_ax_t(int N, const AxLaunch& a, cudaStream_t s) {
  const int64_t groups = (a.E + EPB - 1) / EPB;
  int grid = ax_max_blocks<NP, T, GEO, CG, EPB>();
  if (grid > kRedMax) grid = kRedMax;
  if (groups < grid) grid = static_cast<int>(groups);
  if (a.grid_out) *a.grid_out = grid;
  const GllParam<NP, T> tab = make_gll_param<NP, T>(N);
  k_ax<NP, T, GEO, CG, EPB><<<grid, NP * NP * EPB, ax_smem_bytes<NP, T, GEO, CG, EPB>(), s>>>(
      tab, a.E, static_cast<const T*>(a.u), static_cast<T*>(a.w), static_cast<const T*>(a.G),
      static_cast<const T*>(a.coef), static_cast<const T*>(a.scale), static_cast<const T*>(a.z),
      static_cast<T*>(a.p), static_cast<const T*>(a.r), static_cast<const T*>(a.minv), static_cast<T*>(a.x), a.st,
      a.partials, a.err);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

template <int NP, typename T, int EPB>
sem_status launch_ax_shape(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  if (v == SEM_AX_OTF)
    return cg ? launch_ax_t<NP, T, 1, true, EPB>(N, a, s) : launch_ax_t<NP, T, 1, false, EPB>(N, a, s);
  return cg ? launch_ax_t<NP, T, 0, true, EPB>(N, a, s) : launch_ax_t<NP, T, 0, false, EPB>(N, a, s);
}

// Dispatch over the block shape, the variant and the mode for one order and precision
// (the per-point-scale variant is compiled with the default block shape only).
inline int device_sm_count() {
  static const int n = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
  }();
  return n;
}

// A mesh with fewer element groups than SMs takes the shape with fewer elements per block
// (if there is one), so that more SMs share its FP64 work.
template <int NP, typename T>
sem_status launch_ax_np(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  if (v == SEM_AX_OTF_SCALE)
    return cg ? launch_ax_t<NP, T, 2, true, ax_epb<NP>()>(N, a, s) : launch_ax_t<NP, T, 2, false, ax_epb<NP>()>(N, a, s);
  const bool few_groups = a.shape == 0 && (a.E + ax_epb<NP>() - 1) / ax_epb<NP>() < device_sm_count();
  if ((a.shape == 1 && ax_epb_alt<NP>() != ax_epb<NP>()) || (few_groups && ax_epb_alt<NP>() < ax_epb<NP>()))
    return launch_ax_shape<NP, T, ax_epb_alt<NP>()>(N, v, cg, a, s);
  return launch_ax_shape<NP, T, ax_epb<NP>()>(N, v, cg, a, s);
}

// Orders LO..HI (points per direction) of one precision; each translation unit compiles a range.
template <typename T, int LO, int HI>
sem_status launch_ax_range(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  if constexpr (LO > HI) {
    return fail(SEM_ERR_UNSUPPORTED, "polynomial order not compiled in");
  } else {
    if (N + 1 == LO) return launch_ax_np<LO, T>(N, v, cg, a, s);
    return launch_ax_range<T, LO + 1, HI>(N, v, cg, a, s);
  }
}

}  // namespace sem
