// FP32 local operator with on-the-fly factors whose six line contractions run on the tensor
// cores (mma.sync m16n8k8, TF32 operands, FP32 accumulation), for N + 1 = 8 points per
// direction. It is one more candidate of the autotuner (block shape choice kTensorShape of
// the on-the-fly FP32 variant), kept only where the tuner measures it faster.
//
// Each contraction of Eq. 4 over one direction is a product of the element's 64 lines (rows)
// with D^T (forward: u_r = D u along i, etc.) or D (transposed: D^T v), i.e. four 16 x 8 x 8
// tiles per element and direction; warp q of the element's four warps takes tile q in every
// direction. TF32 keeps 11 significant bits, so each operand is split into a TF32 high part
// and a TF32 remainder (the "3xTF32" scheme: a_h b_h + a_h b_l + a_l b_h, the a_l b_l term
// dropped), which keeps the product to about 2^-22 relative, within the FP32 operator's
// 2e-6 bound. Phases of an element (128 threads, 4 warps):
//   0  the element's input (CG mode: x += alpha p, z = M^-1 r, p = z + beta p) -> sU
//   1  forward contractions of sU along i, j, k -> sR, sS, sT (tensor cores)
//   2  (vr, vs, vt) = G (ur, us, ut) in place, G rebuilt on the fly (OtfColumn; 64 threads)
//   3  transposed contractions in place: sR <- D^T along i, sS along j, sT along k
//   4  w = sR + sS + sT, stored; CG mode adds p.w to the block's partial of <p, w, c>
// The staging layout at(i, j, k) = 72 k + 8 j + (i ^ (j & 4)) makes the A-fragment loads of
// all three directions conflict-free.
#include <cstring>

#include "k_ax.cuh"

namespace sem {
namespace {

constexpr int kTcNP = 8;
constexpr int kTcThreads = 128;
constexpr int kTcPlane = 72;
constexpr int kTcStage = kTcNP * kTcPlane;  // floats per staged array

__device__ __forceinline__ int tc_at(int i, int j, int k) { return k * kTcPlane + j * kTcNP + (i ^ (j & 4)); }

// D split into TF32 high parts and TF32 remainders (host side), in the lane order of the
// m16n8k8 B fragments: fwd[h][g][t] = D[g][t] (B = D^T: b0 = B[t][g] = D[g][t], b1 = D[g][t + 4]),
// tr[h][g][t] = D[t][g] (B = D).
struct TcTab {
  float fwd_hi[8][8], fwd_lo[8][8];  // [g][c]: D[g][c]
  float tr_hi[8][8], tr_lo[8][8];    // [g][c]: D[c][g]
  float xi[8], w[8];
};

inline float tf32_round(float x) {
  // round to nearest (ties away from zero) at 10 explicit significand bits, as cvt.rna.tf32.f32
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

TcTab make_tc_tab() {
  const GllTable& t = gll_table(kTcNP - 1);
  TcTab r{};
  for (int g = 0; g < 8; ++g)
    for (int c = 0; c < 8; ++c) {
      const float d = static_cast<float>(t.D[g * 8 + c]), dt = static_cast<float>(t.D[c * 8 + g]);
      r.fwd_hi[g][c] = tf32_round(d);
      r.fwd_lo[g][c] = tf32_round(d - r.fwd_hi[g][c]);
      r.tr_hi[g][c] = tf32_round(dt);
      r.tr_lo[g][c] = tf32_round(dt - r.tr_hi[g][c]);
    }
  for (int a = 0; a < 8; ++a) {
    r.xi[a] = static_cast<float>(t.xi[a]);
    r.w[a] = static_cast<float>(t.w[a]);
  }
  return r;
}

__device__ __forceinline__ uint32_t tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// c += a * b, m16n8k8, TF32 inputs, FP32 accumulators
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One 16 x 8 x 8 tile in 3xTF32: c = a (split on the fly) times the split B fragment.
__device__ __forceinline__ void tile_3xtf32(float (&c)[4], const float (&a)[4], uint32_t bh0, uint32_t bh1,
                                            uint32_t bl0, uint32_t bl1) {
  uint32_t ah[4], al[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ah[q] = tf32(a[q]);
    al[q] = tf32(a[q] - __uint_as_float(ah[q]));
  }
  c[0] = c[1] = c[2] = c[3] = 0.f;
  mma_tf32(c, al, bh0, bh1);  // small terms first
  mma_tf32(c, ah, bl0, bl1);
  mma_tf32(c, ah, bh0, bh1);
}

// Tile q of direction d of the staged array s: A-fragment values of lane (g, t) and the points
// its C-fragment values belong to. Direction 0 (i): rows (k, j) = (2q + h, g), columns i;
// direction 1 (j): rows (k, i) = (2q + h, g), columns j; direction 2 (k): rows (j, i) = (2q + h, g),
// columns k (h = 0 for a0/a2/c0/c1, 1 for a1/a3/c2/c3).
template <int D>
__device__ __forceinline__ int tc_pt(int q, int g, int h, int col) {
  if constexpr (D == 0) return tc_at(col, g, 2 * q + h);
  else if constexpr (D == 1) return tc_at(g, col, 2 * q + h);
  else return tc_at(g, 2 * q + h, col);
}

template <int D>
__device__ __forceinline__ void tc_direction(const float* src, float* dst, int q, int g, int t, uint32_t bh0,
                                             uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  const float a[4] = {src[tc_pt<D>(q, g, 0, t)], src[tc_pt<D>(q, g, 1, t)], src[tc_pt<D>(q, g, 0, t + 4)],
                      src[tc_pt<D>(q, g, 1, t + 4)]};
  float c[4];
  tile_3xtf32(c, a, bh0, bh1, bl0, bl1);
  __syncwarp();  // in place (dst == src): every lane has read its A values before any store
  dst[tc_pt<D>(q, g, 0, 2 * t)] = c[0];
  dst[tc_pt<D>(q, g, 0, 2 * t + 1)] = c[1];
  dst[tc_pt<D>(q, g, 1, 2 * t)] = c[2];
  dst[tc_pt<D>(q, g, 1, 2 * t + 1)] = c[3];
}

template <bool CG>
__global__ void __launch_bounds__(kTcThreads)
    k_ax_tc(const __grid_constant__ TcTab tab, int64_t E, const float* __restrict__ u, float* __restrict__ w,
            const float* __restrict__ coef, float* __restrict__ p, const float* __restrict__ r,
            const float* __restrict__ minv, float* __restrict__ x, CgScalars* __restrict__ st,
            double* __restrict__ partials) {
  constexpr int P = 512;
  __shared__ __align__(16) float sU[kTcStage], sR[kTcStage], sS[kTcStage], sT[kTcStage];
  __shared__ double sRed[kTcThreads / 32];
  float beta = 0.f, alpha = 0.f;
  if constexpr (CG) {
    if (st->done) return;
    beta = static_cast<float>(st->beta);
    alpha = static_cast<float>(st->alpha);
  }
  const int tid = threadIdx.x, lane = tid & 31, q = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  // B fragments (constant over the kernel): forward B = D^T, transposed B = D
  const uint32_t fh0 = __float_as_uint(tab.fwd_hi[g][t]), fh1 = __float_as_uint(tab.fwd_hi[g][t + 4]);
  const uint32_t fl0 = __float_as_uint(tab.fwd_lo[g][t]), fl1 = __float_as_uint(tab.fwd_lo[g][t + 4]);
  const uint32_t th0 = __float_as_uint(tab.tr_hi[g][t]), th1 = __float_as_uint(tab.tr_hi[g][t + 4]);
  const uint32_t tl0 = __float_as_uint(tab.tr_lo[g][t]), tl1 = __float_as_uint(tab.tr_lo[g][t + 4]);
  // this thread's four points in phases 0 and 4: (i0 .. i0 + 3, j4, k4)
  const int k4 = tid >> 4, j4 = (tid >> 1) & 7, i0 = (tid & 1) * 4;
  const int at4 = tc_at(i0, j4, k4);  // i0 .. i0 + 3 stay consecutive and in order (the swizzle flips bit 2)
  DotAcc<float> dot;
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const int64_t base = e * P + 4 * tid;
    float4 pv;  // the element's input at this thread's points (CG mode: the new p)
    if constexpr (CG) {
      const float4 po = *reinterpret_cast<const float4*>(p + base);
      const float4 rq = *reinterpret_cast<const float4*>(r + base);
      const float4 xq = *reinterpret_cast<const float4*>(x + base);
      const float4 mq = minv ? *reinterpret_cast<const float4*>(minv + base) : make_float4(1.f, 1.f, 1.f, 1.f);
      const float zx = minv ? mq.x * rq.x : rq.x, zy = minv ? mq.y * rq.y : rq.y;
      const float zz = minv ? mq.z * rq.z : rq.z, zw = minv ? mq.w * rq.w : rq.w;
      pv = make_float4(zx + beta * po.x, zy + beta * po.y, zz + beta * po.z, zw + beta * po.w);
      *reinterpret_cast<float4*>(x + base) =
          make_float4(xq.x + alpha * po.x, xq.y + alpha * po.y, xq.z + alpha * po.z, xq.w + alpha * po.w);
      *reinterpret_cast<float4*>(p + base) = pv;
    } else {
      pv = *reinterpret_cast<const float4*>(u + base);
    }
    *reinterpret_cast<float4*>(sU + at4) = pv;
    __syncthreads();
    // phase 1: forward contractions, tile q of each direction
    tc_direction<0>(sU, sR, q, g, t, fh0, fh1, fl0, fl1);
    tc_direction<1>(sU, sS, q, g, t, fh0, fh1, fl0, fl1);
    tc_direction<2>(sU, sT, q, g, t, fh0, fh1, fl0, fl1);
    __syncthreads();
    // phase 2: geometric factors on the fly, one thread per k-column (i, j)
    if (tid < 64) {
      const int i = tid & 7, j = tid >> 3;
      OtfColumn<float> geo;
      geo.init(coef + e * 24, tab.xi[i], tab.xi[j]);
      const float wij = tab.w[i] * tab.w[j];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int a = tc_at(i, j, k);
        float ur = sR[a], us = sS[a], ut = sT[a];
        const float gam = tab.xi[k];
        geo.apply(gam, __fdividef(wij * tab.w[k], geo.det(gam)), ur, us, ut);
        sR[a] = ur;
        sS[a] = us;
        sT[a] = ut;
      }
    }
    __syncthreads();
    // phase 3: transposed contractions in place (each warp reads and writes only its own tiles)
    tc_direction<0>(sR, sR, q, g, t, th0, th1, tl0, tl1);
    tc_direction<1>(sS, sS, q, g, t, th0, th1, tl0, tl1);
    tc_direction<2>(sT, sT, q, g, t, th0, th1, tl0, tl1);
    __syncthreads();
    // phase 4: w = the three sums at this thread's four points
    float4 a = *reinterpret_cast<const float4*>(sR + at4);
    const float4 b = *reinterpret_cast<const float4*>(sS + at4);
    const float4 c = *reinterpret_cast<const float4*>(sT + at4);
    a = make_float4(a.x + b.x + c.x, a.y + b.y + c.y, a.z + b.z + c.z, a.w + b.w + c.w);
    const float4 wv = a;
    *reinterpret_cast<float4*>(w + base) = wv;
    if constexpr (CG) {
      float col = pv.x * wv.x;
      col = fmaf(pv.y, wv.y, col);
      col = fmaf(pv.z, wv.z, col);
      col = fmaf(pv.w, wv.w, col);
      dot.add_sum(col);
    }
    // the next element's phase 0 writes sU only; its phase 1 (which overwrites sR, sS, sT) comes
    // after a barrier that every thread reaches once it has finished this phase
  }
  if constexpr (CG) {
    const double s = block_sum(dot.value(), sRed);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

template <bool CG>
int tc_grid(int64_t E) {
  static const int cap = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_tc<CG>, kTcThreads, 0);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }();
  int grid = cap < kRedMax ? cap : kRedMax;
  return E < grid ? static_cast<int>(E) : grid;
}

}  // namespace

bool ax_tensor_available(int N, sem_prec prec, sem_ax_variant v) {
  return N + 1 == kTcNP && prec == SEM_F32 && v == SEM_AX_OTF;
}

sem_status launch_ax_tc(int N, bool cg_mode, const AxLaunch& a, cudaStream_t s) {
  if (N + 1 != kTcNP) return fail(SEM_ERR_UNSUPPORTED, "the tensor-core operator is compiled for N = 7 only");
  static const TcTab tab = make_tc_tab();
  const uintptr_t al = reinterpret_cast<uintptr_t>(a.u) | reinterpret_cast<uintptr_t>(a.w) |
                       reinterpret_cast<uintptr_t>(a.p) | reinterpret_cast<uintptr_t>(a.r) |
                       reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.minv);
  if (al & 15u) return fail(SEM_ERR_ARG, "the tensor-core operator needs 16-byte aligned vectors");
  const float* coef = static_cast<const float*>(a.coef);
  if (cg_mode) {
    const int grid = tc_grid<true>(a.E);
    if (a.grid_out) *a.grid_out = grid;
    k_ax_tc<true><<<grid, kTcThreads, 0, s>>>(tab, a.E, nullptr, static_cast<float*>(a.w), coef,
                                               static_cast<float*>(a.p), static_cast<const float*>(a.r),
                                               static_cast<const float*>(a.minv), static_cast<float*>(a.x), a.st,
                                               a.partials);
  } else {
    const int grid = tc_grid<false>(a.E);
    if (a.grid_out) *a.grid_out = grid;
    k_ax_tc<false><<<grid, kTcThreads, 0, s>>>(tab, a.E, static_cast<const float*>(a.u), static_cast<float*>(a.w),
                                                coef, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  }
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
