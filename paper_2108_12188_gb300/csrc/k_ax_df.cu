// Local operator A_L = D^T G D (Eq. 4, Section 3.1) for FP64 data with stored FP64 factors,
// computed in double-float arithmetic on the FP32 pipes (k_df.cuh): GB300 issues FP32
// FMAs 61 times faster than FP64 ones, and the FP64 kernel is bound by the FP64 pipe.
//
// Same decomposition as k_ax: thread (i, j) of an element owns the column (i, j, 0..NP-1);
// the element's field and the weighted derivatives vr, vs are staged in shared memory as
// (h, l) float pairs; the k-direction stays in registers. Each contraction forms its
// error-free products first and adds them with a pairwise two-sum tree.
//
// The six factor arrays of an element are one contiguous 24 KB block (N = 7): a bulk TMA
// copy brings the next element group's block into shared memory while the current group
// runs its transposed contractions, so the FP32 pipes do not wait on factor loads.
//
// CG mode (Algorithm 1 steps 5-6): p = z + beta p in FP64 (one FMA per point), stored, and
// the element-interior part of <p, w> accumulated in double-float.
#include "k_ax.cuh"
#include "k_df.cuh"
#include "k_tma.cuh"

namespace sem {
namespace {

template <int NP>
struct DfTab {
  float Dh[NP * NP];  // D[a*NP + b] = Dh + Dl
  float Dl[NP * NP];
};

template <int NP>
DfTab<NP> make_df_tab(int N) {
  const GllTable& t = gll_table(N);
  DfTab<NP> d;
  for (int a = 0; a < NP * NP; ++a) {
    const double v = t.D[a];
    d.Dh[a] = static_cast<float>(v);
    d.Dl[a] = static_cast<float>(v - static_cast<double>(d.Dh[a]));
  }
  return d;
}

template <int NP>
constexpr size_t df_smem_bytes() {
  constexpr int P = NP * NP * NP, EPB = ax_epb<NP>();
  return static_cast<size_t>(EPB) * 6 * P * sizeof(double)  // factors of the element group (TMA target)
         + 3 * static_cast<size_t>(EPB) * P * sizeof(df2)     // u, vr, vs as float pairs
         + 2 * NP * NP * sizeof(float) + 16;                  // D split, mbarrier
}

// Copies the factors of the element group starting at element e0 (count elements, each a
// contiguous [6][P] FP64 block) into sG; one thread announces the bytes and issues the copies.
template <int NP>
__device__ __forceinline__ void prefetch_factors(double* sG, const double* G, int64_t e0, int count, uint64_t* bar) {
  constexpr int P = NP * NP * NP;
  constexpr unsigned kElemBytes = 6u * P * sizeof(double);
  fence_proxy_async();
  mbar_expect_tx(bar, kElemBytes * static_cast<unsigned>(count));
  for (int q = 0; q < count; ++q) tma_load_1d(sG + q * 6 * P, G + (e0 + q) * 6 * P, kElemBytes, bar);
}

template <int NP, bool CG>
__global__ void __launch_bounds__(NP * NP * ax_epb<NP>())
    k_ax_df(const __grid_constant__ DfTab<NP> tab, int64_t E, const double* __restrict__ u, double* __restrict__ w,
            const double* __restrict__ G, const double* __restrict__ z, double* __restrict__ p,
            CgScalars* __restrict__ st, double* __restrict__ partials, int* __restrict__ err) {
  constexpr int NP2 = NP * NP, P = NP2 * NP, EPB = ax_epb<NP>();
  extern __shared__ __align__(128) unsigned char smem[];
  double* sG = reinterpret_cast<double*>(smem);
  df2* sU = reinterpret_cast<df2*>(sG + EPB * 6 * P);
  df2* sR = sU + EPB * P;
  df2* sS = sR + EPB * P;
  float* sDh = reinterpret_cast<float*>(sS + EPB * P);
  float* sDl = sDh + NP2;
  // byte offset of sDl + NP2 is EPB*6*P*8 + 3*EPB*P*8 + 8*NP2: a multiple of 8, as the mbarrier needs
  uint64_t* bar = reinterpret_cast<uint64_t*>(sDl + NP2);
  __shared__ double sRed[32];

  double beta = 0.0;
  if constexpr (CG) {
    if (st->done) return;
    beta = st->beta;
  }
  for (int q = threadIdx.x; q < NP2; q += blockDim.x) {
    sDh[q] = tab.Dh[q];
    sDl[q] = tab.Dl[q];
  }
  const int64_t n_groups = (E + EPB - 1) / EPB;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    const int64_t e0 = static_cast<int64_t>(blockIdx.x) * EPB;
    prefetch_factors<NP>(sG, G, e0, static_cast<int>(E - e0 < EPB ? E - e0 : EPB), bar);
  }
  const int slot = threadIdx.x / NP2, tid = threadIdx.x % NP2;
  const int i = tid % NP, j = tid / NP;
  df2 dot{0.f, 0.f};
  unsigned parity = 0;
  __syncthreads();

  for (int64_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int64_t e = grp * EPB + slot;
    const bool valid = e < E;
    const int64_t base = e * P + tid;
    df2 rU[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      double val = 0.0;
      if (valid) {
        if constexpr (CG) {
          val = fma(beta, p[base + k * NP2], z[base + k * NP2]);
          p[base + k * NP2] = val;
        } else {
          val = u[base + k * NP2];
        }
      }
      rU[k] = df_from_double(val);
      sU[slot * P + k * NP2 + tid] = rU[k];
    }
    const bool ok = mbar_wait_bounded(bar, parity);
    parity ^= 1u;
    if (__syncthreads_or(!ok)) {  // the factor copy did not arrive: report and leave together
      if (threadIdx.x == 0) {
        mbar_wait_bounded(bar, parity ^ 1u);  // give the copy in flight one more bounded wait
        atomicExch(err, static_cast<int>(SEM_ERR_TIMEOUT));
        if constexpr (CG) {
          st->status = SEM_ERR_TIMEOUT;
          st->done = 1;
        }
      }
      return;
    }

    const double* gE = sG + slot * 6 * P;
    df2 rT[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      float pr[NP], er[NP], ps[NP], es[NP], pt[NP], et[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        const df2 a = sU[slot * P + k * NP2 + j * NP + l];
        const df2 b = sU[slot * P + k * NP2 + l * NP + i];
        df_prod(sDh[i * NP + l], sDl[i * NP + l], a.h, a.l, pr[l], er[l]);
        df_prod(sDh[j * NP + l], sDl[j * NP + l], b.h, b.l, ps[l], es[l]);
        df_prod(tab.Dh[k * NP + l], tab.Dl[k * NP + l], rU[l].h, rU[l].l, pt[l], et[l]);
      }
      const df2 ur = df_tree_sum<NP>(pr, er);
      const df2 us = df_tree_sum<NP>(ps, es);
      const df2 ut = df_tree_sum<NP>(pt, et);
      df2 g[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) g[m] = df_from_double(gE[m * P + k * NP2 + tid]);
      float p3[3], e3[3];
      df_prod(g[0].h, g[0].l, ur.h, ur.l, p3[0], e3[0]);
      df_prod(g[1].h, g[1].l, us.h, us.l, p3[1], e3[1]);
      df_prod(g[2].h, g[2].l, ut.h, ut.l, p3[2], e3[2]);
      sR[slot * P + k * NP2 + tid] = df_tree_sum<3>(p3, e3);
      df_prod(g[1].h, g[1].l, ur.h, ur.l, p3[0], e3[0]);
      df_prod(g[3].h, g[3].l, us.h, us.l, p3[1], e3[1]);
      df_prod(g[4].h, g[4].l, ut.h, ut.l, p3[2], e3[2]);
      sS[slot * P + k * NP2 + tid] = df_tree_sum<3>(p3, e3);
      df_prod(g[2].h, g[2].l, ur.h, ur.l, p3[0], e3[0]);
      df_prod(g[4].h, g[4].l, us.h, us.l, p3[1], e3[1]);
      df_prod(g[5].h, g[5].l, ut.h, ut.l, p3[2], e3[2]);
      rT[k] = df_tree_sum<3>(p3, e3);
    }
    __syncthreads();  // sG and sU consumed; sR, sS complete
    if (threadIdx.x == 0 && grp + gridDim.x < n_groups) {
      const int64_t e0 = (grp + gridDim.x) * EPB;
      prefetch_factors<NP>(sG, G, e0, static_cast<int>(E - e0 < EPB ? E - e0 : EPB), bar);
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      float pr[NP], er[NP], ps[NP], es[NP], pt[NP], et[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        const df2 a = sR[slot * P + k * NP2 + j * NP + l];
        const df2 b = sS[slot * P + k * NP2 + l * NP + i];
        df_prod(sDh[l * NP + i], sDl[l * NP + i], a.h, a.l, pr[l], er[l]);
        df_prod(sDh[l * NP + j], sDl[l * NP + j], b.h, b.l, ps[l], es[l]);
        df_prod(tab.Dh[l * NP + k], tab.Dl[l * NP + k], rT[l].h, rT[l].l, pt[l], et[l]);
      }
      const df2 wr = df_tree_sum<NP>(pr, er);
      const df2 ws = df_tree_sum<NP>(ps, es);
      const df2 wt = df_tree_sum<NP>(pt, et);
      const df2 acc = df_add(df_add(wr, ws), wt);
      if (valid) w[base + k * NP2] = df_to_double(acc);
      if constexpr (CG) {
        const bool interior = i > 0 && i < NP - 1 && j > 0 && j < NP - 1 && k > 0 && k < NP - 1;
        if (valid && interior) df_fma_acc(dot, rU[k].h, rU[k].l, acc.h, acc.l);
      }
    }
  }
  if constexpr (CG) {
    const double s = block_sum(static_cast<double>(dot.h) + static_cast<double>(dot.l), sRed);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

template <int NP, bool CG>
sem_status launch_df_t(int N, const AxLaunch& a, cudaStream_t s) {
  constexpr int EPB = ax_epb<NP>();
  constexpr size_t smem = df_smem_bytes<NP>();
  // resident blocks per SM x SMs, with the dynamic shared-memory limit raised first; once
  static const int max_blocks = [] {
    cudaFuncSetAttribute(k_ax_df<NP, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_df<NP, CG>, NP * NP * EPB, smem);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }();
  const int64_t groups = (a.E + EPB - 1) / EPB;
  int grid = max_blocks < kRedMax ? max_blocks : kRedMax;
  if (groups < grid) grid = static_cast<int>(groups);
  if (a.grid_out) *a.grid_out = grid;
  k_ax_df<NP, CG><<<grid, NP * NP * EPB, smem, s>>>(make_df_tab<NP>(N), a.E, static_cast<const double*>(a.u),
                                                     static_cast<double*>(a.w), static_cast<const double*>(a.G),
                                                     static_cast<const double*>(a.z), static_cast<double*>(a.p),
                                                     a.st, a.partials, a.err);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

template <int NP>
sem_status launch_df_np(int N, bool cg, const AxLaunch& a, cudaStream_t s) {
  return cg ? launch_df_t<NP, true>(N, a, s) : launch_df_t<NP, false>(N, a, s);
}

}  // namespace

sem_status launch_ax_f64x(int N, sem_ax_variant v, bool cg, const AxLaunch& a, cudaStream_t s) {
  if (v != SEM_AX_STORED) return fail(SEM_ERR_UNSUPPORTED, "SEM_F64X runs the stored-factor variant only");
  switch (N + 1) {
    case 2: return launch_df_np<2>(N, cg, a, s);
    case 3: return launch_df_np<3>(N, cg, a, s);
    case 4: return launch_df_np<4>(N, cg, a, s);
    case 5: return launch_df_np<5>(N, cg, a, s);
    case 6: return launch_df_np<6>(N, cg, a, s);
    case 7: return launch_df_np<7>(N, cg, a, s);
    case 8: return launch_df_np<8>(N, cg, a, s);
    case 9: return launch_df_np<9>(N, cg, a, s);
    case 10: return launch_df_np<10>(N, cg, a, s);
    case 11: return launch_df_np<11>(N, cg, a, s);
    case 12: return launch_df_np<12>(N, cg, a, s);
    default: return fail(SEM_ERR_UNSUPPORTED, "polynomial order not compiled in");
  }
}

}  // namespace sem
