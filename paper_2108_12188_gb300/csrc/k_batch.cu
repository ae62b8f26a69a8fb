// Batched conjugate-gradient kernels: many independent FP32 CG solves (the inner iteration
// of mixed-precision refinement with on-the-fly geometric factors) advance together, each
// launch striding over the work items of every solve in a device-side table (BatchTable).
// One iteration of Algorithm 1 for the whole table is an operator launch per polynomial order
// present, one gather-scatter launch and one update launch; a flush launch adds the pending
// x updates when a run of iterations ends.
//
// A work item covers a fixed part of one solve: an element group (operator), a chunk of
// kBatchGsSeg segments of one record class (gather-scatter), a chunk of kBatchChunk points
// (update, flush). Its partial sums go to that solve's own arrays, indexed by the item, and
// the item that completes a solve's last part (per-solve ticket) forms the solve's scalars
// from the partials in index order. So a solve's arithmetic is the same whatever else is in
// the table and however many blocks run: results are bit-identical alone and in any mix.
//
// The per-solve arithmetic is that of the single-mesh FP32 CG (k_ax CG mode with the fused
// prologue, k_dssum_cg without the dot, the fused k_cg_update, k_cg_flush): Algorithm 1
// steps 5-13 with z = M^-1 r, the x update one iteration late, <p, w, c> accumulated over the
// unassembled w, compensated float dots combined in FP64.
#include "k_ax.cuh"
#include "k_gs.cuh"

namespace sem {
namespace {

// Operator work items of order NP: the element groups of the solves in table entries
// [s_lo, s_hi), in table order. Each block visits its items in ascending order, so the
// solve index only moves forward.
template <int NP, int EPB>
__global__ void __launch_bounds__(NP * NP * EPB)
    k_ax_batch(const __grid_constant__ GllParam<NP, float> tab, const BatchTable* __restrict__ T) {
  using F = float;
  constexpr int NP2 = NP * NP, P = NP2 * NP, SZ = Stage<NP>::kSize;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sRed[32];
  F* sA0 = reinterpret_cast<F*>(smem_raw);
  F* sB0 = sA0 + EPB * SZ;
  const BatchOrder ord = T->order[NP];
  const int slot = threadIdx.x / NP2, tid = threadIdx.x % NP2;
  const int i = tid % NP, j = tid / NP;  // column (i, j); i-row (j, k) = (i, j); j-line (i, k) = (i, j)
  F* sA = sA0 + slot * SZ;
  F* sB = sB0 + slot * SZ;
  int sv = ord.s_lo;
  for (int64_t q = blockIdx.x; q < ord.items; q += gridDim.x) {
    while (q >= T->s[sv].ax_beg + T->s[sv].ax_cnt) ++sv;
    const BatchSolve* d = &T->s[sv];
    CgScalars* st = d->st;
    if (st->done) continue;  // the same for every thread of the block
    const F beta = static_cast<F>(st->beta), alpha = static_cast<F>(st->alpha);
    const int64_t grp = q - d->ax_beg;
    const int64_t e = grp * EPB + slot;
    const bool valid = e < d->E;
    const int64_t base = e * P + tid;
    F* __restrict__ p = d->p;
    F* __restrict__ x = d->x;
    const F* __restrict__ r = d->r;
    const F* __restrict__ minv = d->minv;
    // phase 0: the deferred x += alpha p, z = M^-1 r and p = z + beta p on the column; all
    // loads of the column first
    F rU[NP];
    {
      F po[NP], rq[NP], xq[NP], mq[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int64_t qq = base + k * NP2;
        po[k] = valid ? p[qq] : F(0);
        rq[k] = valid ? r[qq] : F(0);
        xq[k] = valid ? x[qq] : F(0);
        mq[k] = valid && minv ? minv[qq] : F(1);
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int64_t qq = base + k * NP2;
        const F zq = minv ? mq[k] * rq[k] : rq[k];
        const F val = zq + beta * po[k];
        if (valid) {
          x[qq] = xq[k] + alpha * po[k];
          p[qq] = val;
        }
        rU[k] = val;
        sA[Stage<NP>::at(i, j, k)] = val;
      }
    }
    __syncthreads();
    // phase 1: i-row of A -> ur into B; the column -> ut
    F rT[NP];
    {
      F in[NP], out[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(l, i, j)];
      eo_apply<NP, F>(tab.Df, in, out);
#pragma unroll
      for (int l = 0; l < NP; ++l) sB[Stage<NP>::at(l, i, j)] = out[l];
      eo_apply<NP, F>(tab.Df, rU, rT);
    }
    __syncthreads();
    // phase 2: j-line of A -> us, in place
    {
      F in[NP], out[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(i, l, j)];
      eo_apply<NP, F>(tab.Df, in, out);
#pragma unroll
      for (int l = 0; l < NP; ++l) sA[Stage<NP>::at(i, l, j)] = out[l];
    }
    __syncthreads();
    // phase 3: (vr, vs, vt) = G (ur, us, ut) with G rebuilt from the element's coefficients:
    // G v = (w_i w_j w_k / det J) C (C^T v), C the cofactor rows of J (OtfColumn)
    OtfColumn<F> geo{};
    F wij = F(0);
    if (valid) {
      geo.init(d->coef + e * 24, tab.xi[i], tab.xi[j]);
      wij = tab.w[i] * tab.w[j];
    }
    F rR[NP], rS[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int at = Stage<NP>::at(i, j, k);
      rR[k] = sB[at];
      rS[k] = sA[at];
    }
    otf_lanes<NP, 1>(tab, geo, wij, valid, nullptr, base, rR, rS, rT);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int at = Stage<NP>::at(i, j, k);
      sB[at] = rR[k];
      sA[at] = rS[k];
    }
    __syncthreads();
    // phase 4: D^T on i-rows of B and j-lines of A (in place) and on the column
    F rW[NP];
    {
      F inR[NP], inS[NP], outR[NP], outS[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        inR[l] = sB[Stage<NP>::at(l, i, j)];
        inS[l] = sA[Stage<NP>::at(i, l, j)];
      }
      eo_apply<NP, F>(tab.Dt, inR, outR);
      eo_apply<NP, F>(tab.Dt, inS, outS);
      eo_apply<NP, F>(tab.Dt, rT, rW);
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        sB[Stage<NP>::at(l, i, j)] = outR[l];
        sA[Stage<NP>::at(i, l, j)] = outS[l];
      }
    }
    __syncthreads();
    // phase 5: w on the column, and this group's part of <p, w> (over every point; the column
    // as one multiply-add chain, added to a compensated sum)
    DotAcc<F> dot;
    F* __restrict__ w = d->w;
    F col = F(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int at = Stage<NP>::at(i, j, k);
      const F acc = sB[at] + sA[at] + rW[k];
      if (valid) w[base + k * NP2] = acc;
      col = fmaf(rU[k], acc, col);
    }
    if (valid) dot.add_sum(col);
    // (block_sum's barriers also keep the staging buffers until every thread has read them)
    const double s = block_sum(dot.value(), sRed);
    if (threadIdx.x == 0) d->ax_part[grp] = s;
  }
}

// Segments [lo, lo + kBatchGsSeg) of a fixed-width class (n segments), kBatchGsSeg /
// kBatchThreads per thread; each segment's record and then all its copies are loaded before
// the sum.
template <int W>
__device__ __forceinline__ void gs_chunk(const int32_t* __restrict__ rec, const uint8_t* __restrict__ msk, int64_t lo,
                                         int64_t n, float* __restrict__ w) {
#pragma unroll 1
  for (int64_t sg = lo + threadIdx.x; sg < lo + kBatchGsSeg && sg < n; sg += kBatchThreads) {
    int a[W];
    float va[W];
    load_rec<W>(rec, sg, a);
    const bool masked = msk[sg] != 0;
    seg_load<W>(w, a, va);
    seg_store<W>(w, a, masked ? 0.f : seg_add<W>(a, va));
  }
}

// Algorithm 1 step 7 (QQ^T and the mask) for every solve; the item that completes a solve
// forms <p, w, c> from the operator's group partials and alpha = rho / <p, w, c> (step 8).
__global__ void __launch_bounds__(kBatchThreads) k_gs_batch(const BatchTable* __restrict__ T) {
  __shared__ double sRed[kBatchThreads / 32];
  __shared__ bool last;
  const int64_t items = T->gs_items;
  int sv = 0;
  for (int64_t q = blockIdx.x; q < items; q += gridDim.x) {
    while (q >= T->s[sv].gs_beg + T->s[sv].gs_at[5]) ++sv;
    const BatchSolve* d = &T->s[sv];
    CgScalars* st = d->st;
    if (st->done) continue;
    const int64_t l = q - d->gs_beg;
    int c = 0;
    while (l >= d->gs_at[c + 1]) ++c;
    const int64_t lo = (l - d->gs_at[c]) * kBatchGsSeg;
    const GsPlan& g = d->gs;
    float* w = d->w;
    switch (c) {
      case 0: gs_chunk<2>(g.rec[1], g.msk[1], lo, g.n[1], w); break;
      case 1: gs_chunk<4>(g.rec[2], g.msk[2], lo, g.n[2], w); break;
      case 2: gs_chunk<8>(g.rec[3], g.msk[3], lo, g.n[3], w); break;
      case 3: gs_chunk<1>(g.rec[0], g.msk[0], lo, g.n[0], w); break;
      default: {
        const int64_t hi = lo + kBatchGsSeg < g.nx ? lo + kBatchGsSeg : g.nx;
        for (int64_t x = lo + threadIdx.x; x < hi; x += kBatchThreads) {
          const int o0 = g.xoff[x], o1 = g.xoff[x + 1];
          float s = w[g.xidx[o0]];
          for (int o = o0 + 1; o < o1; ++o) s += w[g.xidx[o]];
          if (g.xmsk[x]) s = 0.f;
          for (int o = o0; o < o1; ++o) w[g.xidx[o]] = s;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(&st->ticket[0], 1u);
      last = t == static_cast<unsigned>(d->gs_at[5] - 1);
      if (last) st->ticket[0] = 0u;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const double pw = sum_partials(d->ax_part, static_cast<int>(d->ax_cnt), 1, 0, sRed);
      if (threadIdx.x == 0) {
        st->pw = pw;
        if (!(pw > 0.0) || !isfinite(pw)) {
          st->status = SEM_ERR_BREAKDOWN;
          st->done = 1;
          st->alpha = 0.0;
        } else {
          st->alpha = st->rho / pw;
        }
      }
    }
  }
}

// Algorithm 1 steps 9-13 (x deferred to the next operator prologue): r -= alpha w, z = M^-1 r,
// partials of <r, z, c> and <r, r, c> per chunk; the item that completes a solve forms rho,
// beta, the iteration count and the stopping decision.
__global__ void __launch_bounds__(kBatchThreads) k_update_batch(const BatchTable* __restrict__ T) {
  __shared__ double sRed[kBatchThreads / 32];
  __shared__ bool last;
  const int64_t items = T->up_items;
  int sv = 0;
  for (int64_t q = blockIdx.x; q < items; q += gridDim.x) {
    while (q >= T->s[sv].up_beg + T->s[sv].up_cnt) ++sv;
    const BatchSolve* d = &T->s[sv];
    CgScalars* st = d->st;
    if (st->done) continue;
    const float alpha = static_cast<float>(st->alpha);
    const int64_t c = q - d->up_beg;
    const int64_t lo = c * kBatchChunk;
    const int64_t hi = lo + kBatchChunk < d->n ? lo + kBatchChunk : d->n;
    float* __restrict__ r = d->r;
    const float* __restrict__ w = d->w;
    const float* __restrict__ minv = d->minv;
    const uint8_t* __restrict__ mult = d->mult;
    const double* __restrict__ ctab = d->ctab;
    DotAcc<float> rz, rr;
    auto point = [&](float& ri, float wi, float mi, unsigned m) {
      ri = ri - alpha * wi;
      const float zi = minv ? mi * ri : ri;
      const float cw = m == 1u ? 1.f : static_cast<float>(__ldg(ctab + m));
      rz.add(ri, cw * zi);
      rr.add(ri, cw * ri);
    };
    if (hi - lo == kBatchChunk) {  // a whole chunk: four 16-byte steps per thread, all loads first
      constexpr int K = kBatchChunk / 4 / kBatchThreads;
      float4 rv[K], wv[K], mv[K];
      uchar4 cv[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int64_t v = lo / 4 + threadIdx.x + k * kBatchThreads;
        rv[k] = reinterpret_cast<const float4*>(r)[v];
        wv[k] = reinterpret_cast<const float4*>(w)[v];
        mv[k] = minv ? reinterpret_cast<const float4*>(minv)[v] : make_float4(1.f, 1.f, 1.f, 1.f);
        cv[k] = reinterpret_cast<const uchar4*>(mult)[v];
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        point(rv[k].x, wv[k].x, mv[k].x, cv[k].x);
        point(rv[k].y, wv[k].y, mv[k].y, cv[k].y);
        point(rv[k].z, wv[k].z, mv[k].z, cv[k].z);
        point(rv[k].w, wv[k].w, mv[k].w, cv[k].w);
        reinterpret_cast<float4*>(r)[lo / 4 + threadIdx.x + k * kBatchThreads] = rv[k];
      }
    } else {
      for (int64_t i = lo + threadIdx.x; i < hi; i += kBatchThreads) {
        float ri = r[i];
        point(ri, w[i], minv ? minv[i] : 1.f, mult[i]);
        r[i] = ri;
      }
    }
    const double vz = block_sum(rz.value(), sRed);
    const double vr = block_sum(rr.value(), sRed);
    if (threadIdx.x == 0) {
      d->up_part[2 * c] = vz;
      d->up_part[2 * c + 1] = vr;
      __threadfence();
      const unsigned t = atomicAdd(&st->ticket[1], 1u);
      last = t == static_cast<unsigned>(d->up_cnt - 1);
      if (last) st->ticket[1] = 0u;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const int cnt = static_cast<int>(d->up_cnt);
      const double srz = sum_partials(d->up_part, cnt, 2, 0, sRed);
      const double srr = sum_partials(d->up_part, cnt, 2, 1, sRed);
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
}

// x += alpha p for every solve with an update pending (alpha != 0); the item that completes a
// solve sets its alpha to 0. Solves that are done are flushed too (their last update).
__global__ void __launch_bounds__(kBatchThreads) k_flush_batch(const BatchTable* __restrict__ T) {
  __shared__ bool last;
  const int64_t items = T->up_items;
  int sv = 0;
  for (int64_t q = blockIdx.x; q < items; q += gridDim.x) {
    while (q >= T->s[sv].up_beg + T->s[sv].up_cnt) ++sv;
    const BatchSolve* d = &T->s[sv];
    CgScalars* st = d->st;
    const double a64 = st->alpha;  // read by every item before the solve's last one clears it
    if (a64 == 0.0) continue;
    const float a = static_cast<float>(a64);
    const int64_t lo = (q - d->up_beg) * kBatchChunk;
    const int64_t hi = lo + kBatchChunk < d->n ? lo + kBatchChunk : d->n;
    float* __restrict__ x = d->x;
    const float* __restrict__ p = d->p;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBatchThreads) x[i] += a * p[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(&st->ticket[4], 1u);
      last = t == static_cast<unsigned>(d->up_cnt - 1);
      if (last) {
        st->ticket[4] = 0u;
        st->alpha = 0.0;
      }
    }
    __syncthreads();
  }
}

__global__ void k_batch_status(const BatchTable* __restrict__ T, int count, CgScalars* __restrict__ out) {
  for (int s = threadIdx.x; s < count; s += blockDim.x) out[s] = *T->s[s].st;
}

template <auto K>
int batch_grid(int threads, size_t smem) {
  static const int cap = [threads, smem] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024) cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K, threads, smem);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }();
  return cap;
}

template <int NP>
sem_status launch_ax_batch_np(const BatchTable* t, cudaStream_t s) {
  constexpr int EPB = ax_epb<NP>();
  constexpr size_t smem = 2 * static_cast<size_t>(EPB) * Stage<NP>::kSize * sizeof(float);
  const int grid = batch_grid<k_ax_batch<NP, EPB>>(NP * NP * EPB, smem);
  const GllParam<NP, float> tab = make_gll_param<NP, float>(NP - 1);
  k_ax_batch<NP, EPB><<<grid, NP * NP * EPB, smem, s>>>(tab, t);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

template <int LO, int HI>
sem_status launch_ax_batch_range(int NP, const BatchTable* t, cudaStream_t s) {
  if constexpr (LO > HI) {
    return fail(SEM_ERR_UNSUPPORTED, "polynomial order not compiled in");
  } else {
    if (NP == LO) return launch_ax_batch_np<LO>(t, s);
    return launch_ax_batch_range<LO + 1, HI>(NP, t, s);
  }
}

template <int LO, int HI>
int epb_range(int NP) {
  if constexpr (LO > HI) {
    return 0;
  } else {
    return NP == LO ? ax_epb<LO>() : epb_range<LO + 1, HI>(NP);
  }
}

}  // namespace

int batch_ax_elements_per_group(int NP) { return epb_range<2, kMaxNp>(NP); }

sem_status launch_batch_ax(int NP, const BatchTable* t, cudaStream_t s) {
  return launch_ax_batch_range<2, kMaxNp>(NP, t, s);
}

sem_status launch_batch_gs(const BatchTable* t, cudaStream_t s) {
  k_gs_batch<<<batch_grid<k_gs_batch>(kBatchThreads, 0), kBatchThreads, 0, s>>>(t);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_batch_update(const BatchTable* t, cudaStream_t s) {
  k_update_batch<<<batch_grid<k_update_batch>(kBatchThreads, 0), kBatchThreads, 0, s>>>(t);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_batch_flush(const BatchTable* t, cudaStream_t s) {
  k_flush_batch<<<batch_grid<k_flush_batch>(kBatchThreads, 0), kBatchThreads, 0, s>>>(t);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

sem_status launch_batch_status(const BatchTable* t, int count, CgScalars* out, cudaStream_t s) {
  if (count <= 0) return SEM_OK;
  k_batch_status<<<1, 128, 0, s>>>(t, count, out);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
