// Local operator A_L = D^T G D (Eq. 4, Section 3.1) for FP64 data, with stored factors or
// factors rebuilt on the fly (Section 5.1), computed in double-float arithmetic on the FP32
// pipes (k_df.cuh): GB300 issues FP32 FMAs 64 times faster than FP64 ones, and the FP64
// kernel is bound by the FP64 pipe. The kernel template is shared by four translation units
// (stored / on the fly, lower / higher orders) that compile in parallel.
//
// Same decomposition as k_ax: thread t of an element contracts whole lines of NP values
// (its i-row, its j-line and its k-column) in registers through the even/odd split of D and
// D^T (EoMat), with the element staged in shared memory as (h, l) float pairs in the
// swizzled layout of Stage. A line costs, per output, about 60 FP32 operations instead of
// about 90 for the plain sums: the even and odd combinations are two-sums, each of the H
// products is error-free, the H terms are added by a pairwise two-sum tree, and the pair
// outputs A + B and B - A are two-sums left unnormalised (the low part may exceed half an ulp
// of the high part; products and sums downstream take such pairs exactly). Each output point
// is renormalised once before it is rounded to FP64.
//
// The six factor arrays of an element are one contiguous block (24 KB at N = 7): a bulk TMA
// copy brings the next element group's first three arrays into shared memory (and a bulk
// prefetch the other three into L2) during the rest of the current group, so the FP32 pipes
// do not wait on factor loads (bounded mbarrier waits; a timeout sets SEM_ERR_TIMEOUT). The factors are FP64 values, split into float pairs by
// integer operations, or (SEM_MESH_F64X_STORED) float pairs already, in the same 8 bytes.
// On the fly (OtfColumnDf), no factor is read: the geometry phase runs point by point through
// a third staging buffer.
//
// CG mode (Algorithm 1 steps 5-6, fused_cg): the previous iteration's x += alpha p, z = M^-1 r
// and p = z + beta p in FP64 (on the FP64 pipe, which this kernel otherwise leaves idle), and
// <p, w> accumulated in double-float over every local point of the unassembled w (equal to
// <p, QQ^T w, c> because p has one value per global node; the gather-scatter reads no p).
#pragma once

#include "k_ax.cuh"
#include "k_df.cuh"
#include "k_tma.cuh"

namespace sem {
namespace {

// Geometric factors the double-float operator takes: FP64 values (split into float pairs in the
// kernel), float pairs stored by the mesh (SEM_MESH_F64X_STORED), or none (rebuilt on the fly
// from the element's trilinear coefficients).
constexpr int kGkF64 = 0, kGkPairs = 1, kGkOtf = 2;

// Even/odd split of D and D^T (EoMat, computed in FP64) with every entry as a float pair.
// For the two-wide FP32 operations of sm_100 and later, the H x H blocks are also kept
// interleaved, (E(i,l), O(i,l)) as one float2: C = high parts, NC and NCL = negated high and
// low parts (eo_apply_df forms the products of both sums at once and carries their error
// terms negated).
template <int NP>
struct DfEo {
  static constexpr int H = NP / 2, HC = (NP + 1) / 2;
  float Eh[H][HC], El[H][HC];
  float Oh[HC][H], Ol[HC][H];
  float2 C[H][H], NC[H][H], NCL[H][H];
};

// On-the-fly geometry: the GLL nodes and weights in FP64 (per-column coefficients) and, per
// column point k, the node as a float pair held in both lanes of float2 values (high part;
// negated high and low parts) and the weight as a float pair.
template <int NP>
struct DfTab {
  DfEo<NP> Df, Dt;
  double xi[NP], w[NP];
  float2 gdh[NP], ngdh[NP], ngdl[NP];
  float wkh[NP], wkl[NP];
};

template <int NP>
DfEo<NP> split_eo(const EoMat<NP, double>& m) {
  constexpr int H = NP / 2, HC = (NP + 1) / 2;
  DfEo<NP> d{};
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < HC; ++b) {
      d.Eh[a][b] = static_cast<float>(m.E[a][b]);
      d.El[a][b] = static_cast<float>(m.E[a][b] - static_cast<double>(d.Eh[a][b]));
    }
  for (int a = 0; a < HC; ++a)
    for (int b = 0; b < H; ++b) {
      d.Oh[a][b] = static_cast<float>(m.O[a][b]);
      d.Ol[a][b] = static_cast<float>(m.O[a][b] - static_cast<double>(d.Oh[a][b]));
    }
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < H; ++b) {
      d.C[a][b] = make_float2(d.Eh[a][b], d.Oh[a][b]);
      d.NC[a][b] = make_float2(-d.Eh[a][b], -d.Oh[a][b]);
      d.NCL[a][b] = make_float2(-d.El[a][b], -d.Ol[a][b]);
    }
  return d;
}

template <int NP>
DfTab<NP> make_df_tab(int N) {
  const GllParam<NP, double> g = make_gll_param<NP, double>(N);
  DfTab<NP> t{};
  t.Df = split_eo<NP>(g.Df);
  t.Dt = split_eo<NP>(g.Dt);
  auto split = [](double v, float& h, float& l) {
    h = static_cast<float>(v);
    l = static_cast<float>(v - static_cast<double>(h));
  };
  for (int k = 0; k < NP; ++k) {
    t.xi[k] = g.xi[k];
    t.w[k] = g.w[k];
  }
  for (int k = 0; k < NP; ++k) {
    float h, l;
    split(g.xi[k], h, l);
    t.gdh[k] = make_float2(h, h);
    t.ngdh[k] = make_float2(-h, -h);
    t.ngdl[k] = make_float2(-l, -l);
    split(g.w[k], t.wkh[k], t.wkl[k]);
  }
  return t;
}

// The sums one after the other (any NP; odd NP: A_i has the extra middle term).
template <int NP>
__device__ __forceinline__ void eo_apply_df_odd(const DfEo<NP>& M, const df2 (&in)[NP], df2 (&out)[NP]) {
  constexpr int H = NP / 2, N = NP - 1, HA = H + NP % 2;
  df2 e[H], o[H];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    e[l] = df_add_nr(in[l], in[N - l]);
    o[l] = df_add_nr(in[l], df_neg(in[N - l]));
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float pa[HA], ea[HA], pb[H], eb[H];
#pragma unroll
    for (int l = 0; l < H; ++l) {
      df_prod(M.Eh[i][l], M.El[i][l], e[l].h, e[l].l, pa[l], ea[l]);
      df_prod(M.Oh[i][l], M.Ol[i][l], o[l].h, o[l].l, pb[l], eb[l]);
    }
    if constexpr (NP % 2 == 1) df_prod(M.Eh[i][H], M.El[i][H], in[H].h, in[H].l, pa[H], ea[H]);
    const df2 A = df_tree_sum_nr<HA>(pa, ea);
    const df2 B = df_tree_sum_nr<H>(pb, eb);
    out[i] = df_add_nr(A, B);  // unnormalised pairs: exact sums, valid operands downstream
    out[N - i] = df_add_nr(B, df_neg(A));
  }
  if constexpr (NP % 2 == 1) {
    float pc[H], ec[H];
#pragma unroll
    for (int l = 0; l < H; ++l) df_prod(M.Oh[H][l], M.Ol[H][l], o[l].h, o[l].l, pc[l], ec[l]);
    out[H] = df_tree_sum<H>(pc, ec);
  }
}

// out = M in in double-float (see EoMat for the split); `in` and `out` may not alias.
// Even NP up to 8: the sums A_i (over the even combinations) and B_i (over the odd ones) have
// the same number of terms, so both run in the two lanes of float2 operations (larger orders keep
// the scalar steps, whose code the compiler handles in far less time): each error-free product
// and each two-sum of the tree is one two-wide instruction per step for both. The error terms
// are carried negated (ne = p - a b, formed by a multiply-add with the negated constants, so
// that p itself needs no negation); round-to-nearest is symmetric, so every lane holds exactly
// the negation of what the scalar steps would hold and the results are the same bit for bit.
template <int NP>
__device__ __forceinline__ void eo_apply_df(const DfEo<NP>& M, const df2 (&in)[NP], df2 (&out)[NP]) {
  constexpr int H = NP / 2, N = NP - 1;
  if constexpr (NP % 2 == 0 && NP <= 8) {
    float2 X[H], XL[H];  // (even, odd) combinations: high parts, low parts
#pragma unroll
    for (int l = 0; l < H; ++l) {
      const df2 ev = df_add_nr(in[l], in[N - l]);
      const df2 od = df_add_nr(in[l], df_neg(in[N - l]));
      X[l] = make_float2(ev.h, od.h);
      XL[l] = make_float2(ev.l, od.l);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
      float2 pp[H], ne[H];
#pragma unroll
      for (int l = 0; l < H; ++l) {
        pp[l] = __fmul2_rn(M.C[i][l], X[l]);
        ne[l] = __ffma2_rn(M.NC[i][l], X[l], pp[l]);  // exact: p - ah bh
        ne[l] = __ffma2_rn(M.NC[i][l], XL[l], ne[l]);
        ne[l] = __ffma2_rn(M.NCL[i][l], X[l], ne[l]);
      }
#pragma unroll
      for (int wd = 1; wd < H; wd *= 2) {
#pragma unroll
        for (int a = 0; a + wd < H; a += 2 * wd) {
          const float2 sm = __fadd2_rn(pp[a], pp[a + wd]);  // Knuth's two-sum in both lanes
          const float2 bb = fsub2_rn(sm, pp[a]);
          const float2 t = __fadd2_rn(fsub2_rn(pp[a], fsub2_rn(sm, bb)), fsub2_rn(pp[a + wd], bb));
          pp[a] = sm;
          ne[a] = __fadd2_rn(ne[a], fsub2_rn(ne[a + wd], t));
        }
      }
      const df2 A{pp[0].x, -ne[0].x}, B{pp[0].y, -ne[0].y};
      out[i] = df_add_nr(A, B);  // unnormalised pairs: exact sums, valid operands downstream
      out[N - i] = df_add_nr(B, df_neg(A));
    }
  } else {
    eo_apply_df_odd<NP>(M, in, out);
  }
}


// a g + c in both lanes for a pair a, the column points' node g (high gh; negated high and
// low ngh, ngl) and a pair c: (s, l) with s + l = a g + c to double-float accuracy (unnormalised).
__device__ __forceinline__ void df2_fma_node(float2 ah, float2 al, float2 gh, float2 ngh, float2 ngl, float2 ch,
                                             float2 cl, float2& sh, float2& sl) {
  const float2 p = __fmul2_rn(ah, gh);
  float2 ne = __ffma2_rn(ah, ngh, p);  // exact: p - ah gh
  ne = __ffma2_rn(ah, ngl, ne);
  ne = __ffma2_rn(al, ngh, ne);
  const float2 s = __fadd2_rn(p, ch);  // Knuth's two-sum of p and the high part of c
  const float2 bb = fsub2_rn(s, p);
  const float2 t = __fadd2_rn(fsub2_rn(p, fsub2_rn(s, bb)), fsub2_rn(ch, bb));
  sh = s;
  sl = __fadd2_rn(t, fsub2_rn(cl, ne));
}

// On-the-fly geometry in double-float (Section 5.1's rematerialised factors, in the cofactor
// form of OtfColumn): the column's polynomial coefficients are formed in FP64 (OtfColumn<double>,
// once per column, on the FP64 pipe that this kernel otherwise leaves idle) and split into float
// pairs; at every point C, det J, w_i w_j w_k / det J and G v = (w_i w_j w_k / det J) C (C^T v)
// run in double-float on the FP32 pipes. The nine cofactor entries and det J are evaluated
// two at a time in the lanes of float2 operations, the coefficients held in these pairs:
//   lin[0] = (c0_x, c0_y), lin[1] = (c0_z, c1_z), lin[2] = (c1_x, c1_y)   (a + gam b)
//   quad[0] = (c2_x, c2_y), quad[1] = (c2_z, det J)                     (a + gam (b + gam c))
struct OtfColumnDf {
  float2 lah[3], lal[3], lbh[3], lbl[3];               // linear pairs: a and b, high and low
  float2 qah[2], qal[2], qbh[2], qbl[2], qch[2], qcl[2];  // quadratic pairs
  df2 wij;                                              // w_i w_j

  __device__ __forceinline__ static void pair(double x, double y, float2& h, float2& l) {
    const df2 a = df_from_double(x), b = df_from_double(y);
    h = make_float2(a.h, b.h);
    l = make_float2(a.l, b.l);
  }
  __device__ __forceinline__ void init(const OtfColumn<double>& g, double w_ij) {
    pair(g.c0a.x, g.c0a.y, lah[0], lal[0]);
    pair(g.c0b.x, g.c0b.y, lbh[0], lbl[0]);
    pair(g.c0a.z, g.c1a.z, lah[1], lal[1]);
    pair(g.c0b.z, g.c1b.z, lbh[1], lbl[1]);
    pair(g.c1a.x, g.c1a.y, lah[2], lal[2]);
    pair(g.c1b.x, g.c1b.y, lbh[2], lbl[2]);
    pair(g.c2a.x, g.c2a.y, qah[0], qal[0]);
    pair(g.c2b.x, g.c2b.y, qbh[0], qbl[0]);
    pair(g.c2c.x, g.c2c.y, qch[0], qcl[0]);
    pair(g.c2a.z, g.da, qah[1], qal[1]);
    pair(g.c2b.z, g.db, qbh[1], qbl[1]);
    pair(g.c2c.z, g.dc, qch[1], qcl[1]);
    wij = df_from_double(w_ij);
  }

  // (ur, us, ut) <- G (ur, us, ut) at column point k (node and weight from the table).
  template <int NP>
  __device__ __forceinline__ void apply(const DfTab<NP>& tab, int k, df2& ur, df2& us, df2& ut) const {
    const float2 gh = tab.gdh[k], ngh = tab.ngdh[k], ngl = tab.ngdl[k];  // (gam, gam)
    float2 lh[3], ll[3], qh[2], ql[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) df2_fma_node(lbh[a], lbl[a], gh, ngh, ngl, lah[a], lal[a], lh[a], ll[a]);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      float2 xh, xl;
      df2_fma_node(qch[a], qcl[a], gh, ngh, ngl, qbh[a], qbl[a], xh, xl);
      df2_fma_node(xh, xl, gh, ngh, ngl, qah[a], qal[a], qh[a], ql[a]);
    }
    // M[r][c]: row r of C (c_r), component c
    const df2 M[3][3] = {{{lh[0].x, ll[0].x}, {lh[0].y, ll[0].y}, {lh[1].x, ll[1].x}},
                         {{lh[2].x, ll[2].x}, {lh[2].y, ll[2].y}, {lh[1].y, ll[1].y}},
                         {{qh[0].x, ql[0].x}, {qh[0].y, ql[0].y}, {qh[1].x, ql[1].x}}};
    const df2 det{qh[1].y, ql[1].y};
    // sc = w_i w_j w_k / det J: y exactly enough, then Dekker's double-length division
    // (q1 = y / det J in FP32, the remainder y - q1 det J, q2 = remainder / det J, sc = q1 + q2)
    float yh, ye;
    df_prod(wij.h, wij.l, tab.wkh[k], tab.wkl[k], yh, ye);
    const float rc = __fdividef(1.f, det.h);
    const float q1 = yh * rc;
    float p2, e2;
    df_prod(q1, 0.f, det.h, det.l, p2, e2);  // q1 det J = p2 + e2
    const float rem = (yh - p2) + (ye - e2);
    const float q2 = rem * rc;
    const float sh = q1 + q2;  // fast two-sum (|q2| << |q1|)
    const df2 sc{sh, q2 - (sh - q1)};
    // q = sc C^T u, then u = C q
    const df2 u[3] = {ur, us, ut};
    df2 q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float pp[3], ee[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) df_prod(M[r][c].h, M[r][c].l, u[r].h, u[r].l, pp[r], ee[r]);
      const df2 t = df_tree_sum_nr<3>(pp, ee);
      float ph, pe;
      df_prod(sc.h, sc.l, t.h, t.l, ph, pe);
      q[c] = {ph, pe};
    }
    df2 v[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float pp[3], ee[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) df_prod(M[r][c].h, M[r][c].l, q[c].h, q[c].l, pp[c], ee[c]);
      v[r] = df_tree_sum<3>(pp, ee);
    }
    ur = v[0];
    us = v[1];
    ut = v[2];
  }
};

// Factor values staged in shared memory per element: the first three arrays (G11, G12, G13)
// when P is even (their bytes are then a multiple of 16, as bulk copies need), all six
// otherwise. Unstaged arrays are prefetched into L2 with the copy and read from there. The
// smaller stage lets more blocks share an SM, which this issue-bound kernel needs.
template <int NP, int GK>
__host__ __device__ constexpr int df_gst() {
  return GK == kGkOtf ? 0 : NP % 2 == 0 ? 3 * NP * NP * NP : 6 * NP * NP * NP;
}
template <int NP, int GK>
constexpr size_t df_smem_bytes() {
  constexpr int EPB = ax_epb<NP>();
  return static_cast<size_t>(EPB) * df_gst<NP, GK>() * sizeof(double)            // factors of the group (TMA target)
         + (GK == kGkOtf ? 3 : 2) * static_cast<size_t>(EPB) * Stage<NP>::kSize * sizeof(df2)  // staging A, B (, C)
         + 16;                                                                                // mbarrier
}

// Copies the staged factors of the element group starting at element e0 (count elements, each
// a contiguous [6][P] block of 8-byte values) into sG and prefetches the rest into L2; one
// thread announces the bytes and issues the copies.
template <int NP>
__device__ __forceinline__ void prefetch_factors(double* sG, const double* G, int64_t e0, int count, uint64_t* bar) {
  constexpr int P = NP * NP * NP, GST = df_gst<NP, kGkF64>();
  constexpr unsigned kElemBytes = GST * sizeof(double);
  fence_proxy_async();
  mbar_expect_tx(bar, kElemBytes * static_cast<unsigned>(count));
  for (int q = 0; q < count; ++q) {
    tma_load_1d(sG + q * GST, G + (e0 + q) * 6 * P, kElemBytes, bar);
    if constexpr (GST != 6 * P) l2_prefetch(G + (e0 + q) * 6 * P + GST, (6 * P - GST) * sizeof(double));
  }
}

// Phases of a group, as in k_ax (barrier between phases; each thread owns one i-row, one
// j-line and one k-column of its element in the in-place phases):
//   0 column of u (or x += alpha p, p = M^-1 r + beta p) -> registers and A;  1 i-rows of A -> ur into B, column -> ut;
//   2 j-lines of A -> us in place;  3 column: G (ur, us, ut);  4 D^T on rows, lines, column;
//   5 column: w = sum of the three, converted to FP64 and stored.
// GK: the factors (kGkF64 / kGkPairs: stored, staged by TMA; kGkOtf: rebuilt from coef).
// Minimum blocks per SM: four at N = 7 in CG mode and for the stored plain kernel (128
// registers; 0.429 -> 0.414 ms against a minimum of 1); on the fly otherwise the compiler's
// default (0: 128 registers at N = 7, 0.748 -> 0.707 ms against a minimum of 1); stored
// otherwise 1 (the default took fewer registers there but ran 4% slower at N = 7).
template <int NP, bool CG, int GK>
__global__ void __launch_bounds__(NP * NP * ax_epb<NP>(),
                                  (NP == 8 && (CG || GK != kGkOtf)) ? 4 : GK == kGkOtf ? 0 : 1)
    k_ax_df(const __grid_constant__ DfTab<NP> tab, int64_t E, const double* __restrict__ u, double* __restrict__ w,
            const double* __restrict__ G, const double* __restrict__ coef, const double* __restrict__ r,
            double* __restrict__ p,
            const double* __restrict__ minv, double* __restrict__ x, CgScalars* __restrict__ st,
            double* __restrict__ partials, int* __restrict__ err) {
  constexpr int NP2 = NP * NP, P = NP2 * NP, EPB = ax_epb<NP>(), SZ = Stage<NP>::kSize;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr bool OTF = GK == kGkOtf;
  constexpr int GST = df_gst<NP, GK>();
  double* sG = reinterpret_cast<double*>(smem);
  df2* sA0 = reinterpret_cast<df2*>(sG + EPB * GST);
  df2* sB0 = sA0 + EPB * SZ;
  df2* sC0 = sB0 + EPB * SZ;  // OTF: ut during the geometry phase
  // byte offset EPB*GST*8 + (2 or 3)*EPB*SZ*8: a multiple of 8, as the mbarrier needs
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB0 + (OTF ? 2 : 1) * EPB * SZ);
  __shared__ double sRed[32];

  double beta = 0.0, alpha = 0.0;
  if constexpr (CG) {
    if (st->done) return;
    beta = st->beta;
    alpha = st->alpha;
  }
  const int64_t n_groups = (E + EPB - 1) / EPB;
  if (!OTF && threadIdx.x == 0) {
    mbar_init(bar, 1);
    const int64_t e0 = static_cast<int64_t>(blockIdx.x) * EPB;
    prefetch_factors<NP>(sG, G, e0, static_cast<int>(E - e0 < EPB ? E - e0 : EPB), bar);
  }
  // CG: bulk L2 prefetches of the vectors need 16-byte aligned element blocks (the library's
  // own vectors are; P even makes every block's offset a multiple of 16 bytes)
  const bool vec_l2 = CG && ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(x) |
                              reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(minv)) & 15u) == 0;
  const int slot = threadIdx.x / NP2, tid = threadIdx.x % NP2;
  const int i = tid % NP, j = tid / NP;  // column (i, j); i-row (j, k) = (i, j); j-line (i, k) = (i, j)
  df2* sA = sA0 + slot * SZ;
  df2* sB = sB0 + slot * SZ;
  df2* sC = sC0 + slot * SZ;
  df2 dot{0.f, 0.f};  // CG mode: this thread's part of <p, w>
  unsigned parity = 0;
  __syncthreads();

  for (int64_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const int64_t e = grp * EPB + slot;
    const bool valid = e < E;
    const int64_t base = e * P + tid;
    // phase 0
    df2 rU[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      double val = 0.0;
      if (valid) {
        if constexpr (CG) {
          const int64_t q = base + k * NP2;
          const double po = p[q], xo = x[q], rr = r[q], mm = minv ? minv[q] : 1.0;
          const double zq = minv ? mm * rr : rr;
          val = fma(beta, po, zq);
          x[q] = fma(alpha, po, xo);
          p[q] = val;
        } else {
          val = u[base + k * NP2];
        }
      }
      rU[k] = df_from_double(val);
      sA[Stage<NP>::at(i, j, k)] = rU[k];
    }
    __syncthreads();
    // phase 1
    df2 rT[NP];
    {
      df2 in[NP], out[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(l, i, j)];
      eo_apply_df<NP>(tab.Df, in, out);
#pragma unroll
      for (int l = 0; l < NP; ++l) sB[Stage<NP>::at(l, i, j)] = out[l];
      eo_apply_df<NP>(tab.Df, rU, rT);
    }
    __syncthreads();
    // phase 2
    {
      df2 in[NP], out[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) in[l] = sA[Stage<NP>::at(i, l, j)];
      eo_apply_df<NP>(tab.Df, in, out);
#pragma unroll
      for (int l = 0; l < NP; ++l) sA[Stage<NP>::at(i, l, j)] = out[l];
    }
    if constexpr (OTF) {
      __syncthreads();
    } else {
      const bool ok = mbar_wait_bounded(bar, parity);  // this group's factors
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
    }
    // phase 3
    if constexpr (OTF) {
      OtfColumn<double> g64{};
      double wij = 0.0;
      if (valid) {
        g64.init(coef + e * 24, tab.xi[i], tab.xi[j]);
        wij = tab.w[i] * tab.w[j];
      } else {
        g64.da = 1.0;  // an absent element: unit det J, zero weight, so its w is 0
      }
      OtfColumnDf col;
      col.init(g64, wij);
      // point by point through shared memory (ut in the third buffer), so that no line of the
      // column is held in registers across the evaluation
#pragma unroll
      for (int k = 0; k < NP; ++k) sC[Stage<NP>::at(i, j, k)] = rT[k];
#pragma unroll 1
      for (int k = 0; k < NP; ++k) {
        const int at = Stage<NP>::at(i, j, k);
        df2 ur = sB[at], us = sA[at], ut = sC[at];
        col.apply<NP>(tab, k, ur, us, ut);
        sB[at] = ur;
        sA[at] = us;
        sC[at] = ut;
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) rT[k] = sC[Stage<NP>::at(i, j, k)];
    } else {
      const double* gE = sG + slot * GST;
      const double* gH = G + (valid ? e : int64_t(0)) * 6 * P;  // arrays 3..5 from L2 when not staged
      df2 rR[NP], rS[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int at = Stage<NP>::at(i, j, k);
        rR[k] = sB[at];
        rS[k] = sA[at];
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        df2 g[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          const double* src = (GST != 6 * P && m >= 3) ? gH : gE;
          if constexpr (GK == kGkPairs) {  // factors stored as float pairs: no split needed
            const float2 v = reinterpret_cast<const float2*>(src)[m * P + k * NP2 + tid];
            g[m] = {v.x, v.y};
          } else {
            g[m] = df_from_double(src[m * P + k * NP2 + tid]);
          }
        }
        const df2 ur = rR[k], us = rS[k], ut = rT[k];
        float p3[3], e3[3];
        df_prod(g[0].h, g[0].l, ur.h, ur.l, p3[0], e3[0]);
        df_prod(g[1].h, g[1].l, us.h, us.l, p3[1], e3[1]);
        df_prod(g[2].h, g[2].l, ut.h, ut.l, p3[2], e3[2]);
        rR[k] = df_tree_sum<3>(p3, e3);
        df_prod(g[1].h, g[1].l, ur.h, ur.l, p3[0], e3[0]);
        df_prod(g[3].h, g[3].l, us.h, us.l, p3[1], e3[1]);
        df_prod(g[4].h, g[4].l, ut.h, ut.l, p3[2], e3[2]);
        rS[k] = df_tree_sum<3>(p3, e3);
        df_prod(g[2].h, g[2].l, ur.h, ur.l, p3[0], e3[0]);
        df_prod(g[4].h, g[4].l, us.h, us.l, p3[1], e3[1]);
        df_prod(g[5].h, g[5].l, ut.h, ut.l, p3[2], e3[2]);
        rT[k] = df_tree_sum<3>(p3, e3);
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int at = Stage<NP>::at(i, j, k);
        sB[at] = rR[k];
        sA[at] = rS[k];
      }
    }
    __syncthreads();  // the factors are consumed
    if (threadIdx.x == 0 && grp + gridDim.x < n_groups) {
      const int64_t e0 = (grp + gridDim.x) * EPB;
      const int cnt = static_cast<int>(E - e0 < EPB ? E - e0 : EPB);
      if constexpr (!OTF) prefetch_factors<NP>(sG, G, e0, cnt, bar);
      if constexpr (CG && P % 2 == 0) {  // the next group's p, x, r, M^-1 into L2 (phase 0 reads them)
        if (vec_l2) {
          for (int q = 0; q < cnt; ++q) {
            const int64_t off = (e0 + q) * P;
            l2_prefetch(p + off, P * sizeof(double));
            l2_prefetch(x + off, P * sizeof(double));
            l2_prefetch(r + off, P * sizeof(double));
            if (minv) l2_prefetch(minv + off, P * sizeof(double));
          }
        }
      }
    }
    // phase 4
    df2 rW[NP];
    {
      df2 inR[NP], inS[NP], outR[NP], outS[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        inR[l] = sB[Stage<NP>::at(l, i, j)];
        inS[l] = sA[Stage<NP>::at(i, l, j)];
      }
      eo_apply_df<NP>(tab.Dt, inR, outR);
      eo_apply_df<NP>(tab.Dt, inS, outS);
      eo_apply_df<NP>(tab.Dt, rT, rW);
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        sB[Stage<NP>::at(l, i, j)] = outR[l];
        sA[Stage<NP>::at(i, l, j)] = outS[l];
      }
    }
    __syncthreads();
    // phase 5
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int at = Stage<NP>::at(i, j, k);
      const df2 acc = df_norm(df_add_nr(df_add_nr(sB[at], sA[at]), rW[k]));
      if (valid) w[CG ? e * P + cg_pos(NP, i, j, k) : base + k * NP2] = df_to_double(acc);  // CG: CG layout
      if constexpr (CG) {
        if (valid) df_fma_acc(dot, rU[k].h, rU[k].l, acc.h, acc.l);
      }
    }
    __syncthreads();  // the staging buffers are free for the next group
  }
  if constexpr (CG) {
    const double s = block_sum(static_cast<double>(dot.h) + static_cast<double>(dot.l), sRed);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

template <int NP, bool CG, int GK>
sem_status launch_df_t(int N, const AxLaunch& a, cudaStream_t s) {
  constexpr int EPB = ax_epb<NP>();
  constexpr size_t smem = df_smem_bytes<NP, GK>();
  // resident blocks per SM x SMs, with the dynamic shared-memory limit raised first; once
  static const int max_blocks = [] {
    cudaFuncSetAttribute(k_ax_df<NP, CG, GK>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_df<NP, CG, GK>, NP * NP * EPB, smem);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }();
  const int64_t groups = (a.E + EPB - 1) / EPB;
  int grid = max_blocks < kRedMax ? max_blocks : kRedMax;
  if (groups < grid) grid = static_cast<int>(groups);
  if (a.grid_out) *a.grid_out = grid;
  k_ax_df<NP, CG, GK><<<grid, NP * NP * EPB, smem, s>>>(
      make_df_tab<NP>(N), a.E, static_cast<const double*>(a.u), static_cast<double*>(a.w),
      static_cast<const double*>(a.G), static_cast<const double*>(a.coef), static_cast<const double*>(a.r),
      static_cast<double*>(a.p), static_cast<const double*>(a.minv), static_cast<double*>(a.x), a.st, a.partials,
      a.err);
  count_launch();
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

// Dispatch over the orders LO <= N + 1 <= HI compiled in one translation unit.
template <template <int> class L, int NP, int HI>
sem_status df_dispatch(int N, bool cg, const AxLaunch& a, cudaStream_t s) {
  if (N + 1 == NP) return L<NP>::run(N, cg, a, s);
  if constexpr (NP < HI) return df_dispatch<L, NP + 1, HI>(N, cg, a, s);
  return fail(SEM_ERR_UNSUPPORTED, "polynomial order not compiled in");
}

}  // namespace
}  // namespace sem
