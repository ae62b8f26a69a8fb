// Double-float arithmetic on the FP32 pipes for FP64 data.
//
// A value is carried as an unevaluated sum h + l of two floats. GB300 issues FP32 fused
// multiply-adds 64 times faster than FP64 ones (128 against 2 per clock per SM), so FP64 contractions are rewritten as
// error-free transformations on floats:
//   product   a * b  ->  p = fl(ah bh), e = fma(ah, bh, -p) (exact error), plus the cross
//                        terms ah bl + al bh (al bl is below the working precision);
//   sum       s + p  ->  Knuth's two-sum, whose rounding error is exact;
// which keeps about 47 significant bits (relative error ~1e-14).
//
// Conversions from FP64 use integer operations only (no FP64 instruction): h takes the top
// 24 significand bits, l the next 23. Values outside FP32's normal exponent range are not
// representable this way: magnitudes below 2^-126 become 0, above 2^128 become inf.
#pragma once

#include <cuda_runtime.h>

namespace sem {

struct df2 {
  float h, l;
};

__device__ __forceinline__ df2 df_from_double(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi32 = static_cast<unsigned>(b >> 32), lo32 = static_cast<unsigned>(b);
  const unsigned sign = hi32 & 0x80000000u;
  const int E = static_cast<int>((hi32 >> 20) & 0x7ffu);
  const int fe = E - 896;  // biased FP32 exponent of the same power of two
  df2 r;
  if (fe >= 1 && fe <= 254) {
    const unsigned mh = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
    r.h = __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | mh);
    // the remaining 29 significand bits are rem * 2^(E - 1075); keep their top 23 exactly:
    // q is the integer rem >> 6, built without a conversion instruction
    const unsigned rem23 = (lo32 & 0x1fffffffu) >> 6;
    const float q = __fsub_rn(__uint_as_float(0x4b000000u | rem23), 8388608.0f);
    const int se = E - 1069 + 127;  // biased exponent of 2^(E - 1069)
    const float scale = se >= 1 ? __uint_as_float(static_cast<unsigned>(se) << 23) : 0.0f;
    r.l = __uint_as_float(__float_as_uint(__fmul_rn(q, scale)) | sign);
  } else if (fe > 254) {
    const bool nan = E == 2047 && ((hi32 & 0xfffffu) | lo32) != 0u;
    r.h = __uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u));
    r.l = 0.0f;
  } else {
    r.h = __uint_as_float(sign);
    r.l = 0.0f;
  }
  return r;
}

// Two-wide FP32 subtraction (sm_100 and later), a - b in each lane, rounded to nearest; the
// CUDA headers provide the add, multiply and multiply-add forms only.
__device__ __forceinline__ float2 fsub2_rn(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

__device__ __forceinline__ double df_to_double(df2 a) {
  return static_cast<double>(a.h) + static_cast<double>(a.l);
}

// acc += a * b with acc kept as (running sum of high products, gathered low terms)
__device__ __forceinline__ void df_fma_acc(df2& acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float s = __fadd_rn(acc.h, p);
  const float bb = __fsub_rn(s, acc.h);
  const float t = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

// first term of an accumulation: acc = a * b
__device__ __forceinline__ df2 df_mul(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  return {p, e};
}

// two-sum renormalisation: returns (s, t) with s = fl(h + l) and h + l = s + t exactly
__device__ __forceinline__ df2 df_norm(df2 a) {
  const float s = __fadd_rn(a.h, a.l);
  const float bb = __fsub_rn(s, a.h);
  const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(a.l, bb));
  return {s, t};
}

// a + b for two (normalised) pairs
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return df_norm({s, __fadd_rn(t, __fadd_rn(a.l, b.l))});
}

}  // namespace sem

namespace sem {

// Error-free product a * b as (p, e): p = fl(ah bh), e = its exact rounding error plus the
// cross terms ah bl + al bh.
__device__ __forceinline__ void df_prod(float ah, float al, float bh, float bl, float& p, float& e) {
  p = __fmul_rn(ah, bh);
  e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
}

// a + b without the final renormalisation: (s, t + a.l + b.l) with s + t = a.h + b.h exactly
// (Knuth's two-sum); the pair is a valid operand of df_prod and df_add.
__device__ __forceinline__ df2 df_add_nr(df2 a, df2 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return {s, __fadd_rn(t, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.h, -a.l}; }

// Sum of K terms (p[q] + e[q]) by a pairwise two-sum tree over the high parts; the exact
// rounding errors are gathered into the low parts along the same tree. The critical path
// is log2(K) two-sums instead of K - 1. Returns the pair without renormalisation.
template <int K>
__device__ __forceinline__ df2 df_tree_sum_nr(float (&p)[K], float (&e)[K]) {
#pragma unroll
  for (int w = 1; w < K; w *= 2) {
#pragma unroll
    for (int a = 0; a + w < K; a += 2 * w) {
      const float s = __fadd_rn(p[a], p[a + w]);
      const float bb = __fsub_rn(s, p[a]);
      const float t = __fadd_rn(__fsub_rn(p[a], __fsub_rn(s, bb)), __fsub_rn(p[a + w], bb));
      p[a] = s;
      e[a] = __fadd_rn(e[a], __fadd_rn(t, e[a + w]));
    }
  }
  return {p[0], e[0]};
}

// The same sum, renormalised.
template <int K>
__device__ __forceinline__ df2 df_tree_sum(float (&p)[K], float (&e)[K]) {
#pragma unroll
  for (int w = 1; w < K; w *= 2) {
#pragma unroll
    for (int a = 0; a + w < K; a += 2 * w) {
      const float s = __fadd_rn(p[a], p[a + w]);
      const float bb = __fsub_rn(s, p[a]);
      const float t = __fadd_rn(__fsub_rn(p[a], __fsub_rn(s, bb)), __fsub_rn(p[a + w], bb));
      p[a] = s;
      e[a] = __fadd_rn(e[a], __fadd_rn(t, e[a + w]));
    }
  }
  return df_norm({p[0], e[0]});
}

}  // namespace sem
