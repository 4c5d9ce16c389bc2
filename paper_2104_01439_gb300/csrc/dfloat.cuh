// Double-float ("float-float") arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)), about 48 significant
// bits. GB300 issues FP64 at 1/58 of its FP32 rate, so the long dense sums of the
// Gram-Schmidt sweeps and of the coarse Gauss-Jordan factorisation run in this
// form. Error-free transformations used: TwoSum (Knuth), FastTwoSum (Dekker,
// |a| >= |b|), and the exact product a*b = p + e with e = fma(a, b, -p).
//
// Complex double-float values are stored in a float4 (hi.re, hi.im, lo.re, lo.im),
// 16 bytes like a complex128.
#pragma once
#include <cuda_runtime.h>

namespace helm {

struct DF {
  float h, l;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return DF{s, (a - (s - bp)) + (b - bp)};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return DF{s, b - (s - a)};
}
// renormalise hi + lo
__device__ __forceinline__ DF df_norm(DF a) { return df_fast_two_sum(a.h, a.l); }
__device__ __forceinline__ DF df_split(double d) {
  const float h = (float)d;
  return DF{h, (float)(d - (double)h)};
}
__device__ __forceinline__ double df_val(DF v) { return (double)v.h + (double)v.l; }
// s += a * b (exact product by FMA, TwoSum of the high parts, errors gathered in s.l;
// the caller renormalises once after a run of accumulations)
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, DF& s) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const DF t = df_two_sum(s.h, p);
  s.h = t.h;
  s.l += t.l + e;
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return df_norm(s);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF s{0.f, 0.f};
  df_mac(a.h, a.l, b.h, b.l, s);
  return df_norm(s);
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }

// ---- complex double-float ------------------------------------------------------
__device__ __forceinline__ DF dfc_re(float4 a) { return DF{a.x, a.z}; }
__device__ __forceinline__ DF dfc_im(float4 a) { return DF{a.y, a.w}; }
__device__ __forceinline__ float4 dfc_make(DF re, DF im) { return make_float4(re.h, im.h, re.l, im.l); }
__device__ __forceinline__ float4 dfc_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 dfc_neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 dfc_from(double2 c) { return dfc_make(df_split(c.x), df_split(c.y)); }
// complex64 value nearest to hi + lo (per component)
__device__ __forceinline__ float2 dfc_round(float4 a) { return make_float2(a.x + a.z, a.y + a.w); }
__device__ __forceinline__ double2 dfc_to_double(float4 a) {
  return make_double2(df_val(dfc_re(a)), df_val(dfc_im(a)));
}
// accumulators (unnormalised re, im) for runs of complex products
struct DFC_ACC {
  DF re, im;
};
__device__ __forceinline__ DFC_ACC dfc_acc(float4 c) { return DFC_ACC{dfc_re(c), dfc_im(c)}; }
// acc += a * b
__device__ __forceinline__ void dfc_mac(float4 a, float4 b, DFC_ACC& s) {
  df_mac(a.x, a.z, b.x, b.z, s.re);
  df_mac(-a.y, -a.w, b.y, b.w, s.re);
  df_mac(a.x, a.z, b.y, b.w, s.im);
  df_mac(a.y, a.w, b.x, b.z, s.im);
}
__device__ __forceinline__ float4 dfc_fin(DFC_ACC s) { return dfc_make(df_norm(s.re), df_norm(s.im)); }
// c + a * b
__device__ __forceinline__ float4 dfc_fma(float4 a, float4 b, float4 c) {
  DFC_ACC s = dfc_acc(c);
  dfc_mac(a, b, s);
  return dfc_fin(s);
}
__device__ __forceinline__ float4 dfc_mul(float4 a, float4 b) { return dfc_fma(a, b, dfc_zero()); }
__device__ __forceinline__ float4 dfc_add(float4 a, float4 b) {
  return dfc_make(df_add(dfc_re(a), dfc_re(b)), df_add(dfc_im(a), dfc_im(b)));
}
__device__ __forceinline__ float4 dfc_sub(float4 a, float4 b) { return dfc_add(a, dfc_neg(b)); }
// 1 / d = conj(d) / |d|^2; the reciprocal of |d|^2 is the float quotient refined by one
// Newton step in double-float. Returns false for a zero or non-finite d.
__device__ __forceinline__ bool dfc_inv(float4 d, float4* out) {
  DF m{0.f, 0.f};
  df_mac(d.x, d.z, d.x, d.z, m);
  df_mac(d.y, d.w, d.y, d.w, m);
  m = df_norm(m);
  if (!(m.h > 0.f) || !isfinite(m.h)) return false;
  const float r0 = 1.0f / m.h;
  DF t{0.f, 0.f};
  df_mac(m.h, m.l, r0, 0.f, t);              // m r0 ~ 1
  const DF e = df_add(DF{1.f, 0.f}, df_neg(df_norm(t)));
  DF r{r0, 0.f};
  df_mac(r0, 0.f, e.h, e.l, r);               // r0 + r0 (1 - m r0)
  r = df_norm(r);
  *out = dfc_make(df_mul(dfc_re(d), r), df_neg(df_mul(dfc_im(d), r)));
  return true;
}

}  // namespace helm
