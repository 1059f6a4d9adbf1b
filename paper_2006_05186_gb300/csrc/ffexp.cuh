// The Laplace-domain kernel c * exp(-s d) in float-float arithmetic on the
// FP32 pipes, for the MACA slices and fibres (Sec. 5.1, Alg. 2: entries of
// the block tensors at one frequency, or at all frequencies of one pair).
//
// GB300 issues FP32 about 60 times faster than FP64, and the entries need
// more than FP32 accuracy (a slice must resolve the MACA tolerance; a fibre
// carries per-frequency rounding, which the inverse transform scales by up
// to R^-N).  A float-float value is an unevaluated sum h + l of two floats;
// the error-free transformations are the FMA product (a b - p = fma(a, b, -p))
// and Knuth's TwoSum, which keep about 48 significant bits.
//
// The distance is split as r = r0 + d with d >= 0: r0 is a lower bound of
// the distances of the pair's points (0 for pairs sharing a vertex), and
// exp(-s r0) is formed once per pair in FP64.  So per point only exp(-s d)
// is needed, with Re(s) d >= 0 (no overflow) and a small phase.
//
// exp(-s d) follows the table method of Tang (ACM TOMS 15(2), 1989) for the
// exponential and the same reduction for the circular functions:
//   u = -Re(s) d = (1024 k + j) ln2/1024 + f,  |f| <= ln2/2048,
//   exp(u) = 2^k 2^(j/1024) exp(f);
//   theta = Im(s) d = m pi/512 + g,  |g| <= pi/1024,
//   cis(-theta) = conj(cis(m pi/512) cis(g)).
// ln2/1024 and pi/512 are split into three floats (the first times an
// integer formed exactly by the FMA product), exp(f) - 1, sin(g) and
// cos(g) - 1 are their Taylor polynomials (the bound of each omitted term is
// stated where it is dropped), and the tables hold 2^(j/1024) and
// cis(m pi/512) as float-float pairs.  The relative error of a value is
// about 2^-47 (|Re(s) d| + |Im(s) d|) + 2^-45.
#pragma once

#include "common.cuh"

namespace cqm {

struct ff {
  float h, l;
};

// ---- error-free transformations ------------------------------------------
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__host__ __device__ __forceinline__ ff ff_of(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

// a * b to about 2^-46 relative (normalised result)
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p, e;
  two_prod(a.h, b.h, p, e);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  ff r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}

// acc += v; acc.l grows by at most an ulp of acc.h per call, renormalise
// with ff_norm every few dozen additions
__device__ __forceinline__ void ff_acc(ff& acc, ff v) {
  float s, e;
  two_sum(acc.h, v.h, s, e);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, v.l));
}
__device__ __forceinline__ void ff_norm(ff& a) {
  float s, e;
  fast_two_sum(a.h, a.l, s, e);
  a.h = s;
  a.l = e;
}
// a + b (normalised)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  ff r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}

// ---- reduction constants (each a float; the three sum to the constant to
// 2^-88 relative) -----------------------------------------------------------
#define CQM_FF_INV_LN2_1024 0x1.715476p+10f    // 1024 / ln 2 (only selects k, j)
#define CQM_FF_LN2_1024_H 0x1.62e43p-11f       // ln 2 / 1024, three parts
#define CQM_FF_LN2_1024_M (-0x1.05c61p-39f)
#define CQM_FF_LN2_1024_L (-0x1.950d88p-64f)
#define CQM_FF_INV_PI_512 0x1.45f306p+7f       // 512 / pi (only selects m)
#define CQM_FF_PI_512_H 0x1.921fb6p-8f         // pi / 512, three parts
#define CQM_FF_PI_512_M (-0x1.777a5cp-33f)
#define CQM_FF_PI_512_L (-0x1.ee59dap-58f)

// Frequency as float-float parts.
struct ffs {
  ff re, im;
};
__device__ __forceinline__ ffs ffs_of(double2 s) { return {ff_of(s.x), ff_of(s.y)}; }

// (vr, vi) = c * exp(-s d) for d >= 0 and Re(s) >= 0 (the CQM frequencies of
// an A-stable BDF method).  t2[j] = 2^(j/1024), cs[m] = (cos hi, cos lo,
// sin hi, sin lo)(m pi/512), both float-float, normally in shared memory.
__device__ __forceinline__ void cexp_ff(ff d, ff c, const ffs& s, const float2* __restrict__ t2,
                                        const float4* __restrict__ cs, ff& vr, ff& vi) {
  // u = -Re(s) d = -(p + e)
  float p, e;
  two_prod(s.re.h, d.h, p, e);
  e = fmaf(s.re.h, d.l, e);
  e = fmaf(s.re.l, d.h, e);
  const float nf = rintf(__fmul_rn(-p, CQM_FF_INV_LN2_1024));  // <= 0
  if (!(nf > -126.0f * 1024.0f)) {  // exp(u) < 2^-126: below every other term of the sum
    vr = {0.f, 0.f};
    vi = {0.f, 0.f};
    return;
  }
  const int n = (int)nf;
  const int j = n & 1023;
  const int k = (n - j) >> 10;  // -126 <= k <= 0
  // f = u - n ln2/1024: -p - n h is exact (Sterbenz), the rest is small
  float q1, q2;
  two_prod(nf, CQM_FF_LN2_1024_H, q1, q2);
  const float fa = __fsub_rn(-p, q1);
  float fb = __fsub_rn(-e, q2);
  fb = fmaf(-nf, CQM_FF_LN2_1024_M, fb);
  fb = fmaf(-nf, CQM_FF_LN2_1024_L, fb);
  float fh, fl;
  two_sum(fa, fb, fh, fl);
  // exp(f) = 1 + fh + (fl + fh^2 (1/2 + fh/6 + fh^2/24)); the next term,
  // f^5/120, is below 4e-20 for |f| <= ln2/2048
  const float tq = __fmul_rn(__fmul_rn(fh, fh), fmaf(fmaf(fh, 1.0f / 24.0f, 1.0f / 6.0f), fh, 0.5f));
  const float pl = __fadd_rn(fl, tq);
  // M = 2^(j/1024) exp(f) = T + T fh + T pl
  const float2 T = t2[j];
  float x1, x1e, mh, ml;
  two_prod(T.x, fh, x1, x1e);
  fast_two_sum(T.x, x1, mh, ml);  // T >= 1 > |x1|
  ml = __fadd_rn(ml, x1e);
  ml = fmaf(T.x, pl, ml);
  ml = fmaf(T.y, fh, ml);
  ml = __fadd_rn(ml, T.y);
  const float sc = __int_as_float((k + 127) << 23);  // 2^k, exact
  ff A = ff_mul(c, ff{__fmul_rn(mh, sc), __fmul_rn(ml, sc)});
  // theta = Im(s) d = p + e
  two_prod(s.im.h, d.h, p, e);
  e = fmaf(s.im.h, d.l, e);
  e = fmaf(s.im.l, d.h, e);
  const float mf = rintf(__fmul_rn(p, CQM_FF_INV_PI_512));
  const int m = ((int)mf) & 1023;
  two_prod(mf, CQM_FF_PI_512_H, q1, q2);
  const float ga = __fsub_rn(p, q1);
  float gb = __fsub_rn(e, q2);
  gb = fmaf(-mf, CQM_FF_PI_512_M, gb);
  gb = fmaf(-mf, CQM_FF_PI_512_L, gb);
  float gh, gl;
  two_sum(ga, gb, gh, gl);
  // sin g = gh + (gl + gh^3 (-1/6 + gh^2/120)) (next term g^7/5040 below 2e-19 |g|);
  // cos g - 1 = -q/2 + (-qe/2 - gh gl + q^2/24) with q + qe = gh^2 exactly
  // (next term g^6/720 below 1.2e-18)
  const float g2 = __fmul_rn(gh, gh);
  const float sl = fmaf(__fmul_rn(gh, g2), fmaf(g2, 1.0f / 120.0f, -1.0f / 6.0f), gl);
  float q, qe;
  two_prod(gh, gh, q, qe);
  const float ch = __fmul_rn(-0.5f, q);
  const float cl = fmaf(__fmul_rn(q, q), 1.0f / 24.0f, fmaf(-gh, gl, __fmul_rn(-0.5f, qe)));
  const float4 W = cs[m];  // cos(m pi/512) = W.x + W.y, sin(m pi/512) = W.z + W.w
  // cos theta = Tc + Tc (cos g - 1) - Ts sin g
  float a1, a1e, a2, a2e, s1, t1, s2, t2v;
  two_prod(W.z, gh, a1, a1e);
  two_prod(W.x, ch, a2, a2e);
  two_sum(W.x, -a1, s1, t1);
  two_sum(s1, a2, s2, t2v);
  float lo = __fadd_rn(__fadd_rn(t1, t2v), __fsub_rn(a2e, a1e));
  lo = __fadd_rn(lo, W.y);
  lo = fmaf(W.x, cl, lo);
  lo = fmaf(-W.z, sl, lo);
  lo = fmaf(-W.w, gh, lo);
  lo = fmaf(W.y, ch, lo);
  ff co, si;
  two_sum(s2, lo, co.h, co.l);  // cos theta may be small: renormalise exactly
  // sin theta = Ts + Ts (cos g - 1) + Tc sin g
  two_prod(W.x, gh, a1, a1e);
  two_prod(W.z, ch, a2, a2e);
  two_sum(W.z, a1, s1, t1);
  two_sum(s1, a2, s2, t2v);
  lo = __fadd_rn(__fadd_rn(t1, t2v), __fadd_rn(a1e, a2e));
  lo = __fadd_rn(lo, W.w);
  lo = fmaf(W.z, cl, lo);
  lo = fmaf(W.x, sl, lo);
  lo = fmaf(W.y, gh, lo);
  lo = fmaf(W.w, ch, lo);
  two_sum(s2, lo, si.h, si.l);
  vr = ff_mul(A, co);
  vi = ff_mul(A, si);
  vi.h = -vi.h;
  vi.l = -vi.l;
}

}  // namespace cqm
