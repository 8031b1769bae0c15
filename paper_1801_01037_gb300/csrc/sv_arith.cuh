// Arithmetic of the three storage/arithmetic modes, as device functions on one amplitude.
//
// The update itself is the paper's strided pair update (Sec. V.A):
//     a <- q11 a + q12 b,   b <- q21 a + q22 b      (a = alpha_k, b = alpha_{k + 2^t}, old values on the right)
// written out per mode.  GB300 executes FP64 at about 1.7 fused multiply-adds per clock per SM and converts
// double <-> float at the same rate, against about 120 FP32 multiply-adds per clock per SM, so complex128 is
// by default computed in "double-float" (DF32) form: every double is split into an unevaluated float pair
// hi + lo with integer bit operations only, the 2x2 complex product becomes four compensated float dot
// products (exact products via FMA, exact sums via TwoSum, Dekker/Knuth), and the pair is re-assembled into
// a double with integer operations, one float multiply and one float-to-int conversion.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "sv_internal.h"

namespace svi {

// ------------------------------------------------------------------------------------------------------
// Double-float primitives
// ------------------------------------------------------------------------------------------------------
struct dfv { float h, l; };

// x (IEEE double) -> hi + lo.  hi = x truncated to 24 significant bits, lo = the remaining 29 mantissa bits
// rounded to 24 bits; |x - (hi + lo)| <= 2^-47 |x|.  Integer and float ops only (no FP64 instruction).
// |x| < 2^-126 gives 0 (absolute error < 1.2e-38); the lo part is dropped for |x| < 2^-74.  Valid for
// |x| < 2^128, which every amplitude of a normalised state satisfies.
__device__ __forceinline__ dfv df_split(double x) {
  const uint32_t lo = (uint32_t)__double2loint(x);
  const uint32_t hi = (uint32_t)__double2hiint(x);
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t eh = hi & 0x7FF00000u;                 // biased exponent e << 20
  const uint32_t t = __funnelshift_l(lo, hi, 3);        // top 23 mantissa bits in t[22:0]
  const uint32_t hb = (t & 0x007FFFFFu) | (eh * 8u - (896u << 23));   // float exponent e - 1023 + 127
  const float rf = __uint2float_rn(lo & 0x1FFFFFFFu);   // residual mantissa bits as an integer
  const float sc = __uint_as_float(eh * 8u - (948u << 23));            // 2^(e - 1075)
  const float l = __fmul_rn(rf, sc);
  dfv r;
  r.h = (eh >= (897u << 20)) ? __uint_as_float(hb | sign) : 0.0f;
  r.l = (eh >= (949u << 20)) ? __uint_as_float(__float_as_uint(l) | sign) : 0.0f;
  return r;
}

// s + e -> nearest double, for |e| <= ulp(s)/2 (as TwoSum leaves it).  The double's bit pattern is s's bits
// re-biased, plus e measured in units of the double ulp of s's binade (|delta| <= 2^28, so an int32).
// When s is a power of two and the correction lowers |s|, the result lies in the binade below, whose ulp
// is half as large, so delta doubles.  Float zero or subnormal s gives (signed) zero.
__device__ __forceinline__ double df_combine(float s, float e) {
  const uint32_t sb = __float_as_uint(s);
  const uint32_t sign = sb & 0x80000000u;
  const uint32_t mag = sb & 0x7FFFFFFFu;
  const uint32_t fexp = mag & 0x7F800000u;
  const uint32_t dhi = ((mag >> 3) + (896u << 20)) | sign;
  const uint32_t dlo = mag << 29;
  const float scale = __uint_as_float(((306u << 23) - fexp) | sign);  // +-2^(52 - (exp(s) - 127))
  int32_t delta = __float2int_rn(__fmul_rn(e, scale));
  if ((mag & 0x007FFFFFu) == 0u && delta < 0) delta *= 2;
  delta = (fexp >= (53u << 23)) ? delta : 0;
  uint64_t bits = (((uint64_t)dhi) << 32 | dlo) + (uint64_t)(int64_t)delta;
  bits = (fexp == 0u) ? (((uint64_t)sign) << 32) : bits;
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Dot products of double-float numbers (a compensated dot product in the manner of Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005).  Each product qh*xh is split exactly into p + e by one multiply and
// one FMA; the p's are summed with TwoSum (Knuth), whose exact rounding errors, the e's and the cross terms
// qh*xl, qm*xh and ql*xh of the three-float gate entry q = qh + qm + ql go to a float accumulator c (the terms
// with xl times qm or ql are below 2^-48 relative and dropped; they depend on the amplitude, so they average
// out, whereas an error in q itself would bias every amplitude the same way).  c carries about 2^-23 of the
// result, so its own rounding leaves an error of a few 2^-47 of the largest term.  A final Fast2Sum
// renormalises the pair (|c| <= |s| except under cancellation, where the error stays that small in absolute
// terms).
__device__ __forceinline__ float df_term(float qh, float qm, float ql, dfv x, float &c) {
  const float p = __fmul_rn(qh, x.h);
  c = __fadd_rn(c, __fmaf_rn(qh, x.h, -p));
  c = __fmaf_rn(qh, x.l, c);
  c = __fmaf_rn(qm, x.h, c);
  c = __fmaf_rn(ql, x.h, c);
  return p;
}

__device__ __forceinline__ dfv fast_two_sum(float s, float c) {
  dfv r;
  r.h = __fadd_rn(s, c);
  r.l = __fsub_rn(c, __fsub_rn(r.h, s));
  return r;
}

// A gate entry in three-float form.
struct q3 { float h, m, l; };

__device__ __forceinline__ dfv df_dot4(q3 q0, dfv x0, q3 q1, dfv x1, q3 q2, dfv x2, q3 q3_, dfv x3) {
  float c = 0.0f, s, e;
  const float p0 = df_term(q0.h, q0.m, q0.l, x0, c);
  const float p1 = df_term(q1.h, q1.m, q1.l, x1, c);
  const float p2 = df_term(q2.h, q2.m, q2.l, x2, c);
  const float p3 = df_term(q3_.h, q3_.m, q3_.l, x3, c);
  two_sum(p0, p1, s, e);
  c = __fadd_rn(c, e);
  two_sum(s, p2, s, e);
  c = __fadd_rn(c, e);
  two_sum(s, p3, s, e);
  c = __fadd_rn(c, e);
  return fast_two_sum(s, c);
}

// Eight terms (one real output of a row of a two-qubit gate), same scheme.
__device__ __forceinline__ dfv df_dot8(const q3 (&q)[8], const dfv (&x)[8]) {
  float c = 0.0f, s, e;
  float p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = df_term(q[i].h, q[i].m, q[i].l, x[i], c);
  s = p[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) {
    two_sum(s, p[i], s, e);
    c = __fadd_rn(c, e);
  }
  return fast_two_sum(s, c);
}

__device__ __forceinline__ dfv df_dot2(q3 q0, dfv x0, q3 q1, dfv x1) {
  float c = 0.0f, s, e;
  const float p0 = df_term(q0.h, q0.m, q0.l, x0, c);
  const float p1 = df_term(q1.h, q1.m, q1.l, x1, c);
  two_sum(p0, p1, s, e);
  c = __fadd_rn(c, e);
  return fast_two_sum(s, c);
}

// ------------------------------------------------------------------------------------------------------
// Lane-packed double-float: two independent double-float values per register pair (the two outputs of a pair
// update), computed with Blackwell's packed FP32x2 instructions (one instruction does the same float
// operation in both lanes).  Each lane's arithmetic is the compensated dot product above with the same error
// bound; subtracted products go through TwoDiff and a separate correction accumulator instead of negated
// coefficients, so no extra negations are needed.
// ------------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  const unsigned long long ua = ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
  const unsigned long long ub = ((unsigned long long)__float_as_uint(b.y) << 32) | __float_as_uint(b.x);
  unsigned long long ud;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
  return make_float2(__uint_as_float((unsigned)ud), __uint_as_float((unsigned)(ud >> 32)));
}
__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }

struct dfv2 { float2 h, l; };   // lane j: h.j + l.j

// A gate entry per lane in three-float form.
struct q3p { float2 h, m, l; };

// p = q.h * x.h per lane; the product's exact rounding error and the cross terms go to c.
__device__ __forceinline__ float2 df_term2(const q3p &q, const dfv2 &x, float2 &c) {
  const float2 p = mul2(q.h, x.h);
  const float2 en = fma2(make_float2(-q.h.x, -q.h.y), x.h, p);  // -(q.h x.h - p), exact
  c = sub2(c, en);
  c = fma2(q.h, x.l, c);
  c = fma2(q.m, x.h, c);
  c = fma2(q.l, x.h, c);
  return p;
}
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2 &s, float2 &e) {
  s = sub2(a, b);
  const float2 bb = sub2(s, a);
  e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
__device__ __forceinline__ dfv2 fast_two_sum2(float2 s, float2 c) {
  dfv2 r;
  r.h = add2(s, c);
  r.l = sub2(c, sub2(r.h, s));
  return r;
}
// q0 x0 - q1 x1 + q2 x2 - q3 x3 (PM) or q0 x0 + q1 x1 + q2 x2 + q3 x3, per lane.
template <bool PM>
__device__ __forceinline__ dfv2 df_dot4_2(const q3p &q0, const dfv2 &x0, const q3p &q1, const dfv2 &x1, const q3p &q2,
                                          const dfv2 &x2, const q3p &q3_, const dfv2 &x3) {
  float2 c = bcast(0.f), cn = bcast(0.f), s, e;
  const float2 p0 = df_term2(q0, x0, c);
  const float2 p1 = df_term2(q1, x1, PM ? cn : c);
  const float2 p2 = df_term2(q2, x2, c);
  const float2 p3 = df_term2(q3_, x3, PM ? cn : c);
  if (PM) two_diff2(p0, p1, s, e); else two_sum2(p0, p1, s, e);
  c = add2(c, e);
  two_sum2(s, p2, s, e);
  c = add2(c, e);
  if (PM) two_diff2(s, p3, s, e); else two_sum2(s, p3, s, e);
  c = add2(c, e);
  if (PM) c = sub2(c, cn);
  return fast_two_sum2(s, c);
}
// ------------------------------------------------------------------------------------------------------
// Per-mode amplitude types.  G: element in global memory.  S: working form in registers / shared memory.
// ------------------------------------------------------------------------------------------------------
template <int MODE> struct Arith;

// Coefficients of one gate in the working precision of a mode, loaded once per gate.
struct CoefF32 { float q[8]; };
struct CoefF64 { double q[8]; };
struct CoefDF { float h[8], m[8], l[8]; };

template <> struct Arith<MODE_C64_F32> {
  using G = float2;
  using S = float2;
  using Coef = CoefF32;
  static __device__ __forceinline__ S load(G v) { return v; }
  static __device__ __forceinline__ G store(S v) { return v; }
  static __device__ __forceinline__ S zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ S one() { return make_float2(1.f, 0.f); }
  static __device__ __forceinline__ void coef(Coef &c, const DevGate &g) {
    // two 16-byte loads (DevGate records are 192 bytes, 16-byte aligned)
    const float4 a = reinterpret_cast<const float4 *>(g.qh)[0], b = reinterpret_cast<const float4 *>(g.qh)[1];
    c.q[0] = a.x; c.q[1] = a.y; c.q[2] = a.z; c.q[3] = a.w;
    c.q[4] = b.x; c.q[5] = b.y; c.q[6] = b.z; c.q[7] = b.w;
  }
  // One output of a two-qubit gate: sum_j V[r][j] x_j with c = row r (entries j = 0..3 as (re, im)).
  static __device__ __forceinline__ S row4(const Coef &c, S x0, S x1, S x2, S x3) {
    const float *q = c.q;
    S r;
    r.x = __fmaf_rn(q[0], x0.x, __fmaf_rn(-q[1], x0.y, __fmaf_rn(q[2], x1.x, __fmaf_rn(-q[3], x1.y,
          __fmaf_rn(q[4], x2.x, __fmaf_rn(-q[5], x2.y, __fmaf_rn(q[6], x3.x, -q[7] * x3.y)))))));
    r.y = __fmaf_rn(q[0], x0.y, __fmaf_rn(q[1], x0.x, __fmaf_rn(q[2], x1.y, __fmaf_rn(q[3], x1.x,
          __fmaf_rn(q[4], x2.y, __fmaf_rn(q[5], x2.x, __fmaf_rn(q[6], x3.y, q[7] * x3.x)))))));
    return r;
  }
  // r = q[j] * a   (q[j] = complex entry j of the matrix: 0 = q11, 1 = q12, 2 = q21, 3 = q22)
  static __device__ __forceinline__ S cmul(const Coef &c, int j, S a) {
    const float qr = c.q[2 * j], qi = c.q[2 * j + 1];
    return make_float2(__fmaf_rn(qr, a.x, -qi * a.y), __fmaf_rn(qr, a.y, qi * a.x));
  }
  static __device__ __forceinline__ void pair(const Coef &c, S &a, S &b) {
    const float *q = c.q;
    S r0, r1;
    r0.x = __fmaf_rn(q[0], a.x, __fmaf_rn(-q[1], a.y, __fmaf_rn(q[2], b.x, -q[3] * b.y)));
    r0.y = __fmaf_rn(q[0], a.y, __fmaf_rn(q[1], a.x, __fmaf_rn(q[2], b.y, q[3] * b.x)));
    r1.x = __fmaf_rn(q[4], a.x, __fmaf_rn(-q[5], a.y, __fmaf_rn(q[6], b.x, -q[7] * b.y)));
    r1.y = __fmaf_rn(q[4], a.y, __fmaf_rn(q[5], a.x, __fmaf_rn(q[6], b.y, q[7] * b.x)));
    a = r0; b = r1;
  }
};

template <> struct Arith<MODE_C128_F64> {
  using G = double2;
  using S = double2;
  using Coef = CoefF64;
  static __device__ __forceinline__ S load(G v) { return v; }
  static __device__ __forceinline__ G store(S v) { return v; }
  static __device__ __forceinline__ S zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ S one() { return make_double2(1.0, 0.0); }
  static __device__ __forceinline__ void coef(Coef &c, const DevGate &g) {
    const double2 *v = reinterpret_cast<const double2 *>(g.q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 t = v[i];
      c.q[2 * i] = t.x;
      c.q[2 * i + 1] = t.y;
    }
  }
  static __device__ __forceinline__ S row4(const Coef &c, S x0, S x1, S x2, S x3) {
    const double *q = c.q;
    S r;
    r.x = __fma_rn(q[0], x0.x, __fma_rn(-q[1], x0.y, __fma_rn(q[2], x1.x, __fma_rn(-q[3], x1.y,
          __fma_rn(q[4], x2.x, __fma_rn(-q[5], x2.y, __fma_rn(q[6], x3.x, -q[7] * x3.y)))))));
    r.y = __fma_rn(q[0], x0.y, __fma_rn(q[1], x0.x, __fma_rn(q[2], x1.y, __fma_rn(q[3], x1.x,
          __fma_rn(q[4], x2.y, __fma_rn(q[5], x2.x, __fma_rn(q[6], x3.y, q[7] * x3.x)))))));
    return r;
  }
  static __device__ __forceinline__ S cmul(const Coef &c, int j, S a) {
    const double qr = c.q[2 * j], qi = c.q[2 * j + 1];
    return make_double2(__fma_rn(qr, a.x, -qi * a.y), __fma_rn(qr, a.y, qi * a.x));
  }
  static __device__ __forceinline__ void pair(const Coef &c, S &a, S &b) {
    const double *q = c.q;
    S r0, r1;
    r0.x = __fma_rn(q[0], a.x, __fma_rn(-q[1], a.y, __fma_rn(q[2], b.x, -q[3] * b.y)));
    r0.y = __fma_rn(q[0], a.y, __fma_rn(q[1], a.x, __fma_rn(q[2], b.y, q[3] * b.x)));
    r1.x = __fma_rn(q[4], a.x, __fma_rn(-q[5], a.y, __fma_rn(q[6], b.x, -q[7] * b.y)));
    r1.y = __fma_rn(q[4], a.y, __fma_rn(q[5], a.x, __fma_rn(q[6], b.y, q[7] * b.x)));
    a = r0; b = r1;
  }
};

// Working form of a DF32 amplitude: (re.hi, re.lo, im.hi, im.lo).
template <> struct Arith<MODE_C128_DF32> {
  using G = double2;
  using S = float4;
  using Coef = CoefDF;
  static __device__ __forceinline__ S load(G v) {
    const dfv r = df_split(v.x), i = df_split(v.y);
    return make_float4(r.h, r.l, i.h, i.l);
  }
  static __device__ __forceinline__ G store(S v) { return make_double2(df_combine(v.x, v.y), df_combine(v.z, v.w)); }
  static __device__ __forceinline__ S zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ S one() { return make_float4(1.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void coef(Coef &c, const DevGate &g) {
    const float4 *h = reinterpret_cast<const float4 *>(g.qh), *m = reinterpret_cast<const float4 *>(g.qm),
                 *l = reinterpret_cast<const float4 *>(g.ql);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float4 a = h[i], b = m[i], d = l[i];
      c.h[4 * i] = a.x; c.h[4 * i + 1] = a.y; c.h[4 * i + 2] = a.z; c.h[4 * i + 3] = a.w;
      c.m[4 * i] = b.x; c.m[4 * i + 1] = b.y; c.m[4 * i + 2] = b.z; c.m[4 * i + 3] = b.w;
      c.l[4 * i] = d.x; c.l[4 * i + 1] = d.y; c.l[4 * i + 2] = d.z; c.l[4 * i + 3] = d.w;
    }
  }
  // Two-qubit rows read their 24 coefficient floats from the record as they are used (L1 hits), which keeps
  // the quadruple update within the register budget.
  static __device__ __forceinline__ S row4g(const DevGate &g, S x0, S x1, S x2, S x3) {
    const dfv xr[4] = {{x0.x, x0.y}, {x1.x, x1.y}, {x2.x, x2.y}, {x3.x, x3.y}};
    const dfv xi[4] = {{x0.z, x0.w}, {x1.z, x1.w}, {x2.z, x2.w}, {x3.z, x3.w}};
    auto q = [&](int i, bool neg) {
      const float h = g.qh[i], m = g.qm[i], l = g.ql[i];
      return neg ? q3{-h, -m, -l} : q3{h, m, l};
    };
    const q3 qre[8] = {q(0, false), q(1, true), q(2, false), q(3, true), q(4, false), q(5, true), q(6, false), q(7, true)};
    const dfv are[8] = {xr[0], xi[0], xr[1], xi[1], xr[2], xi[2], xr[3], xi[3]};
    const dfv re = df_dot8(qre, are);
    const q3 qim[8] = {q(0, false), q(1, false), q(2, false), q(3, false), q(4, false), q(5, false), q(6, false), q(7, false)};
    const dfv aim[8] = {xi[0], xr[0], xi[1], xr[1], xi[2], xr[2], xi[3], xr[3]};
    const dfv im = df_dot8(qim, aim);
    return make_float4(re.h, re.l, im.h, im.l);
  }
  static __device__ __forceinline__ S row4(const Coef &c, S x0, S x1, S x2, S x3) {
    const dfv xr[4] = {{x0.x, x0.y}, {x1.x, x1.y}, {x2.x, x2.y}, {x3.x, x3.y}};
    const dfv xi[4] = {{x0.z, x0.w}, {x1.z, x1.w}, {x2.z, x2.w}, {x3.z, x3.w}};
    const q3 qre[8] = {e(c, 0), ne(c, 1), e(c, 2), ne(c, 3), e(c, 4), ne(c, 5), e(c, 6), ne(c, 7)};
    const dfv are[8] = {xr[0], xi[0], xr[1], xi[1], xr[2], xi[2], xr[3], xi[3]};
    const q3 qim[8] = {e(c, 0), e(c, 1), e(c, 2), e(c, 3), e(c, 4), e(c, 5), e(c, 6), e(c, 7)};
    const dfv aim[8] = {xi[0], xr[0], xi[1], xr[1], xi[2], xr[2], xi[3], xr[3]};
    const dfv re = df_dot8(qre, are), im = df_dot8(qim, aim);
    return make_float4(re.h, re.l, im.h, im.l);
  }
  // Entry e of the matrix (0 = q11 re, 1 = q11 im, ..., 7 = q22 im), optionally negated.
  static __device__ __forceinline__ q3 e(const Coef &c, int i) { return q3{c.h[i], c.m[i], c.l[i]}; }
  static __device__ __forceinline__ q3 ne(const Coef &c, int i) { return q3{-c.h[i], -c.m[i], -c.l[i]}; }
  static __device__ __forceinline__ S cmul(const Coef &c, int j, S a) {
    const dfv ar{a.x, a.y}, ai{a.z, a.w};
    const dfv xr = df_dot2(e(c, 2 * j), ar, ne(c, 2 * j + 1), ai);
    const dfv xi = df_dot2(e(c, 2 * j), ai, e(c, 2 * j + 1), ar);
    return make_float4(xr.h, xr.l, xi.h, xi.l);
  }
  // The dense pair update with both outputs in the two lanes of packed FP32x2 instructions: lane 0 computes
  // a' = q11 a + q12 b, lane 1 computes b' = q21 a + q22 b, with the same compensated dot product per lane.
  static __device__ __forceinline__ void pair(const Coef &c, S &a, S &b) {
    const q3p q11r = qp(c, 0, 4), q11i = qp(c, 1, 5), q12r = qp(c, 2, 6), q12i = qp(c, 3, 7);
    const dfv2 re = df_dot4_2<true>(q11r, bx(a.x, a.y), q11i, bx(a.z, a.w), q12r, bx(b.x, b.y), q12i, bx(b.z, b.w));
    const dfv2 im = df_dot4_2<false>(q11r, bx(a.z, a.w), q11i, bx(a.x, a.y), q12r, bx(b.z, b.w), q12i, bx(b.x, b.y));
    a = make_float4(re.h.x, re.l.x, im.h.x, im.l.x);
    b = make_float4(re.h.y, re.l.y, im.h.y, im.l.y);
  }
  // The same update in scalar instructions, negated entries folded into the terms (one correction
  // accumulator per output): the rounding of the corrections differs from the packed form in the last
  // bits of the low word, within the same error bound.
  static __device__ __forceinline__ void pair_scalar(const Coef &c, S &a, S &b) {
    const dfv ar{a.x, a.y}, ai{a.z, a.w}, br{b.x, b.y}, bi{b.z, b.w};
    const dfv o0r = df_dot4(e(c, 0), ar, ne(c, 1), ai, e(c, 2), br, ne(c, 3), bi);
    const dfv o0i = df_dot4(e(c, 0), ai, e(c, 1), ar, e(c, 2), bi, e(c, 3), br);
    const dfv o1r = df_dot4(e(c, 4), ar, ne(c, 5), ai, e(c, 6), br, ne(c, 7), bi);
    const dfv o1i = df_dot4(e(c, 4), ai, e(c, 5), ar, e(c, 6), bi, e(c, 7), br);
    a = make_float4(o0r.h, o0r.l, o0i.h, o0i.l);
    b = make_float4(o1r.h, o1r.l, o1i.h, o1i.l);
  }
  // Lane pair (entry i for lane 0, entry j for lane 1) of the three-float coefficients.
  static __device__ __forceinline__ q3p qp(const Coef &c, int i, int j) {
    return q3p{make_float2(c.h[i], c.h[j]), make_float2(c.m[i], c.m[j]), make_float2(c.l[i], c.l[j])};
  }
  static __device__ __forceinline__ dfv2 bx(float h, float l) { return dfv2{bcast(h), bcast(l)}; }
};

// Apply one gate class to an amplitude pair (a = target bit 0, b = target bit 1).
// PACK = false selects the scalar double-float pair update (same results, more instructions, fewer registers).
template <int MODE, bool PACK = true>
__device__ __forceinline__ void apply_pair(uint32_t cls, const typename Arith<MODE>::Coef &c,
                                           typename Arith<MODE>::S &a, typename Arith<MODE>::S &b) {
  using M = Arith<MODE>;
  switch (cls) {
    case GC_GENERAL:
      if constexpr (MODE == MODE_C128_DF32 && !PACK) M::pair_scalar(c, a, b);
      else M::pair(c, a, b);
      break;
    case GC_DIAG: a = M::cmul(c, 0, a); b = M::cmul(c, 3, b); break;
    case GC_PHASE: b = M::cmul(c, 3, b); break;
    case GC_ANTIDIAG: { const auto t = M::cmul(c, 1, b); b = M::cmul(c, 2, a); a = t; } break;
    default: { const auto t = a; a = b; b = t; } break;  // GC_X
  }
}

} // namespace svi
