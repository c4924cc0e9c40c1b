// Double-float ("df64") arithmetic on the FP32 pipes: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, giving a 48-bit significand over the FP32 exponent range.
//
// Built from error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2: s + e = a + b exactly
// in 6 flops for any a, b), FastTwoSum (Dekker 1971: exact when |a| >= |b|) and the FMA form of
// TwoProd (p + e = a * b exactly with e = fma(a, b, -p)). The high parts are always added with
// TwoSum; the final renormalisation uses FastTwoSum, whose result is exact except after a
// cancellation of the high parts, where its error stays below ~2^-47 of the operands' magnitudes
// (the normwise bound an FFT or a pointwise product needs).
//
// On GB300 an FP32 FMA issues 63x faster than an FP64 FMA, so transforms and pointwise products in
// this arithmetic run several times faster than in FP64 while staying within ~1e-14 relative error.
#pragma once
#include <cuda_runtime.h>

namespace lmvd {

struct df {
  float hi, lo;
};
struct cdf {
  df re, im;  // 16 bytes, same footprint as a complex double
};

__host__ __device__ inline df df_from_double(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}

// Split of a double into hi + lo with integer operations only (no FP64 instruction): hi takes the
// sign, exponent and the top 23 stored mantissa bits (truncation), lo the remaining 29 bits rounded
// to 24 on the FP32 pipe and scaled by two powers of two; a FastTwoSum renormalises. Relative error
// <= 2^-48 for |x| >= 2^-102; smaller magnitudes keep hi exactly and lose lo gradually (below 2^-126,
// outside the float range, the result is a signed zero). Magnitudes >= 2^128 (outside the float range)
// become a signed infinity, nan a nan. Every case stays off the FP64 pipe: the compiler may evaluate a
// short branch for all threads, so even rare cases must not use FP64 instructions.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e);
__device__ __forceinline__ df df_from_double_int(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32);
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  const unsigned sign = hi32 & 0x80000000u;
  if (e > 1150) {
    const bool nan = e == 2047 && (u & 0xFFFFFFFFFFFFFull) != 0;
    return df{__uint_as_float(nan ? 0x7FC00000u : (sign | 0x7F800000u)), 0.f};
  }
  if (e < 897) return df{__uint_as_float(sign), 0.f};
  const unsigned long long m52 = u & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m52 >> 29));
  const int k = e - 1075;                                         // lo = rem * 2^k, k in [-178, 75]
  const int ka = k >> 1, kb = k - ka;                             // 2^ka, 2^kb are normal floats
  const float sa = __uint_as_float((unsigned)(ka + 127) << 23), sb = __uint_as_float((unsigned)(kb + 127) << 23);
  // the low 29 mantissa bits as a float, rounded to nearest, on the FP32 pipe (an int-to-float
  // conversion instruction would run at the FP64 rate): both 23-bit halves are exact through the 2^23
  // trick (the float 2^23 + r has mantissa r), and one FMA rounds r1 2^23 + r0 once
  const unsigned r = (unsigned)(m52 & 0x1FFFFFFFull);
  const float f0 = __fsub_rn(__uint_as_float(0x4B000000u | (r & 0x7FFFFFu)), 8388608.0f);
  const float f1 = __fsub_rn(__uint_as_float(0x4B000000u | (r >> 23)), 8388608.0f);
  float lo = __fmul_rn(__fmul_rn(__fmaf_rn(f1, 8388608.0f, f0), sa), sb);
  lo = sign ? -lo : lo;
  float s, l;
  fast_two_sum(hi, lo, s, l);
  return df{s, l};
}

// hi + lo rounded to a double with integer operations only (no FP64 instruction). The 24-bit
// mantissa of lo is aligned to the 53-bit mantissa of hi and added (or subtracted); bits of lo below
// the double's last place are rounded to nearest (a denormal lo is handled like a normal one).
// Non-normal hi: inf and nan keep their value (lo is then irrelevant); a denormal hi (below 2^-126,
// where lo of a normalised pair is zero) is converted exactly, with its leading bit found by clz.
__device__ __forceinline__ double df_to_double_int(df a) {
  const unsigned hb = __float_as_uint(a.hi), lb = __float_as_uint(a.lo);
  const unsigned long long sgn = (unsigned long long)(hb & 0x80000000u) << 32;
  if ((hb & 0x7fffffffu) == 0) return __longlong_as_double((long long)sgn);  // a normalised pair has lo = 0 here
  int eh = (int)((hb >> 23) & 0xffu);
  if (eh == 255) {  // inf or nan
    const unsigned long long mh = (unsigned long long)(hb & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull | mh | (mh ? (1ull << 51) : 0ull)));
  }
  if (eh == 0) {  // denormal hi = m 2^-149, m < 2^23: leading bit at 31 - clz(m)
    const unsigned m = hb & 0x7fffffu;
    const int lead = 31 - __clz((int)m);                  // value = 1.f 2^(lead - 149)
    const unsigned long long frac = ((unsigned long long)m << (52 - lead)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(lead - 149 + 1023) << 52) | frac));
  }
  unsigned long long M = (unsigned long long)((hb & 0x7fffffu) | 0x800000u) << 29;  // leading bit 52
  int el = (int)((lb >> 23) & 0xffu);
  if ((lb & 0x7fffffffu) != 0 && el != 255) {
    // a denormal lo has no implicit bit and the exponent of the smallest normal
    const unsigned long long ml = (unsigned long long)((lb & 0x7fffffu) | (el ? 0x800000u : 0u));
    el = el ? el : 1;
    const int sh = 29 - (eh - el);
    unsigned long long add = 0;
    if (sh >= 0) add = ml << sh;
    else if (sh > -26) add = (ml + (1ull << (-sh - 1))) >> (-sh);
    if (((hb ^ lb) & 0x80000000u) == 0) {
      M += add;
      if (M >> 53) {
        M = (M + 1) >> 1;
        ++eh;
      }
    } else {
      M -= add;
      if (!(M >> 52)) {
        M <<= 1;
        --eh;
      }
    }
  }
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(eh + 896) << 52) | (M & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df dadd(df a, df b) {
  float s, e, r, rl;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  fast_two_sum(s, e, r, rl);
  return df{r, rl};
}
// a + b without the final renormalisation: hi + lo is the sum to the same accuracy, but lo may exceed
// ulp(hi) / 2. For intermediates that only feed another dadd (its TwoSum of the high parts is exact for
// any operands and it renormalises its result).
__device__ __forceinline__ df dadd_lazy(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ df dneg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df dsub(df a, df b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ df dmul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float r, rl;
  fast_two_sum(p, e, r, rl);
  return df{r, rl};
}
// a * b for a power of two b (exact)
__device__ __forceinline__ df dscale2(df a, float b) { return df{a.hi * b, a.lo * b}; }
// a * b + c * d with one renormalisation
__device__ __forceinline__ df ddot2(df a, df b, df c, df d) {
  const float p1 = __fmul_rn(a.hi, b.hi), e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = __fmul_rn(c.hi, d.hi), e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s, e3;
  two_sum(p1, p2, s, e3);
  float t = __fadd_rn(__fadd_rn(e1, e2), e3);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fmaf_rn(c.hi, d.lo, t);
  t = __fmaf_rn(c.lo, d.hi, t);
  float r, rl;
  fast_two_sum(s, t, r, rl);
  return df{r, rl};
}
// a * b + c * d without the final renormalisation (see dadd_lazy)
__device__ __forceinline__ df ddot2_lazy(df a, df b, df c, df d) {
  const float p1 = __fmul_rn(a.hi, b.hi), e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = __fmul_rn(c.hi, d.hi), e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s, e3;
  two_sum(p1, p2, s, e3);
  float t = __fadd_rn(__fadd_rn(e1, e2), e3);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fmaf_rn(c.hi, d.lo, t);
  t = __fmaf_rn(c.lo, d.hi, t);
  return df{s, t};
}

// complex helpers
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cdf{dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cdf{dsub(a.re, b.re), dsub(a.im, b.im)}; }
__device__ __forceinline__ cdf cadd_lazy(cdf a, cdf b) { return cdf{dadd_lazy(a.re, b.re), dadd_lazy(a.im, b.im)}; }
__device__ __forceinline__ cdf csub_lazy(cdf a, cdf b) {
  return cdf{dadd_lazy(a.re, dneg(b.re)), dadd_lazy(a.im, dneg(b.im))};
}
__device__ __forceinline__ cdf ctimes_i(cdf a) { return cdf{dneg(a.im), a.re}; }
__device__ __forceinline__ cdf cconj(cdf a) { return cdf{a.re, dneg(a.im)}; }
// v * (wr + i wi), not renormalised (the twiddle products feed only a butterfly's additions)
__device__ __forceinline__ cdf cmulw_lazy(cdf v, df wr, df wi) {
  return cdf{ddot2_lazy(v.re, wr, dneg(v.im), wi), ddot2_lazy(v.re, wi, v.im, wr)};
}

}  // namespace lmvd
