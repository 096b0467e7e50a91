// fd_df.cuh -- double-float ("df") numbers: a value held as the unevaluated sum hi + lo of two
// FP32 numbers, |lo| <= ulp(hi), about 46 significant bits (Dekker 1971).  The arithmetic uses
// the error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProduct with a fused
// multiply-add.  It serves where FP64 arithmetic would queue on the SM's narrow FP64 unit: a df
// operation costs a few tens of FP32 instructions, which this GPU issues about seventy times
// faster than FP64 ones.  The conversions to and from FP64 work on the IEEE-754 bit patterns
// (integer instructions) for the same reason; values below 2^-126 in magnitude are flushed to
// zero, and the caller keeps magnitudes far below 2^128.
//
// The functions are host+device so that a host program can check them (on the host the FP32
// operations must be compiled without contraction into FMAs).
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FD_HD __host__ __device__ __forceinline__
#else
#define FD_HD inline
#endif

namespace fd {
namespace df {

FD_HD uint64_t dbits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}
FD_HD double dfrom(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}
FD_HD uint32_t fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}
FD_HD float ffrom(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
// index of the highest set bit of x > 0
FD_HD int msb64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return 63 - __clzll((long long)x);
#else
  return 63 - __builtin_clzll(x);
#endif
}

// FP32 operations that are never contracted or reassociated.
FD_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
FD_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
FD_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
FD_HD float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return __builtin_fmaf(a, b, c);
#endif
}

// TwoSum: s + e == a + b exactly, s = fl(a + b).
FD_HD void two_sum(float a, float b, float& s, float& e) {
  s = add(a, b);
  const float bb = sub(s, a);
  e = add(sub(a, sub(s, bb)), sub(b, bb));
}

// FP64 -> (hi, lo): hi keeps the leading 24 significant bits of d (truncated), lo the next 24
// bits of the remainder d - hi (truncated), so |d - hi - lo| < 2^-46 |d|.  Integer work only.
FD_HD void split(double d, float& hi, float& lo) {
  const uint64_t b = dbits(d);
  const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const uint64_t m = b & 0xfffffffffffffull;
  const int eh = e - 1023 + 127;
  lo = ffrom(sgn);
  if (eh <= 0) {  // |d| < 2^-126, zero, FP64 subnormal
    hi = ffrom(sgn);
    return;
  }
  if (eh >= 255) {  // too large for FP32, infinity, NaN
    hi = ffrom(sgn | 0x7f800000u | (e == 2047 && m ? 0x400000u : 0u));
    return;
  }
  hi = ffrom(sgn | (uint32_t)eh << 23 | (uint32_t)(m >> 29));
  const uint64_t r = m & ((1ull << 29) - 1);  // d - hi = +-r 2^(e - 1075)
  if (r == 0) return;
  const int p = msb64(r);  // 0..28
  const int el = e - 1075 + p + 127;
  if (el <= 0) return;
  const uint32_t frac = p >= 23 ? (uint32_t)(r >> (p - 23)) : (uint32_t)(r << (23 - p));
  lo = ffrom(sgn | (uint32_t)el << 23 | (frac & 0x7fffffu));
}

// FP32 -> FP64 on the bit pattern (exact for normal numbers; FP32 subnormals become zero).
FD_HD double widen(float f) {
  const uint32_t b = fbits(f);
  const uint64_t sgn = (uint64_t)(b & 0x80000000u) << 32;
  const uint32_t ef = (b >> 23) & 0xff;
  if (ef == 0) return dfrom(sgn);
  const uint64_t ed = ef == 255 ? 2047 : (uint64_t)ef - 127 + 1023;
  return dfrom(sgn | ed << 52 | (uint64_t)(b & 0x7fffffu) << 29);
}

FD_HD double join(float hi, float lo) { return widen(hi) + widen(lo); }

// A complex df number as a float4: x = Re hi, y = Re lo, z = Im hi, w = Im lo.
struct c4 {
  float x, y, z, w;
};

FD_HD c4 csplit(double re, double im) {
  c4 r;
  split(re, r.x, r.y);
  split(im, r.z, r.w);
  return r;
}

// p + e = a * b with a, b df (the lo * lo term, below 2^-46 |a b|, is dropped).
FD_HD void prod(float ah, float al, float bh, float bl, float& p, float& e) {
  p = mul(ah, bh);
  e = fma(ah, bh, -p);
  e = fma(ah, bl, e);
  e = fma(al, bh, e);
}

// (s, t) -> normalised df
FD_HD void renorm(float s, float t, float& h, float& l) {
  h = add(s, t);
  l = sub(t, sub(h, s));
}

// g - a * b for complex df numbers.
FD_HD c4 cms(c4 g, c4 a, c4 b) {
  float p1, e1, p2, e2, p3, e3, p4, e4;
  prod(a.x, a.y, b.x, b.y, p1, e1);  // Re a Re b
  prod(a.z, a.w, b.z, b.w, p2, e2);  // Im a Im b
  prod(a.x, a.y, b.z, b.w, p3, e3);  // Re a Im b
  prod(a.z, a.w, b.x, b.y, p4, e4);  // Im a Re b
  c4 r;
  float s, t, s2, t2;
  // Re: g - Re a Re b + Im a Im b
  two_sum(g.x, -p1, s, t);
  t = add(t, sub(g.y, e1));
  two_sum(s, p2, s2, t2);
  t2 = add(t2, add(t, e2));
  renorm(s2, t2, r.x, r.y);
  // Im: g - Re a Im b - Im a Re b
  two_sum(g.z, -p3, s, t);
  t = add(t, sub(g.w, e3));
  two_sum(s, -p4, s2, t2);
  t2 = add(t2, sub(t, e4));
  renorm(s2, t2, r.z, r.w);
  return r;
}

// |r|^2 of a complex df number, as a normalised df pair.
FD_HD void abs2(c4 r, float& th, float& tl) {
  float p1, e1, p2, e2, s, e;
  prod(r.x, r.y, r.x, r.y, p1, e1);
  prod(r.z, r.w, r.z, r.w, p2, e2);
  two_sum(p1, p2, s, e);
  e = add(e, add(e1, e2));
  renorm(s, e, th, tl);
}

// 1 / t for a df t > 0 (normal range): the FP32 reciprocal refined by one Newton step in df,
// y = y0 + y0 (1 - t y0); 1 - t y0 is exact in FP32 because t y0 is within 2^-22 of 1.
FD_HD void recip(float th, float tl, float& yh, float& yl) {
#ifdef __CUDA_ARCH__
  const float y0 = __frcp_rn(th);
#else
  const float y0 = 1.0f / th;
#endif
  float p, pe;
  prod(th, tl, y0, 0.f, p, pe);
  const float e = sub(sub(1.f, p), pe);
  renorm(y0, mul(y0, e), yh, yl);
}

// a > b for normalised df pairs (the sign of the df difference).
FD_HD bool greater(float ah, float al, float bh, float bl) {
  float s, e;
  two_sum(ah, -bh, s, e);
  e = add(e, sub(al, bl));
  return add(s, e) > 0.f;
}

// a * y for a complex df a and a real df y.
FD_HD c4 scale(c4 a, float yh, float yl) {
  c4 r;
  float p, e;
  prod(a.x, a.y, yh, yl, p, e);
  renorm(p, e, r.x, r.y);
  prod(a.z, a.w, yh, yl, p, e);
  renorm(p, e, r.z, r.w);
  return r;
}

// g + c with c a plain FP32 value added to the real part.
FD_HD c4 add_re(c4 g, float c) {
  float s, t;
  two_sum(g.x, c, s, t);
  t = add(t, g.y);
  renorm(s, t, g.x, g.y);
  return g;
}

}  // namespace df
}  // namespace fd
