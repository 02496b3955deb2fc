// dword.cuh -- double-word ("float-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum h + l of two FP32 numbers with
// |l| <= ulp(h) / 2: about 48 significant bits (unit roundoff u^2 = 2^-48
// with u = 2^-24).  GB300 issues FP32 at 64 times its FP64 rate (128 against
// 2 lanes per clock per SM), so operations of 3-11 FP32 instructions still
// run several times faster than native FP64 ones, with a rounding error
// about 30 times that of FP64.
//
// Building blocks (every FP32 operation written with an explicit-rounding
// intrinsic so that the compiler neither contracts nor reorders them):
//   2Sum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum (Dekker 1971), 2Prod with an
//   FMA; the double-word sum ("sloppy" form), products and reciprocal follow
//   Joldes, Muller & Popescu, "Tight and rigorous error bounds for basic
//   building blocks of double-word arithmetic", ACM TOMS 44(2), 2017.  The
//   sloppy sum has relative error ~3u^2 for operands of one sign and an
//   absolute error ~u^2 (|x| + |y|) under cancellation: the same kind of
//   bound as a binary64 sum of operands that carry their own rounding.
//
// Range: values below 2^-126 in magnitude convert to zero and magnitudes
// must stay below 2^127; lower parts below 2^-126 are flushed.  The solver's
// states, geometry and fluxes are many orders of magnitude inside that range.
#pragma once
#include <cuda_runtime.h>

namespace pmg {

struct dw {
  float h, l;
};

// Host side: nearest double-word of a binary64 constant.
inline dw dw_const(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

#ifdef __CUDACC__

__device__ __forceinline__ dw fast_two_sum(float a, float b) {   // needs |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return {s, __fsub_rn(b, z)};
}

__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  return {s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}

__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = two_sum(x.h, y.h);
  const float w = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
  return fast_two_sum(s.h, w);
}
__device__ __forceinline__ dw operator-(dw x) { return {-x.h, -x.l}; }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }

// x * y: the exact product of the high parts (2Prod) plus the two cross terms.
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float ch = __fmul_rn(x.h, y.h);
  float cl = __fmaf_rn(x.h, y.h, -ch);
  cl = __fmaf_rn(x.h, y.l, cl);
  cl = __fmaf_rn(x.l, y.h, cl);
  return fast_two_sum(ch, cl);
}

// x * 2^k is exact: scale both parts.
__device__ __forceinline__ dw scale2(dw x, float pow2) { return {__fmul_rn(x.h, pow2), __fmul_rn(x.l, pow2)}; }

// 1 / y (y normal, nonzero): the FP32 approximation t (relative error below
// 2^-22) refined by one Newton step t + t (1 - y t), with y t formed exactly
// enough in double-word; the result is within ~2^-44 of 1/y.
__device__ __forceinline__ dw rcp(dw y) {
  float t;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(y.h));
  const float ph = __fmul_rn(y.h, t);
  float pl = __fmaf_rn(y.h, t, -ph);
  pl = __fmaf_rn(y.l, t, pl);
  const float e = __fsub_rn(__fsub_rn(1.0f, ph), pl);   // 1 - ph is exact (ph within 2^-21 of 1)
  return fast_two_sum(t, __fmul_rn(t, e));
}

// sqrt(x) (x > 0 normal): s = x rsqrt(x) in FP32, then one Newton step
// s + (x - s^2) / (2 s) with s^2 formed exactly by 2Prod.
__device__ __forceinline__ dw sqrt_dw(dw x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.h));
  const float s = __fmul_rn(x.h, r);
  const float s2h = __fmul_rn(s, s);
  const float s2l = __fmaf_rn(s, s, -s2h);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.h, s2h), s2l), x.l);
  return fast_two_sum(s, __fmul_rn(d, __fmul_rn(0.5f, r)));
}

__device__ __forceinline__ dw abs_dw(dw x) { return x.h < 0.0f ? -x : x; }
__device__ __forceinline__ bool operator<(dw a, dw b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ dw min_dw(dw a, dw b) { return b < a ? b : a; }
__device__ __forceinline__ dw max_dw(dw a, dw b) { return a < b ? b : a; }

// Accumulator of a sum of double-word products and terms, after the Dot2
// scheme of Ogita, Rump & Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005): the products of the high parts are formed exactly
// (2Prod) and summed exactly (2Sum) into one FP32 word, every low-order term
// is gathered in a second FP32 word, and the pair is renormalised once at the
// end.  12 FP32 operations per product instead of 18 for a double-word
// multiply followed by a double-word add.
struct dw_acc {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add_prod(dw a, dw b) {
    const float ph = __fmul_rn(a.h, b.h);
    float pl = __fmaf_rn(a.h, b.h, -ph);
    pl = __fmaf_rn(a.h, b.l, pl);
    pl = __fmaf_rn(a.l, b.h, pl);
    const dw t = two_sum(s, ph);
    s = t.h;
    c = __fadd_rn(c, __fadd_rn(t.l, pl));
  }
  __device__ __forceinline__ void add(dw a) {
    const dw t = two_sum(s, a.h);
    s = t.h;
    c = __fadd_rn(c, __fadd_rn(t.l, a.l));
  }
  __device__ __forceinline__ dw value() const { return two_sum(s, c); }
};

// binary64 -> double-word with integer and FP32 operations only (no FP64
// instruction): h takes the leading 24 significand bits (truncated), the
// next 23 bits form l, and a Fast2Sum renormalises the pair.  The dropped
// six bits (of the 52 fraction bits) give a relative error below 2^-46.
__device__ __forceinline__ dw dw_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi32 = (unsigned int)(b >> 32), lo32 = (unsigned int)b;
  const unsigned int sgn = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  const unsigned int mh = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const float h = e >= 897 ? __uint_as_float(sgn | ((unsigned int)(e - 896) << 23) | mh) : 0.0f;
  // the remaining 29 bits r, without its last six, as an exact FP32 integer
  // (magic-number conversion), times 2^(e - 1075 + 6) with x's sign
  const float rf = __fsub_rn(__uint_as_float(0x4b000000u | ((lo32 & 0x1fffffffu) >> 6)), 8388608.0f);
  const float sc = __uint_as_float(sgn | ((unsigned int)(e - 942) << 23));
  const float l = e >= 943 ? __fmul_rn(rf, sc) : 0.0f;
  return fast_two_sum(h, l);
}

// FP32 -> binary64 bit pattern (normal numbers and zero; FP32 denormals,
// which never occur here in a high part, read as zero).
__device__ __forceinline__ double f32_bits_to_double(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = (u >> 23) & 0xffu;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(ex + 896u) << 52) | m;
  return ex ? __longlong_as_double((long long)bits) : 0.0;
}

// double-word -> binary64: h + l rounded once (one FP64 addition).
__device__ __forceinline__ double dw_to_double(dw x) {
  return f32_bits_to_double(x.h) + f32_bits_to_double(x.l);
}
#endif  // __CUDACC__

}  // namespace pmg
