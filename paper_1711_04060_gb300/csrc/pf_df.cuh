// pf_df.cuh -- double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits, computed entirely on the FP32 pipes.  The building blocks
// are the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum, FastTwoSum and the
// FMA form of TwoProduct; the exponential follows Tang's table-driven method (ACM TOMS 15, 1989): a
// reduction x = (64 m + j) ln2/64 + r with |r| <= ln2/128, a short series for e^r and a table of 2^(j/64).
//
// On GB300 the FP64 pipe issues about 1/64 of the FP32 rate, so a pointwise kernel whose arithmetic is
// double-float instead of FP64 runs far more operations per clock while keeping about 1e-14 relative accuracy.
// The functions are __host__ __device__ so the same code can be checked on the CPU against exact values.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define PF_HD __host__ __device__ __forceinline__
#else
#define PF_HD inline
#endif

namespace pf {

struct dfl {
  float hi, lo;
};

// Rounded-to-nearest float operations that the compiler may not fuse or reorder (an FMA contraction
// would break the error-free transformations below).
PF_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
PF_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
PF_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
PF_HD float f_fma(float a, float b, float c) { return fmaf(a, b, c); }

PF_HD float f_from_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

// TwoSum (Knuth): s + e = a + b exactly.
PF_HD dfl two_sum(float a, float b) {
  const float s = f_add(a, b);
  const float bb = f_sub(s, a);
  const float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
  return {s, e};
}

// FastTwoSum (Dekker), valid when |a| >= |b| or a = 0: s + e = a + b exactly.
PF_HD dfl fast_two_sum(float a, float b) {
  const float s = f_add(a, b);
  return {s, f_sub(b, f_sub(s, a))};
}

// TwoProduct with an FMA: p + e = a * b exactly.
PF_HD dfl two_prod(float a, float b) {
  const float p = f_mul(a, b);
  return {p, f_fma(a, b, -p)};
}

// a + b, both double-float, with both parts' rounding errors carried (accurate under cancellation).
PF_HD dfl df_add(dfl a, dfl b) {
  dfl s = two_sum(a.hi, b.hi);
  const dfl t = two_sum(a.lo, b.lo);
  s.lo = f_add(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = f_add(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

PF_HD dfl df_add_f(dfl a, float b) {
  dfl s = two_sum(a.hi, b);
  s.lo = f_add(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

PF_HD dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

PF_HD dfl df_mul(dfl a, dfl b) {
  dfl p = two_prod(a.hi, b.hi);
  p.lo = f_fma(a.hi, b.lo, p.lo);
  p.lo = f_fma(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

PF_HD dfl df_mul_f(dfl a, float b) {
  dfl p = two_prod(a.hi, b);
  p.lo = f_fma(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// ln 2 / 64 as C1 + C2 + C3: C1 has 11 significant bits, so k * C1 is exact for |k| < 2^13; C2 and C3
// carry the next 48 bits.  Derived from ln 2 = sum_k 1 / (k 2^k) in exact arithmetic; the split leaves
// 3.6e-21 per unit of k.
constexpr float LN2_64_C1 = 0x1.62cp-7f;
constexpr float LN2_64_C2 = 0x1.217f7ep-18f;
constexpr float LN2_64_C3 = -0x1.c610cap-43f;
constexpr float INV_LN2_64 = 0x1.715476p+6f;  // 64 / ln 2, only used to pick k

// Table of 2^(j/64), j = 0..63, as double-float pairs (hi, lo).
struct Exp2Table {
  float hi[64], lo[64];
};

// The table from the host's exp2 in double (correct to about 1e-16), split into float pairs.
inline Exp2Table make_exp2_table() {
  Exp2Table t;
  for (int j = 0; j < 64; ++j) {
    const double v = exp2((double)j / 64.0);
    t.hi[j] = (float)v;
    t.lo[j] = (float)(v - (double)t.hi[j]);
  }
  return t;
}

// e^x for a double-float x: relative error about 1e-14 for x.hi in [-70, 88].  Below -70 the low part of the
// result is subnormal, so the relative error grows to 2^-24 while the absolute error stays below 2^-125; below
// -87 (e^x < 2^-125) the result is 0.  The callers sum terms of order one, for which neither matters.  Above
// 88 the result is +inf.
PF_HD dfl df_exp(dfl x, const float* thi, const float* tlo) {
  if (!(x.hi >= -87.0f)) return {0.0f, 0.0f};
  if (x.hi > 88.0f) return {INFINITY, 0.0f};
  const float kf = rintf(f_mul(x.hi, INV_LN2_64));
  const int k = (int)kf;
  // r = x - k ln2/64 in double-float: x.hi - k C1 is exact (Sterbenz), k C2 by TwoProduct
  const float r1 = f_sub(x.hi, f_mul(kf, LN2_64_C1));
  const dfl p2 = two_prod(kf, LN2_64_C2);
  dfl r = two_sum(r1, -p2.hi);
  r = df_add_f(r, x.lo);  // x.lo reaches ulp(x.hi) / 2, far above ulp(r.hi): added without loss
  r.lo = f_sub(r.lo, f_fma(kf, LN2_64_C3, p2.lo));
  r = fast_two_sum(r.hi, r.lo);
  // e^r - 1 = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720) + O(r^7), |r| < 0.0055: the first two
  // terms in double-float, the tail (below 2.7e-8) in FP32
  dfl sq = two_prod(r.hi, r.hi);
  sq.lo = f_fma(2.0f * r.hi, r.lo, sq.lo);
  const dfl half_sq = {0.5f * sq.hi, 0.5f * sq.lo};
  const float rh = r.hi;
  const float poly = f_fma(rh, f_fma(rh, f_fma(rh, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f), 1.0f / 6.0f);
  const float tail = f_mul(f_mul(rh, sq.hi), poly);
  dfl em1 = df_add(r, half_sq);
  em1 = df_add_f(em1, tail);
  // 1 + em1, |em1| < 0.0055
  dfl e = two_sum(1.0f, em1.hi);
  e.lo = f_add(e.lo, em1.lo);
  e = fast_two_sum(e.hi, e.lo);
  const int j = k & 63, m = k >> 6;  // k = 64 m + j (arithmetic shift: floor division)
  const dfl y = df_mul({thi[j], tlo[j]}, e);
  // times 2^m, m in [-126, 126]: exact scaling of both parts
  const float sc = f_from_bits((uint32_t)(m + 127) << 23);
  return {f_mul(y.hi, sc), f_mul(y.lo, sc)};
}

// The bit pattern of a double (no arithmetic).
PF_HD uint64_t d_bits(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u;
  memcpy(&u, &v, 8);
  return u;
#endif
}

// A double as a double-float pair without FP64 arithmetic (on GB300 a conversion from double issues on the slow
// FP64 pipe; this split uses integer operations, one integer-to-float conversion and FP32 multiplications).  For
// v = (1.m) 2^E: hi = v with its 52-bit mantissa cut to the first 23 bits, lo = the remaining 29 bits as an integer
// rounded to FP32 and scaled by 2^(E-52); FastTwoSum then gives the usual |lo| <= ulp(hi) / 2.  Relative error at
// most 2^-48 for 2^-97 <= |v| <= the largest float; for 2^-126 <= |v| < 2^-97 lo loses bits (absolute error below
// 2^-149), below 2^-126 the pair is a signed zero; above the largest float hi is a signed infinity once |v|
// reaches it plus half its unit, as a conversion to FP32 would round; NaN gives a NaN.
PF_HD dfl df_from_double_bits(double v) {
  const uint64_t u = d_bits(v);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ffu);
  const uint64_t m = u & 0xfffffffffffffull;
  if (e == 0x7ff) return {f_from_bits(sign | 0x7f800000u | (m ? 0x400000u : 0u)), 0.0f};
  const int E = e - 1023;
  if (E < -126) return {f_from_bits(sign), 0.0f};
  if (E > 127) return {f_from_bits(sign | 0x7f800000u), 0.0f};
  const float hi = f_from_bits(sign | ((uint32_t)(E + 127) << 23) | (uint32_t)(m >> 29));
  const uint32_t rest = (uint32_t)(m & 0x1fffffffu);
  float lo = (float)rest;  // at most 29 bits: rounded to 24
  // times 2^(E-52), E - 52 in [-178, 75]: one power-of-two factor when it is a normal float, else two
  const int k = E - 52;
  if (k >= -126) {
    lo = f_mul(lo, f_from_bits((uint32_t)(k + 127) << 23));
  } else {
    lo = f_mul(f_mul(lo, f_from_bits((uint32_t)(-64 + 127) << 23)), f_from_bits((uint32_t)(k + 64 + 127) << 23));
  }
  if (sign) lo = -lo;
  return fast_two_sum(hi, lo);
}

// The residual r = b + sum_k f_k q_k - d x of one row of a 7-point operator (nk couplings f_k to the neighbour
// values q_k, diagonal d, the node's value x), from FP64 inputs in double-float on the FP32 pipes: each input
// split by df_from_double_bits, the terms added in the order b, f_0 q_0, ..., f_{nk-1} q_{nk-1}, -d x.  The error
// stays within about 2^-44 (|b| + sum_k |f_k q_k| + |d x|) for inputs in the range df_from_double_bits keeps to
// 2^-48, and products within the float range.
PF_HD dfl df_residual_row(double b, double d, double x, const double* f, const double* q, int nk) {
  dfl r = df_from_double_bits(b);
  for (int k = 0; k < nk; ++k) r = df_add(r, df_mul(df_from_double_bits(f[k]), df_from_double_bits(q[k])));
  return df_add(r, df_neg(df_mul(df_from_double_bits(d), df_from_double_bits(x))));
}

}  // namespace pf
