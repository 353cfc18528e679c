// dfloat.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2 (about 48 significant
// bits).  The FP64-accurate parts of the mixed-precision solver (the FP64
// residual, e^u of the FP64 iterate, the ghost values) run on the FP32 pipes
// with it: on GB300 an FP64 instruction costs the issue slots of ~64 FP32 ones.
//
// The building blocks are the error-free transformations of Knuth (two-sum:
// a + b = s + e exactly) and Dekker (two-product, here with one FMA: a b = p + e
// exactly).  On the device every operation is written with the _rn intrinsics
// so that the compiler cannot contract or reassociate them; the same code
// compiles as host C++ (with -ffp-contract=off) for testing.
#pragma once
#include <math.h>
#include <string.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn(a, b)
#define DF_SUB(a, b) __fsub_rn(a, b)
#define DF_MUL(a, b) __fmul_rn(a, b)
#define DF_FMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_FMA(a, b, c) fmaf(a, b, c)
#endif

struct dfl {
  float hi, lo;
};

// a + b = s + e exactly (Knuth)
__host__ __device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = DF_ADD(a, b);
  const float bb = DF_SUB(s, a);
  const float e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
  return dfl{s, e};
}

// a + b = s + e exactly, valid when |a| >= |b| or a == 0
__host__ __device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = DF_ADD(a, b);
  return dfl{s, DF_SUB(b, DF_SUB(s, a))};
}

// a b = p + e exactly (Dekker's product, one FMA)
__host__ __device__ __forceinline__ dfl df_two_prod(float a, float b) {
  const float p = DF_MUL(a, b);
  return dfl{p, DF_FMA(a, b, -p)};
}

__host__ __device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }

// a + b, both double-float (the accurate two-two-sum form)
__host__ __device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = df_two_sum(a.hi, b.hi);
  const dfl t = df_two_sum(a.lo, b.lo);
  s.lo = DF_ADD(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = DF_ADD(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// a + b with error below ~2^-46 (|a| + |b|): the absolute accuracy of the
// inputs themselves, enough where the result is not needed relative to a
// cancelled sum
__host__ __device__ __forceinline__ dfl df_add_abs(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, DF_ADD(s.lo, DF_ADD(a.lo, b.lo)));
}

// a + b with b a float
__host__ __device__ __forceinline__ dfl df_add_f(dfl a, float b) {
  dfl s = df_two_sum(a.hi, b);
  s.lo = DF_ADD(s.lo, a.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

// a b, both double-float (the lo*lo term is below the result's precision)
__host__ __device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  dfl p = df_two_prod(a.hi, b.hi);
  p.lo = DF_FMA(a.hi, b.lo, DF_FMA(a.lo, b.hi, p.lo));
  return df_fast_two_sum(p.hi, p.lo);
}

// a b with b a float
__host__ __device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
  dfl p = df_two_prod(a.hi, b);
  p.lo = DF_FMA(a.lo, b, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

// a times a power of two (exact while both parts stay normal)
__host__ __device__ __forceinline__ dfl df_ldexp(dfl a, int k) {
  return dfl{ldexpf(a.hi, k), ldexpf(a.lo, k)};
}

// conversions with FP64 (these cost FP64 instructions: use at the edges only)
__host__ __device__ __forceinline__ dfl df_from_double(double x) {
  const float hi = (float)x;
  return dfl{hi, (float)(x - (double)hi)};
}
__host__ __device__ __forceinline__ double df_to_double(dfl a) {
  return (double)a.hi + (double)a.lo;
}

// ---- conversions on the integer pipes --------------------------------------
// On GB300 a conversion to or from FP64 issues on the FP64 pipe, like an FP64
// add.  Kernels that only move values between FP64 arrays and FP32 or
// double-float ones use these instead: they take the IEEE bit patterns apart
// with integer instructions.  FP32 results that would be subnormal are
// flushed to zero (|x| < 2^-126), and the low part of a pair is dropped when
// |x| < 2^-74: losses far below the accuracy of every value they carry here.
__host__ __device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double dfrombits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned fbits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned b;
  memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float ffrombits(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, 4);
  return x;
#endif
}

// FP64 -> FP32, rounded to nearest even (the cast's result wherever it is a
// normal number): the 29 dropped significand bits are rounded into the kept
// ones by an integer add, whose carry moves on into the exponent.
__host__ __device__ __forceinline__ float f_from_double_bits(double x) {
  unsigned long long b = dbits(x);
  const unsigned s = (unsigned)(b >> 63) << 31;
  b &= 0x7fffffffffffffffULL;
  if (b >= 0x7ff0000000000000ULL)  // inf, nan
    return ffrombits(s | 0x7f800000u | (b > 0x7ff0000000000000ULL ? 0x400000u : 0u));
  b += 0x0fffffffULL + ((b >> 29) & 1);
  const int e = (int)(b >> 52) - 1023 + 127;
  if (e <= 0) return ffrombits(s);
  if (e >= 255) return ffrombits(s | 0x7f800000u);
  return ffrombits(s | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// FP32 -> FP64, exact (subnormal inputs flushed to zero)
__host__ __device__ __forceinline__ double d_from_float_bits(float x) {
  const unsigned b = fbits(x);
  const unsigned long long s = (unsigned long long)(b >> 31) << 63;
  const int e = (int)((b >> 23) & 255);
  const unsigned long long m = (unsigned long long)(b & 0x7fffffu) << 29;
  if (e == 0) return dfrombits(s);
  if (e == 255) return dfrombits(s | 0x7ff0000000000000ULL | m);
  return dfrombits(s | ((unsigned long long)(e - 127 + 1023) << 52) | m);
}

// FP64 -> double-float: hi = x rounded to FP32, lo = x - hi rounded to FP32
// (the pair df_from_double forms).  With M the 53-bit significand and E the
// exponent, x - hi = (M - H 2^29) 2^(E-52), H = hi's 24-bit significand: an
// integer below 2^28 in magnitude, converted once and scaled exactly.
__host__ __device__ __forceinline__ dfl df_from_double_bits(double x) {
  const unsigned long long b = dbits(x) & 0x7fffffffffffffffULL;
  const float hi = f_from_double_bits(x);
  const int E = (int)(b >> 52) - 1023;
  if (E < -74 || E > 127 || fbits(hi) << 1 == 0u || (fbits(hi) & 0x7f800000u) == 0x7f800000u)
    return dfl{hi, 0.f};
  const long long M = (long long)((b & 0xfffffffffffffULL) | 0x10000000000000ULL);
  // hi's significand scaled to x's exponent (a round-up to 2^24 is included)
  const long long H = (long long)((fbits(hi) & 0x7fffffu) | 0x800000u)
                      << (((fbits(hi) >> 23) & 255) - 127 - E);
  const float r = (float)(int)(M - (H << 29));  // |M - H 2^29| <= 2^28
  const float sc = ffrombits((unsigned)(E - 52 + 127) << 23);
  const float lo = DF_MUL(r, sc);
  return (long long)dbits(x) < 0 ? dfl{hi, -lo} : dfl{hi, lo};
}

// double-float -> FP64: the exact widenings of both parts, one FP64 add
__host__ __device__ __forceinline__ double df_to_double_bits(dfl a) {
  return d_from_float_bits(a.hi) + d_from_float_bits(a.lo);
}

// 2^(j/32), j = 0..31, as double-float pairs: the FP64 value of 2^(j/32)
// (53 bits, more than the pair's 48) split into its two nearest floats
#define DF_EXP2_TABLE                                                                       \
  {                                                                                         \
    {1.0f, 0.0f}, {1.0218971967697144f, -4.811559861650494e-08f},                          \
        {1.0442737340927124f, 4.8334701574503924e-08f},                                     \
        {1.0671404600143433f, -5.9337519786595294e-08f},                                    \
        {1.0905077457427979f, -1.3077539939843064e-08f},                                    \
        {1.114386796951294f, -5.435540018083884e-08f},                                      \
        {1.1387885808944702f, 5.386222312608879e-08f},                                      \
        {1.1637248992919922f, -4.051441493402308e-08f},                                     \
        {1.1892070770263672f, 3.797635272917432e-08f},                                      \
        {1.215247392654419f, -3.267394887984665e-08f},                                      \
        {1.2418577671051025f, 4.496838101886169e-08f},                                      \
        {1.2690509557724f, 1.419333317542737e-09f},                                         \
        {1.2968395948410034f, -4.018999533172973e-08f},                                     \
        {1.3252366781234741f, -3.496373324196611e-08f},                                     \
        {1.3542555570602417f, -1.0123349269974824e-08f},                                    \
        {1.3839099407196045f, -5.875577357983275e-08f},                                     \
        {1.4142135381698608f, 2.4203234971764687e-08f},                                     \
        {1.4451807737350464f, 3.324199937537742e-08f},                                      \
        {1.4768261909484863f, -4.500898853621038e-08f},                                     \
        {1.5091644525527954f, -2.4959373234878512e-08f},                                    \
        {1.5422108173370361f, 8.070904833346049e-09f},                                      \
        {1.5759809017181396f, -5.661025426206834e-08f},                                     \
        {1.610490322113037f, 9.836217174097328e-09f},                                       \
        {1.6457555294036865f, -5.124972091152813e-08f},                                     \
        {1.6817928552627563f, -2.4755326677450284e-08f},                                    \
        {1.7186193466186523f, -4.8496175963919086e-08f},                                    \
        {1.7562521696090698f, -9.235770370707996e-09f},                                     \
        {1.7947090864181519f, -1.141504490931311e-08f},                                     \
        {1.8340080976486206f, -1.1239277952768134e-08f},                                    \
        {1.8741676807403564f, -4.663005626071026e-08f},                                     \
        {1.9152065515518188f, 9.845328108326612e-09f},                                      \
    {                                                                                       \
      1.9571441411972046f, -1.7021804410433106e-08f                                         \
    }                                                                                       \
  }

#ifdef __CUDACC__
static __constant__ dfl kDfExp2Tab[32] = DF_EXP2_TABLE;
#endif
static const dfl kDfExp2TabHost[32] = DF_EXP2_TABLE;
#ifdef __CUDA_ARCH__
#define DF_TAB(j) kDfExp2Tab[j]
#else
#define DF_TAB(j) kDfExp2TabHost[j]
#endif

// e^x for a double-float x with |x| < 87 (the FP32 range of the result), by
// Tang's table-driven method (P. T. P. Tang, ACM TOMS 15 (1989) 144) with a
// Cody-Waite split of the reduction constant (Cody & Waite, "Software Manual
// for the Elementary Functions", 1980), both restated for float pairs:
// x = n ln2/32 + r with n = round(32 x / ln2) and |r| <= ln2/64; e^r from its
// Taylor series through r^7/7! (the omitted terms are below 5e-21 relative);
// e^x = 2^(n div 32) 2^((n mod 32)/32) e^r.  ln2/32 is split as c1 + c2 + c3 + c4:
// c1 and c2 carry 12 significant bits, so n c1 and n c2 are exact for
// |n| < 2^12; n c3 is formed exactly as a two-product; n c4 < 1.2e-14.
__host__ __device__ __forceinline__ dfl df_exp(dfl x) {
  const float kInvL = 46.16624069213867f;  // 32 / ln 2
  const float c1 = 0.02165985107421875f;
  const float c2 = 9.9837779998779297e-07f;
  const float c3 = -5.9520444128935424e-11f;
  const float c4 = -2.7447449183091686e-18f;
  const float nf = rintf(DF_MUL(x.hi, kInvL));
  const int n = (int)nf;
  dfl r = df_add_f(x, -DF_MUL(nf, c1));
  r = df_add_f(r, -DF_MUL(nf, c2));
  r = df_sub(r, df_two_prod(nf, c3));
  r = df_add_f(r, -DF_MUL(nf, c4));
  // e^r = 1 + r (1 + r/2 (1 + r/3 (1 + r/4 (1 + r/5 (1 + r/6 (1 + r/7))))));
  // the inner four brackets enter scaled by r^3/6 < 2.2e-7: FP32 suffices there
  const float rh = r.hi;
  float q = DF_FMA(DF_MUL(rh, 1.f / 7.f), 1.f, 1.f);
  q = DF_FMA(DF_MUL(rh, q), 1.f / 6.f, 1.f);
  q = DF_FMA(DF_MUL(rh, q), 1.f / 5.f, 1.f);
  q = DF_FMA(DF_MUL(rh, q), 1.f / 4.f, 1.f);
  dfl t = df_add_f(df_mul_f(r, DF_MUL(q, 1.f / 3.f)), 1.f);  // 1 + r/3 q
  t = df_add_f(df_mul(df_mul_f(r, 0.5f), t), 1.f);           // 1 + r/2 t
  t = df_add_f(df_mul(r, t), 1.f);                            // e^r
  const int j = n & 31, k = (n - j) / 32;
  return df_ldexp(df_mul(t, DF_TAB(j)), k);
}

// 1/sqrt(a) for a > 0: an FP32 estimate y, then one Newton step
// y + y (1 - a y^2)/2 with a y^2 formed in double-float (relative error about
// 1.5 times the square of the estimate's, ~1e-13)
__host__ __device__ __forceinline__ dfl df_rsqrt(dfl a) {
#ifdef __CUDA_ARCH__
  const float y = rsqrtf(a.hi);
#else
  const float y = 1.f / sqrtf(a.hi);
#endif
  const dfl y2 = df_two_prod(y, y);
  const dfl ay2 = df_mul(a, y2);
  const dfl d = df_add_f(df_neg(ay2), 1.f);  // 1 - a y^2, small
  return df_two_sum(y, DF_MUL(DF_MUL(0.5f, y), d.hi));
}
