// Host check of the double-float primitives (paper_1305_2418_gb300/csrc/dfloat.cuh)
// against long double: prints the largest relative error of each operation
// over seeded random operands.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../paper_1305_2418_gb300/csrc/dfloat.cuh"

static long double val(dfl a) { return (long double)a.hi + (long double)a.lo; }

int main() {
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double e_add = 0, e_mul = 0, e_exp = 0, e_rsqrt = 0, e_conv = 0;
  for (int i = 0; i < 1000000; ++i) {
    const double a = U(g) * std::pow(10.0, 3 * U(g)), b = U(g) * std::pow(10.0, 3 * U(g));
    const dfl A = df_from_double(a), B = df_from_double(b);
    e_conv = std::fmax(e_conv, std::fabs((df_to_double(A) - a) / a));
    const long double s = val(A) + val(B);
    if (fabsl(s) > 1e-6L * (fabsl(val(A)) + fabsl(val(B))))
      e_add = std::fmax(e_add, (double)fabsl((val(df_add(A, B)) - s) / s));
    const long double p = val(A) * val(B);
    e_mul = std::fmax(e_mul, (double)fabsl((val(df_mul(A, B)) - p) / p));
    const dfl X = df_from_double(40.0 * U(g));
    const long double ex = expl(val(X));
    e_exp = std::fmax(e_exp, (double)fabsl((val(df_exp(X)) - ex) / ex));
    const dfl Q = df_from_double(std::exp(30.0 * U(g)));
    const long double rs = 1.0L / sqrtl(val(Q));
    e_rsqrt = std::fmax(e_rsqrt, (double)fabsl((val(df_rsqrt(Q)) - rs) / rs));
  }
  // the integer-pipe conversions against the C casts and df_from_double:
  // identical wherever the FP32 results are normal numbers
  long long bad_bits = 0;
  std::uniform_int_distribution<unsigned long long> R;
  for (int i = 0; i < 2000000; ++i) {
    double x;
    if (i % 4 == 0) {  // arbitrary bit patterns, |x| in [2^-74, 2^120) (pairs kept whole)
      unsigned long long b = R(g);
      const int e = 1023 - 74 + (int)(b % 194);
      b = (b & 0x800fffffffffffffULL) | ((unsigned long long)e << 52);
      memcpy(&x, &b, 8);
    } else if (i % 4 == 1) {  // values next to a rounding tie of the FP32 cast
      const float f = (float)(U(g) * std::pow(10.0, 6 * U(g)));
      const double ulp = std::ldexp(1.0, std::ilogb(f) - 23);
      x = (double)f + ulp * (0.5 + (double)((long long)(R(g) % 5) - 2) * 0x1p-30);
    } else {
      x = U(g) * std::pow(10.0, 20 * U(g));
    }
    const float f = f_from_double_bits(x);
    const float fc = (float)x;
    const dfl A = df_from_double_bits(x), B = df_from_double(x);
    const double w = d_from_float_bits(fc);
    const double back = df_to_double_bits(B);
    const bool whole = std::fabs(x) >= 0x1p-74;  // below, the low part is dropped
    if (memcmp(&f, &fc, 4) || memcmp(&A.hi, &B.hi, 4) || (whole && memcmp(&A.lo, &B.lo, 4)) ||
        w != (double)fc || back != df_to_double(B))
      ++bad_bits;
  }
  // special values: zero, infinities, nan, below the FP32 range
  const double inf = INFINITY;
  if (!(f_from_double_bits(0.0) == 0.f && f_from_double_bits(-inf) == -INFINITY &&
        std::isnan(f_from_double_bits(NAN)) && f_from_double_bits(1e-300) == 0.f &&
        f_from_double_bits(1e300) == INFINITY && df_from_double_bits(0.0).lo == 0.f &&
        std::isnan(d_from_float_bits(NAN)) && d_from_float_bits(-INFINITY) == -inf))
    ++bad_bits;
  std::printf("%.6e %.6e %.6e %.6e %.6e %lld\n", e_conv, e_add, e_mul, e_exp, e_rsqrt, bad_bits);
  return 0;
}
