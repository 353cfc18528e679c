// Host check of the double-float primitives (paper_1305_2418_gb300/csrc/dfloat.cuh)
// against long double: prints the largest relative error of each operation
// over seeded random operands.
#include <cmath>
#include <cstdio>
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
  std::printf("%.6e %.6e %.6e %.6e %.6e\n", e_conv, e_add, e_mul, e_exp, e_rsqrt);
  return 0;
}
