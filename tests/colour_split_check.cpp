// Host check of the colour-split index maps (paper_1305_2418_gb300/csrc/colour_split.cuh):
// dense levels -- pdx is a bijection onto [0, N^3) with plane = red-black colour,
// pcell inverts it, and pnb6 gives the colour-split indices of the six periodic
// neighbours (all in the other plane); oct levels -- pidx is a bijection onto
// [0, 8 n_oct) with plane = parity of the child bits and four cells per float4.
// Prints the number of violations.
#include <cstdio>
#include <vector>

#include "../paper_1305_2418_gb300/csrc/colour_split.cuh"

int main() {
  long long bad = 0;
  for (int lg = 2; lg <= 7; ++lg) {
    const int N = 1 << lg, M = N - 1;
    std::vector<int> seen((size_t)N * N * N, 0);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) {
          const unsigned t = pdx(i, j, k, lg);
          if (t >= (unsigned)(N * N * N)) { ++bad; continue; }
          ++seen[t];
          if ((t >> (3 * lg - 1)) != (unsigned)((i + j + k) & 1)) ++bad;
          int a, b, c;
          pcell(t, lg, &a, &b, &c);
          if (a != i || b != j || c != k) ++bad;
          unsigned q[6];
          pnb6(i, j, k, lg, q);
          const unsigned want[6] = {pdx((i - 1) & M, j, k, lg), pdx((i + 1) & M, j, k, lg),
                                    pdx(i, (j - 1) & M, k, lg), pdx(i, (j + 1) & M, k, lg),
                                    pdx(i, j, (k - 1) & M, lg), pdx(i, j, (k + 1) & M, lg)};
          for (int e = 0; e < 6; ++e) {
            if (q[e] != want[e]) ++bad;
            if ((q[e] >> (3 * lg - 1)) == (t >> (3 * lg - 1))) ++bad;  // other colour
          }
        }
    for (int v : seen)
      if (v != 1) ++bad;
  }
  for (long long no : {1LL, 3LL, 1000LL}) {
    std::vector<int> seen((size_t)(8 * no), 0);
    for (long long c = 0; c < 8 * no; ++c) {
      const long long p = pidx(c, no);
      if (p < 0 || p >= 8 * no) { ++bad; continue; }
      ++seen[p];
      const int ch = (int)(c & 7);
      const int colour = ((ch >> 2) + (ch >> 1) + ch) & 1;
      if (p / (4 * no) != colour) ++bad;         // plane = colour
      if ((p >> 2) % no != (c >> 3)) ++bad;      // the oct's float4
    }
    for (int v : seen)
      if (v != 1) ++bad;
    if (pidx(5, 0) != 5) ++bad;  // dense: identity
  }
  std::printf("%lld\n", bad);
  return 0;
}
