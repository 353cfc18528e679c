// dense_f64.cu -- FP64 kernels of the FAS multigrid Newton-Gauss-Seidel solver
// on dense periodic levels (Puchwein, Baldi & Springel 2013, Sec. 3.2-3.3).
//
// Layout: level of size N = 2^lg, C order index ((i*N)+j)*N+k, k along z
// (fastest).  Each level keeps u and E = e^u side by side so a point update
// needs one exponential (its own new E) instead of seven; on GB300 the FP64
// pipe, not HBM, bounds these kernels.
#include <algorithm>

#include "mgfr_internal.cuh"

namespace {

constexpr int BS = 256;

// linear index of (i, j, k) on an N = 2^lg grid (N <= 1024: fits 32 bits)
__device__ __forceinline__ unsigned cidx(int i, int j, int k, int lg) {
  return ((((unsigned)i << lg) + (unsigned)j) << lg) + (unsigned)k;
}

// e^{-u/(n+1)}: for n = 1 this is 1/sqrt(E).
__device__ __forceinline__ double nl_s(double u, double E, const Model& m) {
  return m.n == 1 ? rsqrt(E) : exp(-u * m.inv_np1);
}

// L_i (Sec. 3.2): flux form with face coefficients b = (E_j + E_i)/2.
__device__ __forceinline__ double Lpoint(const double* __restrict__ u, const double* __restrict__ E,
                                         int i, int j, int k, int lg, const Model& m, double ih2) {
  const int M = (1 << lg) - 1;
  const long long c = cidx(i, j, k, lg);
  const long long nb[6] = {cidx((i - 1) & M, j, k, lg), cidx((i + 1) & M, j, k, lg),
                           cidx(i, (j - 1) & M, k, lg), cidx(i, (j + 1) & M, k, lg),
                           cidx(i, j, (k - 1) & M, lg), cidx(i, j, (k + 1) & M, lg)};
  const double uc = u[c], Ec = E[c];
  double sbd = 0.0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const double un = u[nb[q]];
    sbd = fma(0.5 * (E[nb[q]] + Ec), un - uc, sbd);
  }
  return sbd * ih2 + m.aRt * (1.0 - nl_s(uc, Ec, m));
}

__global__ void k_source(const double* __restrict__ d, double* __restrict__ f, long long n,
                         double src) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) f[t] = src * d[t];
}

// E = e^u of an iterate already in place (the previous solution as the start)
__global__ void k_init_inplace(const double* __restrict__ u, double* __restrict__ E, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) E[t] = exp(u[t]);
}

__global__ void k_init(const double* __restrict__ u0, double* __restrict__ u,
                       double* __restrict__ E, long long n) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (!u0) {  // the zero start: e^0 = 1
    u[t] = 0.0;
    E[t] = 1.0;
    return;
  }
  const double v = u0[t];
  u[t] = v;
  E[t] = exp(v);
}

// One red (colour 0: i+j+k even) or black half-sweep of the Newton update
// u <- u - (L - f) / (dL/du) (Sec. 3.3, Eq. (23)), one thread
// per cell of the active colour.  dL/du holds the neighbours fixed; the step
// is clamped to |du| <= cap.
__global__ void __launch_bounds__(BS) k_sweep(double* __restrict__ u, double* __restrict__ E,
                                              const double* __restrict__ f, int lg, int colour,
                                              Model m, double ih2, double cap,
                                              const float* __restrict__ mask, float mthr) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int N = 1 << lg, M = N - 1;
  if (t >= (1LL << (3 * lg - 1))) return;
  const int k2 = (int)(t & ((N >> 1) - 1));
  const long long r = t >> (lg - 1);
  const int j = (int)(r & M), i = (int)(r >> lg);
  const int k = 2 * k2 + ((i + j + colour) & 1);
  const long long c = cidx(i, j, k, lg);
  if (mask && !(mask[c] > mthr)) return;
  const long long nb[6] = {cidx((i - 1) & M, j, k, lg), cidx((i + 1) & M, j, k, lg),
                           cidx(i, (j - 1) & M, k, lg), cidx(i, (j + 1) & M, k, lg),
                           cidx(i, j, (k - 1) & M, lg), cidx(i, j, (k + 1) & M, lg)};
  const double uc = u[c], Ec = E[c];
  double sbd = 0.0, sd = 0.0, sb = 0.0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const double un = u[nb[q]], b = 0.5 * (E[nb[q]] + Ec), du = un - uc;
    sbd = fma(b, du, sbd);
    sd += du;
    sb += b;
  }
  const double s = nl_s(uc, Ec, m);
  const double L = sbd * ih2 + m.aRt * (1.0 - s);
  const double dL = (0.5 * Ec * sd - sb) * ih2 + m.aRt_np1 * s;
  double step = (L - f[c]) / dL;
  step = fmin(fmax(step, -cap), cap);
  const double unew = uc - step;
  u[c] = unew;
  E[c] = exp(unew);
}

// Per coarse cell: restrict u (average of the 8 daughters, Sec. 3.3) and the
// fine residual f - L(u); the residual average lands in fc (completed into the
// FAS right-hand side by k_fas_rhs).
__global__ void __launch_bounds__(BS) k_restrict_resid(const double* __restrict__ u,
                                                       const double* __restrict__ E,
                                                       const double* __restrict__ f, int lgf,
                                                       double* __restrict__ uc,
                                                       double* __restrict__ Ec,
                                                       double* __restrict__ ucold,
                                                       double* __restrict__ fc, Model m,
                                                       double ih2, const float* __restrict__ mask,
                                                       float mthr) {
  const int lgc = lgf - 1, Nc = 1 << lgc;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (1LL << (3 * lgc))) return;
  const int K = (int)(t & (Nc - 1)), J = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  double su = 0.0, sr = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q >> 2), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q & 1);
    const long long c = cidx(i, j, k, lgf);
    su += u[c];
    if (!mask || mask[c] > mthr) sr += f[c] - Lpoint(u, E, i, j, k, lgf, m, ih2);
  }
  const double um = 0.125 * su;
  uc[t] = um;
  ucold[t] = um;
  Ec[t] = exp(um);
  fc[t] = 0.125 * sr;
}

// FAS right-hand side f^{2h} = L^{2h}(R u) + R(f - L(u)) (Eq. (27)).
__global__ void __launch_bounds__(BS) k_fas_rhs(const double* __restrict__ u,
                                                const double* __restrict__ E,
                                                double* __restrict__ f, int lg, Model m,
                                                double ih2, const float* __restrict__ mask,
                                                float mthr) {
  const int N = 1 << lg;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (1LL << (3 * lg))) return;
  if (mask && !(mask[t] > mthr)) return;
  const int k = (int)(t & (N - 1)), j = (int)((t >> lg) & (N - 1)), i = (int)(t >> (2 * lg));
  f[t] += Lpoint(u, E, i, j, k, lg, m, ih2);
}

// u^h += P(u^{2h} - R u^h) (Eq. (29)), P linear (parent value plus
// s_d (c_{+d} - c_{-d})/8 per axis) or injection; then E = e^u.
__global__ void __launch_bounds__(BS) k_prolong_corr(double* __restrict__ u,
                                                     double* __restrict__ E,
                                                     const double* __restrict__ uc,
                                                     const double* __restrict__ ucold, int lgf,
                                                     int linear, const float* __restrict__ mask,
                                                     float mthr) {
  const int N = 1 << lgf, lgc = lgf - 1, Mc = (N >> 1) - 1;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (1LL << (3 * lgf))) return;
  if (mask && !(mask[t] > mthr)) return;
  const int k = (int)(t & (N - 1)), j = (int)((t >> lgf) & (N - 1)), i = (int)(t >> (2 * lgf));
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  auto corr = [&](int a, int b, int c) {
    const long long q = cidx(a & Mc, b & Mc, c & Mc, lgc);
    return uc[q] - ucold[q];
  };
  double v = corr(I, J, K);
  if (linear) {
    const double sx = (i & 1) ? 0.125 : -0.125, sy = (j & 1) ? 0.125 : -0.125,
                 sz = (k & 1) ? 0.125 : -0.125;
    v += sx * (corr(I + 1, J, K) - corr(I - 1, J, K));
    v += sy * (corr(I, J + 1, K) - corr(I, J - 1, K));
    v += sz * (corr(I, J, K + 1) - corr(I, J, K - 1));
  }
  const double un = u[t] + v;
  u[t] = un;
  E[t] = exp(un);
}

// Direct NGS on the 4^3 grid (Sec. 3.3, step 5): one block of 64 threads,
// red-black sweeps in shared memory until max|r| drops by `rel` or
// max_sweeps is reached (bounded loop); the residual is checked before the
// first sweep and after every kCheck sweeps.
__global__ void __launch_bounds__(64) k_coarse(double* __restrict__ ug, double* __restrict__ Eg,
                                               const double* __restrict__ fg, Model m, double ih2,
                                               double cap, int max_sweeps, double rel,
                                               const float* __restrict__ mask, float mthr) {
  __shared__ double u[64], E[64], f[64], red[64];
  const int t = threadIdx.x;
  const bool active = !mask || mask[t] > mthr;
  u[t] = ug[t];
  E[t] = Eg[t];
  f[t] = fg[t];
  const int i = t >> 4, j = (t >> 2) & 3, k = t & 3;
  const int colour = (i + j + k) & 1;
  const int nb[6] = {(((i + 3) & 3) << 4) | (j << 2) | k, (((i + 1) & 3) << 4) | (j << 2) | k,
                     (i << 4) | (((j + 3) & 3) << 2) | k, (i << 4) | (((j + 1) & 3) << 2) | k,
                     (i << 4) | (j << 2) | ((k + 3) & 3), (i << 4) | (j << 2) | ((k + 1) & 3)};
  __syncthreads();
  constexpr int kCheck = 4;
  double r0 = -1.0;
  for (int s = 0; s <= max_sweeps; ++s) {
    if (s % kCheck == 0 || s == max_sweeps) {
      // residual max (before sweep s)
      double sbd = 0.0;
      for (int q = 0; q < 6; ++q) sbd = fma(0.5 * (E[nb[q]] + E[t]), u[nb[q]] - u[t], sbd);
      const double rr = fabs(f[t] - (sbd * ih2 + m.aRt * (1.0 - nl_s(u[t], E[t], m))));
      red[t] = active ? rr : 0.0;
      __syncthreads();
      for (int w = 32; w > 0; w >>= 1) {
        if (t < w) red[t] = fmax(red[t], red[t + w]);
        __syncthreads();
      }
      const double rmax = red[0];
      __syncthreads();
      if (r0 < 0.0) r0 = rmax;
      if (s == max_sweeps || rmax <= rel * r0) break;
    }
    for (int c = 0; c < 2; ++c) {
      if (colour == c && active) {
        double sb = 0.0, sd = 0.0, sbd = 0.0;
        const double uc = u[t], Ec = E[t];
        for (int q = 0; q < 6; ++q) {
          const double b = 0.5 * (E[nb[q]] + Ec), du = u[nb[q]] - uc;
          sbd = fma(b, du, sbd);
          sd += du;
          sb += b;
        }
        const double sN = nl_s(uc, Ec, m);
        const double L = sbd * ih2 + m.aRt * (1.0 - sN);
        const double dL = (0.5 * Ec * sd - sb) * ih2 + m.aRt_np1 * sN;
        double step = (L - f[t]) / dL;
        step = fmin(fmax(step, -cap), cap);
        u[t] = uc - step;
        E[t] = exp(u[t]);
      }
      __syncthreads();
    }
  }
  ug[t] = u[t];
  Eg[t] = E[t];
}

template <int MODE>  // 0: residual of (u,E,f); 1: plain vector x (in u)
__global__ void __launch_bounds__(BS) k_norm(const double* __restrict__ u,
                                             const double* __restrict__ E,
                                             const double* __restrict__ f, int lg, long long n,
                                             Model m, double ih2, double* __restrict__ partials) {
  double ss = 0.0, mx = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += stride) {
    double r;
    if (MODE == 0) {
      const int N = 1 << lg;
      const int k = (int)(t & (N - 1)), j = (int)((t >> lg) & (N - 1)), i = (int)(t >> (2 * lg));
      r = f[t] - Lpoint(u, E, i, j, k, lg, m, ih2);
    } else {
      r = u[t];
    }
    ss = fma(r, r, ss);
    mx = fmax(mx, fabs(r));
  }
  __shared__ double s1[BS / 32], s2[BS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = ss;
    s2[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < BS / 32; ++w) {
      a += s1[w];
      b = fmax(b, s2[w]);
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_finish(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
    a += partials[2 * q];
    b = fmax(b, partials[2 * q + 1]);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s1[0];
    out[1] = s2[0];
  }
}

// fR = fR_bar e^u and a_MG/c^2 = (fR_{+} - fR_{-}) / (2h) / (2a) per axis
// (Sec. 2, Eq. (13)).  acc is [3][N^3].
__global__ void __launch_bounds__(BS) k_force(const double* __restrict__ E, int lg, double fbar,
                                              double g_scale, double* __restrict__ fr,
                                              double* __restrict__ acc) {
  const int N = 1 << lg, M = N - 1;
  const long long n = 1LL << (3 * lg);
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int k = (int)(t & M), j = (int)((t >> lg) & M), i = (int)(t >> (2 * lg));
  fr[t] = fbar * E[t];
  if (!acc) return;
  acc[t] = g_scale * (E[cidx((i + 1) & M, j, k, lg)] - E[cidx((i - 1) & M, j, k, lg)]);
  acc[n + t] = g_scale * (E[cidx(i, (j + 1) & M, k, lg)] - E[cidx(i, (j - 1) & M, k, lg)]);
  acc[2 * n + t] = g_scale * (E[cidx(i, j, (k + 1) & M, lg)] - E[cidx(i, j, (k - 1) & M, lg)]);
}

}  // namespace

namespace f64 {

void source(const double* delta, double* f, long long n, double src, cudaStream_t s) {
  k_source<<<nblocks(n, BS), BS, 0, s>>>(delta, f, n, src);
}

void init_u(const double* u0, double* u, double* E, long long n, cudaStream_t s) {
  if (u0 == u)
    k_init_inplace<<<nblocks(n, BS), BS, 0, s>>>(u, E, n);
  else
    k_init<<<nblocks(n, BS), BS, 0, s>>>(u0, u, E, n);
}

void sweep(DenseLevel& L, const Model& m, int colour, double cap, cudaStream_t s) {
  k_sweep<<<nblocks(L.n / 2, BS), BS, 0, s>>>(L.u, L.E, L.f, L.lg, colour, m, L.ih2, cap, L.mask,
                                              L.mthr);
}

void restrict_resid(DenseLevel& F, DenseLevel& C, const Model& m, cudaStream_t s) {
  k_restrict_resid<<<nblocks(C.n, BS), BS, 0, s>>>(F.u, F.E, F.f, F.lg, C.u, C.E, C.uold, C.f, m,
                                                   F.ih2, F.mask, F.mthr);
}

void fas_rhs(DenseLevel& C, const Model& m, cudaStream_t s) {
  k_fas_rhs<<<nblocks(C.n, BS), BS, 0, s>>>(C.u, C.E, C.f, C.lg, m, C.ih2, C.mask, C.mthr);
}

void prolong_corr(DenseLevel& F, DenseLevel& C, int linear, cudaStream_t s) {
  k_prolong_corr<<<nblocks(F.n, BS), BS, 0, s>>>(F.u, F.E, C.u, C.uold, F.lg, linear, F.mask,
                                                 F.mthr);
}

void coarse_solve(DenseLevel& C, const Model& m, double cap, int max_sweeps, double rel,
                  cudaStream_t s) {
  k_coarse<<<1, 64, 0, s>>>(C.u, C.E, C.f, m, C.ih2, cap, max_sweeps, rel, C.mask, C.mthr);
}

void resid_norm(DenseLevel& L, const Model& m, double* partials, int nparts, double* out,
                cudaStream_t s) {
  int nb = (int)std::min<long long>(nparts, nblocks(L.n, BS));
  k_norm<0><<<nb, BS, 0, s>>>(L.u, L.E, L.f, L.lg, L.n, m, L.ih2, partials);
  k_finish<<<1, 256, 0, s>>>(partials, nb, out);
}

void norm(const double* x, long long n, double* partials, int nparts, double* out, cudaStream_t s) {
  int nb = (int)std::min<long long>(nparts, nblocks(n, BS));
  Model m{};
  k_norm<1><<<nb, BS, 0, s>>>(x, nullptr, nullptr, 0, n, m, 0.0, partials);
  k_finish<<<1, 256, 0, s>>>(partials, nb, out);
}

void force(const DenseLevel& L, const Model& m, double* fr, double* acc, cudaStream_t s) {
  const double g_scale = m.fbar / (2.0 * L.h) / (2.0 * m.a);
  k_force<<<nblocks(L.n, BS), BS, 0, s>>>(L.E, L.lg, m.fbar, g_scale, fr, acc);
}

}  // namespace f64
