// amr_solve.cu -- one-way solve of a refined level (Puchwein, Baldi & Springel
// 2013, Sec. 3.3, steps 9-12 and the mask function of the multigrid on
// partial levels).
//
// Level L is relaxed with red-black Newton-Gauss-Seidel on its octs, its ghost
// layer fixed from the converged level L-1.  The FAS coarse grids are the
// coarser tree levels and then the dense levels below the base; a coarse cell
// is relaxed only where its mask (1 on level L, the daughters' average below,
// 0 without daughters) exceeds mask_thres.  Unrelaxed coarse cells keep the
// converged coarse solution (or the restriction of their daughters), so the
// coarse solutions themselves are never modified.
//
// Kernels are templated on the working precision T.  The FP64 form runs FP64
// V-cycles to the tolerance.  The mixed form first runs FP32 V-cycles (u in
// FP32, e^u recomputed by the SFU) until the FP32 residual reaches
// mixed_switch or stalls (phase A), then corrects the defect (phase B): the
// residual r = f - L(u) of the level in double-float (FP64-accurate, on the
// FP32 pipes), FP32 linear masked V-cycles on J(u) e = r, u += e in
// double-float; the stopping test is always that FP64-accurate residual.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "amr.cuh"
#include "colour_split.cuh"
#include "dfloat.cuh"

namespace {

constexpr int BS = 256;

template <class T>
struct MT {
  T aRt, aRt_np1, inv_np1;
  int n;
};

template <class T>
MT<T> mt(const Model& m) {
  return MT<T>{(T)m.aRt, (T)m.aRt_np1, (T)m.inv_np1, m.n};
}

__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float ex(float x) { return __expf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// e^{-u/(n+1)} (1/sqrt(E) for n = 1)
template <class T>
__device__ __forceinline__ T nls(T u, T E, const MT<T>& m) {
  return m.n == 1 ? rsq(E) : ex(-u * m.inv_np1);
}

template <class T>
struct NB {
  T u, E;
};

// e^u at slot q.  The FP64 oct arrays store E = e^u beside u; the FP32 oct
// arrays carry u only and e^u is recomputed by the SFU where it is needed
// (a stored FP32 E would add a read and a write stream to every sweep).
__device__ __forceinline__ double Eat(const double* __restrict__ E, const double* __restrict__,
                                      long long q) {
  return E[q];
}
__device__ __forceinline__ float Eat(const float* __restrict__, const float* __restrict__ u,
                                     long long q) {
  return __expf(u[q]);
}

// neighbour of cell (o, ch) in direction d: same oct, neighbouring oct, or
// the ghost slot of that face.
template <class T>
__device__ __forceinline__ NB<T> onb(const T* __restrict__ u, const T* __restrict__ E,
                                     const int* __restrict__ nbr, const T* __restrict__ gh,
                                     const T* __restrict__ ghE, long long o, int ch, int d) {
  const int ax = d >> 1, plus = d & 1;
  const int bit = (ch >> (2 - ax)) & 1;
  const int chn = ch ^ (1 << (2 - ax));
  if (bit != plus) {
    const long long q = 8 * o + chn;
    return NB<T>{u[q], Eat(E, u, q)};
  }
  const int no = nbr[6 * o + d];
  if (no >= 0) {
    const long long q = 8LL * no + chn;
    return NB<T>{u[q], Eat(E, u, q)};
  }
  const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
  const int qi = (((ch >> (2 - t1)) & 1) << 1) | ((ch >> (2 - t2)) & 1);
  const long long g = 4LL * (-no - 1) + qi;  // ghost slot of the face
  return NB<T>{gh[g], Eat(ghE, gh, g)};
}

// L_i (Sec. 3.2) from the centre and its six neighbours
template <class T>
__device__ __forceinline__ T Lval(T uc, T Ec, const NB<T>* nb, const MT<T>& m, T ih2) {
  T sbd = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) sbd = fma((T)0.5 * (nb[q].E + Ec), nb[q].u - uc, sbd);
  return sbd * ih2 + m.aRt * ((T)1 - nls(uc, Ec, m));
}

// Newton step (L - f)/(dL/du), clamped (Sec. 3.3, Eq. (23))
template <class T>
__device__ __forceinline__ T newton(T uc, T Ec, const NB<T>* nb, T f, const MT<T>& m, T ih2, T cap) {
  T sbd = 0, sd = 0, sb = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const T b = (T)0.5 * (nb[q].E + Ec), du = nb[q].u - uc;
    sbd = fma(b, du, sbd);
    sd += du;
    sb += b;
  }
  const T s = nls(uc, Ec, m);
  const T L = sbd * ih2 + m.aRt * ((T)1 - s);
  const T dL = ((T)0.5 * Ec * sd - sb) * ih2 + m.aRt_np1 * s;
  T step = (L - f) / dL;
  return fmin(fmax(step, -cap), cap);
}

__constant__ int kColourChild[2][4] = {{0, 3, 5, 6}, {1, 2, 4, 7}};

template <class T>
__global__ void __launch_bounds__(BS) k_osweep(T* __restrict__ u, T* __restrict__ E,
                                               const T* __restrict__ f, const int* __restrict__ nbr,
                                               const T* __restrict__ gh, const T* __restrict__ ghE,
                                               const unsigned char* __restrict__ act,
                                               long long n_oct, const int* __restrict__ olist,
                                               int colour, MT<T> m, T ih2, T cap) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 4 * n_oct) return;
  const long long o = olist ? olist[t >> 2] : t >> 2;
  const int ch = kColourChild[colour][t & 3];
  const long long c = 8 * o + ch;
  if (act && !(act[c])) return;
  NB<T> nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = onb(u, E, nbr, gh, ghE, o, ch, d);
  const T uc = u[c];
  const T un = uc - newton(uc, Eat(E, u, c), nb, f[c], m, ih2, cap);
  u[c] = un;
  if constexpr (std::is_same<T, double>::value) E[c] = ex(un);
}

// restrict oct level to its parents: u average, masked residual average
template <class T>
__global__ void __launch_bounds__(BS) k_orestrict(
    const T* __restrict__ u, const T* __restrict__ E, const T* __restrict__ f,
    const int* __restrict__ nbr, const T* __restrict__ gh, const T* __restrict__ ghE,
    const unsigned char* __restrict__ act, long long n_oct, const int* __restrict__ olist,
    const int* __restrict__ pcell, MT<T> m, T ih2, T* __restrict__ uc, T* __restrict__ Ec,
    T* __restrict__ ucold, T* __restrict__ fc) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_oct) return;
  const long long o = olist ? olist[t] : t;
  T su = 0, sr = 0;
  for (int ch = 0; ch < 8; ++ch) {
    const long long c = 8 * o + ch;
    su += u[c];
    if (!act || act[c]) {
      NB<T> nb[6];
#pragma unroll
      for (int d = 0; d < 6; ++d) nb[d] = onb(u, E, nbr, gh, ghE, o, ch, d);
      sr += f[c] - Lval(u[c], Eat(E, u, c), nb, m, ih2);
    }
  }
  const int p = pcell[o];
  const T um = (T)0.125 * su;
  uc[p] = um;
  ucold[p] = um;
  Ec[p] = ex(um);
  fc[p] = (T)0.125 * sr;
}

// FAS right-hand side on a coarse oct level: f += L(u) at relaxed cells
template <class T>
__global__ void __launch_bounds__(BS) k_ofas(const T* __restrict__ u, const T* __restrict__ E,
                                             T* __restrict__ f, const int* __restrict__ nbr,
                                             const T* __restrict__ gh, const T* __restrict__ ghE,
                                             const unsigned char* __restrict__ act,
                                             long long ncell, const int* __restrict__ olist,
                                             MT<T> m, T ih2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncell) return;
  const long long o = olist ? olist[t >> 3] : t >> 3;
  const int ch = (int)(t & 7);
  const long long c = 8 * o + ch;
  if (!(act[c])) return;
  NB<T> nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = onb(u, E, nbr, gh, ghE, o, ch, d);
  f[c] += Lval(u[c], Eat(E, u, c), nb, m, ih2);
}

// u += P(uc - ucold) on relaxed cells (Eq. (29)), the parent's
// neighbours from the pnbr table (a gradient component is 0 where one is
// missing).
template <class T>
__global__ void __launch_bounds__(BS) k_oprolong(long long ncell, const int* __restrict__ olist,
                                                 const int* __restrict__ pcell,
                                                 const int* __restrict__ pnbr,
                                                 const T* __restrict__ uc,
                                                 const T* __restrict__ ucold,
                                                 const unsigned char* __restrict__ act,
                                                 int linear, T* __restrict__ u, T* __restrict__ E) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncell) return;
  const long long o = olist ? olist[t >> 3] : t >> 3;
  const int ch = (int)(t & 7);
  const long long c = 8 * o + ch;
  if (act && !(act[c])) return;
  const int p = pcell[o];
  T v = uc[p] - ucold[p];
  if (linear) {
    for (int ax = 0; ax < 3; ++ax) {
      const int pm = pnbr[6 * o + 2 * ax], pp = pnbr[6 * o + 2 * ax + 1];
      if (pm < 0 || pp < 0) continue;
      const T s = ((ch >> (2 - ax)) & 1) ? (T)0.125 : (T)-0.125;
      v += s * ((uc[pp] - ucold[pp]) - (uc[pm] - ucold[pm]));
    }
  }
  const T un = u[c] + v;
  u[c] = un;
  if constexpr (std::is_same<T, double>::value) E[c] = ex(un);
}

// residual norms of level L (sum r^2, max |r|, sum f^2), accumulated in FP64
template <class T>
__global__ void __launch_bounds__(BS) k_onorm(const T* __restrict__ u, const T* __restrict__ E,
                                              const T* __restrict__ f, const int* __restrict__ nbr,
                                              const T* __restrict__ gh, const T* __restrict__ ghE,
                                              long long ncell, MT<T> m, T ih2,
                                              double* __restrict__ partials) {
  double ss = 0.0, mx = 0.0, fs = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long o = c >> 3;
    const int ch = (int)(c & 7);
    NB<T> nb[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = onb(u, E, nbr, gh, ghE, o, ch, d);
    const double r = (double)(f[c] - Lval(u[c], Eat(E, u, c), nb, m, ih2));
    ss = fma(r, r, ss);
    mx = fmax(mx, fabs(r));
    fs = fma((double)f[c], (double)f[c], fs);
  }
  __shared__ double s1[BS / 32], s2[BS / 32], s3[BS / 32];
  for (int q = 16; q > 0; q >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, q);
    fs += __shfl_xor_sync(0xffffffffu, fs, q);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, q));
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = ss;
    s2[threadIdx.x >> 5] = mx;
    s3[threadIdx.x >> 5] = fs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, e = 0.0;
    for (int w = 0; w < BS / 32; ++w) {
      a += s1[w];
      b = fmax(b, s2[w]);
      e += s3[w];
    }
    partials[3 * blockIdx.x] = a;
    partials[3 * blockIdx.x + 1] = b;
    partials[3 * blockIdx.x + 2] = e;
  }
}

__global__ void k_finish3(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
  __shared__ double s1[256], s2[256], s3[256];
  double a = 0.0, b = 0.0, e = 0.0;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
    a += partials[3 * q];
    b = fmax(b, partials[3 * q + 1]);
    e += partials[3 * q + 2];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  s3[threadIdx.x] = e;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + w]);
      s3[threadIdx.x] += s3[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s1[0];
    out[1] = s2[0];
    out[2] = s3[0];
  }
}

// ---- dense levels (base and below) with masks, u and E stored ------------
// linear index of (i, j, k) on an N = 2^lg grid (N <= 1024: fits 32 bits)
__device__ __forceinline__ unsigned cidx(int i, int j, int k, int lg) {
  return ((((unsigned)i << lg) + (unsigned)j) << lg) + (unsigned)k;
}

template <class T>
__device__ __forceinline__ void dnb(const T* __restrict__ u, const T* __restrict__ E, int i, int j,
                                    int k, int lg, NB<T>* nb) {
  const int M = (1 << lg) - 1;
  const unsigned q[6] = {cidx((i - 1) & M, j, k, lg), cidx((i + 1) & M, j, k, lg),
                          cidx(i, (j - 1) & M, k, lg), cidx(i, (j + 1) & M, k, lg),
                          cidx(i, j, (k - 1) & M, lg), cidx(i, j, (k + 1) & M, lg)};
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = NB<T>{u[q[d]], Eat(E, u, q[d])};
}

// the six neighbour values of x at (i, j, k)
__device__ __forceinline__ void dnb_x(const float* __restrict__ x, int i, int j, int k, int lg,
                                      float* out) {
  const int M = (1 << lg) - 1;
  out[0] = x[cidx((i - 1) & M, j, k, lg)];
  out[1] = x[cidx((i + 1) & M, j, k, lg)];
  out[2] = x[cidx(i, (j - 1) & M, k, lg)];
  out[3] = x[cidx(i, (j + 1) & M, k, lg)];
  out[4] = x[cidx(i, j, (k - 1) & M, lg)];
  out[5] = x[cidx(i, j, (k + 1) & M, lg)];
}

// masked Newton-Gauss-Seidel half-sweep of a dense level (the base or one below
// it as a coarse grid of a refined-level solve), one thread per relaxed cell of
// the colour, from a list of their C-order indices
template <class T>
__global__ void __launch_bounds__(BS) k_dsweep_list(T* __restrict__ u, T* __restrict__ E,
                                                    const T* __restrict__ f, int lg,
                                                    const int* __restrict__ list, long long n,
                                                    MT<T> m, T ih2, T cap) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const unsigned c = (unsigned)list[t];
  const int M = (1 << lg) - 1;
  const int k = (int)(c & M), j = (int)((c >> lg) & M), i = (int)(c >> (2 * lg));
  NB<T> nb[6];
  dnb(u, E, i, j, k, lg, nb);
  const T uc = u[c];
  const T un = uc - newton(uc, Eat(E, u, c), nb, f[c], m, ih2, cap);
  u[c] = un;
  if constexpr (std::is_same<T, double>::value) E[c] = ex(un);
}

// the relaxed cells of a masked dense level -> one list per colour (colour q
// at list + q half, in block order: a red-black half-sweep does not depend on
// the order), count[q] += their number; one atomic per block and colour
__global__ void __launch_bounds__(BS) k_dense_list(const unsigned char* __restrict__ act, int lg,
                                                   int* __restrict__ list,
                                                   unsigned long long* __restrict__ count) {
  __shared__ int woff[2][BS / 32];
  __shared__ unsigned long long bbase[2];
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = (1 << lg) - 1;
  const bool live = t < (1u << (3 * lg));
  const int colour = live ? (int)(((t >> (2 * lg)) + ((t >> lg) & M) + (t & M)) & 1) : 0;
  const bool on = live && act[t];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned ballot[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    ballot[q] = __ballot_sync(0xffffffffu, on && colour == q);  // whole warps reach here
    if (lane == 0) woff[q][w] = __popc(ballot[q]);
  }
  __syncthreads();
  if (threadIdx.x < 2) {  // exclusive offsets of the warps, and the block's base
    const int q = threadIdx.x;
    int run = 0;
    for (int v = 0; v < BS / 32; ++v) {
      const int n = woff[q][v];
      woff[q][v] = run;
      run += n;
    }
    bbase[q] = run > 0 ? atomicAdd(count + q, (unsigned long long)run) : 0ULL;
  }
  __syncthreads();
  if (on) {
    const int q = colour;
    list[((long long)q << (3 * lg - 1)) + bbase[q] + woff[q][w] +
         __popc(ballot[q] & ((1u << lane) - 1u))] = (int)t;
  }
}

template <class T>
__global__ void __launch_bounds__(BS) k_drestrict(const T* __restrict__ u, const T* __restrict__ E,
                                                  const T* __restrict__ f, int lgf,
                                                  T* __restrict__ uc, T* __restrict__ Ec,
                                                  T* __restrict__ ucold, T* __restrict__ fc, MT<T> m,
                                                  T ih2, const unsigned char* __restrict__ act) {
  const int lgc = lgf - 1, Nc = 1 << lgc;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lgc))) return;
  const int K = (int)(t & (Nc - 1)), J = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  T su = 0, sr = 0;
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q >> 2), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q & 1);
    const unsigned c = cidx(i, j, k, lgf);
    su += u[c];
    if (!act || act[c]) {
      NB<T> nb[6];
      dnb(u, E, i, j, k, lgf, nb);
      sr += f[c] - Lval(u[c], Eat(E, u, c), nb, m, ih2);
    }
  }
  const T um = (T)0.125 * su;
  uc[t] = um;
  ucold[t] = um;
  if constexpr (std::is_same<T, double>::value) Ec[t] = ex(um);
  fc[t] = (T)0.125 * sr;
}

// The relaxed cells of a masked dense level as the two per-colour lists
// (colour q at p + q half, n[q] entries); p == nullptr: none built (the
// kernels then visit every cell and test the relax flags).
struct CList {
  const int* p;
  long long half, n0, n1;
};

// cell of thread tid: from the lists, else tid itself if its flag is set
__device__ __forceinline__ bool dcell(const CList& L, const unsigned char* __restrict__ act,
                                      int lg, long long tid, unsigned* c) {
  if (L.p) {
    if (tid < L.n0) {
      *c = (unsigned)L.p[tid];
      return true;
    }
    tid -= L.n0;
    if (tid >= L.n1) return false;
    *c = (unsigned)L.p[L.half + tid];
    return true;
  }
  if (tid >= (1LL << (3 * lg))) return false;
  if (act && !act[tid]) return false;
  *c = (unsigned)tid;
  return true;
}

template <class T>
__global__ void __launch_bounds__(BS) k_dfas(const T* __restrict__ u, const T* __restrict__ E,
                                             T* __restrict__ f, int lg, MT<T> m, T ih2,
                                             const unsigned char* __restrict__ act, CList cl) {
  const int N = 1 << lg;
  unsigned t;
  if (!dcell(cl, act, lg, blockIdx.x * (long long)blockDim.x + threadIdx.x, &t)) return;
  const int k = (int)(t & (N - 1)), j = (int)((t >> lg) & (N - 1)), i = (int)(t >> (2 * lg));
  NB<T> nb[6];
  dnb(u, E, i, j, k, lg, nb);
  f[t] += Lval(u[t], Eat(E, u, t), nb, m, ih2);
}

template <class T>
__global__ void __launch_bounds__(BS) k_dprolong(T* __restrict__ u, T* __restrict__ E,
                                                 const T* __restrict__ uc, const T* __restrict__ ucold,
                                                 int lgf, int linear, const unsigned char* __restrict__ act,
                                                 CList cl) {
  const int N = 1 << lgf, lgc = lgf - 1, Mc = (N >> 1) - 1;
  unsigned t;
  if (!dcell(cl, act, lgf, blockIdx.x * (long long)blockDim.x + threadIdx.x, &t)) return;
  const int k = (int)(t & (N - 1)), j = (int)((t >> lgf) & (N - 1)), i = (int)(t >> (2 * lgf));
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  auto corr = [&](int a, int b, int c) {
    const unsigned q = cidx(a & Mc, b & Mc, c & Mc, lgc);
    return uc[q] - ucold[q];
  };
  T v = corr(I, J, K);
  if (linear) {
    v += ((i & 1) ? (T)0.125 : (T)-0.125) * (corr(I + 1, J, K) - corr(I - 1, J, K));
    v += ((j & 1) ? (T)0.125 : (T)-0.125) * (corr(I, J + 1, K) - corr(I, J - 1, K));
    v += ((k & 1) ? (T)0.125 : (T)-0.125) * (corr(I, J, K + 1) - corr(I, J, K - 1));
  }
  const T un = u[t] + v;
  u[t] = un;
  if constexpr (std::is_same<T, double>::value) E[t] = ex(un);
}

// masked NGS on the 4^3 grid, fixed sweep count (one block of 64 threads)
template <class T>
__global__ void __launch_bounds__(64) k_dcoarse(T* __restrict__ ug, T* __restrict__ Eg,
                                                const T* __restrict__ fg, MT<T> m, T ih2, T cap,
                                                int sweeps, const unsigned char* __restrict__ act) {
  __shared__ T u[64], E[64];
  const int t = threadIdx.x;
  u[t] = ug[t];
  E[t] = Eat(Eg, ug, t);
  const T f = fg[t];
  const bool active = !act || act[t];
  const int i = t >> 4, j = (t >> 2) & 3, k = t & 3, colour = (i + j + k) & 1;
  const int q[6] = {(((i + 3) & 3) << 4) | (j << 2) | k, (((i + 1) & 3) << 4) | (j << 2) | k,
                    (i << 4) | (((j + 3) & 3) << 2) | k, (i << 4) | (((j + 1) & 3) << 2) | k,
                    (i << 4) | (j << 2) | ((k + 3) & 3), (i << 4) | (j << 2) | ((k + 1) & 3)};
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int col = 0; col < 2; ++col) {
      if (colour == col && active) {
        NB<T> nb[6];
        for (int d = 0; d < 6; ++d) nb[d] = NB<T>{u[q[d]], E[q[d]]};
        const T un = u[t] - newton(u[t], E[t], nb, f, m, ih2, cap);
        u[t] = un;
        E[t] = ex(un);
      }
      __syncthreads();
    }
  ug[t] = u[t];
  if constexpr (std::is_same<T, double>::value) Eg[t] = E[t];
}


// ---- linear correction scheme (mixed precision, phase B) --------------------
// J(u): Jacobian of L at the FP32 linearisation point u (E = e^u stored):
//   J_ij = (E_j (u_j - u_i) + E_i + E_j) / (2h^2)
//   J_ii = sum_j (E_i (u_j - u_i) - E_i - E_j) / (2h^2) + alpha Rt/(n+1) e^{-u_i/(n+1)}
struct JR {
  float off[6], diag;
};

__device__ __forceinline__ JR jrow(float uc, float Ec, const NB<float>* nb, const MT<float>& m,
                                   float ih2) {
  JR J;
  const float h2 = 0.5f * ih2;
  float d = 0.f;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float du = nb[q].u - uc;
    J.off[q] = h2 * fmaf(nb[q].E, du, Ec + nb[q].E);
    d += fmaf(Ec, du, -Ec - nb[q].E);
  }
  J.diag = d * h2 + m.aRt_np1 * nls(uc, Ec, m);
  return J;
}

// masked Gauss-Seidel half-sweep on J(u) e = r of a dense level, one thread per
// relaxed cell of the colour (list of C-order indices)
__global__ void __launch_bounds__(BS) k_dlin_sweep_list(float* __restrict__ e,
                                                        const float* __restrict__ r,
                                                        const float* __restrict__ u,
                                                        const float* __restrict__ E, int lg,
                                                        const int* __restrict__ list,
                                                        long long n, MT<float> m, float ih2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const unsigned c = (unsigned)list[t];
  const int M = (1 << lg) - 1;
  const int k = (int)(c & M), j = (int)((c >> lg) & M), i = (int)(c >> (2 * lg));
  NB<float> nb[6];
  dnb(u, E, i, j, k, lg, nb);
  const JR J = jrow(u[c], Eat(E, u, c), nb, m, ih2);
  float en[6];
  dnb_x(e, i, j, k, lg, en);
  float acc = r[c];
#pragma unroll
  for (int d = 0; d < 6; ++d) acc = fmaf(-J.off[d], en[d], acc);
  e[c] = __fdividef(acc, J.diag);
}

__global__ void __launch_bounds__(BS) k_dlin_restrict(const float* __restrict__ e,
                                                      const float* __restrict__ r,
                                                      const float* __restrict__ u,
                                                      const float* __restrict__ E, int lgf,
                                                      float* __restrict__ rc, float* __restrict__ uc,
                                                      float* __restrict__ Ec, float* __restrict__ ec,
                                                      MT<float> m, float ih2,
                                                      const unsigned char* __restrict__ act) {
  const int lgc = lgf - 1, Nc = 1 << lgc;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lgc))) return;
  const int K = (int)(t & (Nc - 1)), J0 = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  float su = 0.f, sr = 0.f;
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q >> 2), j = 2 * J0 + ((q >> 1) & 1), k = 2 * K + (q & 1);
    const unsigned c = cidx(i, j, k, lgf);
    su += u[c];
    if (!act || act[c]) {
      NB<float> nb[6];
      float en[6];
      dnb(u, E, i, j, k, lgf, nb);
      dnb_x(e, i, j, k, lgf, en);
      const JR J = jrow(u[c], Eat(E, u, c), nb, m, ih2);
      float Je = J.diag * e[c];
#pragma unroll
      for (int d = 0; d < 6; ++d) Je = fmaf(J.off[d], en[d], Je);
      sr += r[c] - Je;
    }
  }
  const float um = 0.125f * su;
  uc[t] = um;
  rc[t] = 0.125f * sr;
  ec[t] = 0.f;
}

__global__ void __launch_bounds__(BS) k_dlin_prolong(float* __restrict__ e, const float* __restrict__ ec,
                                                     int lgf, int linear,
                                                     const unsigned char* __restrict__ act,
                                                     CList cl) {
  const int N = 1 << lgf, lgc = lgf - 1, Mc = (N >> 1) - 1;
  unsigned t;
  if (!dcell(cl, act, lgf, blockIdx.x * (long long)blockDim.x + threadIdx.x, &t)) return;
  const int k = (int)(t & (N - 1)), j = (int)((t >> lgf) & (N - 1)), i = (int)(t >> (2 * lgf));
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  auto cv = [&](int a, int b, int c) { return ec[cidx(a & Mc, b & Mc, c & Mc, lgc)]; };
  float v = cv(I, J, K);
  if (linear) {
    v += ((i & 1) ? 0.125f : -0.125f) * (cv(I + 1, J, K) - cv(I - 1, J, K));
    v += ((j & 1) ? 0.125f : -0.125f) * (cv(I, J + 1, K) - cv(I, J - 1, K));
    v += ((k & 1) ? 0.125f : -0.125f) * (cv(I, J, K + 1) - cv(I, J, K - 1));
  }
  e[t] += v;
}

__global__ void __launch_bounds__(64) k_dlin_coarse(float* __restrict__ eg, const float* __restrict__ rg,
                                                    const float* __restrict__ ug,
                                                    const float* __restrict__ Eg, MT<float> m,
                                                    float ih2, int sweeps,
                                                    const unsigned char* __restrict__ act) {
  __shared__ float e[64];
  const int t = threadIdx.x;
  const bool active = !act || act[t];
  const int i = t >> 4, j = (t >> 2) & 3, k = t & 3, colour = (i + j + k) & 1;
  const int q[6] = {(((i + 3) & 3) << 4) | (j << 2) | k, (((i + 1) & 3) << 4) | (j << 2) | k,
                    (i << 4) | (((j + 3) & 3) << 2) | k, (i << 4) | (((j + 1) & 3) << 2) | k,
                    (i << 4) | (j << 2) | ((k + 3) & 3), (i << 4) | (j << 2) | ((k + 1) & 3)};
  NB<float> nb[6];
  for (int d = 0; d < 6; ++d) nb[d] = NB<float>{ug[q[d]], Eat(Eg, ug, q[d])};
  const JR J = jrow(ug[t], Eat(Eg, ug, t), nb, m, ih2);
  const float rc = rg[t];
  e[t] = eg[t];
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int col = 0; col < 2; ++col) {
      if (colour == col && active) {
        float acc = rc;
        for (int d = 0; d < 6; ++d) acc = fmaf(-J.off[d], e[q[d]], acc);
        e[t] = acc / J.diag;
      }
      __syncthreads();
    }
  eg[t] = e[t];
}

__global__ void k_zero32(float* __restrict__ x, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.f;
}


// ---- FP32 storage of oct levels -------------------------------------------
// The FP32 arrays of an oct level (u, f or r, e) are stored by colour
// (colour_split.cuh, pidx): one float4 per colour and oct, so that a
// half-sweep moves whole 16-byte vectors of the colour it reads or writes.

struct Oct8 {
  float v[8];
};

__device__ __forceinline__ float4 ldc(const float* __restrict__ p, long long o, long long no,
                                      int col) {
  return *reinterpret_cast<const float4*>(p + 4 * (col * no + o));
}

__device__ __forceinline__ void stc(float* __restrict__ p, long long o, long long no, int col,
                                    float4 v) {
  *reinterpret_cast<float4*>(p + 4 * (col * no + o)) = v;
}

// the float4 of one colour <-> the oct's cells of that colour
__device__ __forceinline__ float f4(const float4& v, int r) {
  return r == 0 ? v.x : r == 1 ? v.y : r == 2 ? v.z : v.w;
}

__device__ __forceinline__ Oct8 ld8(const float* __restrict__ p, long long o, long long no) {
  const float4 a = ldc(p, o, no, 0), b = ldc(p, o, no, 1);
  Oct8 r;
  r.v[0] = a.x; r.v[3] = a.y; r.v[5] = a.z; r.v[6] = a.w;
  r.v[1] = b.x; r.v[2] = b.y; r.v[4] = b.z; r.v[7] = b.w;
  return r;
}

__device__ __forceinline__ void st8(float* __restrict__ p, long long o, long long no,
                                    const Oct8& x) {
  stc(p, o, no, 0, make_float4(x.v[0], x.v[3], x.v[5], x.v[6]));
  stc(p, o, no, 1, make_float4(x.v[1], x.v[2], x.v[4], x.v[7]));
}

// tangential face index of cell ch on a face normal to axis ax
__device__ __forceinline__ int face_q(int ch, int ax) {
  const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
  return (((ch >> (2 - t1)) & 1) << 1) | ((ch >> (2 - t2)) & 1);
}

// ---- thread-per-oct FP32 sweeps ------------------------------------------------
// One thread updates the 4 cells of colour COL in its oct.  It reads both
// colours of its own u, the colour-COL vector of f (or r), and from each face
// the other colour of the neighbouring oct (the cells across the face from
// colour-COL cells have the other colour) or the ghost face; it writes the
// colour-COL vector of u (or e).  e^u is recomputed by the SFU from u.
//   LIN = true : Gauss-Seidel on J(u) e = r  (u fixed; e updated)
//   LIN = false: Newton-Gauss-Seidel on L(u) = f (u updated)
// no: octs of the level (plane stride); n, olist: the octs visited.
template <bool LIN, int COL>
__global__ void __launch_bounds__(BS, 6) k_oct_sweep32(
    float* __restrict__ u, float* __restrict__ e, const float* __restrict__ rf,
    const int* __restrict__ nbr, const float* __restrict__ gh,
    const unsigned char* __restrict__ act, long long n, const int* __restrict__ olist,
    long long no, MT<float> m, float ih2, float cap) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int o = olist ? olist[t] : (int)t;
  constexpr int CC[2][4] = {{0, 3, 5, 6}, {1, 2, 4, 7}};
  constexpr int OC = 1 - COL;
  // 32-bit oct indices into float4 planes (n_oct < 2^31 / 6, checked on the host)
  const float4* __restrict__ u4 = reinterpret_cast<const float4*>(u);
  const float4* __restrict__ uo = u4 + OC * no;  // the other colour's plane
  const float4* __restrict__ e4 = reinterpret_cast<const float4*>(e);
  const float4* __restrict__ g4 = reinterpret_cast<const float4*>(gh);
  const float4 a0 = u4[o], a1 = u4[no + o];
  Oct8 U;
  U.v[0] = a0.x; U.v[3] = a0.y; U.v[5] = a0.z; U.v[6] = a0.w;
  U.v[1] = a1.x; U.v[2] = a1.y; U.v[4] = a1.z; U.v[7] = a1.w;
  const float4 R4 = reinterpret_cast<const float4*>(rf)[COL * no + o];
  Oct8 EE;
#pragma unroll
  for (int i = 0; i < 8; ++i) EE.v[i] = __expf(U.v[i]);
  // LIN: corrections of the other colour (the in-oct neighbours)
  const float4 XO = LIN ? e4[OC * no + o] : make_float4(0.f, 0.f, 0.f, 0.f);
  bool on[4];
  float s1[4], s2[4], s3[4];  // LIN: (sum off*e, diag sum, -); NL: (sum b du, sum du, sum b)
  // the oct's eight relax flags in one 8-byte load
  const unsigned long long a8 = act ? __ldg(reinterpret_cast<const unsigned long long*>(act) + o)
                                    : ~0ULL;
  // the six face neighbours as three 8-byte loads (6 o ints: 8-byte aligned)
  const int2* nb2 = reinterpret_cast<const int2*>(nbr) + 3 * o;
  const int2 n01 = __ldg(nb2), n23 = __ldg(nb2 + 1), n45 = __ldg(nb2 + 2);
  const int nbv[6] = {n01.x, n01.y, n23.x, n23.y, n45.x, n45.y};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int ch = CC[COL][q];
    on[q] = ((a8 >> (8 * ch)) & 0xffULL) != 0ULL;
    s1[q] = s2[q] = s3[q] = 0.f;
    // in-oct neighbours (other colour, unchanged in this half-sweep)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int cn = ch ^ (1 << (2 - a));
      const float du = U.v[cn] - U.v[ch];
      if (LIN) {
        s1[q] = fmaf(0.5f * ih2 * fmaf(EE.v[cn], du, EE.v[ch] + EE.v[cn]), f4(XO, cn >> 1),
                     s1[q]);
        s2[q] += fmaf(EE.v[ch], du, -EE.v[ch] - EE.v[cn]);
      } else {
        const float b = 0.5f * (EE.v[cn] + EE.v[ch]);
        s1[q] = fmaf(b, du, s1[q]);
        s2[q] += du;
        s3[q] += b;
      }
    }
  }
  // faces: the neighbouring oct's other colour, or the ghost face
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int a = d >> 1, plus = d & 1;
    const int nb = nbv[d];
    const bool has = nb >= 0;
    float4 NU, NX = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!LIN) {
      NU = has ? uo[nb] : g4[-nb - 1];  // one load, no divergent branch
    } else if (has) {
      NU = uo[nb];
      NX = e4[OC * no + nb];
    } else {
      NU = g4[-nb - 1];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ch = CC[COL][q];
      if (((ch >> (2 - a)) & 1) != plus) continue;  // not on this face
      const int cn = ch ^ (1 << (2 - a));
      const float un = has ? f4(NU, cn >> 1) : f4(NU, face_q(ch, a));
      const float xn = (LIN && has) ? f4(NX, cn >> 1) : 0.f;
      const float En = __expf(un);
      const float du = un - U.v[ch];
      if (LIN) {
        s1[q] = fmaf(0.5f * ih2 * fmaf(En, du, EE.v[ch] + En), xn, s1[q]);
        s2[q] += fmaf(EE.v[ch], du, -EE.v[ch] - En);
      } else {
        const float b = 0.5f * (En + EE.v[ch]);
        s1[q] = fmaf(b, du, s1[q]);
        s2[q] += du;
        s3[q] += b;
      }
    }
  }
  // the colour-COL vector: new values on relaxed cells, the old ones elsewhere
  float4 out = LIN ? (act ? e4[COL * no + o] : make_float4(0.f, 0.f, 0.f, 0.f))
                   : make_float4(U.v[CC[COL][0]], U.v[CC[COL][1]], U.v[CC[COL][2]],
                                 U.v[CC[COL][3]]);
  float res[4] = {out.x, out.y, out.z, out.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!on[q]) continue;
    const int ch = CC[COL][q];
    const float sN = nls(U.v[ch], EE.v[ch], m);
    if (LIN) {
      const float diag = s2[q] * 0.5f * ih2 + m.aRt_np1 * sN;
      res[q] = __fdividef(f4(R4, q) - s1[q], diag);
    } else {
      const float L = s1[q] * ih2 + m.aRt * (1.f - sN);
      const float dL = (0.5f * EE.v[ch] * s2[q] - s3[q]) * ih2 + m.aRt_np1 * sN;
      float step = __fdividef(L - f4(R4, q), dL);
      step = fminf(fmaxf(step, -cap), cap);
      res[q] = U.v[ch] - step;
    }
  }
  reinterpret_cast<float4*>(LIN ? e : u)[COL * no + o] =
      make_float4(res[0], res[1], res[2], res[3]);
}

// ---- thread-per-oct FP32 operator sums ------------------------------------
// For every cell c of oct o, over its six neighbours j (three in the oct, one
// across each of its three outer faces: the neighbouring oct or the ghost),
// with E = e^u from the SFU:
//   NL : s1_c = sum_j 1/2 (E_j + E_c)(u_j - u_c)          (h^2 times the
//        divergence term of L_c, Sec. 3.2)
//   LIN: s1_c = sum_j (E_j (u_j - u_c) + E_c + E_j) x_j   (2 h^2 times the
//        off-diagonal part of (J x)_c; x = 0 at ghosts)
//        s2_c = sum_j (E_c (u_j - u_c) - E_c - E_j)       (2 h^2 times the
//        divergence part of J_cc)
// Each face is loaded once per oct instead of once per cell.
template <bool LIN>
__device__ __forceinline__ void oct_sums(const float* __restrict__ u, const float* __restrict__ x,
                                         const int* __restrict__ nbr,
                                         const float* __restrict__ gh, long long o, long long no,
                                         const Oct8& U, const Oct8& EE, const Oct8& X, float* s1,
                                         float* s2) {
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    s1[ch] = 0.f;
    s2[ch] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int cn = ch ^ (1 << (2 - a));
      const float du = U.v[cn] - U.v[ch];
      if (LIN) {
        s1[ch] = fmaf(fmaf(EE.v[cn], du, EE.v[ch] + EE.v[cn]), X.v[cn], s1[ch]);
        s2[ch] += fmaf(EE.v[ch], du, -EE.v[ch] - EE.v[cn]);
      } else {
        s1[ch] = fmaf(0.5f * (EE.v[cn] + EE.v[ch]), du, s1[ch]);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int a = d >> 1, plus = d & 1;
    const int nb = nbr[6 * o + d];
    Oct8 NU, NX;
    float G[4];
    if (nb >= 0) {
      NU = ld8(u, nb, no);
      if (LIN) NX = ld8(x, nb, no);
    } else {
      const float4 g = *reinterpret_cast<const float4*>(gh + 4LL * (-nb - 1));
      G[0] = g.x;
      G[1] = g.y;
      G[2] = g.z;
      G[3] = g.w;
    }
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      if (((ch >> (2 - a)) & 1) != plus) continue;  // not on this face
      float un, xn;
      if (nb >= 0) {
        const int cn = ch ^ (1 << (2 - a));
        un = NU.v[cn];
        xn = LIN ? NX.v[cn] : 0.f;
      } else {
        un = G[face_q(ch, a)];
        xn = 0.f;
      }
      const float En = __expf(un), du = un - U.v[ch];
      if (LIN) {
        s1[ch] = fmaf(fmaf(En, du, EE.v[ch] + En), xn, s1[ch]);
        s2[ch] += fmaf(EE.v[ch], du, -EE.v[ch] - En);
      } else {
        s1[ch] = fmaf(0.5f * (En + EE.v[ch]), du, s1[ch]);
      }
    }
  }
}

__device__ __forceinline__ void block_partials3(double ss, double mx, double fs,
                                                double* __restrict__ partials) {
  __shared__ double s1[BS / 32], s2[BS / 32], s3[BS / 32];
  for (int q = 16; q > 0; q >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, q);
    fs += __shfl_xor_sync(0xffffffffu, fs, q);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, q));
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = ss;
    s2[threadIdx.x >> 5] = mx;
    s3[threadIdx.x >> 5] = fs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, e = 0.0;
    for (int w = 0; w < BS / 32; ++w) {
      a += s1[w];
      b = fmax(b, s2[w]);
      e += s3[w];
    }
    partials[3 * blockIdx.x] = a;
    partials[3 * blockIdx.x + 1] = b;
    partials[3 * blockIdx.x + 2] = e;
  }
}

// FP32 residual norms of the solved level (sum r^2, max |r|, sum f^2), one
// thread per oct; the oct's eight terms are summed in FP32, the octs in FP64.
__global__ void __launch_bounds__(BS) k_onorm32(const float* __restrict__ u,
                                                const float* __restrict__ f,
                                                const int* __restrict__ nbr,
                                                const float* __restrict__ gh, long long n_oct,
                                                MT<float> m, float ih2,
                                                double* __restrict__ partials) {
  double ss = 0.0, mx = 0.0, fs = 0.0;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n_oct;
       o += (long long)gridDim.x * blockDim.x) {
    const Oct8 U = ld8(u, o, n_oct), Fv = ld8(f, o, n_oct);
    Oct8 EE;
#pragma unroll
    for (int i = 0; i < 8; ++i) EE.v[i] = __expf(U.v[i]);
    float s1[8], s2[8];
    oct_sums<false>(u, nullptr, nbr, gh, o, n_oct, U, EE, U, s1, s2);
    float ss8 = 0.f, mx8 = 0.f, fs8 = 0.f;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      const float L = s1[ch] * ih2 + m.aRt * (1.f - nls(U.v[ch], EE.v[ch], m));
      const float r = Fv.v[ch] - L;
      ss8 = fmaf(r, r, ss8);
      mx8 = fmaxf(mx8, fabsf(r));
      fs8 = fmaf(Fv.v[ch], Fv.v[ch], fs8);
    }
    ss += ss8;
    mx = fmax(mx, (double)mx8);
    fs += fs8;
  }
  block_partials3(ss, mx, fs, partials);
}

// FAS right-hand side on a coarse oct level (FP32): f += L(u) at relaxed cells
__global__ void __launch_bounds__(BS) k_ofas32(const float* __restrict__ u, float* __restrict__ f,
                                               const int* __restrict__ nbr,
                                               const float* __restrict__ gh,
                                               const unsigned char* __restrict__ act, long long n,
                                               const int* __restrict__ olist, long long no,
                                               MT<float> m, float ih2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long o = olist ? olist[t] : t;
  const Oct8 U = ld8(u, o, no);
  Oct8 EE;
#pragma unroll
  for (int i = 0; i < 8; ++i) EE.v[i] = __expf(U.v[i]);
  float s1[8], s2[8];
  oct_sums<false>(u, nullptr, nbr, gh, o, no, U, EE, U, s1, s2);
  Oct8 Fv = ld8(f, o, no);
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    if (act[8 * o + ch]) Fv.v[ch] += s1[ch] * ih2 + m.aRt * (1.f - nls(U.v[ch], EE.v[ch], m));
  st8(f, o, no, Fv);
}

// FAS restriction of one oct to its parent (FP32): u average, average of the
// residual f - L(u) over the oct's relaxed cells.  pno: octs of the parent
// level (0: dense).
__global__ void __launch_bounds__(BS) k_orestrict32(
    const float* __restrict__ u, const float* __restrict__ f, const int* __restrict__ nbr,
    const float* __restrict__ gh, const unsigned char* __restrict__ act, long long n,
    const int* __restrict__ olist, long long no, const int* __restrict__ pcell, long long pno,
    MT<float> m, float ih2, float* __restrict__ uc, float* __restrict__ ucold,
    float* __restrict__ fc) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long o = olist ? olist[t] : t;
  const Oct8 U = ld8(u, o, no), Fv = ld8(f, o, no);
  Oct8 EE;
#pragma unroll
  for (int i = 0; i < 8; ++i) EE.v[i] = __expf(U.v[i]);
  float s1[8], s2[8];
  oct_sums<false>(u, nullptr, nbr, gh, o, no, U, EE, U, s1, s2);
  float su = 0.f, sr = 0.f;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    su += U.v[ch];
    if (!act || act[8 * o + ch])
      sr += Fv.v[ch] - (s1[ch] * ih2 + m.aRt * (1.f - nls(U.v[ch], EE.v[ch], m)));
  }
  const long long p = pidx(pcell[o], pno);
  const float um = 0.125f * su;
  uc[p] = um;
  ucold[p] = um;
  fc[p] = 0.125f * sr;
}

// Linear-phase restriction of one oct: r_c = R(r - J e) over relaxed cells,
// u_c = R(u), e_c = 0.
__global__ void __launch_bounds__(BS) k_olin_restrict32(
    const float* __restrict__ e, const float* __restrict__ r, const float* __restrict__ u,
    const int* __restrict__ nbr, const float* __restrict__ gh,
    const unsigned char* __restrict__ act, long long n, const int* __restrict__ olist,
    long long no, const int* __restrict__ pcell, long long pno, MT<float> m, float ih2,
    float* __restrict__ rc, float* __restrict__ uc, float* __restrict__ ec) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long o = olist ? olist[t] : t;
  const Oct8 U = ld8(u, o, no), X = ld8(e, o, no), R = ld8(r, o, no);
  Oct8 EE;
#pragma unroll
  for (int i = 0; i < 8; ++i) EE.v[i] = __expf(U.v[i]);
  float s1[8], s2[8];
  oct_sums<true>(u, e, nbr, gh, o, no, U, EE, X, s1, s2);
  const float h2 = 0.5f * ih2;
  float su = 0.f, sr = 0.f;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    su += U.v[ch];
    if (!act || act[8 * o + ch]) {
      const float diag = s2[ch] * h2 + m.aRt_np1 * nls(U.v[ch], EE.v[ch], m);
      sr += R.v[ch] - fmaf(diag, X.v[ch], s1[ch] * h2);
    }
  }
  const long long p = pidx(pcell[o], pno);
  uc[p] = 0.125f * su;
  rc[p] = 0.125f * sr;
  ec[p] = 0.f;
}

// Prolongation of a coarse correction to the relaxed cells of one oct (FP32):
// the parent's value c plus, per axis, s (c+ - c-)/8 from the parent's two
// neighbours (a component is 0 where one is missing), s = +1 or -1 for the
// daughter's high or low position.  NL: c = uc - ucold (FAS), added to u;
// LIN: c = e_c, added to e.  The oct is read and written whole.
template <bool LIN>
__global__ void __launch_bounds__(BS) k_oprolong32(long long n, const int* __restrict__ olist,
                                                   long long no, const int* __restrict__ pcell,
                                                   const int* __restrict__ pnbr, long long pno,
                                                   const float* __restrict__ uc,
                                                   const float* __restrict__ ucold,
                                                   const unsigned char* __restrict__ act,
                                                   int linear, float* __restrict__ u) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long o = olist ? olist[t] : t;
  auto corr = [&](int q) -> float {
    const long long k = pidx(q, pno);
    if constexpr (LIN)
      return uc[k];
    else
      return uc[k] - ucold[k];
  };
  const float v0 = corr(pcell[o]);
  float g[3] = {0.f, 0.f, 0.f};
  bool have[3] = {false, false, false};
  if (linear) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int pm = pnbr[6 * o + 2 * ax], pp = pnbr[6 * o + 2 * ax + 1];
      if (pm < 0 || pp < 0) continue;
      g[ax] = corr(pp) - corr(pm);
      have[ax] = true;
    }
  }
  Oct8 U = ld8(u, o, no);
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    if (act && !(act[8 * o + ch])) continue;
    float v = v0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
      if (have[ax]) v += (((ch >> (2 - ax)) & 1) ? 0.125f : -0.125f) * g[ax];
    U.v[ch] += v;
  }
  st8(u, o, no, U);
}

// ---- phase B in double-float (mixed form) ---------------------------------
// From the end of phase A until the level is finished, the FP64 work arrays of
// the level being solved (w, wE, wf) and its FP64 ghost slots hold
// double-float pairs in their 8 bytes; the FP64-accurate residual, e^u and
// the corrections then run on the FP32 pipes.  k_df2d turns them back into
// FP64 (level output, or the FP64 fallback).

struct MDF {
  dfl aRt, inv_np1, ih2h;  // alpha Rt, 1/(n+1), 1/(2 h^2)
  int n;
};

MDF mdf(const Model& m, double ih2) {
  return MDF{df_from_double(m.aRt), df_from_double(m.inv_np1), df_from_double(0.5 * ih2), m.n};
}

// one double-float value as a single 8-byte load
__device__ __forceinline__ dfl ldf(const dfl* __restrict__ p, long long i) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
  return dfl{v.x, v.y};
}

// the four double-float values of half h of oct o (cells 4h .. 4h+3: 32
// contiguous bytes, two 16-byte loads)
__device__ __forceinline__ void ld4df(const dfl* __restrict__ p, long long o, int h, dfl* x) {
  const float4* q = reinterpret_cast<const float4*>(p + 8 * o + 4 * h);
  const float4 a = __ldg(q), b = __ldg(q + 1);
  x[0] = dfl{a.x, a.y};
  x[1] = dfl{a.z, a.w};
  x[2] = dfl{b.x, b.y};
  x[3] = dfl{b.z, b.w};
}

// r = f - L(u) to FP64 accuracy in double-float (Sec. 3.2 operator); stores r
// and u rounded to FP32 for the linear cycles, zeroes the correction e, and
// accumulates the norms (FP32 within a thread, FP64 across threads: they feed
// only the stopping test).  Two threads per oct, one per x half (cells 4h +
// q, q = 2 y + z): the flux across each inner face, (E_i + E_j)(u_j - u_i),
// is formed once per face inside a half and once by each thread across the
// middle x face, and enters the two cells with opposite signs (the
// double-float sum, difference and product are odd under negation, so each
// cell's terms are those of a cell-by-cell evaluation); every cell sums its
// six terms in the direction order -x, +x, -y, +y, -z, +z.
__global__ void __launch_bounds__(BS, 4) k_oresid_df(
    const dfl* __restrict__ u, const dfl* __restrict__ E, const dfl* __restrict__ f,
    const int* __restrict__ nbr, const dfl* __restrict__ gh, const dfl* __restrict__ ghE,
    MDF m, long long no, float* __restrict__ r32, float* __restrict__ u32,
    float* __restrict__ e32, double* __restrict__ partials) {
  float ss = 0.f, mx = 0.f, fs = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * no;
       t += (long long)gridDim.x * blockDim.x) {
    const long long o = t >> 1;
    const int h = (int)(t & 1);
    dfl U[4], Ev[4], acc[4];
    ld4df(u, o, h, U);
    ld4df(E, o, h, Ev);
    // x: the outer face on side h, and the middle face (cell 4h + q against
    // 4(1-h) + q of the other half)
    {
      dfl Up[4], Ep[4];
      ld4df(u, o, 1 - h, Up);
      ld4df(E, o, 1 - h, Ep);
      const int nb = nbr[6 * o + h];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ch = 4 * h + q;
        dfl ue, Ee;
        if (nb >= 0) {
          ue = ldf(u, 8LL * nb + (ch ^ 4));
          Ee = ldf(E, 8LL * nb + (ch ^ 4));
        } else {
          ue = ldf(gh, 4LL * (-nb - 1) + face_q(ch, 0));
          Ee = ldf(ghE, 4LL * (-nb - 1) + face_q(ch, 0));
        }
        const dfl ext = df_mul(df_add_abs(Ee, Ev[q]), df_add_abs(ue, df_neg(U[q])));
        const dfl zero{0.f, 0.f};
        if (h == 0) {  // this cell is ch0 of the middle face: -x outer, then +x inner
          const dfl Fin = df_mul(df_add_abs(Ep[q], Ev[q]), df_add_abs(Up[q], df_neg(U[q])));
          acc[q] = df_add_abs(df_add_abs(zero, ext), Fin);
        } else {       // ch1: -x inner, then +x outer
          const dfl Fin = df_mul(df_add_abs(Ev[q], Ep[q]), df_add_abs(U[q], df_neg(Up[q])));
          acc[q] = df_add_abs(df_add_abs(zero, df_neg(Fin)), ext);
        }
      }
    }
    // y and z: faces inside the half, outer faces on both sides
#pragma unroll
    for (int ax = 1; ax < 3; ++ax) {
      const int sh = 2 - ax;
      const int nm = nbr[6 * o + 2 * ax], np = nbr[6 * o + 2 * ax + 1];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        // q0 has bit sh clear, q1 is its partner across the face
        const int q0 = ((p >> sh) << (sh + 1)) | (p & ((1 << sh) - 1));
        const int q1 = q0 | (1 << sh);
        const int ch0 = 4 * h + q0, ch1 = 4 * h + q1;
        const int qi = face_q(ch0, ax);
        dfl um, Em, up, Ep;  // across the minus face of ch0, the plus face of ch1
        if (nm >= 0) {
          um = ldf(u, 8LL * nm + ch1);
          Em = ldf(E, 8LL * nm + ch1);
        } else {
          um = ldf(gh, 4LL * (-nm - 1) + qi);
          Em = ldf(ghE, 4LL * (-nm - 1) + qi);
        }
        if (np >= 0) {
          up = ldf(u, 8LL * np + ch0);
          Ep = ldf(E, 8LL * np + ch0);
        } else {
          up = ldf(gh, 4LL * (-np - 1) + qi);
          Ep = ldf(ghE, 4LL * (-np - 1) + qi);
        }
        const dfl Fin = df_mul(df_add_abs(Ev[q1], Ev[q0]), df_add_abs(U[q1], df_neg(U[q0])));
        acc[q0] = df_add_abs(acc[q0], df_mul(df_add_abs(Em, Ev[q0]), df_add_abs(um, df_neg(U[q0]))));
        acc[q0] = df_add_abs(acc[q0], Fin);
        acc[q1] = df_add_abs(acc[q1], df_neg(Fin));
        acc[q1] = df_add_abs(acc[q1], df_mul(df_add_abs(Ep, Ev[q1]), df_add_abs(up, df_neg(U[q1]))));
      }
    }
    dfl F4[4];
    ld4df(f, o, h, F4);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const dfl sN = m.n == 1 ? df_rsqrt(Ev[q]) : df_exp(df_neg(df_mul(U[q], m.inv_np1)));
      const dfl L = df_add(df_mul(acc[q], m.ih2h), df_mul(m.aRt, df_add_f(df_neg(sN), 1.f)));
      const dfl r = df_sub(F4[q], L);
      const long long k = pidx(8 * o + 4 * h + q, no);
      r32[k] = r.hi;
      u32[k] = U[q].hi;
      e32[k] = 0.f;
      ss = fmaf(r.hi, r.hi, ss);
      mx = fmaxf(mx, fabsf(r.hi));
      fs = fmaf(F4[q].hi, F4[q].hi, fs);
    }
  }
  block_partials3((double)ss, (double)mx, (double)fs, partials);
}

// FP32 iterate -> double-float iterate and its e^u
__global__ void k_f2df_exp(const float* __restrict__ w32, long long no, dfl* __restrict__ w,
                           dfl* __restrict__ wE, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dfl v{w32[pidx(i, no)], 0.f};
  w[i] = v;
  wE[i] = df_exp(v);
}

// w += clamp(e), wE = e^w (double-float)
__global__ void k_apply_df(dfl* __restrict__ w, dfl* __restrict__ wE, const float* __restrict__ e,
                           long long no, long long n, float cap) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dfl v = df_add_f(w[i], fminf(fmaxf(e[pidx(i, no)], -cap), cap));
  w[i] = v;
  wE[i] = df_exp(v);
}

// double-float -> FP64 (in place allowed) and back
__global__ void k_df2d(const dfl* __restrict__ x, double* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    const dfl v = x[i];
    y[i] = df_to_double_bits(v);
  }
}
__global__ void k_d2df(const double* __restrict__ x, dfl* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = x[i];
    y[i] = df_from_double_bits(v);
  }
}

// ---- set-up kernels --------------------------------------------------------
// initial guess of level L from the converged level L-1 (linear
// reconstruction with the parent's neighbours), FP64 and FP32 copies
__global__ void k_init_level(long long ncell, const int* __restrict__ pcell,
                             const int* __restrict__ pnbr, const double* __restrict__ up,
                             int linear, double* __restrict__ w, double* __restrict__ wE,
                             float* __restrict__ w32, long long no) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const long long o = c >> 3;
  const int ch = (int)(c & 7);
  if (w32) {
    // mixed form: an FP32 guess (the FP64 iterate is taken from w32 later),
    // with the parent values converted on the integer pipes
    float v = f_from_double_bits(up[pcell[o]]);
    if (linear) {
      for (int ax = 0; ax < 3; ++ax) {
        const int pm = pnbr[6 * o + 2 * ax], pp = pnbr[6 * o + 2 * ax + 1];
        if (pm < 0 || pp < 0) continue;
        v = fmaf(((ch >> (2 - ax)) & 1) ? 0.125f : -0.125f,
                 f_from_double_bits(up[pp]) - f_from_double_bits(up[pm]), v);
      }
    }
    w32[pidx(c, no)] = v;
    return;
  }
  double v = up[pcell[o]];
  if (linear) {
    for (int ax = 0; ax < 3; ++ax) {
      const int pm = pnbr[6 * o + 2 * ax], pp = pnbr[6 * o + 2 * ax + 1];
      if (pm < 0 || pp < 0) continue;
      v += (((ch >> (2 - ax)) & 1) ? 0.125 : -0.125) * (up[pp] - up[pm]);
    }
  }
  w[c] = v;
  wE[c] = exp(v);
}

// Start of level L from the previous particle solve where its octs persist
// (start = MGFR_START_PREVIOUS_ALL): the oct whose parent cell has the same
// Morton key, found by binary search in the previous solve's keys (increasing,
// the storage order), lends its eight converged values; the other octs keep
// the prolonged guess of k_init_level.
__global__ void k_warm_level(const int4* __restrict__ opos, long long n_oct,
                             const unsigned long long* __restrict__ pkey, long long pn,
                             const double* __restrict__ pu, double* __restrict__ w,
                             double* __restrict__ wE, float* __restrict__ w32) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= n_oct) return;
  const int4 p = opos[o];
  const unsigned long long key = morton3((unsigned)p.x, (unsigned)p.y, (unsigned)p.z);
  long long lo = 0, hi = pn;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (pkey[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo >= pn || pkey[lo] != key) return;
  for (int ch = 0; ch < 8; ++ch) {
    const double v = pu[8 * lo + ch];
    if (w32) {
      w32[pidx(8 * o + ch, n_oct)] = f_from_double_bits(v);
    } else {
      w[8 * o + ch] = v;
      wE[8 * o + ch] = exp(v);
    }
  }
}

// Ghost values on the faces of level-l octs that have no neighbouring oct
// (Sec. 3.3), one thread per ghost value: slot s = t / 4 (its face 6 o + d
// from gface), qi = t % 4 the face cell.  The face's four outside cells are
// daughters of one level-(l-1) cell P, the oct's parent shifted along the face
// normal; the four threads of a face look up P and its six neighbours (the
// same addresses).  A ghost is P's value plus, per axis, s (c+ - c-)/8,
// s = +1 or -1 for the ghost's high or low daughter position in P (a
// component is 0 where one of P's neighbours does not exist).  Written as
// (u, e^u) in FP64 (double-float pairs in the mixed form) and FP32 u.
__global__ void k_ghosts(long long n_gslot, int l, TreeView T, const unsigned* __restrict__ gface,
                         const double* __restrict__ up, int linear, double* __restrict__ ghost,
                         double* __restrict__ ghostE, float* __restrict__ g32, int dfmode) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 4 * n_gslot) return;
  const unsigned f = gface[t >> 2];
  const int qi = (int)(t & 3);
  const unsigned o = f / 6u;
  const int d = (int)(f - 6u * o);
  const int ax = d >> 1, plus = d & 1;
  const int t1 = ax == 0 ? 1 : 0;  // the first tangential axis
  const int4 p = T.opos[l][o];
  const long long P0 = p.x + (ax == 0 ? (plus ? 1 : -1) : 0);
  const long long P1 = p.y + (ax == 1 ? (plus ? 1 : -1) : 0);
  const long long P2 = p.z + (ax == 2 ? (plus ? 1 : -1) : 0);
  int lev;
  const long long pc = find_cell(T, l - 1, P0, P1, P2, &lev);
  // per axis, the indices of P's two neighbours (-1: no gradient)
  long long cm[3] = {-1, -1, -1}, cp[3] = {-1, -1, -1};
  if (lev == l - 1 && linear) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int lp, lm;
      const long long qp = find_cell(T, l - 1, P0 + (a == 0), P1 + (a == 1), P2 + (a == 2), &lp);
      const long long qm = find_cell(T, l - 1, P0 - (a == 0), P1 - (a == 1), P2 - (a == 2), &lm);
      if (lp == l - 1 && lm == l - 1) {
        cp[a] = qp;
        cm[a] = qm;
      }
    }
  }
  // daughter bit of the ghost along axis a inside P: along the normal the
  // side facing the oct, tangentially the oct cell's own bits (qi's two bits)
  auto hbit = [&](int a) { return a == ax ? 1 - plus : a == t1 ? (qi >> 1) & 1 : qi & 1; };
  if (dfmode) {
    // double-float slots (phase B of the mixed form): the parent's FP64
    // values converted on the integer pipes, the stencil and e^v on the FP32
    // pipes
    dfl V{0.f, 0.f};
    if (lev == l - 1) V = df_from_double_bits(up[pc]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (cp[a] >= 0) {
        const dfl g = df_mul_f(df_sub(df_from_double_bits(up[cp[a]]),
                                      df_from_double_bits(up[cm[a]])),
                               hbit(a) ? 0.125f : -0.125f);
        V = df_add(V, g);
      }
    reinterpret_cast<dfl*>(ghost)[t] = V;
    reinterpret_cast<dfl*>(ghostE)[t] = df_exp(V);
    g32[t] = V.hi;
    return;
  }
  double v = lev == l - 1 ? up[pc] : 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (cp[a] >= 0) v += (hbit(a) ? 0.125 : -0.125) * (up[cp[a]] - up[cm[a]]);
  ghost[t] = v;
  ghostE[t] = exp(v);
  g32[t] = (float)v;
}

// FP64 cell array -> FP32 array of a level (no: its octs, 0 for dense)
__global__ void k_d2f(const double* __restrict__ x, float* __restrict__ y, long long n,
                      long long no) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[pidx(i, no)] = f_from_double_bits(x[i]);
}

// the same into two arrays
__global__ void k_d2f2(const double* __restrict__ x, float* __restrict__ y, float* __restrict__ z,
                       long long n, long long no) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    const float v = f_from_double_bits(x[i]);
    const long long q = pidx(i, no);
    y[q] = v;
    z[q] = v;
  }
}

// FP64 iterate from the FP32 one: w = w32, wE = e^w
__global__ void k_f2d_exp(const float* __restrict__ w32, long long no, double* __restrict__ w,
                          double* __restrict__ wE, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = (double)w32[pidx(i, no)];
  w[i] = v;
  wE[i] = exp(v);
}

__global__ void k_mask_up(const float* __restrict__ mchild, long long n_oct,
                          const int* __restrict__ pcell, float* __restrict__ mparent) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= n_oct) return;
  float s = 0.f;
  for (int q = 0; q < 8; ++q) s += mchild[8 * o + q];
  mparent[pcell[o]] = 0.125f * s;
}

__global__ void k_mask_dense(const float* __restrict__ mf, int lgf, float* __restrict__ mc) {
  const int lgc = lgf - 1, Nc = 1 << lgc;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lgc))) return;
  const int K = (int)(t & (Nc - 1)), J = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  float s = 0.f;
  for (int q = 0; q < 8; ++q)
    s += mf[cidx(2 * I + (q >> 2), 2 * J + ((q >> 1) & 1), 2 * K + (q & 1), lgf)];
  mc[t] = 0.125f * s;
}

__global__ void k_fill_f(float* __restrict__ x, long long n, float v) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

// act[c] = 1 where the multigrid mask relaxes cell c (mask > threshold): one
// byte per cell for the sweeps instead of the float mask
__global__ void k_act(const float* __restrict__ mask, long long n, float mthr,
                      unsigned char* __restrict__ act) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) act[i] = mask[i] > mthr ? 1 : 0;
}

__global__ void k_count_relaxed(const float* __restrict__ mask, long long n, float mthr,
                                long long* __restrict__ out) {
  long long cnt = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    cnt += mask[i] > mthr;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd((unsigned long long*)out, (unsigned long long)cnt);
}

// Octs of a coarse level holding at least one relaxed cell, appended with one
// atomic per warp (order within a warp kept; any order is valid, since each
// kernel over the list updates cells independently of the visiting order).
__global__ void k_oct_list(const float* __restrict__ mask, long long n_oct, float mthr,
                           int* __restrict__ list, unsigned long long* __restrict__ count) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool act = false;
  if (o < n_oct) {
    const float4* m4 = reinterpret_cast<const float4*>(mask + 8 * o);
    const float4 a = m4[0], b = m4[1];
    act = a.x > mthr || a.y > mthr || a.z > mthr || a.w > mthr || b.x > mthr || b.y > mthr ||
          b.z > mthr || b.w > mthr;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, act);
  if (!bal) return;
  const int lane = threadIdx.x & 31, lead = __ffs(bal) - 1;
  unsigned long long base = 0;
  if (lane == lead) base = atomicAdd(count, (unsigned long long)__popc(bal));
  base = __shfl_sync(0xffffffffu, base, lead);
  if (act) list[base + __popc(bal & ((1u << lane) - 1u))] = (int)o;
}

}  // namespace

// ============================================================================
// host orchestration
// ============================================================================
namespace {

// work arrays of one tree level in precision T
template <class T>
struct TA {
  T *w, *wE, *wf, *wold, *gh, *ghE;
};

template <class T>
TA<T> tarr(AmrLevel& L);
template <>
TA<double> tarr<double>(AmrLevel& L) {
  return TA<double>{L.w, L.wE, L.wf, L.wold, L.ghost, L.ghostE};
}
template <>
TA<float> tarr<float>(AmrLevel& L) {
  return TA<float>{L.w32, L.wE32, L.wf32, L.wold32, L.ghost32, nullptr};
}

// work arrays of dense level k of the hierarchy below the base (k >= 1)
template <class T>
TA<T> darr(DenseLevel& D);
template <>
TA<double> darr<double>(DenseLevel& D) {
  return TA<double>{D.u, D.E, D.f, D.uold, nullptr, nullptr};
}
template <>
TA<float> darr<float>(DenseLevel& D) {
  return TA<float>{D.u32, D.e32, D.f32, D.uold32, nullptr, nullptr};
}

struct SolveCtx {
  mgfr_ctx* c;
  AmrWork* A;
  Model m;
  int L;
  float mthr;
  long long updates;      // nonlinear NGS cell updates (tree levels)
  int kmax;  // deepest dense level below the base holding a relaxed cell (0: none)
  long long lin_updates = 0;  // FP32 linear Gauss-Seidel cell updates (tree levels)
};

// whether the coarse grid below tree level l >= 1 of the level-S.L solve has
// a relaxed cell (otherwise the cycle stops at level l)
// A dense coarse grid (the base or a level below it) costs a pass over all its
// cells per kernel but helps only where cells relax: the cycle descends to it
// only when at least 1/kDenseMinDiv of its cells relax, and otherwise stops at
// the finer level, whose few coarse-covered cells the smoothing settles.
constexpr long long kDenseMinDiv = 64;

bool has_coarse(const SolveCtx& S, int l) {
  const AmrLevel& P = S.A->L[l - 1];
  return l - 1 >= 1 ? P.n_list > 0 : P.relaxed * kDenseMinDiv >= P.ncell;
}

// Octs visited on tree level l >= 1 of the level-S.L solve: every oct of the
// solved level, the active-oct list on a coarser level.
struct ORange {
  const int* list;
  long long n;
};

// the relaxed-cell lists of dense level k (0: the base) where this solve
// built them
CList clist(const SolveCtx& S, int k) {
  const DenseHier& H = S.c->dh;
  if (!(k == 0 || (k <= S.kmax && H.L[k].N > 4))) return CList{nullptr, 0, 0, 0};
  return CList{S.A->dlist[k], H.L[k].n / 2, S.A->dlist_n[k][0], S.A->dlist_n[k][1]};
}
// threads of a launch over dense level cells: the listed ones, else all n
long long cl_threads(const CList& L, long long n) { return L.p ? L.n0 + L.n1 : n; }

// red-black sweeps on tree level l (l < S.L, or k >= 1 dense: a coarse grid)
int sweeps_of(const SolveCtx& S, int l, int n) {
  const int nc = S.c->cfg.n_coarse;
  return l != S.L && nc > 0 ? nc : n;
}
ORange orange(const SolveCtx& S, const AmrLevel& L, int l) {
  return l == S.L ? ORange{nullptr, L.n_oct} : ORange{L.olist, L.n_list};
}

template <class T>
void relax(SolveCtx& S, int l, int sweeps) {
  mgfr_ctx* c = S.c;
  AmrLevel& L = S.A->L[l];
  const mgfr_config& g = c->cfg;
  const MT<T> m = mt<T>(S.m);
  TA<T> a = tarr<T>(L);
  for (int s = 0; s < sweeps; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l >= 1) {
        const ORange R = orange(S, L, l);
        if (R.n == 0) continue;
        if (l == S.L) prof_begin(c, 3, L.ncell);
        if constexpr (std::is_same<T, float>::value) {
          const unsigned char* mk = l == S.L ? nullptr : L.act;
          if (col == 0)
            k_oct_sweep32<false, 0><<<nblocks(R.n, BS), BS, 0, c->s>>>(
                L.w32, nullptr, L.wf32, L.nbr, L.ghost32, mk, R.n, R.list, L.n_oct, m,
                (float)L.ih2, (float)g.step_cap);
          else
            k_oct_sweep32<false, 1><<<nblocks(R.n, BS), BS, 0, c->s>>>(
                L.w32, nullptr, L.wf32, L.nbr, L.ghost32, mk, R.n, R.list, L.n_oct, m,
                (float)L.ih2, (float)g.step_cap);
        } else {
          k_osweep<T><<<nblocks(4 * R.n, BS), BS, 0, c->s>>>(
              a.w, a.wE, a.wf, L.nbr, a.gh, a.ghE, l == S.L ? nullptr : L.act, R.n,
              R.list, col, m, (T)L.ih2, (T)g.step_cap);
        }
        if (l == S.L) prof_end(c);
      } else {
        const long long nl = S.A->dlist_n[0][col];
        if (nl == 0) continue;
        k_dsweep_list<T><<<nblocks(nl, BS), BS, 0, c->s>>>(
            a.w, a.wE, a.wf, L.lgN, S.A->dlist[0] + col * (L.ncell / 2), nl, m, (T)L.ih2,
            (T)g.step_cap);
      }
      c->launches += 1;
    }
    S.updates += L.relaxed;
  }
}

template <class T>
void vcycle_dense(SolveCtx& S, int k) {
  mgfr_ctx* c = S.c;
  const mgfr_config& g = c->cfg;
  DenseHier& H = c->dh;
  DenseLevel& F = H.L[k];
  const unsigned char* mk = S.A->dact[k];
  const MT<T> m = mt<T>(S.m);
  TA<T> a = darr<T>(F);
  if (F.N <= 4) {
    k_dcoarse<T><<<1, 64, 0, c->s>>>(a.w, a.wE, a.wf, m, (T)F.ih2, (T)g.step_cap, 20, mk);
    c->launches += 1;
    return;
  }
  auto sweep = [&](int sweeps) {
    for (int s = 0; s < sweeps; ++s)
      for (int col = 0; col < 2; ++col) {
        const long long nl = S.A->dlist_n[k][col];
        if (nl == 0) continue;
        k_dsweep_list<T><<<nblocks(nl, BS), BS, 0, c->s>>>(a.w, a.wE, a.wf, F.lg,
                                                            S.A->dlist[k] + col * (F.n / 2), nl,
                                                            m, (T)F.ih2, (T)g.step_cap);
        c->launches += 1;
      }
  };
  sweep(sweeps_of(S, -1, g.n_pre));
  if (k + 1 <= S.kmax) {
    DenseLevel& C = H.L[k + 1];
    TA<T> b = darr<T>(C);
    k_drestrict<T><<<nblocks(C.n, BS), BS, 0, c->s>>>(a.w, a.wE, a.wf, F.lg, b.w, b.wE, b.wold,
                                                      b.wf, m, (T)F.ih2, mk);
    const CList cc = clist(S, k + 1);
    if (cl_threads(cc, C.n) > 0)
      k_dfas<T><<<nblocks(cl_threads(cc, C.n), BS), BS, 0, c->s>>>(b.w, b.wE, b.wf, C.lg, m,
                                                                     (T)C.ih2, S.A->dact[k + 1], cc);
    c->launches += 2;
    vcycle_dense<T>(S, k + 1);
    const CList cf = clist(S, k);
    if (cl_threads(cf, F.n) > 0)
      k_dprolong<T><<<nblocks(cl_threads(cf, F.n), BS), BS, 0, c->s>>>(
          a.w, a.wE, b.w, b.wold, F.lg, g.prolong_linear, mk, cf);
    c->launches += 1;
  }
  sweep(sweeps_of(S, -1, g.n_post));
}

// masked FAS V-cycle of the level-S.L solve at tree level l >= 0
template <class T>
void vcycle_tree(SolveCtx& S, int l) {
  mgfr_ctx* c = S.c;
  AmrWork* A = S.A;
  const mgfr_config& g = c->cfg;
  const MT<T> m = mt<T>(S.m);
  AmrLevel& F = A->L[l];
  TA<T> a = tarr<T>(F);
  relax<T>(S, l, sweeps_of(S, l, g.n_pre));
  const unsigned char* fmask = l == S.L ? nullptr : F.act;
  if (l >= 1 && has_coarse(S, l)) {
    AmrLevel& P = A->L[l - 1];
    TA<T> b = tarr<T>(P);
    const ORange R = orange(S, F, l);
    const long long pno = l - 1 >= 1 ? P.n_oct : 0;  // FP32 parent layout (0: dense)
    if (R.n > 0) {
      if constexpr (std::is_same<T, float>::value)
        k_orestrict32<<<nblocks(R.n, BS), BS, 0, c->s>>>(a.w, a.wf, F.nbr, a.gh, fmask,
                                                         R.n, R.list, F.n_oct, F.pcell, pno, m,
                                                         (T)F.ih2, b.w, b.wold, b.wf);
      else
        k_orestrict<T><<<nblocks(R.n, BS), BS, 0, c->s>>>(a.w, a.wE, a.wf, F.nbr, a.gh, a.ghE,
                                                          fmask, R.n, R.list, F.pcell, m,
                                                          (T)F.ih2, b.w, b.wE, b.wold, b.wf);
    }
    if (l - 1 >= 1) {
      if (P.n_list > 0) {
        if constexpr (std::is_same<T, float>::value)
          k_ofas32<<<nblocks(P.n_list, BS), BS, 0, c->s>>>(b.w, b.wf, P.nbr, b.gh, P.act,
                                                           P.n_list, P.olist, P.n_oct, m,
                                                           (T)P.ih2);
        else
          k_ofas<T><<<nblocks(8 * P.n_list, BS), BS, 0, c->s>>>(b.w, b.wE, b.wf, P.nbr, b.gh,
                                                                b.ghE, P.act, 8 * P.n_list,
                                                                P.olist, m, (T)P.ih2);
      }
    } else {
      const CList c0 = clist(S, 0);
      if (cl_threads(c0, P.ncell) > 0)
        k_dfas<T><<<nblocks(cl_threads(c0, P.ncell), BS), BS, 0, c->s>>>(
            b.w, b.wE, b.wf, P.lgN, m, (T)P.ih2, P.act, c0);
    }
    c->launches += 2;
    vcycle_tree<T>(S, l - 1);
    if (R.n > 0) {
      if constexpr (std::is_same<T, float>::value)
        k_oprolong32<false><<<nblocks(R.n, BS), BS, 0, c->s>>>(R.n, R.list, F.n_oct, F.pcell,
                                                              F.pnbr, pno, b.w, b.wold, fmask,
                                                              g.prolong_linear, a.w);
      else
        k_oprolong<T><<<nblocks(8 * R.n, BS), BS, 0, c->s>>>(8 * R.n, R.list, F.pcell, F.pnbr,
                                                             b.w, b.wold, fmask,
                                                             g.prolong_linear, a.w, a.wE);
    }
    c->launches += 1;
  } else if (l == 0 && S.kmax >= 1) {
    DenseHier& H = c->dh;
    DenseLevel& C = H.L[1];
    TA<T> b = darr<T>(C);
    k_drestrict<T><<<nblocks(C.n, BS), BS, 0, c->s>>>(a.w, a.wE, a.wf, F.lgN, b.w, b.wE, b.wold,
                                                      b.wf, m, (T)F.ih2, F.act);
    const CList c1 = clist(S, 1), c0 = clist(S, 0);
    if (cl_threads(c1, C.n) > 0)
      k_dfas<T><<<nblocks(cl_threads(c1, C.n), BS), BS, 0, c->s>>>(b.w, b.wE, b.wf, C.lg, m,
                                                                     (T)C.ih2, A->dact[1], c1);
    c->launches += 2;
    vcycle_dense<T>(S, 1);
    if (cl_threads(c0, F.ncell) > 0)
      k_dprolong<T><<<nblocks(cl_threads(c0, F.ncell), BS), BS, 0, c->s>>>(
          a.w, a.wE, b.w, b.wold, F.lgN, g.prolong_linear, F.act, c0);
    c->launches += 1;
  }
  relax<T>(S, l, sweeps_of(S, l, g.n_post));
}

// residual norms of level L in precision T -> hs[0..2] (sum r^2, max, sum f^2)
template <class T>
mgfr_status level_norm(SolveCtx& S, double* hs) {
  mgfr_ctx* c = S.c;
  AmrLevel& L = S.A->L[S.L];
  DenseHier& H = c->dh;
  TA<T> a = tarr<T>(L);
  int nparts;
  if constexpr (std::is_same<T, float>::value) {
    nparts = (int)std::min<long long>(H.nparts / 2, nblocks(L.n_oct, BS));
    k_onorm32<<<nparts, BS, 0, c->s>>>(a.w, a.wf, L.nbr, a.gh, L.n_oct, mt<float>(S.m),
                                       (float)L.ih2, H.partials);
  } else {
    nparts = (int)std::min<long long>(H.nparts / 2, nblocks(L.ncell, BS));
    k_onorm<T><<<nparts, BS, 0, c->s>>>(a.w, a.wE, a.wf, L.nbr, a.gh, a.ghE, L.ncell,
                                        mt<T>(S.m), (T)L.ih2, H.partials);
  }
  k_finish3<<<1, 256, 0, c->s>>>(H.partials, nparts, H.scal + 8);
  c->launches += 2;
  MG_CK(c, cudaMemcpyAsync(hs, H.scal + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  return MGFR_OK;
}

mgfr_status count_relaxed(mgfr_ctx* c, AmrWork* A, const float* mask, long long n, float mthr,
                          long long* out) {
  MG_CK(c, cudaMemsetAsync(A->d_small + 2, 0, sizeof(long long), c->s));
  k_count_relaxed<<<(unsigned)std::min<long long>(1024, nblocks(n, BS)), BS, 0, c->s>>>(
      mask, n, mthr, A->d_small + 2);
  c->launches += 1;
  MG_CK(c, cudaMemcpyAsync(out, A->d_small + 2, sizeof(long long), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  return MGFR_OK;
}


// per-colour lists of the relaxed cells of masked dense level k (0: the base)
mgfr_status build_dense_lists(mgfr_ctx* c, AmrWork* A, int k, const unsigned char* act, int lg) {
  MG_CK(c, cudaMemsetAsync(A->d_small + 4, 0, 2 * sizeof(long long), c->s));
  k_dense_list<<<nblocks(1LL << (3 * lg), BS), BS, 0, c->s>>>(
      act, lg, A->dlist[k], (unsigned long long*)(A->d_small + 4));
  c->launches += 1;
  long long n[2] = {0, 0};
  MG_CK(c, cudaMemcpyAsync(n, A->d_small + 4, 2 * sizeof(long long), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  A->dlist_n[k][0] = n[0];
  A->dlist_n[k][1] = n[1];
  return MGFR_OK;
}

// active-oct list of coarse tree level P (octs with a relaxed cell) -> P.olist
mgfr_status build_oct_list(mgfr_ctx* c, AmrWork* A, AmrLevel& P, float mthr) {
  MG_CK(c, cudaMemsetAsync(A->d_small + 3, 0, sizeof(long long), c->s));
  k_oct_list<<<nblocks(P.n_oct, BS), BS, 0, c->s>>>(P.mask, P.n_oct, mthr, P.olist,
                                                    (unsigned long long*)(A->d_small + 3));
  c->launches += 1;
  long long n = 0;
  MG_CK(c, cudaMemcpyAsync(&n, A->d_small + 3, sizeof(long long), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  P.n_list = n;
  return MGFR_OK;
}

// ---- linear masked V-cycle (phase B of the mixed form) -------------------------
// level arrays: u = w32 (linearisation point), E = wE32, r = wf32, e = wold32;
// dense levels below the base: u = u32, E = e32, r = r32, e = uold32.
void lin_relax(SolveCtx& S, int l, int sweeps) {
  mgfr_ctx* c = S.c;
  AmrLevel& L = S.A->L[l];
  const MT<float> m = mt<float>(S.m);
  for (int s = 0; s < sweeps; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l >= 1) {
        const unsigned char* mk = l == S.L ? nullptr : L.act;
        const ORange R = orange(S, L, l);
        if (R.n == 0) continue;
        if (l == S.L) prof_begin(c, 4, L.ncell);
        if (col == 0)
          k_oct_sweep32<true, 0><<<nblocks(R.n, BS), BS, 0, c->s>>>(
              L.w32, L.wold32, L.wf32, L.nbr, L.ghost32, mk, R.n, R.list, L.n_oct, m,
              (float)L.ih2, 0.f);
        else
          k_oct_sweep32<true, 1><<<nblocks(R.n, BS), BS, 0, c->s>>>(
              L.w32, L.wold32, L.wf32, L.nbr, L.ghost32, mk, R.n, R.list, L.n_oct, m,
              (float)L.ih2, 0.f);
        if (l == S.L) prof_end(c);
      } else {
        const long long nl = S.A->dlist_n[0][col];
        if (nl == 0) continue;
        k_dlin_sweep_list<<<nblocks(nl, BS), BS, 0, c->s>>>(
            L.wold32, L.wf32, L.w32, L.wE32, L.lgN, S.A->dlist[0] + col * (L.ncell / 2), nl, m,
            (float)L.ih2);
      }
      c->launches += 1;
    }
  }
}

void lin_vcycle_dense(SolveCtx& S, int k) {
  mgfr_ctx* c = S.c;
  const mgfr_config& g = c->cfg;
  DenseHier& H = c->dh;
  DenseLevel& F = H.L[k];
  const unsigned char* mk = S.A->dact[k];
  const MT<float> m = mt<float>(S.m);
  if (F.N <= 4) {
    k_dlin_coarse<<<1, 64, 0, c->s>>>(F.uold32, F.r32, F.u32, F.e32, m, (float)F.ih2, 20, mk);
    c->launches += 1;
    return;
  }
  auto sweep = [&](int sweeps) {
    for (int s = 0; s < sweeps; ++s)
      for (int col = 0; col < 2; ++col) {
        const long long nl = S.A->dlist_n[k][col];
        if (nl == 0) continue;
        k_dlin_sweep_list<<<nblocks(nl, BS), BS, 0, c->s>>>(F.uold32, F.r32, F.u32, F.e32, F.lg,
                                                            S.A->dlist[k] + col * (F.n / 2), nl,
                                                            m, (float)F.ih2);
        c->launches += 1;
      }
  };
  sweep(sweeps_of(S, -1, g.n_pre));
  if (k + 1 <= S.kmax) {
    DenseLevel& C = H.L[k + 1];
    k_dlin_restrict<<<nblocks(C.n, BS), BS, 0, c->s>>>(F.uold32, F.r32, F.u32, F.e32, F.lg,
                                                       C.r32, C.u32, C.e32, C.uold32, m,
                                                       (float)F.ih2, mk);
    c->launches += 1;
    lin_vcycle_dense(S, k + 1);
    const CList cf = clist(S, k);
    if (cl_threads(cf, F.n) > 0)
      k_dlin_prolong<<<nblocks(cl_threads(cf, F.n), BS), BS, 0, c->s>>>(
          F.uold32, C.uold32, F.lg, g.prolong_linear, mk, cf);
    c->launches += 1;
  }
  sweep(sweeps_of(S, -1, g.n_post));
}

void lin_vcycle_tree(SolveCtx& S, int l) {
  mgfr_ctx* c = S.c;
  AmrWork* A = S.A;
  const mgfr_config& g = c->cfg;
  const MT<float> m = mt<float>(S.m);
  AmrLevel& F = A->L[l];
  const int npre = sweeps_of(S, l, g.n_pre), npost = sweeps_of(S, l, g.n_post);
  lin_relax(S, l, npre);
  S.lin_updates += (long long)npre * F.relaxed;
  const unsigned char* fmask = l == S.L ? nullptr : F.act;
  if (l >= 1 && has_coarse(S, l)) {
    AmrLevel& P = A->L[l - 1];
    const ORange R = orange(S, F, l);
    const long long pno = l - 1 >= 1 ? P.n_oct : 0;  // FP32 parent layout (0: dense)
    if (R.n > 0)
      k_olin_restrict32<<<nblocks(R.n, BS), BS, 0, c->s>>>(
          F.wold32, F.wf32, F.w32, F.nbr, F.ghost32, fmask, R.n, R.list, F.n_oct, F.pcell, pno,
          m, (float)F.ih2, P.wf32, P.w32, P.wold32);
    c->launches += 1;
    lin_vcycle_tree(S, l - 1);
    if (R.n > 0)
      k_oprolong32<true><<<nblocks(R.n, BS), BS, 0, c->s>>>(R.n, R.list, F.n_oct, F.pcell,
                                                           F.pnbr, pno, P.wold32, nullptr, fmask,
                                                           g.prolong_linear, F.wold32);
    c->launches += 1;
  } else if (l == 0 && S.kmax >= 1) {
    DenseHier& H = c->dh;
    DenseLevel& C = H.L[1];
    k_dlin_restrict<<<nblocks(C.n, BS), BS, 0, c->s>>>(F.wold32, F.wf32, F.w32, F.wE32, F.lgN,
                                                       C.r32, C.u32, C.e32, C.uold32, m,
                                                       (float)F.ih2, F.act);
    c->launches += 1;
    lin_vcycle_dense(S, 1);
    const CList c0 = clist(S, 0);
    if (cl_threads(c0, F.ncell) > 0)
      k_dlin_prolong<<<nblocks(cl_threads(c0, F.ncell), BS), BS, 0, c->s>>>(
          F.wold32, C.uold32, F.lgN, g.prolong_linear, F.act, c0);
    c->launches += 1;
  }
  lin_relax(S, l, npost);
  S.lin_updates += (long long)npost * F.relaxed;
}

// FP64 residual of level L with the linear system set up for phase B
mgfr_status lin_resid(SolveCtx& S, double* hs) {
  mgfr_ctx* c = S.c;
  AmrLevel& L = S.A->L[S.L];
  DenseHier& H = c->dh;
  const int nparts = (int)std::min<long long>(H.nparts / 2, nblocks(2 * L.n_oct, BS));
  if (c->capturing >= 0) prof_begin(c, 2, L.ncell);
  k_oresid_df<<<nparts, BS, 0, c->s>>>(
      reinterpret_cast<const dfl*>(L.w), reinterpret_cast<const dfl*>(L.wE),
      reinterpret_cast<const dfl*>(L.wf), L.nbr, reinterpret_cast<const dfl*>(L.ghost),
      reinterpret_cast<const dfl*>(L.ghostE), mdf(S.m, L.ih2), L.n_oct, L.wf32, L.w32,
      L.wold32, H.partials);
  if (c->capturing >= 0) prof_end(c);
  k_finish3<<<1, 256, 0, c->s>>>(H.partials, nparts, H.scal + 8);
  c->launches += 2;
  MG_CK(c, cudaMemcpyAsync(hs, H.scal + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  return MGFR_OK;
}

#define TRY(x)                    \
  do {                            \
    mgfr_status s_ = (x);         \
    if (s_ != MGFR_OK) return s_; \
  } while (0)

template <class T>
mgfr_status run_vcycle(SolveCtx& S, mgfr_stats* st, double* hs) {
  S.c->capturing = 3;
  vcycle_tree<T>(S, S.L);
  S.c->capturing = -1;
  TRY(level_norm<T>(S, hs));
  prof_collect(S.c, 3, st);
  return MGFR_OK;
}

}  // namespace

mgfr_status amr_solve_level(mgfr_ctx* c, AmrWork* A, int Lv, const Model& m, mgfr_stats* st) {
  const mgfr_config& g = c->cfg;
  DenseHier& H = c->dh;
  AmrLevel& F = A->L[Lv];
  const bool mixed = g.precision == MGFR_PREC_MIXED;
  const float mthr = (float)g.mask_thres;
  TreeView T = tree_view(A);
  const double* up = Lv - 1 == 0 ? H.L[0].u : A->L[Lv - 1].u;
  // the mixed form keeps the FP64 ghost slots as double-float pairs until the
  // level is finished
  bool gh_df = mixed, w_df = false;
  if (F.n_gslot > 0)
    k_ghosts<<<nblocks(4 * F.n_gslot, BS), BS, 0, c->s>>>(F.n_gslot, Lv, T, F.gface, up,
                                                          g.prolong_linear, F.ghost, F.ghostE,
                                                          F.ghost32, mixed ? 1 : 0);
  c->launches += 1;
  k_init_level<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.ncell, F.pcell, F.pnbr, up,
                                                      g.prolong_linear, F.w, F.wE,
                                                      mixed ? F.w32 : nullptr, F.n_oct);
  if (g.start == MGFR_START_PREVIOUS_ALL && Lv < A->prev_nlev && A->prev_N0 == A->N0 &&
      A->prev_box == A->box && A->prev_noct[Lv] > 0 && F.n_oct > 0) {
    k_warm_level<<<nblocks(F.n_oct, BS), BS, 0, c->s>>>(F.opos, F.n_oct, A->prev_key[Lv],
                                                         A->prev_noct[Lv], A->prev_u[Lv], F.w,
                                                         F.wE, mixed ? F.w32 : nullptr);
    c->launches += 1;
  }
  if (mixed) {
    k_d2df<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.f, reinterpret_cast<dfl*>(F.wf), F.ncell);
  } else {
    MG_CK(c, cudaMemcpyAsync(F.wf, F.f, sizeof(double) * (size_t)F.ncell,
                             cudaMemcpyDeviceToDevice, c->s));
  }
  k_fill_f<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.mask, F.ncell, 1.f);
  c->launches += 3;
  if (mixed) {
    k_d2f<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.f, F.wf32, F.ncell, F.n_oct);
    c->launches += 1;
  }
  F.relaxed = F.ncell;
  // FP64 work copies of the coarser levels: set up front in the FP64 form; in
  // the mixed form only the FP64 fallback V-cycles below need them
  auto fp64_coarse = [&]() -> mgfr_status {
    for (int l = Lv - 1; l >= 0; --l) {
      AmrLevel& P = A->L[l];
      const double* uu = l == 0 ? H.L[0].u : P.u;
      const double* EE = l == 0 ? H.L[0].E : P.E;
      const size_t b8 = sizeof(double) * (size_t)P.ncell;
      MG_CK(c, cudaMemcpyAsync(P.w, uu, b8, cudaMemcpyDeviceToDevice, c->s));
      MG_CK(c, cudaMemcpyAsync(P.wE, EE, b8, cudaMemcpyDeviceToDevice, c->s));
      MG_CK(c, cudaMemcpyAsync(P.wold, uu, b8, cudaMemcpyDeviceToDevice, c->s));
      P.wE_df = false;  // its e^u pairs are overwritten
    }
    return MGFR_OK;
  };
  if (!mixed) TRY(fp64_coarse());
  for (int l = Lv - 1; l >= 0; --l) {
    AmrLevel& P = A->L[l];
    const double* uu = l == 0 ? H.L[0].u : P.u;
    if (mixed) {
      const long long pno = l >= 1 ? P.n_oct : 0;  // FP32 layout (0: dense)
      k_d2f2<<<nblocks(P.ncell, BS), BS, 0, c->s>>>(uu, P.w32, P.wold32, P.ncell, pno);
      c->launches += 1;
    }
    MG_CK(c, cudaMemsetAsync(P.mask, 0, sizeof(float) * (size_t)P.ncell, c->s));
    AmrLevel& Ch = A->L[l + 1];
    k_mask_up<<<nblocks(Ch.n_oct, BS), BS, 0, c->s>>>(Ch.mask, Ch.n_oct, Ch.pcell, P.mask);
    c->launches += 1;
    TRY(count_relaxed(c, A, P.mask, P.ncell, mthr, &P.relaxed));
    k_act<<<nblocks(P.ncell, BS), BS, 0, c->s>>>(P.mask, P.ncell, mthr, P.act);
    c->launches += 1;
    if (l >= 1) TRY(build_oct_list(c, A, P, mthr));
  }
  for (int k = 1; k < H.nlev; ++k) {
    const float* mf = k == 1 ? A->L[0].mask : A->dmask[k - 1];
    k_mask_dense<<<nblocks(H.L[k].n, BS), BS, 0, c->s>>>(mf, H.L[k - 1].lg, A->dmask[k]);
    c->launches += 1;
  }
  // the dense levels below the base the cycles visit: each must relax at
  // least 1/kDenseMinDiv of its cells (and the base too, see has_coarse)
  int kmax = 0;
  if (A->L[0].relaxed * kDenseMinDiv >= A->L[0].ncell) {
    for (int k = 1; k < H.nlev; ++k) {
      long long nk = 0;
      TRY(count_relaxed(c, A, A->dmask[k], H.L[k].n, mthr, &nk));
      if (nk == 0 || nk * kDenseMinDiv < H.L[k].n) break;
      kmax = k;
      k_act<<<nblocks(H.L[k].n, BS), BS, 0, c->s>>>(A->dmask[k], H.L[k].n, mthr, A->dact[k]);
      c->launches += 1;
      if (H.L[k].N > 4) TRY(build_dense_lists(c, A, k, A->dact[k], H.L[k].lg));
    }
  }
  TRY(build_dense_lists(c, A, 0, A->L[0].act, A->L[0].lgN));
  SolveCtx S{c, A, m, Lv, mthr, 0, kmax};
  if (g.profile) prof_reserve_public(c, 64);
  double hs[3];
  // initial norms (the reference ||f|| and whether to iterate at all): FP32
  // arrays in the mixed form, whose FP64 residual decides convergence below
  if (mixed)
    TRY(level_norm<float>(S, hs));
  else
    TRY(level_norm<double>(S, hs));
  const double fn = std::sqrt(hs[2]), r0 = std::sqrt(hs[0]);
  const double ref = fn > 0.0 ? fn : r0;
  const double target = g.tol_rel * ref;
  double r = r0;
  int it = 0, it32 = 0;
  if (mixed && r > target) {
    // FP32 V-cycles until mixed_switch or a stall
    double prev = -1.0;
    while (it32 < g.max_vcycles) {
      TRY(run_vcycle<float>(S, st, hs));
      ++it32;
      const double r32 = std::sqrt(hs[0]);
      if (!std::isfinite(r32) || r32 <= g.mixed_switch * ref || (prev > 0.0 && r32 > 0.7 * prev))
        break;
      prev = r32;
    }
    k_f2df_exp<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.w32, F.n_oct, reinterpret_cast<dfl*>(F.w),
                                                      reinterpret_cast<dfl*>(F.wE), F.ncell);
    c->launches += 1;
    w_df = true;
    // phase B: FP64-accurate residual (double-float), FP32 linear masked
    // V-cycles on J(u) e = r, u += e
    for (int l = Lv - 1; l >= 0; --l) {
      AmrLevel& P = A->L[l];
      k_zero32<<<nblocks(P.ncell, BS), BS, 0, c->s>>>(P.wold32, P.ncell);
      c->launches += 1;
    }
    for (int k = 1; k < H.nlev; ++k) {
      k_zero32<<<nblocks(H.L[k].n, BS), BS, 0, c->s>>>(H.L[k].uold32, H.L[k].n);
      c->launches += 1;
    }
    c->capturing = 3;
    TRY(lin_resid(S, hs));
    c->capturing = -1;
    r = std::sqrt(hs[0]);
    double rprev = r;
    int inner = g.mixed_inner;
    while (r > target && it < g.max_vcycles) {
      c->capturing = 3;
      for (int q = 0; q < inner; ++q) lin_vcycle_tree(S, Lv);
      k_apply_df<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(reinterpret_cast<dfl*>(F.w),
                                                        reinterpret_cast<dfl*>(F.wE), F.wold32,
                                                        F.n_oct, F.ncell, (float)g.step_cap);
      c->launches += 1;
      TRY(lin_resid(S, hs));
      c->capturing = -1;
      prof_collect(c, 3, st);
      r = std::sqrt(hs[0]);
      ++it;
      if (!std::isfinite(r) || r > rprev) break;  // finish with FP64 V-cycles below
      // linear cycles of the next outer iteration: from the reduction per
      // cycle just measured, as many as bring r to half the target (at most
      // mixed_inner); a residual just above the target then costs one cycle
      const double rho = std::pow(r / rprev, 1.0 / inner);
      inner = g.mixed_inner;
      if (r > target && rho > 0.0 && rho < 1.0) {
        const double need = std::ceil(std::log(0.5 * target / r) / std::log(rho));
        inner = (int)std::max(1.0, std::min((double)g.mixed_inner, need));
      }
      rprev = r;
    }
  }
  if (mixed && !(r > target) && it32 == 0) {
    // converged at the start: the FP64 iterate is the FP32 initial guess
    k_f2d_exp<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.w32, F.n_oct, F.w, F.wE, F.ncell);
    c->launches += 1;
  }
  if (mixed && r > target) {
    // FP64 fallback: the iterate, source and ghosts back to FP64
    if (w_df) {
      k_df2d<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(reinterpret_cast<const dfl*>(F.w), F.w,
                                                    F.ncell);
      k_df2d<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(reinterpret_cast<const dfl*>(F.wE), F.wE,
                                                    F.ncell);
      c->launches += 2;
      w_df = false;
    }
    MG_CK(c, cudaMemcpyAsync(F.wf, F.f, sizeof(double) * (size_t)F.ncell,
                             cudaMemcpyDeviceToDevice, c->s));
    if (F.n_gslot > 0)
      k_ghosts<<<nblocks(4 * F.n_gslot, BS), BS, 0, c->s>>>(F.n_gslot, Lv, T, F.gface, up,
                                                            g.prolong_linear, F.ghost, F.ghostE,
                                                            F.ghost32, 0);
    c->launches += 1;
    gh_df = false;
    TRY(fp64_coarse());
  }
  while (r > target && it < g.max_vcycles) {
    TRY(run_vcycle<double>(S, st, hs));
    r = std::sqrt(hs[0]);
    ++it;
    if (!std::isfinite(r)) break;
  }
  if (w_df) {
    k_df2d<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(reinterpret_cast<const dfl*>(F.w), F.u,
                                                  F.ncell);
    k_df2d<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(reinterpret_cast<const dfl*>(F.wE), F.E,
                                                  F.ncell);
    c->launches += 2;
  } else {
    MG_CK(c, cudaMemcpyAsync(F.u, F.w, sizeof(double) * (size_t)F.ncell,
                             cudaMemcpyDeviceToDevice, c->s));
    MG_CK(c, cudaMemcpyAsync(F.E, F.wE, sizeof(double) * (size_t)F.ncell,
                             cudaMemcpyDeviceToDevice, c->s));
  }
  F.ghost_df = gh_df;  // the force kernel reads the ghosts in either form
  F.wE_df = w_df;      // e^u of the result still available as pairs in wE
  if (st) {
    st->level_iters[Lv] = it + it32;
    st->level_res[Lv] = r / ref;
    st->cell_updates += S.updates;
    st->linear_updates += S.lin_updates;
  }
  if (!(r <= target)) return set_err(c, MGFR_E_NOCONVERGE, "refined level did not converge");
  return MGFR_OK;
}
