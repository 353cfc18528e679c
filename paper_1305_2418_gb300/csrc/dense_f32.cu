// dense_f32.cu -- mixed-precision kernels for dense periodic levels.
//
// Phase A (FP32 nonlinear FAS): the same Newton-Gauss-Seidel update, FAS
// restriction/right-hand side/correction as the FP64 path (Puchwein, Baldi &
// Springel 2013, Sec. 3.3), in FP32, with e^u recomputed on the fly by the
// SFU instead of stored.  These are HBM-bound: a half-sweep streams u and f
// once and writes u once.
//
// Phase B (defect correction): r = f - L(u) in FP64 on the FP64 iterate, then
// the linearised system J(u) e = r (J the Jacobian of the discrete L) is
// relaxed by an FP32 linear multigrid V-cycle and u += e in FP64.  Solving
// the linearised correction in FP32 avoids the ~1e-7 cancellation floor of a
// nonlinear FP32 correction.
#include <algorithm>

#include "colour_split.cuh"
#include "dfloat.cuh"
#include "mgfr_internal.cuh"

namespace {

constexpr int BS = 256;

// linear index of (i, j, k) on an N = 2^lg grid (N <= 1024: fits 32 bits)
__device__ __forceinline__ unsigned cidx(int i, int j, int k, int lg) {
  return ((((unsigned)i << lg) + (unsigned)j) << lg) + (unsigned)k;
}

struct ModelF {
  float aRt, aRt_np1, inv_np1;
};

__host__ __device__ inline ModelF to_f(const Model& m) {
  return ModelF{(float)m.aRt, (float)m.aRt_np1, (float)m.inv_np1};
}

// The FP32 arrays of a dense level (u, f, u_old, e, r) are stored by colour
// (colour_split.cuh): a half-sweep reads one plane, reads and writes the
// other, each in whole coalesced rows.

// ---- Phase A: nonlinear FP32 Newton-Gauss-Seidel half-sweep ----------------
// Thread = one cell of the active colour (plane `colour`, index t in it).
__global__ void __launch_bounds__(BS) k_sweep32(float* __restrict__ u, const float* __restrict__ f,
                                                int lg, int colour, ModelF m, float ih2,
                                                float cap) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lg - 1))) return;
  const unsigned c = ((unsigned)colour << (3 * lg - 1)) + t;
  int i, j, k;
  pcell(c, lg, &i, &j, &k);
  unsigned q[6];
  pnb6(i, j, k, lg, q);
  float nb[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) nb[e] = u[q[e]];
  const float uc = u[c];
  const float Ec = __expf(uc);
  float sbd = 0.f, sd = 0.f, sb = 0.f;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float bb = 0.5f * (__expf(nb[e]) + Ec), du = nb[e] - uc;
    sbd = fmaf(bb, du, sbd);
    sd += du;
    sb += bb;
  }
  const float s = __expf(-uc * m.inv_np1);
  const float L = sbd * ih2 + m.aRt * (1.f - s);
  const float dL = (0.5f * Ec * sd - sb) * ih2 + m.aRt_np1 * s;
  float step = __fdividef(L - f[c], dL);
  step = fminf(fmaxf(step, -cap), cap);
  u[c] = uc - step;
}

__device__ __forceinline__ float Lpoint32(const float* __restrict__ u, int i, int j, int k, int lg,
                                          const ModelF& m, float ih2) {
  unsigned q[6];
  pnb6(i, j, k, lg, q);
  const float uc = u[pdx(i, j, k, lg)], Ec = __expf(uc);
  float sbd = 0.f;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float un = u[q[e]];
    sbd = fmaf(0.5f * (__expf(un) + Ec), un - uc, sbd);
  }
  return sbd * ih2 + m.aRt * (1.f - __expf(-uc * m.inv_np1));
}

__device__ __forceinline__ void block_partial(double ss, double mx, double* __restrict__ partials) {
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
    for (int w = 0; w < (int)blockDim.x / 32; ++w) {
      a += s1[w];
      b = fmax(b, s2[w]);
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// Restrict u and the FP32 residual (8-daughter average); the residual norm of
// the fine level is accumulated too (used on the finest level only).
__global__ void __launch_bounds__(BS) k_restrict32(const float* __restrict__ u,
                                                   const float* __restrict__ f, int lgf,
                                                   float* __restrict__ uc, float* __restrict__ ucold,
                                                   float* __restrict__ fc, ModelF m, float ih2) {
  const int lgc = lgf - 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lgc))) return;
  int I, J, K;
  pcell(t, lgc, &I, &J, &K);
  float su = 0.f, sr = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q >> 2), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q & 1);
    const unsigned c = pdx(i, j, k, lgf);
    su += u[c];
    sr += f[c] - Lpoint32(u, i, j, k, lgf, m, ih2);
  }
  uc[t] = 0.125f * su;
  ucold[t] = 0.125f * su;
  fc[t] = 0.125f * sr;
}

__global__ void __launch_bounds__(BS) k_fas_rhs32(const float* __restrict__ u, float* __restrict__ f,
                                                  int lg, ModelF m, float ih2) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lg))) return;
  int i, j, k;
  pcell(t, lg, &i, &j, &k);
  f[t] += Lpoint32(u, i, j, k, lg, m, ih2);
}

// fine += P(coarse - coarse_old) (linear or injection); `sub` selects whether
// coarse_old is subtracted (nonlinear FAS) or not (linear correction scheme).
__global__ void __launch_bounds__(BS) k_prolong32(float* __restrict__ u, const float* __restrict__ uc,
                                                  const float* __restrict__ ucold, int lgf,
                                                  int linear) {
  const int N = 1 << lgf, lgc = lgf - 1, Mc = (N >> 1) - 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lgf))) return;
  int i, j, k;
  pcell(t, lgf, &i, &j, &k);
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  auto corr = [&](int a, int b, int c) {
    const unsigned q = pdx(a & Mc, b & Mc, c & Mc, lgc);
    return ucold ? uc[q] - ucold[q] : uc[q];
  };
  float v = corr(I, J, K);
  if (linear) {
    const float sx = (i & 1) ? 0.125f : -0.125f, sy = (j & 1) ? 0.125f : -0.125f,
                sz = (k & 1) ? 0.125f : -0.125f;
    v += sx * (corr(I + 1, J, K) - corr(I - 1, J, K));
    v += sy * (corr(I, J + 1, K) - corr(I, J - 1, K));
    v += sz * (corr(I, J, K + 1) - corr(I, J, K - 1));
  }
  u[t] += v;
}

__global__ void __launch_bounds__(64) k_coarse32(float* __restrict__ ug, const float* __restrict__ fg,
                                                 ModelF m, float ih2, float cap, int sweeps) {
  __shared__ float u[64];  // C order in shared memory
  const int t = threadIdx.x;
  const int i = t >> 4, j = (t >> 2) & 3, k = t & 3, colour = (i + j + k) & 1;
  const unsigned g = pdx(i, j, k, 2);
  u[t] = ug[g];
  const float fc = fg[g];
  const int nb[6] = {(((i + 3) & 3) << 4) | (j << 2) | k, (((i + 1) & 3) << 4) | (j << 2) | k,
                     (i << 4) | (((j + 3) & 3) << 2) | k, (i << 4) | (((j + 1) & 3) << 2) | k,
                     (i << 4) | (j << 2) | ((k + 3) & 3), (i << 4) | (j << 2) | ((k + 1) & 3)};
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      if (colour == c) {
        const float uc = u[t], Ec = __expf(uc);
        float sbd = 0.f, sd = 0.f, sb = 0.f;
        for (int q = 0; q < 6; ++q) {
          const float un = u[nb[q]], b = 0.5f * (__expf(un) + Ec), du = un - uc;
          sbd = fmaf(b, du, sbd);
          sd += du;
          sb += b;
        }
        const float sN = __expf(-uc * m.inv_np1);
        const float L = sbd * ih2 + m.aRt * (1.f - sN);
        const float dL = (0.5f * Ec * sd - sb) * ih2 + m.aRt_np1 * sN;
        float step = (L - fc) / dL;
        step = fminf(fmaxf(step, -cap), cap);
        u[t] = uc - step;
      }
      __syncthreads();
    }
  ug[g] = u[t];
}

// FP32 residual norm on the finest level (phase A stopping test).
__global__ void __launch_bounds__(BS) k_norm32(const float* __restrict__ u, const float* __restrict__ f,
                                               int lg, long long n, ModelF m, float ih2,
                                               double* __restrict__ partials) {
  double ss = 0.0, mx = 0.0;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += gridDim.x * blockDim.x) {
    int i, j, k;
    pcell(t, lg, &i, &j, &k);
    const double r = (double)(f[t] - Lpoint32(u, i, j, k, lg, m, ih2));
    ss = fma(r, r, ss);
    mx = fmax(mx, fabs(r));
  }
  block_partial(ss, mx, partials);
}

// C-order FP64 -> colour-split FP32
__global__ void k_from64(const double* __restrict__ x, float* __restrict__ y, int lg) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lg))) return;
  const int M = (1 << lg) - 1;
  y[pdx((int)(t >> (2 * lg)), (int)((t >> lg) & M), (int)(t & M), lg)] = f_from_double_bits(x[t]);
}

// FP32 iterate -> double-float iterate and its e^u (start of phase B)
__global__ void k_to_df(const float* __restrict__ u32, dfl* __restrict__ u, dfl* __restrict__ E,
                        int lg) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lg))) return;
  const int M = (1 << lg) - 1;
  const dfl v{u32[pdx((int)(t >> (2 * lg)), (int)((t >> lg) & M), (int)(t & M), lg)], 0.f};
  u[t] = v;
  E[t] = df_exp(v);
}

// ---- Phase B ---------------------------------------------------------------
// Model constants as double-float pairs (phase B in double-float)
struct DFM {
  dfl aRt, inv_np1, ih2h;  // alpha Rt, 1/(n+1), 1/(2 h^2)
  int n;
};

// r = f - L(u) to FP64 accuracy in double-float on the FP32 pipes (u, E, f
// held as hi + lo pairs); stores r and u rounded to FP32, zeroes the
// correction e, and accumulates the norms (FP32 within a thread).
__global__ void __launch_bounds__(BS) k_resid_df(const dfl* __restrict__ u,
                                                 const dfl* __restrict__ E,
                                                 const dfl* __restrict__ f, int lg, DFM m,
                                                 float* __restrict__ r32,
                                                 float* __restrict__ u32, float* __restrict__ e32,
                                                 double* __restrict__ partials) {
  const int M = (1 << lg) - 1;
  const unsigned n = 1u << (3 * lg);
  float ss = 0.f, mx = 0.f;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += gridDim.x * blockDim.x) {
    const int k = (int)(t & M), j = (int)((t >> lg) & M), i = (int)(t >> (2 * lg));
    const unsigned nb[6] = {cidx((i - 1) & M, j, k, lg), cidx((i + 1) & M, j, k, lg),
                             cidx(i, (j - 1) & M, k, lg), cidx(i, (j + 1) & M, k, lg),
                             cidx(i, j, (k - 1) & M, lg), cidx(i, j, (k + 1) & M, lg)};
    const dfl uc = u[t], Ec = E[t];
    dfl acc = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 6; ++q)
      acc = df_add_abs(acc, df_mul(df_add_abs(E[nb[q]], Ec), df_add_abs(u[nb[q]], df_neg(uc))));
    const dfl sN = m.n == 1 ? df_rsqrt(Ec) : df_exp(df_neg(df_mul(uc, m.inv_np1)));
    const dfl L = df_add(df_mul(acc, m.ih2h), df_mul(m.aRt, df_add_f(df_neg(sN), 1.f)));
    const dfl r = df_sub(f[t], L);
    const unsigned p = pdx(i, j, k, lg);
    r32[p] = r.hi;
    u32[p] = uc.hi;
    e32[p] = 0.f;
    ss = fmaf(r.hi, r.hi, ss);
    mx = fmaxf(mx, fabsf(r.hi));
  }
  block_partial((double)ss, (double)mx, partials);
}

// Jacobian of L at u (neighbours j of cell i):
//   dL_i/du_j = (E_j (u_j - u_i) + E_i + E_j) / (2 h^2),
//   dL_i/du_i = sum_j (E_i (u_j - u_i) - E_i - E_j) / (2 h^2)
//               + alpha Rt/(n+1) e^{-u_i/(n+1)}.
struct Jrow {
  float off[6], diag;
};

__device__ __forceinline__ Jrow jac_row(float uc, const float* nb, const ModelF& m, float ih2) {
  Jrow J;
  const float Ec = __expf(uc);
  float d = 0.f;
  const float h2 = 0.5f * ih2;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float En = __expf(nb[q]), du = nb[q] - uc;
    J.off[q] = h2 * fmaf(En, du, Ec + En);
    d += fmaf(Ec, du, -Ec - En);
  }
  J.diag = d * h2 + m.aRt_np1 * __expf(-uc * m.inv_np1);
  return J;
}

__device__ __forceinline__ void nb6(const float* __restrict__ x, const unsigned* q, float* out) {
#pragma unroll
  for (int e = 0; e < 6; ++e) out[e] = x[q[e]];
}

// Gauss-Seidel half-sweep on J e = r: e_i = (r_i - sum_j J_ij e_j) / J_ii.
__global__ void __launch_bounds__(BS) k_lin_sweep(float* __restrict__ e, const float* __restrict__ r,
                                                  const float* __restrict__ u, int lg, int colour,
                                                  ModelF m, float ih2) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lg - 1))) return;
  const unsigned c = ((unsigned)colour << (3 * lg - 1)) + t;
  int i, j, k;
  pcell(c, lg, &i, &j, &k);
  unsigned q[6];
  pnb6(i, j, k, lg, q);
  float un[6], en[6];
  nb6(u, q, un);
  nb6(e, q, en);
  const Jrow J = jac_row(u[c], un, m, ih2);
  float s = r[c];
#pragma unroll
  for (int q = 0; q < 6; ++q) s = fmaf(-J.off[q], en[q], s);
  e[c] = __fdividef(s, J.diag);
}

// Coarse linear problem: r_c = R(r - J e), u_c = R(u), e_c = 0.
__global__ void __launch_bounds__(BS) k_lin_restrict(const float* __restrict__ e,
                                                     const float* __restrict__ r,
                                                     const float* __restrict__ u, int lgf,
                                                     float* __restrict__ ec, float* __restrict__ rc,
                                                     float* __restrict__ uc, ModelF m, float ih2) {
  const int lgc = lgf - 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lgc))) return;
  int I, J, K;
  pcell(t, lgc, &I, &J, &K);
  float su = 0.f, sr = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q >> 2), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q & 1);
    const unsigned c = pdx(i, j, k, lgf);
    unsigned nq[6];
    pnb6(i, j, k, lgf, nq);
    float un[6], en[6];
    nb6(u, nq, un);
    nb6(e, nq, en);
    const Jrow Jr = jac_row(u[c], un, m, ih2);
    float Je = Jr.diag * e[c];
    for (int p = 0; p < 6; ++p) Je = fmaf(Jr.off[p], en[p], Je);
    sr += r[c] - Je;
    su += u[c];
  }
  uc[t] = 0.125f * su;
  rc[t] = 0.125f * sr;
  ec[t] = 0.f;
}

__global__ void __launch_bounds__(64) k_lin_coarse(float* __restrict__ eg, const float* __restrict__ rg,
                                                   const float* __restrict__ ug, ModelF m, float ih2,
                                                   int sweeps) {
  __shared__ float e[64];  // C order in shared memory
  const int t = threadIdx.x;
  const int i = t >> 4, j = (t >> 2) & 3, k = t & 3, colour = (i + j + k) & 1;
  const int nb[6] = {(((i + 3) & 3) << 4) | (j << 2) | k, (((i + 1) & 3) << 4) | (j << 2) | k,
                     (i << 4) | (((j + 3) & 3) << 2) | k, (i << 4) | (((j + 1) & 3) << 2) | k,
                     (i << 4) | (j << 2) | ((k + 3) & 3), (i << 4) | (j << 2) | ((k + 1) & 3)};
  unsigned gq[6];
  pnb6(i, j, k, 2, gq);
  float un[6];
  for (int q = 0; q < 6; ++q) un[q] = ug[gq[q]];
  const unsigned g = pdx(i, j, k, 2);
  const Jrow J = jac_row(ug[g], un, m, ih2);
  const float rc = rg[g];
  e[t] = eg[g];
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      if (colour == c) {
        float acc = rc;
        for (int q = 0; q < 6; ++q) acc = fmaf(-J.off[q], e[nb[q]], acc);
        e[t] = acc / J.diag;
      }
      __syncthreads();
    }
  eg[g] = e[t];
}

__global__ void k_apply_corr(dfl* __restrict__ u, dfl* __restrict__ E, const float* __restrict__ e,
                             int lg, float cap) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (1u << (3 * lg))) return;
  const int M = (1 << lg) - 1;
  const float et = e[pdx((int)(t >> (2 * lg)), (int)((t >> lg) & M), (int)(t & M), lg)];
  const dfl v = df_add_f(u[t], fminf(fmaxf(et, -cap), cap));
  u[t] = v;
  E[t] = df_exp(v);
}

__global__ void k_d2df(const double* __restrict__ x, dfl* __restrict__ y, long long n) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const double v = x[t];
    y[t] = df_from_double_bits(v);
  }
}
__global__ void k_df2d(const dfl* __restrict__ x, double* __restrict__ y, long long n) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const dfl v = x[t];
    y[t] = df_to_double_bits(v);
  }
}

// an FP64 iterate (in place) -> double-float pairs, and e^u as pairs
__global__ void k_d2df_exp(dfl* __restrict__ u, dfl* __restrict__ E, long long n) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const dfl v = df_from_double_bits(reinterpret_cast<const double*>(u)[t]);
    u[t] = v;
    E[t] = df_exp(v);
  }
}

__global__ void k_zero(float* __restrict__ x, long long n) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = 0.f;
}

__global__ void k_finish32(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
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

}  // namespace

namespace f32 {

void from64(const double* x, float* y, const DenseLevel& L, cudaStream_t s) {
  k_from64<<<nblocks(L.n, BS), BS, 0, s>>>(x, y, L.lg);
}
void to_df(DenseLevel& L, cudaStream_t s) {
  k_to_df<<<nblocks(L.n, BS), BS, 0, s>>>(L.u32, reinterpret_cast<dfl*>(L.u),
                                          reinterpret_cast<dfl*>(L.E), L.lg);
}
void f_to_df(const double* f, double* fdf, long long n, cudaStream_t s) {
  k_d2df<<<nblocks(n, BS), BS, 0, s>>>(f, reinterpret_cast<dfl*>(fdf), n);
}
void fp64_to_df(DenseLevel& L, cudaStream_t s) {
  k_d2df_exp<<<nblocks(L.n, BS), BS, 0, s>>>(reinterpret_cast<dfl*>(L.u), reinterpret_cast<dfl*>(L.E),
                                             L.n);
}
void state_to_fp64(DenseLevel& L, cudaStream_t s) {
  k_df2d<<<nblocks(L.n, BS), BS, 0, s>>>(reinterpret_cast<const dfl*>(L.u), L.u, L.n);
  k_df2d<<<nblocks(L.n, BS), BS, 0, s>>>(reinterpret_cast<const dfl*>(L.E), L.E, L.n);
}

void sweep(DenseLevel& L, const Model& m, int colour, float cap, cudaStream_t s) {
  k_sweep32<<<nblocks(L.n / 2, BS), BS, 0, s>>>(L.u32, L.f32, L.lg, colour, to_f(m), (float)L.ih2,
                                                cap);
}
void restrict_resid(DenseLevel& F, DenseLevel& C, const Model& m, double*, int, cudaStream_t s) {
  k_restrict32<<<nblocks(C.n, BS), BS, 0, s>>>(F.u32, F.f32, F.lg, C.u32, C.uold32, C.f32, to_f(m),
                                                (float)F.ih2);
}
void fas_rhs(DenseLevel& C, const Model& m, cudaStream_t s) {
  k_fas_rhs32<<<nblocks(C.n, BS), BS, 0, s>>>(C.u32, C.f32, C.lg, to_f(m), (float)C.ih2);
}
void prolong_corr(DenseLevel& F, DenseLevel& C, int linear, cudaStream_t s) {
  k_prolong32<<<nblocks(F.n, BS), BS, 0, s>>>(F.u32, C.u32, C.uold32, F.lg, linear);
}
void coarse_solve(DenseLevel& C, const Model& m, float cap, int sweeps, cudaStream_t s) {
  k_coarse32<<<1, 64, 0, s>>>(C.u32, C.f32, to_f(m), (float)C.ih2, cap, sweeps);
}
void norm32(DenseLevel& L, const Model& m, double* partials, int nparts, double* out,
            cudaStream_t s) {
  int nb = (int)std::min<long long>(nparts, nblocks(L.n, BS));
  k_norm32<<<nb, BS, 0, s>>>(L.u32, L.f32, L.lg, L.n, to_f(m), (float)L.ih2, partials);
  k_finish32<<<1, 256, 0, s>>>(partials, nb, out);
}
void resid_df(DenseLevel& L, const double* fdf, const Model& m, double* partials, int nparts,
              double* out, cudaStream_t s) {
  int nb = (int)std::min<long long>(nparts, nblocks(L.n, BS));
  const DFM dm{df_from_double(m.aRt), df_from_double(m.inv_np1), df_from_double(0.5 * L.ih2),
               m.n};
  k_resid_df<<<nb, BS, 0, s>>>(reinterpret_cast<const dfl*>(L.u), reinterpret_cast<const dfl*>(L.E),
                               reinterpret_cast<const dfl*>(fdf), L.lg, dm, L.r32, L.u32, L.e32,
                               partials);
  k_finish32<<<1, 256, 0, s>>>(partials, nb, out);
}
void lin_sweep(DenseLevel& L, const Model& m, int colour, cudaStream_t s) {
  k_lin_sweep<<<nblocks(L.n / 2, BS), BS, 0, s>>>(L.e32, L.r32, L.u32, L.lg, colour, to_f(m),
                                                  (float)L.ih2);
}
void lin_restrict(DenseLevel& F, DenseLevel& C, const Model& m, cudaStream_t s) {
  k_lin_restrict<<<nblocks(C.n, BS), BS, 0, s>>>(F.e32, F.r32, F.u32, F.lg, C.e32, C.r32, C.u32,
                                                 to_f(m), (float)F.ih2);
}
void lin_prolong(DenseLevel& F, DenseLevel& C, int linear, cudaStream_t s) {
  k_prolong32<<<nblocks(F.n, BS), BS, 0, s>>>(F.e32, C.e32, nullptr, F.lg, linear);
}
void lin_coarse(DenseLevel& C, const Model& m, int sweeps, cudaStream_t s) {
  k_lin_coarse<<<1, 64, 0, s>>>(C.e32, C.r32, C.u32, to_f(m), (float)C.ih2, sweeps);
}
void zero(float* x, long long n, cudaStream_t s) { k_zero<<<nblocks(n, BS), BS, 0, s>>>(x, n); }
void apply_corr(DenseLevel& L, double cap, cudaStream_t s) {
  k_apply_corr<<<nblocks(L.n, BS), BS, 0, s>>>(reinterpret_cast<dfl*>(L.u),
                                               reinterpret_cast<dfl*>(L.E), L.e32, L.lg, (float)cap);
}

}  // namespace f32
