// pm.cu -- gravitational potential of the last particle solve on a periodic
// particle-mesh grid (Puchwein, Baldi & Springel 2013, Sec. 2.4, Eq. (30)):
//   lap_x phi = 4 pi G a^2 rho_bar (delta_pm - mean) = (3/2) Om H0^2 a^-1 (delta_pm - mean)
// with delta_pm the matter and/or effective-mass contrast assigned to the PM
// grid by volume overlap (amr.cu), x comoving in Mpc/h, H0 = 100 km/s per
// Mpc/h, phi in (km/s)^2.
//
// The 7-point periodic Poisson problem is solved by linear multigrid in
// FP64: red-black Gauss-Seidel smoothing, the residual restricted by the
// 8-daughter average, the coarse correction prolonged by the same linear
// reconstruction as the field solve (parent plus its central-difference
// slopes at the daughter offsets), down to 4^3, where Gauss-Seidel sweeps
// run in one block.  The periodic operator is singular: the right-hand side
// has its mean removed, every coarse right-hand side is the average of a
// zero-sum residual, and phi is returned with zero mean.  The kernels stream
// phi and rhs once per half-sweep (HBM-bound, one thread per updated cell).
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "amr.cuh"

namespace {

constexpr int BS = 256;
constexpr int PM_MAXL = 10;
constexpr double kPoissonScale = 1.5e4;  // (3/2) H0^2 with H0 = 100 km/s per Mpc/h

__device__ __forceinline__ unsigned pidx(unsigned i, unsigned j, unsigned k, int lg) {
  return (((i << lg) + j) << lg) + k;
}

// One red (colour 0: i+j+k even) or black half-sweep of Gauss-Seidel on
// (sum of the 6 neighbours - 6 phi) / h^2 = rhs.
__global__ void __launch_bounds__(BS) k_pm_sweep(double* __restrict__ phi,
                                                 const double* __restrict__ rhs, int lg,
                                                 int colour, double h2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int N = 1 << lg, M = N - 1;
  if (t >= (1LL << (3 * lg - 1))) return;
  const int k2 = (int)(t & ((N >> 1) - 1));
  const long long r = t >> (lg - 1);
  const int j = (int)(r & M), i = (int)(r >> lg);
  const int k = 2 * k2 + ((i + j + colour) & 1);
  const double s = phi[pidx((i - 1) & M, j, k, lg)] + phi[pidx((i + 1) & M, j, k, lg)] +
                   phi[pidx(i, (j - 1) & M, k, lg)] + phi[pidx(i, (j + 1) & M, k, lg)] +
                   phi[pidx(i, j, (k - 1) & M, lg)] + phi[pidx(i, j, (k + 1) & M, lg)];
  phi[pidx(i, j, k, lg)] = (s - h2 * rhs[pidx(i, j, k, lg)]) * (1.0 / 6.0);
}

__device__ __forceinline__ double pm_resid(const double* __restrict__ phi,
                                           const double* __restrict__ rhs, int i, int j, int k,
                                           int lg, double ih2) {
  const int M = (1 << lg) - 1;
  const double c = phi[pidx(i, j, k, lg)];
  const double s = phi[pidx((i - 1) & M, j, k, lg)] + phi[pidx((i + 1) & M, j, k, lg)] +
                   phi[pidx(i, (j - 1) & M, k, lg)] + phi[pidx(i, (j + 1) & M, k, lg)] +
                   phi[pidx(i, j, (k - 1) & M, lg)] + phi[pidx(i, j, (k + 1) & M, lg)];
  return rhs[pidx(i, j, k, lg)] - (s - 6.0 * c) * ih2;
}

// residual rhs - lap phi of every cell (for the stopping test)
__global__ void __launch_bounds__(BS) k_pm_resid(const double* __restrict__ phi,
                                                 const double* __restrict__ rhs, int lg,
                                                 double ih2, double* __restrict__ res) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (1LL << (3 * lg))) return;
  const int M = (1 << lg) - 1;
  const int k = (int)(t & M), j = (int)((t >> lg) & M), i = (int)(t >> (2 * lg));
  res[t] = pm_resid(phi, rhs, i, j, k, lg, ih2);
}

// coarse right-hand side: the 8-daughter average of the fine residual; the
// coarse correction starts from zero
__global__ void __launch_bounds__(BS) k_pm_restrict(const double* __restrict__ phi,
                                                    const double* __restrict__ rhs, int lgf,
                                                    double ih2, double* __restrict__ rhs_c,
                                                    double* __restrict__ phi_c) {
  const int lgc = lgf - 1, Nc = 1 << lgc;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (1LL << (3 * lgc))) return;
  const int K = (int)(t & (Nc - 1)), J = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    s += pm_resid(phi, rhs, 2 * I + (q >> 2), 2 * J + ((q >> 1) & 1), 2 * K + (q & 1), lgf, ih2);
  rhs_c[t] = 0.125 * s;
  phi_c[t] = 0.0;
}

// phi_f += P(phi_c): the parent's value plus its central-difference slopes at
// the daughter's quarter-cell offset, one thread per fine cell
__global__ void __launch_bounds__(BS) k_pm_prolong(double* __restrict__ phi_f,
                                                   const double* __restrict__ phi_c, int lgf) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (1LL << (3 * lgf))) return;
  const int Mf = (1 << lgf) - 1, lgc = lgf - 1, Mc = (1 << lgc) - 1;
  const int k = (int)(t & Mf), j = (int)((t >> lgf) & Mf), i = (int)(t >> (2 * lgf));
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const double sx = (i & 1) ? 1.0 : -1.0, sy = (j & 1) ? 1.0 : -1.0, sz = (k & 1) ? 1.0 : -1.0;
  double v = phi_c[pidx(I, J, K, lgc)];
  v += sx * (phi_c[pidx((I + 1) & Mc, J, K, lgc)] - phi_c[pidx((I - 1) & Mc, J, K, lgc)]) * 0.125;
  v += sy * (phi_c[pidx(I, (J + 1) & Mc, K, lgc)] - phi_c[pidx(I, (J - 1) & Mc, K, lgc)]) * 0.125;
  v += sz * (phi_c[pidx(I, J, (K + 1) & Mc, lgc)] - phi_c[pidx(I, J, (K - 1) & Mc, lgc)]) * 0.125;
  phi_f[t] += v;
}

// the 4^3 grid: Gauss-Seidel sweeps in one block of 32 threads (one colour
// of the 64 cells per pass)
__global__ void k_pm_coarse(double* __restrict__ phi, const double* __restrict__ rhs, double h2,
                            int sweeps) {
  const int t = threadIdx.x;  // 0..31
  for (int s = 0; s < sweeps; ++s)
    for (int col = 0; col < 2; ++col) {
      const int k2 = t & 1, j = (t >> 1) & 3, i = t >> 3;
      const int k = 2 * k2 + ((i + j + col) & 1);
      const double sum = phi[pidx((i + 3) & 3, j, k, 2)] + phi[pidx((i + 1) & 3, j, k, 2)] +
                         phi[pidx(i, (j + 3) & 3, k, 2)] + phi[pidx(i, (j + 1) & 3, k, 2)] +
                         phi[pidx(i, j, (k + 3) & 3, 2)] + phi[pidx(i, j, (k + 1) & 3, 2)];
      const double v = (sum - h2 * rhs[pidx(i, j, k, 2)]) * (1.0 / 6.0);
      __syncthreads();
      phi[pidx(i, j, k, 2)] = v;
      __syncthreads();
    }
}

// per-block sums of x and of x^2 (deterministic: a fixed tree per block,
// the blocks summed on the host in order)
__global__ void __launch_bounds__(BS) k_pm_sums(const double* __restrict__ x, long long n,
                                                double* __restrict__ part) {
  __shared__ double s1[BS], s2[BS];
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)BS + threadIdx.x; i < n; i += (long long)gridDim.x * BS) {
    const double v = x[i];
    a += v;
    b += v * v;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = BS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1[0];
    part[2 * blockIdx.x + 1] = s2[0];
  }
}

// y = scale * (x - shift)
__global__ void k_pm_affine(const double* __restrict__ x, long long n, double scale, double shift,
                            double* __restrict__ y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = scale * (x[i] - shift);
}

// g = -grad phi by central differences (periodic), component-major [3][n]
__global__ void __launch_bounds__(BS) k_pm_grad(const double* __restrict__ phi, int lg, double inv2h,
                                                double* __restrict__ g) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = 1LL << (3 * lg);
  if (t >= n) return;
  const int M = (1 << lg) - 1;
  const int k = (int)(t & M), j = (int)((t >> lg) & M), i = (int)(t >> (2 * lg));
  g[t] = -(phi[pidx((i + 1) & M, j, k, lg)] - phi[pidx((i - 1) & M, j, k, lg)]) * inv2h;
  g[n + t] = -(phi[pidx(i, (j + 1) & M, k, lg)] - phi[pidx(i, (j - 1) & M, k, lg)]) * inv2h;
  g[2 * n + t] = -(phi[pidx(i, j, (k + 1) & M, lg)] - phi[pidx(i, j, (k - 1) & M, lg)]) * inv2h;
}

// cloud-in-cell interpolation of g [3][N^3] (values at cell centres) to the
// particles: position t = x N / box in cell units (wrapped), the 8 cells
// around t - 1/2 with the product of the 1D linear weights
__global__ void __launch_bounds__(BS) k_pm_cic(const double* __restrict__ pos, long long np, int lg,
                                               double inv_h, const double* __restrict__ g,
                                               double* __restrict__ acc) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int N = 1 << lg, M = N - 1;
  const long long n = 1LL << (3 * lg);
  int i0[3];
  double w1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double t = pos[3 * p + a] * inv_h - 0.5;
    const double fl = floor(t);
    w1[a] = t - fl;
    i0[a] = (int)((long long)fl & M);
  }
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int a = q >> 2, b = (q >> 1) & 1, c = q & 1;
    const double w = (a ? w1[0] : 1.0 - w1[0]) * (b ? w1[1] : 1.0 - w1[1]) * (c ? w1[2] : 1.0 - w1[2]);
    const unsigned id = pidx((i0[0] + a) & M, (i0[1] + b) & M, (i0[2] + c) & M, lg);
    s0 = fma(w, g[id], s0);
    s1 = fma(w, g[n + id], s1);
    s2 = fma(w, g[2 * n + id], s2);
  }
  acc[3 * p] = s0;
  acc[3 * p + 1] = s1;
  acc[3 * p + 2] = s2;
}

// leapfrog: v += kick acc, x = wrap(x + drift v); each operation rounded on
// its own (no fused multiply-add), so the step is reproducible elsewhere
__global__ void __launch_bounds__(BS) k_kick_drift(double* __restrict__ pos, double* __restrict__ vel,
                                                   const double* __restrict__ acc, long long n3,
                                                   double kick, double drift, double box) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const double v = __dadd_rn(vel[i], __dmul_rn(kick, acc[i]));
  vel[i] = v;
  double x = __dadd_rn(pos[i], __dmul_rn(drift, v));
  x = __dsub_rn(x, __dmul_rn(box, floor(__ddiv_rn(x, box))));
  if (!(x < box)) x = 0.0;  // rounding at the upper edge
  pos[i] = x;
}

struct PmLevel {
  int lg = 0;
  long long n = 0;
  double h2 = 0.0, ih2 = 0.0;
  double *phi = nullptr, *rhs = nullptr;
};

struct PmWork {
  int lg = 0, nlev = 0;
  PmLevel L[PM_MAXL];
  double* res = nullptr;      // residual of the finest level
  double* grad = nullptr;     // -grad phi [3][n] of the finest level (force)
  double* part = nullptr;     // block sums (device)
  double* part_h = nullptr;   // block sums (page-locked host)
  int nparts = 0;
};

void pm_free_work(PmWork* P) {
  for (auto& L : P->L) {
    if (L.phi) cudaFree(L.phi);
    if (L.rhs) cudaFree(L.rhs);
    L = PmLevel();
  }
  if (P->res) cudaFree(P->res);
  if (P->grad) cudaFree(P->grad);
  if (P->part) cudaFree(P->part);
  if (P->part_h) cudaFreeHost(P->part_h);
  P->res = P->part = P->part_h = P->grad = nullptr;
  P->lg = P->nlev = 0;
}

mgfr_status pm_alloc(mgfr_ctx* c, PmWork* P, int lg, double box) {
  if (P->lg != lg) {
    pm_free_work(P);
    P->lg = lg;
    P->nlev = lg - 1;  // N ... 4
    for (int l = 0; l < P->nlev; ++l) {
      PmLevel& L = P->L[l];
      L.lg = lg - l;
      L.n = 1LL << (3 * L.lg);
      MG_CK(c, cudaMalloc(&L.phi, sizeof(double) * (size_t)L.n));
      MG_CK(c, cudaMalloc(&L.rhs, sizeof(double) * (size_t)L.n));
    }
    MG_CK(c, cudaMalloc(&P->res, sizeof(double) * (size_t)P->L[0].n));
    P->nparts = 152 * 8;
    MG_CK(c, cudaMalloc(&P->part, sizeof(double) * 2 * P->nparts));
    MG_CK(c, cudaMallocHost(&P->part_h, sizeof(double) * 2 * P->nparts));
  }
  for (int l = 0; l < P->nlev; ++l) {
    const double h = box / (double)(1LL << P->L[l].lg);
    P->L[l].h2 = h * h;
    P->L[l].ih2 = 1.0 / (h * h);
  }
  return MGFR_OK;
}

// (sum x, sum x^2) of n values, summed in a fixed order
mgfr_status pm_sums(mgfr_ctx* c, PmWork* P, const double* x, long long n, double* sum,
                    double* sumsq) {
  const int nb = (int)std::min<long long>(P->nparts, (n + BS - 1) / BS);
  k_pm_sums<<<nb, BS, 0, c->s>>>(x, n, P->part);
  c->launches += 1;
  MG_CK(c, cudaMemcpyAsync(P->part_h, P->part, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nb; ++q) {
    a += P->part_h[2 * q];
    b += P->part_h[2 * q + 1];
  }
  *sum = a;
  *sumsq = b;
  return MGFR_OK;
}

void pm_vcycle(mgfr_ctx* c, PmWork* P, int l, long long& updates) {
  const mgfr_config& g = c->cfg;
  PmLevel& F = P->L[l];
  auto sweep = [&](int k) {
    for (int q = 0; q < k; ++q) {
      for (int col = 0; col < 2; ++col)
        k_pm_sweep<<<nblocks(F.n / 2, BS), BS, 0, c->s>>>(F.phi, F.rhs, F.lg, col, F.h2);
      c->launches += 2;
      updates += F.n;
    }
  };
  sweep(g.n_pre);
  PmLevel& C = P->L[l + 1];
  k_pm_restrict<<<nblocks(C.n, BS), BS, 0, c->s>>>(F.phi, F.rhs, F.lg, F.ih2, C.rhs, C.phi);
  c->launches += 1;
  if (C.lg > 2) {
    pm_vcycle(c, P, l + 1, updates);
  } else {
    k_pm_coarse<<<1, 32, 0, c->s>>>(C.phi, C.rhs, C.h2, 60);
    c->launches += 1;
    updates += 60 * C.n;
  }
  k_pm_prolong<<<nblocks(F.n, BS), BS, 0, c->s>>>(F.phi, C.phi, F.lg);
  c->launches += 1;
  sweep(g.n_post);
}

}  // namespace

void pm_free(mgfr_ctx* c) {
  PmWork* P = (PmWork*)c->pm;
  if (!P) return;
  pm_free_work(P);
  delete P;
  c->pm = nullptr;
}

// The potential of Eq. (30) on the PM grid of level lpm, left (zero mean) in
// the workspace's finest phi; phi_out (nullable) receives a copy.  Runs after
// the caller's stream, on the context's stream; synchronises.
static mgfr_status pm_solve(mgfr_ctx* c, int lpm, int what, double* phi_out_dev,
                            double* dens_out_dev, mgfr_stats* st, PmWork** work) {
  int lg = 0;
  double om = 0.3, a = 1.0;
  mgfr_status rs = amr_density_pm(c, lpm, what, nullptr, &lg, &om, &a);
  if (rs != MGFR_OK) return rs;
  if (lg < 3) return set_err(c, MGFR_E_INVALID, "the PM grid needs at least 8 cells per axis");
  auto w0 = std::chrono::steady_clock::now();
  MG_CK(c, cudaSetDevice(c->device));
  if (st) std::memset(st, 0, sizeof(*st));
  c->launches = 0;
  if (!c->pm) c->pm = new PmWork();
  PmWork* P = (PmWork*)c->pm;
  const double box = ((AmrWork*)c->amr)->box;
  if ((rs = pm_alloc(c, P, lg, box)) != MGFR_OK) return rs;
  PmLevel& L0 = P->L[0];
  MG_CK(c, cudaEventRecord(c->ev_in, c->user));
  MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_in, 0));
  MG_CK(c, cudaEventRecord(c->t0, c->s));
  // density contrast on the PM grid, then rhs = (3/2) Om H0^2 / a (delta - mean)
  if ((rs = amr_density_pm(c, lpm, what, L0.rhs, nullptr, nullptr, nullptr)) != MGFR_OK) return rs;
  if (dens_out_dev)
    MG_CK(c, cudaMemcpyAsync(dens_out_dev, L0.rhs, sizeof(double) * (size_t)L0.n,
                             cudaMemcpyDeviceToDevice, c->s));
  double sum = 0.0, sq = 0.0;
  if ((rs = pm_sums(c, P, L0.rhs, L0.n, &sum, &sq)) != MGFR_OK) return rs;
  const double scale = kPoissonScale * om / a;
  k_pm_affine<<<nblocks(L0.n, BS), BS, 0, c->s>>>(L0.rhs, L0.n, scale, sum / (double)L0.n, L0.rhs);
  MG_CK(c, cudaMemsetAsync(L0.phi, 0, sizeof(double) * (size_t)L0.n, c->s));
  c->launches += 1;
  if ((rs = pm_sums(c, P, L0.rhs, L0.n, &sum, &sq)) != MGFR_OK) return rs;
  const double fn = std::sqrt(sq), target = c->cfg.tol_rel * fn;
  double r = fn;
  int it = 0;
  long long updates = 0;
  while (r > target && it < c->cfg.max_vcycles) {
    pm_vcycle(c, P, 0, updates);
    k_pm_resid<<<nblocks(L0.n, BS), BS, 0, c->s>>>(L0.phi, L0.rhs, L0.lg, L0.ih2, P->res);
    c->launches += 1;
    if ((rs = pm_sums(c, P, P->res, L0.n, &sum, &sq)) != MGFR_OK) return rs;
    r = std::sqrt(sq);
    ++it;
    if (!std::isfinite(r)) break;
  }
  // zero mean
  if ((rs = pm_sums(c, P, L0.phi, L0.n, &sum, &sq)) != MGFR_OK) return rs;
  k_pm_affine<<<nblocks(L0.n, BS), BS, 0, c->s>>>(L0.phi, L0.n, 1.0, sum / (double)L0.n, L0.phi);
  c->launches += 1;
  if (phi_out_dev)
    MG_CK(c, cudaMemcpyAsync(phi_out_dev, L0.phi, sizeof(double) * (size_t)L0.n,
                             cudaMemcpyDeviceToDevice, c->s));
  MG_CK(c, cudaEventRecord(c->t1, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  MG_CK(c, cudaGetLastError());
  *work = P;
  if (st) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->t0, c->t1);
    st->vcycles = it;
    st->linear_updates = updates;
    st->res_l2_init = fn;
    st->res_l2_final = r;
    st->f_l2 = fn;
    st->t_solve_ms = ms;
    st->n_levels = 1;
    st->cells_per_level[0] = L0.n;
    st->gpu_launches = c->launches;
    st->t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  }
  if (!(r <= target))
    return set_err(c, MGFR_E_NOCONVERGE, "PM Poisson solve did not reach the tolerance");
  return MGFR_OK;
}

static mgfr_status pm_finish(mgfr_ctx* c, mgfr_status rs) {
  MG_CK(c, cudaEventRecord(c->ev_out, c->s));
  MG_CK(c, cudaStreamWaitEvent(c->user, c->ev_out, 0));
  MG_CK(c, cudaStreamSynchronize(c->s));
  MG_CK(c, cudaGetLastError());
  return rs;
}

extern "C" mgfr_status mgfr_pm_potential(mgfr_ctx* c, int lpm, int what, double* phi_out_dev,
                                         double* dens_out_dev, mgfr_stats* st) {
  if (!c) return MGFR_E_INVALID;
  if (!phi_out_dev) return set_err(c, MGFR_E_INVALID, "phi_out_dev is required");
  PmWork* P = nullptr;
  mgfr_status rs = pm_solve(c, lpm, what, phi_out_dev, dens_out_dev, st, &P);
  if (rs != MGFR_OK && rs != MGFR_E_NOCONVERGE) return rs;
  return pm_finish(c, rs);
}

extern "C" mgfr_status mgfr_pm_accel(mgfr_ctx* c, int lpm, int what, const double* pos_dev,
                                     long long Np, double* acc_out_dev, mgfr_stats* st) {
  if (!c) return MGFR_E_INVALID;
  if (!pos_dev || !acc_out_dev || Np <= 0 || Np >= (1LL << 40))
    return set_err(c, MGFR_E_INVALID, "need positions and a force array of Np >= 1 particles");
  PmWork* P = nullptr;
  mgfr_status rs = pm_solve(c, lpm, what, nullptr, nullptr, st, &P);
  if (rs != MGFR_OK && rs != MGFR_E_NOCONVERGE) return rs;
  PmLevel& L0 = P->L[0];
  if (!P->grad) MG_CK(c, cudaMalloc(&P->grad, sizeof(double) * 3 * (size_t)L0.n));
  const double box = ((AmrWork*)c->amr)->box;
  const double h = box / (double)(1LL << L0.lg);
  k_pm_grad<<<nblocks(L0.n, BS), BS, 0, c->s>>>(L0.phi, L0.lg, 0.5 / h, P->grad);
  k_pm_cic<<<nblocks(Np, BS), BS, 0, c->s>>>(pos_dev, Np, L0.lg, 1.0 / h, P->grad, acc_out_dev);
  c->launches += 2;
  if (st) st->gpu_launches = c->launches;
  return pm_finish(c, rs);
}

extern "C" mgfr_status mgfr_kick_drift(double* pos_dev, double* vel_dev, const double* acc_dev,
                                       long long Np, double kick, double drift, double box,
                                       void* cuda_stream) {
  if (!pos_dev || !vel_dev || !acc_dev || Np <= 0 || Np >= (1LL << 40) || !(box > 0.0) ||
      !std::isfinite(kick) || !std::isfinite(drift))
    return MGFR_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_kick_drift<<<nblocks(3 * Np, BS), BS, 0, s>>>(pos_dev, vel_dev, acc_dev, 3 * Np, kick, drift,
                                                  box);
  if (cudaGetLastError() != cudaSuccess) return MGFR_E_CUDA;
  return MGFR_OK;
}
