// noalloc.cu -- mgfr_solve_density_noalloc: the FP64 dense-grid solve for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool or a fixed-budget service that forbids allocation
// on its request path, or code that must not trigger an allocation in the
// middle of its own work.  For them this entry point keeps every scratch
// array of the multigrid hierarchy in one file-scope device array of fixed
// size (NA_MAX_N = 64, i.e. grids up to 64^3; about 7.5 MB that every GPU
// which loads this library holds until the process exits).  The caller still
// passes the input and output buffers.  No cudaMalloc, cudaFree or other
// allocating routine is called, and no context object is needed.
//
// The arithmetic is the same FP64 FAS V-cycle as mgfr_solve_density's FP64
// path, built from the same kernels.
#include <cmath>
#include <cstring>
#include <mutex>

#include "mgfr_internal.cuh"

namespace {

constexpr int NA_MAX_N = 64;
constexpr int NA_MAX_DEV = 64;
constexpr int NA_PARTS = 152 * 8;

// doubles per level (u, E, f and uold on coarse levels), each array padded to
// a multiple of 32 doubles (256 B)
constexpr size_t pad32(size_t n) { return (n + 31) / 32 * 32; }
constexpr size_t na_level_doubles(int N, bool coarse) {
  return (coarse ? 4 : 3) * pad32((size_t)N * N * N);
}
constexpr size_t na_total() {
  size_t s = 0;
  bool coarse = false;
  for (int N = NA_MAX_N; N >= 4; N /= 2) {
    s += na_level_doubles(N, coarse);
    coarse = true;
  }
  return s + pad32(2 * NA_PARTS) + pad32(16);
}
constexpr size_t NA_DOUBLES = na_total();

// The scratch.  Host code must not use this name as an address: in host code
// it is only a stand-in symbol; the device address comes from
// cudaGetSymbolAddress (see na_scratch below).
static __device__ __align__(256) double g_na_scratch[NA_DOUBLES];

std::mutex g_na_mu;
double* g_na_ptr[NA_MAX_DEV] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does it; make that first call before any
// stream capture).
mgfr_status na_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEV) return MGFR_E_CUDA;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return MGFR_E_CUDA;
    g_na_ptr[dev] = (double*)p;
  }
  *out = g_na_ptr[dev];
  return MGFR_OK;
}

struct NaHier {
  int nlev = 0;
  DenseLevel L[MGFR_MAX_DENSE];
  double* partials = nullptr;
  double* scal = nullptr;
};

void na_carve(double* base, int N, double box, NaHier& H) {
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  H.nlev = lg - 1;
  double* p = base;
  for (int l = 0; l < H.nlev; ++l) {
    DenseLevel& L = H.L[l];
    L = DenseLevel();
    L.lg = lg - l;
    L.N = 1 << L.lg;
    L.n = 1LL << (3 * L.lg);
    L.h = box / L.N;
    L.ih2 = 1.0 / (L.h * L.h);
    const size_t a = pad32((size_t)L.n);
    L.u = p;
    p += a;
    L.E = p;
    p += a;
    L.f = p;
    p += a;
    if (l > 0) {
      L.uold = p;
      p += a;
    }
  }
  H.partials = p;
  p += pad32(2 * NA_PARTS);
  H.scal = p;
}

void na_vcycle(NaHier& H, const mgfr_config& g, const Model& m, int l, cudaStream_t s,
               long long& upd) {
  DenseLevel& F = H.L[l];
  DenseLevel& C = H.L[l + 1];
  for (int q = 0; q < g.n_pre; ++q) {
    f64::sweep(F, m, 0, g.step_cap, s);
    f64::sweep(F, m, 1, g.step_cap, s);
    upd += F.n;
  }
  f64::restrict_resid(F, C, m, s);
  f64::fas_rhs(C, m, s);
  if (C.N > 4)
    na_vcycle(H, g, m, l + 1, s, upd);
  else
    f64::coarse_solve(C, m, g.step_cap, 200, kCoarseRel64, s);
  f64::prolong_corr(F, C, g.prolong_linear, s);
  for (int q = 0; q < g.n_post; ++q) {
    f64::sweep(F, m, 0, g.step_cap, s);
    f64::sweep(F, m, 1, g.step_cap, s);
    upd += F.n;
  }
}

}  // namespace

extern "C" mgfr_status mgfr_solve_density_noalloc(const mgfr_config* cfg, const double* delta_dev,
                                                  int N, double box, double a, double* fr_out_dev,
                                                  double* acc_out_dev, void* cuda_stream,
                                                  mgfr_stats* st) {
  if (!cfg || !delta_dev || !fr_out_dev) return MGFR_E_INVALID;
  if (N < 8 || N > NA_MAX_N || (N & (N - 1))) return MGFR_E_INVALID;  // beyond the scratch
  if (!(box > 0.0) || !std::isfinite(box) || !(a > 0.0) || !std::isfinite(a)) return MGFR_E_INVALID;
  const mgfr_config& g = *cfg;
  std::string why;
  if (!validate_cfg(cfg, why)) return MGFR_E_INVALID;  // the same checks as mgfr_create
  if (st) std::memset(st, 0, sizeof(*st));
  double* base = nullptr;
  mgfr_status rs = na_scratch(&base);
  if (rs != MGFR_OK) return rs;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  NaHier H;
  na_carve(base, N, box, H);
  const Model m = make_model(g, a);
  DenseLevel& L0 = H.L[0];
  f64::source(delta_dev, L0.f, L0.n, m.src, s);
  f64::init_u(nullptr, L0.u, L0.E, L0.n, s);
  f64::norm(L0.f, L0.n, H.partials, NA_PARTS, H.scal + 2, s);
  f64::resid_norm(L0, m, H.partials, NA_PARTS, H.scal, s);
  double hs[4];
  if (cudaMemcpyAsync(hs, H.scal, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MGFR_E_CUDA;
  const double fn = std::sqrt(hs[2]), r0 = std::sqrt(hs[0]);
  if (!std::isfinite(fn) || !std::isfinite(r0)) return MGFR_E_INVALID;
  const double target = g.tol_rel * (fn > 0.0 ? fn : r0);
  double r = r0;
  int it = 0;
  long long upd = 0;
  while (r > target && it < g.max_vcycles) {
    na_vcycle(H, g, m, 0, s, upd);
    f64::resid_norm(L0, m, H.partials, NA_PARTS, H.scal, s);
    if (cudaMemcpyAsync(hs, H.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return MGFR_E_CUDA;
    r = std::sqrt(hs[0]);
    ++it;
    if (!std::isfinite(r)) break;
  }
  f64::force(L0, m, fr_out_dev, acc_out_dev, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return MGFR_E_CUDA;
  if (st) {
    st->vcycles = it;
    st->cell_updates = upd;
    st->res_l2_init = r0;
    st->res_l2_final = r;
    st->res_max_final = hs[1];
    st->f_l2 = fn;
    st->n_levels = 1;
    st->cells_per_level[0] = L0.n;
  }
  return r <= target ? MGFR_OK : MGFR_E_NOCONVERGE;
}
