// solver.cu -- context, C ABI and host orchestration of the dense-level solve.
//
// One base-level solve (Puchwein, Baldi & Springel 2013, Sec. 3.3, steps 1-8):
// source f from delta, FAS V-cycles down to 4^3 until
// ||f - L(u)||_2 <= tol ||f||_2, then f_R and the force.  A V-cycle plus the
// residual norm and its read-back is captured once as a CUDA graph and
// replayed; the host reads one norm per V-cycle to test convergence.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <vector>

#include "mgfr_internal.cuh"
#include "amr.cuh"

#define CLIGHT_OVER_H0 2997.92458

Model make_model(const mgfr_config& cfg, double a) {
  Model m;
  const double om = cfg.omega_m, ol = 1.0 - om;
  const double kappa = 1.0 / (CLIGHT_OVER_H0 * CLIGHT_OVER_H0);
  m.Rt = om / (a * a * a) + 4.0 * ol;
  const double Rt1 = om + 4.0 * ol;
  m.fbar = -cfg.fr0_abs * std::pow(Rt1 / m.Rt, (double)(cfg.n + 1));
  m.alpha = a * a * kappa / m.fbar;
  m.src = -m.alpha * om / (a * a * a);
  m.aRt = m.alpha * m.Rt;
  m.aRt_np1 = m.aRt / (cfg.n + 1);
  m.inv_np1 = 1.0 / (cfg.n + 1);
  m.a = a;
  m.n = cfg.n;
  return m;
}

void prof_clear(mgfr_ctx* c, int g) {
  for (auto& r : c->prof[g]) {
    c->evpool.push_back(r.a);
    c->evpool.push_back(r.b);
  }
  c->prof[g].clear();
}

// Timing events are created before a capture starts (no event creation while
// the stream is capturing); prof_begin takes a pair from the pool.
static void prof_reserve(mgfr_ctx* c, size_t pairs) {
  while (c->evpool.size() < 2 * pairs) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->evpool.push_back(e);
  }
}

void prof_reserve_public(mgfr_ctx* c, size_t pairs) { prof_reserve(c, pairs); }

void prof_begin(mgfr_ctx* c, int fam, long long cells) {
  if (!c->cfg.profile || c->capturing < 0 || c->evpool.size() < 2) return;
  mgfr_ctx::ProfRec r{fam, c->evpool.back(), nullptr, cells};
  c->evpool.pop_back();
  r.b = c->evpool.back();
  c->evpool.pop_back();
  cudaEventRecord(r.a, c->s);
  c->prof[c->capturing].push_back(r);
}

void prof_end(mgfr_ctx* c) {
  if (!c->cfg.profile || c->capturing < 0 || c->prof[c->capturing].empty()) return;
  cudaEventRecord(c->prof[c->capturing].back().b, c->s);
}

void prof_collect(mgfr_ctx* c, int g, mgfr_stats* st) {
  if (!c->cfg.profile) return;
  for (auto& r : c->prof[g]) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      if (st) {
        st->kern_ms[r.fam] += ms;
        st->kern_launches[r.fam] += 1;
        st->kern_cells[r.fam] += r.cells;
      }
    } else {
      (void)cudaGetLastError();
    }
  }
  prof_clear(c, g);
}

long long count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  long long k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

mgfr_status set_err(mgfr_ctx* c, mgfr_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

extern "C" {

const char* mgfr_version(void) { return "mgfr 0.1 (sm_103a)"; }

void mgfr_config_default(mgfr_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->omega_m = 0.3;
  c->fr0_abs = 1e-5;
  c->n = 1;
  c->precision = MGFR_PREC_FP64;
  c->tol_rel = 1e-8;
  c->n_pre = 2;
  c->n_post = 2;
  c->max_vcycles = 100;
  c->prolong_linear = 1;
  c->step_cap = 2.0;
  c->max_level = 0;
  c->refine_count = 8;
  c->mixed_switch = 3e-6;
  c->mixed_inner = 3;
  c->max_spins = 1LL << 26;
  c->mask_thres = 0.99;
  c->n_coarse = 0;
  c->start = MGFR_START_ZERO;
}

}  // extern "C"

bool validate_cfg(const mgfr_config* c, std::string& why) {
  auto bad = [&](const char* w) {
    why = w;
    return false;
  };
  if (!c) return bad("config is NULL");
  if (!(c->omega_m > 0.0 && c->omega_m <= 1.0)) return bad("omega_m must be in (0, 1]");
  if (!(c->fr0_abs > 0.0) || !std::isfinite(c->fr0_abs)) return bad("fr0_abs must be > 0");
  if (c->n < 1 || c->n > 16) return bad("n must be in [1, 16]");
  if (c->precision != MGFR_PREC_FP64 && c->precision != MGFR_PREC_MIXED)
    return bad("precision must be 0 (FP64) or 1 (mixed)");
  if (!(c->tol_rel > 0.0 && c->tol_rel < 1.0)) return bad("tol_rel must be in (0, 1)");
  if (c->n_pre < 0 || c->n_post < 0 || c->n_pre + c->n_post < 1 || c->n_pre > 16 ||
      c->n_post > 16)
    return bad("n_pre + n_post must be >= 1 (each <= 16)");
  if (c->max_vcycles < 1 || c->max_vcycles > 100000) return bad("max_vcycles out of range");
  if (!(c->step_cap > 0.0)) return bad("step_cap must be > 0");
  if (c->max_level < 0 || c->max_level > 8) return bad("max_level must be in [0, 8]");
  if (c->refine_count < -1) return bad("refine_count must be >= -1");
  if (!(c->mixed_switch > 0.0 && c->mixed_switch < 1.0)) return bad("mixed_switch in (0,1)");
  if (c->mixed_inner < 1 || c->mixed_inner > 16) return bad("mixed_inner in [1, 16]");
  if (c->max_spins < 0) return bad("max_spins must be >= 0");
  if (!(c->mask_thres >= 0.0 && c->mask_thres < 1.0)) return bad("mask_thres in [0, 1)");
  if (c->n_coarse < 0 || c->n_coarse > 16) return bad("n_coarse in [0, 16]");
  if (c->start < MGFR_START_ZERO || c->start > MGFR_START_PREVIOUS_ALL)
    return bad("start must be 0 (zero), 1 (user), 2 (learned), 3 (previous) or 4 (previous, all levels)");
  return true;
}

mgfr_status start_guess(mgfr_ctx* c, int N, const double* x, double dscale, const double* u_init,
                        const double** u0) {
  *u0 = u_init;
  if (c->cfg.start == MGFR_START_USER && !u_init)
    return set_err(c, MGFR_E_INVALID, "start = user needs u_init");
  if (c->cfg.start == MGFR_START_PREVIOUS || c->cfg.start == MGFR_START_PREVIOUS_ALL) {
    if (u_init) return set_err(c, MGFR_E_INVALID, "start = previous takes no u_init");
    if (c->u_prev_N != N || c->dh.N != N) {
      if (c->cfg.start == MGFR_START_PREVIOUS_ALL) return MGFR_OK;  // nothing held: zero start
      return set_err(c, MGFR_E_INVALID, "start = previous: no solution of this size in the context");
    }
    *u0 = c->dh.L[0].u;  // kept in place; the initialisation forms e^u from it
    return MGFR_OK;
  }
  if (c->cfg.start != MGFR_START_LEARNED) return MGFR_OK;
  if (u_init) return set_err(c, MGFR_E_INVALID, "start = learned takes no u_init");
  const long long n = (long long)N * N * N;
  if (c->u_learn_cap < n) {
    if (c->u_learn) cudaFree(c->u_learn);
    c->u_learn = nullptr;
    c->u_learn_cap = 0;
    MG_CK(c, cudaMalloc(&c->u_learn, sizeof(double) * (size_t)n));
    c->u_learn_cap = n;
  }
  const double fr0 = c->cfg.fr0_abs;
  mgfr_status rs = unet_predict_batch(c, 1, N, x, dscale, &fr0, c->u_learn);
  if (rs != MGFR_OK) return rs;
  *u0 = c->u_learn;
  return MGFR_OK;
}

static void free_dense(DenseHier& H) {
  for (int l = 0; l < MGFR_MAX_DENSE; ++l) {
    DenseLevel& L = H.L[l];
    void* ps[] = {L.u, L.E, L.f, L.uold, L.u32, L.f32, L.uold32, L.e32, L.r32, L.w32};
    for (void* p : ps)
      if (p) cudaFree(p);
    L = DenseLevel();
  }
  if (H.partials) cudaFree(H.partials);
  if (H.scal) cudaFree(H.scal);
  if (H.fdf) cudaFree(H.fdf);
  H = DenseHier();
}

static void drop_graphs(mgfr_ctx* c) {
  if (c->g_v64) cudaGraphExecDestroy(c->g_v64);
  if (c->g_v32) cudaGraphExecDestroy(c->g_v32);
  if (c->g_lin) cudaGraphExecDestroy(c->g_lin);
  c->g_v64 = c->g_v32 = c->g_lin = nullptr;
  c->graph_key[0] = c->key32[0] = c->keylin[0] = 0;
  for (int g = 0; g < 3; ++g) prof_clear(c, g);
}

// Allocate the dense hierarchy N, N/2, ..., 4 (FP64 arrays always; FP32 ones
// for the mixed form).
static mgfr_status ensure_dense(mgfr_ctx* c, int N, bool mixed) {
  DenseHier& H = c->dh;
  if (H.N == N && (H.mixed || !mixed)) return MGFR_OK;
  drop_graphs(c);
  free_dense(H);
  c->u_prev_N = 0;
  H.N = N;
  H.mixed = mixed;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  H.nlev = lg - 1;  // N ... 4
  for (int l = 0; l < H.nlev; ++l) {
    DenseLevel& L = H.L[l];
    L.lg = lg - l;
    L.N = 1 << L.lg;
    L.n = 1LL << (3 * L.lg);
    size_t b8 = sizeof(double) * (size_t)L.n, b4 = sizeof(float) * (size_t)L.n;
    MG_CK(c, cudaMalloc(&L.u, b8));
    MG_CK(c, cudaMalloc(&L.E, b8));
    MG_CK(c, cudaMalloc(&L.f, b8));
    if (l > 0) MG_CK(c, cudaMalloc(&L.uold, b8));
    if (mixed) {
      MG_CK(c, cudaMalloc(&L.u32, b4));
      MG_CK(c, cudaMalloc(&L.f32, b4));
      MG_CK(c, cudaMalloc(&L.e32, b4));
      MG_CK(c, cudaMalloc(&L.r32, b4));
      if (l > 0) MG_CK(c, cudaMalloc(&L.uold32, b4));
    }
  }
  H.nparts = 152 * 8;
  if (mixed) MG_CK(c, cudaMalloc(&H.fdf, sizeof(double) * (size_t)H.L[0].n));
  MG_CK(c, cudaMalloc(&H.partials, sizeof(double) * 2 * H.nparts));
  MG_CK(c, cudaMalloc(&H.scal, sizeof(double) * 16));
  return MGFR_OK;
}

static void set_spacing(DenseHier& H, double box) {
  for (int l = 0; l < H.nlev; ++l) {
    H.L[l].h = box / H.L[l].N;
    H.L[l].ih2 = 1.0 / (H.L[l].h * H.L[l].h);
  }
}

mgfr_status ensure_dense_public(mgfr_ctx* c, int N, bool mixed, double box) {
  mgfr_status rs = ensure_dense(c, N, mixed);
  if (rs != MGFR_OK) return rs;
  set_spacing(c->dh, box);
  return MGFR_OK;
}

// ---- FP64 V-cycle (Sec. 3.3, steps 3-7) ------------------------------------
static void vcycle64(mgfr_ctx* c, const Model& m, int l, long long& updates) {
  DenseHier& H = c->dh;
  DenseLevel& F = H.L[l];
  DenseLevel& C = H.L[l + 1];
  const mgfr_config& g = c->cfg;
  for (int s = 0; s < g.n_pre; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l == 0) prof_begin(c, 0, F.n);
      f64::sweep(F, m, col, g.step_cap, c->s);
      if (l == 0) prof_end(c);
    }
    updates += F.n;
  }
  f64::restrict_resid(F, C, m, c->s);
  f64::fas_rhs(C, m, c->s);
  if (C.N > 4)
    vcycle64(c, m, l + 1, updates);
  else
    f64::coarse_solve(C, m, g.step_cap, 200, kCoarseRel64, c->s);
  f64::prolong_corr(F, C, g.prolong_linear, c->s);
  for (int s = 0; s < g.n_post; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l == 0) prof_begin(c, 0, F.n);
      f64::sweep(F, m, col, g.step_cap, c->s);
      if (l == 0) prof_end(c);
    }
    updates += F.n;
  }
}

// Capture `body` on the work stream into an executable graph.
template <class Fn>
mgfr_status capture(mgfr_ctx* c, int gid, cudaGraphExec_t* out, Fn body) {
  cudaGraph_t g = nullptr;
  MG_CK(c, cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
  c->capturing = -1;
  body();
  cudaError_t e = cudaStreamEndCapture(c->s, &g);
  if (e != cudaSuccess) return set_err(c, MGFR_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  c->graph_kernels[gid] = count_kernel_nodes(g);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return set_err(c, MGFR_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return MGFR_OK;
}

// Issue one cycle: replay its graph, or with cfg.profile run the same launch
// sequence directly on the stream with timing events around the profiled
// kernels (events are not recorded inside graphs).
template <class Fn>
mgfr_status issue(mgfr_ctx* c, int gid, cudaGraphExec_t gx, Fn body) {
  if (c->cfg.profile) {
    prof_clear(c, gid);
    prof_reserve(c, 4 + 2 * (size_t)(c->cfg.n_pre + c->cfg.n_post) * (size_t)c->cfg.mixed_inner);
    c->capturing = gid;
    body();
    c->capturing = -1;
  } else {
    MG_CK(c, cudaGraphLaunch(gx, c->s));
  }
  c->launches += c->graph_kernels[gid];
  return MGFR_OK;
}

void make_key(char* key, size_t n, const char* tag, int N, double box, const Model& m,
                     const mgfr_config& g) {
  std::snprintf(key, n, "%s|%d|%.17g|%.17g|%.17g|%d|%d|%d|%d|%.17g|%d|%d", tag, N, box, m.alpha,
                m.Rt, m.n, g.n_pre, g.n_post, g.prolong_linear, g.step_cap, g.mixed_inner,
                g.profile);
}

static mgfr_status sync_read(mgfr_ctx* c) {
  MG_CK(c, cudaStreamSynchronize(c->s));
  return MGFR_OK;
}

// FP64 base-level solve on the already-filled hierarchy (f on level 0, u/E
// initialised).  Fills stats (vcycles, updates, norms).
mgfr_status dense_solve64(mgfr_ctx* c, const Model& m, double box, mgfr_stats* st) {
  DenseHier& H = c->dh;
  DenseLevel& L0 = H.L[0];
  const mgfr_config& g = c->cfg;
  double* hs = c->host_scal;
  f64::norm(L0.f, L0.n, H.partials, H.nparts, H.scal + 2, c->s);
  f64::resid_norm(L0, m, H.partials, H.nparts, H.scal, c->s);
  c->launches += 4;
  MG_CK(c, cudaMemcpyAsync(hs, H.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  mgfr_status rs = sync_read(c);
  if (rs != MGFR_OK) return rs;
  const double fn = std::sqrt(hs[2]), r0 = std::sqrt(hs[0]);
  if (!std::isfinite(fn) || !std::isfinite(r0))
    return set_err(c, MGFR_E_INVALID, "non-finite density or initial guess");
  const double target = g.tol_rel * (fn > 0.0 ? fn : r0);
  long long updates_per = 0;
  char key[256];
  make_key(key, sizeof(key), "v64", H.N, box, m, g);
  auto body64 = [&]() {
    updates_per = 0;
    vcycle64(c, m, 0, updates_per);
    f64::resid_norm(L0, m, H.partials, H.nparts, H.scal, c->s);
    cudaMemcpyAsync(hs, H.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s);
  };
  if (!c->g_v64 || std::strcmp(key, c->graph_key) != 0) {
    if (c->g_v64) cudaGraphExecDestroy(c->g_v64);
    c->g_v64 = nullptr;
    mgfr_status cs = capture(c, 0, &c->g_v64, body64);
    if (cs != MGFR_OK) return cs;
    std::strcpy(c->graph_key, key);
    c->updates_v64 = updates_per;
  }
  double r = r0;
  int it = 0;
  while (r > target && it < g.max_vcycles) {
    if ((rs = issue(c, 0, c->g_v64, body64)) != MGFR_OK) return rs;
    rs = sync_read(c);
    if (rs != MGFR_OK) return rs;
    prof_collect(c, 0, st);
    r = std::sqrt(hs[0]);
    ++it;
    if (!std::isfinite(r)) break;
  }
  if (st) {
    st->vcycles = it;
    st->cell_updates += (long long)it * c->updates_v64;
    st->res_l2_init = r0;
    st->res_l2_final = r;
    st->res_max_final = hs[1];
    st->f_l2 = fn;
  }
  if (!(r <= target))
    return set_err(c, MGFR_E_NOCONVERGE, "base level did not converge within max_vcycles");
  return MGFR_OK;
}


// ---- mixed precision ---------------------------------------------------------
// Phase A: FP32 nonlinear FAS V-cycle (same steps as vcycle64).
static void vcycle32(mgfr_ctx* c, const Model& m, int l, long long& updates) {
  DenseHier& H = c->dh;
  DenseLevel& F = H.L[l];
  DenseLevel& C = H.L[l + 1];
  const mgfr_config& g = c->cfg;
  const float cap = (float)g.step_cap;
  for (int s = 0; s < g.n_pre; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l == 0) prof_begin(c, 0, F.n);
      f32::sweep(F, m, col, cap, c->s);
      if (l == 0) prof_end(c);
    }
    updates += F.n;
  }
  f32::restrict_resid(F, C, m, H.partials, H.nparts, c->s);
  f32::fas_rhs(C, m, c->s);
  if (C.N > 4)
    vcycle32(c, m, l + 1, updates);
  else
    f32::coarse_solve(C, m, cap, 40, c->s);
  f32::prolong_corr(F, C, g.prolong_linear, c->s);
  for (int s = 0; s < g.n_post; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l == 0) prof_begin(c, 0, F.n);
      f32::sweep(F, m, col, cap, c->s);
      if (l == 0) prof_end(c);
    }
    updates += F.n;
  }
}

// Phase B: FP32 linear V-cycle on J(u) e = r (correction scheme).
static void vcycle_lin(mgfr_ctx* c, const Model& m, int l, long long& updates) {
  DenseHier& H = c->dh;
  DenseLevel& F = H.L[l];
  DenseLevel& C = H.L[l + 1];
  const mgfr_config& g = c->cfg;
  for (int s = 0; s < g.n_pre; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l == 0) prof_begin(c, 1, F.n);
      f32::lin_sweep(F, m, col, c->s);
      if (l == 0) prof_end(c);
    }
    updates += F.n;
  }
  f32::lin_restrict(F, C, m, c->s);
  if (C.N > 4)
    vcycle_lin(c, m, l + 1, updates);
  else
    f32::lin_coarse(C, m, 40, c->s);
  f32::lin_prolong(F, C, g.prolong_linear, c->s);
  for (int s = 0; s < g.n_post; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l == 0) prof_begin(c, 1, F.n);
      f32::lin_sweep(F, m, col, c->s);
      if (l == 0) prof_end(c);
    }
    updates += F.n;
  }
}

// Mixed form: FP32 nonlinear V-cycles until ||r|| <= mixed_switch ||f|| (or
// they stall), then FP64 defect correction: r = f - L(u) in FP64, FP32 linear
// V-cycles on J e = r, u += e in FP64, until the FP64 stopping test holds.
// warm: the start is not zero; its FP64-accurate residual is formed first,
// and if it already meets the switch point the FP32 phase (which would round
// the start to FP32) is skipped.
mgfr_status dense_solve_mixed(mgfr_ctx* c, const Model& m, double box, mgfr_stats* st, bool warm) {
  DenseHier& H = c->dh;
  DenseLevel& L0 = H.L[0];
  const mgfr_config& g = c->cfg;
  double* hs = c->host_scal;
  // ||f|| in FP64 (a sum of squares); the initial residual, which only decides
  // whether to iterate, from the FP32 copies the V-cycles start from
  f64::norm(L0.f, L0.n, H.partials, H.nparts, H.scal + 2, c->s);
  f32::from64(L0.f, L0.f32, L0, c->s);
  f32::from64(L0.u, L0.u32, L0, c->s);
  f32::norm32(L0, m, H.partials, H.nparts, H.scal, c->s);
  c->launches += 6;
  MG_CK(c, cudaMemcpyAsync(hs, H.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  mgfr_status rs = sync_read(c);
  if (rs != MGFR_OK) return rs;
  const double fn = std::sqrt(hs[2]), r0 = std::sqrt(hs[0]);
  if (!std::isfinite(fn) || !std::isfinite(r0))
    return set_err(c, MGFR_E_INVALID, "non-finite density or initial guess");
  const double ref = fn > 0.0 ? fn : r0;
  const double target = g.tol_rel * ref;
  if (st) {
    st->res_l2_init = r0;
    st->f_l2 = fn;
  }
  char key[256];
  make_key(key, sizeof(key), "v32", H.N, box, m, g);
  long long upd = 0;
  auto body32 = [&]() {
    upd = 0;
    vcycle32(c, m, 0, upd);
    f32::norm32(L0, m, H.partials, H.nparts, H.scal, c->s);
    cudaMemcpyAsync(hs, H.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s);
  };
  if (!c->g_v32 || std::strcmp(key, c->key32) != 0) {
    if (c->g_v32) cudaGraphExecDestroy(c->g_v32);
    c->g_v32 = nullptr;
    rs = capture(c, 1, &c->g_v32, body32);
    if (rs != MGFR_OK) return rs;
    std::strcpy(c->key32, key);
    c->updates_v32 = upd;
  }
  make_key(key, sizeof(key), "lin", H.N, box, m, g);
  auto bodylin = [&]() {
    upd = 0;
    for (int q = 0; q < g.mixed_inner; ++q) vcycle_lin(c, m, 0, upd);
    f32::apply_corr(L0, g.step_cap, c->s);
    prof_begin(c, 2, L0.n);
    f32::resid_df(L0, H.fdf, m, H.partials, H.nparts, H.scal, c->s);
    prof_end(c);
    cudaMemcpyAsync(hs, H.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s);
  };
  if (!c->g_lin || std::strcmp(key, c->keylin) != 0) {
    if (c->g_lin) cudaGraphExecDestroy(c->g_lin);
    c->g_lin = nullptr;
    rs = capture(c, 2, &c->g_lin, bodylin);
    if (rs != MGFR_OK) return rs;
    std::strcpy(c->keylin, key);
    c->updates_lin = upd;
  }
  int vc = 0, outer = 0;
  double r = r0;
  bool state_df = false;  // L0.u, L0.E hold double-float pairs (phase B)
  bool skip_a = false;    // the start already meets the switch point
  if (r > target || warm) {
    f32::f_to_df(L0.f, H.fdf, L0.n, c->s);
    c->launches += 1;
  }
  if (warm) {
    f32::fp64_to_df(L0, c->s);
    f32::resid_df(L0, H.fdf, m, H.partials, H.nparts, H.scal, c->s);
    c->launches += 3;
    state_df = true;
    MG_CK(c, cudaMemcpyAsync(hs, H.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    if ((rs = sync_read(c)) != MGFR_OK) return rs;
    r = std::sqrt(hs[0]);
    if (st) st->res_l2_init = r;
    skip_a = r <= g.mixed_switch * ref;
  }
  // Phases alternate: A until it reaches mixed_switch or stalls, then B while
  // the FP64 residual keeps falling; a rise in B sends the iterate back to A.
  for (int round = 0; round < 8 && r > target; ++round) {
    if (!(skip_a && round == 0)) {
      double prev = -1.0;
      while (vc < g.max_vcycles) {
        if ((rs = issue(c, 1, c->g_v32, body32)) != MGFR_OK) return rs;
        if ((rs = sync_read(c)) != MGFR_OK) return rs;
        prof_collect(c, 1, st);
        ++vc;
        const double r32 = std::sqrt(hs[0]);
        if (!std::isfinite(r32)) break;
        if (r32 <= g.mixed_switch * ref) break;
        if (prev > 0.0 && r32 > 0.7 * prev) break;
        prev = r32;
      }
      f32::to_df(L0, c->s);
      f32::resid_df(L0, H.fdf, m, H.partials, H.nparts, H.scal, c->s);
      c->launches += 3;
      state_df = true;
      MG_CK(c, cudaMemcpyAsync(hs, H.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
      if ((rs = sync_read(c)) != MGFR_OK) return rs;
      r = std::sqrt(hs[0]);
    }
    bool rose = false;
    while (r > target && outer < g.max_vcycles) {
      if ((rs = issue(c, 2, c->g_lin, bodylin)) != MGFR_OK) return rs;
      if ((rs = sync_read(c)) != MGFR_OK) return rs;
      prof_collect(c, 2, st);
      ++outer;
      const double rn = std::sqrt(hs[0]);
      if (!(rn < r)) {
        rose = true;
        r = rn;
        break;
      }
      r = rn;
    }
    if (!rose || vc >= g.max_vcycles) break;
    // back to phase A from the current FP64 iterate (u32 = fp32(u) already)
  }
  if (state_df) {  // the FP64 iterate and e^u for the caller
    f32::state_to_fp64(L0, c->s);
    c->launches += 2;
  }
  if (st) {
    st->vcycles = vc;
    st->outer_iters = outer;
    st->cell_updates += (long long)vc * c->updates_v32;
    st->linear_updates += (long long)outer * c->updates_lin;
    st->res_l2_final = r;
    st->res_max_final = hs[1];
  }
  if (!(r <= target))
    return set_err(c, MGFR_E_NOCONVERGE, "mixed solve did not reach the FP64 tolerance");
  return MGFR_OK;
}

extern "C" {

mgfr_status mgfr_create(mgfr_ctx** out, const mgfr_config* cfg, int device, void* stream) {
  if (!out) return MGFR_E_INVALID;
  *out = nullptr;
  std::string why;
  if (!validate_cfg(cfg, why)) return MGFR_E_INVALID;
  mgfr_ctx* c = new mgfr_ctx();
  c->cfg = *cfg;
  c->device = device;
  c->user = (cudaStream_t)stream;
  auto fail = [&](cudaError_t e) {
    (void)e;
    mgfr_destroy(c);
    return e == cudaErrorMemoryAllocation ? MGFR_E_OOM : MGFR_E_CUDA;
  };
  cudaError_t e;
  if ((e = cudaSetDevice(device)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
  cudaEvent_t* evs[] = {&c->ev_in, &c->ev_out};
  for (auto* ev : evs)
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreate(&c->t0)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreate(&c->t1)) != cudaSuccess) return fail(e);
  if ((e = cudaMallocHost(&c->host_scal, 64 * sizeof(double))) != cudaSuccess) return fail(e);
  *out = c;
  return MGFR_OK;
}

mgfr_status mgfr_set_config(mgfr_ctx* c, const mgfr_config* cfg) {
  if (!c) return MGFR_E_INVALID;
  std::string why;
  if (!validate_cfg(cfg, why)) return set_err(c, MGFR_E_INVALID, why);
  c->cfg = *cfg;
  drop_graphs(c);
  return MGFR_OK;
}

const char* mgfr_last_error(const mgfr_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void mgfr_destroy(mgfr_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->s) cudaStreamSynchronize(c->s);
  if (c->cs) cudaStreamSynchronize(c->cs);
  drop_graphs(c);
  free_dense(c->dh);
  amr_free(c);
  batch_free(c);
  unet_free(c);
  pm_free(c);
  if (c->u_learn) cudaFree(c->u_learn);
  for (auto e : c->evpool) cudaEventDestroy(e);
  c->evpool.clear();
  if (c->host_scal) cudaFreeHost(c->host_scal);
  cudaEvent_t evs[] = {c->ev_in, c->ev_out, c->t0, c->t1, c->ev_copy};
  for (auto ev : evs)
    if (ev) cudaEventDestroy(ev);
  for (auto ev : c->ev_chunk)
    if (ev) cudaEventDestroy(ev);
  if (c->s) cudaStreamDestroy(c->s);
  if (c->cs) cudaStreamDestroy(c->cs);
  delete c;
}

static bool pow2_in(int N, int lo, int hi) { return N >= lo && N <= hi && (N & (N - 1)) == 0; }

mgfr_status mgfr_solve_density(mgfr_ctx* c, const double* delta, int N, double box, double a,
                               const double* u_init, double* fr_out, double* acc_out,
                               double* u_out, mgfr_stats* st) {
  if (!c) return MGFR_E_INVALID;
  if (!delta || !fr_out) return set_err(c, MGFR_E_INVALID, "delta and fr_out are required");
  if (!pow2_in(N, 8, 1024)) return set_err(c, MGFR_E_INVALID, "N must be a power of two in [8, 1024]");
  if (!(box > 0.0) || !std::isfinite(box)) return set_err(c, MGFR_E_INVALID, "box must be > 0");
  if (!(a > 0.0) || !std::isfinite(a)) return set_err(c, MGFR_E_INVALID, "a must be > 0");
  auto w0 = std::chrono::steady_clock::now();
  MG_CK(c, cudaSetDevice(c->device));
  if (st) std::memset(st, 0, sizeof(*st));
  const bool mixed = c->cfg.precision == MGFR_PREC_MIXED;
  // the base level of a particle solve lives in the dense workspace this
  // solve overwrites: its hierarchy is no longer queryable
  amr_invalidate(c);
  mgfr_status rs = ensure_dense(c, N, mixed);
  if (rs != MGFR_OK) return rs;
  DenseHier& H = c->dh;
  set_spacing(H, box);
  const Model m = make_model(c->cfg, a);
  MG_CK(c, cudaEventRecord(c->ev_in, c->user));
  MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_in, 0));
  DenseLevel& L0 = H.L[0];
  c->launches = 0;
  const double* u0 = nullptr;
  if ((rs = start_guess(c, N, delta, 1.0, u_init, &u0)) != MGFR_OK) return rs;
  f64::source(delta, L0.f, L0.n, m.src, c->s);
  f64::init_u(u0, L0.u, L0.E, L0.n, c->s);
  c->u_prev_N = 0;  // valid again once solved
  c->launches += 2;
  MG_CK(c, cudaEventRecord(c->t0, c->s));
  rs = mixed ? dense_solve_mixed(c, m, box, st, u0 != nullptr) : dense_solve64(c, m, box, st);
  MG_CK(c, cudaEventRecord(c->t1, c->s));
  if (rs == MGFR_OK || rs == MGFR_E_NOCONVERGE) {
    f64::force(L0, m, fr_out, acc_out, c->s);
    c->launches += 1;
    if (u_out) MG_CK(c, cudaMemcpyAsync(u_out, L0.u, sizeof(double) * L0.n, cudaMemcpyDeviceToDevice, c->s));
    c->u_prev_N = N;  // the next solve may start from it
  } else {
    c->u_prev_N = 0;
  }
  MG_CK(c, cudaEventRecord(c->ev_out, c->s));
  MG_CK(c, cudaStreamWaitEvent(c->user, c->ev_out, 0));
  MG_CK(c, cudaStreamSynchronize(c->s));
  MG_CK(c, cudaGetLastError());
  if (st) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->t0, c->t1);
    st->t_solve_ms = ms;
    st->n_levels = 1;
    st->cells_per_level[0] = L0.n;
    st->gpu_launches = c->launches;
    st->t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  }
  return rs;
}

}  // extern "C"
