// mgfr_internal.cuh -- shared declarations of the GB300 f(R) solver library.
//
// Notation follows Puchwein, Baldi & Springel (arXiv:1305.2418), Sec. 3.2:
// u = ln(f_R / fR_bar), E = e^u, face coefficient b = (E_j + E_i)/2, and
//   L_i(u) = (1/h^2) sum_j b_ij (u_j - u_i) + alpha Rt (1 - e^{-u_i/(n+1)}),
//   f_i    = -alpha Om a^-3 delta_i,
// in comoving units (the physical equation divided by a^-2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mgfr.h"

#define MGFR_MAX_DENSE 12

// Constants of one solve (background of Sec. 2 at scale factor a).
struct Model {
  double Rt;       // Om a^-3 + 4 OL
  double fbar;     // fR_bar(a) < 0
  double alpha;    // a^2 (H0/c)^2 / fbar
  double src;      // -alpha Om a^-3  (f = src * delta)
  double aRt;      // alpha * Rt
  double aRt_np1;  // alpha * Rt / (n+1)
  double inv_np1;  // 1/(n+1)
  double a;
  int n;
};

Model make_model(const mgfr_config& cfg, double a);


// One dense periodic level of the multigrid hierarchy (N = 2^lg).
struct DenseLevel {
  int lg = 0, N = 0;
  long long n = 0;
  double h = 0, ih2 = 0;
  // FP64 nonlinear FAS
  double *u = nullptr, *E = nullptr, *f = nullptr, *uold = nullptr;
  // FP32 nonlinear FAS (mixed precision, phase A)
  float *u32 = nullptr, *f32 = nullptr, *uold32 = nullptr;
  // FP32 linear multigrid on the Jacobian system (mixed precision, phase B)
  float *e32 = nullptr, *r32 = nullptr, *w32 = nullptr;
  // multigrid mask of partial-level solves (Sec. 3.3): only cells with
  // mask > mthr are relaxed; nullptr = all cells.
  const float* mask = nullptr;
  float mthr = 0.4f;
};

struct DenseHier {
  int N = 0, nlev = 0;
  bool mixed = false;
  DenseLevel L[MGFR_MAX_DENSE];
  double* partials = nullptr;  // reduction scratch (2 doubles per block)
  double* scal = nullptr;      // device scalars: [0..1] last norm, [2..7] spare
  double* fdf = nullptr;       // base-level f as double-float pairs (mixed form)
  int nparts = 0;
};

// ---- FP64 dense kernels (dense_f64.cu) -----------------------------------
// Relative drop of the max residual at which the FP64 4^3 coarsest-grid
// solve stops (an accelerator: the fixed point does not depend on it).
constexpr double kCoarseRel64 = 1e-6;
namespace f64 {
void source(const double* delta, double* f, long long n, double src, cudaStream_t s);
void init_u(const double* u0, double* u, double* E, long long n, cudaStream_t s);
void sweep(DenseLevel& L, const Model& m, int colour, double step_cap, cudaStream_t s);
void restrict_resid(DenseLevel& F, DenseLevel& C, const Model& m, cudaStream_t s);
void fas_rhs(DenseLevel& C, const Model& m, cudaStream_t s);
void prolong_corr(DenseLevel& F, DenseLevel& C, int linear, cudaStream_t s);
void coarse_solve(DenseLevel& C, const Model& m, double step_cap, int max_sweeps, double rel,
                  cudaStream_t s);
// ||f - L(u)||_2^2 and max|f - L(u)| into out[0], out[1] (device).
void resid_norm(DenseLevel& L, const Model& m, double* partials, int nparts, double* out,
                cudaStream_t s);
// sum x^2 and max|x| into out[0], out[1] (device).
void norm(const double* x, long long n, double* partials, int nparts, double* out, cudaStream_t s);
void force(const DenseLevel& L, const Model& m, double* fr, double* acc, cudaStream_t s);
}  // namespace f64

// ---- FP32 dense kernels, mixed precision (dense_f32.cu) -------------------
// The FP32 arrays of a dense level (u32, f32, uold32, e32, r32) are stored by
// red-black colour (plane (i + j + k) & 1, then C order of (i, j, k >> 1));
// the FP64 and double-float arrays are in C order.
namespace f32 {
// C-order FP64 x -> colour-split FP32 y on level L's grid
void from64(const double* x, float* y, const DenseLevel& L, cudaStream_t s);
void sweep(DenseLevel& L, const Model& m, int colour, float step_cap, cudaStream_t s);
void restrict_resid(DenseLevel& F, DenseLevel& C, const Model& m, double* partials, int nparts,
                    cudaStream_t s);
void fas_rhs(DenseLevel& C, const Model& m, cudaStream_t s);
void prolong_corr(DenseLevel& F, DenseLevel& C, int linear, cudaStream_t s);
void coarse_solve(DenseLevel& C, const Model& m, float step_cap, int max_sweeps, cudaStream_t s);
// FP32 residual norms of the FP32 iterate (sum r^2, max|r|) into out.
void norm32(DenseLevel& L, const Model& m, double* partials, int nparts, double* out,
            cudaStream_t s);
// Phase B.  From to_df until state_to_fp64, L.u and L.E hold the iterate and
// e^u as double-float pairs (hi + lo floats in each 8-byte slot).
// FP64-accurate residual in double-float (fdf: f as pairs, see f_to_df);
// writes r32 = f - L(u), u32 = u rounded, e32 = 0, and the norms (sum r^2,
// max|r|) into out.
void resid_df(DenseLevel& L, const double* fdf, const Model& m, double* partials, int nparts,
              double* out, cudaStream_t s);
// Linear Gauss-Seidel on J(u32) e = r (J: Jacobian of L at u32).
void lin_sweep(DenseLevel& L, const Model& m, int colour, cudaStream_t s);
void lin_restrict(DenseLevel& F, DenseLevel& C, const Model& m, cudaStream_t s);
void lin_prolong(DenseLevel& F, DenseLevel& C, int linear, cudaStream_t s);
void lin_coarse(DenseLevel& C, const Model& m, int sweeps, cudaStream_t s);
void zero(float* x, long long n, cudaStream_t s);
// u += clamp(e, cap); E = e^u (double-float)
void apply_corr(DenseLevel& L, double cap, cudaStream_t s);
// u = u32, E = e^u as double-float pairs
void to_df(DenseLevel& L, cudaStream_t s);
// the FP64 iterate in L.u -> double-float pairs in place, E = e^u as pairs
void fp64_to_df(DenseLevel& L, cudaStream_t s);
// f (FP64) -> fdf (double-float pairs, same size)
void f_to_df(const double* f, double* fdf, long long n, cudaStream_t s);
// L.u, L.E: double-float pairs -> FP64 (in place)
void state_to_fp64(DenseLevel& L, cudaStream_t s);
}  // namespace f32

// ---- context ---------------------------------------------------------------
struct mgfr_ctx {
  mgfr_config cfg;
  int device = 0;
  cudaStream_t user = nullptr;  // caller's stream
  cudaStream_t s = nullptr;     // internal work stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
  // host-buffer particle solve: copy stream and per-chunk events (created on
  // first use)
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_chunk[8] = {}, ev_copy = nullptr;
  std::string err;
  DenseHier dh;
  double* host_scal = nullptr;  // pinned: norms read back by the host
  // captured V-cycle graphs (FP64 / FP32 nonlinear / linear phase)
  cudaGraphExec_t g_v64 = nullptr, g_v32 = nullptr, g_lin = nullptr;
  char graph_key[256] = {0}, key32[256] = {0}, keylin[256] = {0};
  long long updates_v64 = 0, updates_v32 = 0, updates_lin = 0;
  void* amr = nullptr;    // refined hierarchy workspace (amr.cu)
  void* batch = nullptr;  // batched-solve workspace (batch.cu)
  void* unet = nullptr;   // learned initial guess network (unet.cu)
  void* pm = nullptr;     // particle-mesh potential workspace (pm.cu)
  // profiling: events recorded around base-level kernels inside each graph
  struct ProfRec {
    int fam;
    cudaEvent_t a, b;
    long long cells;
  };
  std::vector<ProfRec> prof[4];  // per graph: 0 v64, 1 v32, 2 lin, 3 refined
  std::vector<cudaEvent_t> evpool;
  int capturing = -1;            // graph being captured (-1: none)
  long long graph_kernels[4] = {0, 0, 0, 0};  // kernel nodes per captured graph
  long long launches = 0;        // kernels launched by the current call
  int u_prev_N = 0;              // grid of the solution held in dh.L[0].u (0: none)
  double* u_learn = nullptr;     // learned initial guess of a solve (MGFR_START_LEARNED)
  long long u_learn_cap = 0;
};

// Network prediction for B boxes of D^3 cells (unet.cu): u_out [B][D^3] from
// the density contrast dscale * x [B][D^3] (device) and |fR0| per box (host),
// on the context's stream, without synchronising.  MGFR_E_INVALID when there
// is no network or D is not a power of two in [32, 512].
mgfr_status unet_predict_batch(mgfr_ctx* c, int B, int D, const double* x, double dscale,
                               const double* fr0_host, double* u_out);
// The initial guess of a base-level solve under cfg.start: *u0 = u_init
// (zero / user start) or the network's prediction from dscale * x (learned),
// held in context workspace (solver.cu).
mgfr_status start_guess(mgfr_ctx* c, int N, const double* x, double dscale, const double* u_init,
                        const double** u0);

// Count of kernel nodes in a graph.
long long count_kernel_nodes(cudaGraph_t g);

// Record a timing event pair around a kernel launch while capturing graph
// `c->capturing` with profiling on.
void prof_begin(mgfr_ctx* c, int fam, long long cells);
void prof_end(mgfr_ctx* c);
void prof_collect(mgfr_ctx* c, int graph, mgfr_stats* st);
void prof_clear(mgfr_ctx* c, int graph);

mgfr_status set_err(mgfr_ctx* c, mgfr_status st, const std::string& msg);
// Range checks of a configuration (false and the reason in why if invalid).
bool validate_cfg(const mgfr_config* c, std::string& why);
void batch_free(mgfr_ctx* c);
void unet_free(mgfr_ctx* c);
void pm_free(mgfr_ctx* c);
#define MG_CK(ctx, call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err((ctx), e_ == cudaErrorMemoryAllocation ? MGFR_E_OOM : MGFR_E_CUDA,   \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

static inline unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
