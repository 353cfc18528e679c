/*
 * mgfr.h -- C ABI of the GB300 f(R) modified-gravity field solver.
 *
 * The library solves the quasi-static scalar-field equation of Hu-Sawicki
 * f(R) gravity in the log variable u = ln(f_R / fR_bar(a)) (Puchwein, Baldi &
 * Springel, arXiv:1305.2418, Sec. 3.2, Eqs. (15) and (16)) with
 * red-black Newton-Gauss-Seidel relaxation accelerated by FAS multigrid
 * (Sec. 3.3, Eqs. (23), (27), (29)), on a
 * periodic base grid or on a hierarchy refined where particle counts are high
 * (Sec. 3.1), and returns f_R = fR_bar e^u and the extra acceleration
 * a_MG = (c^2/2) grad f_R (Sec. 2, Eq. (13)).
 *
 * Conventions shared by every entry point:
 *  - Lengths are comoving Mpc/h; positions are wrapped periodically into
 *    [0, box).  The model is flat LCDM background (Omega_L = 1 - Omega_m)
 *    with fR_bar0 = -fr0_abs < 0.
 *  - The discrete equation, in comoving units, is
 *      L_i(u) = (1/h^2) sum_{6 nbrs j} (e^{u_j} + e^{u_i})/2 (u_j - u_i)
 *               + alpha Rt (1 - e^{-u_i/(n+1)})  =  f_i = -alpha Om a^-3 delta_i,
 *    Rt = Om a^-3 + 4 OL, fR_bar(a) = -fr0_abs (Rt(1)/Rt(a))^{n+1},
 *    alpha = a^2 (H0/c)^2 / fR_bar(a)  (Sec. 3.2 divided by a^-2).
 *  - A solve stops when ||f - L(u)||_2 <= tol_rel ||f||_2 on the level being
 *    solved (||f - L(0)||_2 = ||f||_2 is the zero-start residual).
 *  - Output force unit: acc = a_MG / c^2 = grad_x f_R / (2a), in h/Mpc;
 *    multiply by c^2 for physical units.
 *  - Dense grids are C order a[i][j][k] with i along x (slowest), k along z.
 *    Grid force arrays are component-major [3][N^3]; particle arrays are
 *    [Np][3].
 *  - Memory: every pointer named *_dev is device memory owned by the caller;
 *    it must stay valid until the call returns.  The library allocates its
 *    own workspaces inside the context (freed by mgfr_destroy).  Work runs on
 *    the context's stream (given at mgfr_create; 0 = legacy default stream)
 *    and every solve call returns only after its results are written.
 *  - Errors: every call returns an mgfr_status and never aborts; the text of
 *    the last error is available from mgfr_last_error.  Kernel waits are
 *    bounded; no call traps the GPU.
 */
#ifndef MGFR_H
#define MGFR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgfr_ctx mgfr_ctx; /* opaque, owned by the library */

typedef enum {
  MGFR_OK = 0,
  MGFR_E_INVALID = 1,     /* bad argument (size, NaN, pointer, parameter) */
  MGFR_E_CUDA = 2,        /* a CUDA runtime call failed                   */
  MGFR_E_OOM = 3,         /* device workspace allocation failed           */
  MGFR_E_NOCONVERGE = 4,  /* max_vcycles reached; outputs hold last iterate */
  MGFR_E_TIMEOUT = 5,     /* a bounded device wait gave up                */
  MGFR_E_UNSUPPORTED = 6  /* case the library does not handle               */
} mgfr_status;

typedef enum { MGFR_PREC_FP64 = 0, MGFR_PREC_MIXED = 1 } mgfr_precision;

typedef struct {
  /* model (Sec. 2) */
  double omega_m;      /* matter density parameter; Omega_L = 1 - omega_m  */
  double fr0_abs;      /* |fR_bar0| > 0                                     */
  int n;               /* Hu-Sawicki exponent n >= 1                        */
  /* solver (Sec. 3.3) */
  int precision;       /* mgfr_precision                                    */
  double tol_rel;      /* stopping test, default 1e-8                       */
  int n_pre, n_post;   /* red-black sweeps before/after the coarse grid     */
  int max_vcycles;     /* per level solve, default 100                      */
  int prolong_linear;  /* 1: linear reconstruction, 0: straight injection   */
  double step_cap;     /* clamp on a Newton step |du| (default 2)           */
  /* refinement (Sec. 3.1) */
  int max_level;       /* number of refinement levels above the base       */
  int refine_count;    /* a cell is refined when it holds > refine_count    */
  /* mixed precision: FP32 nonlinear V-cycles until the relative residual is
   * below mixed_switch, then FP64 defect-correction iterations, each with
   * mixed_inner FP32 linear V-cycles on the Jacobian system.               */
  double mixed_switch; /* default 3e-6                                      */
  int mixed_inner;     /* default 3                                         */
  long long max_spins; /* bound on any device-side wait (default 1<<26)     */
  int profile;         /* 1: time the base-level sweep kernels with CUDA
                          events recorded around each launch (see stats)   */
  double mask_thres;   /* refined-level multigrid: coarse cells are relaxed
                          where the mask exceeds this (Sec. 3.3 uses 0.4;
                          default 0.99 relaxes only fully covered cells,
                          which converges also for weak screening)        */
  int n_coarse;        /* red-black sweeps before and after the coarse grid
                          on the coarser levels of a refined-level solve
                          (0: n_pre and n_post, the default)               */
  int start;           /* mgfr_start: initial guess of the (base-level) solve */
} mgfr_config;

/* Initial guess of a solve.  The paper starts each step from the previous
 * step's solution (Sec. 3.3, step 2); the learned start is an addition of
 * this library.
 *   MGFR_START_ZERO    u = 0 unless the call passes u_init (the default);
 *   MGFR_START_USER    u = u_init, which the call must pass (MGFR_E_INVALID
 *                      if it is NULL): the previous-step warm start;
 *   MGFR_START_LEARNED u = the context's network (mgfr_unet_init or
 *                      mgfr_unet_load) applied to the density contrast with
 *                      the context's |fR0|, n and Omega_m; u_init must be
 *                      NULL.  The grid (the base grid of a particle solve)
 *                      must be a power of two in [32, 512].  Batch items
 *                      keep a u_init_dev they pass; the others of 32^3 and
 *                      more are predicted in groups of one size, those below
 *                      32^3 start from zero.  The prediction runs inside the
 *                      call, on the context's stream.
 *   MGFR_START_PREVIOUS u = the base-level solution of the context's last
 *                      density or particle solve of the same grid size (the
 *                      previous step's u, kept in the context: no copy);
 *                      u_init must be NULL; MGFR_E_INVALID if there is none
 *                      (first solve, another size or precision since).  Not
 *                      for batches.
 *   MGFR_START_PREVIOUS_ALL  as MGFR_START_PREVIOUS on the base level, and in
 *                      a particle solve also on the refined levels: every oct
 *                      that the context's previous particle solve (same base
 *                      grid and box, made in this mode) also had starts from
 *                      that solve's u there; the other octs start from the
 *                      prolonged coarser solution (Sec. 3.3).  The paper's
 *                      step list starts only the base level from the previous
 *                      step; this carries the previous solution to the
 *                      refined levels too, an accelerator that leaves the
 *                      answer unchanged.  When nothing of a previous solve is
 *                      held (first solve of the context) it is the zero
 *                      start; u_init must be NULL; not for batches. */
typedef enum {
  MGFR_START_ZERO = 0,
  MGFR_START_USER = 1,
  MGFR_START_LEARNED = 2,
  MGFR_START_PREVIOUS = 3,
  MGFR_START_PREVIOUS_ALL = 4
} mgfr_start;

typedef struct {
  int vcycles;               /* nonlinear V-cycles (all precisions), base level */
  int outer_iters;           /* FP64 defect-correction iterations (mixed)  */
  long long cell_updates;    /* nonlinear NGS updates, all levels          */
  long long linear_updates;  /* FP32 linear Gauss-Seidel updates (mixed)   */
  double res_l2_init;        /* ||f - L(u0)||_2 on the base level          */
  double res_l2_final;       /* ||f - L(u)||_2 on the base level           */
  double res_max_final;      /* max |f - L(u)| on the base level           */
  double f_l2;               /* ||f||_2 on the base level                  */
  double t_total_ms;         /* wall time of the call                      */
  double t_solve_ms;         /* time of the base-level solve               */
  int n_levels;              /* levels of the hierarchy (1 = base only)    */
  long long cells_per_level[16];
  long long octs_per_level[16];
  int level_iters[16];       /* V-cycles (or sweeps) per refined level     */
  double level_res[16];      /* final relative residual per level          */
  /* per-kernel device time with cfg.profile = 1 (0 otherwise):
   * [0] nonlinear NGS half-sweeps on the base level (FP64 or FP32),
   * [1] FP32 linear Gauss-Seidel half-sweeps on the base level (mixed),
   * [2] FP64 residuals of the mixed form (base and refined levels),
   * [3] nonlinear NGS half-sweeps on the refined level being solved,
   * [4] FP32 linear Gauss-Seidel half-sweeps on the refined level being
   *     solved (mixed), [5] reserved.                                      */
  double kern_ms[6];
  long long kern_launches[6];
  long long kern_cells[6];   /* cells of the levels those launches covered   */
  long long gpu_launches;    /* kernels this call launched (graph nodes included) */
} mgfr_stats;

/* Fill *cfg with the defaults above (omega_m 0.3, fr0_abs 1e-5, n 1, FP64,
 * tol 1e-8, 2+2 sweeps, 100 V-cycles, linear prolongation, step cap 2,
 * max_level 0, refine_count 8, mixed_switch 3e-6, mixed_inner 3,
 * mask_thres 0.99, n_coarse 0, start MGFR_START_ZERO). */
void mgfr_config_default(mgfr_config* cfg);

/* Create a context on CUDA device `device`, working on `cuda_stream`
 * (a cudaStream_t; NULL = default stream).  Validates cfg. */
mgfr_status mgfr_create(mgfr_ctx** out, const mgfr_config* cfg, int device, void* cuda_stream);

/* Replace the configuration of an existing context (validated). */
mgfr_status mgfr_set_config(mgfr_ctx* ctx, const mgfr_config* cfg);

/*
 * Solve on a periodic N^3 grid given the density contrast (Sec. 3.2-3.3).
 *   delta_dev   [N^3] FP64 density contrast rho/rho_bar - 1 (C order).
 *   N           power of two, 8 <= N <= 1024.   box > 0, a > 0.
 *   u_init_dev  [N^3] FP64 initial guess for u, or NULL for u = 0
 *               (the previous-step warm start of Sec. 3.3, step 2); see
 *               cfg.start for the learned start.
 *   fr_out_dev  [N^3] FP64 f_R (required).
 *   acc_out_dev [3][N^3] FP64 a_MG / c^2, or NULL.
 *   u_out_dev   [N^3] FP64 solution u, or NULL.
 *   st          statistics, or NULL.
 * Returns MGFR_E_NOCONVERGE (outputs filled from the last iterate) when the
 * stopping test fails within max_vcycles.
 */
mgfr_status mgfr_solve_density(mgfr_ctx* ctx, const double* delta_dev, int N, double box, double a,
                               const double* u_init_dev, double* fr_out_dev, double* acc_out_dev,
                               double* u_out_dev, mgfr_stats* st);

/*
 * Solve on the refined hierarchy built from particles (Sec. 3.1 and 3.3).
 *   pos_dev      [Np][3] FP64 comoving positions (Mpc/h), wrapped into [0, box).
 *   N_base       base grid size (power of two, 8..1024); cfg.max_level
 *                refinement levels are added where a cell holds more than
 *                cfg.refine_count particles (nearest-grid-point count), the
 *                flags dilated by one cell over the 26 neighbours, each
 *                flagged cell refined into a full oct of 8 daughters.
 *   Masses: adaptive cloud-in-cell (cube of the particle's leaf-cell side),
 *   summed into every coarser cell; delta_l = m N_l^3 / Np - 1 per level.
 *   Solve: base level as mgfr_solve_density, then each refined level in turn
 *   with ghost cells and initial guess prolonged from the converged coarser
 *   level (one-way interface); the coarser solutions are not modified.
 *   u_init_dev   [N_base^3] initial guess of the base level or NULL (cfg.start
 *                as for mgfr_solve_density; the learned start predicts the
 *                base level from its deposited density contrast).
 *   fr_base_out_dev [N_base^3] f_R on the base level, or NULL.
 *   acc_out_dev  [Np][3] a_MG / c^2 at the particles, gathered from the leaf
 *                cells with the mass-assignment weights, or NULL.
 * The hierarchy and the per-level fields stay in the context until the next
 * solve (see mgfr_get_level_*).  Returns MGFR_E_NOCONVERGE if a level missed
 * its tolerance (outputs filled), MGFR_E_INVALID on a non-finite position.
 */
mgfr_status mgfr_solve_particles(mgfr_ctx* ctx, const double* pos_dev, long long Np, int N_base,
                                 double box, double a, const double* u_init_dev,
                                 double* fr_base_out_dev, double* acc_out_dev, mgfr_stats* st);

/*
 * mgfr_solve_particles with the particle arrays in host memory: the same
 * solve (Sec. 3.1 and 3.3) on positions copied to the device by the call, and
 * the force at the particles copied back while it is being gathered (the
 * gather runs in chunks; each chunk's copy overlaps the next chunk's gather).
 *   pos_host     [Np][3] FP64 positions in host memory (page-locked memory,
 *                e.g. from cudaHostAlloc, lets the copies run asynchronously;
 *                pageable memory works but the copies then stage through the
 *                driver).
 *   acc_out_host [Np][3] host memory for a_MG / c^2 at the particles (required).
 *   u_init_dev, fr_base_out_dev: device pointers or NULL, as above.
 * The device copies of the particle arrays are context workspace (grown to
 * Np, kept for the next call).  The call returns when acc_out_host is filled.
 * Errors as mgfr_solve_particles; MGFR_E_INVALID if acc_out_host is NULL.
 */
mgfr_status mgfr_solve_particles_host(mgfr_ctx* ctx, const double* pos_host, long long Np,
                                      int N_base, double box, double a, const double* u_init_dev,
                                      double* fr_base_out_dev, double* acc_out_host,
                                      mgfr_stats* st);

/* Size of level `level` of the last particle solve: octs (0 on the base)
 * and cells (N_base^3 on the base, 8 per oct above). */
mgfr_status mgfr_get_level_info(mgfr_ctx* ctx, int level, long long* n_oct, long long* ncell);

/* Parent key of every oct of refined level `level` >= 1, in storage order:
 * the parent's linear index (I N_{l-1} + J) N_{l-1} + K on level l-1.
 * keys_host: host array of n_oct entries.  Cell c of oct o is its daughter
 * (di, dj, dk) with c = 8 o + 4 di + 2 dj + dk. */
mgfr_status mgfr_get_level_keys(mgfr_ctx* ctx, int level, long long* keys_host);

typedef enum {
  MGFR_FIELD_U = 0,      /* u, [ncell]                                   */
  MGFR_FIELD_FR = 1,     /* f_R, [ncell]                                 */
  MGFR_FIELD_SOURCE = 2, /* f = -alpha Om a^-3 delta, [ncell]            */
  MGFR_FIELD_MASS = 3,   /* deposited mass in particle masses, [ncell]   */
  MGFR_FIELD_ACC = 4,    /* a_MG / c^2: base [3][ncell], refined [ncell][3] */
  MGFR_FIELD_COUNT = 5   /* particles per cell (nearest grid point)      */
} mgfr_field;

/* Copy a per-level field of the last particle solve to host memory
 * (out_host: ncell doubles, 3 ncell for MGFR_FIELD_ACC). */
mgfr_status mgfr_get_level_field(mgfr_ctx* ctx, int level, int what, double* out_host);

/*
 * Effective mass density of the last particle solve (Sec. 2.4, Eqs.
 * (30) and (31)): in units of the mean
 * matter density, delta_eff = delta / 3 - delta R / (24 pi G rho_bar) with
 * delta R = R_bar ((fR_bar / f_R)^{1/(n+1)} - 1) (Eq. (11)), i.e.
 * delta / 3 + Rt / (3 Om a^-3) (1 - e^{-u/(n+1)}), with the model and a of
 * that solve.
 *   mgfr_get_effective_density: per cell of one level, out_dev [ncell] device
 *     FP64, cells in the order of the level fields.
 *   mgfr_effective_mass_pm: on the periodic PM grid of level lpm (N_pm =
 *     N_base 2^lpm <= 1024 per axis), out_dev [N_pm^3] device FP64, C order:
 *     each leaf cell (a cell with no daughters) shares its effective mass
 *     among the PM cells it overlaps in proportion to the overlapping volume
 *     (Sec. 2.4, long-range part), expressed as a density contrast.
 * Both are ordered on the context's stream after the solve; the PM grid sums
 * contributions with FP64 atomics (order-dependent rounding).
 * MGFR_E_INVALID without a particle solve or for an invalid level / lpm.
 */
mgfr_status mgfr_get_effective_density(mgfr_ctx* ctx, int level, double* out_dev);
mgfr_status mgfr_effective_mass_pm(mgfr_ctx* ctx, int lpm, double* out_dev);

/*
 * Gravitational potential of the last particle solve on the periodic PM grid
 * of level lpm (N_pm = N_base 2^lpm, 8 <= N_pm <= 1024 per axis), Sec. 2.4,
 * Eq. (30): lap_x phi = 4 pi G a^2 rho_bar (delta_pm - mean(delta_pm))
 * = (3/2) Omega_m H0^2 a^-1 (delta_pm - mean), with x comoving in Mpc/h,
 * H0 = 100 km/s per Mpc/h, phi in (km/s)^2 and mean(phi) = 0.  delta_pm is
 * each leaf cell's density contrast shared among the PM cells it overlaps by
 * volume (as in mgfr_effective_mass_pm) for
 *   what = MGFR_PM_EFFECTIVE: delta_eff alone (the modified-gravity part, whose
 *          potential is -(c^2/2) f_R up to a constant and discretisation),
 *          MGFR_PM_MATTER: the matter contrast delta (Newtonian gravity),
 *          MGFR_PM_TOTAL: delta + delta_eff (Eq. (30)).
 * The 7-point periodic Poisson problem is solved in FP64 by linear multigrid
 * V-cycles (cfg.n_pre / n_post red-black Gauss-Seidel sweeps, down to 4^3) to
 * ||rhs - lap phi||_2 <= cfg.tol_rel ||rhs||_2 (at most cfg.max_vcycles).
 *   phi_out_dev  [N_pm^3] device FP64, C order (required).
 *   dens_out_dev [N_pm^3] device FP64: delta_pm, or NULL.
 *   st           vcycles, res_l2_init / final (of the scaled right-hand side),
 *                linear_updates, t_solve_ms; or NULL.
 * Workspace (three FP64 arrays of the PM grid and its coarse levels) is held
 * by the context.  MGFR_E_INVALID without a particle solve, for a bad lpm or
 * what; MGFR_E_NOCONVERGE (phi filled) if the tolerance is not reached.
 */
typedef enum { MGFR_PM_EFFECTIVE = 0, MGFR_PM_MATTER = 1, MGFR_PM_TOTAL = 2 } mgfr_pm_what;
mgfr_status mgfr_pm_potential(mgfr_ctx* ctx, int lpm, int what, double* phi_out_dev,
                              double* dens_out_dev, mgfr_stats* st);

/*
 * The force of that potential at the particles: after solving phi as
 * mgfr_pm_potential does, g = -grad_x phi by central differences on the PM
 * grid (periodic) is interpolated to each particle with cloud-in-cell weights
 * of the PM grid (the 8 cells around x N_pm / box - 1/2).  With what =
 * MGFR_PM_TOTAL this is the long-range force of Eq. (30) including the
 * effective mass (Sec. 2.4); MGFR_PM_MATTER gives the Newtonian one.
 *   pos_dev     [Np][3] FP64 comoving positions (Mpc/h), any values (wrapped).
 *   acc_out_dev [Np][3] FP64 -grad_x phi in (km/s)^2 per Mpc/h (the comoving
 *               gradient; the peculiar acceleration is this divided by a).
 * Errors as mgfr_pm_potential; MGFR_E_INVALID without positions or output.
 */
mgfr_status mgfr_pm_accel(mgfr_ctx* ctx, int lpm, int what, const double* pos_dev, long long Np,
                          double* acc_out_dev, mgfr_stats* st);

/*
 * One leapfrog kick-drift step of Np particles on `cuda_stream` (an addition
 * for time-stepped use, Sec. 3.3, step 2: each step's solve starts from the
 * previous step's solution): vel += kick * acc, then pos = wrap(pos + drift *
 * vel) into [0, box).  pos_dev, vel_dev, acc_dev: [Np][3] FP64 device arrays.
 * Asynchronous: returns after the launch.  MGFR_E_INVALID for NULL arrays, Np
 * < 1, box <= 0 or a non-finite kick or drift.
 */
mgfr_status mgfr_kick_drift(double* pos_dev, double* vel_dev, const double* acc_dev, long long Np,
                            double kick, double drift, double box, void* cuda_stream);

/* One independent periodic solve of a batch (Sec. 3.2-3.3 per item). */
typedef struct {
  int N;                     /* power of two, 8..512                          */
  double box, a;             /* box [Mpc/h] and scale factor                  */
  double fr0_abs;            /* |fR_bar0| of this solve (omega_m from cfg)    */
  int n;                     /* Hu-Sawicki exponent                           */
  const double* delta_dev;   /* [N^3] density contrast                        */
  const double* u_init_dev;  /* [N^3] initial guess or NULL (cfg.start)       */
  double* fr_out_dev;        /* [N^3] f_R                                     */
  double* acc_out_dev;       /* [3][N^3] a_MG / c^2, or NULL                  */
  double* u_out_dev;         /* [N^3] the solution u = ln(f_R / fR_bar), or NULL */
} mgfr_batch_item;

/*
 * Solve `nsolves` independent periodic grids of mixed sizes in ONE persistent
 * cooperative kernel launch (replayed from a CUDA graph): every solve runs the
 * mixed-precision form of mgfr_solve_density (FP32 FAS V-cycles, then FP64
 * residual with FP32 linear V-cycles on the Jacobian system) to
 * ||f - L(u)||_2 <= tol_rel ||f||_2.  Solves of different sizes share each
 * V-cycle phase (aligned on grid size); phases are separated by a software
 * grid barrier whose waits are bounded by cfg.max_spins (MGFR_E_TIMEOUT if
 * one gives up; the context stays usable).  per_solve (nullable) receives one
 * mgfr_stats per item, in item order.  The launch shape (threads per block,
 * blocks per SM) comes from mgfr_batch_autotune for the same list of sizes,
 * else 256 x 2.
 */
mgfr_status mgfr_batch_solve(mgfr_ctx* ctx, int nsolves, const mgfr_batch_item* items,
                             mgfr_stats* per_solve);

/* Time the candidate launch shapes (128/256/512 threads x 1/2/4 blocks per
 * SM) on this batch, keep the fastest for batches with the same sizes (and
 * append it to the file named by the environment variable MGFR_TUNE_CACHE,
 * when set).  Runs the batch 9 times; outputs are overwritten. */
mgfr_status mgfr_batch_autotune(mgfr_ctx* ctx, int nsolves, const mgfr_batch_item* items,
                                int* best_threads, int* best_blocks_per_sm);

/*
 * Learned initial guess (an addition to the paper's method: the paper starts
 * from the previous step's u, Sec. 3.3 step 2).  A 4-level 3D U-Net
 * (16/32/64/128 channels, 3^3 kernels, circular padding, BF16 weights and
 * activations, FP32 accumulation) maps per-voxel features (ln(1+delta),
 * log10|fR0| + 5, 1, and the local screening value -(n+1) ln(1 + Om delta/Rt)
 * at a = 1, see mgfr_unet_params) to u; the multigrid then drives the
 * residual to the same tolerance from that start (pass it as u_init or use
 * MGFR_START_LEARNED).  Training and inference run on this library's own
 * tensor-core kernels (tcgen05 with TMEM accumulators for the forward,
 * input-gradient and weight-gradient convolutions).  D (box cells per side) must be
 * a power of two in [32, 512]; the network applies at the cell size it was
 * trained at.
 */
/* (Re)create the network: He-normal convolution weights from `seed`, zero
 * biases and a zero head (the first prediction is u = 0). */
mgfr_status mgfr_unet_init(mgfr_ctx* ctx, unsigned long long seed);
/* One Adam step (learning rate lr) on B samples of D^3: delta_dev [B][D^3],
 * fr0_host [B] (|fR0| per sample, host), u_target_dev [B][D^3]; *loss_out =
 * mean squared error before the step, measured in v = asinh(u / 0.01), the
 * variable the network predicts (u = 0.01 sinh(v)). */
mgfr_status mgfr_unet_train_step(mgfr_ctx* ctx, int B, int D, const double* delta_dev,
                                 const double* fr0_host, const double* u_target_dev, float lr,
                                 double* loss_out);
/* u_out_dev [D^3] = network(delta_dev [D^3], |fR0|). */
mgfr_status mgfr_unet_predict(mgfr_ctx* ctx, int D, const double* delta_dev, double fr0_abs,
                              double* u_out_dev);
/* Copy the FP32 master parameters to (set = 0) or from (set = 1) host memory;
 * *count receives their number (host may be NULL to query it).
 * Network and parameter layout: the input is 16 channels per voxel
 * [ln(1 + delta), log10|fR0| + 5, 1, asinh(u_scr / 0.01) / 5, 0 x 12] with
 * the local screening value u_scr = -(n+1) ln(1 + Om delta / Rt) at a = 1
 * (clamped to [-20, 5]; logarithm arguments floored at 1e-3 and 1e-6).  Encoder levels 0..2:
 * e_l = relu(conv(relu(conv(p_l)))) with 16/32/64 channels, p_0 = input,
 * p_{l+1} = 2^3 average of e_l; bottom: the same with 128 channels on p_3;
 * decoder levels 2..0: d_l = relu(conv(relu(conv([up(d_{l+1}), e_l])))) with
 * 64/32/16 channels (nearest upsampling, upsampled channels first);
 * head v = w . d_0 + c; u = 0.01 sinh(v).  Activations, pre-activation
 * gradients and the convolutions' weight copies are BF16; accumulation,
 * biases, the head and the master parameters are FP32.  The flat parameter
 * vector holds, for the 14 convolutions in the order enc0a, enc0b, enc1a,
 * enc1b, enc2a, enc2b, bottom a, bottom b, dec2a, dec2b, dec1a, dec1b, dec0a,
 * dec0b, W [27][Cin][Cout] then b [Cout]; then the head's 16 weights and its
 * bias (1,466,065 values). */
mgfr_status mgfr_unet_params(mgfr_ctx* ctx, int set, float* host, long long* count);
/* Write the network's FP32 master parameters to the file `path` (8-byte
 * tag "MGFRUNT1", the parameter count as a little-endian int64, then the
 * parameters as little-endian FP32), or read such a file into the context's
 * network (created if needed; the optimiser state restarts).  MGFR_E_INVALID
 * if the file cannot be opened, is truncated or holds another count. */
mgfr_status mgfr_unet_save(mgfr_ctx* ctx, const char* path);
mgfr_status mgfr_unet_load(mgfr_ctx* ctx, const char* path);
/* Gradients of the last training step (same layout as the parameters). */
mgfr_status mgfr_unet_grads(mgfr_ctx* ctx, float* host);
/* One convolution of the network on caller device buffers (NDHWC, channel
 * counts multiples of 16, Cout <= 128, D a power of two >= 4; W [27][Cin][Cout]
 * BF16 with tap = (dx+1)*9 + (dy+1)*3 + (dz+1) for input offset (dx,dy,dz)):
 *   op 0: out (BF16 [B D^3][Cout]) = relu?(conv(x) + bias)   (bias nullable)
 *   op 1: out (FP32 [B D^3][Cin])  = gradient w.r.t. x for output gradient g
 *   op 2: out (FP32 [27][Cin][Cout]) = gradient w.r.t. W, db (FP32 [Cout],
 *         nullable) = gradient w.r.t. the bias; allocates its own scratch.
 * Runs on `stream` and returns when done. */
mgfr_status mgfr_nn_conv3d(int op, int B, int D, int Cin, int Cout, const void* x_bf16,
                           const void* w_bf16, const float* bias, int relu, const void* g_bf16,
                           void* out, float* db, void* stream);

/*
 * FP64 dense-grid solve that allocates nothing (no counterpart in the paper:
 * an addition of this library for callers that cannot allocate device
 * memory, such as code running inside another framework's memory pool or a
 * service whose request path forbids allocation).
 *
 * Same arguments and results as mgfr_solve_density with precision FP64, a
 * zero initial guess and no u output, but without a context: the
 * configuration and the stream are passed in, and all multigrid scratch lives
 * in one fixed device array inside the library (grids up to 64^3; about
 * 7.5 MB that every GPU which loads the library keeps until the process
 * exits).  N must be a power of two in [8, 64]; anything larger returns
 * MGFR_E_INVALID.  cfg->precision and cfg->profile are ignored.
 *   delta_dev [N^3], fr_out_dev [N^3], acc_out_dev [3][N^3] or NULL: caller's
 *   device buffers; cuda_stream: the stream to run on (NULL = default).
 * The first call on a device looks up that device's scratch address; make
 * that first call before any stream capture.  Every call reuses the same
 * scratch and writes it before reading it, so nothing carries over from one
 * call to the next; calls that overlap on the GPU (two streams or two host
 * threads at once) race on the scratch and must be serialised by the caller.
 * The call returns after its results are written.  No cudaMalloc, cudaFree
 * or other allocating routine is called.
 */
mgfr_status mgfr_solve_density_noalloc(const mgfr_config* cfg, const double* delta_dev, int N,
                                       double box, double a, double* fr_out_dev,
                                       double* acc_out_dev, void* cuda_stream, mgfr_stats* st);

/* Text of the last error seen by this context ("" if none). */
const char* mgfr_last_error(const mgfr_ctx* ctx);

/* Release the context and its device workspaces (NULL is accepted). */
void mgfr_destroy(mgfr_ctx* ctx);

/* Library version string. */
const char* mgfr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MGFR_H */
