// amr.cuh -- refined hierarchy built from particle counts (Puchwein, Baldi &
// Springel 2013, Sec. 3.1) and its one-way level solves (Sec. 3.3, steps
// 9-12, with the mask function of the multigrid on partial levels).
//
// Levels: 0 is the dense periodic base grid (N0^3, C order).  Level l >= 1
// is a list of octs (8 daughters of one refined level-(l-1) cell); cell
// index 8*o + (4 di + 2 dj + dk).  son[l][cell] is the oct at l+1 of a
// refined cell (-1 otherwise).  Octs of level 1 are stored in Morton (Z)
// order of their base-level parents, and octs of level l+1 >= 2 in the
// storage order of their parents (a stream compaction of level l), which
// continues the same Z curve; a parent's position is given by opos (its
// level-(l-1) coordinates) and keys are reported as the parent's linear index
// (I N + J) N + K at level l.
#pragma once
#include "mgfr_internal.cuh"

#define AMR_MAXL 9

struct AmrLevel {
  int lgN = 0;                        // log2 of N_l = N0 << l
  long long n_oct = 0, ncell = 0;
  double h = 0, ih2 = 0;
  int* son = nullptr;                 // [ncell]
  unsigned char* refined = nullptr;   // [ncell]
  int* count = nullptr;               // [ncell]
  int4* opos = nullptr;               // [n_oct] parent coordinates at level l-1
  int* pcell = nullptr;               // [n_oct] parent cell index at level l-1
  int* nbr = nullptr;                 // [n_oct*6] face-neighbour oct, or -(1 + ghost slot)
  long long n_gslot = 0, gcap = 0;    // ghost faces (faces without a neighbouring oct), capacity
  double* mass = nullptr;             // [ncell] deposited mass (particle units)
  double *u = nullptr, *E = nullptr, *f = nullptr;  // converged solution, source
  double *w = nullptr, *wE = nullptr, *wf = nullptr, *wold = nullptr;  // work
  float* mask = nullptr;              // [ncell] multigrid mask
  double *ghost = nullptr, *ghostE = nullptr;  // [n_gslot*4], 4 per ghost face
  double* acc = nullptr;              // [ncell*3] (level >= 1)
  float4* acc32 = nullptr;            // [ncell] FP32 force for the mixed-form gather
  int* pnbr = nullptr;                // [n_oct*6] parent's face-neighbour cells (-1: none)
  // FP32 work arrays (mixed precision phase of the level solves)
  float *w32 = nullptr, *wE32 = nullptr, *wf32 = nullptr, *wold32 = nullptr;
  float* ghost32 = nullptr;           // [n_gslot*4] FP32 ghost u (e^u recomputed)
  unsigned* gface = nullptr;          // [n_gslot] face 6 o + d of each ghost slot
  long long relaxed = 0;              // cells relaxed in the current level solve
  bool ghost_df = false;              // FP64 ghost slots hold double-float pairs (mixed form)
  bool wE_df = false;                 // wE holds e^u as double-float pairs after the solve
  bool force_stale = false;           // FP64 f_R (in w) and acc not yet formed (mixed form)
  unsigned char* act = nullptr;       // [ncell] mask > threshold (coarse level of a solve)
  int* olist = nullptr;               // [n_oct] octs with a relaxed cell (coarse level of a solve)
  long long n_list = 0;               // entries of olist in use
};

struct TreeView {
  int nlev, lg0;
  const int* son[AMR_MAXL];
  const int4* opos[AMR_MAXL];
  const int* nbr[AMR_MAXL];
};

// ---- tree lookups ----------------------------------------------------------
// Cell at level l with level-l coordinates (I,J,K) (wrapped).  Returns the
// cell index at the deepest level m <= l that exists on the path, m in *lev.
static __device__ __forceinline__ long long find_cell(const TreeView& T, int l, long long I, long long J,
                                               long long K, int* lev) {
  const long long Nl = 1LL << (T.lg0 + l);
  I &= Nl - 1;
  J &= Nl - 1;
  K &= Nl - 1;
  long long c = (((I >> l) << T.lg0) + (J >> l) << T.lg0) + (K >> l);
  for (int m = 1; m <= l; ++m) {
    const int o = T.son[m - 1][c];
    if (o < 0) {
      *lev = m - 1;
      return c;
    }
    const int sh = l - m;
    c = 8LL * o + (((I >> sh) & 1) << 2) + (((J >> sh) & 1) << 1) + ((K >> sh) & 1);
  }
  *lev = l;
  return c;
}

static __device__ __forceinline__ void cell_coords(const TreeView& T, int l, long long c, long long* I,
                                            long long* J, long long* K) {
  if (l == 0) {
    const long long M = (1LL << T.lg0) - 1;
    *K = c & M;
    *J = (c >> T.lg0) & M;
    *I = c >> (2 * T.lg0);
    return;
  }
  const int4 p = T.opos[l][c >> 3];
  const int ch = (int)(c & 7);
  *I = 2LL * p.x + ((ch >> 2) & 1);
  *J = 2LL * p.y + ((ch >> 1) & 1);
  *K = 2LL * p.z + (ch & 1);
}


struct AmrWork {
  int N0 = 0, lg0 = 0, nlev = 0;
  double box = 0;
  long long Np = 0;
  AmrLevel L[AMR_MAXL];
  float* dmask[MGFR_MAX_DENSE] = {};  // masks of the dense levels below the base
  unsigned char* dact[MGFR_MAX_DENSE] = {};  // their mask > threshold flags
  // relaxed cells of the masked dense levels (index 0: the base, k >= 1: the
  // dense levels below it), per colour: colour q at [q n/2, q n/2 + dlist_n[k][q])
  int* dlist[MGFR_MAX_DENSE] = {};
  long long dlist_n[MGFR_MAX_DENSE][2] = {};
  int* blocksums = nullptr;
  long long blocksums_cap = 0;
  long long* d_small = nullptr;       // device scalars (totals, error flags)
  double* acc0 = nullptr;             // base force [3][N0^3]
  double* fr0 = nullptr;              // base fR [N0^3]
  double fbar = 0.0, a = 1.0;         // of the last particle solve (deferred level forces)
  double omega_m = 0.3;               // of the last particle solve (effective density)
  int nexp = 1;
  float4* acc0_32 = nullptr;          // base force, FP32 (x, y, z, 0) per cell
  double *pos_dev = nullptr, *acc_dev = nullptr;  // particle arrays of the host-buffer call
  long long pio_cap = 0;                          // their capacity (particles)
  // the deposit's record for the FP32 gather (mixed form): the 8 cells of
  // each particle's cube, and the particles whose cube split over finer cells
  unsigned* rec_idx = nullptr;
  int* split_list = nullptr;                      // per chunk q at q rec_per
  long long* d_split = nullptr;                   // [8] split particles per chunk
  long long rec_cap = 0, rec_per = 0, n_split[8] = {};
  bool rec_on = false;                            // the last deposit recorded
  long long cap_cells[AMR_MAXL] = {}; // allocated capacity per level (cells)
  long long cap_oct[AMR_MAXL] = {};
  // the refined levels of the previous particle solve made with start =
  // MGFR_START_PREVIOUS_ALL: per level, the Morton keys of the octs' parent
  // cells (increasing: the storage order) and the converged u of their cells
  int prev_nlev = 0, prev_N0 = 0;
  double prev_box = 0.0;
  unsigned long long* prev_key[AMR_MAXL] = {};
  double* prev_u[AMR_MAXL] = {};
  long long prev_noct[AMR_MAXL] = {}, prev_cap[AMR_MAXL] = {};
};

// Morton key of cell (i, j, k) (21 bits each): the bits of i, j and k
// interleaved with i's the most significant of each triple, the order in
// which the base level's flag scan visits cells and every level stores octs.
__host__ __device__ inline unsigned long long morton3(unsigned i, unsigned j, unsigned k) {
  unsigned long long m = 0;
  for (int b = 0; b < 21; ++b)
    m |= ((unsigned long long)((i >> b) & 1u) << (3 * b + 2)) |
         ((unsigned long long)((j >> b) & 1u) << (3 * b + 1)) |
         ((unsigned long long)((k >> b) & 1u) << (3 * b));
  return m;
}

// Keep the refined levels of this particle solve for the next one (start =
// MGFR_START_PREVIOUS_ALL), or forget them (any other start).
mgfr_status amr_keep_previous(mgfr_ctx* c, AmrWork* A, bool keep);

void amr_free(mgfr_ctx* c);
// Forget the hierarchy of the last particle solve (its level-0 arrays live in
// the dense workspace, which other solves reuse); the level getters then
// return MGFR_E_INVALID until the next particle solve completes.
void amr_invalidate(mgfr_ctx* c);
// Density contrast of the last particle solve on the periodic PM grid of
// level lpm (what 0: delta_eff, 1: delta, 2: both), written to out_dev
// [N_pm^3] on the context's stream (out_dev NULL: checks only); returns
// log2 N_pm and the model's Omega_m and a of that solve.
mgfr_status amr_density_pm(mgfr_ctx* c, int lpm, int what, double* out_dev, int* lg_pm,
                           double* omega_m, double* a);
TreeView tree_view(const AmrWork* A);
// One-way solve of refined level L >= 1 (amr_solve.cu).
mgfr_status amr_solve_level(mgfr_ctx* c, AmrWork* A, int L, const Model& m, mgfr_stats* st);
void prof_reserve_public(mgfr_ctx* c, size_t pairs);
