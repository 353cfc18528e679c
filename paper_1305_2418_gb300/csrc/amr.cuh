// amr.cuh -- refined hierarchy built from particle counts (Puchwein, Baldi &
// Springel 2013, Sec. 3.1) and its one-way level solves (Sec. 3.3, steps
// 9-12, with the mask function of the multigrid on partial levels).
//
// Levels: 0 is the dense periodic base grid (N0^3, C order).  Level l >= 1
// is a list of octs (8 daughters of one refined level-(l-1) cell); cell
// index 8*o + (4 di + 2 dj + dk).  son[l][cell] is the oct at l+1 of a
// refined cell (-1 otherwise).  Octs of level l+1 are stored in the storage
// order of their parents (a stream compaction of level l), so a parent's
// position is given by opos (its level-(l-1)... coordinates) and keys are
// reported as the parent's linear index (I N + J) N + K at level l.
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
  int* nbr = nullptr;                 // [n_oct*6] face-neighbour octs (-1: none)
  double* mass = nullptr;             // [ncell] deposited mass (particle units)
  double *u = nullptr, *E = nullptr, *f = nullptr;  // converged solution, source
  double *w = nullptr, *wE = nullptr, *wf = nullptr, *wold = nullptr;  // work
  float* mask = nullptr;              // [ncell] multigrid mask
  double *ghost = nullptr, *ghostE = nullptr;  // [n_oct*24]
  double* acc = nullptr;              // [ncell*3] (level >= 1)
  long long relaxed = 0;              // cells relaxed in the current level solve
};

struct TreeView {
  int nlev, lg0;
  const int* son[AMR_MAXL];
  const int4* opos[AMR_MAXL];
  const int* nbr[AMR_MAXL];
};

struct AmrWork {
  int N0 = 0, lg0 = 0, nlev = 0;
  double box = 0;
  long long Np = 0;
  AmrLevel L[AMR_MAXL];
  float* dmask[MGFR_MAX_DENSE] = {};  // masks of the dense levels below the base
  int* blocksums = nullptr;
  long long blocksums_cap = 0;
  long long* d_small = nullptr;       // device scalars (totals, error flags)
  double* acc0 = nullptr;             // base force [3][N0^3]
  double* fr0 = nullptr;              // base fR [N0^3]
  long long cap_cells[AMR_MAXL] = {}; // allocated capacity per level (cells)
  long long cap_oct[AMR_MAXL] = {};
};

void amr_free(mgfr_ctx* c);
