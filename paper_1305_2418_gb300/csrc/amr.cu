// amr.cu -- refined hierarchy from particle counts, adaptive cloud-in-cell,
// one-way refined-level solves and the force at the particles
// (Puchwein, Baldi & Springel 2013, Sec. 3.1 and 3.3, eq. modgrav_accel).
//
// Structure build, per level l < lmax: nearest-grid-point counts (int32
// atomics), flags = count > refine_count dilated over the 26 neighbours,
// stream compaction of the flags into the octs of level l+1 (their order
// follows the parents' storage order), parent links and face-neighbour octs.
// Particle cell indices use floor(t 2^l) on t = x N0 / box computed in FP64
// with explicit round-to-nearest operations, so the hierarchy is bit-exact
// with a CPU evaluation of the same expression.
//
// Refined level L is solved with the paper's masked FAS multigrid: the level
// itself (all cells relaxed, ghost layer fixed from level L-1), then every
// coarser tree level and the dense levels below the base, where only cells
// whose mask (1 on level L, averaged down, 0 without daughters) exceeds
// mask_thres are relaxed; the other coarse cells keep the restricted or the
// converged coarse value.  The converged coarse solutions themselves are not
// modified (one-way interface).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "amr.cuh"

namespace {

constexpr int BS = 256;

// ---- particle coordinates ------------------------------------------------
__device__ __forceinline__ double wrap_coord(double x, double inv, double N0) {
  double t = __dmul_rn(x, inv);
  if (t < 0.0 || t >= N0) {
    const double q = floor(__ddiv_rn(t, N0));
    t = __dsub_rn(t, __dmul_rn(N0, q));
    if (t >= N0 || t < 0.0) t = 0.0;
  }
  return t;
}

struct P3 {
  double x, y, z;
};

__device__ __forceinline__ P3 particle_t(const double* __restrict__ pos, long long p, double inv,
                                         double N0) {
  return P3{wrap_coord(pos[3 * p], inv, N0), wrap_coord(pos[3 * p + 1], inv, N0),
            wrap_coord(pos[3 * p + 2], inv, N0)};
}

// ---- tree lookups ----------------------------------------------------------
// Cell at level l with level-l coordinates (I,J,K) (wrapped).  Returns the
// cell index at the deepest level m <= l that exists on the path, m in *lev.
__device__ __forceinline__ long long find_cell(const TreeView& T, int l, long long I, long long J,
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

__device__ __forceinline__ void cell_coords(const TreeView& T, int l, long long c, long long* I,
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

// ---- structure kernels -----------------------------------------------------
__global__ void k_count(const double* __restrict__ pos, long long Np, double inv, double N0, int l,
                        TreeView T, int* __restrict__ count) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Np) return;
  const P3 t = particle_t(pos, p, inv, N0);
  int lev;
  const long long c = find_cell(T, l, (long long)floor(ldexp(t.x, l)),
                                (long long)floor(ldexp(t.y, l)), (long long)floor(ldexp(t.z, l)),
                                &lev);
  if (lev == l) atomicAdd(count + c, 1);
}

// Flag cells holding more than thr particles and their 26 neighbours.
__global__ void k_flag(const int* __restrict__ count, long long ncell, int thr, int l, TreeView T,
                       unsigned char* __restrict__ refined) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell || count[c] <= thr) return;
  long long I, J, K;
  cell_coords(T, l, c, &I, &J, &K);
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int d = -1; d <= 1; ++d) {
        int lev;
        const long long nb = find_cell(T, l, I + a, J + b, K + d, &lev);
        if (lev == l) refined[nb] = 1;
      }
}

// Exclusive scan of the refinement flags -> son indices (three passes).
constexpr int SCAN_BS = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_BS * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_BS) k_scan_count(const unsigned char* __restrict__ flags,
                                                        long long n, int* __restrict__ sums) {
  __shared__ int red[SCAN_BS / 32];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int cnt = 0;
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    const long long i = base + (long long)q * SCAN_BS + threadIdx.x;
    if (i < n) cnt += flags[i] != 0;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < SCAN_BS / 32; ++w) s += red[w];
    sums[blockIdx.x] = s;
  }
}

// single block: exclusive scan of the per-tile sums; total -> *total
__global__ void __launch_bounds__(SCAN_BS) k_scan_sums(int* __restrict__ sums, long long nb,
                                                       long long* __restrict__ total) {
  __shared__ int buf[SCAN_BS];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < nb; base += SCAN_BS) {
    const long long i = base + threadIdx.x;
    const int v = i < nb ? sums[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BS; off <<= 1) {
      const int add = threadIdx.x >= (unsigned)off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nb) sums[i] = (int)(carry + buf[threadIdx.x] - v);
    __syncthreads();
    if (threadIdx.x == SCAN_BS - 1) carry += buf[SCAN_BS - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(SCAN_BS) k_scan_scatter(const unsigned char* __restrict__ flags,
                                                          long long n,
                                                          const int* __restrict__ offs,
                                                          int* __restrict__ son) {
  __shared__ int buf[SCAN_BS];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int run = offs[blockIdx.x];
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    const long long i = base + (long long)q * SCAN_BS + threadIdx.x;
    const int v = (i < n && flags[i]) ? 1 : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BS; off <<= 1) {
      const int add = threadIdx.x >= (unsigned)off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) son[i] = v ? run + buf[threadIdx.x] - 1 : -1;
    const int tot = buf[SCAN_BS - 1];
    __syncthreads();
    run += tot;
  }
}

__global__ void k_make_octs(const int* __restrict__ son, long long ncell, int l, TreeView T,
                            int* __restrict__ pcell, int4* __restrict__ opos) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int o = son[c];
  if (o < 0) return;
  long long I, J, K;
  cell_coords(T, l, c, &I, &J, &K);
  pcell[o] = (int)c;
  opos[o] = make_int4((int)I, (int)J, (int)K, 0);
}

// face-neighbour octs of the octs of level l (their parents live on l-1)
__global__ void k_oct_nbrs(long long n_oct, int l, TreeView T, int* __restrict__ nbr) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= n_oct) return;
  const int4 p = T.opos[l][o];
  const int dd[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int d = 0; d < 6; ++d) {
    int lev;
    const long long q = find_cell(T, l - 1, p.x + dd[d][0], p.y + dd[d][1], p.z + dd[d][2], &lev);
    nbr[6 * o + d] = lev == l - 1 ? T.son[l - 1][q] : -1;
  }
}

// ---- adaptive cloud-in-cell (Sec. 3.1) -------------------------------------
// The particle is a cube with the side of its leaf cell (level lam).  Its 8
// level-lam pieces go to the leaf cell holding each piece; a piece whose cell
// is refined is split among the daughters (explicit stack); a piece whose
// cell does not exist goes to the deepest existing ancestor, a leaf.
struct LevelPtrs {
  double* a[AMR_MAXL];  // per-level array (mass for deposit)
};

struct GatherPtrs {
  const double* acc[AMR_MAXL];  // level 0: [3][N0^3]; l >= 1: [ncell][3]
  long long n0;
};

template <bool GATHER>
__device__ __forceinline__ void touch(int lev, long long c, double w, LevelPtrs& D,
                                      const GatherPtrs& G, double* out) {
  if (GATHER) {
    if (lev == 0) {
      out[0] += w * G.acc[0][c];
      out[1] += w * G.acc[0][G.n0 + c];
      out[2] += w * G.acc[0][2 * G.n0 + c];
    } else {
      out[0] += w * G.acc[lev][3 * c];
      out[1] += w * G.acc[lev][3 * c + 1];
      out[2] += w * G.acc[lev][3 * c + 2];
    }
  } else {
    atomicAdd(D.a[lev] + c, w);
  }
}

struct StackEnt {
  double lo[3], hi[3];  // interval in level-`l` units
  long long c;          // refined cell index at level l
  int l;
  int pad;
};

template <bool GATHER>
__device__ void visit_particle(const TreeView& T, const P3& t, LevelPtrs& D, const GatherPtrs& G,
                               double* out, unsigned long long* err) {
  // leaf level of the particle
  int lam = 0;
  {
    long long c = (((long long)floor(t.x) << T.lg0) + (long long)floor(t.y) << T.lg0) +
                  (long long)floor(t.z);
    for (int m = 1; m < T.nlev; ++m) {
      const int o = T.son[m - 1][c];
      if (o < 0) break;
      const long long I = (long long)floor(ldexp(t.x, m)), J = (long long)floor(ldexp(t.y, m)),
                      K = (long long)floor(ldexp(t.z, m));
      c = 8LL * o + ((I & 1) << 2) + ((J & 1) << 1) + (K & 1);
      lam = m;
    }
  }
  const double tl[3] = {ldexp(t.x, lam) - 0.5, ldexp(t.y, lam) - 0.5, ldexp(t.z, lam) - 0.5};
  long long i0[3];
  double w1[3];
  for (int a = 0; a < 3; ++a) {
    i0[a] = (long long)floor(tl[a]);
    w1[a] = tl[a] - (double)i0[a];
  }
  StackEnt st[48];
  int sp = 0;
  for (int q = 0; q < 8; ++q) {
    const int ba = (q >> 2) & 1, bb = (q >> 1) & 1, bc = q & 1;
    const double w = (ba ? w1[0] : 1.0 - w1[0]) * (bb ? w1[1] : 1.0 - w1[1]) *
                     (bc ? w1[2] : 1.0 - w1[2]);
    if (!(w > 0.0)) continue;
    int lev;
    const long long c = find_cell(T, lam, i0[0] + ba, i0[1] + bb, i0[2] + bc, &lev);
    const bool refined = lev == lam && lam + 1 < T.nlev && T.son[lam][c] >= 0;
    if (!refined) {
      touch<GATHER>(lev, c, w, D, G, out);
      continue;
    }
    if (sp >= 48) {
      atomicOr(err, 1ULL);
      continue;
    }
    StackEnt& e = st[sp++];
    const long long P[3] = {i0[0] + ba, i0[1] + bb, i0[2] + bc};
    const int bits[3] = {ba, bb, bc};
    for (int a = 0; a < 3; ++a) {
      // the cube is [tl, tl + 1] in level-lam units; clip to the cell [P, P+1]
      e.lo[a] = bits[a] ? (double)P[a] : tl[a];
      e.hi[a] = bits[a] ? tl[a] + 1.0 : (double)P[a] + 1.0;
    }
    e.c = c;
    e.l = lam;
  }
  // split refined pieces among daughters (volumes in level-lam units)
  while (sp > 0) {
    const StackEnt e = st[--sp];
    const int o = T.son[e.l][e.c];
    const int lc = e.l + 1;
    const double scale = ldexp(1.0, -3 * (lc - lam));  // daughter-unit volume -> cube fraction
    long long I0[3];
    double lo2[3], hi2[3];
    for (int a = 0; a < 3; ++a) {
      lo2[a] = 2.0 * e.lo[a];
      hi2[a] = 2.0 * e.hi[a];
      I0[a] = 2 * (long long)floor(e.lo[a] + 0.0);  // parent coordinate * 2
    }
    // parent cell coordinate: floor of the interval start (interval lies in it)
    for (int ch = 0; ch < 8; ++ch) {
      const int b[3] = {(ch >> 2) & 1, (ch >> 1) & 1, ch & 1};
      double lo[3], hi[3];
      bool empty = false;
      for (int a = 0; a < 3; ++a) {
        const double c0 = (double)(I0[a] + b[a]);
        lo[a] = fmax(lo2[a], c0);
        hi[a] = fmin(hi2[a], c0 + 1.0);
        if (!(hi[a] > lo[a])) empty = true;
      }
      if (empty) continue;
      const long long cc = 8LL * o + ch;
      const bool ref = lc + 1 < T.nlev && T.son[lc][cc] >= 0;
      if (!ref) {
        const double vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]) * scale;
        touch<GATHER>(lc, cc, vol, D, G, out);
      } else if (sp < 48) {
        StackEnt& n = st[sp++];
        for (int a = 0; a < 3; ++a) {
          n.lo[a] = lo[a];
          n.hi[a] = hi[a];
        }
        n.c = cc;
        n.l = lc;
      } else {
        atomicOr(err, 1ULL);
      }
    }
  }
}

__global__ void k_deposit(const double* __restrict__ pos, long long Np, double inv, double N0,
                          TreeView T, LevelPtrs D, unsigned long long* err) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Np) return;
  const P3 t = particle_t(pos, p, inv, N0);
  GatherPtrs G{};
  visit_particle<false>(T, t, D, G, nullptr, err);
}

__global__ void k_gather(const double* __restrict__ pos, long long Np, double inv, double N0,
                         TreeView T, GatherPtrs G, double* __restrict__ acc,
                         unsigned long long* err) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Np) return;
  const P3 t = particle_t(pos, p, inv, N0);
  LevelPtrs D{};
  double out[3] = {0.0, 0.0, 0.0};
  visit_particle<true>(T, t, D, G, out, err);
  acc[3 * p] = out[0];
  acc[3 * p + 1] = out[1];
  acc[3 * p + 2] = out[2];
}

// coarse cell mass = sum of its daughters (Sec. 3.1)
__global__ void k_mass_up(const double* __restrict__ mchild, long long n_oct,
                          const int* __restrict__ pcell, double* __restrict__ mparent) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= n_oct) return;
  double s = 0.0;
  for (int q = 0; q < 8; ++q) s += mchild[8 * o + q];
  mparent[pcell[o]] = s;
}

__global__ void k_source_lvl(const double* __restrict__ mass, long long n, double scale, double src,
                             double* __restrict__ f) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) f[c] = src * (mass[c] * scale - 1.0);
}

__global__ void k_nan_check(const double* __restrict__ x, long long n,
                            unsigned long long* __restrict__ err) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicOr(err, 2ULL);
}

// ---- refined-level operators -----------------------------------------------
__device__ __forceinline__ double nl_s(double u, double E, const Model& m) {
  return m.n == 1 ? rsqrt(E) : exp(-u * m.inv_np1);
}

// value of the neighbour of cell (o, ch) in direction d: same oct, the
// neighbouring oct, or the ghost slot (ghost != nullptr).
struct OctNb {
  double u, E;
};

__device__ __forceinline__ OctNb oct_nb(const double* __restrict__ u, const double* __restrict__ E,
                                        const int* __restrict__ nbr,
                                        const double* __restrict__ ghost,
                                        const double* __restrict__ ghostE, long long o, int ch,
                                        int d) {
  const int ax = d >> 1, plus = d & 1;
  const int bit = (ch >> (2 - ax)) & 1;
  const int chn = ch ^ (1 << (2 - ax));
  if (bit != plus) {  // inside the oct
    const long long q = 8 * o + chn;
    return OctNb{u[q], E[q]};
  }
  const int no = nbr[6 * o + d];
  if (no >= 0) {
    const long long q = 8LL * no + chn;
    return OctNb{u[q], E[q]};
  }
  // ghost slot: face d, index from the two tangential bits
  const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
  const int qi = (((ch >> (2 - t1)) & 1) << 1) | ((ch >> (2 - t2)) & 1);
  const long long g = 24 * o + 4 * d + qi;
  return OctNb{ghost[g], ghostE[g]};
}

// red (colour 0) cells of an oct: children with even di+dj+dk
__constant__ int kColourChild[2][4] = {{0, 3, 5, 6}, {1, 2, 4, 7}};

__global__ void __launch_bounds__(BS) k_oct_sweep(double* __restrict__ u, double* __restrict__ E,
                                                  const double* __restrict__ f,
                                                  const int* __restrict__ nbr,
                                                  const double* __restrict__ ghost,
                                                  const double* __restrict__ ghostE,
                                                  const float* __restrict__ mask, float mthr,
                                                  long long n_oct, int colour, Model m, double ih2,
                                                  double cap) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 4 * n_oct) return;
  const long long o = t >> 2;
  const int ch = kColourChild[colour][t & 3];
  const long long c = 8 * o + ch;
  if (mask && !(mask[c] > mthr)) return;
  const double uc = u[c], Ec = E[c];
  double sbd = 0.0, sd = 0.0, sb = 0.0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const OctNb nb = oct_nb(u, E, nbr, ghost, ghostE, o, ch, d);
    const double b = 0.5 * (nb.E + Ec), du = nb.u - uc;
    sbd = fma(b, du, sbd);
    sd += du;
    sb += b;
  }
  const double s = nl_s(uc, Ec, m);
  const double L = sbd * ih2 + m.aRt * (1.0 - s);
  const double dL = (0.5 * Ec * sd - sb) * ih2 + m.aRt_np1 * s;
  double step = (L - f[c]) / dL;
  step = fmin(fmax(step, -cap), cap);
  const double un = uc - step;
  u[c] = un;
  E[c] = exp(un);
}

__device__ __forceinline__ double oct_L(const double* __restrict__ u, const double* __restrict__ E,
                                        const int* __restrict__ nbr,
                                        const double* __restrict__ ghost,
                                        const double* __restrict__ ghostE, long long o, int ch,
                                        const Model& m, double ih2) {
  const long long c = 8 * o + ch;
  const double uc = u[c], Ec = E[c];
  double sbd = 0.0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const OctNb nb = oct_nb(u, E, nbr, ghost, ghostE, o, ch, d);
    sbd = fma(0.5 * (nb.E + Ec), nb.u - uc, sbd);
  }
  return sbd * ih2 + m.aRt * (1.0 - nl_s(uc, Ec, m));
}

// residual norm over all cells of a level (ghost layer fixed)
__global__ void __launch_bounds__(BS) k_oct_norm(const double* __restrict__ u,
                                                 const double* __restrict__ E,
                                                 const double* __restrict__ f,
                                                 const int* __restrict__ nbr,
                                                 const double* __restrict__ ghost,
                                                 const double* __restrict__ ghostE,
                                                 long long ncell, Model m, double ih2,
                                                 double* __restrict__ partials) {
  double ss = 0.0, mx = 0.0, fs = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const double r = f[c] - oct_L(u, E, nbr, ghost, ghostE, c >> 3, (int)(c & 7), m, ih2);
    ss = fma(r, r, ss);
    mx = fmax(mx, fabs(r));
    fs = fma(f[c], f[c], fs);
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

// Restrict oct level k to its parents on level k-1: u average, masked
// residual average (cells with mask <= mthr contribute 0), saved old value.
__global__ void __launch_bounds__(BS) k_oct_restrict(
    const double* __restrict__ u, const double* __restrict__ E, const double* __restrict__ f,
    const int* __restrict__ nbr, const double* __restrict__ ghost,
    const double* __restrict__ ghostE, const float* __restrict__ mask, float mthr,
    long long n_oct, const int* __restrict__ pcell, Model m, double ih2, double* __restrict__ uc,
    double* __restrict__ Ec, double* __restrict__ ucold, double* __restrict__ fc) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= n_oct) return;
  double su = 0.0, sr = 0.0;
  for (int ch = 0; ch < 8; ++ch) {
    const long long c = 8 * o + ch;
    su += u[c];
    if (!mask || mask[c] > mthr) sr += f[c] - oct_L(u, E, nbr, ghost, ghostE, o, ch, m, ih2);
  }
  const int p = pcell[o];
  const double um = 0.125 * su;
  uc[p] = um;
  ucold[p] = um;
  Ec[p] = exp(um);
  fc[p] = 0.125 * sr;
}

// FAS right-hand side on a coarse oct level: f += L(u) at relaxed cells.
__global__ void __launch_bounds__(BS) k_oct_fas(const double* __restrict__ u,
                                                const double* __restrict__ E,
                                                double* __restrict__ f,
                                                const int* __restrict__ nbr,
                                                const float* __restrict__ mask, float mthr,
                                                long long ncell, Model m, double ih2) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell || !(mask[c] > mthr)) return;
  f[c] += oct_L(u, E, nbr, nullptr, nullptr, c >> 3, (int)(c & 7), m, ih2);
}

// parent value of level-l cell (I,J,K) with the linear reconstruction from
// the parent's neighbours (a component is 0 where a neighbour is missing);
// `val` reads the parent level's field (a difference of two arrays for
// corrections).
template <class F>
__device__ __forceinline__ double prolong_value(const TreeView& T, int l, long long I, long long J,
                                                long long K, long long pc, int linear, F val) {
  double v = val(pc);
  if (!linear) return v;
  const long long P[3] = {I >> 1, J >> 1, K >> 1};
  const long long C[3] = {I, J, K};
  for (int ax = 0; ax < 3; ++ax) {
    long long Qp[3] = {P[0], P[1], P[2]}, Qm[3] = {P[0], P[1], P[2]};
    Qp[ax] += 1;
    Qm[ax] -= 1;
    int lp, lm;
    const long long cp = find_cell(T, l - 1, Qp[0], Qp[1], Qp[2], &lp);
    const long long cm = find_cell(T, l - 1, Qm[0], Qm[1], Qm[2], &lm);
    if (lp != l - 1 || lm != l - 1) continue;
    const double s = (C[ax] & 1) ? 0.125 : -0.125;
    v += s * (val(cp) - val(cm));
  }
  return v;
}

// Initial guess of level l from the converged level l-1 (Sec. 3.3, step 9).
__global__ void k_oct_init(long long ncell, int l, TreeView T, const int* __restrict__ pcell,
                           const double* __restrict__ up, int linear, double* __restrict__ u,
                           double* __restrict__ E) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  long long I, J, K;
  cell_coords(T, l, c, &I, &J, &K);
  const double v = prolong_value(T, l, I, J, K, pcell[c >> 3], linear,
                                 [&](long long q) { return up[q]; });
  u[c] = v;
  E[c] = exp(v);
}

// Ghost values of level l: for every oct face without a neighbouring oct, the
// 4 level-l cells across it take the linear reconstruction of their parent
// (level l-1, converged) -- fixed during the level solve.
__global__ void k_ghosts(long long n_oct, int l, TreeView T, const int* __restrict__ nbr,
                         const double* __restrict__ up, int linear, double* __restrict__ ghost,
                         double* __restrict__ ghostE) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 24 * n_oct) return;
  const long long o = t / 24;
  const int d = (int)((t % 24) >> 2), qi = (int)(t & 3);
  if (nbr[6 * o + d] >= 0) return;
  const int ax = d >> 1, plus = d & 1;
  const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
  int b[3];
  b[ax] = plus;  // the oct's cell on that face has this bit
  b[t1] = (qi >> 1) & 1;
  b[t2] = qi & 1;
  const int4 p = T.opos[l][o];
  long long C[3] = {2LL * p.x + b[0], 2LL * p.y + b[1], 2LL * p.z + b[2]};
  C[ax] += plus ? 1 : -1;
  const long long Nl = 1LL << (T.lg0 + l);
  for (int a = 0; a < 3; ++a) C[a] &= Nl - 1;
  int lev;
  const long long pc = find_cell(T, l - 1, C[0] >> 1, C[1] >> 1, C[2] >> 1, &lev);
  double v = 0.0;
  if (lev == l - 1)
    v = prolong_value(T, l, C[0], C[1], C[2], pc, linear, [&](long long q) { return up[q]; });
  ghost[t] = v;
  ghostE[t] = exp(v);
}

// Correction of relaxed level-l cells from the coarse level l-1:
// u += P(uc - ucold) (eq. fine_correction).
__global__ void k_oct_prolong(long long ncell, int l, TreeView T, const int* __restrict__ pcell,
                              const double* __restrict__ uc, const double* __restrict__ ucold,
                              const float* __restrict__ mask, float mthr, int linear,
                              double* __restrict__ u, double* __restrict__ E) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  if (mask && !(mask[c] > mthr)) return;
  long long I, J, K;
  cell_coords(T, l, c, &I, &J, &K);
  const double v = prolong_value(T, l, I, J, K, pcell[c >> 3], linear,
                                 [&](long long q) { return uc[q] - ucold[q]; });
  const double un = u[c] + v;
  u[c] = un;
  E[c] = exp(un);
}

// mask of level l-1 cells from their daughters: average of the 8 masks for
// cells with daughters (cells without daughters keep 0).
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
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (1LL << (3 * lgc))) return;
  const int K = (int)(t & (Nc - 1)), J = (int)((t >> lgc) & (Nc - 1)), I = (int)(t >> (2 * lgc));
  float s = 0.f;
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q >> 2), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q & 1);
    s += mf[((((long long)i << lgf) + j) << lgf) + k];
  }
  mc[t] = 0.125f * s;
}

__global__ void k_fill_f(float* __restrict__ x, long long n, float v) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
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

// f_R and a_MG/c^2 on a refined level (central differences, ghosts at edges)
__global__ void k_oct_force(const double* __restrict__ E, const int* __restrict__ nbr,
                            const double* __restrict__ ghostE, long long ncell, double fbar,
                            double g_scale, double* __restrict__ fr, double* __restrict__ acc) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const long long o = c >> 3;
  const int ch = (int)(c & 7);
  fr[c] = fbar * E[c];
  for (int ax = 0; ax < 3; ++ax) {
    const OctNb m = oct_nb(E, E, nbr, ghostE, ghostE, o, ch, 2 * ax);
    const OctNb p = oct_nb(E, E, nbr, ghostE, ghostE, o, ch, 2 * ax + 1);
    acc[3 * c + ax] = g_scale * (p.E - m.E);
  }
}

}  // namespace

// ============================================================================
// host side
// ============================================================================

static AmrWork* W(mgfr_ctx* c) { return (AmrWork*)c->amr; }

static void free_level(AmrLevel& L) {
  void* ps[] = {L.son, L.refined, L.count, L.opos, L.pcell, L.nbr, L.mass, L.w, L.wE, L.wf,
                L.wold, L.mask, L.ghost, L.ghostE, L.acc};
  for (void* p : ps)
    if (p) cudaFree(p);
  // u, E, f of level >= 1 are owned here too
}

void amr_free(mgfr_ctx* c) {
  AmrWork* A = W(c);
  if (!A) return;
  for (int l = 0; l < AMR_MAXL; ++l) {
    free_level(A->L[l]);
    if (l > 0) {
      if (A->L[l].u) cudaFree(A->L[l].u);
      if (A->L[l].E) cudaFree(A->L[l].E);
      if (A->L[l].f) cudaFree(A->L[l].f);
    }
  }
  for (int l = 0; l < MGFR_MAX_DENSE; ++l)
    if (A->dmask[l]) cudaFree(A->dmask[l]);
  if (A->blocksums) cudaFree(A->blocksums);
  if (A->d_small) cudaFree(A->d_small);
  if (A->acc0) cudaFree(A->acc0);
  if (A->fr0) cudaFree(A->fr0);
  delete A;
  c->amr = nullptr;
}

static TreeView tree_view(const AmrWork* A) {
  TreeView T{};
  T.nlev = A->nlev;
  T.lg0 = A->lg0;
  for (int l = 0; l < AMR_MAXL; ++l) {
    T.son[l] = A->L[l].son;
    T.opos[l] = A->L[l].opos;
    T.nbr[l] = A->L[l].nbr;
  }
  return T;
}

template <class T>
static mgfr_status grow(mgfr_ctx* c, T** p, long long n, long long* cap_unused = nullptr) {
  (void)cap_unused;
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (n <= 0) return MGFR_OK;
  MG_CK(c, cudaMalloc((void**)p, sizeof(T) * (size_t)n));
  return MGFR_OK;
}

#define TRY(x)                               \
  do {                                       \
    mgfr_status s_ = (x);                    \
    if (s_ != MGFR_OK) return s_;            \
  } while (0)

// Allocate the per-cell arrays of level l (ncell cells, n_oct octs).
static mgfr_status alloc_level(mgfr_ctx* c, AmrWork* A, int l) {
  AmrLevel& L = A->L[l];
  const long long n = L.ncell, no = L.n_oct;
  if (A->cap_cells[l] == n && A->cap_oct[l] == no && L.son) return MGFR_OK;
  free_level(L);
  if (l > 0) {
    if (L.u) cudaFree(L.u);
    if (L.E) cudaFree(L.E);
    if (L.f) cudaFree(L.f);
    L.u = L.E = L.f = nullptr;
  }
  L.son = nullptr; L.refined = nullptr; L.count = nullptr; L.opos = nullptr; L.pcell = nullptr;
  L.nbr = nullptr; L.mass = nullptr; L.w = nullptr; L.wE = nullptr; L.wf = nullptr;
  L.wold = nullptr; L.mask = nullptr; L.ghost = nullptr; L.ghostE = nullptr; L.acc = nullptr;
  TRY(grow(c, &L.son, n));
  TRY(grow(c, &L.refined, n));
  TRY(grow(c, &L.count, n));
  TRY(grow(c, &L.mass, n));
  TRY(grow(c, &L.w, n));
  TRY(grow(c, &L.wE, n));
  TRY(grow(c, &L.wf, n));
  TRY(grow(c, &L.wold, n));
  TRY(grow(c, &L.mask, n));
  if (l > 0) {
    TRY(grow(c, &L.opos, no));
    TRY(grow(c, &L.pcell, no));
    TRY(grow(c, &L.nbr, 6 * no));
    TRY(grow(c, &L.ghost, 24 * no));
    TRY(grow(c, &L.ghostE, 24 * no));
    TRY(grow(c, &L.acc, 3 * n));
    TRY(grow(c, &L.u, n));
    TRY(grow(c, &L.E, n));
    TRY(grow(c, &L.f, n));
  }
  A->cap_cells[l] = n;
  A->cap_oct[l] = no;
  return MGFR_OK;
}

static mgfr_status scan_flags(mgfr_ctx* c, AmrWork* A, const unsigned char* flags, long long n,
                              int* son, long long* total) {
  const long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb > A->blocksums_cap) {
    if (A->blocksums) cudaFree(A->blocksums);
    A->blocksums = nullptr;
    MG_CK(c, cudaMalloc(&A->blocksums, sizeof(int) * (size_t)nb));
    A->blocksums_cap = nb;
  }
  k_scan_count<<<(unsigned)nb, SCAN_BS, 0, c->s>>>(flags, n, A->blocksums);
  k_scan_sums<<<1, SCAN_BS, 0, c->s>>>(A->blocksums, nb, A->d_small);
  k_scan_scatter<<<(unsigned)nb, SCAN_BS, 0, c->s>>>(flags, n, A->blocksums, son);
  c->launches += 3;
  MG_CK(c, cudaMemcpyAsync(total, A->d_small, sizeof(long long), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  return MGFR_OK;
}

// Counts, flags, compaction and oct tables for every level (Sec. 3.1).
static mgfr_status build_structure(mgfr_ctx* c, AmrWork* A, const double* pos) {
  const mgfr_config& g = c->cfg;
  const double inv = (double)A->N0 / A->box, N0d = (double)A->N0;
  A->nlev = 1;
  A->L[0].ncell = 1LL << (3 * A->lg0);
  A->L[0].n_oct = 0;
  TRY(alloc_level(c, A, 0));
  for (int l = 0;; ++l) {
    AmrLevel& L = A->L[l];
    L.lgN = A->lg0 + l;
    L.h = A->box / (double)(1LL << L.lgN);
    L.ih2 = 1.0 / (L.h * L.h);
    MG_CK(c, cudaMemsetAsync(L.count, 0, sizeof(int) * (size_t)L.ncell, c->s));
    MG_CK(c, cudaMemsetAsync(L.refined, 0, (size_t)L.ncell, c->s));
    TreeView T = tree_view(A);
    if (A->Np > 0)
      k_count<<<nblocks(A->Np, BS), BS, 0, c->s>>>(pos, A->Np, inv, N0d, l, T, L.count);
    c->launches += 1;
    if (l >= g.max_level || l + 1 >= AMR_MAXL) {
      MG_CK(c, cudaMemsetAsync(L.son, 0xff, sizeof(int) * (size_t)L.ncell, c->s));
      break;
    }
    k_flag<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.count, L.ncell, g.refine_count, l, T,
                                                  L.refined);
    c->launches += 1;
    long long nref = 0;
    TRY(scan_flags(c, A, L.refined, L.ncell, L.son, &nref));
    if (nref == 0) break;
    AmrLevel& N = A->L[l + 1];
    N.n_oct = nref;
    N.ncell = 8 * nref;
    TRY(alloc_level(c, A, l + 1));
    A->nlev = l + 2;
    T = tree_view(A);
    k_make_octs<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.son, L.ncell, l, T, N.pcell, N.opos);
    T = tree_view(A);
    k_oct_nbrs<<<nblocks(N.n_oct, BS), BS, 0, c->s>>>(N.n_oct, l + 1, T, N.nbr);
    c->launches += 2;
  }
  // the deepest level has no sons
  AmrLevel& D = A->L[A->nlev - 1];
  MG_CK(c, cudaMemsetAsync(D.son, 0xff, sizeof(int) * (size_t)D.ncell, c->s));
  MG_CK(c, cudaMemsetAsync(D.refined, 0, (size_t)D.ncell, c->s));
  return MGFR_OK;
}

static mgfr_status deposit(mgfr_ctx* c, AmrWork* A, const double* pos) {
  const double inv = (double)A->N0 / A->box, N0d = (double)A->N0;
  LevelPtrs D{};
  for (int l = 0; l < A->nlev; ++l) {
    MG_CK(c, cudaMemsetAsync(A->L[l].mass, 0, sizeof(double) * (size_t)A->L[l].ncell, c->s));
    D.a[l] = A->L[l].mass;
  }
  TreeView T = tree_view(A);
  k_deposit<<<nblocks(A->Np, BS), BS, 0, c->s>>>(pos, A->Np, inv, N0d, T, D,
                                                 (unsigned long long*)(A->d_small + 1));
  c->launches += 1;
  for (int l = A->nlev - 1; l >= 1; --l) {
    k_mass_up<<<nblocks(A->L[l].n_oct, BS), BS, 0, c->s>>>(A->L[l].mass, A->L[l].n_oct,
                                                           A->L[l].pcell, A->L[l - 1].mass);
    c->launches += 1;
  }
  return MGFR_OK;
}

// ---- level solves -------------------------------------------------------------
struct AmrSolveCtx {
  mgfr_ctx* c;
  AmrWork* A;
  Model m;
  int L;          // level being solved
  float mthr;
  long long updates;
};

// Dense view of the base level's work arrays (mask included).
static DenseLevel base_work(AmrWork* A, const DenseHier& H) {
  DenseLevel D = H.L[0];
  AmrLevel& B = A->L[0];
  D.u = B.w;
  D.E = B.wE;
  D.f = B.wf;
  D.uold = B.wold;
  D.mask = B.mask;
  return D;
}

static DenseLevel sub_work(AmrWork* A, const DenseHier& H, int k, float mthr) {
  DenseLevel D = H.L[k];
  D.mask = A->dmask[k];
  D.mthr = mthr;
  return D;
}

void prof_reserve_public(mgfr_ctx* c, size_t pairs);

static void relax_tree(AmrSolveCtx& S, int l, int sweeps) {
  mgfr_ctx* c = S.c;
  AmrWork* A = S.A;
  const mgfr_config& g = c->cfg;
  AmrLevel& L = A->L[l];
  for (int s = 0; s < sweeps; ++s) {
    for (int col = 0; col < 2; ++col) {
      if (l >= 1) {
        if (l == S.L) prof_begin(c, 3, L.ncell);
        k_oct_sweep<<<nblocks(4 * L.n_oct, BS), BS, 0, c->s>>>(
            L.w, L.wE, L.wf, L.nbr, L.ghost, L.ghostE, l == S.L ? nullptr : L.mask, S.mthr,
            L.n_oct, col, S.m, L.ih2, g.step_cap);
        if (l == S.L) prof_end(c);
      } else {
        DenseLevel D = base_work(A, c->dh);
        D.mthr = S.mthr;
        f64::sweep(D, S.m, col, g.step_cap, c->s);
      }
      c->launches += 1;
    }
    S.updates += L.relaxed;
  }
}

static void vcycle_dense_masked(AmrSolveCtx& S, int k);

// Masked FAS V-cycle of the level-S.L solve, entered at tree level l >= 0.
static void vcycle_tree(AmrSolveCtx& S, int l) {
  mgfr_ctx* c = S.c;
  AmrWork* A = S.A;
  const mgfr_config& g = c->cfg;
  AmrLevel& F = A->L[l];
  relax_tree(S, l, g.n_pre);
  if (l >= 1) {
    AmrLevel& P = A->L[l - 1];
    k_oct_restrict<<<nblocks(F.n_oct, BS), BS, 0, c->s>>>(
        F.w, F.wE, F.wf, F.nbr, F.ghost, F.ghostE, l == S.L ? nullptr : F.mask, S.mthr, F.n_oct,
        F.pcell, S.m, F.ih2, P.w, P.wE, P.wold, P.wf);
    if (l - 1 >= 1) {
      k_oct_fas<<<nblocks(P.ncell, BS), BS, 0, c->s>>>(P.w, P.wE, P.wf, P.nbr, P.mask, S.mthr,
                                                       P.ncell, S.m, P.ih2);
    } else {
      DenseLevel D = base_work(A, c->dh);
      D.mthr = S.mthr;
      f64::fas_rhs(D, S.m, c->s);
    }
    c->launches += 2;
    vcycle_tree(S, l - 1);
    TreeView T = tree_view(A);
    k_oct_prolong<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(
        F.ncell, l, T, F.pcell, P.w, P.wold, l == S.L ? nullptr : F.mask, S.mthr,
        g.prolong_linear, F.w, F.wE);
    c->launches += 1;
  } else {
    // base level -> dense levels below it
    DenseHier& H = c->dh;
    DenseLevel B = base_work(A, H);
    B.mthr = S.mthr;
    DenseLevel C1 = sub_work(A, H, 1, S.mthr);
    f64::restrict_resid(B, C1, S.m, c->s);
    f64::fas_rhs(C1, S.m, c->s);
    c->launches += 2;
    vcycle_dense_masked(S, 1);
    f64::prolong_corr(B, C1, g.prolong_linear, c->s);
    c->launches += 1;
  }
  relax_tree(S, l, g.n_post);
}

static void vcycle_dense_masked(AmrSolveCtx& S, int k) {
  mgfr_ctx* c = S.c;
  DenseHier& H = c->dh;
  const mgfr_config& g = c->cfg;
  DenseLevel F = sub_work(S.A, H, k, S.mthr);
  if (F.N <= 4) {
    f64::coarse_solve(F, S.m, g.step_cap, 60, 1e-12, c->s);
    c->launches += 1;
    return;
  }
  for (int s = 0; s < g.n_pre; ++s) {
    f64::sweep(F, S.m, 0, g.step_cap, c->s);
    f64::sweep(F, S.m, 1, g.step_cap, c->s);
    c->launches += 2;
  }
  DenseLevel C = sub_work(S.A, H, k + 1, S.mthr);
  f64::restrict_resid(F, C, S.m, c->s);
  f64::fas_rhs(C, S.m, c->s);
  c->launches += 2;
  vcycle_dense_masked(S, k + 1);
  f64::prolong_corr(F, C, g.prolong_linear, c->s);
  c->launches += 1;
  for (int s = 0; s < g.n_post; ++s) {
    f64::sweep(F, S.m, 0, g.step_cap, c->s);
    f64::sweep(F, S.m, 1, g.step_cap, c->s);
    c->launches += 2;
  }
}

// residual norm of level l (sum r^2, max |r|, sum f^2) -> host hs[0..2]
static mgfr_status level_norm(mgfr_ctx* c, AmrWork* A, int l, const Model& m, double* hs) {
  AmrLevel& L = A->L[l];
  DenseHier& H = c->dh;
  const int nparts = std::min<long long>(H.nparts / 2, nblocks(L.ncell, BS));
  k_oct_norm<<<nparts, BS, 0, c->s>>>(L.w, L.wE, L.wf, L.nbr, L.ghost, L.ghostE, L.ncell, m,
                                      L.ih2, H.partials);
  k_finish3<<<1, 256, 0, c->s>>>(H.partials, nparts, H.scal + 8);
  c->launches += 2;
  MG_CK(c, cudaMemcpyAsync(hs, H.scal + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  return MGFR_OK;
}

static mgfr_status count_relaxed(mgfr_ctx* c, AmrWork* A, const float* mask, long long n,
                                 float mthr, long long* out) {
  MG_CK(c, cudaMemsetAsync(A->d_small + 2, 0, sizeof(long long), c->s));
  k_count_relaxed<<<std::min<long long>(1024, nblocks(n, BS)), BS, 0, c->s>>>(mask, n, mthr,
                                                                              A->d_small + 2);
  c->launches += 1;
  MG_CK(c, cudaMemcpyAsync(out, A->d_small + 2, sizeof(long long), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  return MGFR_OK;
}

// One-way solve of refined level L (Sec. 3.3, steps 9-10).
static mgfr_status solve_level(mgfr_ctx* c, AmrWork* A, int Lv, const Model& m, mgfr_stats* st) {
  const mgfr_config& g = c->cfg;
  DenseHier& H = c->dh;
  AmrLevel& F = A->L[Lv];
  const float mthr = (float)g.mask_thres;
  TreeView T = tree_view(A);
  const double* up = Lv - 1 == 0 ? H.L[0].u : A->L[Lv - 1].u;
  // ghosts and initial guess from the converged parent level
  k_ghosts<<<nblocks(24 * F.n_oct, BS), BS, 0, c->s>>>(F.n_oct, Lv, T, F.nbr, up, g.prolong_linear,
                                                       F.ghost, F.ghostE);
  k_oct_init<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.ncell, Lv, T, F.pcell, up,
                                                    g.prolong_linear, F.w, F.wE);
  MG_CK(c, cudaMemcpyAsync(F.wf, F.f, sizeof(double) * (size_t)F.ncell, cudaMemcpyDeviceToDevice, c->s));
  k_fill_f<<<nblocks(F.ncell, BS), BS, 0, c->s>>>(F.mask, F.ncell, 1.f);
  c->launches += 3;
  F.relaxed = F.ncell;
  // coarse tree levels: work = converged solution; masks averaged down
  for (int l = Lv - 1; l >= 0; --l) {
    AmrLevel& P = A->L[l];
    const double* uu = l == 0 ? H.L[0].u : P.u;
    const double* EE = l == 0 ? H.L[0].E : P.E;
    MG_CK(c, cudaMemcpyAsync(P.w, uu, sizeof(double) * (size_t)P.ncell, cudaMemcpyDeviceToDevice, c->s));
    MG_CK(c, cudaMemcpyAsync(P.wE, EE, sizeof(double) * (size_t)P.ncell, cudaMemcpyDeviceToDevice, c->s));
    MG_CK(c, cudaMemcpyAsync(P.wold, uu, sizeof(double) * (size_t)P.ncell, cudaMemcpyDeviceToDevice, c->s));
    MG_CK(c, cudaMemsetAsync(P.mask, 0, sizeof(float) * (size_t)P.ncell, c->s));
    AmrLevel& Ch = A->L[l + 1];
    k_mask_up<<<nblocks(Ch.n_oct, BS), BS, 0, c->s>>>(Ch.mask, Ch.n_oct, Ch.pcell, P.mask);
    c->launches += 1;
    TRY(count_relaxed(c, A, P.mask, P.ncell, mthr, &P.relaxed));
  }
  for (int k = 1; k < H.nlev; ++k) {
    const float* mf = k == 1 ? A->L[0].mask : A->dmask[k - 1];
    k_mask_dense<<<nblocks(H.L[k].n, BS), BS, 0, c->s>>>(mf, H.L[k - 1].lg, A->dmask[k]);
    c->launches += 1;
  }
  AmrSolveCtx S{c, A, m, Lv, mthr, 0};
  if (g.profile) prof_reserve_public(c, 64);
  double hs[3];
  TRY(level_norm(c, A, Lv, m, hs));
  const double fn = std::sqrt(hs[2]), r0 = std::sqrt(hs[0]);
  const double target = g.tol_rel * (fn > 0.0 ? fn : r0);
  double r = r0;
  int it = 0;
  while (r > target && it < g.max_vcycles) {
    c->capturing = 3;
    vcycle_tree(S, Lv);
    c->capturing = -1;
    TRY(level_norm(c, A, Lv, m, hs));
    prof_collect(c, 3, st);
    r = std::sqrt(hs[0]);
    ++it;
    if (!std::isfinite(r)) break;
  }
  MG_CK(c, cudaMemcpyAsync(F.u, F.w, sizeof(double) * (size_t)F.ncell, cudaMemcpyDeviceToDevice, c->s));
  MG_CK(c, cudaMemcpyAsync(F.E, F.wE, sizeof(double) * (size_t)F.ncell, cudaMemcpyDeviceToDevice, c->s));
  if (st) {
    st->level_iters[Lv] = it;
    st->level_res[Lv] = fn > 0.0 ? r / fn : r;
    st->cell_updates += S.updates;
  }
  if (!(r <= target)) return set_err(c, MGFR_E_NOCONVERGE, "refined level did not converge");
  return MGFR_OK;
}

mgfr_status dense_solve64(mgfr_ctx* c, const Model& m, double box, mgfr_stats* st);
mgfr_status dense_solve_mixed(mgfr_ctx* c, const Model& m, double box, mgfr_stats* st);
mgfr_status ensure_dense_public(mgfr_ctx* c, int N, bool mixed, double box);

extern "C" {

mgfr_status mgfr_solve_particles(mgfr_ctx* c, const double* pos, long long Np, int N0, double box,
                                 double a, const double* u_init, double* fr_out, double* acc_out,
                                 mgfr_stats* st) {
  if (!c) return MGFR_E_INVALID;
  if (!pos || Np <= 0) return set_err(c, MGFR_E_INVALID, "need Np >= 1 particle positions");
  if (Np >= (1LL << 40)) return set_err(c, MGFR_E_INVALID, "Np too large");
  if (N0 < 8 || N0 > 1024 || (N0 & (N0 - 1))) return set_err(c, MGFR_E_INVALID, "N_base must be a power of two in [8, 1024]");
  if (!(box > 0.0) || !std::isfinite(box)) return set_err(c, MGFR_E_INVALID, "box must be > 0");
  if (!(a > 0.0) || !std::isfinite(a)) return set_err(c, MGFR_E_INVALID, "a must be > 0");
  const mgfr_config& g = c->cfg;
  MG_CK(c, cudaSetDevice(c->device));
  if (st) std::memset(st, 0, sizeof(*st));
  c->launches = 0;
  const bool mixed = g.precision == MGFR_PREC_MIXED;
  TRY(ensure_dense_public(c, N0, mixed, box));
  if (!c->amr) c->amr = new AmrWork();
  AmrWork* A = W(c);
  if (!A->d_small) MG_CK(c, cudaMalloc(&A->d_small, sizeof(long long) * 8));
  int lg0 = 0;
  while ((1 << lg0) < N0) ++lg0;
  if (A->N0 != N0) {
    for (int k = 0; k < MGFR_MAX_DENSE; ++k)
      if (A->dmask[k]) {
        cudaFree(A->dmask[k]);
        A->dmask[k] = nullptr;
      }
    if (A->acc0) cudaFree(A->acc0);
    if (A->fr0) cudaFree(A->fr0);
    A->acc0 = A->fr0 = nullptr;
  }
  A->N0 = N0;
  A->lg0 = lg0;
  A->box = box;
  A->Np = Np;
  DenseHier& H = c->dh;
  for (int k = 1; k < H.nlev; ++k)
    if (!A->dmask[k]) MG_CK(c, cudaMalloc(&A->dmask[k], sizeof(float) * (size_t)H.L[k].n));
  if (!A->acc0) MG_CK(c, cudaMalloc(&A->acc0, sizeof(double) * 3 * (size_t)H.L[0].n));
  if (!A->fr0) MG_CK(c, cudaMalloc(&A->fr0, sizeof(double) * (size_t)H.L[0].n));
  auto w0 = std::chrono::steady_clock::now();
  MG_CK(c, cudaEventRecord(c->ev_in, c->user));
  MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_in, 0));
  MG_CK(c, cudaMemsetAsync(A->d_small, 0, sizeof(long long) * 8, c->s));
  k_nan_check<<<nblocks(3 * Np, BS), BS, 0, c->s>>>(pos, 3 * Np, (unsigned long long*)(A->d_small + 1));
  c->launches += 1;
  // structure, deposit, sources
  TRY(build_structure(c, A, pos));
  TRY(deposit(c, A, pos));
  const Model m = make_model(g, a);
  for (int l = 0; l < A->nlev; ++l) {
    AmrLevel& L = A->L[l];
    const double Nl = (double)(1LL << L.lgN);
    double* f = l == 0 ? H.L[0].f : L.f;
    k_source_lvl<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.mass, L.ncell, Nl * Nl * Nl / (double)Np,
                                                        m.src, f);
    c->launches += 1;
  }
  long long flags = 0;
  MG_CK(c, cudaMemcpyAsync(&flags, A->d_small + 1, sizeof(long long), cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  if (flags & 2) return set_err(c, MGFR_E_INVALID, "non-finite particle position");
  if (flags & 1) return set_err(c, MGFR_E_UNSUPPORTED, "cloud-in-cell split stack overflow");
  // base level
  DenseLevel& L0 = H.L[0];
  f64::init_u(u_init, L0.u, L0.E, L0.n, c->s);
  c->launches += 1;
  MG_CK(c, cudaEventRecord(c->t0, c->s));
  mgfr_status rs = mixed ? dense_solve_mixed(c, m, box, st) : dense_solve64(c, m, box, st);
  if (rs != MGFR_OK && rs != MGFR_E_NOCONVERGE) return rs;
  mgfr_status worst = rs;
  for (int l = 1; l < A->nlev; ++l) {
    mgfr_status ls = solve_level(c, A, l, m, st);
    if (ls != MGFR_OK && ls != MGFR_E_NOCONVERGE) return ls;
    if (ls != MGFR_OK) worst = ls;
  }
  MG_CK(c, cudaEventRecord(c->t1, c->s));
  // force per level, then at the particles
  f64::force(L0, m, A->fr0, A->acc0, c->s);
  c->launches += 1;
  if (fr_out)
    MG_CK(c, cudaMemcpyAsync(fr_out, A->fr0, sizeof(double) * (size_t)L0.n,
                             cudaMemcpyDeviceToDevice, c->s));
  GatherPtrs G{};
  G.acc[0] = A->acc0;
  G.n0 = L0.n;
  for (int l = 1; l < A->nlev; ++l) {
    AmrLevel& L = A->L[l];
    const double gs = m.fbar / (2.0 * L.h) / (2.0 * m.a);
    k_oct_force<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.E, L.nbr, L.ghostE, L.ncell, m.fbar, gs,
                                                       L.w, L.acc);
    G.acc[l] = L.acc;
    c->launches += 1;
  }
  if (acc_out) {
    TreeView T = tree_view(A);
    k_gather<<<nblocks(Np, BS), BS, 0, c->s>>>(pos, Np, (double)N0 / box, (double)N0, T, G,
                                               acc_out, (unsigned long long*)(A->d_small + 1));
    c->launches += 1;
  }
  MG_CK(c, cudaEventRecord(c->ev_out, c->s));
  MG_CK(c, cudaStreamWaitEvent(c->user, c->ev_out, 0));
  MG_CK(c, cudaStreamSynchronize(c->s));
  MG_CK(c, cudaGetLastError());
  if (st) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->t0, c->t1);
    st->t_solve_ms = ms;
    st->n_levels = A->nlev;
    for (int l = 0; l < A->nlev; ++l) {
      st->cells_per_level[l] = A->L[l].ncell;
      st->octs_per_level[l] = A->L[l].n_oct;
    }
    st->gpu_launches = c->launches;
    st->t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  }
  return worst;
}

mgfr_status mgfr_get_level_info(mgfr_ctx* c, int level, long long* n_oct, long long* ncell) {
  if (!c) return MGFR_E_INVALID;
  AmrWork* A = W(c);
  if (!A || level < 0 || level >= A->nlev) return set_err(c, MGFR_E_INVALID, "no such level");
  if (n_oct) *n_oct = A->L[level].n_oct;
  if (ncell) *ncell = A->L[level].ncell;
  return MGFR_OK;
}

mgfr_status mgfr_get_level_keys(mgfr_ctx* c, int level, long long* keys_host) {
  if (!c || !keys_host) return MGFR_E_INVALID;
  AmrWork* A = W(c);
  if (!A || level < 1 || level >= A->nlev) return set_err(c, MGFR_E_INVALID, "no such refined level");
  AmrLevel& L = A->L[level];
  std::vector<int4> p((size_t)L.n_oct);
  MG_CK(c, cudaMemcpy(p.data(), L.opos, sizeof(int4) * (size_t)L.n_oct, cudaMemcpyDeviceToHost));
  const long long Np = 1LL << (A->lg0 + level - 1);
  for (long long o = 0; o < L.n_oct; ++o)
    keys_host[o] = ((long long)p[o].x * Np + p[o].y) * Np + p[o].z;
  return MGFR_OK;
}

mgfr_status mgfr_get_level_field(mgfr_ctx* c, int level, int what, double* out_host) {
  if (!c || !out_host) return MGFR_E_INVALID;
  AmrWork* A = W(c);
  if (!A || level < 0 || level >= A->nlev) return set_err(c, MGFR_E_INVALID, "no such level");
  AmrLevel& L = A->L[level];
  const size_t n = (size_t)L.ncell;
  const double* src = nullptr;
  size_t cnt = n;
  std::vector<double> tmp;
  switch (what) {
    case MGFR_FIELD_U: src = level == 0 ? c->dh.L[0].u : L.u; break;
    case MGFR_FIELD_SOURCE: src = level == 0 ? c->dh.L[0].f : L.f; break;
    case MGFR_FIELD_MASS: src = L.mass; break;
    case MGFR_FIELD_FR: src = level == 0 ? A->fr0 : L.w; break;
    case MGFR_FIELD_ACC:
      src = level == 0 ? A->acc0 : L.acc;
      cnt = 3 * n;
      break;
    case MGFR_FIELD_COUNT: {
      std::vector<int> ci(n);
      MG_CK(c, cudaMemcpy(ci.data(), L.count, sizeof(int) * n, cudaMemcpyDeviceToHost));
      for (size_t q = 0; q < n; ++q) out_host[q] = ci[q];
      return MGFR_OK;
    }
    default: return set_err(c, MGFR_E_INVALID, "unknown field");
  }
  MG_CK(c, cudaMemcpy(out_host, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
  return MGFR_OK;
}

}  // extern "C"
