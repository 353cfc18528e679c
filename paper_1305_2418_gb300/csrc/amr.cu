// amr.cu -- refined hierarchy from particle counts, adaptive cloud-in-cell,
// one-way refined-level solves and the force at the particles
// (Puchwein, Baldi & Springel 2013, Sec. 3.1 and 3.3, Eq. (13)).
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
#include <type_traits>
#include <vector>

#include "amr.cuh"
#include "dfloat.cuh"

namespace {

constexpr int BS = 256;

// ---- particle coordinates ------------------------------------------------
__device__ __forceinline__ double wrap_coord(double x, double inv, double N0) {
  double t = __dmul_rn(x, inv);
  // 0 <= t < N0 tested on the bit patterns (ordered like the values for
  // non-negative doubles; -0.0 and negatives have the sign bit set)
  const long long tb = __double_as_longlong(t);
  if (tb < 0 || tb >= __double_as_longlong(N0)) {
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

// Fixed point for the traversal: a coordinate is held as X = floor(t 2^52),
// t in level-0 cell units (t < N0 <= 2^10, so X < 2^62).  For every level m,
// X >> (52 - m) = floor(t 2^m) exactly (nested floors), so the cells chosen are
// those of the floating-point definition; every overlap length is an integer,
// exact in double, and a weight is rounded only by its two products.  All of
// the traversal but those products runs on the integer pipes.
constexpr int QB = 52;

// floor(t 2^52) for 0 <= t < 2^10, read off t's bits: with t = 1.f 2^e and
// s = 2^52 + f the 53-bit significand, t 2^52 = s 2^e, so X = s << e for
// e >= 0 and s >> -e (the floor) for e < 0.  Equal to the truncating FP64
// conversion of t 2^52, without FP64 instructions.
__device__ __forceinline__ long long qfix(double t) {
  const long long b = __double_as_longlong(t);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const long long sig = (b & ((1LL << 52) - 1)) | (1LL << 52);
  if (e >= 0) return sig << e;
  return e > -53 ? sig >> -e : 0;  // also t = +-0 and subnormals: 0
}

// v as a double for 0 <= v <= 2^52 (exact), built on the integer pipes: the
// leading bit gives the exponent, the bits below it the significand
// (times 2^k, exact while the result is a normal number)
__device__ __forceinline__ double exact_i2d(long long v, int k = 0) {
  if (v == 0) return 0.0;
  const int e = 63 - __clzll(v);  // v in [2^e, 2^(e+1)), e <= 52
  const unsigned long long m = ((unsigned long long)v << (52 - e)) & 0xfffffffffffffULL;
  return __longlong_as_double((long long)(((unsigned long long)(e + k + 1023) << 52) | m));
}

// ---- structure kernels -----------------------------------------------------
__global__ void k_count(const double* __restrict__ pos, long long Np, double inv, double N0, int l,
                        TreeView T, int* __restrict__ count) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Np) return;
  const P3 t = particle_t(pos, p, inv, N0);
  int lev;
  const int sh = QB - l;  // X >> (52 - l) = floor(t 2^l)
  const long long c =
      find_cell(T, l, qfix(t.x) >> sh, qfix(t.y) >> sh, qfix(t.z) >> sh, &lev);
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
// On the base level the scan runs in Morton (Z) order of the cells: scan
// element i is the cell whose coordinates interleave the bits of i, so the
// octs of level 1, and through their daughters every deeper level, are stored
// along a Z curve and face-neighbouring octs lie close together in memory.
constexpr int SCAN_BS = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_BS * SCAN_ITEMS;

// every third bit of x (bits 0, 3, 6, ...) packed into the low bits
__device__ __forceinline__ unsigned long long take3(unsigned long long x) {
  unsigned long long r = 0;
#pragma unroll
  for (int b = 0; b < 21; ++b) r |= ((x >> (3 * b)) & 1ULL) << b;
  return r;
}

// scan position -> cell index: identity, or Morton order on an N = 2^mlg base
__device__ __forceinline__ long long scan_cell(long long i, int mlg) {
  if (mlg == 0) return i;
  const unsigned long long x = (unsigned long long)i;
  const long long I = (long long)take3(x >> 2), J = (long long)take3(x >> 1),
                  K = (long long)take3(x);
  return (((I << mlg) + J) << mlg) + K;
}

__global__ void __launch_bounds__(SCAN_BS) k_scan_count(const unsigned char* __restrict__ flags,
                                                        long long n, int mlg,
                                                        int* __restrict__ sums) {
  __shared__ int red[SCAN_BS / 32];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int cnt = 0;
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    const long long i = base + (long long)q * SCAN_BS + threadIdx.x;
    if (i < n) cnt += flags[scan_cell(i, mlg)] != 0;
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
                                                          long long n, int mlg,
                                                          const int* __restrict__ offs,
                                                          int* __restrict__ son) {
  // rank of a set flag = set flags before it in its warp (ballot) + in the
  // warps before (a scan of the 32 warp counts)
  __shared__ int wsum[SCAN_BS / 32];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int run = offs[blockIdx.x];
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    const long long i = base + (long long)q * SCAN_BS + threadIdx.x;
    const long long c = i < n ? scan_cell(i, mlg) : 0;
    const bool v = i < n && flags[c];
    const unsigned ballot = __ballot_sync(0xffffffffu, v);
    if (lane == 0) wsum[w] = __popc(ballot);
    __syncthreads();
    if (w == 0) {
      int x = wsum[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
      }
      wsum[lane] = x;  // inclusive
    }
    __syncthreads();
    const int before = (w > 0 ? wsum[w - 1] : 0) + __popc(ballot & ((1u << lane) - 1u));
    if (i < n) son[c] = v ? run + before : -1;
    run += wsum[SCAN_BS / 32 - 1];
    __syncthreads();
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
  // the deposit's record of each particle's cells for the FP32 gather (NULL:
  // none): 8 slots per particle (its cube's corners q = 4 bx + 2 by + bz),
  // cell level << rb | index (rb = 32 minus the bits of the deepest level);
  // slot q of particle p at q np + p
  unsigned* rec_idx;
  long long np;
  int rb;
};

// record slot values: a zero-width corner, and (slot 0) a particle whose cube
// splits over finer cells (its pieces are not recorded)
constexpr unsigned kRecSkip = 0xffffffffu, kRecSplit = 0xfffffffeu;

// index bits of a record slot for a hierarchy of nlev levels: the level takes
// the top max(1, ceil(log2 nlev)) bits; cells of a level must stay below
// 2^rb - 2 so that no slot equals a marker
static inline int rec_bits(int nlev) {
  int lb = 1;
  while ((1 << lb) < nlev) ++lb;
  return 32 - lb;
}

struct GatherPtrs {
  const double* acc[AMR_MAXL];    // FP64: level 0 [3][N0^3]; l >= 1 [ncell][3]
  const float4* acc32[AMR_MAXL];  // FP32 (mixed form): [ncell] (x, y, z, 0)
  long long n0;
};

// Weight arithmetic of the traversal.  double: the integer overlap lengths
// exactly, the scale 2^(-3F) to the fraction of the cube in the exponent of
// the x lengths (deposit and the FP64 gather).  float (gather of the mixed form): the top 24 bits of each
// length relative to the cube side 2^F, scale 2^-72; the weights then carry
// a relative error of about 2^-24.
template <class W>
struct Wt;
template <>
struct Wt<double> {
  static __device__ __forceinline__ double len(long long v, int) { return exact_i2d(v); }
  // len(v) 2^(-3F), the scale entering the exponent (exact: v = 0, or v >= 1 and
  // the result >= 2^-156, a normal number)
  static __device__ __forceinline__ double len_scaled(long long v, int F) {
    return exact_i2d(v, -3 * F);
  }
};
template <>
struct Wt<float> {
  static __device__ __forceinline__ float len(long long v, int F) {
    return (float)(int)((v + (1LL << (F - 25))) >> (F - 24));  // rounded to nearest
  }
  static __device__ __forceinline__ float scale(int) { return 0x1p-72f; }
  static __device__ __forceinline__ float len_scaled(long long v, int F) {
    return len(v, F) * scale(F);
  }
};

template <bool GATHER, class W>
__device__ __forceinline__ void touch(int lev, long long c, W w, LevelPtrs& D,
                                      const GatherPtrs& G, W* out) {
  if constexpr (GATHER && std::is_same<W, float>::value) {
    const float4 a = G.acc32[lev][c];
    out[0] = fmaf(w, a.x, out[0]);
    out[1] = fmaf(w, a.y, out[1]);
    out[2] = fmaf(w, a.z, out[2]);
  } else if (GATHER) {
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
  long long lo[3], hi[3];  // piece [lo, hi) per axis, fixed-point units
  long long c;             // refined cell index at level l holding the piece
  int l;
  int pad;
};

// Split the piece [lo, hi) of refined cell c at level l among its daughters:
// per axis the daughter boundary is mid = (2P + 1) 2^(QB - l - 1) and the
// two overlaps are [lo, min(hi, mid)) and [max(lo, mid), hi).  A daughter
// that is refined again is split one more level in registers (DEPTH = 2) or
// pushed on the explicit stack (DEPTH = 1).  No recursion: the stack frame
// size is static.
template <bool GATHER, class W, int DEPTH>
__device__ __forceinline__ void split_q(const TreeView& T, int l, long long c, const long long* lo,
                                        const long long* hi, int F, LevelPtrs& D,
                                        const GatherPtrs& G, W* out, StackEnt* st, int& sp,
                                        unsigned long long* err) {
  const int o = T.son[l][c];
  const int lc = l + 1, sh = QB - lc;
  long long clo[3][2], chi[3][2];
  W len[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long mid = ((lo[a] >> sh) | 1LL) * (1LL << sh);
    clo[a][0] = lo[a];
    chi[a][0] = min(hi[a], mid);
    clo[a][1] = max(lo[a], mid);
    chi[a][1] = hi[a];
#pragma unroll
    for (int b = 0; b < 2; ++b)  // the fraction of the cube enters through axis 0
      len[a][b] = a == 0 ? Wt<W>::len_scaled(chi[a][b] - clo[a][b], F)
                         : Wt<W>::len(chi[a][b] - clo[a][b], F);
  }
  for (int ch = 0; ch < 8; ++ch) {
    const int b0 = (ch >> 2) & 1, b1 = (ch >> 1) & 1, b2 = ch & 1;
    if (chi[0][b0] <= clo[0][b0] || chi[1][b1] <= clo[1][b1] || chi[2][b2] <= clo[2][b2]) continue;
    const long long cc = 8LL * o + ch;
    const bool ref = lc + 1 < T.nlev && T.son[lc][cc] >= 0;
    if (!ref) {
      touch<GATHER, W>(lc, cc, len[0][b0] * len[1][b1] * len[2][b2], D, G, out);
      continue;
    }
    const long long nlo[3] = {clo[0][b0], clo[1][b1], clo[2][b2]};
    const long long nhi[3] = {chi[0][b0], chi[1][b1], chi[2][b2]};
    if constexpr (DEPTH > 1) {
      split_q<GATHER, W, DEPTH - 1>(T, lc, cc, nlo, nhi, F, D, G, out, st, sp, err);
    } else {
      if (sp < 48) {
        StackEnt& n = st[sp++];
        for (int a = 0; a < 3; ++a) {
          n.lo[a] = nlo[a];
          n.hi[a] = nhi[a];
        }
        n.c = cc;
        n.l = lc;
      } else {
        atomicOr(err, 1ULL);
      }
    }
  }
}

// Visits the pieces of a particle's cube (deposit: adds the weights; gather:
// sums weight x force).  Returns whether the cube split over finer cells.
// ri (deposit with a record): the record's 8 slots, which the caller stores
// once its warp has reconverged (whole-warp, coalesced stores).
// MODE 0: every piece.  MODE 1: only the corners that are not refined (the
// split ones are left to a MODE 2 pass over the listed particles, so that the
// warps of the first pass do not wait on the few lanes that split).  MODE 2:
// only the pieces of refined corners.
constexpr int kVisitAll = 0, kVisitUnsplit = 1, kVisitSplit = 2;
template <bool GATHER, class W, int MODE = kVisitAll>
__device__ bool visit_particle(const TreeView& T, const P3& t, LevelPtrs& D, const GatherPtrs& G,
                               W* out, unsigned long long* err, unsigned* ri = nullptr) {
  const bool rec = !GATHER && D.rec_idx;
  bool split = false;
  const long long X[3] = {qfix(t.x), qfix(t.y), qfix(t.z)};
  // leaf level lam of the particle and the oct holding its leaf cell
  int lam = 0, own = -1;
  long long c = ((((X[0] >> QB) << T.lg0) + (X[1] >> QB)) << T.lg0) + (X[2] >> QB);
  for (int m = 1; m < T.nlev; ++m) {
    const int o = T.son[m - 1][c];
    if (o < 0) break;
    const int sh = QB - m;
    c = 8LL * o + (((X[0] >> sh) & 1) << 2) + (((X[1] >> sh) & 1) << 1) + ((X[2] >> sh) & 1);
    lam = m;
    own = o;
  }
  // the cube: side one level-lam cell, centred on the particle: [cl, cl + 2^F)
  const int F = QB - lam;
  const long long one = 1LL << F;
  long long cl[3], i0[3], edge[3];
  W Lw[3][2];
  // fixed-point volume -> fraction of the cube
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cl[a] = X[a] - (one >> 1);
    i0[a] = cl[a] >> F;
    edge[a] = (i0[a] + 1) * one;  // boundary between the two cells the cube spans
    // the fraction of the cube (scale) enters through axis 0
    Lw[a][0] = a == 0 ? Wt<W>::len_scaled(edge[a] - cl[a], F) : Wt<W>::len(edge[a] - cl[a], F);
    Lw[a][1] = a == 0 ? Wt<W>::len_scaled(cl[a] + one - edge[a], F)
                      : Wt<W>::len(cl[a] + one - edge[a], F);
  }
  // x-y products of the corner weights, shared by the two z pieces
  W Lxy[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) Lxy[b] = Lw[0][b >> 1] * Lw[1][b & 1];
  StackEnt st[48];
  int sp = 0;
  for (int q = 0; q < 8; ++q) {
    const int bits[3] = {(q >> 2) & 1, (q >> 1) & 1, q & 1};
    if ((bits[0] && edge[0] == cl[0] + one) || (bits[1] && edge[1] == cl[1] + one) ||
        (bits[2] && edge[2] == cl[2] + one)) {
      if (rec) ri[q] = kRecSkip;
      continue;  // zero-width piece
    }
    const long long K[3] = {i0[0] + bits[0], i0[1] + bits[1], i0[2] + bits[2]};
    int lev;
    long long cq;
    if (lam > 0 && (K[0] >> 1) == (X[0] >> (F + 1)) && (K[1] >> 1) == (X[1] >> (F + 1)) &&
        (K[2] >> 1) == (X[2] >> (F + 1))) {
      // same oct as the particle's leaf cell
      cq = 8LL * own + ((K[0] & 1) << 2) + ((K[1] & 1) << 1) + (K[2] & 1);
      lev = lam;
    } else {
      cq = find_cell(T, lam, K[0], K[1], K[2], &lev);
    }
    const bool refined = lev == lam && lam + 1 < T.nlev && T.son[lam][cq] >= 0;
    if (!refined) {
      if (MODE != kVisitSplit) {
        const W w = Lxy[(bits[0] << 1) | bits[1]] * Lw[2][bits[2]];
        touch<GATHER, W>(lev, cq, w, D, G, out);
        if (rec) ri[q] = ((unsigned)lev << D.rb) | (unsigned)cq;
      }
      continue;
    }
    split = true;
    if (rec) ri[q] = kRecSkip;
    if (MODE == kVisitUnsplit) continue;
    long long lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = bits[a] ? edge[a] : cl[a];
      hi[a] = bits[a] ? cl[a] + one : edge[a];
    }
    split_q<GATHER, W, 2>(T, lam, cq, lo, hi, F, D, G, out, st, sp, err);
  }
  // pieces refined three or more levels below the particle's leaf
  while (sp > 0) {
    const StackEnt e = st[--sp];
    split_q<GATHER, W, 1>(T, e.l, e.c, e.lo, e.hi, F, D, G, out, st, sp, err);
  }
  if (rec && split) ri[0] = kRecSplit;
  return split;
}

// With a record (D.rec_idx), the particles whose cube split are appended to
// the list of their chunk (chunk = p / per, its list at split_list + chunk per,
// counted in n_split[chunk]; one atomic per block, any order within the
// chunk).  Launched with 256 threads; per = 256 bpc, so a block lies in one
// chunk (a 32-bit division: a 64-bit one would be a call, which costs the
// traversal registers).
__global__ void __launch_bounds__(256, 4) k_deposit(const double* __restrict__ pos, long long Np, double inv, double N0,
                          TreeView T, LevelPtrs D, unsigned long long* err,
                          int* __restrict__ split_list, unsigned long long* __restrict__ n_split,
                          unsigned bpc) {
  __shared__ int woff[8];
  __shared__ unsigned long long bbase;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool split = false;
  unsigned ri[8];
  if (p < Np) {
    const P3 t = particle_t(pos, p, inv, N0);
    GatherPtrs G{};
    if (D.rec_idx)  // the split pieces are left to k_deposit_split
      split = visit_particle<false, double, kVisitUnsplit>(T, t, D, G, nullptr, err, ri);
    else
      split = visit_particle<false, double>(T, t, D, G, nullptr, err, ri);
  }
  if (!D.rec_idx) return;  // uniform over the launch
  // whole blocks reach here (no early exit above)
  const unsigned b = __ballot_sync(0xffffffffu, split);
  if (p < Np) {  // the warp has reconverged at the ballot: full-sector stores
#pragma unroll
    for (int q = 0; q < 8; ++q) D.rec_idx[q * D.np + p] = ri[q];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) woff[w] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int v = 0; v < 8; ++v) {
      const int k = woff[v];
      woff[v] = run;
      run += k;
    }
    const unsigned q = blockIdx.x / bpc;
    bbase = 256ULL * bpc * q + (run > 0 ? atomicAdd(n_split + q, (unsigned long long)run) : 0ULL);
  }
  __syncthreads();
  if (split) split_list[bbase + woff[w] + __popc(b & ((1u << lane) - 1u))] = (int)p;
}

// The split pieces of the particles listed by k_deposit (chunk q's list at
// split_list + q per, n_split[q] entries): a grid-stride loop over the eight
// lists, whose lengths are read on the device.
__global__ void __launch_bounds__(256, 4) k_deposit_split(
    const double* __restrict__ pos, double inv, double N0, TreeView T, LevelPtrs D,
    unsigned long long* err, const int* __restrict__ split_list,
    const unsigned long long* __restrict__ n_split, long long per) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int q = 0; q < 8; ++q) {
    const long long n = (long long)n_split[q];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += stride) {
      const long long p = split_list[q * per + t];
      const P3 tp = particle_t(pos, p, inv, N0);
      GatherPtrs G{};
      visit_particle<false, double, kVisitSplit>(T, tp, D, G, nullptr, err);
    }
  }
}

__global__ void k_gather(const double* __restrict__ pos, long long Np, double inv, double N0,
                         TreeView T, GatherPtrs G, double* __restrict__ acc,
                         unsigned long long* err) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Np) return;
  const P3 t = particle_t(pos, p, inv, N0);
  LevelPtrs D{};
  double out[3] = {0.0, 0.0, 0.0};
  visit_particle<true, double>(T, t, D, G, out, err);
  acc[3 * p] = out[0];
  acc[3 * p + 1] = out[1];
  acc[3 * p + 2] = out[2];
}

// mixed form: FP32 weights and FP32 force fields, FP64 output
__global__ void __launch_bounds__(256, 4) k_gather32(const double* __restrict__ pos, long long Np, double inv, double N0,
                           TreeView T, GatherPtrs G, double* __restrict__ acc,
                           unsigned long long* err) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= Np) return;
  const P3 t = particle_t(pos, p, inv, N0);
  LevelPtrs D{};
  float out[3] = {0.f, 0.f, 0.f};
  visit_particle<true, float>(T, t, D, G, out, err);
  acc[3 * p] = out[0];
  acc[3 * p + 1] = out[1];
  acc[3 * p + 2] = out[2];
}

// mixed form, from the deposit's record: the cells of each particle's cube
// are read from the record instead of found by walking the tree; the FP32
// weights and the sum are those of the traversal (same arithmetic, same
// order).  The particle's leaf level is the deepest recorded level (its leaf
// cell is one of the corners).  Particles whose cube split are left to
// k_gather32_list.  Particles p0 .. p0 + n - 1; np: the record's slot stride.
__global__ void __launch_bounds__(256) k_gather32_rec(const double* __restrict__ pos,
                                                      const unsigned* __restrict__ rec_idx,
                                                      long long np, int rb, long long p0,
                                                      long long n, double inv, double N0,
                                                      GatherPtrs G, double* __restrict__ acc) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long p = p0 + t;
  unsigned id[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) id[q] = __ldg(rec_idx + q * np + p);
  if (id[0] == kRecSplit) return;
  int lam = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (id[q] != kRecSkip) lam = max(lam, (int)(id[q] >> rb));
  const P3 tp = particle_t(pos, p, inv, N0);
  const long long X[3] = {qfix(tp.x), qfix(tp.y), qfix(tp.z)};
  const int F = QB - lam;
  const long long one = 1LL << F;
  float Lw[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long cl = X[a] - (one >> 1);
    const long long edge = ((cl >> F) + 1) * one;
    Lw[a][0] = Wt<float>::len(edge - cl, F);
    Lw[a][1] = Wt<float>::len(cl + one - edge, F);
  }
  const float scale = Wt<float>::scale(F);
  Lw[0][0] *= scale;
  Lw[0][1] *= scale;
  float Lxy[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) Lxy[b] = Lw[0][b >> 1] * Lw[1][b & 1];
  float out[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (id[q] == kRecSkip) continue;
    const float w = Lxy[q >> 1] * Lw[2][q & 1];
    const float4 a = __ldg(G.acc32[id[q] >> rb] + (id[q] & ((1u << rb) - 1u)));
    out[0] = fmaf(w, a.x, out[0]);
    out[1] = fmaf(w, a.y, out[1]);
    out[2] = fmaf(w, a.z, out[2]);
  }
  acc[3 * p] = out[0];
  acc[3 * p + 1] = out[1];
  acc[3 * p + 2] = out[2];
}

// mixed form, the listed particles (those whose cube split): full traversal
__global__ void __launch_bounds__(256, 4) k_gather32_list(const double* __restrict__ pos,
                                                          const int* __restrict__ list, long long n,
                                                          double inv, double N0, TreeView T,
                                                          GatherPtrs G, double* __restrict__ acc,
                                                          unsigned long long* err) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long p = list[t];
  const P3 tp = particle_t(pos, p, inv, N0);
  LevelPtrs D{};
  float out[3] = {0.f, 0.f, 0.f};
  visit_particle<true, float>(T, tp, D, G, out, err);
  acc[3 * p] = out[0];
  acc[3 * p + 1] = out[1];
  acc[3 * p + 2] = out[2];
}

// base-level force [3][n] (FP64) -> (x, y, z, 0) per cell (FP32)
__global__ void k_acc_pack(const double* __restrict__ acc, long long n, float4* __restrict__ a32) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n)
    a32[t] = make_float4(f_from_double_bits(acc[t]), f_from_double_bits(acc[n + t]),
                         f_from_double_bits(acc[2 * n + t]), 0.f);
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

// ---- effective mass density [Sec. 2.4] ---------------------------------------
// delta rho_eff / rho_bar = delta / 3 - delta R / (24 pi G rho_bar), delta R =
// R_bar (e^{-u/(n+1)} - 1) [Eq. (11)]: with R_bar = 3 H0^2 Rt and
// 24 pi G rho_bar = 9 H0^2 Om a^-3, delta / 3 + c3 (1 - e^{-u/(n+1)}),
// c3 = Rt / (3 Om a^-3); delta = mass scale - 1 per level (mass in particle
// masses, scale = N_l^3 / Np).
struct EffPar {
  double scale, c3, inv_np1;
};

__device__ __forceinline__ double eff_density(double mass, double u, const EffPar& q) {
  return (mass * q.scale - 1.0) / 3.0 + q.c3 * (1.0 - exp(-u * q.inv_np1));
}

__global__ void k_eff_level(const double* __restrict__ mass, const double* __restrict__ u,
                            long long n, EffPar q, double* __restrict__ out) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) out[c] = eff_density(mass[c], u[c], q);
}

// Each leaf cell of level l hands its mass to the cells of the nested
// periodic PM grid of level lpm (N_pm = N0 2^lpm) by overlapping volume: a
// leaf at l <= lpm covers 2^(lpm-l) PM cells per axis and gives each its
// contrast as a density (plain stores: leaves do not overlap); a leaf at
// l > lpm lies in one PM cell and adds its contrast 8^-(l-lpm) (atomics).
// The contrast is delta_eff (what 0), delta (what 1) or delta + delta_eff
// (what 2, the right-hand side of Eq. (30)).
__global__ void k_eff_pm(int l, int lpm, TreeView T, const double* __restrict__ mass,
                         const double* __restrict__ u, long long n, EffPar q, int what,
                         double* __restrict__ out) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= n || T.son[l][c] >= 0) return;  // not a leaf
  const double d = mass[c] * q.scale - 1.0;
  const double eff = what == 1 ? d : (what == 0 ? eff_density(mass[c], u[c], q)
                                                : d + eff_density(mass[c], u[c], q));
  long long I, J, K;
  cell_coords(T, l, c, &I, &J, &K);
  const long long Npm = 1LL << (T.lg0 + lpm);
  if (l <= lpm) {
    const long long s = 1LL << (lpm - l);
    for (long long a = 0; a < s; ++a)
      for (long long b = 0; b < s; ++b)
        for (long long e = 0; e < s; ++e)
          out[((I * s + a) * Npm + (J * s + b)) * Npm + (K * s + e)] = eff;
  } else {
    const int sh = l - lpm;
    atomicAdd(out + ((I >> sh) * Npm + (J >> sh)) * Npm + (K >> sh),
              eff / (double)(1LL << (3 * sh)));
  }
}

__global__ void k_nan_check(const double* __restrict__ x, long long n,
                            unsigned long long* __restrict__ err) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicOr(err, 2ULL);
}

// ---- refined-level force --------------------------------------------------
struct OctNbE {
  double E;
};

// E of the neighbour of cell (o, ch) in direction d (same oct, neighbouring
// oct, or the ghost slot of the face).
__device__ __forceinline__ double oct_nbE(const double* __restrict__ E,
                                         const int* __restrict__ nbr,
                                         const double* __restrict__ ghostE, int gdf, long long o,
                                         int ch, int d) {
  const int ax = d >> 1, plus = d & 1;
  const int bit = (ch >> (2 - ax)) & 1;
  const int chn = ch ^ (1 << (2 - ax));
  if (bit != plus) return E[8 * o + chn];
  const int no = nbr[6 * o + d];
  if (no >= 0) return E[8LL * no + chn];
  const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
  const int qi = (((ch >> (2 - t1)) & 1) << 1) | ((ch >> (2 - t2)) & 1);
  const long long g = 4LL * (-no - 1) + qi;  // ghost slot of the face
  return gdf ? df_to_double(reinterpret_cast<const dfl*>(ghostE)[g]) : ghostE[g];
}

// Ghost faces (faces without a neighbouring oct) get consecutive slots in
// storage order: flag them, scan, and store -(1 + slot) in the neighbour table.
__global__ void k_face_flags(const int* __restrict__ nbr, long long n,
                             unsigned char* __restrict__ flags) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) flags[i] = nbr[i] < 0 ? 1 : 0;
}
__global__ void k_face_slots(const int* __restrict__ slot, long long n, int* __restrict__ nbr,
                             unsigned* __restrict__ gface) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && slot[i] >= 0) {
    nbr[i] = -(slot[i] + 1);
    gface[slot[i]] = (unsigned)i;
  }
}

// FP32 force copy of a refined level from e^u as double-float pairs (mixed
// form): the central difference is formed exactly enough in double-float and
// rounded once, on the FP32 pipes.  acc32 = g_scale (E+ - E-) per axis.
__device__ __forceinline__ dfl oct_nbE_df(const dfl* __restrict__ E, const int* __restrict__ nbr,
                                          const dfl* __restrict__ ghostE, long long o, int ch,
                                          int d) {
  const int ax = d >> 1, plus = d & 1;
  const int bit = (ch >> (2 - ax)) & 1;
  const int chn = ch ^ (1 << (2 - ax));
  if (bit != plus) return E[8 * o + chn];
  const int no = nbr[6 * o + d];
  if (no >= 0) return E[8LL * no + chn];
  const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
  const int qi = (((ch >> (2 - t1)) & 1) << 1) | ((ch >> (2 - t2)) & 1);
  return ghostE[4LL * (-no - 1) + qi];
}

__global__ void k_oct_acc32_df(const dfl* __restrict__ E, const int* __restrict__ nbr,
                               const dfl* __restrict__ ghostE, long long ncell, float g_scale,
                               float4* __restrict__ acc32) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const long long o = c >> 3;
  const int ch = (int)(c & 7);
  float a[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const dfl em = oct_nbE_df(E, nbr, ghostE, o, ch, 2 * ax);
    const dfl ep = oct_nbE_df(E, nbr, ghostE, o, ch, 2 * ax + 1);
    a[ax] = g_scale * df_add_abs(ep, df_neg(em)).hi;
  }
  acc32[c] = make_float4(a[0], a[1], a[2], 0.f);
}

__global__ void k_oct_pnbrs(long long n_oct, int l, TreeView T, int* __restrict__ pnbr) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= n_oct) return;
  const int4 p = T.opos[l][o];
  const int dd[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int d = 0; d < 6; ++d) {
    int lev;
    const long long q = find_cell(T, l - 1, p.x + dd[d][0], p.y + dd[d][1], p.z + dd[d][2], &lev);
    pnbr[6 * o + d] = lev == l - 1 ? (int)q : -1;
  }
}

// f_R and a_MG/c^2 on a refined level (central differences, ghosts at edges)
__global__ void k_oct_force(const double* __restrict__ E, const int* __restrict__ nbr,
                            const double* __restrict__ ghostE, int gdf, long long ncell,
                            double fbar,
                            double g_scale, double* __restrict__ fr, double* __restrict__ acc,
                            float4* __restrict__ acc32) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const long long o = c >> 3;
  const int ch = (int)(c & 7);
  fr[c] = fbar * E[c];
  for (int ax = 0; ax < 3; ++ax) {
    const double em = oct_nbE(E, nbr, ghostE, gdf, o, ch, 2 * ax);
    const double ep = oct_nbE(E, nbr, ghostE, gdf, o, ch, 2 * ax + 1);
    acc[3 * c + ax] = g_scale * (ep - em);
  }
  if (acc32)
    acc32[c] = make_float4((float)acc[3 * c], (float)acc[3 * c + 1], (float)acc[3 * c + 2], 0.f);
}

}  // namespace

// ============================================================================
// host side
// ============================================================================

static AmrWork* W(mgfr_ctx* c) { return (AmrWork*)c->amr; }

static void free_level(AmrLevel& L) {
  void* ps[] = {L.son,  L.refined, L.count,  L.opos, L.pcell,   L.nbr,     L.mass,
                L.w,    L.wE,      L.wf,     L.wold, L.mask,    L.ghost,   L.ghostE,
                L.acc,  L.pnbr,    L.w32,    L.wE32, L.wf32,    L.wold32,  L.ghost32, L.gface,
                L.olist,  L.acc32, L.act};
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
  for (int l = 0; l < MGFR_MAX_DENSE; ++l) {
    if (A->dmask[l]) cudaFree(A->dmask[l]);
    if (A->dact[l]) cudaFree(A->dact[l]);
    if (A->dlist[l]) cudaFree(A->dlist[l]);
  }
  if (A->blocksums) cudaFree(A->blocksums);
  if (A->d_small) cudaFree(A->d_small);
  if (A->acc0) cudaFree(A->acc0);
  if (A->fr0) cudaFree(A->fr0);
  if (A->acc0_32) cudaFree(A->acc0_32);
  if (A->pos_dev) cudaFree(A->pos_dev);
  if (A->acc_dev) cudaFree(A->acc_dev);
  if (A->rec_idx) cudaFree(A->rec_idx);
  if (A->split_list) cudaFree(A->split_list);
  if (A->d_split) cudaFree(A->d_split);
  for (int l = 0; l < AMR_MAXL; ++l) {
    if (A->prev_key[l]) cudaFree(A->prev_key[l]);
    if (A->prev_u[l]) cudaFree(A->prev_u[l]);
  }
  delete A;
  c->amr = nullptr;
}

// Morton keys of the octs' parent cells (parent coordinates at level l - 1)
__global__ void k_oct_keys(const int4* __restrict__ opos, long long n_oct,
                           unsigned long long* __restrict__ key) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o >= n_oct) return;
  const int4 p = opos[o];
  key[o] = morton3((unsigned)p.x, (unsigned)p.y, (unsigned)p.z);
}

mgfr_status amr_keep_previous(mgfr_ctx* c, AmrWork* A, bool keep) {
  A->prev_nlev = 0;
  if (!keep) return MGFR_OK;
  // 21 bits per coordinate in the keys: parents of level l have coordinates
  // below N0 2^(l-1)
  if ((long long)A->N0 << (A->nlev > 1 ? A->nlev - 2 : 0) > (1LL << 21)) return MGFR_OK;
  for (int l = 1; l < A->nlev; ++l) {
    const AmrLevel& L = A->L[l];
    if (L.n_oct > A->prev_cap[l]) {
      if (A->prev_key[l]) cudaFree(A->prev_key[l]);
      if (A->prev_u[l]) cudaFree(A->prev_u[l]);
      A->prev_key[l] = nullptr;
      A->prev_u[l] = nullptr;
      A->prev_cap[l] = 0;
      MG_CK(c, cudaMalloc(&A->prev_key[l], sizeof(unsigned long long) * (size_t)L.n_oct));
      MG_CK(c, cudaMalloc(&A->prev_u[l], sizeof(double) * 8 * (size_t)L.n_oct));
      A->prev_cap[l] = L.n_oct;
    }
    A->prev_noct[l] = L.n_oct;
    if (L.n_oct == 0) continue;
    k_oct_keys<<<nblocks(L.n_oct, BS), BS, 0, c->s>>>(L.opos, L.n_oct, A->prev_key[l]);
    MG_CK(c, cudaMemcpyAsync(A->prev_u[l], L.u, sizeof(double) * 8 * (size_t)L.n_oct,
                             cudaMemcpyDeviceToDevice, c->s));
    c->launches += 1;
  }
  A->prev_nlev = A->nlev;
  A->prev_N0 = A->N0;
  A->prev_box = A->box;
  return MGFR_OK;
}

void amr_invalidate(mgfr_ctx* c) {
  if (c && c->amr) W(c)->nlev = 0;
}

TreeView tree_view(const AmrWork* A) {
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
  L.pnbr = nullptr; L.w32 = nullptr; L.wE32 = nullptr; L.wf32 = nullptr; L.wold32 = nullptr;
  L.ghost32 = nullptr; L.olist = nullptr; L.acc32 = nullptr; L.act = nullptr; L.gface = nullptr;
  L.gcap = 0;
  TRY(grow(c, &L.son, n));
  TRY(grow(c, &L.refined, n));
  TRY(grow(c, &L.count, n));
  TRY(grow(c, &L.mass, n));
  TRY(grow(c, &L.w, n));
  TRY(grow(c, &L.wE, n));
  TRY(grow(c, &L.wf, n));
  TRY(grow(c, &L.wold, n));
  TRY(grow(c, &L.mask, n));
  TRY(grow(c, &L.act, n));
  TRY(grow(c, &L.w32, n));
  TRY(grow(c, &L.wE32, n));
  TRY(grow(c, &L.wf32, n));
  TRY(grow(c, &L.wold32, n));
  if (l > 0) {
    TRY(grow(c, &L.pnbr, 6 * no));
    TRY(grow(c, &L.olist, no));
    TRY(grow(c, &L.opos, no));
    TRY(grow(c, &L.pcell, no));
    TRY(grow(c, &L.nbr, 6 * no));
    TRY(grow(c, &L.acc, 3 * n));
    TRY(grow(c, &L.acc32, n));
    TRY(grow(c, &L.u, n));
    TRY(grow(c, &L.E, n));
    TRY(grow(c, &L.f, n));
  }
  A->cap_cells[l] = n;
  A->cap_oct[l] = no;
  return MGFR_OK;
}

static mgfr_status scan_flags(mgfr_ctx* c, AmrWork* A, const unsigned char* flags, long long n,
                              int mlg, int* son, long long* total) {
  const long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb > A->blocksums_cap) {
    if (A->blocksums) cudaFree(A->blocksums);
    A->blocksums = nullptr;
    MG_CK(c, cudaMalloc(&A->blocksums, sizeof(int) * (size_t)nb));
    A->blocksums_cap = nb;
  }
  k_scan_count<<<(unsigned)nb, SCAN_BS, 0, c->s>>>(flags, n, mlg, A->blocksums);
  k_scan_sums<<<1, SCAN_BS, 0, c->s>>>(A->blocksums, nb, A->d_small);
  k_scan_scatter<<<(unsigned)nb, SCAN_BS, 0, c->s>>>(flags, n, mlg, A->blocksums, son);
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
    TRY(scan_flags(c, A, L.refined, L.ncell, l == 0 ? A->lg0 : 0, L.son, &nref));
    if (nref == 0) break;
    // oct and face indices are 32-bit (neighbour tables, ghost slots)
    if (6 * nref > 0x7fffffffLL) return set_err(c, MGFR_E_INVALID, "refined level too large");
    AmrLevel& N = A->L[l + 1];
    N.n_oct = nref;
    N.ncell = 8 * nref;
    TRY(alloc_level(c, A, l + 1));
    A->nlev = l + 2;
    T = tree_view(A);
    k_make_octs<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.son, L.ncell, l, T, N.pcell, N.opos);
    T = tree_view(A);
    k_oct_nbrs<<<nblocks(N.n_oct, BS), BS, 0, c->s>>>(N.n_oct, l + 1, T, N.nbr);
    k_oct_pnbrs<<<nblocks(N.n_oct, BS), BS, 0, c->s>>>(N.n_oct, l + 1, T, N.pnbr);
    c->launches += 3;
    // ghost-face slots (scratch: the new level's refined and son arrays, set
    // for real in the next pass)
    k_face_flags<<<nblocks(6 * N.n_oct, BS), BS, 0, c->s>>>(N.nbr, 6 * N.n_oct, N.refined);
    TRY(scan_flags(c, A, N.refined, 6 * N.n_oct, 0, N.son, &N.n_gslot));
    if (N.n_gslot > N.gcap) {
      TRY(grow(c, &N.ghost, 4 * N.n_gslot));
      TRY(grow(c, &N.ghostE, 4 * N.n_gslot));
      TRY(grow(c, &N.ghost32, 4 * N.n_gslot));
      TRY(grow(c, &N.gface, N.n_gslot));
      N.gcap = N.n_gslot;
    }
    k_face_slots<<<nblocks(6 * N.n_oct, BS), BS, 0, c->s>>>(N.son, 6 * N.n_oct, N.nbr, N.gface);
    c->launches += 2;
  }
  // the deepest level has no sons
  AmrLevel& D = A->L[A->nlev - 1];
  MG_CK(c, cudaMemsetAsync(D.son, 0xff, sizeof(int) * (size_t)D.ncell, c->s));
  MG_CK(c, cudaMemsetAsync(D.refined, 0, (size_t)D.ncell, c->s));
  return MGFR_OK;
}

// record: keep each particle's cells for the FP32 gather (cell indices must
// fit the record's index bits, rec_bits), with the split particles listed per
// chunk of `per` particles (per a multiple of 256, at most 8 chunks)
static mgfr_status deposit(mgfr_ctx* c, AmrWork* A, const double* pos, bool record,
                           long long per) {
  const double inv = (double)A->N0 / A->box, N0d = (double)A->N0;
  LevelPtrs D{};
  for (int l = 0; l < A->nlev; ++l) {
    MG_CK(c, cudaMemsetAsync(A->L[l].mass, 0, sizeof(double) * (size_t)A->L[l].ncell, c->s));
    D.a[l] = A->L[l].mass;
    if (A->L[l].ncell > (1LL << rec_bits(A->nlev)) - 2) record = false;
  }
  A->rec_on = record;
  A->rec_per = per;
  for (auto& n : A->n_split) n = 0;
  if (record) {
    if (!A->d_split) MG_CK(c, cudaMalloc(&A->d_split, sizeof(long long) * 8));
    MG_CK(c, cudaMemsetAsync(A->d_split, 0, sizeof(long long) * 8, c->s));
    if (A->Np > A->rec_cap) {
      if (A->rec_idx) cudaFree(A->rec_idx);
      if (A->split_list) cudaFree(A->split_list);
      A->rec_idx = nullptr;
      A->split_list = nullptr;
      A->rec_cap = 0;
      MG_CK(c, cudaMalloc(&A->rec_idx, sizeof(unsigned) * 8 * (size_t)A->Np));
      MG_CK(c, cudaMalloc(&A->split_list, sizeof(int) * 8 * (size_t)((A->Np + 7) / 8 + 256)));
      A->rec_cap = A->Np;
    }
    D.rec_idx = A->rec_idx;
    D.np = A->Np;
    D.rb = rec_bits(A->nlev);
  }
  TreeView T = tree_view(A);
  k_deposit<<<nblocks(A->Np, BS), BS, 0, c->s>>>(pos, A->Np, inv, N0d, T, D,
                                                 (unsigned long long*)(A->d_small + 1),
                                                 A->split_list,
                                                 (unsigned long long*)A->d_split,
                                                 (unsigned)(per / 256));
  c->launches += 1;
  if (record) {
    LevelPtrs Ds = D;  // the split pieces add masses only (no record)
    Ds.rec_idx = nullptr;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    k_deposit_split<<<std::max(nsm, 1) * 8, BS, 0, c->s>>>(pos, inv, N0d, T, Ds,
                                                 (unsigned long long*)(A->d_small + 1),
                                                 A->split_list,
                                                 (const unsigned long long*)A->d_split, per);
    c->launches += 1;
  }
  for (int l = A->nlev - 1; l >= 1; --l) {
    k_mass_up<<<nblocks(A->L[l].n_oct, BS), BS, 0, c->s>>>(A->L[l].mass, A->L[l].n_oct,
                                                           A->L[l].pcell, A->L[l - 1].mass);
    c->launches += 1;
  }
  return MGFR_OK;
}

mgfr_status dense_solve64(mgfr_ctx* c, const Model& m, double box, mgfr_stats* st);
mgfr_status dense_solve_mixed(mgfr_ctx* c, const Model& m, double box, mgfr_stats* st, bool warm);
mgfr_status ensure_dense_public(mgfr_ctx* c, int N, bool mixed, double box);

extern "C" {

// The particle solve; acc_out is a device array, and acc_host (if not NULL)
// receives it chunk by chunk while the gather runs.
static mgfr_status check_particle_args(mgfr_ctx* c, const double* pos, long long Np, int N0,
                                       double box, double a) {
  if (!pos || Np <= 0) return set_err(c, MGFR_E_INVALID, "need Np >= 1 particle positions");
  if (Np >= (1LL << 40)) return set_err(c, MGFR_E_INVALID, "Np too large");
  if (N0 < 8 || N0 > 1024 || (N0 & (N0 - 1))) return set_err(c, MGFR_E_INVALID, "N_base must be a power of two in [8, 1024]");
  if (!(box > 0.0) || !std::isfinite(box)) return set_err(c, MGFR_E_INVALID, "box must be > 0");
  if (!(a > 0.0) || !std::isfinite(a)) return set_err(c, MGFR_E_INVALID, "a must be > 0");
  return MGFR_OK;
}

static mgfr_status solve_particles(mgfr_ctx* c, const double* pos, long long Np, int N0, double box,
                                   double a, const double* u_init, double* fr_out,
                                   double* acc_out, double* acc_host, mgfr_stats* st) {
  if (!c) return MGFR_E_INVALID;
  TRY(check_particle_args(c, pos, Np, N0, box, a));
  const mgfr_config& g = c->cfg;
  MG_CK(c, cudaSetDevice(c->device));
  if (st) std::memset(st, 0, sizeof(*st));
  c->launches = 0;
  const bool mixed = g.precision == MGFR_PREC_MIXED;
  amr_invalidate(c);  // valid again only once this solve has built its levels
  TRY(ensure_dense_public(c, N0, mixed, box));
  if (!c->amr) c->amr = new AmrWork();
  AmrWork* A = W(c);
  if (!A->d_small) MG_CK(c, cudaMalloc(&A->d_small, sizeof(long long) * 8));
  int lg0 = 0;
  while ((1 << lg0) < N0) ++lg0;
  if (A->N0 != N0) {
    for (int k = 0; k < MGFR_MAX_DENSE; ++k) {
      if (A->dmask[k]) {
        cudaFree(A->dmask[k]);
        A->dmask[k] = nullptr;
      }
      if (A->dact[k]) {
        cudaFree(A->dact[k]);
        A->dact[k] = nullptr;
      }
      if (A->dlist[k]) {
        cudaFree(A->dlist[k]);
        A->dlist[k] = nullptr;
      }
    }
    if (A->acc0) cudaFree(A->acc0);
    if (A->fr0) cudaFree(A->fr0);
    if (A->acc0_32) cudaFree(A->acc0_32);
    A->acc0 = A->fr0 = nullptr;
    A->acc0_32 = nullptr;
  }
  A->N0 = N0;
  A->lg0 = lg0;
  A->box = box;
  A->Np = Np;
  DenseHier& H = c->dh;
  for (int k = 1; k < H.nlev; ++k) {
    if (!A->dmask[k]) MG_CK(c, cudaMalloc(&A->dmask[k], sizeof(float) * (size_t)H.L[k].n));
    if (!A->dact[k]) MG_CK(c, cudaMalloc(&A->dact[k], (size_t)H.L[k].n));
  }
  for (int k = 0; k < H.nlev; ++k)
    if (!A->dlist[k]) MG_CK(c, cudaMalloc(&A->dlist[k], sizeof(int) * (size_t)H.L[k].n));
  if (!A->acc0) MG_CK(c, cudaMalloc(&A->acc0, sizeof(double) * 3 * (size_t)H.L[0].n));
  if (!A->fr0) MG_CK(c, cudaMalloc(&A->fr0, sizeof(double) * (size_t)H.L[0].n));
  if (mixed && !A->acc0_32)
    MG_CK(c, cudaMalloc(&A->acc0_32, sizeof(float4) * (size_t)H.L[0].n));
  auto w0 = std::chrono::steady_clock::now();
  MG_CK(c, cudaEventRecord(c->ev_in, c->user));
  MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_in, 0));
  MG_CK(c, cudaMemsetAsync(A->d_small, 0, sizeof(long long) * 8, c->s));
  k_nan_check<<<nblocks(3 * Np, BS), BS, 0, c->s>>>(pos, 3 * Np, (unsigned long long*)(A->d_small + 1));
  c->launches += 1;
  // structure, deposit, sources
  TRY(build_structure(c, A, pos));
  // the FP32 gather of the mixed form replays the deposit's record; with a
  // host destination it runs (and is copied back) in 8 chunks
  const int nch = acc_host ? 8 : 1;
  const long long per = ((Np + nch - 1) / nch + 255) / 256 * 256;
  TRY(deposit(c, A, pos, mixed && acc_out, per));
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
  if (A->rec_on)
    MG_CK(c, cudaMemcpyAsync(A->n_split, A->d_split, sizeof(long long) * 8,
                             cudaMemcpyDeviceToHost, c->s));
  MG_CK(c, cudaStreamSynchronize(c->s));
  if (flags & 2) return set_err(c, MGFR_E_INVALID, "non-finite particle position");
  if (flags & 1) return set_err(c, MGFR_E_UNSUPPORTED, "cloud-in-cell split stack overflow");
  // base level (the learned start predicts it from delta = f / src)
  DenseLevel& L0 = H.L[0];
  const double* u0 = nullptr;
  TRY(start_guess(c, N0, L0.f, 1.0 / m.src, u_init, &u0));
  f64::init_u(u0, L0.u, L0.E, L0.n, c->s);
  c->u_prev_N = 0;  // valid again once the base level is solved
  c->launches += 1;
  MG_CK(c, cudaEventRecord(c->t0, c->s));
  mgfr_status rs =
      mixed ? dense_solve_mixed(c, m, box, st, u0 != nullptr) : dense_solve64(c, m, box, st);
  if (rs != MGFR_OK && rs != MGFR_E_NOCONVERGE) return rs;
  c->u_prev_N = N0;  // the refined levels never write the base level's u
  mgfr_status worst = rs;
  for (int l = 1; l < A->nlev; ++l) {
    mgfr_status ls = amr_solve_level(c, A, l, m, st);
    if (ls != MGFR_OK && ls != MGFR_E_NOCONVERGE) return ls;
    if (ls != MGFR_OK) worst = ls;
  }
  TRY(amr_keep_previous(c, A, g.start == MGFR_START_PREVIOUS_ALL));
  MG_CK(c, cudaEventRecord(c->t1, c->s));
  // force per level, then at the particles
  f64::force(L0, m, A->fr0, A->acc0, c->s);
  c->launches += 1;
  if (fr_out)
    MG_CK(c, cudaMemcpyAsync(fr_out, A->fr0, sizeof(double) * (size_t)L0.n,
                             cudaMemcpyDeviceToDevice, c->s));
  // the mixed form gathers FP32 copies of the force fields with FP32 weights
  const bool g32 = mixed && acc_out;
  GatherPtrs G{};
  G.acc[0] = A->acc0;
  G.acc32[0] = A->acc0_32;
  G.n0 = L0.n;
  if (g32) {
    k_acc_pack<<<nblocks(L0.n, BS), BS, 0, c->s>>>(A->acc0, L0.n, A->acc0_32);
    c->launches += 1;
  }
  A->fbar = m.fbar;
  A->omega_m = g.omega_m;
  A->nexp = g.n;
  A->a = m.a;
  for (int l = 1; l < A->nlev; ++l) {
    AmrLevel& L = A->L[l];
    const double gs = m.fbar / (2.0 * L.h) / (2.0 * m.a);
    if (g32 && L.wE_df && L.ghost_df) {
      // mixed form: the FP32 force copy straight from the double-float e^u; the
      // FP64 f_R and force of the level are formed on request
      k_oct_acc32_df<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(
          reinterpret_cast<const dfl*>(L.wE), L.nbr, reinterpret_cast<const dfl*>(L.ghostE),
          L.ncell, (float)gs, L.acc32);
      L.force_stale = true;
    } else {
      k_oct_force<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.E, L.nbr, L.ghostE,
                                                         L.ghost_df ? 1 : 0, L.ncell, m.fbar, gs,
                                                         L.w, L.acc, g32 ? L.acc32 : nullptr);
      L.force_stale = false;
    }
    G.acc[l] = L.acc;
    G.acc32[l] = L.acc32;
    c->launches += 1;
  }
  if (acc_out) {
    TreeView T = tree_view(A);
    // FP32 gather from the deposit's record, per chunk: the particles whose
    // cube split (full traversal), then the rest from their recorded cells.
    // With a host destination each chunk is copied back on the copy stream
    // while the next one is gathered.
    const bool replay = g32 && A->rec_on;
    for (int q = 0; q < nch; ++q) {
      const long long p0 = q * per, n = std::min(per, Np - p0);
      if (n <= 0) break;
      if (replay && A->n_split[q] > 0) {
        k_gather32_list<<<nblocks(A->n_split[q], BS), BS, 0, c->s>>>(
            pos, A->split_list + q * per, A->n_split[q], (double)N0 / box, (double)N0, T, G,
            acc_out, (unsigned long long*)(A->d_small + 1));
        c->launches += 1;
      }
      if (replay)
        k_gather32_rec<<<nblocks(n, BS), BS, 0, c->s>>>(pos, A->rec_idx, Np,
                                                        rec_bits(A->nlev), p0, n,
                                                        (double)N0 / box, (double)N0, G, acc_out);
      else if (g32)
        k_gather32<<<nblocks(n, BS), BS, 0, c->s>>>(pos + 3 * p0, n, (double)N0 / box, (double)N0,
                                                    T, G, acc_out + 3 * p0,
                                                    (unsigned long long*)(A->d_small + 1));
      else
        k_gather<<<nblocks(n, BS), BS, 0, c->s>>>(pos + 3 * p0, n, (double)N0 / box, (double)N0, T,
                                                  G, acc_out + 3 * p0,
                                                  (unsigned long long*)(A->d_small + 1));
      c->launches += 1;
      if (acc_host) {
        MG_CK(c, cudaEventRecord(c->ev_chunk[q], c->s));
        MG_CK(c, cudaStreamWaitEvent(c->cs, c->ev_chunk[q], 0));
        MG_CK(c, cudaMemcpyAsync(acc_host + 3 * p0, acc_out + 3 * p0, sizeof(double) * 3 * (size_t)n,
                                 cudaMemcpyDeviceToHost, c->cs));
      }
    }
    if (acc_host) {
      MG_CK(c, cudaEventRecord(c->ev_copy, c->cs));
      MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_copy, 0));
    }
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

mgfr_status mgfr_solve_particles(mgfr_ctx* c, const double* pos, long long Np, int N0, double box,
                                 double a, const double* u_init, double* fr_out, double* acc_out,
                                 mgfr_stats* st) {
  return solve_particles(c, pos, Np, N0, box, a, u_init, fr_out, acc_out, nullptr, st);
}

mgfr_status mgfr_solve_particles_host(mgfr_ctx* c, const double* pos_host, long long Np, int N0,
                                      double box, double a, const double* u_init, double* fr_out,
                                      double* acc_host, mgfr_stats* st) {
  if (!c) return MGFR_E_INVALID;
  TRY(check_particle_args(c, pos_host, Np, N0, box, a));
  if (!acc_host) return set_err(c, MGFR_E_INVALID, "acc_out_host is required");
  MG_CK(c, cudaSetDevice(c->device));
  if (!c->cs) {
    MG_CK(c, cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking));
    for (auto& ev : c->ev_chunk) MG_CK(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    MG_CK(c, cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming));
  }
  if (!c->amr) c->amr = new AmrWork();
  AmrWork* A = W(c);
  if (Np > A->pio_cap) {
    if (A->pos_dev) cudaFree(A->pos_dev);
    if (A->acc_dev) cudaFree(A->acc_dev);
    A->pos_dev = A->acc_dev = nullptr;
    A->pio_cap = 0;
    MG_CK(c, cudaMalloc(&A->pos_dev, sizeof(double) * 3 * (size_t)Np));
    MG_CK(c, cudaMalloc(&A->acc_dev, sizeof(double) * 3 * (size_t)Np));
    A->pio_cap = Np;
  }
  // in the caller's stream order
  MG_CK(c, cudaEventRecord(c->ev_in, c->user));
  MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_in, 0));
  MG_CK(c, cudaMemcpyAsync(A->pos_dev, pos_host, sizeof(double) * 3 * (size_t)Np,
                           cudaMemcpyHostToDevice, c->s));
  const mgfr_status rs =
      solve_particles(c, A->pos_dev, Np, N0, box, a, u_init, fr_out, A->acc_dev, acc_host, st);
  if (rs != MGFR_OK && rs != MGFR_E_NOCONVERGE) {
    // the host arrays may still be in use by copies queued before the error
    cudaStreamSynchronize(c->s);
    if (c->cs) cudaStreamSynchronize(c->cs);
  }
  return rs;
}

static EffPar eff_par(const AmrWork* A, int l) {
  const double Nl = (double)(1LL << (A->lg0 + l));
  const double a3 = A->a * A->a * A->a, rho = A->omega_m / a3;
  const double Rt = rho + 4.0 * (1.0 - A->omega_m);
  return EffPar{Nl * Nl * Nl / (double)A->Np, Rt / (3.0 * rho), 1.0 / (A->nexp + 1)};
}

mgfr_status mgfr_get_effective_density(mgfr_ctx* c, int level, double* out_dev) {
  if (!c || !out_dev) return MGFR_E_INVALID;
  AmrWork* A = W(c);
  if (!A || A->nlev == 0 || level < 0 || level >= A->nlev)
    return set_err(c, MGFR_E_INVALID, "no such level of a particle solve");
  MG_CK(c, cudaSetDevice(c->device));
  // out_dev is written in the caller's stream order
  MG_CK(c, cudaEventRecord(c->ev_in, c->user));
  MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_in, 0));
  AmrLevel& L = A->L[level];
  const double* u = level == 0 ? c->dh.L[0].u : L.u;
  k_eff_level<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.mass, u, L.ncell, eff_par(A, level),
                                                     out_dev);
  MG_CK(c, cudaEventRecord(c->ev_out, c->s));
  MG_CK(c, cudaStreamWaitEvent(c->user, c->ev_out, 0));
  MG_CK(c, cudaGetLastError());
  return MGFR_OK;
}

}  // extern "C"

mgfr_status amr_density_pm(mgfr_ctx* c, int lpm, int what, double* out_dev, int* lg_pm,
                           double* omega_m, double* a) {
  AmrWork* A = W(c);
  if (!A || A->nlev == 0) return set_err(c, MGFR_E_INVALID, "no particle solve yet");
  if (lpm < 0 || A->lg0 + lpm > 10) return set_err(c, MGFR_E_INVALID, "PM grid of 2^0..2^10 cells per axis");
  if (what < 0 || what > 2) return set_err(c, MGFR_E_INVALID, "what: 0 effective, 1 matter, 2 total");
  if (lg_pm) *lg_pm = A->lg0 + lpm;
  if (omega_m) *omega_m = A->omega_m;
  if (a) *a = A->a;
  if (!out_dev) return MGFR_OK;
  const long long Npm = 1LL << (A->lg0 + lpm);
  MG_CK(c, cudaMemsetAsync(out_dev, 0, sizeof(double) * (size_t)(Npm * Npm * Npm), c->s));
  TreeView T = tree_view(A);
  for (int l = 0; l < A->nlev; ++l) {
    AmrLevel& L = A->L[l];
    const double* u = l == 0 ? c->dh.L[0].u : L.u;
    k_eff_pm<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(l, lpm, T, L.mass, u, L.ncell,
                                                    eff_par(A, l), what, out_dev);
    c->launches += 1;
  }
  return MGFR_OK;
}

extern "C" {

mgfr_status mgfr_effective_mass_pm(mgfr_ctx* c, int lpm, double* out_dev) {
  if (!c || !out_dev) return MGFR_E_INVALID;
  TRY(amr_density_pm(c, lpm, 0, nullptr, nullptr, nullptr, nullptr));  // checks only
  MG_CK(c, cudaSetDevice(c->device));
  MG_CK(c, cudaEventRecord(c->ev_in, c->user));
  MG_CK(c, cudaStreamWaitEvent(c->s, c->ev_in, 0));
  TRY(amr_density_pm(c, lpm, 0, out_dev, nullptr, nullptr, nullptr));
  MG_CK(c, cudaEventRecord(c->ev_out, c->s));
  MG_CK(c, cudaStreamWaitEvent(c->user, c->ev_out, 0));
  MG_CK(c, cudaGetLastError());
  return MGFR_OK;
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
    case MGFR_FIELD_FR:
    case MGFR_FIELD_ACC:
      if (level >= 1 && L.force_stale) {  // deferred in the mixed form: form it now
        const double gs = A->fbar / (2.0 * L.h) / (2.0 * A->a);
        k_oct_force<<<nblocks(L.ncell, BS), BS, 0, c->s>>>(L.E, L.nbr, L.ghostE,
                                                           L.ghost_df ? 1 : 0, L.ncell, A->fbar,
                                                           gs, L.w, L.acc, nullptr);
        MG_CK(c, cudaStreamSynchronize(c->s));
        MG_CK(c, cudaGetLastError());
        L.force_stale = false;
      }
      if (what == MGFR_FIELD_FR) {
        src = level == 0 ? A->fr0 : L.w;
      } else {
        src = level == 0 ? A->acc0 : L.acc;
        cnt = 3 * n;
      }
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
