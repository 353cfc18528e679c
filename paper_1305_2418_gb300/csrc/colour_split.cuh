// colour_split.cuh -- index maps of the colour-split FP32 storage.  The
// red-black colour of a cell is the parity of its coordinates; every FP32
// array of the solver is stored by colour so that a half-sweep moves whole
// vectors of the colours it reads and writes.  The same code compiles as host
// C++ for testing.
#pragma once

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

#ifdef __CUDA_ARCH__
#define CS_POPC(x) __popc(x)
#else
#define CS_POPC(x) __builtin_popcount(x)
#endif

// ---- dense levels (N = 2^lg, 2 <= lg <= 10) --------------------------------
// Plane q = (i + j + k) & 1 holds the cells of that colour, in C order of
// (i, j, k >> 1).  The six neighbours of a cell all lie in the other plane,
// four of them at the same (k >> 1) in neighbouring rows and two in the same
// row (at k >> 1 and one step along it).
__host__ __device__ __forceinline__ unsigned prow(int i, int j, int lg) {
  return (((unsigned)i << lg) + (unsigned)j) << (lg - 1);
}
// colour-split index of (i, j, k), each in [0, N)
__host__ __device__ __forceinline__ unsigned pdx(int i, int j, int k, int lg) {
  return ((unsigned)((i + j + k) & 1) << (3 * lg - 1)) + prow(i, j, lg) + ((unsigned)k >> 1);
}
// cell of colour-split index t
__host__ __device__ __forceinline__ void pcell(unsigned t, int lg, int* i, int* j, int* k) {
  const int M = (1 << lg) - 1;
  const unsigned q = t >> (3 * lg - 1);
  const unsigned p = t & ((1u << (3 * lg - 1)) - 1u);
  *i = (int)(p >> (2 * lg - 1));
  *j = (int)((p >> (lg - 1)) & M);
  *k = 2 * (int)(p & (M >> 1)) + (int)((q + *i + *j) & 1);
}
// colour-split indices of the six periodic neighbours (-x, +x, -y, +y, -z, +z)
__host__ __device__ __forceinline__ void pnb6(int i, int j, int k, int lg, unsigned* q) {
  const int M = (1 << lg) - 1, hm = M >> 1;
  const unsigned ob = (unsigned)((i + j + k + 1) & 1) << (3 * lg - 1);
  const int kh = k >> 1;
  q[0] = ob + prow((i - 1) & M, j, lg) + kh;
  q[1] = ob + prow((i + 1) & M, j, lg) + kh;
  q[2] = ob + prow(i, (j - 1) & M, lg) + kh;
  q[3] = ob + prow(i, (j + 1) & M, lg) + kh;
  const unsigned r = ob + prow(i, j, lg);
  q[4] = r + ((k & 1) ? kh : ((kh - 1) & hm));
  q[5] = r + ((k & 1) ? ((kh + 1) & hm) : kh);
}

// ---- oct levels --------------------------------------------------------------
// Plane k (k = 0, 1) holds, for every oct o, the four cells of colour k as one
// float4 at floats (k n_oct + o) 4.  The colour is the parity of the
// child-index bits (parent coordinates contribute an even amount), and a
// cell's place in its float4 is ch >> 1 (colour 0: children 0, 3, 5, 6;
// colour 1: 1, 2, 4, 7).  n_oct = 0 marks a dense level (C order).
__host__ __device__ __forceinline__ long long pidx(long long c, long long n_oct) {
  if (n_oct == 0) return c;
  const int ch = (int)(c & 7);
  return (((long long)(CS_POPC(ch) & 1) * n_oct + (c >> 3)) << 2) + (ch >> 1);
}
