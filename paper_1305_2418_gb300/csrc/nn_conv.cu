// nn_conv.cu -- 3^3 convolutions on BF16 tensor cores (mma.sync m16n8k16,
// FP32 accumulation), circular padding, NDHWC activations.
//
// Forward and input-gradient are one implicit GEMM: rows = voxels, columns =
// output channels, reduction = (tap, input channel).  Per tap the weight
// slice is staged in shared memory as [n][k] (k contiguous) so B fragments
// are 32-bit shared loads; A fragments are gathered straight from the
// activation tensor (each row is the contiguous channel vector of one
// neighbour voxel).  The input-gradient uses the mirrored tap and the
// transposed weight slice.  The weight gradient is a GEMM over voxels with
// both operands staged transposed (voxel index contiguous) in shared memory;
// per-chunk partial sums are reduced by a second kernel (deterministic).
// The network's own channel pairs run on the tcgen05 kernels of nn_tc.cu;
// these serve the others.  nn_wgrad_finish (the reduction of the partial dW
// and the bias gradient) serves both.
#include <algorithm>

#include "nn_kernels.cuh"

namespace {

__device__ __forceinline__ void mma16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const unsigned*>(p);
}

// neighbour voxel of m at offset (dx,dy,dz), periodic in each sample
__device__ __forceinline__ long long nbr_vox(long long m, int lgD, int dx, int dy, int dz) {
  const int D = 1 << lgD, M = D - 1;
  const long long per = 1LL << (3 * lgD);
  const long long b = m >> (3 * lgD), r = m & (per - 1);
  const int i = (int)(r >> (2 * lgD)), j = (int)((r >> lgD) & M), k = (int)(r & M);
  return b * per + ((((long long)((i + dx) & M) << lgD) + ((j + dy) & M)) << lgD) + ((k + dz) & M);
}

constexpr int KPAD = 8;

// DGRAD = false: y[m][n] = sum_{tap,k} x[m + tap][k] W[tap][k][n]      (n = co)
// DGRAD = true : gx[m][n] = sum_{tap,k} g[m - tap][k] W[tap][n][k]     (n = ci)
template <int NT, bool DGRAD>
__global__ void __launch_bounds__(128) k_conv(const __nv_bfloat16* __restrict__ x, int ldx, int offx,
                                              int K, const __nv_bfloat16* __restrict__ W, int Cin,
                                              int Cout, const float* __restrict__ bias, int relu,
                                              __nv_bfloat16* __restrict__ y, int ldy, int offy,
                                              float* __restrict__ gx, int ldg, int offg,
                                              int accumulate, int lgD) {
  extern __shared__ __nv_bfloat16 Ws[];  // [NT*8][K + KPAD]
  const int KP = K + KPAD;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int n0 = blockIdx.y * NT * 8;
  const long long m0 = ((long long)blockIdx.x * 4 + warp) * 16;
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    const int dx = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dz = tap % 3 - 1;
    __syncthreads();
    // stage the weight slice [n][k] of this tap
    for (int e = threadIdx.x; e < NT * 8 * K; e += blockDim.x) {
      const int n = e / K, k = e % K;
      const __nv_bfloat16 v = DGRAD ? W[((long long)tap * Cin + (n0 + n)) * Cout + k]
                                    : W[((long long)tap * Cin + k) * Cout + (n0 + n)];
      Ws[n * KP + k] = v;
    }
    __syncthreads();
    const long long r0 = DGRAD ? nbr_vox(m0 + gid, lgD, -dx, -dy, -dz)
                               : nbr_vox(m0 + gid, lgD, dx, dy, dz);
    const long long r1 = DGRAD ? nbr_vox(m0 + gid + 8, lgD, -dx, -dy, -dz)
                               : nbr_vox(m0 + gid + 8, lgD, dx, dy, dz);
    const __nv_bfloat16* x0 = x + r0 * ldx + offx + tig * 2;
    const __nv_bfloat16* x1 = x + r1 * ldx + offx + tig * 2;
    for (int kc = 0; kc < K; kc += 16) {
      unsigned a[4];
      a[0] = ld32(x0 + kc);
      a[1] = ld32(x1 + kc);
      a[2] = ld32(x0 + kc + 8);
      a[3] = ld32(x1 + kc + 8);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const __nv_bfloat16* wp = Ws + (t * 8 + gid) * KP + kc + tig * 2;
        unsigned b[2] = {ld32(wp), ld32(wp + 8)};
        mma16816(acc[t], a, b);
      }
    }
  }
  // epilogue: rows gid, gid+8; columns t*8 + tig*2 + {0,1}
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int n = n0 + t * 8 + tig * 2;
    for (int h = 0; h < 2; ++h) {
      const long long m = m0 + gid + 8 * h;
      float v0 = acc[t][2 * h], v1 = acc[t][2 * h + 1];
      if (!DGRAD) {
        if (bias) {
          v0 += bias[n];
          v1 += bias[n + 1];
        }
        if (relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        __nv_bfloat162 o;
        o.x = __float2bfloat16(v0);
        o.y = __float2bfloat16(v1);
        *reinterpret_cast<__nv_bfloat162*>(y + m * ldy + offy + n) = o;
      } else {
        float* q = gx + m * ldg + offg + n;
        if (accumulate) {
          q[0] += v0;
          q[1] += v1;
        } else {
          q[0] = v0;
          q[1] = v1;
        }
      }
    }
  }
}

// weight gradient partials: block (tap, 16-row ci tile, voxel chunk z)
template <int NT>
__global__ void __launch_bounds__(128) k_wgrad(const __nv_bfloat16* __restrict__ x, int ldx, int offx,
                                               int Cin, const __nv_bfloat16* __restrict__ g, int ldg,
                                               int offg, int Cout, float* __restrict__ partials,
                                               long long Mtot, long long chunk, int lgD) {
  constexpr int MC = 64;  // voxels per staging step
  constexpr int STAGE_BYTES = (16 + NT * 8) * (MC + KPAD) * 2;
  constexpr int RED_BYTES = 4 * 16 * NT * 8 * 4;
  __shared__ __align__(16) unsigned char raw[STAGE_BYTES > RED_BYTES ? STAGE_BYTES : RED_BYTES];
  auto Xs = reinterpret_cast<__nv_bfloat16(*)[MC + KPAD]>(raw);
  auto Gs = reinterpret_cast<__nv_bfloat16(*)[MC + KPAD]>(raw + 16 * (MC + KPAD) * 2);
  auto red = reinterpret_cast<float(*)[16 * NT * 8]>(raw);
  const int tap = blockIdx.x, ci0 = blockIdx.y * 16;
  const int dx = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dz = tap % 3 - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
  const long long mbeg = (long long)blockIdx.z * chunk;
  const long long mend = min(Mtot, mbeg + chunk);
  for (long long mb = mbeg; mb < mend; mb += MC) {
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * MC; e += blockDim.x) {
      const int mm = e >> 4, ci = e & 15;
      const long long m = mb + mm;
      Xs[ci][mm] = m < mend ? x[nbr_vox(m, lgD, dx, dy, dz) * ldx + offx + ci0 + ci]
                            : __float2bfloat16(0.f);
    }
    for (int e = threadIdx.x; e < NT * 8 * MC; e += blockDim.x) {
      const int mm = e / (NT * 8), co = e % (NT * 8);
      const long long m = mb + mm;
      Gs[co][mm] = m < mend ? g[m * ldg + offg + co] : __float2bfloat16(0.f);
    }
    __syncthreads();
    const int k0 = warp * 16;
    unsigned a[4];
    a[0] = ld32(&Xs[gid][k0 + tig * 2]);
    a[1] = ld32(&Xs[gid + 8][k0 + tig * 2]);
    a[2] = ld32(&Xs[gid][k0 + tig * 2 + 8]);
    a[3] = ld32(&Xs[gid + 8][k0 + tig * 2 + 8]);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      unsigned b[2] = {ld32(&Gs[t * 8 + gid][k0 + tig * 2]), ld32(&Gs[t * 8 + gid][k0 + tig * 2 + 8])};
      mma16816(acc[t], a, b);
    }
  }
  // reduce the 4 warps' partial tiles (the staging buffers are reused)
  __syncthreads();
#pragma unroll
  for (int t = 0; t < NT; ++t)
    for (int h = 0; h < 2; ++h) {
      const int row = gid + 8 * h, col = t * 8 + tig * 2;
      red[warp][row * NT * 8 + col] = acc[t][2 * h];
      red[warp][row * NT * 8 + col + 1] = acc[t][2 * h + 1];
    }
  __syncthreads();
  for (int e = threadIdx.x; e < 16 * NT * 8; e += blockDim.x) {
    const float v = red[0][e] + red[1][e] + red[2][e] + red[3][e];
    const int row = e / (NT * 8), col = e % (NT * 8);
    partials[(((long long)blockIdx.z * 27 + tap) * Cin + ci0 + row) * Cout + col] = v;
  }
}

__global__ void k_wgrad_reduce(const float* __restrict__ partials, int S, long long n,
                               float* __restrict__ dW) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int z = 0; z < S; ++z) s += partials[(long long)z * n + i];
  dW[i] = s;
}

// db[c] = sum over voxels of g[m][c].  The additions follow one fixed order:
// for each slot t < 256 the voxels m = t, t + 256, t + 512, ... in turn, then
// a pairwise tree over the 256 slot sums (stride 128, 64, ..., 1).  Stage 1
// gives every (slot, channel) pair its own thread (consecutive threads take
// consecutive channels of one voxel, so a warp's loads are contiguous) and
// keeps 32 loads of the chain in flight; stage 2 runs the tree, one block
// per channel.
constexpr int BG_SLOTS = 256;

__global__ void __launch_bounds__(128) k_bias_slots(const __nv_bfloat16* __restrict__ g, int ldg,
                                                    int offg, long long Mtot, int Cout,
                                                    float* __restrict__ part) {
  const long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (T >= (long long)BG_SLOTS * Cout) return;
  const int c = (int)(T % Cout), t = (int)(T / Cout);
  constexpr int U = 32;
  float s = 0.f;
  long long m = t;
  for (; m + (U - 1) * (long long)BG_SLOTS < Mtot; m += U * (long long)BG_SLOTS) {
    float v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) v[q] = __bfloat162float(g[(m + q * BG_SLOTS) * ldg + offg + c]);
#pragma unroll
    for (int q = 0; q < U; ++q) s += v[q];
  }
  for (; m < Mtot; m += BG_SLOTS) s += __bfloat162float(g[m * ldg + offg + c]);
  part[(long long)t * Cout + c] = s;
}

__global__ void __launch_bounds__(BG_SLOTS) k_bias_tree(const float* __restrict__ part, int Cout,
                                                        float* __restrict__ db) {
  __shared__ float red[BG_SLOTS];
  const int c = blockIdx.x, t = threadIdx.x;
  red[t] = part[(long long)t * Cout + c];
  __syncthreads();
  for (int w = BG_SLOTS / 2; w > 0; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  if (t == 0) db[c] = red[0];
}

constexpr int WG_S_TARGET = 608;  // about 4 blocks per SM of partial tiles

int pick_nt(int n) { return n % 64 == 0 ? 8 : (n % 32 == 0 ? 4 : 2); }

}  // namespace

void nn_conv_fwd(TView x, int Cin, const __nv_bfloat16* W, const float* bias, int relu, TView y,
                 int Cout, int B, int lgD, cudaStream_t s) {
  const long long Mtot = (long long)B << (3 * lgD);
  const int nt = pick_nt(Cout);
  dim3 grid((unsigned)(Mtot / 64), Cout / (nt * 8));
  const size_t smem = sizeof(__nv_bfloat16) * nt * 8 * (Cin + KPAD);
#define LAUNCH_F(NT)                                                                            \
  k_conv<NT, false><<<grid, 128, smem, s>>>(x.p, x.ld, x.off, Cin, W, Cin, Cout, bias, relu,    \
                                            y.p, y.ld, y.off, nullptr, 0, 0, 0, lgD)
  if (nt == 8) LAUNCH_F(8); else if (nt == 4) LAUNCH_F(4); else LAUNCH_F(2);
#undef LAUNCH_F
}

void nn_conv_dgrad(TView g, int Cout, const __nv_bfloat16* W, FView gx, int Cin, int accumulate,
                   int B, int lgD, cudaStream_t s) {
  const long long Mtot = (long long)B << (3 * lgD);
  const int nt = pick_nt(Cin);
  dim3 grid((unsigned)(Mtot / 64), Cin / (nt * 8));
  const size_t smem = sizeof(__nv_bfloat16) * nt * 8 * (Cout + KPAD);
#define LAUNCH_D(NT)                                                                            \
  k_conv<NT, true><<<grid, 128, smem, s>>>(g.p, g.ld, g.off, Cout, W, Cin, Cout, nullptr, 0,    \
                                           nullptr, 0, 0, gx.p, gx.ld, gx.off, accumulate, lgD)
  if (nt == 8) LAUNCH_D(8); else if (nt == 4) LAUNCH_D(4); else LAUNCH_D(2);
#undef LAUNCH_D
}

void nn_wgrad_finish(float* partials, int S, int Cin, int Cout, float* dW, TView g,
                     float* db, long long Mtot, cudaStream_t s) {
  const long long n = 27LL * Cin * Cout;
  k_wgrad_reduce<<<nblocks(n, 256), 256, 0, s>>>(partials, S, n, dW);
  if (!db) return;
  // the bias stages reuse the partials (read by k_wgrad_reduce before them on
  // this stream); they hold S * 27 * Cin * Cout >= 432 * Cout floats (Cin >= 16)
  const long long nt = (long long)BG_SLOTS * Cout;
  k_bias_slots<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(g.p, g.ld, g.off, Mtot, Cout, partials);
  k_bias_tree<<<Cout, BG_SLOTS, 0, s>>>(partials, Cout, db);
}

long long nn_wgrad_scratch(int Cin, int Cout) {
  const int S = std::max(1, WG_S_TARGET / (27 * (Cin / 16)));
  return (long long)S * 27 * Cin * Cout;
}

void nn_conv_wgrad(TView x, int Cin, TView g, int Cout, float* dW, float* db, float* partials,
                   int B, int lgD, cudaStream_t s) {
  const long long Mtot = (long long)B << (3 * lgD);
  const int S = std::max(1, WG_S_TARGET / (27 * (Cin / 16)));
  const long long chunk = ((Mtot + S - 1) / S + 63) / 64 * 64;
  dim3 grid(27, Cin / 16, S);
  // Cout in {16, 32, 64, 128}: one launch covers all output channels
#define LAUNCH_W(NT)                                                                            \
  k_wgrad<NT><<<grid, 128, 0, s>>>(x.p, x.ld, x.off, Cin, g.p, g.ld, g.off, Cout, partials, Mtot, \
                                   chunk, lgD)
  switch (Cout / 8) {
    case 2: LAUNCH_W(2); break;
    case 4: LAUNCH_W(4); break;
    case 8: LAUNCH_W(8); break;
    default: LAUNCH_W(16); break;
  }
#undef LAUNCH_W
  nn_wgrad_finish(partials, S, Cin, Cout, dW, g, db, Mtot, s);
}
