// nn_tc.cu -- the network's 3^3 convolutions (forward, input gradient and
// weight gradient) on the fifth-generation tensor cores: tcgen05.mma with the
// FP32 accumulator in tensor memory (TMEM), BF16 operands in shared memory.
// Three forms: the per-tap kernel (k_conv_tc, below), the halo-tiled kernels
// of the full- and second-resolution layers (k_conv_halo, k_conv_halo_s: the
// input block with its one-voxel halo staged once per CTA, each tap a shifted
// descriptor into it) and the weight gradient (k_wgrad_tc).
//
// Implicit GEMM per CTA (128 threads): rows = an M tile of 128 consecutive
// voxels, columns = all N output channels (N <= 256), reduction = 27 taps x
// the K input channels.  Per tap:
//   A (128 x K): each row the channel vector of the row voxel's neighbour at
//     the tap offset (periodic), copied by cp.async in 16-byte chunks;
//   B (N x K): the tap's weight slice, packed in advance in the shared-memory
//     layout and brought in by one bulk asynchronous copy (cp.async.bulk,
//     completion counted on an mbarrier).
// Both tiles use the canonical K-major layout without swizzle: core matrices
// of 8 rows x 16 bytes; for each 8-channel chunk the rows are contiguous (so
// the 8-row groups are 128 B apart: SBO), and the chunks follow each other one
// tile-height apart (LBO).  Thread 0 issues the tap's MMAs (K = 16 each) and
// commits them to the stage's mbarrier; two stages overlap the copies of tap
// t+1 with the MMAs of tap t.  The epilogue reads the accumulator with
// tcgen05.ld (warp w its 32 TMEM lanes = rows 32w..32w+31).
//
// Forward: y[m][co] = sum_{tap,ci} x[m + d_tap][ci] W[tap][ci][co] (+bias,
// ReLU), stored BF16.  Input gradient: gx[m][ci] = sum_{tap,co}
// g[m - d_tap][co] W[tap][ci][co], stored (or added) FP32.
//
// Weight gradient (k_wgrad_tc): dW[t][ci][co] = sum_v x[v][ci] g[v - d_t][co]
// as the transposed GEMM rows = (tap, co) (128 / Cout taps per CTA), columns
// = ci, reduction = voxels.  Both operands are then contiguous along their
// row index in the NDHWC tensors (the channels), so they are staged in the
// MN-major canonical layout (core matrices of 8 voxels x 16 bytes of
// channels) by 16-byte cp.async copies, without a transpose.  The voxels are
// split over CTAs; each CTA writes its partial dW, reduced in a fixed order.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets *err and the
// CTA leaves through the normal exit (TMEM freed).
#include <algorithm>
#include <cstdint>

#include "nn_kernels.cuh"

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;
constexpr long long kSpin = 1LL << 22;  // try_wait rounds before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the completion of the phase with this parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long long i = 0; i < kSpin; ++i)
    if (mbar_try(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // 0: fill with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// one bulk copy global -> shared, its bytes counted on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// canonical K-major shared-memory descriptor, no swizzle (version 1)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor: BF16 x BF16 -> FP32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// MN-major operands without swizzle: the field at bits 32-45 (SBO) holds the
// stride between core matrices along M (or N), the field at bits 16-29 (LBO)
// the stride between core matrices along K
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t mn_stride,
                                             uint32_t k_stride) {
  return sdesc(saddr, k_stride, mn_stride);
}

// instruction descriptor: BF16 x BF16 -> FP32, A and B MN-major (bits 15, 16)
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) {
  return idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// neighbour voxel of m at offset (dx,dy,dz), periodic in each sample
__device__ __forceinline__ long long tc_nbr(long long m, int lgD, int dx, int dy, int dz) {
  const int D = 1 << lgD, M = D - 1;
  const long long per = 1LL << (3 * lgD);
  const long long b = m >> (3 * lgD), r = m & (per - 1);
  const int i = (int)(r >> (2 * lgD)), j = (int)((r >> lgD) & M), k = (int)(r & M);
  return b * per + ((((long long)((i + dx) & M) << lgD) + ((j + dy) & M)) << lgD) + ((k + dz) & M);
}

// KC: channels of an A row (the reduction per tap); NC: output columns.
// DGRAD: the input-gradient form (mirrored tap, FP32 output, optional add).
template <int KC, int NC, bool DGRAD>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(
    const __nv_bfloat16* __restrict__ x, int ldx, int offx, const __nv_bfloat16* __restrict__ Wp,
    const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ y, int ldy, int offy,
    float* __restrict__ gx, int ldg, int offg, int accumulate, int lgD, long long Mtot,
    int tmem_cols, int* __restrict__ err) {
  constexpr int A_BYTES = TC_M * KC * 2, B_BYTES = NC * KC * 2;
  constexpr uint32_t A_LBO = TC_M * 16, B_LBO = NC * 16, SBO = 128;
  constexpr uint32_t IDESC = idesc_bf16(TC_M, NC);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;                        // [2][A_BYTES]
  unsigned char* Bs = smem + 2 * A_BYTES;          // [2][B_BYTES]
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + 2 * B_BYTES);  // full[2], done[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long m0 = (long long)blockIdx.x * TC_M;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(bars + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  bool ok = true;

  // A copies of tap t into stage s (every thread a share of the 16-byte chunks)
  auto load_a = [&](int t, int s) {
    const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
    const int sg = DGRAD ? -1 : 1;
    unsigned char* A = As + s * A_BYTES;
    constexpr int CH = KC / 8;  // 16-byte chunks per row
    for (int e = tid; e < TC_M * CH; e += TC_THREADS) {
      const int r = e / CH, c = e - r * CH;
      const long long m = m0 + r;
      const bool v = m < Mtot;
      const long long src = v ? tc_nbr(m, lgD, sg * dx, sg * dy, sg * dz) : 0;
      cp_async16(A + c * (TC_M * 16) + r * 16, x + src * ldx + offx + 8 * c, v);
    }
    cp_async_commit();
  };

  // thread 0's account of what is in flight: bulk copies issued per stage
  // (their completions are waited in order) and the stage of the last commit
  int issued[2] = {0, 0}, landed[2] = {0, 0}, commits[2] = {0, 0}, last_commit = -1;
  auto issue_b = [&](int t, int st) {
    bulk_load(Bs + st * B_BYTES, Wp + (long long)t * NC * KC, B_BYTES, bars + st);
    ++issued[st];
  };
  load_a(0, 0);
  if (tid == 0) issue_b(0, 0);
  for (int t = 0; t < 27; ++t) {
    const int s = t & 1;
    if (t + 1 < 27) {
      const int s1 = (t + 1) & 1;
      // stage s1 was last read by the MMAs of tap t-1
      if (t >= 1 && !mbar_wait(bars + 2 + s1, ((t - 1) >> 1) & 1, err)) ok = false;
      ok = __syncthreads_and(ok);
      if (!ok) break;
      load_a(t + 1, s1);
      if (tid == 0) issue_b(t + 1, s1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    // this thread's A copies of tap t are done; make them visible to the
    // tensor cores (async proxy) and to the issuing thread
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(bars + s, (t >> 1) & 1, err)) {
        ok = false;
      } else {
        ++landed[s];
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(As + s * A_BYTES), b0 = smem_u32(Bs + s * B_BYTES);
#pragma unroll
        for (int kk = 0; kk < KC / 16; ++kk) {
          // K step of 16 = two 8-channel chunks
          const uint64_t ad = sdesc(a0 + kk * 2 * A_LBO, A_LBO, SBO);
          const uint64_t bd = sdesc(b0 + kk * 2 * B_LBO, B_LBO, SBO);
          mma_bf16(tbase, ad, bd, IDESC, (t > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(bars + 2 + s);
        ++commits[s];
        last_commit = s;
      }
    }
  }
  // the last tap's MMAs (and so all earlier ones) completed
  ok = __syncthreads_and(ok);
  if (ok && !mbar_wait(bars + 2 + (26 & 1), (26 >> 1) & 1, err)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok);
  if (ok) {
    const int row = warp * 32 + (tid & 31);
    const long long m = m0 + row;
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int n0 = 0; n0 < NC; n0 += 16) {
      float v[16];
      tmem_ld16(lane_addr + n0, v);
      if (m < Mtot) {
        if (!DGRAD) {
          __align__(16) __nv_bfloat16 o[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float a = v[i] + (bias ? bias[n0 + i] : 0.f);
            if (relu) a = fmaxf(a, 0.f);
            o[i] = __float2bfloat16(a);
          }
          uint4* dst = reinterpret_cast<uint4*>(y + m * ldy + offy + n0);
          dst[0] = reinterpret_cast<const uint4*>(o)[0];
          dst[1] = reinterpret_cast<const uint4*>(o)[1];
        } else {
          float* q = gx + m * ldg + offg + n0;
#pragma unroll
          for (int i = 0; i < 16; ++i) q[i] = accumulate ? q[i] + v[i] : v[i];
        }
      }
    }
  } else {
    // a wait ran out: let the copies and MMAs still in flight finish (each
    // wait bounded) before the shared memory and TMEM are given up
    cp_async_wait<0>();
    if (tid == 0) {
      for (int q = 0; q < 2; ++q)
        while (landed[q] < issued[q]) {
          if (!mbar_wait(bars + q, (uint32_t)(landed[q] & 1), err)) break;
          ++landed[q];
        }
      if (last_commit >= 0)
        mbar_wait(bars + 2 + last_commit, (uint32_t)((commits[last_commit] - 1) & 1), err);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(tmem_cols)
                 : "memory");
}

// ---- weight gradient ------------------------------------------------------
constexpr int WG_KC = 64;     // voxels per stage (4 MMAs of K = 16)
constexpr int WG_STAGES = 3;  // stages in flight
constexpr int WG_CTAS = 608;  // target CTAs of a launch (4 per SM)

// CI input channels (MMA N), CO output channels (128 / CO taps per CTA).
// blockIdx.x: tap group; blockIdx.y: voxel range [q chunk, (q + 1) chunk).
template <int CI, int CO>
__global__ void __launch_bounds__(TC_THREADS) k_wgrad_tc(
    const __nv_bfloat16* __restrict__ x, int ldx, int offx, const __nv_bfloat16* __restrict__ g,
    int ldg, int offg, int lgD, long long Mtot, long long chunk, float* __restrict__ part,
    int tmem_cols, int* __restrict__ err) {
  constexpr int TPM = TC_M / CO;                 // taps per CTA
  constexpr int A_BYTES = TC_M * WG_KC * 2;      // 16 KB
  constexpr int B_BYTES = CI * WG_KC * 2;
  constexpr int ST_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t A_KSTR = (TC_M / 8) * 128;  // bytes between 8-voxel groups
  constexpr uint32_t B_KSTR = (CI / 8) * 128;
  constexpr uint32_t IDESC = idesc_bf16_mn(TC_M, CI);
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* done = reinterpret_cast<uint64_t*>(smem + WG_STAGES * ST_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + WG_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile = blockIdx.x;
  const long long v0 = (long long)blockIdx.y * chunk;
  const long long v1 = v0 + chunk < Mtot ? v0 + chunk : Mtot;
  const int nk = v1 > v0 ? (int)((v1 - v0 + WG_KC - 1) / WG_KC) : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < WG_STAGES; ++q) mbar_init(done + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  bool ok = true;

  // stage st <- voxels [v0 + k WG_KC, +WG_KC): chunk e of a tile lands at 16 e
  // (A: e = (8-voxel group, 8-row group, voxel in group); B likewise with the
  // 8-channel groups of x)
  auto load = [&](int k, int st) {
    unsigned char* As = smem + st * ST_BYTES;
    unsigned char* Bs = As + A_BYTES;
    const long long vb = v0 + (long long)k * WG_KC;
    for (int e = tid; e < TC_M * WG_KC / 8; e += TC_THREADS) {
      const int r8 = e & 7, mg = (e >> 3) & (TC_M / 8 - 1), kg = e >> 7;
      const int tl = mg / (CO / 8), co8 = mg - tl * (CO / 8);
      const int t = tile * TPM + tl;
      const long long v = vb + kg * 8 + r8;
      const bool ok_e = t < 27 && v < v1;
      long long src = 0;
      if (ok_e) {
        const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
        src = tc_nbr(v, lgD, -dx, -dy, -dz) * ldg + offg + 8 * co8;
      }
      cp_async16(As + 16 * e, g + src, ok_e);
    }
    for (int e = tid; e < CI * WG_KC / 8; e += TC_THREADS) {
      const int r8 = e & 7, ng = (e >> 3) % (CI / 8), kg = (e >> 3) / (CI / 8);
      const long long v = vb + kg * 8 + r8;
      const bool ok_e = v < v1;
      cp_async16(Bs + 16 * e, x + (ok_e ? v * ldx + offx + 8 * ng : 0), ok_e);
    }
  };

  int commits[WG_STAGES] = {}, last_commit = -1;
  for (int k = 0; k < WG_STAGES - 1; ++k) {
    if (k < nk) load(k, k);
    cp_async_commit();
  }
  for (int k = 0; k < nk; ++k) {
    const int st = k % WG_STAGES;
    const int kn = k + WG_STAGES - 1;
    if (kn < nk) {
      const int sn = kn % WG_STAGES;  // last read by the MMAs of chunk k - 1
      if (k >= 1 && tid == 0 &&
          !mbar_wait(done + sn, (uint32_t)(((k - 1) / WG_STAGES) & 1), err))
        ok = false;
      ok = __syncthreads_and(ok);
      if (!ok) break;
      load(kn, sn);
    }
    cp_async_commit();
    cp_async_wait<WG_STAGES - 1>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + st * ST_BYTES), b0 = a0 + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < WG_KC / 16; ++kk) {
        const uint64_t ad = sdesc_mn(a0 + 2 * kk * A_KSTR, 128, A_KSTR);
        const uint64_t bd = sdesc_mn(b0 + 2 * kk * B_KSTR, 128, B_KSTR);
        mma_bf16(tbase, ad, bd, IDESC, (k > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(done + st);
      ++commits[st];
      last_commit = st;
    }
  }
  ok = __syncthreads_and(ok);
  if (ok && nk > 0 && tid == 0 &&
      !mbar_wait(done + (nk - 1) % WG_STAGES, (uint32_t)(((nk - 1) / WG_STAGES) & 1), err))
    ok = false;
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // row = (tap in group, co); its CI accumulators go to part[q][t][ci][co]
    const int row = warp * 32 + (tid & 31);
    const int tl = row / CO, co = row - tl * CO, t = tile * TPM + tl;
    const long long base = ((long long)blockIdx.y * 27 + (t < 27 ? t : 0)) * CI * CO + co;
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int n0 = 0; n0 < CI; n0 += 16) {
      float v[16];
      tmem_ld16(lane_addr + n0, v);
      if (t < 27) {
#pragma unroll
        for (int i = 0; i < 16; ++i) part[base + (long long)(n0 + i) * CO] = nk > 0 ? v[i] : 0.f;
      }
    }
  } else {
    // a wait ran out: let the copies and MMAs in flight finish (bounded)
    cp_async_wait<0>();
    if (tid == 0 && last_commit >= 0)
      mbar_wait(done + last_commit, (uint32_t)((commits[last_commit] - 1) & 1), err);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(tmem_cols)
                 : "memory");
}

// splits of the voxel range: about WG_CTAS CTAs in all, none empty
void wgrad_split(int Cout, long long Mtot, int* S, long long* chunk) {
  const int nt = (27 + TC_M / Cout - 1) / (TC_M / Cout);
  const long long nch = (Mtot + WG_KC - 1) / WG_KC;
  long long s = std::max(1, WG_CTAS / nt);
  if (s > nch) s = nch;
  const long long per = (nch + s - 1) / s;
  *S = (int)((nch + per - 1) / per);
  *chunk = per * WG_KC;
}

template <int CI, int CO>
void launch_wgrad(TView x, TView g, int lgD, long long Mtot, float* part, int* err, int* S_out,
                  cudaStream_t s) {
  constexpr int ST_BYTES = TC_M * WG_KC * 2 + CI * WG_KC * 2;
  const int cols = CI <= 32 ? 32 : (CI <= 64 ? 64 : (CI <= 128 ? 128 : 256));
  const size_t need = (size_t)WG_STAGES * ST_BYTES + WG_STAGES * 8 + 16;
  const int k = 512 / cols;
  const size_t cap = 233472 / (k + 1) - 1024 + 16;
  const size_t smem = need > cap ? need : cap;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_wgrad_tc<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  int S;
  long long chunk;
  wgrad_split(CO, Mtot, &S, &chunk);
  const int nt = (27 + TC_M / CO - 1) / (TC_M / CO);
  k_wgrad_tc<CI, CO><<<dim3(nt, S), TC_THREADS, smem, s>>>(x.p, x.ld, x.off, g.p, g.ld, g.off,
                                                           lgD, Mtot, chunk, part, cols, err);
  *S_out = S;
}

// ---- halo-tiled forward and input gradient for the full-resolution layers ---
// A CTA computes TX x-slices of a 16 (y) x 8 (z) block of output voxels, one
// M = 128 tile per slice (row m = 8 y + z).  It stages the input once as a
// (TX + 2) x 18 x 10 voxel block with its one-voxel periodic halo, laid out
// [8-channel group][x][y][z] with 16 bytes per voxel, and all 27 taps'
// packed weights by one bulk copy.  The A operand of tap (dx, dy, dz) is then
// a K-major no-swizzle view of the halo block: core matrices of 8 z-
// consecutive voxels x 16 bytes, 8-row groups (y) 10 x 16 bytes apart (SBO),
// 8-channel groups one block-plane apart (LBO), the start shifted by the tap
// offset.  So the block is read from global memory once instead of 27 times,
// and a tile costs 27 (KC / 16) MMAs on shared-memory operands.
template <int KC, int NC, bool DGRAD, int TX>
__global__ void __launch_bounds__(TC_THREADS) k_conv_halo(
    const __nv_bfloat16* __restrict__ x, int ldx, int offx, const __nv_bfloat16* __restrict__ Wp,
    const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ y, int ldy, int offy,
    float* __restrict__ gx, int ldg, int offg, int accumulate, int lgD, int tmem_cols,
    int* __restrict__ err) {
  constexpr int HX = TX + 2, HY = 18, HZ = 10, CH = KC / 8;
  constexpr int PLANE = HX * HY * HZ * 16;  // bytes of one 8-channel group
  constexpr int H_BYTES = CH * PLANE;
  constexpr int W_BYTES = 27 * NC * KC * 2;
  constexpr uint32_t SBO = HZ * 16, B_LBO = NC * 16;
  constexpr uint32_t IDESC = idesc_bf16(TC_M, NC);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* Hs = smem;
  unsigned char* Ws = smem + H_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Ws + W_BYTES);  // weights, MMAs
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int D = 1 << lgD, M = D - 1;
  // tile coordinates: z blocks of 8, y blocks of 16, x blocks of TX, samples
  const int nz = D >> 3, ny = D >> 4, nx = D / TX;
  long long bid = blockIdx.x;
  const int bz = (int)(bid % nz);
  bid /= nz;
  const int by = (int)(bid % ny);
  bid /= ny;
  const int bx = (int)(bid % nx);
  const long long b = bid / nx;
  const int x0 = bx * TX, y0 = by * 16, z0 = bz * 8;
  const long long sbase = b << (3 * lgD);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  bool ok = true;
  if (tid == 0) bulk_load(Ws, Wp, (uint32_t)W_BYTES, bars);
  // the halo block: chunk e = ((c8 HX + hx) HY + hy) HZ + hz lands at 16 e
  for (int e = tid; e < CH * HX * HY * HZ; e += TC_THREADS) {
    int r = e;
    const int hz = r % HZ;
    r /= HZ;
    const int hy = r % HY;
    r /= HY;
    const int hx = r % HX;
    const int c8 = r / HX;
    const long long v = sbase + ((((long long)((x0 + hx - 1) & M) << lgD) + ((y0 + hy - 1) & M))
                                 << lgD) +
                        ((z0 + hz - 1) & M);
    cp_async16(Hs + 16 * e, x + v * ldx + offx + 8 * c8, true);
  }
  cp_async_commit();
  cp_async_wait<0>();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  bool issued = false;
  if (tid == 0) {
    if (!mbar_wait(bars, 0, err)) {
      ok = false;
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t h0 = smem_u32(Hs), w0 = smem_u32(Ws);
      const int sg = DGRAD ? -1 : 1;
#pragma unroll 1
      for (int t = 0; t < 27; ++t) {
        const int dx = sg * (t / 9 - 1), dy = sg * ((t / 3) % 3 - 1), dz = sg * (t % 3 - 1);
#pragma unroll 1
        for (int tx = 0; tx < TX; ++tx) {
          const uint32_t a_off = (uint32_t)((((tx + dx + 1) * HY + (dy + 1)) * HZ + (dz + 1)) * 16);
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
            const uint64_t ad = sdesc(h0 + a_off + 2 * kk * PLANE, PLANE, SBO);
            const uint64_t bd = sdesc(w0 + t * (NC * KC * 2) + 2 * kk * B_LBO, B_LBO, 128);
            mma_bf16(tbase + tx * NC, ad, bd, IDESC, (t > 0 || kk > 0) ? 1u : 0u);
          }
        }
      }
      mma_commit(bars + 1);
      issued = true;
    }
  }
  ok = __syncthreads_and(ok);
  if (ok && tid == 0 && !mbar_wait(bars + 1, 0, err)) ok = false;
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = warp * 32 + (tid & 31);
    const int yy = row >> 3, zz = row & 7;
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int tx = 0; tx < TX; ++tx) {
      const long long m = sbase + ((((long long)(x0 + tx) << lgD) + (y0 + yy)) << lgD) + (z0 + zz);
#pragma unroll 1
      for (int n0 = 0; n0 < NC; n0 += 16) {
        float v[16];
        tmem_ld16(lane_addr + tx * NC + n0, v);
        if (!DGRAD) {
          __align__(16) __nv_bfloat16 o[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float a = v[i] + (bias ? bias[n0 + i] : 0.f);
            if (relu) a = fmaxf(a, 0.f);
            o[i] = __float2bfloat16(a);
          }
          uint4* dst = reinterpret_cast<uint4*>(y + m * ldy + offy + n0);
          dst[0] = reinterpret_cast<const uint4*>(o)[0];
          dst[1] = reinterpret_cast<const uint4*>(o)[1];
        } else {
          float* q = gx + m * ldg + offg + n0;
#pragma unroll
          for (int i = 0; i < 16; ++i) q[i] = accumulate ? q[i] + v[i] : v[i];
        }
      }
    }
  } else if (tid == 0) {
    // a wait ran out: the weights' copy and the MMAs in flight (each bounded)
    if (issued) mbar_wait(bars + 1, 0, err);
    else mbar_wait(bars, 0, err);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(tmem_cols)
                 : "memory");
}

template <int KC, int NC, bool DG, int TX>
void launch_halo(const TcArgs& a, cudaStream_t s) {
  constexpr int H_BYTES = (KC / 8) * (TX + 2) * 18 * 10 * 16, W_BYTES = 27 * NC * KC * 2;
  const int cols0 = TX * NC;
  const int cols = cols0 <= 32 ? 32 : (cols0 <= 64 ? 64 : (cols0 <= 128 ? 128 : 256));
  const size_t need = (size_t)H_BYTES + W_BYTES + 2 * 8 + 16;
  const int k = 512 / cols;
  const size_t cap = 233472 / (k + 1) - 1024 + 16;
  const size_t smem = need > cap ? need : cap;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_halo<KC, NC, DG, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  const long long tiles = a.Mtot / (TX * 16 * 8);
  k_conv_halo<KC, NC, DG, TX><<<(unsigned)tiles, TC_THREADS, smem, s>>>(
      a.x, a.ldx, a.offx, a.Wp, a.bias, a.relu, a.y, a.ldy, a.offy, a.gx, a.ldg, a.offg,
      a.accumulate, a.lgD, cols, a.err);
}

// The same halo-tiled form for layers whose 27 weight slices do not fit beside
// the input block: the block stays resident while the taps' weight slices
// stream through two shared-memory stages (one bulk copy each).  Thread 0
// alone loads the slices and issues the MMAs, so the loop over taps has no
// block-wide synchronisation.
template <int KC, int NC, bool DGRAD, int TX>
__global__ void __launch_bounds__(TC_THREADS) k_conv_halo_s(
    const __nv_bfloat16* __restrict__ x, int ldx, int offx, const __nv_bfloat16* __restrict__ Wp,
    const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ y, int ldy, int offy,
    float* __restrict__ gx, int ldg, int offg, int accumulate, int lgD, int tmem_cols,
    int* __restrict__ err) {
  constexpr int HX = TX + 2, HY = 18, HZ = 10, CH = KC / 8;
  constexpr int PLANE = HX * HY * HZ * 16;
  constexpr int H_BYTES = CH * PLANE;
  constexpr int T_BYTES = NC * KC * 2;  // one tap's weight slice
  constexpr uint32_t SBO = HZ * 16, B_LBO = NC * 16;
  constexpr uint32_t IDESC = idesc_bf16(TC_M, NC);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* Hs = smem;
  unsigned char* Ws = smem + H_BYTES;  // [2][T_BYTES]
  uint64_t* bars = reinterpret_cast<uint64_t*>(Ws + 2 * T_BYTES);  // full[2], done[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int D = 1 << lgD, M = D - 1;
  const int nz = D >> 3, ny = D >> 4, nx = D / TX;
  long long bid = blockIdx.x;
  const int bz = (int)(bid % nz);
  bid /= nz;
  const int by = (int)(bid % ny);
  bid /= ny;
  const int bx = (int)(bid % nx);
  const long long b = bid / nx;
  const int x0 = bx * TX, y0 = by * 16, z0 = bz * 8;
  const long long sbase = b << (3 * lgD);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(bars + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  // thread 0's account of the copies and MMAs in flight
  int issued[2] = {0, 0}, landed[2] = {0, 0}, commits[2] = {0, 0}, last_commit = -1;
  if (tid == 0) {
    bulk_load(Ws, Wp, (uint32_t)T_BYTES, bars);
    ++issued[0];
  }
  for (int e = tid; e < CH * HX * HY * HZ; e += TC_THREADS) {
    int r = e;
    const int hz = r % HZ;
    r /= HZ;
    const int hy = r % HY;
    r /= HY;
    const int hx = r % HX;
    const int c8 = r / HX;
    const long long v = sbase + ((((long long)((x0 + hx - 1) & M) << lgD) + ((y0 + hy - 1) & M))
                                 << lgD) +
                        ((z0 + hz - 1) & M);
    cp_async16(Hs + 16 * e, x + v * ldx + offx + 8 * c8, true);
  }
  cp_async_commit();
  cp_async_wait<0>();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  bool ok = true;
  if (tid == 0) {
    const uint32_t h0 = smem_u32(Hs), w0 = smem_u32(Ws);
    const int sg = DGRAD ? -1 : 1;
    for (int t = 0; t < 27 && ok; ++t) {
      const int st = t & 1;
      if (t + 1 < 27) {
        const int s1 = (t + 1) & 1;  // last read by the MMAs of tap t - 1
        if (t >= 1 && !mbar_wait(bars + 2 + s1, ((t - 1) >> 1) & 1, err)) {
          ok = false;
          break;
        }
        bulk_load(Ws + s1 * T_BYTES, Wp + (long long)(t + 1) * NC * KC, (uint32_t)T_BYTES,
                  bars + s1);
        ++issued[s1];
      }
      if (!mbar_wait(bars + st, (t >> 1) & 1, err)) {
        ok = false;
        break;
      }
      ++landed[st];
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int dx = sg * (t / 9 - 1), dy = sg * ((t / 3) % 3 - 1), dz = sg * (t % 3 - 1);
#pragma unroll 1
      for (int tx = 0; tx < TX; ++tx) {
        const uint32_t a_off = (uint32_t)((((tx + dx + 1) * HY + (dy + 1)) * HZ + (dz + 1)) * 16);
#pragma unroll
        for (int kk = 0; kk < KC / 16; ++kk) {
          const uint64_t ad = sdesc(h0 + a_off + 2 * kk * PLANE, PLANE, SBO);
          const uint64_t bd = sdesc(w0 + st * T_BYTES + 2 * kk * B_LBO, B_LBO, 128);
          mma_bf16(tbase + tx * NC, ad, bd, IDESC, (t > 0 || kk > 0) ? 1u : 0u);
        }
      }
      mma_commit(bars + 2 + st);
      ++commits[st];
      last_commit = st;
    }
    if (ok && !mbar_wait(bars + 2 + (26 & 1), (26 >> 1) & 1, err)) ok = false;
    if (!ok) {
      // a wait ran out: the copies and MMAs in flight (each wait bounded)
      for (int q = 0; q < 2; ++q)
        while (landed[q] < issued[q]) {
          if (!mbar_wait(bars + q, (uint32_t)(landed[q] & 1), err)) break;
          ++landed[q];
        }
      if (last_commit >= 0)
        mbar_wait(bars + 2 + last_commit, (uint32_t)((commits[last_commit] - 1) & 1), err);
    }
  }
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = warp * 32 + (tid & 31);
    const int yy = row >> 3, zz = row & 7;
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int tx = 0; tx < TX; ++tx) {
      const long long m = sbase + ((((long long)(x0 + tx) << lgD) + (y0 + yy)) << lgD) + (z0 + zz);
#pragma unroll 1
      for (int n0 = 0; n0 < NC; n0 += 16) {
        float v[16];
        tmem_ld16(lane_addr + tx * NC + n0, v);
        if (!DGRAD) {
          __align__(16) __nv_bfloat16 o[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float a = v[i] + (bias ? bias[n0 + i] : 0.f);
            if (relu) a = fmaxf(a, 0.f);
            o[i] = __float2bfloat16(a);
          }
          uint4* dst = reinterpret_cast<uint4*>(y + m * ldy + offy + n0);
          dst[0] = reinterpret_cast<const uint4*>(o)[0];
          dst[1] = reinterpret_cast<const uint4*>(o)[1];
        } else {
          float* q = gx + m * ldg + offg + n0;
#pragma unroll
          for (int i = 0; i < 16; ++i) q[i] = accumulate ? q[i] + v[i] : v[i];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(tmem_cols)
                 : "memory");
}

template <int KC, int NC, bool DG, int TX>
void launch_halo_s(const TcArgs& a, cudaStream_t s) {
  constexpr int H_BYTES = (KC / 8) * (TX + 2) * 18 * 10 * 16, T_BYTES = NC * KC * 2;
  const int cols0 = TX * NC;
  const int cols = cols0 <= 32 ? 32 : (cols0 <= 64 ? 64 : (cols0 <= 128 ? 128 : 256));
  const size_t need = (size_t)H_BYTES + 2 * T_BYTES + 4 * 8 + 16;
  const int k = 512 / cols;
  const size_t cap = 233472 / (k + 1) - 1024 + 16;
  const size_t smem = need > cap ? need : cap;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_halo_s<KC, NC, DG, TX>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  const long long tiles = a.Mtot / (TX * 16 * 8);
  k_conv_halo_s<KC, NC, DG, TX><<<(unsigned)tiles, TC_THREADS, smem, s>>>(
      a.x, a.ldx, a.offx, a.Wp, a.bias, a.relu, a.y, a.ldy, a.offy, a.gx, a.ldg, a.offg,
      a.accumulate, a.lgD, cols, a.err);
}

// Packed weight slices.  Forward (N = Cout, K = Cin):
//   Wp[t][c][n][k8] = W[t][8c + k8][n]
// Input gradient (N = Cin, K = Cout):
//   Wp[t][c][n][k8] = W[t][n][8c + k8]
// i.e. per tap the K-major N x K tile, 8-channel chunks of K one after the
// other, the N rows of a chunk contiguous (the shared-memory layout).
__global__ void k_pack_tc(const __nv_bfloat16* __restrict__ W, int Cin, int Cout, int dgrad,
                          __nv_bfloat16* __restrict__ Wp) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long per = (long long)Cin * Cout;
  if (e >= 27 * per) return;
  const int t = (int)(e / per);
  const long long r = e - t * per;
  const int N = dgrad ? Cin : Cout;
  const int k8 = (int)(r & 7), n = (int)((r >> 3) % N), c = (int)((r >> 3) / N);
  const int kidx = 8 * c + k8;
  const int ci = dgrad ? n : kidx, co = dgrad ? kidx : n;
  Wp[e] = W[((long long)t * Cin + ci) * Cout + co];
}

template <int KC, int NC, bool DG>
void launch_tc(const TcArgs& a, cudaStream_t s) {
  constexpr int A_BYTES = TC_M * KC * 2, B_BYTES = NC * KC * 2;
  const int cols = NC <= 32 ? 32 : (NC <= 64 ? 64 : (NC <= 128 ? 128 : 256));
  const size_t need = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + 4 * 8 + 16;
  // at most 512 / cols CTAs per SM may hold TMEM at once: pad the shared
  // memory so that no more are resident (tcgen05.alloc would wait)
  // (each CTA also holds 1 KB of reserved shared memory)
  const int k = 512 / cols;
  const size_t cap = 233472 / (k + 1) - 1024 + 16;
  const size_t smem = need > cap ? need : cap;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_tc<KC, NC, DG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  const unsigned grid = (unsigned)((a.Mtot + TC_M - 1) / TC_M);
  k_conv_tc<KC, NC, DG><<<grid, TC_THREADS, smem, s>>>(
      a.x, a.ldx, a.offx, a.Wp, a.bias, a.relu, a.y, a.ldy, a.offy, a.gx, a.ldg, a.offg,
      a.accumulate, a.lgD, a.Mtot, cols, a.err);
}

}  // namespace

long long nn_tc_packed_size(int Cin, int Cout) { return 27LL * Cin * Cout; }

void nn_tc_pack(const __nv_bfloat16* W, int Cin, int Cout, int dgrad, __nv_bfloat16* Wp,
                cudaStream_t s) {
  const long long n = 27LL * Cin * Cout;
  k_pack_tc<<<nblocks(n, 256), 256, 0, s>>>(W, Cin, Cout, dgrad, Wp);
}

// (K, N) pairs of the network's convolutions: forward (Cin, Cout) and input
// gradient (Cout, Cin)
bool nn_tc_supported(int K, int N) {
  static const int kn[][2] = {{16, 16},  {16, 32},  {32, 32},  {32, 64},  {64, 64},  {64, 128},
                              {128, 128}, {192, 64}, {96, 32},  {48, 16},  {32, 16},  {64, 32},
                              {128, 64}, {64, 192}, {32, 96},  {16, 48}};
  for (auto& p : kn)
    if (p[0] == K && p[1] == N) return true;
  return false;
}

bool nn_tc_conv(const TcArgs& a, int K, int N, bool dgrad, cudaStream_t s) {
  // the layers of the two finest levels whose input block and 27 weight
  // slices fit one CTA's shared memory run on the halo-tiled kernel when the
  // grid holds its tiles (16^3 and more)
  if (a.lgD >= 4 && a.lgD <= 10) {
#define HALO_CASE(KK, NN, TXF, TXD)                                                       \
  if (K == KK && N == NN) {                                                             \
    if (dgrad) launch_halo<KK, NN, true, TXD>(a, s); else launch_halo<KK, NN, false, TXF>(a, s); \
    return true;                                                                        \
  }
    HALO_CASE(16, 16, 4, 4) HALO_CASE(16, 32, 4, 4) HALO_CASE(32, 32, 2, 2)
    HALO_CASE(32, 16, 2, 2)
#undef HALO_CASE
    // larger channel counts: the weight slices stream beside the resident block
#define HALO_S(KK, NN, TXX, DGR)                           \
  if (K == KK && N == NN && dgrad == DGR) {                \
    launch_halo_s<KK, NN, DGR, TXX>(a, s);                  \
    return true;                                            \
  }
    HALO_S(96, 32, 2, false) HALO_S(32, 96, 2, true) HALO_S(32, 64, 2, false)
    HALO_S(64, 32, 2, true) HALO_S(64, 64, 2, false) HALO_S(64, 64, 2, true)
    HALO_S(64, 128, 2, false) HALO_S(128, 64, 1, true) HALO_S(128, 128, 1, false)
    HALO_S(128, 128, 1, true) HALO_S(64, 192, 1, true)
#undef HALO_S
    if (!dgrad && K == 48 && N == 16) {
      launch_halo<48, 16, false, 2>(a, s);
      return true;
    }
    if (dgrad && K == 16 && N == 48) {
      launch_halo<16, 48, true, 2>(a, s);
      return true;
    }
  }
#define TC_CASE(KK, NN)                                              \
  if (K == KK && N == NN) {                                          \
    if (dgrad) launch_tc<KK, NN, true>(a, s); else launch_tc<KK, NN, false>(a, s); \
    return true;                                                     \
  }
  TC_CASE(16, 16) TC_CASE(16, 32) TC_CASE(32, 32) TC_CASE(32, 64) TC_CASE(64, 64)
  TC_CASE(64, 128) TC_CASE(128, 128) TC_CASE(192, 64) TC_CASE(96, 32) TC_CASE(48, 16)
  TC_CASE(32, 16) TC_CASE(64, 32) TC_CASE(128, 64) TC_CASE(64, 192) TC_CASE(32, 96)
  TC_CASE(16, 48)
#undef TC_CASE
  return false;
}

// (Cin, Cout) pairs of the network's weight gradients
bool nn_tc_wgrad_supported(int Cin, int Cout) {
  static const int p[][2] = {{16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 64},
                             {64, 128}, {128, 128}, {192, 64}, {96, 32}, {48, 16}};
  for (auto& q : p)
    if (q[0] == Cin && q[1] == Cout) return true;
  return false;
}

long long nn_tc_wgrad_scratch(int Cin, int Cout) {
  const int nt = (27 + TC_M / Cout - 1) / (TC_M / Cout);
  return (long long)std::max(1, WG_CTAS / nt) * 27 * Cin * Cout;
}

bool nn_tc_wgrad(TView x, int Cin, TView g, int Cout, float* dW, float* db, float* partials,
                 int B, int lgD, int* err, cudaStream_t s) {
  const long long Mtot = (long long)B << (3 * lgD);
  int S = 0;
#define WG_CASE(CI, CO)                                                  \
  if (Cin == CI && Cout == CO) {                                         \
    launch_wgrad<CI, CO>(x, g, lgD, Mtot, partials, err, &S, s);         \
  } else
  WG_CASE(16, 16) WG_CASE(16, 32) WG_CASE(32, 32) WG_CASE(32, 64) WG_CASE(64, 64)
  WG_CASE(64, 128) WG_CASE(128, 128) WG_CASE(192, 64) WG_CASE(96, 32) WG_CASE(48, 16)
  return false;
#undef WG_CASE
  nn_wgrad_finish(partials, S, Cin, Cout, dW, g, db, Mtot, s);
  return true;
}
