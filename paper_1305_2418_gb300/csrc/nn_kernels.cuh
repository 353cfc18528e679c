// nn_kernels.cuh -- BF16 tensor-core 3D convolution primitives (3^3 taps,
// circular padding, NDHWC) with FP32 accumulation, for the learned initial
// guess of the field solve.  Declarations shared by unet.cu.
#pragma once
#include <cuda_bf16.h>

#include "mgfr_internal.cuh"

// Activation tensor view: element (voxel m, channel c) at p[m * ld + off + c].
struct TView {
  __nv_bfloat16* p;
  int ld, off;
};
struct FView {
  float* p;
  int ld, off;
};

// y = conv(x, W) + b (+ReLU): x [B*D^3][Cin] bf16, W [27][Cin][Cout] bf16
// (tap = (dx+1)*9 + (dy+1)*3 + (dz+1), x index i + dx), y bf16.
// Cin, Cout multiples of 16 (Cout <= 128).
void nn_conv_fwd(TView x, int Cin, const __nv_bfloat16* W, const float* bias, int relu, TView y,
                 int Cout, int B, int lgD, cudaStream_t s);
// gx (+)= conv^T(g, W): g [B*D^3][Cout] bf16 (gradient of the pre-activation),
// gx FP32 [.][Cin] (accumulate if acc).
void nn_conv_dgrad(TView g, int Cout, const __nv_bfloat16* W, FView gx, int Cin, int accumulate,
                   int B, int lgD, cudaStream_t s);
// dW[27][Cin][Cout] (FP32, overwritten) = sum_m x[nbr(m,tap)][ci] g[m][co];
// db[Cout] = sum_m g[m][co].  `partials` is scratch of nn_wgrad_scratch()
// floats.
void nn_conv_wgrad(TView x, int Cin, TView g, int Cout, float* dW, float* db, float* partials,
                   int B, int lgD, cudaStream_t s);
long long nn_wgrad_scratch(int Cin, int Cout);
// dW[i] = sum over the S slices of partials[s][i] (in order), then db (the
// bias stages reuse `partials` as their scratch: Cin >= 16, S >= 1)
void nn_wgrad_finish(float* partials, int S, int Cin, int Cout, float* dW, TView g,
                     float* db, long long Mtot, cudaStream_t s);

// ---- tensor-core (tcgen05) forward and input-gradient convolutions (nn_tc.cu)
struct TcArgs {
  const __nv_bfloat16* x;  // A rows: x (forward) or g (input gradient), view
  int ldx, offx;
  const __nv_bfloat16* Wp;  // packed weights (nn_tc_pack)
  const float* bias;        // forward, nullable
  int relu;
  __nv_bfloat16* y;  // forward output view
  int ldy, offy;
  float* gx;  // input-gradient output view
  int ldg, offg, accumulate;
  int lgD;
  long long Mtot;  // voxels (B D^3)
  int* err;        // set to 1 if a bounded wait in the kernel gave up
};
// whether the (K, N) pair (forward: Cin, Cout; gradient: Cout, Cin) is built
bool nn_tc_supported(int K, int N);
// elements of a packed weight tensor (27 Cin Cout)
long long nn_tc_packed_size(int Cin, int Cout);
// W [27][Cin][Cout] BF16 -> the per-tap K-major tiles of the forward
// (dgrad = 0) or input-gradient (dgrad = 1) convolution
void nn_tc_pack(const __nv_bfloat16* W, int Cin, int Cout, int dgrad, __nv_bfloat16* Wp,
                cudaStream_t s);
// launch; false if (K, N) is not built
bool nn_tc_conv(const TcArgs& a, int K, int N, bool dgrad, cudaStream_t s);
// weight gradient on tcgen05 (same result and arguments as nn_conv_wgrad;
// partials: nn_tc_wgrad_scratch floats); false if (Cin, Cout) is not built
bool nn_tc_wgrad_supported(int Cin, int Cout);
long long nn_tc_wgrad_scratch(int Cin, int Cout);
bool nn_tc_wgrad(TView x, int Cin, TView g, int Cout, float* dW, float* db, float* partials,
                 int B, int lgD, int* err, cudaStream_t s);
