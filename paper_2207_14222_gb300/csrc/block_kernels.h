// block_kernels.h -- launchers of the block-form steps (block_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace usp {

enum : int { BLOCK_ANTISYMMETRIC = 1, BLOCK_FLUX = 2 };
constexpr int BLOCK_KMAX = 4;   // components per point (flux form in 3-D)

struct BlockArgs {
  int kind;            // BLOCK_ANTISYMMETRIC or BLOCK_FLUX
  int K;               // components: 2 (antisymmetric), 1 + ndim (flux)
  int ndim;
  int n[3];
  int64_t N;           // points per component plane
  float ks[3];         // 2 pi / (n dx) per axis
  float inv_n;         // 1 / N
  float sym[4];        // antisymmetric: a_re, a_im, b_re, b_im of l = a|p|^2 + b;
                       // flux: alpha, beta, s
  const float2* V;     // per point: v (antisymmetric) or (Vu, VJ) (flux)
  const float2* y;     // K planes
  const float2* x_in;  // K planes
  float2* x_out;       // K planes
  float2* buf;         // K planes of scratch
  DevState* st;
  double* partials;    // one per block of the post step
  double* hist;
  float alpha;
  int flags;           // F_XZERO, F_REF
};

int block_grid(int64_t N);
cudaError_t launch_block_pre(const BlockArgs& a, cudaStream_t s);
cudaError_t launch_block_mul(const BlockArgs& a, cudaStream_t s);
cudaError_t launch_block_post(const BlockArgs& a, cudaStream_t s);
// out[0] = alpha* (min Re 1/lambda of B), out[1] = max ||V|| per point,
// out[2] = non-finite count; partials: 3 per block.
cudaError_t launch_block_stats(const BlockArgs& a, double* partials, double* out, cudaStream_t s);
cudaError_t launch_pack2(const float* a, const float* b, int64_t n, float2* out, cudaStream_t s);

}  // namespace usp
