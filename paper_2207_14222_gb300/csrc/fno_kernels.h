// fno_kernels.h -- launchers of the Fourier-neural-operator kernels
// (fno_kernels.cu) used by the warm-start network (fno_api.cpp).
//
// Tensors are FP32, batch-major.  A "strided field" addresses element
// (b, c, p) of a batch of multi-channel images at b * bs + c * cs + p * ps
// (planar: bs = C P, cs = P, ps = 1; a complex64 field read as two
// channels: bs = 2 P, cs = 1, ps = 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace usp {

struct Strided {
  float* ptr;
  int64_t bs, cs, ps;
};
struct CStrided {
  const float* ptr;
  int64_t bs, cs, ps;
};

// out(b, o, p) = (accumulate ? out : 0) + bias[o] + sum_c Wt(o, c) in(b, c, p)
// with Wt(o, c) = W[o * so + c * sc].  cin, cout <= 64.
cudaError_t fno_conv(CStrided in, int cin, const float* W, int64_t so, int64_t sc,
                     const float* bias, Strided out, int cout, int batch, int64_t P,
                     bool accumulate, cudaStream_t s);

// Dynamic shared memory the truncated transforms need for H x W planes.
size_t fno_smem_bytes(int H, int W, int modes);

// Truncated forward 2-D DFT of `planes` real H x W planes (contiguous):
// out[plane][m1][m2] = sum_{i,j} in[plane][i][j] e^{-2 pi i (k1 i / H + k2 j / W)},
// k = mode index of the slot.  twh/tww: e^{-2 pi i k(s) n / N} as [n][s].
cudaError_t fno_dft2(const float* in, int64_t planes, int H, int W, int modes,
                     const float2* twh, const float2* tww, float2* out, cudaStream_t s);

// Truncated inverse: acc[plane][i][j] += scale * Re sum_{m} Z[plane][m1][m2]
// e^{+2 pi i (k1 i / H + k2 j / W)}; then act[plane] = gelu(acc[plane]) if
// act is not null.
cudaError_t fno_idft2(const float2* Z, int64_t planes, int H, int W, int modes,
                      const float2* twh, const float2* tww, float scale, float* acc,
                      float* act, cudaStream_t s);

// Per-mode channel mixing: Z[b][o][m] = sum_c R[o][c][m] X[b][c][m]
// (adjoint: Z[b][c][m] = sum_o conj(R[o][c][m]) X[b][o][m]).  R: complex as
// (re, im) float pairs.  nout/nin: channels of Z / X.
cudaError_t fno_mix(const float2* X, const float* R, int batch, int nin, int nout, int mm,
                    bool adjoint, float2* Z, cudaStream_t s);

// dR[o][c][m] = scale * sum_b G[b][o][m] conj(X[b][c][m]).
cudaError_t fno_dR(const float2* G, const float2* X, int batch, int O, int C, int mm,
                   float scale, float* dR, cudaStream_t s);

// Weight gradients of a 1x1 convolution, deterministic: dW[o][c] = sum_{b,p}
// g(b, o, p) v(b, c, p) and db[o] = sum_{b,p} g(b, o, p) (db may be null),
// written (not accumulated).  partials: scratch of
// fno_wgrad_partials(O, C) floats.
int64_t fno_wgrad_partials(int O, int C);
cudaError_t fno_wgrad(CStrided g, int O, CStrided v, int C, int batch, int64_t P,
                      float* partials, float* dW, float* db, cudaStream_t s);

// x <- x * gelu'(z), elementwise.
cudaError_t fno_gelu_bwd(float* x, const float* z, int64_t n, cudaStream_t s);

// Loss mean_b ||xh_b - x_b||^2 / ||x_b||^2 over complex64 fields (batch x P)
// into *loss (device double), and gu = 2 (xh - x) / (batch ||x_b||^2).
// partials: scratch of fno_loss_partials(batch) doubles.
int64_t fno_loss_partials(int batch);
cudaError_t fno_loss(const float2* xh, const float2* x, int batch, int64_t P, double* partials,
                     double* loss, float2* gu, cudaStream_t s);

// Adam step on n parameters: m, v moments; c1 = 1/(1 - beta1^t),
// c2 = 1/(1 - beta2^t).
cudaError_t fno_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                     float beta1, float beta2, float eps, float c1, float c2, cudaStream_t s);

}  // namespace usp
