// block_kernels.cu -- the pointwise and spectral steps of Algorithm 1 for the
// block forms of the canonical system (Sec. 2.2 Eq. antisymmetrised; Sec. 3.2
// Eq. diffusion-equation-matrix-form), whose unknown has K components per
// grid point stored as K consecutive planes of N points.  The transforms of
// each plane run on the line and strided-axis kernels of pencil_kernels.cu;
// these kernels couple the components:
//   k_block_pre   t = B x + y                      (B = I - V, K x K per point)
//   k_block_mul   T <- (L^(p) + I)^-1 T / N         (K x K per frequency)
//   k_block_post  Delta = B (u - x), x += alpha Delta, ||Delta||^2 (FP64),
//                 then the last block updates the iteration state.
#include "block_kernels.h"
#include "fft_core.cuh"
#include "iteration_state.cuh"

namespace usp {

namespace {

constexpr int BT = 256;

__device__ __forceinline__ float2 cm(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmc(float2 a, float2 b) {   // conj(a) b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// B x at point i for the block kind (x: K planes).
__device__ __forceinline__ void apply_B(const BlockArgs& a, int64_t i, const float2* xk, float2* out) {
  const float2 vv = a.V[i];
  if (a.kind == BLOCK_ANTISYMMETRIC) {
    // B = [[1, conj(v)], [-v, 1]]
    const float2 c = cmc(vv, xk[1]), d = cm(vv, xk[0]);
    out[0] = make_float2(xk[0].x + c.x, xk[0].y + c.y);
    out[1] = make_float2(xk[1].x - d.x, xk[1].y - d.y);
  } else {
    // B = diag(1 - Vu, (1 - VJ) I), (Vu, VJ) = (vv.x, vv.y)
    const float bu = 1.f - vv.x, bj = 1.f - vv.y;
    out[0] = make_float2(bu * xk[0].x, bu * xk[0].y);
    for (int k = 1; k < a.K; ++k) out[k] = make_float2(bj * xk[k].x, bj * xk[k].y);
  }
}

__global__ void __launch_bounds__(BT) k_block_pre(const BlockArgs a) {
  if (a.st->done) return;
  const bool xzero = (a.flags & F_XZERO) != 0;
  for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * BT) {
    float2 xk[BLOCK_KMAX], t[BLOCK_KMAX];
    for (int k = 0; k < a.K; ++k) xk[k] = xzero ? make_float2(0.f, 0.f) : a.x_in[k * a.N + i];
    apply_B(a, i, xk, t);
    for (int k = 0; k < a.K; ++k) {
      const float2 yv = a.y[k * a.N + i];
      a.buf[k * a.N + i] = make_float2(t[k].x + yv.x, t[k].y + yv.y);
    }
  }
}

__global__ void __launch_bounds__(BT) k_block_mul(const BlockArgs a) {
  if (a.st->done) return;
  for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * BT) {
    // frequency of each axis (C order, last axis fastest)
    float p[3] = {0.f, 0.f, 0.f};
    int64_t r = i;
    for (int ax = a.ndim - 1; ax >= 0; --ax) {
      const int k = int(r % a.n[ax]);
      r /= a.n[ax];
      p[ax] = a.ks[ax] * float(signed_freq(k, a.n[ax]));
    }
    const float p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    float2 T[BLOCK_KMAX];
    for (int k = 0; k < a.K; ++k) T[k] = a.buf[k * a.N + i];
    if (a.kind == BLOCK_ANTISYMMETRIC) {
      // (L+I)^-1 = [[1, conj(l)], [-l, 1]] / (1 + |l|^2), l = a |p|^2 + b
      const float2 l = make_float2(a.sym[0] * p2 + a.sym[2], a.sym[1] * p2 + a.sym[3]);
      const float sc = a.inv_n / (1.f + l.x * l.x + l.y * l.y);
      const float2 c = cmc(l, T[1]), d = cm(l, T[0]);
      a.buf[i] = make_float2(sc * (T[0].x + c.x), sc * (T[0].y + c.y));
      a.buf[a.N + i] = make_float2(sc * (T[1].x - d.x), sc * (T[1].y - d.y));
    } else {
      // Schur complement of [[alpha, i s p^T], [i s p, beta I]]
      const float al = a.sym[0], be = a.sym[1], s = a.sym[2];
      const float S = al + s * s * p2 / be;
      const int d = a.K - 1;
      float2 pT = make_float2(0.f, 0.f);   // p . T_J
      for (int k = 0; k < d; ++k) pT = make_float2(pT.x + p[k] * T[1 + k].x, pT.y + p[k] * T[1 + k].y);
      const float iS = a.inv_n / S;
      // u = (T_u - i s pT / beta) / S
      a.buf[i] = make_float2(iS * (T[0].x + s * pT.y / be), iS * (T[0].y - s * pT.x / be));
      // J_k = T_k / beta - s^2 p_k pT / (beta^2 S) - i s p_k T_u / (beta S)
      for (int k = 0; k < d; ++k) {
        const float c1 = a.inv_n / be, c2 = s * s * p[k] / (be * be * S) * a.inv_n;
        const float c3 = s * p[k] / (be * S) * a.inv_n;
        a.buf[(1 + k) * a.N + i] = make_float2(c1 * T[1 + k].x - c2 * pT.x + c3 * T[0].y,
                                               c1 * T[1 + k].y - c2 * pT.y - c3 * T[0].x);
      }
    }
  }
}

__global__ void __launch_bounds__(BT) k_block_post(const BlockArgs a) {
  __shared__ double red[BT / 32];
  __shared__ int is_last;
  if (a.st->done) return;
  const bool xzero = (a.flags & F_XZERO) != 0;
  const bool ref = (a.flags & F_REF) != 0;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * BT) {
    float2 dk[BLOCK_KMAX], xk[BLOCK_KMAX], del[BLOCK_KMAX];
    for (int k = 0; k < a.K; ++k) {
      xk[k] = xzero ? make_float2(0.f, 0.f) : a.x_in[k * a.N + i];
      const float2 u = a.buf[k * a.N + i];
      dk[k] = make_float2(u.x - xk[k].x, u.y - xk[k].y);
    }
    apply_B(a, i, dk, del);
    for (int k = 0; k < a.K; ++k) {
      acc += (double)del[k].x * del[k].x + (double)del[k].y * del[k].y;
      if (!ref)
        a.x_out[k * a.N + i] = make_float2(xk[k].x + a.alpha * del[k].x, xk[k].y + a.alpha * del[k].y);
    }
  }
  // block sum, then the last block to finish sums the partials in block
  // order (deterministic) and updates the iteration state
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs = 0.0;
    for (int w = 0; w < BT / 32; ++w) bs += red[w];
    a.partials[blockIdx.x] = bs;
    __threadfence();
    is_last = atomicAdd(&a.st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last || threadIdx.x != 0) return;
  __threadfence();
  double tot = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) tot += __ldcg(a.partials + b);
  finalize_iteration(a.st, a.hist, tot, a.flags);
  a.st->ticket = 0u;
}

// alpha* = min over points of the smallest Re 1/lambda over B's eigenvalues,
// and max ||V|| (per point operator norm), non-finite count: per block.
__global__ void __launch_bounds__(BT) k_block_stats(const BlockArgs a, double* partials) {
  __shared__ float r0[BT / 32], r1[BT / 32];
  __shared__ int r2[BT / 32];
  float amin = 3.0e38f, vmax = 0.f;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * BT) {
    const float2 v = a.V[i];
    if (!isfinite(v.x) || !isfinite(v.y)) {
      ++bad;
      continue;
    }
    if (a.kind == BLOCK_ANTISYMMETRIC) {
      const float m2 = v.x * v.x + v.y * v.y;     // eigenvalues 1 -+ i |v|
      vmax = fmaxf(vmax, sqrtf(m2));
      amin = fminf(amin, 1.f / (1.f + m2));
    } else {
      vmax = fmaxf(vmax, fmaxf(fabsf(v.x), fabsf(v.y)));
      amin = fminf(amin, fminf(1.f / (1.f - v.x), 1.f / (1.f - v.y)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    amin = fminf(amin, __shfl_down_sync(0xffffffffu, amin, o));
    vmax = fmaxf(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = amin;
    r1[threadIdx.x >> 5] = vmax;
    r2[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < BT / 32; ++w) {
      r0[0] = fminf(r0[0], r0[w]);
      r1[0] = fmaxf(r1[0], r1[w]);
      r2[0] += r2[w];
    }
    partials[3 * blockIdx.x] = r0[0];
    partials[3 * blockIdx.x + 1] = r1[0];
    partials[3 * blockIdx.x + 2] = r2[0];
  }
}

__global__ void k_block_stats_final(const double* partials, int nb, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double amin = 1e300, vmax = 0.0, bad = 0.0;
  for (int b = 0; b < nb; ++b) {
    amin = fmin(amin, partials[3 * b]);
    vmax = fmax(vmax, partials[3 * b + 1]);
    bad += partials[3 * b + 2];
  }
  out[0] = amin;
  out[1] = vmax;
  out[2] = bad;
}

// Pack two real planes (Vu, VJ) into one float2 per point.
__global__ void k_pack2(const float* a, const float* b, int64_t n, float2* out) {
  for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < n; i += (int64_t)gridDim.x * BT)
    out[i] = make_float2(a[i], b[i]);
}

}  // namespace

int block_grid(int64_t N) {
  int64_t g = (N + BT - 1) / BT;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_block_pre(const BlockArgs& a, cudaStream_t s) {
  k_block_pre<<<block_grid(a.N), BT, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_block_mul(const BlockArgs& a, cudaStream_t s) {
  k_block_mul<<<block_grid(a.N), BT, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_block_post(const BlockArgs& a, cudaStream_t s) {
  k_block_post<<<block_grid(a.N), BT, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_block_stats(const BlockArgs& a, double* partials, double* out, cudaStream_t s) {
  const int nb = block_grid(a.N);
  k_block_stats<<<nb, BT, 0, s>>>(a, partials);
  k_block_stats_final<<<1, 32, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}
cudaError_t launch_pack2(const float* a, const float* b, int64_t n, float2* out, cudaStream_t s) {
  k_pack2<<<block_grid(n), BT, 0, s>>>(a, b, n, out);
  return cudaGetLastError();
}

}  // namespace usp
