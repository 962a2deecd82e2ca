// fno_kernels.cu -- kernels of the Fourier neural operator that proposes the
// iteration's initial estimate x0 (the paper's Algorithm 1 starts from any
// x0; this network is the library's own addition, Li et al.'s operator
// restated).  FP32 arithmetic; every reduction runs in a fixed order, so a
// training step is deterministic.
//
// The spectral layer keeps modes x modes frequencies, so its transforms are
// truncated DFTs evaluated directly: a plane of H x W pixels contracts with a
// modes x W and a modes x H table of unit roots (staged in shared memory),
// which costs 2 modes (H W + modes H) multiply-adds per plane instead of a
// full FFT and leaves the retained modes in shared memory for the mixing.
#include <math.h>

#include "fno_kernels.h"

namespace usp {

namespace {

constexpr int FNO_THREADS = 256;
constexpr int WGRAD_BLOCKS = 512;   // blocks of the weight-gradient reduction
constexpr int WGRAD_TILE = 32;      // pixels per shared-memory tile
constexpr int LOSS_BLOCKS = 16;     // blocks per sample of the loss

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// ------------------------------------------------------------ 1x1 conv ---

template <int CMAX>
__global__ void __launch_bounds__(FNO_THREADS) k_conv(CStrided in, int cin, const float* W,
                                                      int64_t so, int64_t sc, const float* bias,
                                                      Strided out, int cout, int64_t P,
                                                      bool accumulate) {
  __shared__ float w[64 * 64];
  __shared__ float bsh[64];
  for (int i = threadIdx.x; i < cout * cin; i += FNO_THREADS) {
    const int o = i / cin, c = i % cin;
    w[i] = W[o * so + c * sc];
  }
  for (int o = threadIdx.x; o < cout; o += FNO_THREADS) bsh[o] = bias ? bias[o] : 0.f;
  __syncthreads();
  const int64_t b = blockIdx.y;
  const int64_t p = (int64_t)blockIdx.x * FNO_THREADS + threadIdx.x;
  if (p >= P) return;
  float x[CMAX];
#pragma unroll
  for (int c = 0; c < CMAX; ++c) x[c] = c < cin ? in.ptr[b * in.bs + c * in.cs + p * in.ps] : 0.f;
  for (int o = 0; o < cout; ++o) {
    float a = bsh[o];
#pragma unroll
    for (int c = 0; c < CMAX; ++c)
      if (c < cin) a = fmaf(w[o * cin + c], x[c], a);
    float* dst = out.ptr + b * out.bs + o * out.cs + p * out.ps;
    *dst = accumulate ? *dst + a : a;
  }
}

// --------------------------------------------------------- truncated DFT ---

__global__ void __launch_bounds__(FNO_THREADS) k_dft2(const float* in, int H, int W, int modes,
                                                      const float2* twh, const float2* tww,
                                                      float2* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sw = reinterpret_cast<float2*>(smem_raw);   // [W][modes]
  float2* sh = sw + W * modes;                         // [H][modes]
  float2* T = sh + H * modes;                          // [H][modes]
  float* rows = reinterpret_cast<float*>(T + H * modes);
  const int RC = FNO_THREADS / modes;                  // rows per chunk
  const int tid = threadIdx.x;
  for (int i = tid; i < W * modes; i += FNO_THREADS) sw[i] = tww[i];
  for (int i = tid; i < H * modes; i += FNO_THREADS) sh[i] = twh[i];
  const float* pin = in + (int64_t)blockIdx.x * H * W;
  const int r = tid / modes, s = tid % modes;
  for (int r0 = 0; r0 < H; r0 += RC) {
    __syncthreads();  // the previous chunk's rows are consumed
    for (int idx = tid; idx < RC * W; idx += FNO_THREADS) {
      const int rr = r0 + idx / W;
      rows[idx] = rr < H ? pin[(int64_t)rr * W + idx % W] : 0.f;
    }
    __syncthreads();
    if (r0 + r < H) {
      float ax = 0.f, ay = 0.f;
      const float* row = rows + r * W;
      for (int j = 0; j < W; ++j) {
        const float xv = row[j];
        const float2 t = sw[j * modes + s];
        ax = fmaf(xv, t.x, ax);
        ay = fmaf(xv, t.y, ay);
      }
      T[(r0 + r) * modes + s] = make_float2(ax, ay);
    }
  }
  __syncthreads();
  const int mm = modes * modes;
  float2* po = out + (int64_t)blockIdx.x * mm;
  for (int o = tid; o < mm; o += FNO_THREADS) {
    const int m1 = o / modes, s2 = o % modes;
    float ax = 0.f, ay = 0.f;
    for (int i = 0; i < H; ++i) {
      const float2 t = T[i * modes + s2], w = sh[i * modes + m1];
      ax = fmaf(t.x, w.x, fmaf(-t.y, w.y, ax));
      ay = fmaf(t.x, w.y, fmaf(t.y, w.x, ay));
    }
    po[o] = make_float2(ax, ay);
  }
}

__global__ void __launch_bounds__(FNO_THREADS) k_idft2(const float2* Z, int H, int W, int modes,
                                                       const float2* twh, const float2* tww,
                                                       float scale, float* acc, float* act) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sh = reinterpret_cast<float2*>(smem_raw);   // [H][modes]
  float2* swT = sh + H * modes;                        // [modes][W]
  float2* U = swT + modes * W;                         // [H][modes]
  float2* Zs = U + H * modes;                          // [modes][modes]
  const int tid = threadIdx.x;
  const int mm = modes * modes;
  for (int i = tid; i < H * modes; i += FNO_THREADS) sh[i] = twh[i];
  for (int i = tid; i < W * modes; i += FNO_THREADS) {
    const int j = i / modes, s = i % modes;
    swT[s * W + j] = tww[i];
  }
  const float2* pz = Z + (int64_t)blockIdx.x * mm;
  for (int i = tid; i < mm; i += FNO_THREADS) Zs[i] = pz[i];
  __syncthreads();
  // U[i][s] = sum_m1 Z[m1][s] e^{+2 pi i k1 i / H}
  for (int o = tid; o < H * modes; o += FNO_THREADS) {
    const int i = o / modes, s = o % modes;
    float ax = 0.f, ay = 0.f;
    for (int m1 = 0; m1 < modes; ++m1) {
      const float2 z = Zs[m1 * modes + s], w = sh[i * modes + m1];   // z conj(w)
      ax = fmaf(z.x, w.x, fmaf(z.y, w.y, ax));
      ay = fmaf(z.y, w.x, fmaf(-z.x, w.y, ay));
    }
    U[o] = make_float2(ax, ay);
  }
  __syncthreads();
  float* pa = acc + (int64_t)blockIdx.x * H * W;
  float* pact = act ? act + (int64_t)blockIdx.x * H * W : nullptr;
  for (int idx = tid; idx < H * W; idx += FNO_THREADS) {
    const int i = idx / W, j = idx % W;
    float v = 0.f;
    for (int s = 0; s < modes; ++s) {
      const float2 u = U[i * modes + s], w = swT[s * W + j];   // Re(u conj(w))
      v = fmaf(u.x, w.x, fmaf(u.y, w.y, v));
    }
    const float a = pa[idx] + scale * v;
    pa[idx] = a;
    if (pact) pact[idx] = gelu_f(a);
  }
}

// --------------------------------------------------------------- mixing ---

// R and dR live inside the flat parameter vector at any float offset, so
// they are accessed as separate floats (a float2 access needs 8-byte
// alignment).
__global__ void k_mix(const float2* X, const float* R, int batch, int nin, int nout, int mm,
                      bool adjoint, float2* Z) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)batch * nout * mm;
  if (idx >= total) return;
  const int m = int(idx % mm);
  const int oc = int((idx / mm) % nout);
  const int64_t b = idx / ((int64_t)mm * nout);
  float ax = 0.f, ay = 0.f;
  for (int c = 0; c < nin; ++c) {
    const float2 x = X[(b * nin + c) * mm + m];
    if (!adjoint) {
      const int64_t ri = 2 * (((int64_t)oc * nin + c) * mm + m);
      const float2 r = make_float2(R[ri], R[ri + 1]);                 // r x
      ax = fmaf(r.x, x.x, fmaf(-r.y, x.y, ax));
      ay = fmaf(r.x, x.y, fmaf(r.y, x.x, ay));
    } else {
      const int64_t ri = 2 * (((int64_t)c * nout + oc) * mm + m);
      const float2 r = make_float2(R[ri], R[ri + 1]);                 // conj(r) x
      ax = fmaf(r.x, x.x, fmaf(r.y, x.y, ax));
      ay = fmaf(r.x, x.y, fmaf(-r.y, x.x, ay));
    }
  }
  Z[idx] = make_float2(ax, ay);
}

__global__ void k_dR(const float2* G, const float2* X, int batch, int O, int C, int mm,
                     float scale, float* dR) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)O * C * mm) return;
  const int m = int(idx % mm);
  const int c = int((idx / mm) % C);
  const int o = int(idx / ((int64_t)mm * C));
  float ax = 0.f, ay = 0.f;
  for (int b = 0; b < batch; ++b) {
    const float2 g = G[((int64_t)b * O + o) * mm + m], x = X[((int64_t)b * C + c) * mm + m];
    ax = fmaf(g.x, x.x, fmaf(g.y, x.y, ax));      // g conj(x)
    ay = fmaf(g.y, x.x, fmaf(-g.x, x.y, ay));
  }
  dR[2 * idx] = scale * ax;
  dR[2 * idx + 1] = scale * ay;
}

// ------------------------------------------------------ weight gradients ---

__global__ void __launch_bounds__(FNO_THREADS) k_wgrad(CStrided g, int O, CStrided v, int C,
                                                       int64_t P, int64_t N, int64_t chunk,
                                                       float* partials) {
  __shared__ float gt[64][WGRAD_TILE];
  __shared__ float vt[64][WGRAD_TILE + 1];
  const int tid = threadIdx.x;
  const int pairs = O * C;
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.f;
  float dacc = 0.f;
  const int64_t n_begin = (int64_t)blockIdx.x * chunk;
  const int64_t n_end = n_begin + chunk < N ? n_begin + chunk : N;
  for (int64_t n0 = n_begin; n0 < n_end; n0 += WGRAD_TILE) {
    for (int idx = tid; idx < O * WGRAD_TILE; idx += FNO_THREADS) {
      const int o = idx / WGRAD_TILE, k = idx % WGRAD_TILE;
      const int64_t n = n0 + k;
      float val = 0.f;
      if (n < n_end) {
        const int64_t b = n / P, p = n % P;
        val = g.ptr[b * g.bs + o * g.cs + p * g.ps];
      }
      gt[o][k] = val;
    }
    for (int idx = tid; idx < C * WGRAD_TILE; idx += FNO_THREADS) {
      const int c = idx / WGRAD_TILE, k = idx % WGRAD_TILE;
      const int64_t n = n0 + k;
      float val = 0.f;
      if (n < n_end) {
        const int64_t b = n / P, p = n % P;
        val = v.ptr[b * v.bs + c * v.cs + p * v.ps];
      }
      vt[c][k] = val;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int pr = tid + q * FNO_THREADS;
      if (pr < pairs) {
        const int o = pr / C, c = pr % C;
        float a = acc[q];
#pragma unroll 8
        for (int k = 0; k < WGRAD_TILE; ++k) a = fmaf(gt[o][k], vt[c][k], a);
        acc[q] = a;
      }
    }
    if (tid < O) {
      for (int k = 0; k < WGRAD_TILE; ++k) dacc += gt[tid][k];
    }
    __syncthreads();
  }
  float* pp = partials + (int64_t)blockIdx.x * (pairs + O);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int pr = tid + q * FNO_THREADS;
    if (pr < pairs) pp[pr] = acc[q];
  }
  if (tid < O) pp[pairs + tid] = dacc;
}

// Sum the blocks' partials in block order (deterministic) into dW and db.
__global__ void k_wgrad_sum(const float* partials, int nblocks, int O, int C, float* dW,
                            float* db) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int pairs = O * C;
  if (e >= pairs + O) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += (double)partials[(int64_t)b * (pairs + O) + e];
  if (e < pairs) dW[e] = (float)s;
  else if (db) db[e - pairs] = (float)s;
}

// ---------------------------------------------------------- elementwise ---

__global__ void k_gelu_bwd(float* x, const float* z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= gelu_grad_f(z[i]);
}

// ----------------------------------------------------------------- loss ---

__global__ void __launch_bounds__(FNO_THREADS) k_loss_part(const float2* xh, const float2* x,
                                                           int64_t P, double* partials) {
  __shared__ double r0[FNO_THREADS / 32], r1[FNO_THREADS / 32];
  const int64_t b = blockIdx.y;
  const int64_t chunk = (P + LOSS_BLOCKS - 1) / LOSS_BLOCKS;
  const int64_t p0 = blockIdx.x * chunk, p1 = p0 + chunk < P ? p0 + chunk : P;
  double num = 0.0, den = 0.0;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += FNO_THREADS) {
    const float2 a = xh[b * P + p], t = x[b * P + p];
    const double dx = (double)a.x - t.x, dy = (double)a.y - t.y;
    num += dx * dx + dy * dy;
    den += (double)t.x * t.x + (double)t.y * t.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = num;
    r1[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int i = 0; i < FNO_THREADS / 32; ++i) {
      a += r0[i];
      c += r1[i];
    }
    partials[(b * LOSS_BLOCKS + blockIdx.x) * 2] = a;
    partials[(b * LOSS_BLOCKS + blockIdx.x) * 2 + 1] = c;
  }
}

// One thread: per-sample sums in block order, the mean loss, and the
// per-sample gradient scales 2 / (batch ||x_b||^2) after the partials.
__global__ void k_loss_finish(double* partials, int batch, double* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* scales = partials + (int64_t)batch * LOSS_BLOCKS * 2;
  double tot = 0.0;
  for (int b = 0; b < batch; ++b) {
    double num = 0.0, den = 0.0;
    for (int k = 0; k < LOSS_BLOCKS; ++k) {
      num += partials[(b * LOSS_BLOCKS + k) * 2];
      den += partials[(b * LOSS_BLOCKS + k) * 2 + 1];
    }
    tot += den > 0.0 ? num / den : 0.0;
    scales[b] = den > 0.0 ? 2.0 / (batch * den) : 0.0;
  }
  *loss = tot / batch;
}

__global__ void k_loss_grad(const float2* xh, const float2* x, int64_t P, int64_t n,
                            const double* scales, float2* gu) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float sc = (float)scales[i / P];
    const float2 a = xh[i], t = x[i];
    gu[i] = make_float2(sc * (a.x - t.x), sc * (a.y - t.y));
  }
}

// ----------------------------------------------------------------- adam ---

__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                       float beta1, float beta2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t fno_conv(CStrided in, int cin, const float* W, int64_t so, int64_t sc,
                     const float* bias, Strided out, int cout, int batch, int64_t P,
                     bool accumulate, cudaStream_t s) {
  if (cin < 1 || cin > 64 || cout < 1 || cout > 64) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((P + FNO_THREADS - 1) / FNO_THREADS), (unsigned)batch);
  if (cin <= 8)
    k_conv<8><<<grid, FNO_THREADS, 0, s>>>(in, cin, W, so, sc, bias, out, cout, P, accumulate);
  else if (cin <= 32)
    k_conv<32><<<grid, FNO_THREADS, 0, s>>>(in, cin, W, so, sc, bias, out, cout, P, accumulate);
  else
    k_conv<64><<<grid, FNO_THREADS, 0, s>>>(in, cin, W, so, sc, bias, out, cout, P, accumulate);
  return cudaGetLastError();
}

static size_t dft2_smem(int H, int W, int modes) {
  return sizeof(float2) * ((size_t)W * modes + 2 * (size_t)H * modes) +
         sizeof(float) * (size_t)(FNO_THREADS / modes) * W;
}
static size_t idft2_smem(int H, int W, int modes) {
  return sizeof(float2) * (2 * (size_t)H * modes + (size_t)W * modes + (size_t)modes * modes);
}

size_t fno_smem_bytes(int H, int W, int modes) {
  const size_t a = dft2_smem(H, W, modes), b = idft2_smem(H, W, modes);
  return a > b ? a : b;
}

cudaError_t fno_dft2(const float* in, int64_t planes, int H, int W, int modes,
                     const float2* twh, const float2* tww, float2* out, cudaStream_t s) {
  if (modes < 2 || modes > 32 || (FNO_THREADS % modes) != 0) return cudaErrorInvalidValue;
  const size_t sm = dft2_smem(H, W, modes);
  cudaError_t e = cudaFuncSetAttribute(k_dft2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_dft2<<<(unsigned)planes, FNO_THREADS, sm, s>>>(in, H, W, modes, twh, tww, out);
  return cudaGetLastError();
}

cudaError_t fno_idft2(const float2* Z, int64_t planes, int H, int W, int modes,
                      const float2* twh, const float2* tww, float scale, float* acc,
                      float* act, cudaStream_t s) {
  const size_t sm = idft2_smem(H, W, modes);
  cudaError_t e = cudaFuncSetAttribute(k_idft2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_idft2<<<(unsigned)planes, FNO_THREADS, sm, s>>>(Z, H, W, modes, twh, tww, scale, acc, act);
  return cudaGetLastError();
}

cudaError_t fno_mix(const float2* X, const float* R, int batch, int nin, int nout, int mm,
                    bool adjoint, float2* Z, cudaStream_t s) {
  const int64_t total = (int64_t)batch * nout * mm;
  k_mix<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, R, batch, nin, nout, mm, adjoint, Z);
  return cudaGetLastError();
}

cudaError_t fno_dR(const float2* G, const float2* X, int batch, int O, int C, int mm,
                   float scale, float* dR, cudaStream_t s) {
  const int64_t total = (int64_t)O * C * mm;
  k_dR<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(G, X, batch, O, C, mm, scale, dR);
  return cudaGetLastError();
}

int64_t fno_wgrad_partials(int O, int C) { return (int64_t)WGRAD_BLOCKS * (O * C + O); }

cudaError_t fno_wgrad(CStrided g, int O, CStrided v, int C, int batch, int64_t P,
                      float* partials, float* dW, float* db, cudaStream_t s) {
  if (O < 1 || O > 64 || C < 1 || C > 64 || O * C > 16 * FNO_THREADS) return cudaErrorInvalidValue;
  const int64_t N = (int64_t)batch * P;
  int64_t nb = (N + 1023) / 1024;
  if (nb > WGRAD_BLOCKS) nb = WGRAD_BLOCKS;
  if (nb < 1) nb = 1;
  int64_t chunk = (N + nb - 1) / nb;
  chunk = (chunk + WGRAD_TILE - 1) / WGRAD_TILE * WGRAD_TILE;
  nb = (N + chunk - 1) / chunk;
  k_wgrad<<<(unsigned)nb, FNO_THREADS, 0, s>>>(g, O, v, C, P, N, chunk, partials);
  const int outs = O * C + O;
  k_wgrad_sum<<<(unsigned)((outs + 255) / 256), 256, 0, s>>>(partials, (int)nb, O, C, dW, db);
  return cudaGetLastError();
}

cudaError_t fno_gelu_bwd(float* x, const float* z, int64_t n, cudaStream_t s) {
  k_gelu_bwd<<<grid_for(n, 256), 256, 0, s>>>(x, z, n);
  return cudaGetLastError();
}

int64_t fno_loss_partials(int batch) { return (int64_t)batch * LOSS_BLOCKS * 2 + batch; }

cudaError_t fno_loss(const float2* xh, const float2* x, int batch, int64_t P, double* partials,
                     double* loss, float2* gu, cudaStream_t s) {
  k_loss_part<<<dim3(LOSS_BLOCKS, (unsigned)batch), FNO_THREADS, 0, s>>>(xh, x, P, partials);
  k_loss_finish<<<1, 32, 0, s>>>(partials, batch, loss);
  if (gu) {
    const int64_t n = (int64_t)batch * P;
    k_loss_grad<<<grid_for(n, 256), 256, 0, s>>>(xh, x, P, n,
                                                 partials + (int64_t)batch * LOSS_BLOCKS * 2, gu);
  }
  return cudaGetLastError();
}

cudaError_t fno_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                     float beta1, float beta2, float eps, float c1, float c2, cudaStream_t s) {
  k_adam<<<grid_for(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace usp
