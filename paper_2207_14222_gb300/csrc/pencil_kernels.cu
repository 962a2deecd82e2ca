// pencil_kernels.cu -- the pencil schedule of one fixed-point iteration
// (paper Algorithm 1 on the forward-eliminated operator of Sec. 2.1):
//
//   rows pass   : t = (1-V) x + y ; FFT along the contiguous axis      [B x + y]
//   column pass : FFT along each strided axis; on the outermost axis
//                 FFT -> multiply by 1/(N (Lhat(p)+1)) -> inverse FFT   [(L+I)^-1,
//                                                                        Eq. laplacian_inverse]
//   column pass : inverse FFT along the remaining strided axes
//   rows pass   : inverse FFT along the contiguous axis;
//                 Delta = (1-V)(u - x); x += alpha Delta; ||Delta||^2   [Delta, update,
//                                                                        convergence test]
//
// The same kernels, instantiated in FP64 (here) and double-float
// (df_kernels.cu) with the multiplier Lhat(p)/N, form the residual y - A x
// used by iterative refinement.
//
// The kernel templates are in pencil_core.cuh; this unit instantiates them
// for float and double and holds their twiddle tables and the auxiliary
// kernels.
#include "pencil_core.cuh"

namespace usp {

// W_256^m = exp(-2 pi i m/256), m in [0,256).  W_n^m = W_256^(m 256/n).
__device__ float2 g_tw32[256];
__device__ double2 g_tw64[256];

template <>
__device__ __forceinline__ float2 tw_entry<float>(int m) { return g_tw32[m]; }
template <>
__device__ __forceinline__ double2 tw_entry<double>(int m) { return g_tw64[m]; }

// W_1536^m, m in [0,1536)
__device__ float2 g_twx32[TWX_LEN];
__device__ double2 g_twx64[TWX_LEN];

template <>
__device__ __forceinline__ float2 twx_entry<float>(int m) { return g_twx32[m]; }
template <>
__device__ __forceinline__ double2 twx_entry<double>(int m) { return g_twx64[m]; }

cudaError_t launch_rows_f32(int n, const RowsArgs<float>& a, int64_t grid, cudaStream_t s) {
#define C_(N) rows_go<float, N>(a, grid, s)
  USP_SWITCH_N(n, C_)
#undef C_
}
cudaError_t launch_rows_f64(int n, const RowsArgs<double>& a, int64_t grid, cudaStream_t s) {
#define C_(N) rows_go<double, N>(a, grid, s)
  USP_SWITCH_N(n, C_)
#undef C_
}
cudaError_t launch_cols_f32(int n, const ColsArgs<float>& a, cudaStream_t s) {
#define C_(N) cols_go<float, N>(a, s)
  USP_SWITCH_N(n, C_)
#undef C_
}
cudaError_t launch_cols_f64(int n, const ColsArgs<double>& a, cudaStream_t s) {
#define C_(N) cols_go<double, N>(a, s)
  USP_SWITCH_N(n, C_)
#undef C_
}

static int switch_rows_f32(int n) {
#define C_(N) RowsShape<float, N>::F
  USP_SWITCH_N(n, C_)
#undef C_
}
static int switch_rows_f64(int n) {
#define C_(N) RowsShape<double, N>::F
  USP_SWITCH_N(n, C_)
#undef C_
}
static int switch_cols(int n) {
#define C_(N) ColsShape<N>::COLS
  USP_SWITCH_N(n, C_)
#undef C_
}
int rows_per_block_f32(int n) { return switch_rows_f32(n); }
int rows_per_block_f64(int n) { return switch_rows_f64(n); }
int cols_per_block(int n) { return switch_cols(n); }

// Twiddles from the first octant by symmetry, so W^(64 j) are exactly
// 1, -i, -1, i and the table is exactly symmetric.
const float2* twiddle_x_table_f32() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_twx32) != cudaSuccess) return nullptr;
  return reinterpret_cast<const float2*>(p);
}

const float2* twiddle_table_f32() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tw32) != cudaSuccess) return nullptr;
  return static_cast<const float2*>(p);
}

// exp(-2 pi i m / L) for m in [0, L), L a multiple of 8, from the first
// octant by symmetry (quarter turns are exact).
static void unit_roots(int L, double2* out) {
  const double two_pi = 6.283185307179586476925286766559;
  const int Q = L / 4;
  for (int m = 0; m < L; ++m) {
    const int q = m / Q, r = m % Q;
    double c, s;  // cos, sin of 2 pi r/L, r in [0, L/4)
    if (2 * r <= Q) {
      c = cos(two_pi * r / L);
      s = sin(two_pi * r / L);
    } else {
      c = sin(two_pi * (Q - r) / L);
      s = cos(two_pi * (Q - r) / L);
    }
    if (r == 0) { c = 1.0; s = 0.0; }
    for (int k = 0; k < q; ++k) {  // rotate by q quarter turns
      const double t = c;
      c = -s;
      s = t;
    }
    out[m] = make_double2(c, -s);
  }
}

cudaError_t init_twiddles() {
  static double2 h64[256], x64[TWX_LEN];
  static float2 h32[256], x32[TWX_LEN];
  unit_roots(256, h64);
  unit_roots(TWX_LEN, x64);
  for (int m = 0; m < 256; ++m) h32[m] = make_float2((float)h64[m].x, (float)h64[m].y);
  for (int m = 0; m < TWX_LEN; ++m) x32[m] = make_float2((float)x64[m].x, (float)x64[m].y);
  cudaError_t e = cudaMemcpyToSymbol(g_tw32, h32, sizeof(h32));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_tw64, h64, sizeof(h64));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_twx32, x32, sizeof(x32));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_twx64, x64, sizeof(x64));
  if (e != cudaSuccess) return e;
  if ((e = attrs_all<float>()) != cudaSuccess) return e;
  if ((e = attrs_all<double>()) != cudaSuccess) return e;
  return init_twiddles_df(h64, x64);
}

// -------------------------------------------------------- auxiliaries ---

// Statistics of V for validation and alpha = Re[B^-1] = min_r Re 1/(1 - V):
// per-thread FP32 (V is FP32 data; Re 1/(1-V) = (1-Re V)/|1-V|^2 needs no
// more), block and grid reductions in FP64.
__global__ void k_v_stats(const void* V, int vreal, int64_t n, double* partials) {
  float vmax = 0.f, amin = 3.0e38f;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = vreal ? make_float2(reinterpret_cast<const float*>(V)[i], 0.f)
                           : reinterpret_cast<const float2*>(V)[i];
    if (!isfinite(v.x) || !isfinite(v.y)) {
      ++bad;
      continue;
    }
    vmax = fmaxf(vmax, sqrtf(v.x * v.x + v.y * v.y));
    const float br = 1.f - v.x;                       // B = 1 - V
    amin = fminf(amin, br / (br * br + v.y * v.y));   // Re 1/B
  }
  __shared__ float r0[8], r1[8];
  __shared__ int r2[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vmax = fmaxf(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    amin = fminf(amin, __shfl_down_sync(0xffffffffu, amin, o));
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    r0[w] = vmax;
    r1[w] = amin;
    r2[w] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      r0[0] = fmaxf(r0[0], r0[i]);
      r1[0] = fminf(r1[0], r1[i]);
      r2[0] += r2[i];
    }
    partials[3 * blockIdx.x] = r0[0];
    partials[3 * blockIdx.x + 1] = r1[0];
    partials[3 * blockIdx.x + 2] = r2[0];
  }
}

__global__ void k_v_stats_final(const double* partials, int nb, double* out) {
  double vmax = 0.0, amin = 1e300, bad = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) {
    vmax = fmax(vmax, partials[3 * b]);
    amin = fmin(amin, partials[3 * b + 1]);
    bad += partials[3 * b + 2];
  }
  __shared__ double s0[256], s1[256], s2[256];
  s0[threadIdx.x] = vmax;
  s1[threadIdx.x] = amin;
  s2[threadIdx.x] = bad;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s0[threadIdx.x] = fmax(s0[threadIdx.x], s0[threadIdx.x + h]);
      s1[threadIdx.x] = fmin(s1[threadIdx.x], s1[threadIdx.x + h]);
      s2[threadIdx.x] += s2[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
    out[2] = s2[0];
  }
}

cudaError_t launch_v_stats(const void* V, int vreal, int64_t n, double* partials, int nblocks,
                           double* out, cudaStream_t s) {
  k_v_stats<<<nblocks, 256, 0, s>>>(V, vreal, n, partials);
  k_v_stats_final<<<1, 256, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

// min over the table of Re(Lhat) + 1 and the count of non-finite entries.
__global__ void k_table_stats(const float2* t, int64_t n, double* partials) {
  float rmin = 3.0e38f;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 l = t[i];
    if (!isfinite(l.x) || !isfinite(l.y)) {
      ++bad;
      continue;
    }
    rmin = fminf(rmin, l.x + 1.f);
  }
  __shared__ float r0[8];
  __shared__ int r1[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmin = fminf(rmin, __shfl_down_sync(0xffffffffu, rmin, o));
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = rmin;
    r1[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      r0[0] = fminf(r0[0], r0[i]);
      r1[0] += r1[i];
    }
    partials[2 * blockIdx.x] = r0[0];
    partials[2 * blockIdx.x + 1] = r1[0];
  }
}

__global__ void k_table_stats_final(const double* partials, int nb, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rmin = 1e300, bad = 0.0;
  for (int b = 0; b < nb; ++b) {
    rmin = fmin(rmin, partials[2 * b]);
    bad += partials[2 * b + 1];
  }
  out[0] = rmin;
  out[1] = bad;
}

cudaError_t launch_table_stats(const float2* table, int64_t n, double* partials, int nblocks,
                               double* out, cudaStream_t s) {
  k_table_stats<<<nblocks, 256, 0, s>>>(table, n, partials);
  k_table_stats_final<<<1, 32, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

__global__ void k_axpy1(float2* x, const float2* z, int64_t n, const int* mask, int64_t n_per) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask && !mask[i / n_per]) continue;
    const float2 a = x[i], b = z[i];
    x[i] = make_float2(a.x + b.x, a.y + b.y);
  }
}

cudaError_t launch_axpy1(float2* x, const float2* z, int64_t n, cudaStream_t s, const int* mask,
                         int64_t n_per) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_axpy1<<<(unsigned)blocks, 256, 0, s>>>(x, z, n, mask, n_per > 0 ? n_per : n);
  return cudaGetLastError();
}

// Block b sums the `count` partial pairs of group b (2 doubles per block).
__global__ void k_sum_pairs(const double* partials, int count, double* out) {
  __shared__ double red[8];
  const double* pp = partials + 2 * (int64_t)blockIdx.x * count;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < count; i += 256) {
    a += pp[2 * i];
    b += pp[2 * i + 1];
  }
  const double sa = block_sum<256>(a, red);
  const double sb = block_sum<256>(b, red);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sa;
    out[2 * blockIdx.x + 1] = sb;
  }
}

cudaError_t launch_sum_pairs(const double* partials, int count, int groups, double* out,
                             cudaStream_t s) {
  k_sum_pairs<<<groups, 256, 0, s>>>(partials, count, out);
  return cudaGetLastError();
}

cudaError_t launch_copy_bytes(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

}  // namespace usp
