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
// The same kernels, instantiated in FP64 with the multiplier Lhat(p)/N, form
// the residual y - A x used by iterative refinement.
//
// Memory layout: C order, last axis fastest.  Rows kernels: G = N2 adjacent
// lanes own one row, each thread holds N1 values (see fft_core.cuh), so for
// a fixed register the G threads touch G consecutive elements.  Column
// kernels: one warp per stage-1 thread index g, the 32 lanes own 32
// consecutive columns, so every global access of a warp is 32 consecutive
// complex values.
#include <math.h>

#include "fft_core.cuh"
#include "iteration_state.cuh"
#include "kernels.h"

namespace usp {

// W_256^m = exp(-2 pi i m/256), m in [0,256).  W_n^m = W_256^(m 256/n).
__device__ float2 g_tw32[256];
__device__ double2 g_tw64[256];

template <typename T>
__device__ __forceinline__ typename cplx_of<T>::type tw_entry(int m);
template <>
__device__ __forceinline__ float2 tw_entry<float>(int m) { return g_tw32[m]; }
template <>
__device__ __forceinline__ double2 tw_entry<double>(int m) { return g_tw64[m]; }

// FP32 rows: 4 blocks of 256 threads per SM (64 registers) -- measured
// 3.77 TB/s for the fused rows pass versus 3.45 TB/s at 3 blocks (80
// registers) and 1.88 TB/s when ptxas is left to use 210 registers.
template <typename T> struct RowsCfg;
template <> struct RowsCfg<float> {
  static constexpr int THREADS = 256;
  static constexpr int MINB = 4;
};
template <> struct RowsCfg<double> {
  static constexpr int THREADS = 128;
  static constexpr int MINB = 1;
};

// ------------------------------------------------------------ reductions ---

template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < THREADS / 32; ++i) s += red[i];
  }
  return s;  // valid in thread 0
}

// Block partial of ||Delta||^2 into partials[part_index]; the last of the
// problem's part_count blocks to finish sums the problem's partials
// [part_first, part_first + part_count) in a fixed order (deterministic) and
// updates its state.
template <int THREADS>
__device__ void reduce_and_finalize(double acc, double* partials, int64_t part_index,
                                    int64_t part_first, int64_t part_count, DevState* st,
                                    double* hist, int flags) {
  __shared__ double red[THREADS / 32];
  __shared__ int is_last;
  const double bs = block_sum<THREADS>(acc, red);
  if (threadIdx.x == 0) {
    partials[part_index] = bs;
    __threadfence();
    const unsigned t = atomicAdd(&st->ticket, 1u);
    is_last = (t == (unsigned)(part_count - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < part_count; i += THREADS) s += __ldcg(partials + part_first + i);
  const double tot = block_sum<THREADS>(s, red);
  if (threadIdx.x == 0) {
    finalize_iteration(st, hist, tot, flags);
    st->ticket = 0u;
  }
}

// ------------------------------------------------------- spectral factor ---

// a / b: FP32 uses the fast reciprocal-based division (about 2 ulp, enough for
// the multiplier 1/(N(Lhat+1)), whose denominator is at least 1); FP64 (the
// refinement residual) divides exactly.
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double quot(double a, double b) { return a / b; }

template <typename T, typename V>
__device__ __forceinline__ V spectral_factor(T p2, const Sym<T>& s, int mul) {
  const T lr = s.a_re * p2 + s.b_re;
  const T li = s.a_im * p2 + s.b_im;
  if (mul == MUL_L) return mkc<V>(lr * s.inv_n, li * s.inv_n);
  const T dr = lr + T(1);
  const T sc = quot(s.inv_n, dr * dr + li * li);
  return mkc<V>(dr * sc, -li * sc);
}

// |p|^2 contributed by axis `ax` at frequency index k.
template <typename T>
__device__ __forceinline__ T axis_p2(const Sym<T>& s, int ax, int k) {
  const T p = s.ks[ax] * T(signed_freq(k, s.n[ax]));
  return p * p;
}

// --------------------------------------------------------------- rows ---

template <int N, bool INV, typename V>
__device__ __forceinline__ void fft_rows(V* v, V* exr, const V* tw, int g) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  stage1<N, INV>(v, g, tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) exr[k1 * N2 + (g ^ (k1 & (N2 - 1)))] = v[k1];
  __syncthreads();
  V w[N1];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k1 = g + G * s;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) w[s * N2 + n2] = exr[k1 * N2 + (n2 ^ (k1 & (N2 - 1)))];
  }
  __syncthreads();
  stage2<N, INV>(w);
#pragma unroll
  for (int q = 0; q < N1; ++q) v[q] = w[q];
}

__device__ __forceinline__ float2 load_v(const void* V, int64_t i, bool vreal) {
  if (vreal) return make_float2(__ldg(reinterpret_cast<const float*>(V) + i), 0.f);
  return __ldg(reinterpret_cast<const float2*>(V) + i);
}

template <typename T, int N>
__global__ void __launch_bounds__(RowsCfg<T>::THREADS, RowsCfg<T>::MINB) k_rows(const RowsArgs<T> a) {
  typedef typename cplx_of<T>::type V;
  constexpr int N1 = Split<N>::N1, G = Split<N>::G;
  constexpr int THREADS = RowsCfg<T>::THREADS;
  constexpr int F = THREADS / G;  // rows per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* ex = tw + N;

  // the problem of this block (blocks never straddle problems)
  const int p = a.bt.count > 1 ? int((int64_t)blockIdx.x * F / a.bt.rows_per) : 0;
  DevState* st = a.st + p;
  if (!(a.flags & F_NOSTATE) && st->done) return;

  const int tid = threadIdx.x, f = tid / G, g = tid % G;
  const int64_t row = (int64_t)blockIdx.x * F + f;
  const bool active = row < a.nrows;
  const int64_t base = row * N;
  const bool xzero = (a.flags & F_XZERO) != 0;
  const bool vreal = (a.flags & F_VREAL) != 0;
  for (int m = tid; m < N; m += THREADS) tw[m] = tw_entry<T>(stage1_twiddle_exponent(m, Split<N>::N2) * (256 / N));
  __syncthreads();
  V* exr = ex + f * N;

  V v[N1];
  // ---- input stage (stage-1 distribution: register q holds index N2 q + g)
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    const int64_t i = base + in_index<N>(g, q);
    V t = mkc<V>(T(0), T(0));
    if (active) {
      if (a.mode & R_IN_BUF) {
        t = reinterpret_cast<const V*>(a.buf)[i];
      } else if (a.mode & R_IN_X) {
        const float2 xv = a.x_in[i];
        t = mkc<V>(T(xv.x), T(xv.y));
      } else {  // R_IN_PRE: B x + y
        const float2 yv = a.y[i];
        float2 tv = yv;
        if (!xzero) {
          const float2 vv = load_v(a.V, i, vreal);
          const float2 xv = a.x_in[i];
          const float br = 1.f - vv.x, bi = -vv.y;
          tv.x += br * xv.x - bi * xv.y;
          tv.y += br * xv.y + bi * xv.x;
        }
        t = mkc<V>(T(tv.x), T(tv.y));
      }
    }
    v[q] = t;
  }
  // ---- transforms
  if (a.mode & R_FWD) fft_rows<N, false>(v, exr, tw, g);
  if (a.mode & R_MUL) {
    const Sym<T> sy = problem_sym(a.sym, a.bt, p);
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const int k = out_index<N>(g, q);
      v[q] = cmul(v[q], spectral_factor<T, V>(axis_p2(sy, 0, k), sy, a.mul));
    }
  }
  if (a.mode & R_INV) {
    if (a.mode & R_FWD) {
      V t[N1];
      out_to_in<N>(v, t);
#pragma unroll
      for (int q = 0; q < N1; ++q) v[q] = t[q];
    }
    fft_rows<N, true>(v, exr, tw, g);
  }
  // ---- output stage (register q holds index out_index(g, q))
  if (a.mode & R_OUT_BUF) {
    if (active) {
#pragma unroll
      for (int q = 0; q < N1; ++q)
        reinterpret_cast<V*>(a.buf)[base + out_index<N>(g, q)] = v[q];
    }
    return;
  }
  if (a.mode & R_OUT_POST) {
    // Delta = (1-V)(u - x) ; x += alpha Delta  (Algorithm 1)
    float acc = 0.f;
    const bool then_pre = (a.mode & R_THEN_PRE_FWD) != 0;
    if (active) {
      const float al = a.bt.alpha ? a.bt.alpha[p] : float(a.alpha);
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        const int64_t i = base + out_index<N>(g, q);
        const float2 vv = load_v(a.V, i, vreal);
        const float2 xv = xzero ? make_float2(0.f, 0.f) : a.x_in[i];
        const float ur = float(v[q].x) - xv.x, ui = float(v[q].y) - xv.y;
        const float br = 1.f - vv.x, bi = -vv.y;
        const float dr = br * ur - bi * ui, di = br * ui + bi * ur;
        acc += dr * dr + di * di;
        const float2 xn = make_float2(xv.x + al * dr, xv.y + al * di);
        if (!(a.flags & F_REF)) a.x_out[i] = xn;
        if (then_pre) {
          // next iteration's B x + y, from the updated iterate
          const float2 yv = a.y[i];
          v[q] = mkc<V>(T(yv.x + br * xn.x - bi * xn.y), T(yv.y + br * xn.y + bi * xn.x));
        }
      }
    }
    if (then_pre) {
      V t[N1];
      out_to_in<N>(v, t);
#pragma unroll
      for (int q = 0; q < N1; ++q) v[q] = t[q];
      fft_rows<N, false>(v, exr, tw, g);
      if (active) {
#pragma unroll
        for (int q = 0; q < N1; ++q)
          reinterpret_cast<V*>(a.buf)[base + out_index<N>(g, q)] = v[q];
      }
    }
    const int64_t bpp = a.bt.count > 1 ? a.bt.rows_per / F : (int64_t)gridDim.x;
    reduce_and_finalize<THREADS>((double)acc, a.partials, blockIdx.x, p * bpp, bpp, st,
                                 a.hist + (int64_t)p * a.bt.hist_stride, a.flags);
    return;
  }
  if (a.mode & R_OUT_RESID) {
    // u = L x ; A x = u + V x ; r = y - A x  (fp64)
    double acc_r = 0.0, acc_y = 0.0;
    if (active) {
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        const int64_t i = base + out_index<N>(g, q);
        const float2 vv = load_v(a.V, i, vreal);
        const float2 xv = a.x_in[i];
        const double ax = double(v[q].x) + (double(vv.x) * xv.x - double(vv.y) * xv.y);
        const double ay = double(v[q].y) + (double(vv.x) * xv.y + double(vv.y) * xv.x);
        double rx = ax, ry = ay;
        if (!(a.flags & F_APPLY_A)) {
          const float2 yv = a.y[i];
          rx = double(yv.x) - ax;
          ry = double(yv.y) - ay;
          acc_y += double(yv.x) * yv.x + double(yv.y) * yv.y;
        }
        acc_r += rx * rx + ry * ry;
        if (a.r_out) a.r_out[i] = make_float2(float(rx), float(ry));
      }
    }
    __shared__ double red[THREADS / 32];
    const double sr = block_sum<THREADS>(acc_r, red);
    const double sy = block_sum<THREADS>(acc_y, red);
    if (threadIdx.x == 0) {
      a.partials[2 * blockIdx.x] = sr;
      a.partials[2 * blockIdx.x + 1] = sy;
    }
  }
}

// ------------------------------------------------------------ columns ---

template <int N, bool INV, typename V>
__device__ __forceinline__ void fft_cols(V* v, V* ex, const V* tw, int g, int lane) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  stage1<N, INV>(v, g, tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) ex[(k1 * N2 + g) * 32 + lane] = v[k1];
  __syncthreads();
  V w[N1];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k1 = g + G * s;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) w[s * N2 + n2] = ex[(k1 * N2 + n2) * 32 + lane];
  }
  __syncthreads();
  stage2<N, INV>(w);
#pragma unroll
  for (int q = 0; q < N1; ++q) v[q] = w[q];
}

template <typename T, int N>
__global__ void __launch_bounds__(32 * Split<N>::G) k_cols(const ColsArgs<T> a) {
  typedef typename cplx_of<T>::type V;
  constexpr int N1 = Split<N>::N1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* ex = tw + N;

  const int64_t ib = blockIdx.x % a.inner_blocks, o = blockIdx.x / a.inner_blocks;
  const int p = a.bt.count > 1 ? int(o / a.bt.outer_per) : 0;
  if (!(a.flags & F_NOSTATE) && a.st[p].done) return;

  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t col = ib * 32 + lane;
  const bool active = col < a.inner;
  const int64_t base = o * (int64_t)N * a.inner + col;
  V* buf = reinterpret_cast<V*>(a.buf);
  for (int m = threadIdx.x; m < N; m += blockDim.x) tw[m] = tw_entry<T>(stage1_twiddle_exponent(m, Split<N>::N2) * (256 / N));
  __syncthreads();

  V v[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q)
    v[q] = active ? buf[base + (int64_t)in_index<N>(g, q) * a.inner] : mkc<V>(T(0), T(0));

  if (a.mode == COL_INV) {
    fft_cols<N, true>(v, ex, tw, g, lane);
  } else {
    fft_cols<N, false>(v, ex, tw, g, lane);
    if (a.mode == COL_FWD_MUL_INV) {
      // This pass runs on axis 0 after all faster axes were transformed, so
      // the column index decomposes into their frequency indices.
      const Sym<T> sy = problem_sym(a.sym, a.bt, p);
      T p2in = T(0);
      if (a.flags & F_CBLOCK) {
        // column-block layout of the fused schedule: col = (cb * 256 + ky) * 32 + xl
        p2in = axis_p2(sy, 2, int((col >> 13) * 32 + (col & 31))) +
               axis_p2(sy, 1, int((col >> 5) & 255));
      } else if (sy.ndim == 3) {
        p2in = axis_p2(sy, 2, int(col % sy.n[2])) + axis_p2(sy, 1, int(col / sy.n[2]));
      } else if (sy.ndim == 2) {
        p2in = axis_p2(sy, 1, int(col));
      }
      V t[N1];
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        const int k = out_index<N>(g, q);
        v[q] = cmul(v[q], spectral_factor<T, V>(p2in + axis_p2(sy, 0, k), sy, a.mul));
      }
      out_to_in<N>(v, t);
#pragma unroll
      for (int q = 0; q < N1; ++q) v[q] = t[q];
      fft_cols<N, true>(v, ex, tw, g, lane);
    }
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < N1; ++q) buf[base + (int64_t)out_index<N>(g, q) * a.inner] = v[q];
  }
}

// ------------------------------------------------------------ launchers ---

template <typename T, int N>
static size_t rows_smem() {
  typedef typename cplx_of<T>::type V;
  return sizeof(V) * (N + (RowsCfg<T>::THREADS / Split<N>::G) * N);
}
template <typename T, int N>
static size_t cols_smem() {
  typedef typename cplx_of<T>::type V;
  return sizeof(V) * (N + 32 * N);
}

template <typename T, int N>
static cudaError_t rows_attr() {
  return cudaFuncSetAttribute(k_rows<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rows_smem<T, N>());
}
template <typename T, int N>
static cudaError_t cols_attr() {
  return cudaFuncSetAttribute(k_cols<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cols_smem<T, N>());
}

template <typename T, int N>
static cudaError_t rows_go(const RowsArgs<T>& a, int64_t grid, cudaStream_t s) {
  k_rows<T, N><<<(unsigned)grid, RowsCfg<T>::THREADS, rows_smem<T, N>(), s>>>(a);
  return cudaGetLastError();
}
template <typename T, int N>
static cudaError_t cols_go(const ColsArgs<T>& a, cudaStream_t s) {
  const int64_t grid = a.inner_blocks * a.outer;
  k_cols<T, N><<<(unsigned)grid, 32 * Split<N>::G, cols_smem<T, N>(), s>>>(a);
  return cudaGetLastError();
}

#define USP_SWITCH_N(n, CALL)                     \
  switch (n) {                                    \
    case 2: return CALL(2);                       \
    case 4: return CALL(4);                       \
    case 8: return CALL(8);                       \
    case 16: return CALL(16);                     \
    case 32: return CALL(32);                     \
    case 64: return CALL(64);                     \
    case 128: return CALL(128);                   \
    case 256: return CALL(256);                   \
    default: return cudaErrorInvalidValue;        \
  }

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

int rows_per_block_f32(int n) { return RowsCfg<float>::THREADS / (n / (1 << ((ilog2c(n) + 1) / 2))); }
int rows_per_block_f64(int n) { return RowsCfg<double>::THREADS / (n / (1 << ((ilog2c(n) + 1) / 2))); }

template <typename T, int N>
static cudaError_t attrs_one() {
  cudaError_t e = rows_attr<T, N>();
  if (e != cudaSuccess) return e;
  return cols_attr<T, N>();
}
template <typename T>
static cudaError_t attrs_all() {
  cudaError_t e;
  if ((e = attrs_one<T, 2>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 4>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 8>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 16>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 32>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 64>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 128>()) != cudaSuccess) return e;
  return attrs_one<T, 256>();
}

// Twiddles from the first octant by symmetry, so W^(64 j) are exactly
// 1, -i, -1, i and the table is exactly symmetric.
const float2* twiddle_table_f32() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tw32) != cudaSuccess) return nullptr;
  return static_cast<const float2*>(p);
}

cudaError_t init_twiddles() {
  float2 h32[256];
  double2 h64[256];
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < 256; ++m) {
    const int q = m / 64, r = m % 64;
    double c, s;  // cos, sin of 2 pi r/256, r in [0, 64)
    if (r <= 32) {
      c = cos(two_pi * r / 256.0);
      s = sin(two_pi * r / 256.0);
    } else {
      c = sin(two_pi * (64 - r) / 256.0);
      s = cos(two_pi * (64 - r) / 256.0);
    }
    if (r == 0) { c = 1.0; s = 0.0; }
    // rotate by q quarter turns: angle 2 pi m/256 = q pi/2 + 2 pi r/256
    for (int k = 0; k < q; ++k) {
      const double t = c;
      c = -s;
      s = t;
    }
    h64[m] = make_double2(c, -s);  // exp(-i angle)
    h32[m] = make_float2((float)c, (float)-s);
  }
  cudaError_t e = cudaMemcpyToSymbol(g_tw32, h32, sizeof(h32));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_tw64, h64, sizeof(h64));
  if (e != cudaSuccess) return e;
  if ((e = attrs_all<float>()) != cudaSuccess) return e;
  return attrs_all<double>();
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
