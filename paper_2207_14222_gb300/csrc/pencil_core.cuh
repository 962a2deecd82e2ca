// pencil_core.cuh -- the pencil passes as templates over the arithmetic type
// T: float (the FP32 iteration), double and double-float (the refinement
// residual y - A x, Sec. 2.1's A = L + V applied with the multiplier
// Lhat(p)/N).  Each translation unit that instantiates them defines the
// twiddle tables of its types (tw_entry<T>, twx_entry<T>).
//
// Memory layout: C order, last axis fastest.  Rows kernels: G = N2 adjacent
// lanes own one row, each thread holds N1 values (see fft_core.cuh), so for
// a fixed register the G threads touch G consecutive elements.  Column
// kernels: one warp per stage-1 thread index g, the 32 lanes own 32
// consecutive columns, so every global access of a warp is 32 consecutive
// complex values.
#pragma once

#include <math.h>

#include <type_traits>

#include "dfloat.cuh"
#include "fft_core.cuh"
#include "iteration_state.cuh"
#include "kernels.h"

namespace usp {

// W_256^m = exp(-2 pi i m/256), m in [0,256); W_n^m = W_256^(m 256/n).
template <typename T>
__device__ __forceinline__ typename cplx_of<T>::type tw_entry(int m);

// W_1536^m, m in [0,1536): the radix stage of lines of length 96, 192, 384
// (W_N^m = W_1536^(m 1536/N)) and 512.
constexpr int TWX_LEN = 1536;
template <typename T>
__device__ __forceinline__ typename cplx_of<T>::type twx_entry(int m);

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
// double-float (the refinement residual): the FP64 block shape (same row
// blocks), at four blocks per SM -- the 256-point pass fits 128 registers
// without spilling, and twice the warps hide its global loads
template <> struct RowsCfg<dfl> {
  static constexpr int THREADS = 128;
  static constexpr int MINB = 4;
};
// Block shape of the line pass for lines of length N: radix-3 lines use
// 3/4 of the threads so that whole lines fill a block.
template <typename T, int N>
struct RowsShape {
  static constexpr int THREADS = Line<N>::R == 3 ? RowsCfg<T>::THREADS * 3 / 4 : RowsCfg<T>::THREADS;
  static constexpr int F = THREADS / Line<N>::G;  // lines per block
  // the radix stage of the longest lines needs more than 64 registers
  static constexpr int MINB = N >= 384 && RowsCfg<T>::MINB > 2 ? 2 : RowsCfg<T>::MINB;
  static_assert(F * Line<N>::G == THREADS, "lines must fill the block");
};
// Columns per block of the strided-axis pass (lanes per line thread):
// 512-point lines 8 (113 against 119 us with 16, one pass over a batch of 68
// problems of 512^2), 96- and 192-point lines 16 (24.6 against 28.6 us with
// 32 on 70 problems of 192^2), 384-point lines 16 (8: 72 against 70 us).
template <int N>
struct ColsShape {
  static constexpr int COLS = N == 512 ? 8 : (N % 3 == 0 ? 16 : 32);
  static constexpr int THREADS = COLS * Line<N>::G;
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

// The same factors from a tabulated symbol value l = Lhat(p).
template <typename T, typename V>
__device__ __forceinline__ V table_factor(float2 l, const Sym<T>& s, int mul) {
  const T lr = T(l.x), li = T(l.y);
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

// Line transforms (rows): forward from the stage-1 spatial order to the
// spectral output order, inverse from the spectral input order to the
// spatial output order (Line<N>).  exr: the line's N-element exchange area.
template <int N, typename V>
__device__ __forceinline__ void line_fwd_rows(V* v, V* exr, const V* tw, const V* rtw, int l) {
  typedef Line<N> L;
  fft_rows<L::M, false>(v, exr + (l / L::GM) * L::M, tw, l % L::GM);
  radix_fwd<N, 1>(v, exr, rtw, l, 0);
}
template <int N, typename V>
__device__ __forceinline__ void line_inv_rows(V* v, V* exr, const V* tw, const V* rtw, int l) {
  typedef Line<N> L;
  radix_inv<N, 1>(v, exr, rtw, l, 0);
  fft_rows<L::M, true>(v, exr + (l / L::GM) * L::M, tw, l % L::GM);
}

__device__ __forceinline__ float2 load_v(const void* V, int64_t i, bool vreal) {
  if (vreal) return make_float2(__ldg(reinterpret_cast<const float*>(V) + i), 0.f);
  return __ldg(reinterpret_cast<const float2*>(V) + i);
}

template <typename T, int N>
__global__ void __launch_bounds__(RowsShape<T, N>::THREADS, RowsShape<T, N>::MINB) k_rows(const RowsArgs<T> a) {
  typedef typename cplx_of<T>::type V;
  typedef Line<N> L;
  constexpr int N1 = L::NV, G = L::G, M = L::M;
  constexpr int THREADS = RowsShape<T, N>::THREADS;
  constexpr int F = RowsShape<T, N>::F;  // rows per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);   // M-point stage-1 twiddles
  V* rtw = tw + M;                          // W_N^m (radix stage), R > 1
  V* ex = rtw + (L::R > 1 ? N : 0);

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
  for (int m = tid; m < M; m += THREADS) tw[m] = tw_entry<T>(stage1_twiddle_exponent(m, Split<M>::N2) * (256 / M));
  if (L::R > 1)
    for (int m = tid; m < N; m += THREADS) rtw[m] = twx_entry<T>(m * (TWX_LEN / N));
  __syncthreads();
  V* exr = ex + f * N;
  // spectral input (an inverse transform without a forward one) or spatial
  const bool in_spec = (a.mode & R_IN_BUF) && !(a.mode & R_FWD);

  V v[N1];
  // ---- input stage (register q holds position L::sp_in / L::fr_in)
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    const int64_t i = base + (in_spec ? L::fr_in(g, q) : L::sp_in(g, q));
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
  if (a.mode & R_FWD) line_fwd_rows<N>(v, exr, tw, rtw, g);
  if (a.mode & R_MUL) {
    const Sym<T> sy = problem_sym(a.sym, a.bt, p);
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const int k = L::fr_out(g, q);
      v[q] = cmul(v[q], sy.table ? table_factor<T, V>(sy.table[k], sy, a.mul)
                                 : spectral_factor<T, V>(axis_p2(sy, 0, k), sy, a.mul));
    }
  }
  if (a.mode & R_INV) {
    if (a.mode & R_FWD) {
      V t[N1];
      out_to_in<M>(v, t);
#pragma unroll
      for (int q = 0; q < N1; ++q) v[q] = t[q];
    }
    line_inv_rows<N>(v, exr, tw, rtw, g);
  }
  // ---- output stage (register q holds position L::sp_out after an
  // inverse, L::fr_out after a forward transform alone)
  if (a.mode & R_OUT_BUF) {
    if (active) {
      const bool spec = !(a.mode & R_INV);
#pragma unroll
      for (int q = 0; q < N1; ++q)
        reinterpret_cast<V*>(a.buf)[base + (spec ? L::fr_out(g, q) : L::sp_out(g, q))] = v[q];
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
        const int64_t i = base + L::sp_out(g, q);
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
      out_to_in<M>(v, t);
#pragma unroll
      for (int q = 0; q < N1; ++q) v[q] = t[q];
      line_fwd_rows<N>(v, exr, tw, rtw, g);
      if (active) {
#pragma unroll
        for (int q = 0; q < N1; ++q)
          reinterpret_cast<V*>(a.buf)[base + L::fr_out(g, q)] = v[q];
      }
    }
    const int64_t bpp = a.bt.count > 1 ? a.bt.rows_per / F : (int64_t)gridDim.x;
    reduce_and_finalize<THREADS>((double)acc, a.partials, blockIdx.x, p * bpp, bpp, st,
                                 a.hist + (int64_t)p * a.bt.hist_stride, a.flags);
    return;
  }
  if (a.mode & R_OUT_RESID) {
    // u = L x ; A x = u + V x ; r = y - A x  (in T: FP64 or double-float)
    double acc_r = 0.0, acc_y = 0.0;
    if constexpr (std::is_same<T, dfl>::value) {
      // products of two floats are exact in two words; the squared norms
      // are summed per thread in double-float, per block in FP64
      dfl sr(0.f), sy(0.f);
      if (active) {
#pragma unroll
        for (int q = 0; q < N1; ++q) {
          const int64_t i = base + L::sp_out(g, q);
          const float2 vv = load_v(a.V, i, vreal);
          const float2 xv = a.x_in[i];
          const dfl ax = v[q].x + (two_prod(vv.x, xv.x) - two_prod(vv.y, xv.y));
          const dfl ay = v[q].y + (two_prod(vv.x, xv.y) + two_prod(vv.y, xv.x));
          dfl rx = ax, ry = ay;
          if (!(a.flags & F_APPLY_A)) {
            const float2 yv = a.y[i];
            rx = dfl(yv.x) - ax;
            ry = dfl(yv.y) - ay;
            sy = sy + (two_prod(yv.x, yv.x) + two_prod(yv.y, yv.y));
          }
          sr = sr + (rx * rx + ry * ry);
          if (a.r_out) a.r_out[i] = make_float2(float(rx), float(ry));
        }
      }
      acc_r = double(sr);
      acc_y = double(sy);
    } else if (active) {
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        const int64_t i = base + L::sp_out(g, q);
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

// Exchange rows XOR-swizzled as in the TMA column passes (bank halves).
template <int N, bool INV, int COLS, typename V>
__device__ __forceinline__ void fft_cols(V* v, V* ex, const V* tw, int g, int lane) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  stage1<N, INV>(v, g, tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) ex[(k1 * N2 + (g ^ (k1 & (N2 - 1)))) * COLS + lane] = v[k1];
  __syncthreads();
  V w[N1];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k1 = g + G * s;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) w[s * N2 + n2] = ex[(k1 * N2 + (n2 ^ (k1 & (N2 - 1)))) * COLS + lane];
  }
  __syncthreads();
  stage2<N, INV>(w);
#pragma unroll
  for (int q = 0; q < N1; ++q) v[q] = w[q];
}

// Line transforms along a strided axis (COLS columns per block, lane =
// column); orders as line_fwd_rows / line_inv_rows.
template <int N, int COLS, typename V>
__device__ __forceinline__ void line_fwd_cols(V* v, V* ex, const V* tw, const V* rtw, int l, int lane) {
  typedef Line<N> L;
  fft_cols<L::M, false, COLS>(v, ex + (l / L::GM) * L::M * COLS, tw, l % L::GM, lane);
  radix_fwd<N, COLS>(v, ex, rtw, l, lane);
}
template <int N, int COLS, typename V>
__device__ __forceinline__ void line_inv_cols(V* v, V* ex, const V* tw, const V* rtw, int l, int lane) {
  typedef Line<N> L;
  radix_inv<N, COLS>(v, ex, rtw, l, lane);
  fft_cols<L::M, true, COLS>(v, ex + (l / L::GM) * L::M * COLS, tw, l % L::GM, lane);
}

template <typename T, int N>
__global__ void __launch_bounds__(ColsShape<N>::THREADS) k_cols(const ColsArgs<T> a) {
  typedef typename cplx_of<T>::type V;
  typedef Line<N> L;
  constexpr int N1 = L::NV, M = L::M, COLS = ColsShape<N>::COLS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);   // M-point stage-1 twiddles
  V* rtw = tw + M;                          // W_N^m (radix stage), R > 1
  V* ex = rtw + (L::R > 1 ? N : 0);

  // F_REVERSE: the blocks take the tiles from the last one down (the blocks
  // are dispatched in index order), so the end of the field, which the pass
  // before wrote last, is read first
  const int64_t bt = (a.flags & F_REVERSE) ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
  const int64_t ib = bt % a.inner_blocks, o = bt / a.inner_blocks;
  const int p = a.bt.count > 1 ? int(o / a.bt.outer_per) : 0;
  if (!(a.flags & F_NOSTATE) && a.st[p].done) return;

  const int lane = threadIdx.x % COLS, g = threadIdx.x / COLS;
  const int64_t col = ib * COLS + lane;
  const bool active = col < a.inner;
  const int64_t base = o * (int64_t)N * a.inner + col;
  V* buf = reinterpret_cast<V*>(a.buf);
  for (int m = threadIdx.x; m < M; m += blockDim.x)
    tw[m] = tw_entry<T>(stage1_twiddle_exponent(m, Split<M>::N2) * (256 / M));
  if (L::R > 1)
    for (int m = threadIdx.x; m < N; m += blockDim.x) rtw[m] = twx_entry<T>(m * (TWX_LEN / N));
  __syncthreads();

  // COL_INV reads a spectrum along this axis, the other modes spatial values
  const bool in_spec = a.mode == COL_INV;
  V v[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q)
    v[q] = active ? buf[base + (int64_t)(in_spec ? L::fr_in(g, q) : L::sp_in(g, q)) * a.inner]
                  : mkc<V>(T(0), T(0));

  bool out_spec = false;
  if (a.mode == COL_INV) {
    line_inv_cols<N, COLS>(v, ex, tw, rtw, g, lane);
  } else {
    line_fwd_cols<N, COLS>(v, ex, tw, rtw, g, lane);
    out_spec = true;
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
        const int k = L::fr_out(g, q);
        v[q] = cmul(v[q], sy.table
                              ? table_factor<T, V>(sy.table[kspace_index(sy, k, col, (a.flags & F_CBLOCK) != 0)],
                                                   sy, a.mul)
                              : spectral_factor<T, V>(p2in + axis_p2(sy, 0, k), sy, a.mul));
      }
      out_to_in<M>(v, t);
#pragma unroll
      for (int q = 0; q < N1; ++q) v[q] = t[q];
      line_inv_cols<N, COLS>(v, ex, tw, rtw, g, lane);
      out_spec = false;
    }
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < N1; ++q)
      buf[base + (int64_t)(out_spec ? L::fr_out(g, q) : L::sp_out(g, q)) * a.inner] = v[q];
  }
}

// ------------------------------------------------------------ launchers ---

template <typename T, int N>
static size_t rows_smem() {
  typedef typename cplx_of<T>::type V;
  return sizeof(V) * (Line<N>::M + (Line<N>::R > 1 ? N : 0) + RowsShape<T, N>::F * N);
}
template <typename T, int N>
static size_t cols_smem() {
  typedef typename cplx_of<T>::type V;
  return sizeof(V) * (Line<N>::M + (Line<N>::R > 1 ? N : 0) + ColsShape<N>::COLS * N);
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
  k_rows<T, N><<<(unsigned)grid, RowsShape<T, N>::THREADS, rows_smem<T, N>(), s>>>(a);
  return cudaGetLastError();
}
template <typename T, int N>
static cudaError_t cols_go(const ColsArgs<T>& a, cudaStream_t s) {
  const int64_t grid = a.inner_blocks * a.outer;
  k_cols<T, N><<<(unsigned)grid, ColsShape<N>::THREADS, cols_smem<T, N>(), s>>>(a);
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
    case 96: return CALL(96);                     \
    case 192: return CALL(192);                   \
    case 384: return CALL(384);                   \
    case 512: return CALL(512);                   \
    default: return cudaErrorInvalidValue;        \
  }

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
  if ((e = attrs_one<T, 256>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 96>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 192>()) != cudaSuccess) return e;
  if ((e = attrs_one<T, 384>()) != cudaSuccess) return e;
  return attrs_one<T, 512>();
}

}  // namespace usp
