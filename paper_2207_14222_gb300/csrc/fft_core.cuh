// fft_core.cuh -- building blocks of the FFT that applies (L+I)^-1 =
// F^-1 diag(1/(Lhat+1)) F (paper Eq. laplacian_inverse).
//
// A length-N transform (N = 2^k, 2 <= N <= 256) is split as N = N1 * N2 with
// N2 <= N1 <= 16 (N1 = 2^ceil(k/2)):
//   n = N2*n1 + n2,  k = k1 + N1*k2,
//   X[k1 + N1 k2] = sum_n2 W_N^(n2 k1) W_N2^(n2 k2) sum_n1 x[N2 n1 + n2] W_N1^(n1 k1)
// G = N2 cooperating threads each hold N1 values.  Stage 1: thread g holds
// x[N2 q + g] (q = 0..N1-1), does an in-register DFT_N1 and multiplies by the
// twiddle W_N^(g k1).  One exchange through shared memory.  Stage 2: thread g
// does S = N1/N2 in-register DFT_N2's for k1 = g + G s and ends up holding
// X[g + G s + N1 k2] in register s*N2 + k2.  That set of indices is the set
// {g + G m}, the same set the thread held on input, so a forward transform,
// a pointwise spectral multiply and an inverse transform chain in registers
// with one compile-time register permutation (m = s + S k2).
//
// Forward transforms are unnormalised with W_N = exp(-2 pi i / N); inverse
// transforms use the conjugate twiddles and no 1/N (the caller folds 1/N
// into the spectral multiplier).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace usp {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };

template <typename V>
__device__ __forceinline__ V mkc(decltype(V().x) re, decltype(V().x) im) {
  V r; r.x = re; r.y = im; return r;
}
template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return mkc<V>(a.x + b.x, a.y + b.y); }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return mkc<V>(a.x - b.x, a.y - b.y); }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return mkc<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {
  return mkc<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// a * (-i) for the forward direction, a * (+i) for the inverse.
template <bool INV, typename V>
__device__ __forceinline__ V rot_quarter(V a) {
  return INV ? mkc<V>(-a.y, a.x) : mkc<V>(a.y, -a.x);
}

// cos(pi/8), sin(pi/8), sqrt(1/2): the non-trivial values of exp(2 pi i e/16).
#define USP_COS_PI_8 0.92387953251128675613
#define USP_SIN_PI_8 0.38268343236508977173
#define USP_SQRT_HALF 0.70710678118654752440

// a * W_16^e (forward: W_16 = exp(-2 pi i/16); inverse: its conjugate).
// e is a compile-time constant after unrolling, so the switch folds away.
template <bool INV, typename V>
__device__ __forceinline__ V tw16(V a, int e) {
  typedef decltype(a.x) T;
  e &= 15;
  const int q = e >> 2, r = e & 3;
  V b = a;
  if (r == 2) {
    // exp(-+ i pi/4) = sqrt(1/2) (1 -+ i)
    const T h = T(USP_SQRT_HALF);
    b = INV ? mkc<V>(h * (a.x - a.y), h * (a.x + a.y))
            : mkc<V>(h * (a.x + a.y), h * (a.y - a.x));
  } else if (r == 1 || r == 3) {
    const T c = T(r == 1 ? USP_COS_PI_8 : USP_SIN_PI_8);
    const T s = T(r == 1 ? USP_SIN_PI_8 : USP_COS_PI_8);
    // forward W = c - i s ; inverse W = c + i s
    b = INV ? mkc<V>(a.x * c - a.y * s, a.x * s + a.y * c)
            : mkc<V>(a.x * c + a.y * s, a.y * c - a.x * s);
  }
  if (q & 2) b = mkc<V>(-b.x, -b.y);
  if (q & 1) b = rot_quarter<INV>(b);
  return b;
}

// In-register DFT of size R in {1,2,4,8,16}, natural order in and out
// (radix-2 decimation in time, fully unrolled).
template <int R, bool INV, typename V>
struct DFT {
  static __device__ __forceinline__ void run(V* v) {
    constexpr int H = R / 2;
    V e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    DFT<H, INV, V>::run(e);
    DFT<H, INV, V>::run(o);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      V t = tw16<INV>(o[k], k * (16 / R));
      v[k] = cadd(e[k], t);
      v[k + H] = csub(e[k], t);
    }
  }
};
template <bool INV, typename V>
struct DFT<1, INV, V> {
  static __device__ __forceinline__ void run(V*) {}
};
template <bool INV, typename V>
struct DFT<2, INV, V> {
  static __device__ __forceinline__ void run(V* v) {
    V t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  }
};

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

template <int N>
struct Split {
  static constexpr int LOG = ilog2c(N);
  static constexpr int N1 = 1 << ((LOG + 1) / 2);
  static constexpr int N2 = N / N1;
  static constexpr int G = N2;        // threads per transform
  static constexpr int S = N1 / N2;   // stage-2 sub-transforms per thread (1 or 2)
  static_assert(N1 * N2 == N && N2 <= N1 && N1 <= 16, "unsupported FFT size");
};

// Stage-1 twiddle table layout: tw[k1 * N2 + g] = W_N^(g k1) (k1 < N1,
// g < N2), so that the threads g of one transform read consecutive entries
// (no shared-memory bank conflicts) and a warp sharing g reads one entry.
__host__ __device__ __forceinline__ int stage1_twiddle_exponent(int m, int N2) {
  return (m % N2) * (m / N2);
}

// Stage 1: in-register DFT_N1, then v[k1] *= W_N^(g k1) (conjugate if INV).
template <int N, bool INV, typename V>
__device__ __forceinline__ void stage1(V* v, int g, const V* tw) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  DFT<N1, INV, V>::run(v);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) {
    const V w = tw[k1 * N2 + g];
    v[k1] = INV ? cmulc(v[k1], w) : cmul(v[k1], w);
  }
}

// Stage 2 on values already gathered: w[s*N2 + n2] = A[k1 = g + G s][n2];
// out in place: w[s*N2 + k2] = X[g + G s + N1 k2].
template <int N, bool INV, typename V>
__device__ __forceinline__ void stage2(V* w) {
  constexpr int N2 = Split<N>::N2, S = Split<N>::S;
#pragma unroll
  for (int s = 0; s < S; ++s) DFT<N2, INV, V>::run(w + s * N2);
}

// Index held in output register q (= s*N2 + k2) by thread g.
template <int N>
__device__ __forceinline__ int out_index(int g, int q) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G;
  return g + G * (q / N2) + N1 * (q % N2);
}
// Index held in input register q by thread g (stage-1 distribution).
template <int N>
__device__ __forceinline__ int in_index(int g, int q) {
  return Split<N>::N2 * q + g;
}
// Reorder output registers into the stage-1 input distribution, so that a
// second transform can start from them: in[s + S k2] = out[s N2 + k2].
template <int N, typename V>
__device__ __forceinline__ void out_to_in(const V* o, V* i) {
  constexpr int N2 = Split<N>::N2, S = Split<N>::S;
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) i[s + S * k2] = o[s * N2 + k2];
}

// ---- lines of length N = R * M (R in {1, 2, 3}, M = 2^k <= 256) -----------
//
// A length-N transform with N = R M splits by decimation in time into R
// interleaved sub-sequences x[R m + r] (m < M), each transformed by the
// M-point code above:  X[k + M j] = sum_r W_3^(r j) (W_N^(r k) Y_r[k]),
// Y_r = DFT_M(x[R . + r]) (W_R for R = 2: +-1).  A line uses G = R * G_M
// threads; thread l = r G_M + g runs sub-sequence r with the M-point layout of
// thread g and, after one exchange through shared memory, holds the outputs
// X[k + M r] for the frequencies k of thread g.  The inverse runs the same
// steps backwards.  Positions of register q of line thread l (r = l / G_M,
// g = l % G_M):
//   spatial input  (stage-1 order)   R in_index<M>(g, q)  + r
//   spatial output (after inverse)   R out_index<M>(g, q) + r
//   spectral output (after forward)  out_index<M>(g, q) + M r
//   spectral input (for an inverse)  in_index<M>(g, q)  + M r
// For R = 1 these are the plain M-point positions.
template <int N>
struct Line {
  static constexpr int R = (N % 3 == 0) ? 3 : (N > 256 ? 2 : 1);
  static constexpr int M = N / R;
  static constexpr int GM = Split<M>::G;
  static constexpr int G = R * GM;        // threads per line
  static constexpr int NV = Split<M>::N1;  // values per thread
  static_assert(R * M == N && (M & (M - 1)) == 0 && M <= 256, "unsupported line length");
  static __device__ __forceinline__ int sp_in(int l, int q) { return R * in_index<M>(l % GM, q) + l / GM; }
  static __device__ __forceinline__ int sp_out(int l, int q) { return R * out_index<M>(l % GM, q) + l / GM; }
  static __device__ __forceinline__ int fr_out(int l, int q) { return out_index<M>(l % GM, q) + M * (l / GM); }
  static __device__ __forceinline__ int fr_in(int l, int q) { return in_index<M>(l % GM, q) + M * (l / GM); }
};

// sqrt(3)/2: the imaginary part of exp(2 pi i / 3).
#define USP_SQRT3_HALF 0.86602540378443864676

// Output j of the radix-R butterfly over a[0..R) (forward: W_3 = exp(-2 pi i/3)).
template <int R, bool INV, typename V>
__device__ __forceinline__ V radix_out(const V* a, int j) {
  typedef decltype(a[0].x) T;
  if (R == 2) return j == 0 ? cadd(a[0], a[1]) : csub(a[0], a[1]);
  const V s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
  if (j == 0) return cadd(a[0], s);
  const V t = mkc<V>(a[0].x - T(0.5) * s.x, a[0].y - T(0.5) * s.y);
  const V u = mkc<V>(T(USP_SQRT3_HALF) * d.x, T(USP_SQRT3_HALF) * d.y);
  // forward: X1 = t - i u, X2 = t + i u; the inverse swaps the signs
  const bool minus_i = (j == 1) != INV;
  return minus_i ? mkc<V>(t.x + u.y, t.y - u.x) : mkc<V>(t.x - u.y, t.y + u.x);
}

// The radix-R stage after the M-point forward transforms.  v: this
// thread's outputs Y_r[k], k = out_index<M>(g, q); ex: the line's exchange
// area, element e at ex[e * STRIDE + lane]; rtw[m] = W_N^m.  On return
// v[q] = X[out_index<M>(g, q) + M r].  Begins and ends with a barrier-free
// hand-off: the caller's transform already synchronised after its own use of
// ex, and this function synchronises after its reads.
template <int N, int STRIDE, typename V>
__device__ __forceinline__ void radix_fwd(V* v, V* ex, const V* rtw, int l, int lane) {
  typedef Line<N> L;
  if (L::R == 1) return;
  constexpr int M = L::M, NV = L::NV;
  const int r = l / L::GM, g = l % L::GM;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int k = out_index<M>(g, q);
    const V w = v[q];
    ex[(r * M + k) * STRIDE + lane] = r == 0 ? w : cmul(w, rtw[r * k]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int k = out_index<M>(g, q);
    V a[L::R];
#pragma unroll
    for (int i = 0; i < L::R; ++i) a[i] = ex[(i * M + k) * STRIDE + lane];
    v[q] = radix_out<L::R, false>(a, r);
  }
  __syncthreads();
}

// The radix-R stage before the M-point inverse transforms: v[q] =
// X[in_index<M>(g, q) + M r] in; Z_r[k] = W_N^(-r k) sum_j W_R^(-r j)
// X[k + M j] out (k = in_index<M>(g, q)), ready for the M-point inverse.
template <int N, int STRIDE, typename V>
__device__ __forceinline__ void radix_inv(V* v, V* ex, const V* rtw, int l, int lane) {
  typedef Line<N> L;
  if (L::R == 1) return;
  constexpr int M = L::M, NV = L::NV;
  const int r = l / L::GM, g = l % L::GM;
#pragma unroll
  for (int q = 0; q < NV; ++q) ex[(r * M + in_index<M>(g, q)) * STRIDE + lane] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int k = in_index<M>(g, q);
    V a[L::R];
#pragma unroll
    for (int i = 0; i < L::R; ++i) a[i] = ex[(i * M + k) * STRIDE + lane];
    const V z = radix_out<L::R, true>(a, r);
    v[q] = r == 0 ? z : cmulc(z, rtw[r * k]);
  }
  __syncthreads();
}

// Frequency index k in [0,n) to signed FFT-order m in [-n/2, n/2).
__device__ __forceinline__ int signed_freq(int k, int n) { return k < (n >> 1) ? k : k - n; }

}  // namespace usp
