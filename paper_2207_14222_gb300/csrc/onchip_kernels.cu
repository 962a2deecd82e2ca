// onchip_kernels.cu -- whole phases of Algorithm 1 for small square 2-D grids
// (n x n, n in {32, 64, 96, 128, 192, 256}) with every field resident in the
// shared memory of one thread-block cluster.
//
// The pencil schedule streams the field through HBM two or three times per
// iteration; at n <= 256 a field is at most 512 KiB, so those passes are
// latency-bound launches of a few dozen blocks.  Here one cluster of C CTAs
// holds the problem: CTA c owns rows [c R, c R + R) of x, V and y and, in
// k-space, columns [c R, c R + R).  One iteration is
//   A  t = (1 - V) x + y on the own rows, FFT along x, each k-space value
//      stored into the shared memory of the CTA that owns its column;
//   B  FFT along y of the own columns, the multiplier 1/(N (Lhat + 1)),
//      inverse FFT along y, each value stored back to the owner of its row;
//   C  inverse FFT along x, Delta = (1 - V)(u - x), x += alpha Delta, and
//      the CTA's sum of |Delta|^2 stored into every CTA of the cluster.
// The stores between CTAs are asynchronous (st.async) and count their bytes
// on an mbarrier of the receiving CTA, so a CTA waits only for the data it
// needs, not for the whole cluster.  No buffer is overwritten early: a CTA
// sends the next round into a buffer only after it has received data that
// its owner sends after reading that buffer, and every CTA arms the next
// phase of its mbarriers right after a wait completes, before it sends the
// data that lets anyone produce for that phase.  Every CTA adds the C sums
// in the same order and runs the same convergence test (Algorithm 1's) on
// its own copy of the device state, so all CTAs leave the loop together;
// rank 0 writes the history and the state.  The next iteration's step A runs
// before the test of the current one is read (its result is dropped if the
// test stops the phase).
//
// The block forms (Sec. 2.2 antisymmetrised, K = 2; Sec. 3.2 flux form,
// K = 3 in 2-D) run the same steps on K component planes: B = I - V is a
// K x K matrix per point and (L+I)^-1 a K x K matrix per frequency.
//
// One launch runs a whole phase (until the state says done), one cluster per
// problem of a batch.  Every wait is bounded; one that gives up records
// ST_TIMEOUT and the CTAs meet at a final cluster barrier before they exit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_core.cuh"
#include "iteration_state.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace usp {
namespace {

// Kinds of unknown: one component (the scalar form), or the block forms of
// Sec. 2.2 (antisymmetrised, K = 2) and Sec. 3.2 (flux form in 2-D, K = 3).
template <int KIND>
struct Comps {
  static constexpr int K = KIND == ONCHIP_SCALAR ? 1 : (KIND == ONCHIP_ANTISYMMETRIC ? 2 : 3);
};

template <int N, int RR, int KIND>
struct OnchipCfg {
  static constexpr int K = Comps<KIND>::K;   // components per point
  static constexpr int R = RR;               // rows (and k-space columns) per CTA
  static constexpr int C = N / R;            // CTAs per cluster
  typedef Line<N> Ln;                        // N = R' M with a radix-R' outer stage (R' = 3 at 96, 192)
  static constexpr int G = Ln::G;            // threads per line
  static constexpr int NV = Ln::NV;          // values per thread
  static constexpr int T = R * G;            // threads per CTA
  static constexpr int P = N + 8;            // line stride (float2): rows of a warp on both bank halves
  static constexpr int FIELD = R * P;        // float2 per resident array
  // K fields each of x, y, row buffer, column buffer; one of V; twiddles of
  // the M-point stage and W_N^m of the outer stage; then C + T/32 doubles
  static constexpr size_t SMEM =
      sizeof(float2) * ((4 * (size_t)K + 1) * FIELD + 2 * N) + sizeof(double) * (C + T / 32);
  static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
  static_assert(Ln::G * Ln::NV == N, "length");
  static_assert(T % 32 == 0, "whole warps");
  static_assert(C >= 2 && C <= 16, "cluster size");
  static_assert(32 % Split<Ln::M>::G == 0, "the threads of an M-point sub-line share a warp");
  // lines of a radix-3 outer stage straddle warps: their hand-offs take
  // block barriers, those of the power-of-two lines warp barriers
  static constexpr bool WARP_LINES = Ln::R == 1 && 32 % G == 0;
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Shared-memory address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// Asynchronous store into the shared memory of a CTA of the cluster; its
// bytes complete on the mbarrier `mbar` (same CTA, shared::cluster address).
__device__ __forceinline__ void st_async(uint32_t addr, float2 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
               "l"(__double_as_longlong(v)), "r"(mbar)
               : "memory");
}
// Bounded wait for a phase of a local mbarrier whose bytes come from other
// CTAs of the cluster (acquire at cluster scope makes their stores visible).
// Polls with test_wait (no suspension between polls: the CTA has nothing
// else to run while it waits for its lines).
__device__ __forceinline__ bool wait_cluster(uint64_t* b, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// All threads of all CTAs of the cluster.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Position of element e of line l in a line buffer (stride P): an XOR of
// bits 1-3 of e that puts the values one warp stores into one line each
// (step A into columns, step B into rows) and the values it loads along its
// lines on distinct banks.
template <int G>
__device__ __forceinline__ int swz(int l, int e) {
  return e ^ (((l >> 1) * (16 / G)) & 7);
}

__device__ __forceinline__ float axis_p2(const Sym<float>& s, int ax, int k) {
  const float p = s.ks[ax] * (float)signed_freq(k, s.n[ax]);
  return p * p;
}
// 1 / (N (Lhat + 1)) from Lhat = lr + i li.
__device__ __forceinline__ float2 linv_factor(float lr, float li, float inv_n) {
  const float dr = lr + 1.f;
  const float sc = __fdividef(inv_n, fmaf(dr, dr, li * li));
  return make_float2(dr * sc, -li * sc);
}

// Line transforms of one line held by its G threads (Line<N>): forward from
// the spatial input order to the spectral output order, inverse from the
// spectral input order to the spatial output order.  ex: the line's N-entry
// exchange area; tw: M-point twiddles; rtw[m] = W_N^m (outer stage).
template <int N>
__device__ __forceinline__ void line_fwd(float2* v, float2* ex, const float2* tw, const float2* rtw, int l);
template <int N>
__device__ __forceinline__ void line_inv(float2* v, float2* ex, const float2* tw, const float2* rtw, int l);

// B = I - V at one point, applied to the K components of `in` (v: the
// point's entry of V: the complex potential; the antisymmetrised form's v,
// B = [[1, conj(v)], [-v, 1]]; the flux form's (Vu, VJ), B = diag(1 - Vu,
// (1 - VJ) I)).
template <int KIND>
__device__ __forceinline__ void apply_B(float2 v, const float2* in, float2* out) {
  if constexpr (KIND == ONCHIP_SCALAR) {
    const float br = 1.f - v.x;
    out[0] = make_float2(fmaf(br, in[0].x, v.y * in[0].y), fmaf(br, in[0].y, -v.y * in[0].x));
  } else if constexpr (KIND == ONCHIP_ANTISYMMETRIC) {
    out[0] = make_float2(in[0].x + v.x * in[1].x + v.y * in[1].y, in[0].y + v.x * in[1].y - v.y * in[1].x);
    out[1] = make_float2(in[1].x - (v.x * in[0].x - v.y * in[0].y), in[1].y - (v.x * in[0].y + v.y * in[0].x));
  } else {
    const float bu = 1.f - v.x, bj = 1.f - v.y;
    out[0] = make_float2(bu * in[0].x, bu * in[0].y);
    out[1] = make_float2(bj * in[1].x, bj * in[1].y);
    out[2] = make_float2(bj * in[2].x, bj * in[2].y);
  }
}

// (Lhat(p) + I)^-1 / N applied to the K spectral components T at one
// frequency (py along axis 0, px along axis 1).  Block forms: b = (a_re,
// a_im, b_re, b_im) of l = a |p|^2 + b, (L+I)^-1 = [[1, conj(l)], [-l, 1]] /
// (1 + |l|^2); flux: b = (alpha, beta, s), the Schur complement of
// [[alpha, i s p^T], [i s p, beta I]].
template <int KIND>
__device__ __forceinline__ void block_multiply(float2* T, float py, float px, const float* b, float inv_n) {
  const float p2 = py * py + px * px;
  if constexpr (KIND == ONCHIP_ANTISYMMETRIC) {
    const float lr = fmaf(b[0], p2, b[2]), li = fmaf(b[1], p2, b[3]);
    const float sc = __fdividef(inv_n, 1.f + lr * lr + li * li);
    const float2 t0 = T[0], t1 = T[1];
    T[0] = make_float2(sc * (t0.x + lr * t1.x + li * t1.y), sc * (t0.y + lr * t1.y - li * t1.x));
    T[1] = make_float2(sc * (t1.x - (lr * t0.x - li * t0.y)), sc * (t1.y - (lr * t0.y + li * t0.x)));
  } else if constexpr (KIND == ONCHIP_FLUX) {
    const float al = b[0], be = b[1], sg = b[2];
    const float S = al + sg * sg * p2 / be;
    const float pk[2] = {py, px};
    const float2 pT = make_float2(py * T[1].x + px * T[2].x, py * T[1].y + px * T[2].y);
    const float iS = inv_n / S;
    const float2 t0 = T[0];
    T[0] = make_float2(iS * (t0.x + sg * pT.y / be), iS * (t0.y - sg * pT.x / be));
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float c1 = inv_n / be, c2 = sg * sg * pk[k] / (be * be * S) * inv_n;
      const float c3 = sg * pk[k] / (be * S) * inv_n;
      const float2 tk = T[1 + k];
      T[1 + k] = make_float2(c1 * tk.x - c2 * pT.x + c3 * t0.y, c1 * tk.y - c2 * pT.y - c3 * t0.x);
    }
  }
}

// A line of N values held by its G threads (one warp holds whole lines, so
// the exchange needs only warp synchronisation).
template <int N>
__device__ __forceinline__ void fft_line(float2* v, float2* ex, const float2* tw, int g, bool inv) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  if (inv) stage1<N, true>(v, g, tw);
  else stage1<N, false>(v, g, tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) ex[k1 * N2 + (g ^ (k1 & (N2 - 1)))] = v[k1];
  __syncwarp();
  float2 w[N1];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k1 = g + G * s;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) w[s * N2 + n2] = ex[k1 * N2 + (n2 ^ (k1 & (N2 - 1)))];
  }
  __syncwarp();
  if (inv) stage2<N, true>(w);
  else stage2<N, false>(w);
#pragma unroll
  for (int q = 0; q < N1; ++q) v[q] = w[q];
}

template <int N>
__device__ __forceinline__ void line_fwd(float2* v, float2* ex, const float2* tw, const float2* rtw, int l) {
  typedef Line<N> Ln;
  fft_line<Ln::M>(v, ex + (l / Ln::GM) * Ln::M, tw, l % Ln::GM, false);
  if constexpr (Ln::R > 1) radix_fwd<N, 1>(v, ex, rtw, l, 0);
}
template <int N>
__device__ __forceinline__ void line_inv(float2* v, float2* ex, const float2* tw, const float2* rtw, int l) {
  typedef Line<N> Ln;
  if constexpr (Ln::R > 1) radix_inv<N, 1>(v, ex, rtw, l, 0);
  fft_line<Ln::M>(v, ex + (l / Ln::GM) * Ln::M, tw, l % Ln::GM, true);
}

template <int N, int RR, int KIND>
__global__ void __launch_bounds__(OnchipCfg<N, RR, KIND>::T, 1) k_onchip(OnchipArgs a) {
  typedef OnchipCfg<N, RR, KIND> Cf;
  typedef typename Cf::Ln Ln;
  constexpr int MM = Ln::M;
  constexpr int K = Cf::K, C = Cf::C, R = Cf::R, G = Cf::G, NV = Cf::NV, T = Cf::T, P = Cf::P;
  constexpr int F = Cf::FIELD;
  constexpr uint32_t LINE_BYTES = (uint32_t)(K * R * N * sizeof(float2));   // one round into rb or cb
  constexpr uint32_t SLOT_BYTES = (uint32_t)(C * sizeof(double));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* xs = reinterpret_cast<float2*>(smem_raw);   // K fields (component k at xs + k F)
  float2* ys = xs + K * F;
  float2* vs = ys + K * F;      // one field: the point's entry of V
  float2* rb = vs + F;          // K fields, rows: k-space along x (exchange of step A, input of step C)
  float2* cb = rb + K * F;      // K fields, k-space columns (input of step B)
  float2* tw = cb + K * F;      // M-point stage-1 twiddles
  float2* rtw = tw + N;         // W_N^m, m < N (outer stage)
  double* slots = reinterpret_cast<double*>(rtw + N);   // |Delta|^2 of each CTA
  double* red = slots + C;
  __shared__ DevState S;
  __shared__ __align__(8) uint64_t mb[3];   // cb, rb, slots full
  __shared__ uint32_t r_rb[C], r_cb[C], r_sl[C], m_rb[C], m_cb[C], m_sl[C];
  __shared__ int fail;

  const int tid = threadIdx.x;
  const uint32_t c = cluster_rank();
  const int p = blockIdx.x / C;
  const int64_t NN = (int64_t)N * N;
  const int64_t base = (int64_t)p * K * NN;
  DevState* gst = a.st + p;
  double* hist = c == 0 ? a.hist + (int64_t)p * a.bt.hist_stride : nullptr;
  const Sym<float> sy = problem_sym(a.sym, a.bt, p);
  const float alpha = a.bt.alpha ? a.bt.alpha[p] : a.alpha;
  const bool vreal = (a.flags & F_VREAL) != 0;
  const bool ref_pass = (a.flags & F_REF) != 0;
  const bool xzero = (a.flags & F_XZERO) != 0;
  const uint32_t lim = a.wait_limit ? a.wait_limit : (1u << 26);   // about a second of polls

  if (tid == 0) {
    S = *gst;
    fail = 0;
    if (!S.done) {
      for (int b = 0; b < 3; ++b) mbar_init(&mb[b], 1);
      fence_mbar_init();
      // first phase of each barrier armed before any CTA can send
      mbar_arrive_expect_tx(&mb[0], LINE_BYTES + a.fault_tx);
      mbar_arrive_expect_tx(&mb[1], LINE_BYTES);
      mbar_arrive_expect_tx(&mb[2], SLOT_BYTES);
    }
  }
  for (int m = tid; m < MM; m += T) tw[m] = a.tw[stage1_twiddle_exponent(m, Split<MM>::N2) * (256 / MM)];
  if (Ln::R > 1)
    for (int m = tid; m < N; m += T) {
      double sn, cs;
      sincospi(-2.0 * m / N, &sn, &cs);   // W_N^m
      rtw[m] = make_float2((float)cs, (float)sn);
    }
  if (tid < C) {
    r_rb[tid] = map_rank(rb, tid);
    r_cb[tid] = map_rank(cb, tid);
    r_sl[tid] = map_rank(slots, tid);
    m_cb[tid] = map_rank(&mb[0], tid);
    m_rb[tid] = map_rank(&mb[1], tid);
    m_sl[tid] = map_rank(&mb[2], tid);
  }
  __syncthreads();
  // Every CTA of the cluster read the same state (nothing writes it before
  // all of them have passed the first cluster barrier): a uniform exit.
  if (S.done) return;
  const int row0 = (int)c * R;
  for (int i = tid; i < R * N; i += T) {
    const int jj = i / N, col = i % N;
    const int64_t gi = (int64_t)(row0 + jj) * N + col;   // within a plane
    const int64_t vi = (int64_t)p * NN + gi;              // V: one entry per point
#pragma unroll
    for (int k = 0; k < K; ++k) {
      xs[k * F + jj * P + col] = xzero ? make_float2(0.f, 0.f) : a.x_in[base + k * NN + gi];
      ys[k * F + jj * P + col] = a.y[base + k * NN + gi];
    }
    vs[jj * P + col] = vreal ? make_float2(reinterpret_cast<const float*>(a.V)[vi], 0.f)
                             : reinterpret_cast<const float2*>(a.V)[vi];
  }
  cluster_barrier();  // every CTA has started and armed its barriers

  const int j = tid / G, g = tid % G;    // step A / C: row j, line thread g
  const int kk = j, g2 = g;              // step B: k-space column kk
  const int kx = row0 + kk;              // its frequency index along x
  const float p2x = axis_p2(sy, 1, kx);
  const float px = sy.ks[1] * (float)signed_freq(kx, N);
  uint32_t ph_cb = 0, ph_rb = 0, ph_sl = 0;
  float2 v[K][NV];
  bool first = true;
  // Bounded by the state's own limit: finalize_iteration stops at it_limit.
  for (int iter = 0;; ++iter) {
    // ---- A: t = B x + y, FFT along x, k-space values to column owners
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int col = Ln::sp_in(g, q);
      float2 xk[K], t[K];
#pragma unroll
      for (int k = 0; k < K; ++k) xk[k] = xs[k * F + j * P + col];
      apply_B<KIND>(vs[j * P + col], xk, t);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float2 yv = ys[k * F + j * P + col];
        v[k][q] = make_float2(t[k].x + yv.x, t[k].y + yv.y);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) line_fwd<N>(v[k], rb + k * F + j * P, tw, rtw, g);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int kq = Ln::fr_out(g, q), d = kq / R, l = kq % R;
      const uint32_t off = (uint32_t)((l * P + swz<G>(l, row0 + j)) * sizeof(float2));
#pragma unroll
      for (int k = 0; k < K; ++k)
        st_async(r_cb[d] + off + (uint32_t)(k * F * sizeof(float2)), v[k][q], m_cb[d]);
    }
    // a phase is re-armed only by a thread that saw it complete (arming an
    // incomplete phase would over-count its arrivals)
    if (!wait_cluster(&mb[0], ph_cb, lim)) fail = 1;
    else if (tid == 0) mbar_arrive_expect_tx(&mb[0], LINE_BYTES);   // next round of columns
    ph_cb ^= 1u;
    if (!first) {
      // the previous iteration's sums (they were sent before its step C ended)
      const bool got = wait_cluster(&mb[2], ph_sl, lim);
      if (!got) fail = 1;
      ph_sl ^= 1u;
      if (tid == 0 && got) {
        mbar_arrive_expect_tx(&mb[2], SLOT_BYTES);
        double tot = 0.0;
        for (int r = 0; r < C; ++r) tot += slots[r];
        finalize_iteration(&S, hist, tot, 0);
        if (!S.done && iter > S.it_limit + 1) {  // the state machine did not stop: never spin
          S.status = ST_MAXIT;
          S.done = 1;
        }
      }
    }
    __syncthreads();
    if (fail && tid == 0) {
      S.status = ST_TIMEOUT;
      S.done = 1;
    }
    __syncthreads();
    if (S.done) break;
    first = false;

    // ---- B: FFT along y, multiply, inverse FFT along y, values to row owners
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int q = 0; q < NV; ++q) v[k][q] = cb[k * F + kk * P + swz<G>(kk, Ln::sp_in(g2, q))];
    if (Cf::WARP_LINES) __syncwarp();  // a column's threads share a warp
    else __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) line_fwd<N>(v[k], cb + k * F + kk * P, tw, rtw, g2);
    if constexpr (KIND == ONCHIP_SCALAR) {
      if (sy.table) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const float2 l = sy.table[Ln::fr_out(g2, q) * N + kx];
          v[0][q] = cmul(v[0][q], linv_factor(l.x, l.y, sy.inv_n));
        }
      } else {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const float p2 = p2x + axis_p2(sy, 0, Ln::fr_out(g2, q));
          v[0][q] = cmul(v[0][q],
                         linv_factor(fmaf(sy.a_re, p2, sy.b_re), fmaf(sy.a_im, p2, sy.b_im), sy.inv_n));
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        float2 tq[K];
#pragma unroll
        for (int k = 0; k < K; ++k) tq[k] = v[k][q];
        const float py = sy.ks[0] * (float)signed_freq(Ln::fr_out(g2, q), N);
        block_multiply<KIND>(tq, py, px, a.bsym, sy.inv_n);
#pragma unroll
        for (int k = 0; k < K; ++k) v[k][q] = tq[k];
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float2 t[NV];
      out_to_in<MM>(v[k], t);
#pragma unroll
      for (int q = 0; q < NV; ++q) v[k][q] = t[q];
      line_inv<N>(v[k], cb + k * F + kk * P, tw, rtw, g2);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int jy = Ln::sp_out(g2, q), d = jy / R, l = jy % R;
      const uint32_t off = (uint32_t)((l * P + swz<G>(l, kx)) * sizeof(float2));
#pragma unroll
      for (int k = 0; k < K; ++k)
        st_async(r_rb[d] + off + (uint32_t)(k * F * sizeof(float2)), v[k][q], m_rb[d]);
    }
    if (!wait_cluster(&mb[1], ph_rb, lim)) fail = 1;
    else if (tid == 0) mbar_arrive_expect_tx(&mb[1], LINE_BYTES);   // next round of rows
    ph_rb ^= 1u;

    // ---- C: inverse FFT along x, Delta, update, |Delta|^2 to every CTA
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int q = 0; q < NV; ++q) v[k][q] = rb[k * F + j * P + swz<G>(j, Ln::fr_in(g, q))];
    if (Cf::WARP_LINES) __syncwarp();  // a row's threads share a warp
    else __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) line_inv<N>(v[k], rb + k * F + j * P, tw, rtw, g);
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int col = Ln::sp_out(g, q);
      float2 xk[K], u[K], d[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        xk[k] = xs[k * F + j * P + col];
        u[k] = make_float2(v[k][q].x - xk[k].x, v[k][q].y - xk[k].y);
      }
      apply_B<KIND>(vs[j * P + col], u, d);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        ss = fmaf(d[k].x, d[k].x, fmaf(d[k].y, d[k].y, ss));
        if (!ref_pass)
          xs[k * F + j * P + col] = make_float2(fmaf(alpha, d[k].x, xk[k].x), fmaf(alpha, d[k].y, xk[k].y));
      }
    }
    double sd = (double)ss;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sd += __shfl_down_sync(0xffffffffu, sd, o);
    if ((tid & 31) == 0) red[tid >> 5] = sd;
    __syncthreads();  // also orders this step's updates of x before the next step A
    if (tid < C) {
      double cta = 0.0;
      for (int w = 0; w < T / 32; ++w) cta += red[w];
      st_async(r_sl[tid] + (uint32_t)(c * sizeof(double)), cta, m_sl[tid]);
    }
    if (ref_pass) {
      if (!wait_cluster(&mb[2], ph_sl, lim)) fail = 1;
      ph_sl ^= 1u;
      if (tid == 0) {
        double tot = 0.0;
        for (int r = 0; r < C; ++r) tot += slots[r];
        finalize_iteration(&S, nullptr, tot, F_REF);  // stores ||Delta|| as the reference
      }
      __syncthreads();
      if (fail && tid == 0) {
        S.status = ST_TIMEOUT;
        S.done = 1;
      }
      break;
    }
  }
  // Every byte sent to this CTA has been waited for (or a wait gave up):
  // meet the other CTAs before any of them leaves.
  cluster_barrier();
  if (c == 0 && tid == 0) *gst = S;
  if (!ref_pass && !fail) {
    for (int i = tid; i < R * N; i += T) {
      const int jj = i / N, col = i % N;
#pragma unroll
      for (int k = 0; k < K; ++k)
        a.x_out[base + k * NN + (int64_t)(row0 + jj) * N + col] = xs[k * F + jj * P + col];
    }
  }
}

template <int N, int RR, int KIND>
cudaError_t launch_n(const OnchipArgs& a, int problems, cudaStream_t s) {
  typedef OnchipCfg<N, RR, KIND> Cf;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(Cf::C * problems), 1, 1);
  cfg.blockDim = dim3(Cf::T, 1, 1);
  cfg.dynamicSmemBytes = Cf::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = Cf::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_onchip<N, RR, KIND>, a);
}

template <int N, int RR, int KIND>
int prepare_n() {
  typedef OnchipCfg<N, RR, KIND> Cf;
  if (cudaFuncSetAttribute(k_onchip<N, RR, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Cf::SMEM) != cudaSuccess)
    return 0;
  if (Cf::C > 8 && cudaFuncSetAttribute(k_onchip<N, RR, KIND>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                        1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Cf::C, 1, 1);
  cfg.blockDim = dim3(Cf::T, 1, 1);
  cfg.dynamicSmemBytes = Cf::SMEM;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = Cf::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_onchip<N, RR, KIND>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// The instantiations: (n, rows) for the scalar form; rows 8 and n <= 128 for
// the block forms (their K fields per array would not fit otherwise).
template <int KIND>
bool instantiated(int n, int rows) {
  if (KIND == ONCHIP_SCALAR) return onchip_rows_ok(n, rows);
  return rows == 8 && (n == 32 || n == 64 || n == 128);
}
// (the radix-3 sides 96 and 192 are built for the scalar form only)

template <int KIND>
int clusters_kind(int n, int rows) {
  if (!instantiated<KIND>(n, rows)) return 0;
  if (rows == 8) {
    switch (n) {
      case 32: return prepare_n<32, 8, KIND>();
      case 64: return prepare_n<64, 8, KIND>();
      case 128: return prepare_n<128, 8, KIND>();
    }
    if constexpr (KIND == ONCHIP_SCALAR)
      if (n == 96) return prepare_n<96, 8, KIND>();
    return 0;
  }
  if constexpr (KIND == ONCHIP_SCALAR) {
    switch (n) {
      case 32: return prepare_n<32, 16, KIND>();
      case 64: return prepare_n<64, 16, KIND>();
      case 96: return prepare_n<96, 16, KIND>();
      case 128: return prepare_n<128, 16, KIND>();
      case 192: return prepare_n<192, 16, KIND>();
      case 256: return prepare_n<256, 16, KIND>();
    }
  }
  return 0;
}

template <int KIND>
cudaError_t launch_kind(int n, int rows, const OnchipArgs& a, int problems, cudaStream_t s) {
  if (!instantiated<KIND>(n, rows)) return cudaErrorInvalidValue;
  if (rows == 8) {
    switch (n) {
      case 32: return launch_n<32, 8, KIND>(a, problems, s);
      case 64: return launch_n<64, 8, KIND>(a, problems, s);
      case 128: return launch_n<128, 8, KIND>(a, problems, s);
    }
    if constexpr (KIND == ONCHIP_SCALAR)
      if (n == 96) return launch_n<96, 8, KIND>(a, problems, s);
    return cudaErrorInvalidValue;
  }
  if constexpr (KIND == ONCHIP_SCALAR) {
    switch (n) {
      case 32: return launch_n<32, 16, KIND>(a, problems, s);
      case 64: return launch_n<64, 16, KIND>(a, problems, s);
      case 96: return launch_n<96, 16, KIND>(a, problems, s);
      case 128: return launch_n<128, 16, KIND>(a, problems, s);
      case 192: return launch_n<192, 16, KIND>(a, problems, s);
      case 256: return launch_n<256, 16, KIND>(a, problems, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool onchip_side(int n) { return n == 32 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256; }

// rows: rows per CTA, 16 or 8 (8 only for n <= 128: at most 16 CTAs).
bool onchip_rows_ok(int n, int rows) { return onchip_side(n) && (rows == 16 || (rows == 8 && n <= 128)); }

int onchip_clusters(int n, int rows, int kind) {
  switch (kind) {
    case ONCHIP_SCALAR: return clusters_kind<ONCHIP_SCALAR>(n, rows);
    case ONCHIP_ANTISYMMETRIC: return clusters_kind<ONCHIP_ANTISYMMETRIC>(n, rows);
    case ONCHIP_FLUX: return clusters_kind<ONCHIP_FLUX>(n, rows);
  }
  return 0;
}

cudaError_t launch_onchip(int n, int rows, const OnchipArgs& a, int problems, cudaStream_t s) {
  switch (a.kind) {
    case ONCHIP_SCALAR: return launch_kind<ONCHIP_SCALAR>(n, rows, a, problems, s);
    case ONCHIP_ANTISYMMETRIC: return launch_kind<ONCHIP_ANTISYMMETRIC>(n, rows, a, problems, s);
    case ONCHIP_FLUX: return launch_kind<ONCHIP_FLUX>(n, rows, a, problems, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace usp
