// onchip_kernels.cu -- whole phases of Algorithm 1 for small square 2-D grids
// (n x n, n in {32, 64, 128, 256}) with every field resident in the shared
// memory of one thread-block cluster.
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

template <int N, int RR>
struct OnchipCfg {
  static constexpr int R = RR;               // rows (and k-space columns) per CTA
  static constexpr int C = N / R;            // CTAs per cluster
  static constexpr int G = Split<N>::G;      // threads per line
  static constexpr int NV = Split<N>::N1;    // values per thread
  static constexpr int T = R * G;            // threads per CTA
  static constexpr int P = N + 8;            // line stride (float2): rows of a warp on both bank halves
  static constexpr int FIELD = R * P;        // float2 per resident array
  // x, V, y, row buffer, column buffer, twiddles; then C + T/32 doubles
  static constexpr size_t SMEM = sizeof(float2) * (5 * (size_t)FIELD + N) + sizeof(double) * (C + T / 32);
  static_assert(Split<N>::N1 * Split<N>::N2 == N, "length");
  static_assert(T % 32 == 0, "whole warps");
  static_assert(C >= 2 && C <= 16, "cluster size");
  static_assert(G <= 32 && 32 % G == 0, "the threads of a line share a warp");
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
__device__ __forceinline__ bool wait_cluster(uint64_t* b, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
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

template <int N, int RR>
__global__ void __launch_bounds__(OnchipCfg<N, RR>::T, 1) k_onchip(OnchipArgs a) {
  typedef OnchipCfg<N, RR> K;
  constexpr int C = K::C, R = K::R, G = K::G, NV = K::NV, T = K::T, P = K::P;
  constexpr uint32_t LINE_BYTES = (uint32_t)(R * N * sizeof(float2));   // one round into rb or cb
  constexpr uint32_t SLOT_BYTES = (uint32_t)(C * sizeof(double));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  float2* vs = xs + K::FIELD;
  float2* ys = vs + K::FIELD;
  float2* rb = ys + K::FIELD;   // rows: k-space along x (exchange area of step A, input of step C)
  float2* cb = rb + K::FIELD;   // k-space columns (input of step B)
  float2* tw = cb + K::FIELD;
  double* slots = reinterpret_cast<double*>(tw + N);   // |Delta|^2 of each CTA
  double* red = slots + C;
  __shared__ DevState S;
  __shared__ __align__(8) uint64_t mb[3];   // cb, rb, slots full
  __shared__ uint32_t r_rb[C], r_cb[C], r_sl[C], m_rb[C], m_cb[C], m_sl[C];
  __shared__ int fail;

  const int tid = threadIdx.x;
  const uint32_t c = cluster_rank();
  const int p = blockIdx.x / C;
  const int64_t base = (int64_t)p * N * N;
  DevState* gst = a.st + p;
  double* hist = c == 0 ? a.hist + (int64_t)p * a.bt.hist_stride : nullptr;
  const Sym<float> sy = problem_sym(a.sym, a.bt, p);
  const float alpha = a.bt.alpha ? a.bt.alpha[p] : a.alpha;
  const bool vreal = (a.flags & F_VREAL) != 0;
  const bool ref_pass = (a.flags & F_REF) != 0;
  const bool xzero = (a.flags & F_XZERO) != 0;
  const uint32_t lim = a.wait_limit ? a.wait_limit : (1u << 22);

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
  for (int m = tid; m < N; m += T) tw[m] = a.tw[stage1_twiddle_exponent(m, Split<N>::N2) * (256 / N)];
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
    const int j = i / N, col = i % N;
    const int64_t gi = base + (int64_t)(row0 + j) * N + col;
    xs[j * P + col] = xzero ? make_float2(0.f, 0.f) : a.x_in[gi];
    vs[j * P + col] = vreal ? make_float2(reinterpret_cast<const float*>(a.V)[gi], 0.f)
                            : reinterpret_cast<const float2*>(a.V)[gi];
    ys[j * P + col] = a.y[gi];
  }
  cluster_barrier();  // every CTA has started and armed its barriers

  const int j = tid / G, g = tid % G;    // step A / C: row j, line thread g
  const int kk = j, g2 = g;              // step B: k-space column kk
  const int kx = row0 + kk;              // its frequency index along x
  const float p2x = axis_p2(sy, 1, kx);
  uint32_t ph_cb = 0, ph_rb = 0, ph_sl = 0;
  float2 v[NV];
  bool first = true;
  // Bounded by the state's own limit: finalize_iteration stops at it_limit.
  for (int iter = 0;; ++iter) {
    // ---- A: t = (1 - V) x + y, FFT along x, k-space values to column owners
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int col = in_index<N>(g, q);
      const float2 xv = xs[j * P + col], vv = vs[j * P + col], yv = ys[j * P + col];
      const float br = 1.f - vv.x;
      v[q] = make_float2(fmaf(br, xv.x, fmaf(vv.y, xv.y, yv.x)), fmaf(br, xv.y, fmaf(-vv.y, xv.x, yv.y)));
    }
    fft_line<N>(v, rb + j * P, tw, g, false);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int k = out_index<N>(g, q), d = k / R, l = k % R;
      st_async(r_cb[d] + (uint32_t)((l * P + swz<G>(l, row0 + j)) * sizeof(float2)), v[q], m_cb[d]);
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
    for (int q = 0; q < NV; ++q) v[q] = cb[kk * P + swz<G>(kk, in_index<N>(g2, q))];
    __syncwarp();  // a column's threads share a warp
    fft_line<N>(v, cb + kk * P, tw, g2, false);
    if (sy.table) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const float2 l = sy.table[out_index<N>(g2, q) * N + kx];
        v[q] = cmul(v[q], linv_factor(l.x, l.y, sy.inv_n));
      }
    } else {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const float p2 = p2x + axis_p2(sy, 0, out_index<N>(g2, q));
        v[q] = cmul(v[q], linv_factor(fmaf(sy.a_re, p2, sy.b_re), fmaf(sy.a_im, p2, sy.b_im), sy.inv_n));
      }
    }
    {
      float2 t[NV];
      out_to_in<N>(v, t);
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] = t[q];
    }
    fft_line<N>(v, cb + kk * P, tw, g2, true);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int jy = out_index<N>(g2, q), d = jy / R, l = jy % R;
      st_async(r_rb[d] + (uint32_t)((l * P + swz<G>(l, kx)) * sizeof(float2)), v[q], m_rb[d]);
    }
    if (!wait_cluster(&mb[1], ph_rb, lim)) fail = 1;
    else if (tid == 0) mbar_arrive_expect_tx(&mb[1], LINE_BYTES);   // next round of rows
    ph_rb ^= 1u;

    // ---- C: inverse FFT along x, Delta, update, |Delta|^2 to every CTA
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = rb[j * P + swz<G>(j, in_index<N>(g, q))];
    __syncwarp();  // a row's threads share a warp
    fft_line<N>(v, rb + j * P, tw, g, true);
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int col = out_index<N>(g, q);
      const float2 xv = xs[j * P + col], vv = vs[j * P + col];
      const float2 u = make_float2(v[q].x - xv.x, v[q].y - xv.y);
      const float br = 1.f - vv.x;
      const float2 d = make_float2(fmaf(br, u.x, vv.y * u.y), fmaf(br, u.y, -vv.y * u.x));
      ss = fmaf(d.x, d.x, fmaf(d.y, d.y, ss));
      if (!ref_pass) xs[j * P + col] = make_float2(fmaf(alpha, d.x, xv.x), fmaf(alpha, d.y, xv.y));
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
      a.x_out[base + (int64_t)(row0 + jj) * N + col] = xs[jj * P + col];
    }
  }
}

template <int N, int RR>
cudaError_t launch_n(const OnchipArgs& a, int problems, cudaStream_t s) {
  typedef OnchipCfg<N, RR> K;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(K::C * problems), 1, 1);
  cfg.blockDim = dim3(K::T, 1, 1);
  cfg.dynamicSmemBytes = K::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = K::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_onchip<N, RR>, a);
}

template <int N, int RR>
int prepare_n() {
  typedef OnchipCfg<N, RR> K;
  if (cudaFuncSetAttribute(k_onchip<N, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM) !=
      cudaSuccess)
    return 0;
  if (K::C > 8 && cudaFuncSetAttribute(k_onchip<N, RR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(K::C, 1, 1);
  cfg.blockDim = dim3(K::T, 1, 1);
  cfg.dynamicSmemBytes = K::SMEM;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = K::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_onchip<N, RR>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

bool onchip_side(int n) { return n == 32 || n == 64 || n == 128 || n == 256; }

// rows: rows per CTA, 16 or 8 (8 only for n <= 128: at most 16 CTAs).
bool onchip_rows_ok(int n, int rows) { return onchip_side(n) && (rows == 16 || (rows == 8 && n <= 128)); }

int onchip_clusters(int n, int rows) {
  if (!onchip_rows_ok(n, rows)) return 0;
  if (rows == 8) {
    switch (n) {
      case 32: return prepare_n<32, 8>();
      case 64: return prepare_n<64, 8>();
      case 128: return prepare_n<128, 8>();
    }
    return 0;
  }
  switch (n) {
    case 32: return prepare_n<32, 16>();
    case 64: return prepare_n<64, 16>();
    case 128: return prepare_n<128, 16>();
    case 256: return prepare_n<256, 16>();
  }
  return 0;
}

cudaError_t launch_onchip(int n, int rows, const OnchipArgs& a, int problems, cudaStream_t s) {
  if (!onchip_rows_ok(n, rows)) return cudaErrorInvalidValue;
  if (rows == 8) {
    switch (n) {
      case 32: return launch_n<32, 8>(a, problems, s);
      case 64: return launch_n<64, 8>(a, problems, s);
      case 128: return launch_n<128, 8>(a, problems, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (n) {
    case 32: return launch_n<32, 16>(a, problems, s);
    case 64: return launch_n<64, 16>(a, problems, s);
    case 128: return launch_n<128, 16>(a, problems, s);
    case 256: return launch_n<256, 16>(a, problems, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace usp
