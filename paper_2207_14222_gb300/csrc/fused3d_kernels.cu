// fused3d_kernels.cu -- the two-pass schedule of one fixed-point iteration
// (paper Algorithm 1, forward-eliminated operator of Sec. 2.1) for grids
// nz x 256 x 256:
//
//   plane pass (one 8-CTA thread-block cluster per xy-plane):
//       u = F_xy^-1 U ; Delta = (1-V)(u - x) ; x += alpha Delta ; ||Delta||^2 ;
//       t = (1-V) x + y ; T = F_xy t                      [a5 (xy), a6-a8, a2, a3 (xy)]
//   z pass (k_cols on the z axis):
//       U = F_z^-1 [ F_z T / (N (Lhat(p) + 1)) ]          [a3 (z), a4, a5 (z)]
//
// Algorithmic HBM bytes per point and iteration: plane 48 (read U, x, V, y;
// write x, T) + z 16 = 64, versus 112 for the pencil schedule.
//
// The plane's 256 x 256 complex values (512 KB) do not fit one CTA, so each of
// the 8 CTAs of a cluster owns 32 rows (row phase) or 32 columns (column
// phase) and the transposes between the two go through distributed shared
// memory.  The scratch field is stored in a column-block layout,
//   T[z][cb][y][xl],  x = 32 cb + xl,
// so that a CTA's column block of one plane is one contiguous 64 KB chunk and
// a z-pencil group of 32 consecutive columns is 256 contiguous bytes.
#include <cooperative_groups.h>

#include "fft_core.cuh"
#include "iteration_state.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace usp {

namespace {

constexpr int PN = 256;            // plane side (ny = nx)
constexpr int PC = 8;              // CTAs per plane (cluster size)
constexpr int PR = PN / PC;        // rows / columns per CTA
constexpr int PTHREADS = 512;      // 16 warps
constexpr size_t PSMEM = sizeof(float2) * (PN + PR * PN);
// staged variant: + V rows (complex64 worst case) + y rows
constexpr size_t PSMEM_TMA = sizeof(float2) * (PN + 3 * PR * PN);
constexpr uint32_t CHUNK_BYTES = sizeof(float2) * PR * PN;   // 64 KB

__device__ __forceinline__ double block_sum512(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < PTHREADS / 32; ++i) s += red[i];
  return s;
}

}  // namespace

template <int N, bool INV, typename V>
__device__ __forceinline__ void fft_cols_x(V* v, V* ex, const V* tw, int g, int lane) {
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

template <int N, bool INV, typename V>
__device__ __forceinline__ void fft_rows_x(V* v, V* exr, const V* tw, int g) {
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

__device__ __forceinline__ float2 ld_v(const void* V, int64_t i, bool vreal) {
  if (vreal) return make_float2(__ldg(reinterpret_cast<const float*>(V) + i), 0.f);
  return __ldg(reinterpret_cast<const float2*>(V) + i);
}

// One xy-plane per cluster; cluster rank r owns rows / column block r.
// STAGED: the scratch column block, V rows and y rows arrive by bulk copies
// issued at CTA start (the column block straight into the exchange buffer),
// and x is prefetched into registers, so all inputs are in flight before
// the first transform.  Bounded waits; a CTA whose wait times out still
// takes every cluster barrier so its siblings cannot hang.
template <bool STAGED>
__global__ void __cluster_dims__(PC, 1, 1) __launch_bounds__(PTHREADS, STAGED ? 1 : 2)
    k_plane(const PlaneArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* B = tw + PN;          // 32 x 256 complex: exchange and transpose buffer
  float2* SV = B + PR * PN;     // staged V rows (STAGED)
  float2* SY = SV + PR * PN;    // staged y rows (STAGED)
  __shared__ double red[PTHREADS / 32];
  __shared__ int is_last;
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int ok_flag;

  if (!(a.flags & F_NOSTATE) && a.st->done) return;

  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int64_t z = blockIdx.x / PC;
  const int tid = threadIdx.x;
  const int w = tid >> 5, l = tid & 31;      // column layout: warp = stage index, lane = column
  const int rho = tid >> 4, g = tid & 15;    // row layout: 16 threads per row
  const bool xzero = (a.flags & F_XZERO) != 0;
  const bool vreal = (a.flags & F_VREAL) != 0;
  const bool do_post = a.mode != PL_PRE;
  const bool do_pre = a.mode != PL_POST;
  const int64_t cblk = (z * PC + r) * (int64_t)(PN * PR);      // this CTA's column block
  const int64_t rows0 = z * (int64_t)(PN * PN) + (int64_t)(PR * r) * PN;  // its first row
  const int64_t row0 = rows0 + (int64_t)rho * PN;               // this thread's row
  bool ok = true;

  if (STAGED && tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  for (int m = tid; m < PN; m += PTHREADS) tw[m] = a.tw[stage1_twiddle_exponent(m, 16)];
  __syncthreads();
  if (STAGED && tid == 0) {
    if (do_post) {
      mbar_arrive_expect_tx(&bars[0], CHUNK_BYTES);
      bulk_load(B, a.buf + cblk, CHUNK_BYTES, &bars[0]);
    }
    const uint32_t vbytes = vreal ? CHUNK_BYTES / 2 : CHUNK_BYTES;
    const bool need_v = do_post || !xzero;
    const bool need_y = do_pre;
    mbar_arrive_expect_tx(&bars[1], (need_v ? vbytes : 0u) + (need_y ? CHUNK_BYTES : 0u));
    if (need_v) {
      const void* vsrc = vreal ? (const void*)(reinterpret_cast<const float*>(a.V) + rows0)
                               : (const void*)(reinterpret_cast<const float2*>(a.V) + rows0);
      bulk_load(SV, vsrc, vbytes, &bars[1]);
    }
    if (need_y) bulk_load(SY, a.y + rows0, CHUNK_BYTES, &bars[1]);
  }
  auto wait_bar = [&](int i) {   // uniform outcome for the whole CTA
    if (tid == 0) ok_flag = mbar_wait(&bars[i], 0) ? 1 : 0;
    __syncthreads();
    ok = ok && ok_flag;
  };
  // V, y of this thread's point x (row layout)
  auto vval = [&](int x) -> float2 {
    if (STAGED) return vreal ? make_float2(reinterpret_cast<const float*>(SV)[rho * PN + x], 0.f)
                             : SV[rho * PN + x];
    return ld_v(a.V, row0 + x, vreal);
  };
  auto yval = [&](int x) -> float2 { return STAGED ? SY[rho * PN + x] : a.y[row0 + x]; };

  float2* exr = B + rho * PN;
  float2 v[16];
  float acc = 0.f;

  if (do_post) {
    float2 xr[16];
    if (STAGED) {
#pragma unroll
      for (int q = 0; q < 16; ++q)
        xr[q] = xzero ? make_float2(0.f, 0.f) : a.x_in[row0 + g + 16 * q];
      wait_bar(0);
    }
    // ---- inverse FFT along y on this CTA's 32 columns
#pragma unroll
    for (int q = 0; q < 16; ++q)
      v[q] = STAGED ? B[(16 * q + w) * PR + l] : a.buf[cblk + (16 * q + w) * PR + l];
    if (STAGED) __syncthreads();    // B becomes the exchange buffer
    fft_cols_x<PN, true>(v, B, tw, w, l);
#pragma unroll
    for (int q = 0; q < 16; ++q) B[(w + 16 * q) * PR + l] = v[q];   // B[y][xl]
    cluster.sync();
    // ---- transpose: this CTA's 32 rows, gathered from all column blocks
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float2* src = cluster.map_shared_rank(B, q >> 1);
      v[q] = src[(PR * r + rho) * PR + 16 * (q & 1) + g];       // x = 16 q + g
    }
    cluster.sync();
    // ---- inverse FFT along x; Delta, update, next B x + y
    fft_rows_x<PN, true>(v, exr, tw, g);
    if (STAGED) wait_bar(1);
    const float al = a.alpha;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = g + 16 * q;
      const int64_t i = row0 + x;
      const float2 vv = vval(x);
      const float2 xv = STAGED ? xr[q] : (xzero ? make_float2(0.f, 0.f) : a.x_in[i]);
      const float ur = v[q].x - xv.x, ui = v[q].y - xv.y;
      const float br = 1.f - vv.x, bi = -vv.y;
      const float dr = br * ur - bi * ui, di = br * ui + bi * ur;
      acc += dr * dr + di * di;
      const float2 xn = make_float2(xv.x + al * dr, xv.y + al * di);
      if (!(a.flags & F_REF)) a.x_out[i] = xn;
      if (do_pre) {
        const float2 yv = yval(x);
        v[q] = make_float2(yv.x + br * xn.x - bi * xn.y, yv.y + br * xn.y + bi * xn.x);
      }
    }
  } else {
    // prologue: t = (1-V) x + y at x = 16 q + g
    float2 xr[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
      xr[q] = xzero ? make_float2(0.f, 0.f) : a.x_in[row0 + 16 * q + g];
    if (STAGED) wait_bar(1);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = 16 * q + g;
      float2 t = yval(x);
      if (!xzero) {
        const float2 vv = vval(x);
        const float br = 1.f - vv.x, bi = -vv.y;
        t.x += br * xr[q].x - bi * xr[q].y;
        t.y += br * xr[q].y + bi * xr[q].x;
      }
      v[q] = t;
    }
  }

  if (do_pre) {
    // ---- forward FFT along x (register order is the stage-1 order for 256)
    fft_rows_x<PN, false>(v, exr, tw, g);
#pragma unroll
    for (int q = 0; q < 16; ++q) exr[g + 16 * q] = v[q];     // B[row][kx]
    cluster.sync();
    // ---- transpose: this CTA's 32 columns (kx), gathered from all row blocks
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float2* src = cluster.map_shared_rank(B, q >> 1);
      v[q] = src[(16 * (q & 1) + w) * PN + PR * r + l];         // y = 16 q + w
    }
    cluster.sync();
    // ---- forward FFT along y, store the column block
    fft_cols_x<PN, false>(v, B, tw, w, l);
#pragma unroll
    for (int q = 0; q < 16; ++q) a.buf[cblk + (w + 16 * q) * PR + l] = v[q];
  }

  if (STAGED && !ok && tid == 0) {
    // let late copies land before this CTA's shared memory is released
    if (do_post) mbar_wait(&bars[0], 0);
    mbar_wait(&bars[1], 0);
    a.st->status = ST_TIMEOUT;
    a.st->done = 1;
  }

  if (do_post) {
    const double bs = block_sum512((double)acc, red);
    if (threadIdx.x == 0) {
      a.partials[blockIdx.x] = bs;
      __threadfence();
      const unsigned t = atomicAdd(&a.st->ticket, 1u);
      is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      double s = 0.0;
      for (unsigned i = threadIdx.x; i < gridDim.x; i += PTHREADS) s += __ldcg(a.partials + i);
      const double tot = block_sum512(s, red);
      if (threadIdx.x == 0) {
        if (a.st->status != ST_TIMEOUT) finalize_iteration(a.st, a.hist, tot, a.flags);
        a.st->ticket = 0u;
      }
    }
  }
}

cudaError_t plane_kernel_init() {
  cudaError_t e = cudaFuncSetAttribute(k_plane<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)PSMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_plane<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PSMEM_TMA);
}

cudaError_t launch_plane(const PlaneArgs& a, cudaStream_t s) {
  if (a.staged)
    k_plane<true><<<(unsigned)(a.nz * PC), PTHREADS, PSMEM_TMA, s>>>(a);
  else
    k_plane<false><<<(unsigned)(a.nz * PC), PTHREADS, PSMEM, s>>>(a);
  return cudaGetLastError();
}

int plane_max_active_clusters() {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PC * 256, 1, 1);
  cfg.blockDim = dim3(PTHREADS, 1, 1);
  cfg.dynamicSmemBytes = PSMEM_TMA;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = PC;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_plane<true>, &cfg) != cudaSuccess) return -1;
  return n;
}

}  // namespace usp
