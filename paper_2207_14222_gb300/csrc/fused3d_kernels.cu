// fused3d_kernels.cu -- the two-pass schedule of one fixed-point iteration
// (paper Algorithm 1, forward-eliminated operator of Sec. 2.1) for grids
// nz x 256 x 256:
//
//   plane pass (8-CTA thread-block clusters, persistent over xy-planes):
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
constexpr int CHUNK = PR * PN;     // complex values a CTA owns per plane
constexpr uint32_t CHUNK_BYTES = sizeof(float2) * CHUNK;     // 64 KB
constexpr size_t PSMEM = sizeof(float2) * (3 * CHUNK + PN);  // C, SV, SY, twiddles

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

// Persistent: cluster c processes planes c, c + nclusters, ...  CTA rank r
// owns column block r (columns 32r..32r+31) in the column phases and rows
// 32r..32r+31 in the row phase.  Three 64 KB slots, all filled by bulk
// copies issued during the previous plane:
//   C : scratch column block; exchange of the inverse FFT y; transpose source
//       (column results); exchange of the inverse FFT x; refilled with the
//       next plane's column block right after that.
//   SV: V rows; exchange of the forward FFT y; refilled after it.
//   SY: y rows; exchange of the forward FFT x; transpose source (row
//       results); refilled after the peers have read it.
// x of the next plane is prefetched into registers after the pointwise step.
// Per plane: cluster barriers after each transpose source is written and
// after the peers have read it (4 for an iteration, 2 for the prologue and
// the reference pass).  Waits are bounded; a CTA whose wait timed out still
// takes every barrier, so its peers cannot hang.
__global__ void __cluster_dims__(PC, 1, 1) __launch_bounds__(PTHREADS, 1)
    k_plane(const PlaneArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* C = reinterpret_cast<float2*>(smem_raw);
  float2* SV = C + CHUNK;
  float2* SY = SV + CHUNK;
  float2* tw = SY + CHUNK;
  __shared__ double red[PTHREADS / 32];
  __shared__ int is_last;
  __shared__ __align__(8) uint64_t bars[3];   // C (U column block), SV, SY
  __shared__ int ok_flag;

  if (!(a.flags & F_NOSTATE) && a.st->done) return;

  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int ncl = gridDim.x / PC, cid = blockIdx.x / PC;
  const int tid = threadIdx.x;
  const int w = tid >> 5, l = tid & 31;      // column layout: warp = stage index, lane = column
  const int rho = tid >> 4, g = tid & 15;    // row layout: 16 threads per row
  const bool xzero = (a.flags & F_XZERO) != 0;
  const bool vreal = (a.flags & F_VREAL) != 0;
  const bool do_post = a.mode != PL_PRE;
  const bool do_pre = a.mode != PL_POST;
  const bool need_v = do_post || !xzero;
  bool ok = true;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  for (int m = tid; m < PN; m += PTHREADS) tw[m] = a.tw[stage1_twiddle_exponent(m, 16)];
  __syncthreads();

  auto issue = [&](int which, int64_t zz) {   // 0: U column block, 1: V rows, 2: y rows
    const int64_t rows0 = zz * (int64_t)(PN * PN) + (int64_t)(PR * r) * PN;
    if (which == 0) {
      mbar_arrive_expect_tx(&bars[0], CHUNK_BYTES);
      bulk_load(C, a.buf + (zz * PC + r) * (int64_t)CHUNK, CHUNK_BYTES, &bars[0]);
    } else if (which == 1) {
      const uint32_t bytes = vreal ? CHUNK_BYTES / 2 : CHUNK_BYTES;
      const void* src = vreal ? (const void*)(reinterpret_cast<const float*>(a.V) + rows0)
                              : (const void*)(reinterpret_cast<const float2*>(a.V) + rows0);
      mbar_arrive_expect_tx(&bars[1], bytes);
      bulk_load(SV, src, bytes, &bars[1]);
    } else {
      mbar_arrive_expect_tx(&bars[2], CHUNK_BYTES);
      bulk_load(SY, a.y + rows0, CHUNK_BYTES, &bars[2]);
    }
  };
  auto wait_bar = [&](int i, uint32_t parity) {   // one outcome for the whole CTA
    if (tid == 0) ok_flag = mbar_wait(&bars[i], parity) ? 1 : 0;
    __syncthreads();
    ok = ok && ok_flag;
  };
  auto refill = [&](int which, int64_t zz) {   // slot free (all threads) -> next plane
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && zz < a.nz) issue(which, zz);
  };

  float2 xr[16];
  auto prefetch_x = [&](int64_t zz) {    // row layout: x = g + 16 q of row 32 r + rho
    const int64_t row0 = zz * (int64_t)(PN * PN) + (int64_t)(PR * r + rho) * PN;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      xr[q] = xzero ? make_float2(0.f, 0.f) : a.x_in[row0 + g + 16 * q];
  };

  if (cid < a.nz) {
    if (tid == 0) {
      if (do_post) issue(0, cid);
      if (need_v) issue(1, cid);
      if (do_pre) issue(2, cid);
    }
    prefetch_x(cid);
  }

  float acc = 0.f;
  int it = 0;
  for (int64_t z = cid; z < a.nz; z += ncl, ++it) {
    const uint32_t par = uint32_t(it & 1);
    const int64_t znext = z + ncl;
    const int64_t row0 = z * (int64_t)(PN * PN) + (int64_t)(PR * r + rho) * PN;
    float2 v[16];
    if (do_post) {
      // ---- inverse FFT y on this CTA's column block (exchange in C)
      wait_bar(0, par);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = C[(16 * q + w) * PR + l];
      __syncthreads();
      fft_cols_x<PN, true>(v, C, tw, w, l);                    // v[q]: y = w + 16 q
#pragma unroll
      for (int q = 0; q < 16; ++q) C[(w + 16 * q) * PR + l] = v[q];   // C[y][xl]
      cluster.sync();
      // ---- transpose: this CTA's rows from every column block
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float2* src = cluster.map_shared_rank(C, q >> 1);
        v[q] = src[(PR * r + rho) * PR + 16 * (q & 1) + g];     // x = 16 q + g
      }
      cluster.sync();
      // ---- inverse FFT x (exchange in C), then C takes the next block
      fft_rows_x<PN, true>(v, C + rho * PN, tw, g);             // v[q]: x = g + 16 q
      refill(0, znext);
    }
    if (need_v) wait_bar(1, par);
    if (do_pre) wait_bar(2, par);
    // ---- pointwise: Delta, update, norm, next B x + y (row layout)
    const float al = a.alpha;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = do_post ? g + 16 * q : 16 * q + g;
      const int c = rho * PN + x;
      float2 vv = make_float2(0.f, 0.f);
      if (need_v)
        vv = vreal ? make_float2(reinterpret_cast<const float*>(SV)[c], 0.f) : SV[c];
      const float br = 1.f - vv.x, bi = -vv.y;
      float2 xn = xr[q];
      if (do_post) {
        const float ur = v[q].x - xr[q].x, ui = v[q].y - xr[q].y;
        const float dr = br * ur - bi * ui, di = br * ui + bi * ur;
        acc += dr * dr + di * di;
        xn = make_float2(xr[q].x + al * dr, xr[q].y + al * di);
        if (!(a.flags & F_REF)) a.x_out[row0 + x] = xn;
      }
      if (do_pre) {
        const float2 yv = SY[c];
        v[q] = make_float2(yv.x + br * xn.x - bi * xn.y, yv.y + br * xn.y + bi * xn.x);
      }
    }
    if (znext < a.nz) prefetch_x(znext);
    if (!do_pre) {
      refill(1, need_v ? znext : a.nz);   // V slot free
      cluster.sync();                     // peers are done with C before it is rewritten
      continue;
    }
    // ---- forward FFT x (exchange in SY, consumed); row results stay in SY
    __syncthreads();
    fft_rows_x<PN, false>(v, SY + rho * PN, tw, g);             // v[q]: kx = g + 16 q
#pragma unroll
    for (int q = 0; q < 16; ++q) SY[rho * PN + g + 16 * q] = v[q];
    cluster.sync();
    // ---- transpose: this CTA's column block from every row block
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float2* src = cluster.map_shared_rank(SY, q >> 1);
      v[q] = src[(16 * (q & 1) + w) * PN + PR * r + l];         // y = 16 q + w
    }
    cluster.sync();
    refill(2, znext);                                            // peers have read SY
    // ---- forward FFT y (exchange in SV, consumed), store the column block
    fft_cols_x<PN, false>(v, SV, tw, w, l);                      // v[q]: ky = w + 16 q
    const int64_t cblk = (z * PC + r) * (int64_t)CHUNK;
#pragma unroll
    for (int q = 0; q < 16; ++q) a.buf[cblk + (w + 16 * q) * PR + l] = v[q];
    refill(1, need_v ? znext : a.nz);
  }

  if (!ok && tid == 0) {
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
      double sm = 0.0;
      for (unsigned i = threadIdx.x; i < gridDim.x; i += PTHREADS) sm += __ldcg(a.partials + i);
      const double tot = block_sum512(sm, red);
      if (threadIdx.x == 0) {
        if (a.st->status != ST_TIMEOUT) finalize_iteration(a.st, a.hist, tot, a.flags);
        a.st->ticket = 0u;
      }
    }
  }
}

cudaError_t plane_kernel_init() {
  return cudaFuncSetAttribute(k_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PSMEM);
}

cudaError_t launch_plane(const PlaneArgs& a, int clusters, cudaStream_t s) {
  k_plane<<<(unsigned)(clusters * PC), PTHREADS, PSMEM, s>>>(a);
  return cudaGetLastError();
}

int plane_max_active_clusters() {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PC * 256, 1, 1);
  cfg.blockDim = dim3(PTHREADS, 1, 1);
  cfg.dynamicSmemBytes = PSMEM;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = PC;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_plane, &cfg) != cudaSuccess) return -1;
  return n;
}

}  // namespace usp
