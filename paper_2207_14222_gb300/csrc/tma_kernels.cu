// tma_kernels.cu -- FFT passes along a strided axis with TMA-staged tiles.
//
// A tile is 32 consecutive columns x the whole axis (N values each), i.e. a
// box {32, N, 1} of the field viewed as [outer][N][inner].  A persistent CTA
// (one per SM, G = N2 warps) walks its tiles through a ring of three shared
// memory slots: while tile k is transformed in its slot, the TMA loads of
// tiles k+1 and k+2 are in flight, so the bytes in flight per SM do not
// depend on registers.  The result is written back into the slot and stored
// by TMA; a slot is reloaded only after the bulk group that stored from it
// has finished reading it.
//
// Used for every strided-axis pass of the FP32 iteration: the y and z passes
// of the pencil schedule and the z pass of the fused schedule (Eq.
// laplacian_inverse: forward FFT, multiply by 1/(N (Lhat+1)), inverse FFT).
#include "fft_core.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace usp {

namespace {

constexpr int SLOTS = 3;

template <int N, bool INV>
__device__ __forceinline__ void fft_cols_slot(float2* v, float2* ex, const float2* tw, int g,
                                              int lane) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  stage1<N, INV>(v, g, tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) ex[(k1 * N2 + g) * 32 + lane] = v[k1];
  __syncthreads();
  float2 w[N1];
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

__device__ __forceinline__ float2 spectral_factor_f(float p2, const Sym<float>& s, int mul) {
  const float lr = s.a_re * p2 + s.b_re;
  const float li = s.a_im * p2 + s.b_im;
  if (mul == MUL_L) return make_float2(lr * s.inv_n, li * s.inv_n);
  const float dr = lr + 1.f;
  // fast reciprocal division (about 2 ulp); the denominator |Lhat + 1|^2 >= 1
  const float sc = __fdividef(s.inv_n, dr * dr + li * li);
  return make_float2(dr * sc, -li * sc);
}

__device__ __forceinline__ float axis_p2_f(const Sym<float>& s, int ax, int k) {
  const float p = s.ks[ax] * float(signed_freq(k, s.n[ax]));
  return p * p;
}

}  // namespace

template <int N>
__global__ void __launch_bounds__(32 * Split<N>::G, 1)
    k_cols_tma(const __grid_constant__ CUtensorMap map, const ColsTmaArgs a) {
  constexpr int N1 = Split<N>::N1, G = Split<N>::G;
  constexpr int THREADS = 32 * G;
  constexpr int TILE = N * 32;
  constexpr uint32_t TILE_BYTES = TILE * sizeof(float2);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* slots = reinterpret_cast<float2*>(smem_raw);
  float2* tw = slots + SLOTS * TILE;
  __shared__ __align__(8) uint64_t full[SLOTS];
  __shared__ int ok_flag;

  if (!(a.flags & F_NOSTATE) && a.st->done) return;

  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t t0 = blockIdx.x, stride = gridDim.x;
  const int64_t my = t0 < a.tiles ? (a.tiles - t0 + stride - 1) / stride : 0;
  for (int m = threadIdx.x; m < N; m += THREADS)
    tw[m] = a.tw[stage1_twiddle_exponent(m, Split<N>::N2) * (256 / N)];
  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  int64_t issued = 0;  // tiles whose loads were issued (thread 0 only)
  if (threadIdx.x == 0) {
    for (; issued < 2 && issued < my; ++issued) {
      const int64_t t = t0 + issued * stride;
      mbar_arrive_expect_tx(&full[issued], TILE_BYTES);
      tma_load_3d(slots + issued * TILE, &map, int((t % a.inner_blocks) * 32), 0,
                  int(t / a.inner_blocks), &full[issued]);
    }
  }

  int64_t k = 0;
  bool failed = false;
  for (; k < my; ++k) {
    const int s = int(k % SLOTS);
    if (threadIdx.x == 0) ok_flag = mbar_wait(&full[s], uint32_t((k / SLOTS) & 1)) ? 1 : 0;
    __syncthreads();
    if (!ok_flag) {
      failed = true;
      break;
    }
    float2* slot = slots + s * TILE;
    const int64_t t = t0 + k * stride;
    const int64_t col = (t % a.inner_blocks) * 32 + lane;
    float2 v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = slot[in_index<N>(g, q) * 32 + lane];
    __syncthreads();  // the slot now serves as the exchange buffer
    if (a.mode == COL_INV) {
      fft_cols_slot<N, true>(v, slot, tw, g, lane);
    } else {
      fft_cols_slot<N, false>(v, slot, tw, g, lane);
      if (a.mode == COL_FWD_MUL_INV) {
        // outermost axis: the column index holds the faster axes' frequencies
        float p2in = 0.f;
        if (a.flags & F_CBLOCK) {
          p2in = axis_p2_f(a.sym, 2, int((col >> 13) * 32 + (col & 31))) +
                 axis_p2_f(a.sym, 1, int((col >> 5) & 255));
        } else if (a.sym.ndim == 3) {
          p2in = axis_p2_f(a.sym, 2, int(col % a.sym.n[2])) +
                 axis_p2_f(a.sym, 1, int(col / a.sym.n[2]));
        } else if (a.sym.ndim == 2) {
          p2in = axis_p2_f(a.sym, 1, int(col));
        }
        float2 tmp[N1];
#pragma unroll
        for (int q = 0; q < N1; ++q) {
          const int kk = out_index<N>(g, q);
          v[q] = cmul(v[q], spectral_factor_f(p2in + axis_p2_f(a.sym, 0, kk), a.sym, a.mul));
        }
        out_to_in<N>(v, tmp);
#pragma unroll
        for (int q = 0; q < N1; ++q) v[q] = tmp[q];
        fft_cols_slot<N, true>(v, slot, tw, g, lane);
      }
    }
#pragma unroll
    for (int q = 0; q < N1; ++q) slot[out_index<N>(g, q) * 32 + lane] = v[q];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_store_3d(&map, int((t % a.inner_blocks) * 32), 0, int(t / a.inner_blocks), slot);
      bulk_commit();
      if (issued < my) {
        // the slot of tile k+2 held tile k-1, whose store was committed one
        // tile ago: wait until at most the newest group still reads
        bulk_wait_read<1>();
        const int s2 = int(issued % SLOTS);
        const int64_t t2 = t0 + issued * stride;
        mbar_arrive_expect_tx(&full[s2], TILE_BYTES);
        tma_load_3d(slots + s2 * TILE, &map, int((t2 % a.inner_blocks) * 32), 0,
                    int(t2 / a.inner_blocks), &full[s2]);
        ++issued;
      }
    }
  }
  if (threadIdx.x == 0) {
    bulk_wait<0>();
    if (failed) {
      // let the loads still in flight land before the CTA's shared memory goes
      for (int64_t j = k; j < issued; ++j) mbar_wait(&full[j % SLOTS], uint32_t((j / SLOTS) & 1));
      a.st->status = ST_TIMEOUT;
      a.st->done = 1;
    }
  }
}

template <int N>
static size_t cols_tma_smem() {
  return sizeof(float2) * (SLOTS * N * 32 + N);
}

template <int N>
static cudaError_t cols_tma_go(const CUtensorMap& map, const ColsTmaArgs& a, int grid,
                               cudaStream_t s) {
  k_cols_tma<N><<<grid, 32 * Split<N>::G, cols_tma_smem<N>(), s>>>(map, a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t cols_tma_attr() {
  return cudaFuncSetAttribute(k_cols_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cols_tma_smem<N>());
}

cudaError_t cols_tma_init() {
  cudaError_t e;
  if ((e = cols_tma_attr<2>()) != cudaSuccess) return e;
  if ((e = cols_tma_attr<4>()) != cudaSuccess) return e;
  if ((e = cols_tma_attr<8>()) != cudaSuccess) return e;
  if ((e = cols_tma_attr<16>()) != cudaSuccess) return e;
  if ((e = cols_tma_attr<32>()) != cudaSuccess) return e;
  if ((e = cols_tma_attr<64>()) != cudaSuccess) return e;
  if ((e = cols_tma_attr<128>()) != cudaSuccess) return e;
  return cols_tma_attr<256>();
}

cudaError_t launch_cols_tma(int n, const CUtensorMap& map, const ColsTmaArgs& a, int grid,
                            cudaStream_t s) {
  switch (n) {
    case 2: return cols_tma_go<2>(map, a, grid, s);
    case 4: return cols_tma_go<4>(map, a, grid, s);
    case 8: return cols_tma_go<8>(map, a, grid, s);
    case 16: return cols_tma_go<16>(map, a, grid, s);
    case 32: return cols_tma_go<32>(map, a, grid, s);
    case 64: return cols_tma_go<64>(map, a, grid, s);
    case 128: return cols_tma_go<128>(map, a, grid, s);
    case 256: return cols_tma_go<256>(map, a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace usp
