// tc_kernels.cu -- the 256-point transforms of a strided-axis pass on the
// 5th-generation tensor cores (tcgen05.mma, operands in shared memory,
// accumulator in tensor memory).
//
// A tile is 8 columns x 256 points (TMA box {8, 256, 1}, the same ring of
// three slots as the CUDA-core pass).  With n = 16 n1 + n2 and
// k = k1 + 16 k2 the forward transform is
//   stage A  Y[k1](n2, c) = sum_n1 W16^(n1 k1) X[16 n1 + n2](c)
//   twiddle  Y'[k1](n2, c) = W256^(n2 k1) Y[k1](n2, c)
//   stage B  X^[k1 + 16 k2](c) = sum_n2 W16^(n2 k2) Y'[k1](n2, c)
// and the inverse runs the conjugate stages in reverse order.  Each stage is
// one real GEMM D[128 x 32] = A[128 x 32] B[32 x 32]: the 128 rows are the
// (n2 or k1, column) pairs of the tile, the 32 K entries the real and
// imaginary parts of the 16 inputs, the 32 outputs the real and imaginary
// parts of the 16 results, B the DFT-16 matrix in real form.  Thread r of
// the CTA owns row r of A and of D (tensor-memory lane r).
//
// Precision: kind::tf32 products with the split a = a_hi + a_lo (each part
// rounded to TF32): D = A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in
// FP32, which keeps the transform at FP32-level accuracy.  Twiddles, the
// spectral multiply and the hi/lo splits run on the CUDA cores.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "fft_core.cuh"
#include "iteration_state.cuh"
#include "tc_kernels.h"
#include "tma.cuh"

namespace usp {

namespace {

constexpr int TC_SLOTS = 3;
constexpr int TC_COLS = 8;
constexpr int TC_N = 256;
constexpr int TC_THREADS = 128;
constexpr int TC_TILE = TC_N * TC_COLS;                     // complex values per tile
constexpr uint32_t TC_TILE_BYTES = TC_TILE * sizeof(float2);
constexpr int OP_FLOATS = 128 * 32;                         // one A operand (16 KB)
constexpr int B_FLOATS = 32 * 32;                           // one B operand (4 KB)
constexpr uint32_t TMEM_COLS = 32;

// F hi, F lo, conj(F) hi, conj(F) lo in the operand layout (B_FLOATS each)
__device__ float g_tc_b[4 * B_FLOATS];

// Offset (floats) of element (row, k) of a 32-wide K-major operand in the
// canonical no-swizzle layout: core matrices of 8 rows x 4 K entries (16 B
// per row), 128 B apart along K, 1024 B apart between 8-row groups.
__host__ __device__ __forceinline__ int cofs(int row, int k) {
  return (row >> 3) * 256 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading (K) and stride (8-row
// group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major,
// N = 32, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Row `row` of the operand from this thread's 16 complex values (K order).
__device__ __forceinline__ void put_row(float* Ahi, float* Alo, int row, const float2* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float4 h, l;
    h.x = tf32_rna(v[4 * q].x);     l.x = tf32_rna(v[4 * q].x - h.x);
    h.y = tf32_rna(v[4 * q + 1].x); l.y = tf32_rna(v[4 * q + 1].x - h.y);
    h.z = tf32_rna(v[4 * q + 2].x); l.z = tf32_rna(v[4 * q + 2].x - h.z);
    h.w = tf32_rna(v[4 * q + 3].x); l.w = tf32_rna(v[4 * q + 3].x - h.w);
    *reinterpret_cast<float4*>(Ahi + cofs(row, 4 * q)) = h;
    *reinterpret_cast<float4*>(Alo + cofs(row, 4 * q)) = l;
    h.x = tf32_rna(v[4 * q].y);     l.x = tf32_rna(v[4 * q].y - h.x);
    h.y = tf32_rna(v[4 * q + 1].y); l.y = tf32_rna(v[4 * q + 1].y - h.y);
    h.z = tf32_rna(v[4 * q + 2].y); l.z = tf32_rna(v[4 * q + 2].y - h.z);
    h.w = tf32_rna(v[4 * q + 3].y); l.w = tf32_rna(v[4 * q + 3].y - h.w);
    *reinterpret_cast<float4*>(Ahi + cofs(row, 16 + 4 * q)) = h;
    *reinterpret_cast<float4*>(Alo + cofs(row, 16 + 4 * q)) = l;
  }
}

// Entry kpos of rows (8 j + col), j = 0..15, from this thread's 16 values:
// the transpose between the two stages.
__device__ __forceinline__ void put_col(float* Ahi, float* Alo, int col, int kpos, const float2* v) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int row = 8 * j + col;
    const float hr = tf32_rna(v[j].x), hi = tf32_rna(v[j].y);
    Ahi[cofs(row, kpos)] = hr;
    Alo[cofs(row, kpos)] = tf32_rna(v[j].x - hr);
    Ahi[cofs(row, 16 + kpos)] = hi;
    Alo[cofs(row, 16 + kpos)] = tf32_rna(v[j].y - hi);
  }
}

// One stage: D = A B (three TF32 products), then this thread's row of D
// into v (16 complex).  Returns false if the tensor core did not report
// completion within the wait limit.
__device__ __forceinline__ bool run_stage(const float* Ahi, const float* Alo, const float* Bhi,
                                          const float* Blo, uint32_t tmem, uint64_t* bar,
                                          uint32_t& phase, int* ok_flag, float2* v) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operands -> async proxy
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {   // K = 32 in steps of 8 (256 B of each operand)
      const uint64_t ah = sdesc(saddr(Ahi) + 256 * j), al = sdesc(saddr(Alo) + 256 * j);
      const uint64_t bh = sdesc(saddr(Bhi) + 256 * j), bl = sdesc(saddr(Blo) + 256 * j);
      mma_tf32(tmem, ah, bh, j > 0 ? 1u : 0u);
      mma_tf32(tmem, ah, bl, 1u);
      mma_tf32(tmem, al, bh, 1u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
    *ok_flag = mbar_wait(bar, phase) ? 1 : 0;
  }
  __syncthreads();
  phase ^= 1u;
  if (!*ok_flag) return false;
  tc_fence_after();
  uint32_t r[32];
  const uint32_t taddr = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = make_float2(__uint_as_float(r[c]), __uint_as_float(r[16 + c]));
  tc_fence_before();
  return true;
}

__device__ __forceinline__ float p2_axis(const Sym<float>& s, int ax, int k) {
  const float p = s.ks[ax] * float(signed_freq(k, s.n[ax]));
  return p * p;
}

__global__ void __launch_bounds__(TC_THREADS, 2)
    k_cols_tc(const __grid_constant__ CUtensorMap map, const ColsTmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float2* slots = reinterpret_cast<float2*>(smem_raw);
  float* Ahi = reinterpret_cast<float*>(slots + TC_SLOTS * TC_TILE);
  float* Alo = Ahi + OP_FLOATS;
  float* Bs = Alo + OP_FLOATS;                     // F hi, F lo, conj F hi, conj F lo
  float2* tw = reinterpret_cast<float2*>(Bs + 4 * B_FLOATS);
  __shared__ __align__(8) uint64_t full[TC_SLOTS];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int ok_flag;

  if (a.st->done) return;

  const int tid = threadIdx.x;
  const int col = tid & 7, hq = tid >> 3;          // (row group index, column) of row tid
  const int64_t t0 = blockIdx.x, stride = gridDim.x;
  const int64_t my = t0 < a.tiles ? (a.tiles - t0 + stride - 1) / stride : 0;
  for (int i = tid; i < 4 * B_FLOATS; i += TC_THREADS) Bs[i] = g_tc_b[i];
  for (int m = tid; m < TC_N; m += TC_THREADS) tw[m] = a.tw[m];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < TC_SLOTS; ++s) mbar_init(&full[s], 1);
    mbar_init(&mma_bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const bool fwd = a.mode != COL_INV, mul = a.mode == COL_FWD_MUL_INV, inv = a.mode != COL_FWD;

  int64_t issued = 0;  // tiles whose loads were issued (thread 0 only)
  if (tid == 0) {
    for (; issued < 2 && issued < my; ++issued) {
      const int64_t t = t0 + issued * stride;
      mbar_arrive_expect_tx(&full[issued], TC_TILE_BYTES);
      tma_load_3d(slots + issued * TC_TILE, &map, int((t % a.inner_blocks) * TC_COLS), 0,
                  int(t / a.inner_blocks), &full[issued]);
    }
  }
  uint32_t phase = 0;
  bool failed = false;
  int64_t k = 0;
  for (; k < my && !failed; ++k) {
    const int s = int(k % TC_SLOTS);
    if (tid == 0) ok_flag = mbar_wait(&full[s], uint32_t((k / TC_SLOTS) & 1)) ? 1 : 0;
    __syncthreads();
    if (!ok_flag) {
      failed = true;
      break;
    }
    float2* slot = slots + s * TC_TILE;
    const int64_t t = t0 + k * stride;
    const int64_t gcol = (t % a.inner_blocks) * TC_COLS + col;
    float2 v[16];
    if (fwd) {
      // stage A: row (n2 = hq, col), K = n1
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) v[n1] = slot[(16 * n1 + hq) * TC_COLS + col];
      put_row(Ahi, Alo, tid, v);
      if (!run_stage(Ahi, Alo, Bs, Bs + B_FLOATS, tmem, &mma_bar, phase, &ok_flag, v)) { failed = true; break; }
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw[(hq * k1) & 255]);
      // stage B: rows (k1, col), K = n2
      put_col(Ahi, Alo, col, hq, v);
      if (!run_stage(Ahi, Alo, Bs, Bs + B_FLOATS, tmem, &mma_bar, phase, &ok_flag, v)) { failed = true; break; }
      // thread (k1 = hq, col) holds X^[k1 + 16 k2]
      if (mul) {
        const Sym<float>& sy = a.sym;
        float p2in = 0.f;
        if (sy.ndim == 3) p2in = p2_axis(sy, 2, int(gcol % sy.n[2])) + p2_axis(sy, 1, int(gcol / sy.n[2]));
        else if (sy.ndim == 2) p2in = p2_axis(sy, 1, int(gcol));
        const float b1 = sy.b_re + 1.f;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          float dr, di;
          if (sy.table) {   // tabulated symbol
            const float2 l = sy.table[kspace_index(sy, hq + 16 * k2, gcol, false)];
            dr = l.x + 1.f;
            di = l.y;
          } else {
            const float p2 = p2in + p2_axis(sy, 0, hq + 16 * k2);
            dr = fmaf(sy.a_re, p2, b1);
            di = fmaf(sy.a_im, p2, sy.b_im);
          }
          const float sc = __fdividef(sy.inv_n, fmaf(dr, dr, di * di));
          v[k2] = cmul(v[k2], make_float2(dr * sc, -di * sc));
        }
      }
    } else {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) v[k2] = slot[(hq + 16 * k2) * TC_COLS + col];
    }
    if (inv) {
      // stage B^-1: row (k1 = hq, col), K = k2
      put_row(Ahi, Alo, tid, v);
      if (!run_stage(Ahi, Alo, Bs + 2 * B_FLOATS, Bs + 3 * B_FLOATS, tmem, &mma_bar, phase, &ok_flag, v)) {
        failed = true;
        break;
      }
#pragma unroll
      for (int n2 = 0; n2 < 16; ++n2) v[n2] = cmulc(v[n2], tw[(hq * n2) & 255]);
      // stage A^-1: rows (n2, col), K = k1
      put_col(Ahi, Alo, col, hq, v);
      if (!run_stage(Ahi, Alo, Bs + 2 * B_FLOATS, Bs + 3 * B_FLOATS, tmem, &mma_bar, phase, &ok_flag, v)) {
        failed = true;
        break;
      }
      // thread (n2 = hq, col) holds x[16 n1 + n2]
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) slot[(16 * n1 + hq) * TC_COLS + col] = v[n1];
    } else {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) slot[(hq + 16 * k2) * TC_COLS + col] = v[k2];
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_3d(&map, int((t % a.inner_blocks) * TC_COLS), 0, int(t / a.inner_blocks), slot);
      bulk_commit();
      if (issued < my) {
        bulk_wait_read<1>();
        const int s2 = int(issued % TC_SLOTS);
        const int64_t t2 = t0 + issued * stride;
        mbar_arrive_expect_tx(&full[s2], TC_TILE_BYTES);
        tma_load_3d(slots + s2 * TC_TILE, &map, int((t2 % a.inner_blocks) * TC_COLS), 0,
                    int(t2 / a.inner_blocks), &full[s2]);
        ++issued;
      }
    }
  }
  if (tid == 0) {
    bulk_wait<0>();
    if (failed) {
      // let the loads still in flight land before the shared memory goes
      for (int64_t j = k; j < issued; ++j) mbar_wait(&full[j % TC_SLOTS], uint32_t((j / TC_SLOTS) & 1));
      a.st->status = ST_TIMEOUT;
      a.st->done = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

size_t tc_smem() {
  return sizeof(float2) * TC_SLOTS * TC_TILE + sizeof(float) * (2 * OP_FLOATS + 4 * B_FLOATS) +
         sizeof(float2) * TC_N;
}

}  // namespace

cudaError_t tc_cols_init() {
  // DFT-16 in real form: output n' (re for n' < 16, im above), input k (re
  // for k < 16, im above); M[k][n] = exp(-+ 2 pi i k n / 16)
  static float h[4 * B_FLOATS];
  const double two_pi = 6.283185307179586476925286766559;
  for (int dir = 0; dir < 2; ++dir)
    for (int np = 0; np < 32; ++np)
      for (int k = 0; k < 32; ++k) {
        const int n = np & 15, kk = k & 15;
        const int e = (kk * n) & 15;
        const double c = std::cos(two_pi * e / 16.0);
        const double sn = (dir == 0 ? -1.0 : 1.0) * std::sin(two_pi * e / 16.0);  // Im M
        double val;
        if (np < 16) val = k < 16 ? c : -sn;    // Re d = Re a Re M - Im a Im M
        else val = k < 16 ? sn : c;             // Im d = Re a Im M + Im a Re M
        // exact zeros and ones stay exact
        if (std::fabs(val) < 1e-15) val = 0.0;
        uint32_t bits;
        float hi = (float)val;
        std::memcpy(&bits, &hi, 4);
        bits = (bits + 0x1000u) & 0xFFFFE000u;   // round to TF32 (nearest, ties away)
        std::memcpy(&hi, &bits, 4);
        float lo = (float)(val - (double)hi);
        std::memcpy(&bits, &lo, 4);
        bits = (bits + 0x1000u) & 0xFFFFE000u;
        std::memcpy(&lo, &bits, 4);
        h[(2 * dir) * B_FLOATS + cofs(np, k)] = hi;
        h[(2 * dir + 1) * B_FLOATS + cofs(np, k)] = lo;
      }
  cudaError_t e = cudaMemcpyToSymbol(g_tc_b, h, sizeof(h));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cols_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem());
}

cudaError_t launch_cols_tc(const CUtensorMap& map, const ColsTmaArgs& a, int grid, cudaStream_t s) {
  k_cols_tc<<<grid, TC_THREADS, tc_smem(), s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace usp
