// tma_kernels.cu -- FFT passes along a strided axis with TMA-staged tiles.
//
// A tile is COLS (32, 16 or 8) consecutive columns x the whole axis (N
// values each), i.e. a box {COLS, N, 1} of the field viewed as
// [outer][N][inner].  32 / COLS persistent CTAs of COLS x G threads share an
// SM (while one waits at a barrier, the others compute); each walks its
// tiles through a ring of three shared
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
#include "iteration_state.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace usp {

namespace {

constexpr int SLOTS = 3;

// The exchange row of (k1, n2) is k1 N2 + (n2 ^ (k1 mod N2)): the warps'
// reads (fixed n2, consecutive k1) then alternate between the two bank
// halves of a 64-byte row instead of all landing on one.
template <int N, bool INV, int COLS>
__device__ __forceinline__ void fft_cols_slot(float2* v, float2* ex, const float2* tw, int g,
                                              int lane) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  stage1<N, INV>(v, g, tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) ex[(k1 * N2 + (g ^ (k1 & (N2 - 1)))) * COLS + lane] = v[k1];
  __syncthreads();
  float2 w[N1];
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

__device__ __forceinline__ float2 spectral_factor_f(float p2, const Sym<float>& s, int mul) {
  const float lr = s.a_re * p2 + s.b_re;
  const float li = s.a_im * p2 + s.b_im;
  if (mul == MUL_L) return make_float2(lr * s.inv_n, li * s.inv_n);
  const float dr = lr + 1.f;
  // fast reciprocal division (about 2 ulp); the denominator |Lhat + 1|^2 >= 1
  const float sc = __fdividef(s.inv_n, dr * dr + li * li);
  return make_float2(dr * sc, -li * sc);
}

__device__ __forceinline__ float2 table_factor_f(float2 l, const Sym<float>& s, int mul) {
  if (mul == MUL_L) return make_float2(l.x * s.inv_n, l.y * s.inv_n);
  const float dr = l.x + 1.f;
  const float sc = __fdividef(s.inv_n, dr * dr + l.y * l.y);
  return make_float2(dr * sc, -l.y * sc);
}

__device__ __forceinline__ float axis_p2_f(const Sym<float>& s, int ax, int k) {
  const float p = s.ks[ax] * float(signed_freq(k, s.n[ax]));
  return p * p;
}

}  // namespace

template <int N, int COLS>
__global__ void __launch_bounds__(COLS * Split<N>::G, 32 / COLS)
    k_cols_tma(const __grid_constant__ CUtensorMap map, const ColsTmaArgs a) {
  constexpr int N1 = Split<N>::N1, G = Split<N>::G;
  constexpr int THREADS = COLS * G;
  constexpr int TILE = N * COLS;
  constexpr uint32_t TILE_BYTES = TILE * sizeof(float2);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* slots = reinterpret_cast<float2*>(smem_raw);
  float2* tw = slots + SLOTS * TILE;
  __shared__ __align__(8) uint64_t full[SLOTS];
  __shared__ int ok_flag;

  const bool batched = a.bt.count > 1;
  if (!batched && !(a.flags & F_NOSTATE) && a.st->done) return;

  const int lane = threadIdx.x % COLS, g = threadIdx.x / COLS;
  const int64_t t0 = blockIdx.x, stride = gridDim.x;
  const int64_t my = t0 < a.tiles ? (a.tiles - t0 + stride - 1) / stride : 0;
  for (int m = threadIdx.x; m < N; m += THREADS)
    tw[m] = a.tw[stage1_twiddle_exponent(m, Split<N>::N2) * (256 / N)];
  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // the multiply of the outermost axis: this thread's axis frequencies are
  // the same in every tile, so |p_axis|^2 is evaluated once
  const bool mul = a.mode == COL_FWD_MUL_INV;
  float pz2[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) pz2[q] = mul ? axis_p2_f(a.sym, 0, out_index<N>(g, q)) : 0.f;

  // The CTA walks its tiles k (tile t0 + k stride) in order, skipping the
  // tiles of finished problems of a batch (their done flags do not change
  // during the pass): no loads are issued for them.  j counts the tiles
  // walked, which sets the ring slot and the barrier phase.
  // Tile of walk step kk; with F_REVERSE the walk starts at the last tile
  // (the end of the field, which the pass before this one wrote last and
  // left in L2).
  const bool rev = (a.flags & F_REVERSE) != 0;
  auto tile_of = [&](int64_t kk) { return rev ? a.tiles - 1 - (t0 + kk * stride) : t0 + kk * stride; };
  auto active = [&](int64_t kk) {
    if (!batched || (a.flags & F_NOSTATE)) return true;
    const int64_t tt = tile_of(kk);
    return !a.st[int((tt / a.inner_blocks) / a.bt.outer_per)].done;
  };
  auto next_active = [&](int64_t kk) {
    do ++kk; while (kk < my && !active(kk));
    return kk;
  };
  auto issue = [&](int64_t kk, int64_t jj) {   // thread 0: tile kk into slot jj
    const int sl = int(jj % SLOTS);
    const int64_t tt = tile_of(kk);
    mbar_arrive_expect_tx(&full[sl], TILE_BYTES);
    tma_load_3d(slots + sl * TILE, &map, int((tt % a.inner_blocks) * COLS), 0,
                int(tt / a.inner_blocks), &full[sl]);
  };

  int64_t ik = next_active(-1), ij = 0;   // next tile to load and its walk index (thread 0)
  if (threadIdx.x == 0)
    for (; ij < 2 && ik < my; ++ij, ik = next_active(ik)) issue(ik, ij);

  int64_t k = next_active(-1), j = 0;
  bool failed = false;
  for (; k < my; k = next_active(k), ++j) {
    const int s = int(j % SLOTS);
    if (threadIdx.x == 0) ok_flag = mbar_wait(&full[s], uint32_t((j / SLOTS) & 1)) ? 1 : 0;
    __syncthreads();
    if (!ok_flag) {
      failed = true;
      break;
    }
    float2* slot = slots + s * TILE;
    const int64_t t = tile_of(k);
    const int64_t col = (t % a.inner_blocks) * COLS + lane;
    const int pb = batched ? int((t / a.inner_blocks) / a.bt.outer_per) : 0;
    const Sym<float> sy = problem_sym(a.sym, a.bt, pb);
    const float b1 = sy.b_re + 1.f;
    float2 v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = slot[in_index<N>(g, q) * COLS + lane];
    __syncthreads();  // the slot now serves as the exchange buffer
    if (a.mode == COL_INV) {
      fft_cols_slot<N, true, COLS>(v, slot, tw, g, lane);
    } else {
      fft_cols_slot<N, false, COLS>(v, slot, tw, g, lane);
      if (a.mode == COL_FWD_MUL_INV) {
        // outermost axis: the column index holds the faster axes' frequencies
        float p2in = 0.f;
        if (a.flags & F_CBLOCK) {
          p2in = axis_p2_f(sy, 2, int((col >> 13) * 32 + (col & 31))) +
                 axis_p2_f(sy, 1, int((col >> 5) & 255));
        } else if (sy.ndim == 3) {
          p2in = axis_p2_f(sy, 2, int(col % sy.n[2])) + axis_p2_f(sy, 1, int(col / sy.n[2]));
        } else if (sy.ndim == 2) {
          p2in = axis_p2_f(sy, 1, int(col));
        }
        float2 tmp[N1];
        if (sy.table) {
          // tabulated symbol: one lookup per point
#pragma unroll
          for (int q = 0; q < N1; ++q)
            v[q] = cmul(v[q], table_factor_f(sy.table[kspace_index(sy, out_index<N>(g, q), col,
                                                                   (a.flags & F_CBLOCK) != 0)],
                                             sy, a.mul));
        } else if (a.mul == MUL_LINV && sy.a_re == 0.f) {
          // Helmholtz form: a purely imaginary, so Re(Lhat + 1) = Re b + 1
          const float dr2 = b1 * b1;
#pragma unroll
          for (int q = 0; q < N1; ++q) {
            const float di = fmaf(sy.a_im, p2in + pz2[q], sy.b_im);
            const float sc = __fdividef(sy.inv_n, fmaf(di, di, dr2));
            v[q] = cmul(v[q], make_float2(b1 * sc, -di * sc));
          }
        } else if (a.mul == MUL_LINV && sy.a_im == 0.f && sy.b_im == 0.f) {
          // real symbol (diffusion): a real factor
#pragma unroll
          for (int q = 0; q < N1; ++q) {
            const float sc = __fdividef(sy.inv_n, fmaf(sy.a_re, p2in + pz2[q], b1));
            v[q] = make_float2(v[q].x * sc, v[q].y * sc);
          }
        } else if (a.mul == MUL_LINV) {
          // 1 / (N (Lhat + 1)), Lhat = a |p|^2 + b
#pragma unroll
          for (int q = 0; q < N1; ++q) {
            const float p2 = p2in + pz2[q];
            const float dr = fmaf(sy.a_re, p2, b1);
            const float di = fmaf(sy.a_im, p2, sy.b_im);
            const float sc = __fdividef(sy.inv_n, fmaf(dr, dr, di * di));
            v[q] = cmul(v[q], make_float2(dr * sc, -di * sc));
          }
        } else {
#pragma unroll
          for (int q = 0; q < N1; ++q)
            v[q] = cmul(v[q], spectral_factor_f(p2in + pz2[q], sy, a.mul));
        }
        out_to_in<N>(v, tmp);
#pragma unroll
        for (int q = 0; q < N1; ++q) v[q] = tmp[q];
        fft_cols_slot<N, true, COLS>(v, slot, tw, g, lane);
      }
    }
#pragma unroll
    for (int q = 0; q < N1; ++q) slot[out_index<N>(g, q) * COLS + lane] = v[q];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_store_3d(&map, int((t % a.inner_blocks) * COLS), 0, int(t / a.inner_blocks), slot);
      bulk_commit();
      if (ik < my) {
        // the slot of walk position j+2 held position j-1, whose store was
        // committed one tile ago: wait until at most the newest group reads
        bulk_wait_read<1>();
        issue(ik, ij);
        ++ij;
        ik = next_active(ik);
      }
    }
  }
  if (threadIdx.x == 0) {
    bulk_wait<0>();
    if (failed) {
      // let the loads still in flight land before the CTA's shared memory goes
      for (int64_t p = j; p < ij; ++p) mbar_wait(&full[p % SLOTS], uint32_t((p / SLOTS) & 1));
      for (int q = 0; q < (batched ? a.bt.count : 1); ++q) {
        a.st[q].status = ST_TIMEOUT;
        a.st[q].done = 1;
      }
    }
  }
}

// ---------------------------------------------------------------- rows ---
//
// The fused rows pass of an iteration (inverse FFT x, Delta, update, ||Delta||^2,
// next B x + y, forward FFT x) as a persistent kernel: one 512-thread CTA per
// SM walks tiles of F = 512/G rows with three shared-memory slots of one tile
// each, all filled by bulk copies:
//   U slot: scratch rows; exchange buffer of the inverse transform, after
//           which it is refilled with the next tile's rows;
//   V slot: potential; refilled after the pointwise step;
//   Y slot: source; exchange buffer of the forward transform (after the
//           pointwise step consumed it), refilled at the end of the tile.
// x of the next tile is loaded into registers right after the pointwise
// step, so its latency overlaps the forward transform and the stores.

template <int N, bool INV>
__device__ __forceinline__ void fft_rows_slot(float2* v, float2* exr, const float2* tw, int g) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  stage1<N, INV>(v, g, tw);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) exr[k1 * N2 + (g ^ (k1 & (N2 - 1)))] = v[k1];
  __syncthreads();
  float2 w[N1];
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

// Block shape of the staged rows pass: G line threads per row (Line<N>).
// Lines of 256 points and more: 256 threads (192 for radix-3 lines, so that
// whole rows fill the block), tiles of 8 rows, two CTAs per SM -- measured
// on batches of 2-D problems against one CTA of twice the threads: 512
// points 175 vs 208 us, 384 points 115 vs 131 us, 256 points 56 vs 60 us,
// and the 3-D pencil rows pass at 256^3 124 vs 126 us.  Shorter lines: 512
// threads in one CTA per SM.
template <int N>
struct RowsTma {
  static constexpr bool LONG = N >= 256;
  static constexpr int THREADS = (Line<N>::R == 3 ? 384 : 512) / (LONG ? 2 : 1);
  static constexpr int MINB = LONG ? 2 : 1;
  static constexpr int F = THREADS / Line<N>::G;   // rows per tile
  static_assert(F * Line<N>::G == THREADS, "rows must fill the block");
};

// Line transforms of one row held by G threads, exchange in the row's N
// values of a slot (radix stage over the whole row, M-point transforms on
// the sub-rows).
template <int N>
__device__ __forceinline__ void line_inv_slot(float2* v, float2* exr, const float2* tw,
                                              const float2* rtw, int l) {
  typedef Line<N> L;
  radix_inv<N, 1>(v, exr, rtw, l, 0);
  fft_rows_slot<L::M, true>(v, exr + (l / L::GM) * L::M, tw, l % L::GM);
}
template <int N>
__device__ __forceinline__ void line_fwd_slot(float2* v, float2* exr, const float2* tw,
                                              const float2* rtw, int l) {
  typedef Line<N> L;
  fft_rows_slot<L::M, false>(v, exr + (l / L::GM) * L::M, tw, l % L::GM);
  radix_fwd<N, 1>(v, exr, rtw, l, 0);
}

template <int N>
__global__ void __launch_bounds__(RowsTma<N>::THREADS, RowsTma<N>::MINB) k_rows_tma(const RowsTmaArgs a) {
  typedef Line<N> L;
  constexpr int N1 = L::NV, G = L::G, M = L::M;
  constexpr int THREADS = RowsTma<N>::THREADS;
  constexpr int F = RowsTma<N>::F;      // rows per tile
  constexpr int TILE = F * N;           // complex values per tile
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* SU = reinterpret_cast<float2*>(smem_raw);
  float2* SV = SU + TILE;
  float2* SY = SV + TILE;
  float2* tw = SY + TILE;               // M-point stage-1 twiddles
  float2* rtw = tw + M;                 // W_N^m (radix stage), R > 1
  __shared__ __align__(8) uint64_t bars[3];   // U, V, Y slots
  __shared__ double red[THREADS / 32];
  __shared__ int is_last, ok_flag;

  const bool batched = a.bt.count > 1;
  if (!batched && a.st->done) return;

  const int tid = threadIdx.x, f = tid / G, g = tid % G;
  const bool xzero = (a.flags & F_XZERO) != 0;
  const bool vreal = (a.flags & F_VREAL) != 0;
  const int64_t tiles = (a.nrows + F - 1) / F;
  const int64_t t0 = blockIdx.x, stride = gridDim.x;
  const int64_t my = t0 < tiles ? (tiles - t0 + stride - 1) / stride : 0;
  bool ok = true;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  for (int m = tid; m < M; m += THREADS)
    tw[m] = a.tw[stage1_twiddle_exponent(m, Split<M>::N2) * (256 / M)];
  if (L::R > 1)
    for (int m = tid; m < N; m += THREADS) rtw[m] = a.twx[m * (1536 / N)];
  __syncthreads();

  auto first_row = [&](int64_t k) { return (t0 + k * stride) * F; };
  auto rows_in = [&](int64_t k) -> int64_t {   // valid rows of this CTA's k-th tile
    const int64_t r0 = first_row(k);
    return a.nrows - r0 < F ? a.nrows - r0 : F;
  };
  auto issue = [&](int which, int64_t k) {    // 0: U rows, 1: V, 2: y
    const int64_t off = first_row(k) * N;
    const int64_t n = rows_in(k) * N;
    const bool real = which == 1 && vreal;
    const uint32_t bytes = uint32_t(n * (real ? sizeof(float) : sizeof(float2)));
    const void* src;
    if (which == 0) src = a.buf + off;
    else if (which == 2) src = a.y + off;
    else src = real ? (const void*)(reinterpret_cast<const float*>(a.V) + off)
                    : (const void*)(reinterpret_cast<const float2*>(a.V) + off);
    float2* dst = which == 0 ? SU : (which == 1 ? SV : SY);
    mbar_arrive_expect_tx(&bars[which], bytes);
    bulk_load(dst, src, bytes, &bars[which]);
  };
  auto wait_bar = [&](int i, uint32_t parity) {
    if (tid == 0) ok_flag = mbar_wait(&bars[i], parity) ? 1 : 0;
    __syncthreads();
    ok = ok && ok_flag;
  };
  auto release_then = [&](int which, int64_t k) {   // slot free -> refill for tile k
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && k < my) issue(which, k);
  };

  float2 xr[N1];
  auto prefetch_x = [&](int64_t k) {    // this thread's x at points L::sp_out(g, q)
    const int64_t row = first_row(k) + f;
    const bool act = row < a.nrows && !xzero;
#pragma unroll
    for (int q = 0; q < N1; ++q)
      xr[q] = act ? a.x_in[row * N + L::sp_out(g, q)] : make_float2(0.f, 0.f);
  };

  // The CTA walks its tiles in order, skipping the tiles of finished
  // problems of a batch (their done flags do not change during the pass), so
  // no copies are issued for them; the walk index j sets the barrier phase.
  auto active = [&](int64_t kk) { return !batched || !a.st[int(first_row(kk) / a.bt.rows_per)].done; };
  auto next_active = [&](int64_t kk) {
    do ++kk; while (kk < my && !active(kk));
    return kk;
  };
  const int64_t k_first = next_active(-1);
  if (tid == 0 && k_first < my) {
    issue(0, k_first);
    issue(1, k_first);
    issue(2, k_first);
  }
  if (k_first < my) prefetch_x(k_first);

  float acc = 0.f;
  int64_t j = 0;
  for (int64_t k = k_first; k < my; ++j) {
    const int64_t kn = next_active(k);
    const uint32_t par = uint32_t(j & 1);
    const int64_t row = first_row(k) + f;
    const int pb = batched ? int(first_row(k) / a.bt.rows_per) : 0;
    const bool act = row < a.nrows;
    wait_bar(0, par);
    float2 v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q)
      v[q] = act ? SU[f * N + L::fr_in(g, q)] : make_float2(0.f, 0.f);
    __syncthreads();
    // inverse FFT along x, exchange in the U slot, which is then refilled
    line_inv_slot<N>(v, SU + f * N, tw, rtw, g);
    release_then(0, kn);
    wait_bar(1, par);
    wait_bar(2, par);
    // Delta = (1-V)(u - x); x += alpha Delta; next t = (1-V) x + y
    const float al = batched && a.bt.alpha ? a.bt.alpha[pb] : a.alpha;
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const int c = f * N + L::sp_out(g, q);
      const float2 vv = vreal ? make_float2(reinterpret_cast<const float*>(SV)[c], 0.f) : SV[c];
      const float2 yv = SY[c];
      const float br = 1.f - vv.x, bi = -vv.y;
      const float ur = v[q].x - xr[q].x, ui = v[q].y - xr[q].y;
      const float dr = br * ur - bi * ui, di = br * ui + bi * ur;
      const float2 xn = make_float2(xr[q].x + al * dr, xr[q].y + al * di);
      if (act) {
        acc += dr * dr + di * di;
        a.x_out[row * N + L::sp_out(g, q)] = xn;
      }
      v[q] = make_float2(yv.x + br * xn.x - bi * xn.y, yv.y + br * xn.y + bi * xn.x);
    }
    release_then(1, kn);
    if (kn < my) prefetch_x(kn);
    // forward FFT along x, exchange in the Y slot (consumed), which is then
    // refilled; the output index set equals the input set, so the registers
    // are reordered once into the stage-1 order
    float2 t[N1];
    out_to_in<M>(v, t);
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = t[q];
    line_fwd_slot<N>(v, SY + f * N, tw, rtw, g);
    if (act) {
#pragma unroll
      for (int q = 0; q < N1; ++q) a.buf[row * N + L::fr_out(g, q)] = v[q];
    }
    release_then(2, kn);
    if (batched) {
      // per-tile partial of ||Delta||^2 (the problems are finalised once, at
      // the end of the kernel)
      double dv = (double)acc;
      acc = 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dv += __shfl_down_sync(0xffffffffu, dv, o);
      if ((tid & 31) == 0) red[tid >> 5] = dv;
      __syncthreads();
      if (tid == 0) {
        double bs = 0.0;
        for (int i = 0; i < THREADS / 32; ++i) bs += red[i];
        a.partials[t0 + k * stride] = bs;
      }
      __syncthreads();
    }
    k = kn;
  }

  if (!ok && tid == 0) {
    for (int q = 0; q < (batched ? a.bt.count : 1); ++q) {
      a.st[q].status = ST_TIMEOUT;
      a.st[q].done = 1;
    }
  }
  if (batched) {
    // The last CTA to finish sums each running problem's tile partials in
    // tile order (deterministic), one thread per problem, and updates its
    // state; one grid-wide ticket (problem 0's) per launch.
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      is_last = atomicAdd(&a.st[0].ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const int64_t tpp = a.bt.rows_per / F;
    for (int pb = tid; pb < a.bt.count; pb += THREADS) {   // one thread per problem
      if (__ldcg(&a.st[pb].done)) continue;   // its tiles were skipped
      double sm = 0.0;
      for (int64_t i = 0; i < tpp; ++i) sm += __ldcg(a.partials + pb * tpp + i);
      if (a.st[pb].status != ST_TIMEOUT)
        finalize_iteration(a.st + pb, a.hist + (int64_t)pb * a.bt.hist_stride, sm, a.flags);
    }
    __syncthreads();
    if (tid == 0) a.st[0].ticket = 0u;
    return;
  }
  // ||Delta||^2: block partial, the last block finalises (fixed order)
  double dv = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dv += __shfl_down_sync(0xffffffffu, dv, o);
  if ((tid & 31) == 0) red[tid >> 5] = dv;
  __syncthreads();
  if (tid == 0) {
    double bs = 0.0;
    for (int i = 0; i < THREADS / 32; ++i) bs += red[i];
    a.partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned tk = atomicAdd(&a.st->ticket, 1u);
    is_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double sm = 0.0;
    for (unsigned i = tid; i < gridDim.x; i += THREADS) sm += __ldcg(a.partials + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sm += __shfl_down_sync(0xffffffffu, sm, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = sm;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < THREADS / 32; ++i) tot += red[i];
      if (a.st->status != ST_TIMEOUT) finalize_iteration(a.st, a.hist, tot, a.flags);
      a.st->ticket = 0u;
    }
  }
}

template <int N>
static size_t rows_tma_smem() {
  return sizeof(float2) * (3 * RowsTma<N>::F * N + Line<N>::M + (Line<N>::R > 1 ? N : 0));
}

template <int N>
static cudaError_t rows_tma_go(const RowsTmaArgs& a, int grid, cudaStream_t s) {
  k_rows_tma<N><<<grid, RowsTma<N>::THREADS, rows_tma_smem<N>(), s>>>(a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t rows_tma_attr() {
  return cudaFuncSetAttribute(k_rows_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rows_tma_smem<N>());
}

cudaError_t rows_tma_init() {
  cudaError_t e;
  if ((e = rows_tma_attr<96>()) != cudaSuccess) return e;
  if ((e = rows_tma_attr<128>()) != cudaSuccess) return e;
  if ((e = rows_tma_attr<192>()) != cudaSuccess) return e;
  if ((e = rows_tma_attr<256>()) != cudaSuccess) return e;
  if ((e = rows_tma_attr<384>()) != cudaSuccess) return e;
  return rows_tma_attr<512>();
}

int rows_tma_ctas_per_sm(int n) {
  switch (n) {
    case 128: return RowsTma<128>::MINB;
    case 256: return RowsTma<256>::MINB;
    case 384: return RowsTma<384>::MINB;
    case 512: return RowsTma<512>::MINB;
    default: return 1;
  }
}

int rows_tma_tile_rows(int n) {
  // 96 and 192: the plain line pass is faster (tiles of 16-32 short rows
  // leave too little work between the slot hand-offs)
  switch (n) {
    case 128: return RowsTma<128>::F;
    case 256: return RowsTma<256>::F;
    case 384: return RowsTma<384>::F;
    case 512: return RowsTma<512>::F;
    default: return 0;
  }
}

cudaError_t launch_rows_tma(int n, const RowsTmaArgs& a, int grid, cudaStream_t s) {
  switch (n) {
    case 96: return rows_tma_go<96>(a, grid, s);
    case 128: return rows_tma_go<128>(a, grid, s);
    case 192: return rows_tma_go<192>(a, grid, s);
    case 256: return rows_tma_go<256>(a, grid, s);
    case 384: return rows_tma_go<384>(a, grid, s);
    case 512: return rows_tma_go<512>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, int COLS>
static size_t cols_tma_smem() {
  return sizeof(float2) * (SLOTS * N * COLS + N);
}

template <int N, int COLS>
static cudaError_t cols_tma_go(const CUtensorMap& map, const ColsTmaArgs& a, int grid,
                               cudaStream_t s) {
  k_cols_tma<N, COLS><<<grid, COLS * Split<N>::G, cols_tma_smem<N, COLS>(), s>>>(map, a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t cols_tma_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_cols_tma<N, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cols_tma_smem<N, 32>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cols_tma<N, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cols_tma_smem<N, 16>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cols_tma<N, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cols_tma_smem<N, 8>());
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

cudaError_t launch_cols_tma(int n, int cols, const CUtensorMap& map, const ColsTmaArgs& a,
                            int grid, cudaStream_t s) {
#define C_(N)                                                        \
  (cols == 8 ? cols_tma_go<N, 8>(map, a, grid, s)                     \
             : (cols == 16 ? cols_tma_go<N, 16>(map, a, grid, s) : cols_tma_go<N, 32>(map, a, grid, s)))
  if (cols != 8 && cols != 16 && cols != 32) return cudaErrorInvalidValue;
  switch (n) {
    case 2: return C_(2);
    case 4: return C_(4);
    case 8: return C_(8);
    case 16: return C_(16);
    case 32: return C_(32);
    case 64: return C_(64);
    case 128: return C_(128);
    case 256: return C_(256);
    default: return cudaErrorInvalidValue;
  }
#undef C_
}

}  // namespace usp
