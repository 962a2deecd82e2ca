// split3d_kernels.cu -- the split-y two-pass schedule of one fixed-point
// iteration (Algorithm 1 with the forward-eliminated operator of Sec. 2.1;
// (L+I)^-1 = F^-1 diag(1/(Lhat+1)) F, Eq. laplacian_inverse) for grids
// nz x 256 x 256, nz a power of two in [32, 256].
//
// The y transform (length 256) is split as y = 16 y1 + y2, k = k1 + 16 k2:
//   Y[k1 + 16 k2] = sum_y2 W_16^(y2 k2) [ W_256^(y2 k1) sum_y1 t[16 y1 + y2] W_16^(y1 k1) ].
// The inner 16-point transform over y1 needs only the 16 rows {16 y1 + y2}
// of one plane, so the rows pass does it beside the x transform; the outer
// 16-point transform over y2 joins the z transform in the column pass.
// Neither pass needs a whole plane on chip, and no CTA waits for another:
//
//   rows pass (tile = plane z and residue y2: 16 rows of 256 values):
//       inverse y1 stage, inverse FFT x, Delta = (1-V)(u - x), x += alpha Delta,
//       ||Delta||^2, t = (1-V) x + y, FFT x, forward y1 stage
//   column pass (tile = k1 and 2 consecutive kx, over all y2 and z):
//       y2 stage, FFT z, x 1/(N (Lhat + 1)), inverse FFT z, inverse y2 stage
//
// Algorithmic HBM bytes per point and iteration: rows 48 (read scratch, x, V,
// y; write x, scratch; 44 with a real V) + columns 16 = 64, against 96 for the
// pencil schedule.
//
// Scratch layout (complex64), chosen so that a column tile lies inside one
// k1 slab:
//   S[k1][z][y2][kx]  (a k1 slab is nz x 16 rows of 256 values, 8 MB at
//                      nz = 256).
// The rows pass reads its tile (z, y2) as 16 bulk copies of 2 KB rows, one
// per k1, and writes it back with coalesced 2 KB stores; the column pass
// gathers its tile (k1, two kx, all y2 and z) with one 4-D tensor load of
// 16-byte pieces and scatters it back with one tensor store.  The pieces of
// one column tile then span one 8 MB slab (a few address-translation pages)
// instead of the whole 128 MB field, and the tiles in flight at one time
// (consecutive xb of one or two k1) share their slabs.  The tensor map lists
// z before y2, so the tile arrives in shared memory as [y2][z][xi]: a warp's
// 16 z x 2 xi of one y2 are 256 consecutive bytes.
//
// Both kernels are persistent and stage their tiles with the copy engine;
// every wait is bounded and a wait that gives up marks the solve ST_TIMEOUT
// after the copies in flight have landed.
#include "fft_core.cuh"
#include "iteration_state.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace usp {

namespace {

constexpr int SP_N = 256;           // nx = ny
constexpr int SP_R1 = 16;           // y1 points (rows pass)
constexpr int SP_R2 = 16;           // y2 points (column pass)
constexpr int SP_XB = 2;            // kx per column tile
constexpr int SP_NXB = SP_N / SP_XB;
constexpr int SP_ROW = SP_R2 * SP_XB;   // values per z of a column tile
constexpr int SA_THREADS = 256;         // 16 rows x 16 line threads = 256 kx
constexpr int SA_TILE = SP_R1 * SP_N;   // values per rows tile
constexpr uint32_t SA_TILE_BYTES = SA_TILE * sizeof(float2);
constexpr int SC_TILES = SP_R1 * SP_NXB;   // column tiles (k1, xb)

// 4-D tiled TMA load global -> shared, completing on an mbarrier.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// 4-D tiled TMA store shared -> global (this thread's bulk async-group).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                             const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
      : "memory");
}

// The N-point transform of one line held by the G = Split<N>::G threads g of
// one warp (a row of the rows pass, a column of the column pass), exchanging
// through the line's own N values in shared memory: exchange row k1 holds
// position n2 at k1 N2 + (n2 ^ (k1 mod N2)).  The line's threads share a
// warp, so a warp barrier orders the exchange; the caller's warp must not
// touch another warp's line between its own last access and this call.
template <int N, bool INV>
__device__ __forceinline__ void fft_line(float2* v, float2* exl, const float2* tws, int g) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, G = Split<N>::G, S = Split<N>::S;
  stage1<N, INV>(v, g, tws);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) exl[k1 * N2 + (g ^ (k1 & (N2 - 1)))] = v[k1];
  __syncwarp();
  float2 w[N1];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k1 = g + G * s;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) w[s * N2 + n2] = exl[k1 * N2 + (n2 ^ (k1 & (N2 - 1)))];
  }
  __syncwarp();
  stage2<N, INV>(w);
#pragma unroll
  for (int q = 0; q < N1; ++q) v[q] = w[q];
}

__device__ __forceinline__ float axis_p2(const Sym<float>& s, int ax, int k) {
  const float p = s.ks[ax] * float(signed_freq(k, s.n[ax]));
  return p * p;
}

// Stage-1 twiddle table of the M-point transform from the W_256^e table.
template <int M>
__device__ __forceinline__ void load_stage1_twiddles(float2* dst, const float2* w256) {
  for (int m = threadIdx.x; m < M; m += blockDim.x)
    dst[m] = w256[stage1_twiddle_exponent(m, Split<M>::N2) * (256 / M)];
}

}  // namespace

// ------------------------------------------------------------ rows pass ---
//
// Two 256-thread CTAs per SM walk tiles u = (z, y2) (u = 16 z + y2), each
// with three 32 KB shared-memory slots:
//   SU: the tile's scratch values [k1][kx] (16 bulk copies); exchange of the
//       inverse transforms, then refilled with the next tile's values;
//   SV: V rows [y1][x] (16 bulk copies); refilled once the pointwise step
//       has read it;
//   SY: y rows [y1][x] (16 bulk copies); exchange of the forward transforms,
//       refilled once the forward y1 stage has read it.
// Each slot is issued exactly once per tile, behind a block barrier that
// follows its last read; x of the next tile is loaded into registers right
// after the pointwise step, so its latency overlaps the forward transforms.
// Thread roles: rows (f = tid / 16 is the row y1, g = tid % 16 its line
// thread) for the x transform and the pointwise step; columns (kx = tid) for
// the y1 stage, a 16-point transform in registers.
template <int MODE>
__global__ void __launch_bounds__(SA_THREADS, 2)
    k_split_rows(const SplitArgs a) {
  constexpr bool POST = MODE != SPLIT_PRE;   // the tile starts from the scratch (inverse part)
  constexpr bool PRE = MODE != SPLIT_POST;   // the tile ends with t = B x + y and its transform
  constexpr bool FULL = POST && PRE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* SU = reinterpret_cast<float2*>(smem_raw);
  float2* SV = SU + SA_TILE;
  float2* SY = SV + SA_TILE;
  float2* w256 = SY + SA_TILE;     // W_256^e
  float2* tws = w256 + SP_N;       // stage-1 twiddles of the 256-point row transform
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ double red[SA_THREADS / 32];
  __shared__ int is_last, ok_flag;

  if (a.st->done) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const int f = tid >> 4, g = tid & 15;     // row roles
  const int kx = tid;                       // column role
  const bool xzero = (a.flags & F_XZERO) != 0;
  const bool vreal = (a.flags & F_VREAL) != 0;
  const bool ref = (a.flags & F_REF) != 0;
  const bool need_x = !xzero;
  const int64_t tiles = (int64_t)a.nz * SP_R2;
  const int64_t t0 = blockIdx.x, stride = gridDim.x;
  const int64_t my = t0 < tiles ? (tiles - t0 + stride - 1) / stride : 0;
  bool ok = true;
  // thread 0 counts, per slot, the loads issued and the phases it saw
  // complete, so that a failed wait can let the copies in flight land
  int64_t n_issued[3] = {0, 0, 0}, n_waited[3] = {0, 0, 0};

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  for (int m = tid; m < SP_N; m += SA_THREADS) w256[m] = a.tw[m];
  load_stage1_twiddles<256>(tws, a.tw);
  __syncthreads();

  auto tile_of = [&](int64_t k) { return t0 + k * stride; };
  // global row (z * 256 + y) of row y1 of tile u
  auto row_of = [&](int64_t u, int y1) { return (u >> 4) * SP_N + SP_R2 * y1 + (u & 15); };
  // warp 0: issue the copies of slot `which` for the k-th tile (lanes < 16
  // each copy one row of V or y)
  auto issue = [&](int which, int64_t k) {
    const int64_t u = tile_of(k);
    if (lane == 0) ++n_issued[which];
    if (which == 0) {
      // the tile's 16 k1 rows, one k1 slab apart
      if (lane == 0) mbar_arrive_expect_tx(&bars[0], SA_TILE_BYTES);
      __syncwarp();
      if (lane < SP_R1)
        bulk_load(SU + lane * SP_N, a.buf + (lane * tiles + u) * SP_N, SP_N * 8u, &bars[0]);
      return;
    }
    const bool real = which == 1 && vreal;
    const uint32_t rb = real ? SP_N * 4u : SP_N * 8u;
    // rows of y that are all zero are not copied (the pointwise step reads
    // them as zeros)
    const uint32_t rows = which == 2 && a.ymask ? a.ymask[u] & 0xFFFFu : 0xFFFFu;
    if (lane == 0) mbar_arrive_expect_tx(&bars[which], __popc(rows) * rb);
    __syncwarp();
    if (lane < SP_R1 && ((rows >> lane) & 1u)) {
      const int64_t r = row_of(u, lane);
      const char* src = which == 1 ? reinterpret_cast<const char*>(a.V) + r * rb
                                   : reinterpret_cast<const char*>(a.y + r * SP_N);
      char* dst = reinterpret_cast<char*>(which == 1 ? SV : SY) + lane * rb;
      bulk_load(dst, src, rb, &bars[which]);
    }
  };
  auto wait_bar = [&](int i, uint32_t parity) {
    if (tid == 0) {
      ok_flag = mbar_wait(&bars[i], parity) ? 1 : 0;
      n_waited[i] += ok_flag;
    }
    __syncthreads();
    ok = ok && ok_flag;
  };
  // the V slot, and with last == 2 the y slot too, behind one block barrier
  auto wait_bars = [&](int last, uint32_t parity) {
    if (tid == 0) {
      int good = 1;
      for (int i = 1; i <= last && good; ++i) {
        good = mbar_wait(&bars[i], parity) ? 1 : 0;
        n_waited[i] += good;
      }
      ok_flag = good;
    }
    __syncthreads();
    ok = ok && ok_flag;
  };
  auto release_then = [&](int which, int64_t k) {   // slot free -> refill for tile k
    fence_proxy_async_smem();
    __syncthreads();
    if (tid < 32 && k < my) issue(which, k);
  };
  float2 xr[16];
  auto prefetch_x = [&](int64_t k) {   // this thread's x at points g + 16 q of its row
    const int64_t row = row_of(tile_of(k), f);
#pragma unroll
    for (int q = 0; q < 16; ++q)
      xr[q] = need_x ? a.x_in[row * SP_N + g + 16 * q] : make_float2(0.f, 0.f);
  };

  if (tid < 32 && my > 0) {
    if (POST) issue(0, 0);
    issue(1, 0);
    if (PRE) issue(2, 0);
  }
  if (my > 0) prefetch_x(0);

  float acc = 0.f;
  for (int64_t k = 0; k < my && ok; ++k) {
    const uint32_t par = uint32_t(k & 1);
    const int64_t u = tile_of(k);
    const int y2 = int(u & 15);
    const int64_t row = row_of(u, f);
    // this thread's row of y was copied (else it is zero)
    const bool yrow = !a.ymask || ((a.ymask[u] >> f) & 1u);
    float2 v[16];
    if (POST) {
      wait_bar(0, par);
      if (!ok) break;
      // inverse y1 stage: undo W_256^(y2 k1), inverse 16-point DFT over k1
      float2 c[16];
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) c[k1] = cmulc(SU[k1 * SP_N + kx], w256[(y2 * k1) & 255]);
      DFT<16, true, float2>::run(c);   // rows y1
      __syncthreads();                 // SU read by all
#pragma unroll
      for (int i = 0; i < 16; ++i) SU[i * SP_N + kx] = c[i];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = SU[f * SP_N + 16 * q + g];
      __syncwarp();   // row f (this warp's) is read before its exchange reuses it
      fft_line<256, true>(v, SU + f * SP_N, tws, g);   // u at x = g + 16 q
      if (FULL) {
        // the next scratch tile goes into SU behind the barrier of the V and
        // y waits (every warp has finished its inverse transform by then)
        fence_proxy_async_smem();
        wait_bars(2, par);
        if (tid < 32 && k + 1 < my) issue(0, k + 1);
      } else {
        release_then(0, k + 1);
        wait_bars(1, par);
      }
      if (!ok) break;
      // Delta = (1-V)(u - x); x += alpha Delta; next t = (1-V) x + y
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int cidx = f * SP_N + g + 16 * q;
        const float2 vv = vreal ? make_float2(reinterpret_cast<const float*>(SV)[cidx], 0.f) : SV[cidx];
        const float br = 1.f - vv.x, bi = -vv.y;
        const float ur = v[q].x - xr[q].x, ui = v[q].y - xr[q].y;
        const float dr = br * ur - bi * ui, di = br * ui + bi * ur;
        acc += dr * dr + di * di;
        const float2 xn = make_float2(xr[q].x + a.alpha * dr, xr[q].y + a.alpha * di);
        if (!ref) a.x_out[row * SP_N + g + 16 * q] = xn;
        if (PRE) {
          const float2 yv = yrow ? SY[cidx] : make_float2(0.f, 0.f);
          v[q] = make_float2(yv.x + br * xn.x - bi * xn.y, yv.y + br * xn.y + bi * xn.x);
        }
      }
      // FULL: the next V tile is issued behind the barrier that follows the
      // forward x transform (SV is read only above)
      if (!FULL) release_then(1, k + 1);
      if (k + 1 < my) prefetch_x(k + 1);
    } else {
      wait_bars(2, par);
      if (!ok) break;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int cidx = f * SP_N + g + 16 * q;
        const float2 vv = vreal ? make_float2(reinterpret_cast<const float*>(SV)[cidx], 0.f) : SV[cidx];
        const float br = 1.f - vv.x, bi = -vv.y;
        const float2 yv = yrow ? SY[cidx] : make_float2(0.f, 0.f);
        v[q] = make_float2(yv.x + br * xr[q].x - bi * xr[q].y, yv.y + br * xr[q].y + bi * xr[q].x);
      }
      release_then(1, k + 1);
      if (k + 1 < my) prefetch_x(k + 1);
    }
    if (PRE) {
      // forward FFT x (positions g + 16 q in -> frequencies g + 16 q out)
      float2 tmp[16];
      out_to_in<256>(v, tmp);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = tmp[q];
      fft_line<256, false>(v, SY + f * SP_N, tws, g);
#pragma unroll
      for (int q = 0; q < 16; ++q) SY[f * SP_N + g + 16 * q] = v[q];
      fence_proxy_async_smem();
      __syncthreads();
      if (FULL && tid < 32 && k + 1 < my) issue(1, k + 1);
      // forward y1 stage: 16-point DFT over the rows, then W_256^(y2 k1)
      float2 c[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) c[i] = SY[i * SP_N + kx];
      release_then(2, k + 1);
      DFT<16, false, float2>::run(c);
      float2* dst = a.buf + u * SP_N + kx;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) dst[k1 * tiles * SP_N] = cmul(c[k1], w256[(y2 * k1) & 255]);
    }
  }

  if (!ok && tid == 0) {
    // let the copies still in flight land before the CTA's shared memory goes
    for (int i = 0; i < 3; ++i)
      for (int64_t p = n_waited[i]; p < n_issued[i]; ++p) mbar_wait(&bars[i], uint32_t(p & 1));
    a.st->status = ST_TIMEOUT;
    a.st->done = 1;
  }
  // ||Delta||^2: block partial, the last block finalises (fixed order)
  if (!POST) return;
  double dv = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dv += __shfl_down_sync(0xffffffffu, dv, o);
  if (lane == 0) red[tid >> 5] = dv;
  __syncthreads();
  if (tid == 0) {
    double bs = 0.0;
    for (int i = 0; i < SA_THREADS / 32; ++i) bs += red[i];
    a.partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned tk = atomicAdd(&a.st->ticket, 1u);
    is_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double sm = 0.0;
    for (unsigned i = tid; i < gridDim.x; i += SA_THREADS) sm += __ldcg(a.partials + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sm += __shfl_down_sync(0xffffffffu, sm, o);
    __syncthreads();
    if (lane == 0) red[tid >> 5] = sm;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < SA_THREADS / 32; ++i) tot += red[i];
      if (a.st->status != ST_TIMEOUT) finalize_iteration(a.st, a.hist, tot, a.flags);
      a.st->ticket = 0u;
    }
  }
}

// ---------------------------------------------------------- column pass ---
//
// Tiles (k1, xb): the values S[k1][z][y2][2 xb + xi] of all z and y2, moved
// by 4-D tensor copies (16-byte pieces) through a ring of three slots (two
// loads in flight while one tile is transformed in its slot); in a slot the
// tile is laid out [y2][z][xi].  In the slot, thread
// roles change twice: (z, xi) pairs for the 16-point y2 stage, then columns
// c = 2 k2 + xi, each held by the G threads of one warp, for the z
// transform.  The values move between the two through the slot itself,
// column-major: column c at c nz, position z ^ (8 (c & 1)) (the XOR puts
// the even and odd columns of one y2-stage store on different banks).  The
// z transform's exchange then stays inside each column, so only the two
// transposes need block barriers.
template <int NZ>
struct SplitCols {
  static constexpr int G = Split<NZ>::G, N1 = Split<NZ>::N1;
  static constexpr int THREADS = 32 * G;
  static constexpr int MINB = 512 / THREADS;
  static constexpr int TILE = NZ * SP_ROW;
  static constexpr uint32_t TILE_BYTES = TILE * sizeof(float2);
  // (z, xi) pairs per thread in the y2 stage (threads beyond the pairs idle)
  static constexpr int PAIRS = (NZ * SP_XB + THREADS - 1) / THREADS;
  static constexpr int ZSTEP = THREADS / SP_XB;
  static constexpr int SLOTS = 3;
  static_assert(NZ >= 16, "column swizzle needs 16-value blocks");
};

// Position of z in column c of the column-major view of a slot.
template <int NZ>
__device__ __forceinline__ int colpos(int c, int z) {
  return c * NZ + (z ^ (8 * (c & 1)));
}

// Position in column c of register q of line thread g (input order with IN,
// else output order).  For NZ = 256 both orders are g + 16 q, and the XOR
// touches only g, so the position is a per-thread base plus a constant.
template <int NZ, bool IN>
__device__ __forceinline__ int zpos(int cbase, int c, int g, int q) {
  if (Split<NZ>::N2 >= 16 && Split<NZ>::S == 1) return cbase + 16 * q;
  return colpos<NZ>(c, IN ? in_index<NZ>(g, q) : out_index<NZ>(g, q));
}

// x 1/(N (Lhat + 1)) on the spectrum of one z column (frequencies kxx,
// ky; this thread's kz = out_index(g, q)), then the registers reordered for
// the inverse transform.  Specialised for the Helmholtz form (a purely
// imaginary: Re(Lhat + 1) constant) and real symbols (diffusion).
template <int NZ>
__device__ __forceinline__ void spectral_multiply(float2* v, const Sym<float>& sy, const float* pz2,
                                                  float b1, int g, int kxx, int ky) {
  constexpr int N1 = Split<NZ>::N1;
  const float p2in = axis_p2(sy, 2, kxx) + axis_p2(sy, 1, ky);
  if (sy.table) {
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const float2 l = sy.table[((int64_t)out_index<NZ>(g, q) * SP_N + ky) * SP_N + kxx];
      const float dr = l.x + 1.f;
      const float sc = __fdividef(sy.inv_n, fmaf(dr, dr, l.y * l.y));
      v[q] = cmul(v[q], make_float2(dr * sc, -l.y * sc));
    }
  } else if (sy.a_re == 0.f) {
    // Helmholtz form: a purely imaginary, so Re(Lhat + 1) = Re b + 1
    const float dr2 = b1 * b1;
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const float di = fmaf(sy.a_im, p2in + pz2[q], sy.b_im);
      const float sc = __fdividef(sy.inv_n, fmaf(di, di, dr2));
      v[q] = cmul(v[q], make_float2(b1 * sc, -di * sc));
    }
  } else if (sy.a_im == 0.f && sy.b_im == 0.f) {
    // real symbol (diffusion): a real factor
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const float sc = __fdividef(sy.inv_n, fmaf(sy.a_re, p2in + pz2[q], b1));
      v[q] = make_float2(v[q].x * sc, v[q].y * sc);
    }
  } else {
    // 1 / (N (Lhat + 1)), Lhat = a |p|^2 + b
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const float p2 = p2in + pz2[q];
      const float dr = fmaf(sy.a_re, p2, b1);
      const float di = fmaf(sy.a_im, p2, sy.b_im);
      const float sc = __fdividef(sy.inv_n, fmaf(dr, dr, di * di));
      v[q] = cmul(v[q], make_float2(dr * sc, -di * sc));
    }
  }
  float2 tmp[N1];
  out_to_in<NZ>(v, tmp);
#pragma unroll
  for (int q = 0; q < N1; ++q) v[q] = tmp[q];
}

template <int NZ>
__global__ void __launch_bounds__(SplitCols<NZ>::THREADS, SplitCols<NZ>::MINB)
    k_split_cols(const __grid_constant__ CUtensorMap cmap, const SplitColsArgs a) {
  typedef SplitCols<NZ> C;
  constexpr int N1 = C::N1, TILE = C::TILE, G = C::G;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* slots = reinterpret_cast<float2*>(smem_raw);
  float2* tws = slots + C::SLOTS * TILE;   // stage-1 twiddles of the z transform
  __shared__ __align__(8) uint64_t full[C::SLOTS];
  __shared__ int ok_flag;

  if (a.st->done) return;
  const int tid = threadIdx.x;
  const int c = tid / G, g = tid % G;      // z-transform roles: column c = 2 k2 + xi
  const int xi = tid & 1, zb = tid >> 1;   // y2-stage roles
  // z-transform base of column c (the same in every tile)
  const int cbase = c * NZ + (g ^ (8 * (c & 1)));
  const int64_t t0 = blockIdx.x, stride = gridDim.x;
  const int64_t my = t0 < SC_TILES ? (SC_TILES - t0 + stride - 1) / stride : 0;
  load_stage1_twiddles<NZ>(tws, a.tw);
  if (tid == 0) {
    for (int s = 0; s < C::SLOTS; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const Sym<float> sy = a.sym;
  const float b1 = sy.b_re + 1.f;
  float pz2[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) pz2[q] = axis_p2(sy, 0, out_index<NZ>(g, q));

  const bool rev = (a.flags & F_REVERSE) != 0;
  auto tile_of = [&](int64_t kk) { return rev ? SC_TILES - 1 - (t0 + kk * stride) : t0 + kk * stride; };
  auto issue = [&](int64_t kk) {   // thread 0: tile kk into slot kk % SLOTS
    const int sl = int(kk % C::SLOTS);
    const int64_t tt = tile_of(kk);
    mbar_arrive_expect_tx(&full[sl], C::TILE_BYTES);
    tma_load_4d(slots + sl * TILE, &cmap, int(SP_XB * (tt % SP_NXB)), 0, 0, int(tt / SP_NXB), &full[sl]);
  };
  int64_t ik = 0;
  if (tid == 0)
    for (; ik < 2 && ik < my; ++ik) issue(ik);

  int64_t k = 0;
  bool failed = false;
  for (; k < my; ++k) {
    const int s = int(k % C::SLOTS);
    if (tid == 0) ok_flag = mbar_wait(&full[s], uint32_t((k / C::SLOTS) & 1)) ? 1 : 0;
    __syncthreads();
    if (!ok_flag) {
      failed = true;
      break;
    }
    float2* T = slots + s * TILE;
    const int64_t t = tile_of(k);
    const int k1 = int(t / SP_NXB), xb = int(t % SP_NXB);

    // forward y2 stage on the (z, xi) pairs
    float2 w[C::PAIRS][SP_R2];
#pragma unroll
    for (int p = 0; p < C::PAIRS; ++p) {
      const int z = zb + p * C::ZSTEP;
      if (z < NZ) {
        const float2* Tz = T + z * SP_XB + xi;
#pragma unroll
        for (int y2 = 0; y2 < SP_R2; ++y2) w[p][y2] = Tz[y2 * NZ * SP_XB];
        DFT<SP_R2, false, float2>::run(w[p]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < C::PAIRS; ++p) {
      const int z = zb + p * C::ZSTEP;
      if (z < NZ) {
        float2* Te = T + colpos<NZ>(xi, z);
#pragma unroll
        for (int k2 = 0; k2 < SP_R2; ++k2) Te[2 * NZ * k2] = w[p][k2];
      }
    }
    __syncthreads();
    // z transform of column c (this warp's lines only from here on)
    float2 v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = T[zpos<NZ, true>(cbase, c, g, q)];
    __syncwarp();
    fft_line<NZ, false>(v, T + c * NZ, tws, g);
    spectral_multiply<NZ>(v, sy, pz2, b1, g, SP_XB * xb + (c & 1), k1 + SP_R1 * (c >> 1));
    fft_line<NZ, true>(v, T + c * NZ, tws, g);
#pragma unroll
    for (int q = 0; q < N1; ++q) T[zpos<NZ, false>(cbase, c, g, q)] = v[q];
    __syncthreads();
    // inverse y2 stage
#pragma unroll
    for (int p = 0; p < C::PAIRS; ++p) {
      const int z = zb + p * C::ZSTEP;
      if (z < NZ) {
        const float2* Te = T + colpos<NZ>(xi, z);
#pragma unroll
        for (int k2 = 0; k2 < SP_R2; ++k2) w[p][k2] = Te[2 * NZ * k2];
        DFT<SP_R2, true, float2>::run(w[p]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < C::PAIRS; ++p) {
      const int z = zb + p * C::ZSTEP;
      if (z < NZ) {
        float2* Tz = T + z * SP_XB + xi;
#pragma unroll
        for (int y2 = 0; y2 < SP_R2; ++y2) Tz[y2 * NZ * SP_XB] = w[p][y2];
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_4d(&cmap, SP_XB * xb, 0, 0, k1, T);
      bulk_commit();
      if (ik < my) {
        // the slot of tile k+2 held tile k-1, whose store was committed one
        // tile ago: wait until at most the newest group still reads
        bulk_wait_read<1>();
        issue(ik);
        ++ik;
      }
    }
  }
  if (tid == 0) {
    bulk_wait<0>();
    if (failed) {
      for (int64_t p = k; p < ik; ++p) mbar_wait(&full[p % C::SLOTS], uint32_t((p / C::SLOTS) & 1));
      a.st->status = ST_TIMEOUT;
      a.st->done = 1;
    }
  }
}

// ------------------------------------------------------ source row mask ---
//
// One warp per row of y (256 values, 2 KB): any value other than zero sets
// bit y1 of its rows tile's word.  NaN compares unequal to zero, so a
// non-finite source is always copied and reaches the iteration's check.
__global__ void __launch_bounds__(256) k_split_ymask(const float4* y, int64_t nrows, uint32_t* mask) {
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const float4* p = y + r * (SP_N / 2);
  bool nz = false;
#pragma unroll
  for (int i = 0; i < SP_N / 2 / 32; ++i) {
    const float4 v = __ldcs(p + lane + 32 * i);
    nz = nz || v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f;
  }
  if (__any_sync(0xffffffffu, nz) && lane == 0) {
    const int64_t z = r / SP_N;
    const int yy = int(r % SP_N);
    atomicOr(mask + z * SP_R2 + (yy % SP_R2), 1u << (yy / SP_R2));
  }
}

// ----------------------------------------------------------- launchers ---

static size_t split_rows_smem() { return sizeof(float2) * (3 * SA_TILE + 2 * SP_N); }
template <int NZ>
static size_t split_cols_smem() {
  return sizeof(float2) * (SplitCols<NZ>::SLOTS * SplitCols<NZ>::TILE + NZ);
}

template <int NZ>
static cudaError_t split_cols_attr() {
  return cudaFuncSetAttribute(k_split_cols<NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)split_cols_smem<NZ>());
}

cudaError_t split_init() {
  cudaError_t e;
  const int sm = (int)split_rows_smem();
  if ((e = cudaFuncSetAttribute(k_split_rows<SPLIT_PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_split_rows<SPLIT_FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_split_rows<SPLIT_POST>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
  if ((e = split_cols_attr<32>()) != cudaSuccess) return e;
  if ((e = split_cols_attr<64>()) != cudaSuccess) return e;
  if ((e = split_cols_attr<128>()) != cudaSuccess) return e;
  return split_cols_attr<256>();
}

bool split_nz_ok(int nz) { return nz == 32 || nz == 64 || nz == 128 || nz == 256; }

int split_cols_ctas_per_sm(int nz) {
  switch (nz) {
    case 32: return SplitCols<32>::MINB;
    case 64: return SplitCols<64>::MINB;
    case 128: return SplitCols<128>::MINB;
    case 256: return SplitCols<256>::MINB;
    default: return 0;
  }
}

cudaError_t launch_split_ymask(const float2* y, int nz, uint32_t* mask, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(mask, 0, sizeof(uint32_t) * (size_t)nz * SP_R2, s);
  if (e != cudaSuccess) return e;
  const int64_t nrows = (int64_t)nz * SP_N;
  k_split_ymask<<<(unsigned)((nrows + 7) / 8), 256, 0, s>>>(reinterpret_cast<const float4*>(y), nrows, mask);
  return cudaGetLastError();
}

cudaError_t launch_split_rows(int mode, const SplitArgs& a, int grid, cudaStream_t s) {
  const size_t sm = split_rows_smem();
  switch (mode) {
    case SPLIT_PRE: k_split_rows<SPLIT_PRE><<<grid, SA_THREADS, sm, s>>>(a); break;
    case SPLIT_FULL: k_split_rows<SPLIT_FULL><<<grid, SA_THREADS, sm, s>>>(a); break;
    case SPLIT_POST: k_split_rows<SPLIT_POST><<<grid, SA_THREADS, sm, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NZ>
static cudaError_t split_cols_go(const CUtensorMap& map, const SplitColsArgs& a, int grid,
                                 cudaStream_t s) {
  k_split_cols<NZ><<<grid, SplitCols<NZ>::THREADS, split_cols_smem<NZ>(), s>>>(map, a);
  return cudaGetLastError();
}

cudaError_t launch_split_cols(int nz, const CUtensorMap& map, const SplitColsArgs& a, int grid,
                              cudaStream_t s) {
  switch (nz) {
    case 32: return split_cols_go<32>(map, a, grid, s);
    case 64: return split_cols_go<64>(map, a, grid, s);
    case 128: return split_cols_go<128>(map, a, grid, s);
    case 256: return split_cols_go<256>(map, a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace usp
