// kernels.h -- internal interface between the solver runtime (usp_api.cpp)
// and the CUDA kernels.  Not part of the public ABI (include/usp.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace usp {

// Device-side iteration state: one per solver.  Written by the last block
// of the kernel that finishes an iteration (the update pass), read by every
// kernel at entry (done != 0: skip all work) and by the host between CUDA
// graph launches.
enum DevStatus : int {
  ST_RUNNING = 0,
  ST_CONVERGED = 1,   // ||Delta||/ref < tol
  ST_MAXIT = 2,       // it reached it_limit
  ST_NONFINITE = 3,   // NaN/Inf norm
  ST_DIVERGED = 4,    // ||Delta|| above 4x its first value in this phase
  ST_STAGNATED = 5,   // no 0.1% improvement over stall_window iterations
  ST_TIMEOUT = 6      // a bounded wait inside a kernel gave up (copy engine)
};

struct DevState {
  int done;           // nonzero: every kernel returns at entry
  int status;         // DevStatus
  int it;             // Delta evaluations completed (all phases)
  int it_limit;       // stop at this count (status ST_MAXIT)
  int phase_start;    // value of `it` when the current phase began
  int best_it;        // iteration of best_r
  int stall_window;   // 0 disables the stagnation test
  unsigned int ticket;  // last-block-done counter of the update pass
  double tol;         // stop when r < tol
  double ref;         // ||Delta_ref||; <= 0: taken from the next Delta (x0 = 0)
  double last_r;      // last ||Delta||/ref
  double best_r;
  double phase_first_r;
  double sumsq;       // last ||Delta||^2 (FP64)
};

// Kernel flags.
enum : int {
  F_XZERO = 1,      // the iterate is zero: do not read x
  F_REF = 2,        // reference pass: Delta at x = 0, store ||Delta|| in ref, no update
  F_NOSTATE = 4,    // ignore the device state (stand-alone transforms)
  F_APPLY_A = 8,    // residual pass writes A x instead of y - A x
  F_VREAL = 16,     // V is float32 (real potential)
  F_CBLOCK = 32,    // z pass over the column-block layout of the fused schedule
  F_REVERSE = 64    // strided-axis pass walks its tiles from the last one down
};

// Rows pass (transform along the contiguous last axis): a bit set of
// input, transform and output stages.
enum RowMode : int {
  R_IN_PRE = 1,      // t = (1-V) x + y from complex64 x, y        (fp32 only)
  R_IN_X = 2,        // t = x (complex64, upcast)                   (fp64 only)
  R_IN_BUF = 4,      // t = scratch row
  R_FWD = 8,         // forward transform
  R_MUL = 16,        // multiply by the spectral factor (needs R_FWD)
  R_INV = 32,        // inverse transform
  R_OUT_BUF = 64,    // scratch row = result
  R_OUT_POST = 128,  // Delta = (1-V)(u - x); x += alpha Delta; ||Delta||^2 (fp32)
  R_OUT_RESID = 256, // r = y - (u + V x)  [or A x = u + V x]; norms  (fp64)
  R_THEN_PRE_FWD = 512  // with R_OUT_POST: then t = (1-V) x_new + y and
                        // the forward transform of the next iteration -> scratch
};

// Strided-axis pass modes.
enum ColMode : int {
  COL_FWD = 0,
  COL_INV = 1,
  COL_FWD_MUL_INV = 2   // transform, multiply by the spectral factor, inverse
};

enum MulKind : int {
  MUL_LINV = 0,   // 1 / (N (Lhat(p) + 1))
  MUL_L = 1       // Lhat(p) / N
};

// Spectral symbol Lhat(p) = a |p|^2 + b on the grid; p_ax = ks[ax] * m_ax.
// Double-float: a real number as the unevaluated sum hi + lo of two floats,
// |lo| <= ulp(hi)/2 (a 48-bit significand); the arithmetic is in
// dfloat.cuh.  The working type of the refinement residual's transforms.
struct __align__(8) dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfl(float v) : hi(v), lo(0.f) {}
  // exact for |v| < 2^24 (frequency indices)
  __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}
  // the double split into its nearest float and the float nearest the rest
  __host__ __device__ constexpr dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
struct __align__(16) dfl2 {
  dfl x, y;
};

template <typename T>
struct Sym {
  T a_re, a_im, b_re, b_im;
  T inv_n;        // 1 / (total number of points)
  T ks[3];        // 2 pi / (n_ax dx) per axis (axis 0 slowest)
  int n[3];
  int ndim;
  const float2* table;   // Lhat per k-space point (C order), or nullptr: a |p|^2 + b
};

// k-space linear index of frequency index k along axis 0 and the flat
// index `col` over the faster axes (natural order, or the column-block
// layout col = (cb * 256 + ky) * 32 + xl of the fused schedule).
template <typename T>
__host__ __device__ __forceinline__ int64_t kspace_index(const Sym<T>& s, int k, int64_t col, bool cblock) {
  const int64_t inner = s.ndim == 3 ? (int64_t)s.n[1] * s.n[2] : (s.ndim == 2 ? s.n[1] : 1);
  if (cblock) col = ((col >> 5) & 255) * 256 + (col >> 13) * 32 + (col & 31);
  return (int64_t)k * inner + col;
}

// Independent problems on the same grid, stacked along a new slowest axis.
// count == 1 is the single-problem solver (the kernels then use the scalar
// symbol and step of their arguments).  Every block or tile belongs to one
// problem: rows_per and outer_per are multiples of the kernels' tile sizes.
struct Batch {
  int count;              // problems
  int64_t rows_per;       // last-axis lines per problem (rows kernels)
  int64_t outer_per;      // outer slabs per problem (strided-axis kernels)
  const float4* sym32;    // per problem (a_re, a_im, b_re, b_im), or nullptr
  const double* sym64;    // per problem 4 doubles, or nullptr
  const float* alpha;     // per problem step, or nullptr
  int hist_stride;        // history entries per problem
};

template <typename T>
struct RowsArgs {
  int mode;             // RowMode bit set
  int mul;              // MulKind for R_MUL
  int flags;
  int64_t nrows;        // number of rows (length-N lines along the last axis)
  const float2* x_in;   // complex64 iterate (or correction z)
  float2* x_out;        // complex64 iterate out (may alias x_in)
  const float2* y;      // complex64 source
  const void* V;        // complex64, or float32 with F_VREAL
  void* buf;            // complex scratch of type cplx_of<T>
  float2* r_out;        // ROW_INV_RESID output (complex64)
  double* partials;     // one (or two) doubles per block
  DevState* st;
  double* hist;
  T alpha;
  Sym<T> sym;
  Batch bt;
};

template <typename T>
struct ColsArgs {
  int mode;
  int mul;              // MulKind for COL_FWD_MUL_INV
  int flags;
  int64_t inner;        // S: stride of the axis = number of columns per outer slab
  int64_t outer;        // number of outer slabs
  int64_t inner_blocks; // ceil(inner / 32)
  void* buf;            // complex scratch of type cplx_of<T>, in place
  DevState* st;
  Sym<T> sym;
  Batch bt;
};

// Plane pass of the fused schedule (fused3d_kernels.cu), grids nz x 256 x 256.
enum PlaneMode : int {
  PL_PRE = 0,    // t = (1-V) x + y ; T = F_xy t           (phase prologue)
  PL_FULL = 1,   // F_xy^-1 ; Delta, update, norm ; next t ; F_xy
  PL_POST = 2    // F_xy^-1 ; Delta, norm (reference pass, no update)
};

struct PlaneArgs {
  int mode;
  int flags;
  int nz;
  const float2* x_in;
  float2* x_out;
  const float2* y;      // bulk-copied: 16-byte aligned
  const void* V;
  float2* buf;          // column-block layout T[z][cb][y][xl]
  const float2* tw;     // W_256^m table (device)
  double* partials;     // one double per CTA
  DevState* st;
  double* hist;
  float alpha;
};

cudaError_t plane_kernel_init();
cudaError_t launch_plane(const PlaneArgs& a, int clusters, cudaStream_t s);
int plane_max_active_clusters();
const float2* twiddle_table_f32();
const float2* twiddle_x_table_f32();   // W_1536^m, m < 1536

// Strided-axis pass with TMA-staged tiles (tma_kernels.cu).  The tensor map
// views the field as [outer][N][inner] (3-D, 8-byte elements, box {32, N, 1}).
struct ColsTmaArgs {
  int mode;             // ColMode
  int mul;              // MulKind
  int flags;
  int64_t inner_blocks; // ceil(inner / 32)
  int64_t tiles;        // outer * inner_blocks
  DevState* st;
  const float2* tw;     // W_256^m table (device)
  Sym<float> sym;
  Batch bt;
};
cudaError_t cols_tma_init();
cudaError_t launch_cols_tma(int n, int cols, const CUtensorMap& map, const ColsTmaArgs& a, int grid,
                            cudaStream_t s);

// Whole phases of the iteration for square 2-D grids n x n, n in {32, 64,
// 128, 256}, resident in the shared memory of one cluster of n / 16 CTAs per
// problem (onchip_kernels.cu).  One launch runs until every problem's state
// says done; with F_REF it evaluates the reference norm only.
enum : int { ONCHIP_SCALAR = 0, ONCHIP_ANTISYMMETRIC = 1, ONCHIP_FLUX = 2 };
struct OnchipArgs {
  int kind;             // ONCHIP_SCALAR, or a block form (K = 2 or 3 components as K planes)
  int flags;            // F_XZERO, F_REF, F_VREAL
  const float2* x_in;   // iterate in (not read with F_XZERO)
  float2* x_out;        // iterate out (may alias x_in; not written with F_REF)
  const float2* y;
  const void* V;        // complex64, or float32 with F_VREAL
  const float2* tw;     // W_256^m table (device)
  DevState* st;
  double* hist;
  float alpha;          // single problem (batches: bt.alpha)
  Sym<float> sym;       // block forms: ks, n and inv_n only
  float bsym[4];        // block forms: (a_re, a_im, b_re, b_im) of l, or (alpha, beta, s)
  Batch bt;
  uint32_t wait_limit;  // polls per bounded wait (0: the default, about a second)
  uint32_t fault_tx;    // test hook: bytes added to the first exchange's expected count
};
bool onchip_side(int n);
// rows: rows (and k-space columns) per CTA, 16 or 8 (8 for n <= 128).
bool onchip_rows_ok(int n, int rows);
// Clusters of the kernel for (n, rows, kind) that fit on the device at once
// (0: it cannot be launched here or is not built for these sizes).
int onchip_clusters(int n, int rows, int kind);
cudaError_t launch_onchip(int n, int rows, const OnchipArgs& a, int problems, cudaStream_t s);

// Fused rows pass of the pencil schedule as a persistent, bulk-copy staged
// kernel (tma_kernels.cu); row lengths 128 and 256.
struct RowsTmaArgs {
  int flags;            // F_XZERO, F_VREAL
  int64_t nrows;
  const float2* x_in;
  float2* x_out;
  const float2* y;
  const void* V;
  float2* buf;
  const float2* tw;     // W_256^m table (device)
  const float2* twx;    // W_1536^m table (device): radix stage of 96..512
  double* partials;     // one double per CTA (single problem) or per tile (batch)
  DevState* st;
  double* hist;
  float alpha;
  Batch bt;
};
cudaError_t rows_tma_init();
// Rows per tile of the staged rows pass for rows of length n (0: no staged
// kernel for this length).
int rows_tma_tile_rows(int n);
int rows_tma_ctas_per_sm(int n);
cudaError_t launch_rows_tma(int n, const RowsTmaArgs& a, int grid, cudaStream_t s);

// Split-y two-pass schedule (split3d_kernels.cu), grids nz x 256 x 256 with
// nz in {32, 64, 128, 256}: the rows pass does the x transform and the
// 16-point y1 stage of each tile (plane z, rows y = 16 y1 + y2); the column
// pass the 16-point y2 stage, the z transform and the spectral multiply.
// Scratch layout S[k1][z][y2][kx].
enum SplitMode : int {
  SPLIT_PRE = 0,    // t = (1-V) x + y ; forward x and y1 stages      (phase prologue)
  SPLIT_FULL = 1,   // inverse y1, x ; Delta, update, norm ; next t ; forward x, y1
  SPLIT_POST = 2    // inverse y1, x ; Delta, norm (reference pass: no update)
};
struct SplitArgs {
  int flags;            // F_XZERO, F_REF, F_VREAL
  int nz;
  const float2* x_in;
  float2* x_out;
  const float2* y;      // bulk-copied rows: 16-byte aligned
  const uint32_t* ymask;  // per rows tile u = 16 z + y2: bit y1 set when row
                          // 16 y1 + y2 of plane z of y is not all zero (rows
                          // left out are read as zeros); nullptr: every row
  const void* V;        // bulk-copied rows: 16-byte aligned
  float2* buf;          // scratch in the split layout
  const float2* tw;     // W_256^m table (device)
  double* partials;     // one double per CTA
  DevState* st;
  double* hist;
  float alpha;
};
struct SplitColsArgs {
  int flags;            // F_REVERSE
  float2* buf;          // scratch in the split layout
  const float2* tw;     // W_256^m table (device)
  DevState* st;
  Sym<float> sym;       // quadratic symbol or table (k-space C order)
};
cudaError_t split_init();
bool split_nz_ok(int nz);
int split_cols_ctas_per_sm(int nz);
cudaError_t launch_split_rows(int mode, const SplitArgs& a, int grid, cudaStream_t s);
// mask[u] (nz * 16 words, u = 16 z + y2) = the rows of tile u in which y has
// a value other than zero (NaN and Inf count as nonzero).
cudaError_t launch_split_ymask(const float2* y, int nz, uint32_t* mask, cudaStream_t s);
// map: the scratch viewed as 4-D {kx 256, z nz, y2 16, k1 16} (8-byte
// elements, strides in that order 32768 / 2048 / nz * 32768 bytes), box {2, nz, 16, 1}.
cudaError_t launch_split_cols(int nz, const CUtensorMap& map, const SplitColsArgs& a, int grid,
                              cudaStream_t s);

// Launchers (pencil_kernels.cu).  n = transform length (power of two, 2..256).
cudaError_t launch_rows_f32(int n, const RowsArgs<float>& a, int64_t grid, cudaStream_t s);
cudaError_t launch_rows_f64(int n, const RowsArgs<double>& a, int64_t grid, cudaStream_t s);
cudaError_t launch_cols_f32(int n, const ColsArgs<float>& a, cudaStream_t s);
cudaError_t launch_cols_f64(int n, const ColsArgs<double>& a, cudaStream_t s);
// The same passes in double-float (df_kernels.cu): the refinement residual.
cudaError_t launch_rows_df(int n, const RowsArgs<dfl>& a, int64_t grid, cudaStream_t s);
cudaError_t launch_cols_df(int n, const ColsArgs<dfl>& a, cudaStream_t s);
int rows_per_block_f32(int n);
int rows_per_block_f64(int n);
int cols_per_block(int n);   // columns per block of the plain strided-axis pass

// Auxiliary kernels (pencil_kernels.cu).
cudaError_t init_twiddles();
// The double-float twiddle tables from the FP64 ones (W_256^m, W_1536^m).
cudaError_t init_twiddles_df(const double2* tw256, const double2* tw1536);
// Per-block statistics of V (max |V|, min Re 1/(1-V), nonfinite count) then
// their reduction into out[3] (device).
cudaError_t launch_v_stats(const void* V, int vreal, int64_t n, double* partials,
                           int nblocks, double* out, cudaStream_t s);
// A symbol table's min Re(Lhat) + 1 and non-finite count into out[0..1].
cudaError_t launch_table_stats(const float2* table, int64_t n, double* partials, int nblocks,
                               double* out, cudaStream_t s);
// x += z (complex64); with `mask` (per problem, n_per points each) only where
// mask[problem] != 0.
cudaError_t launch_axpy1(float2* x, const float2* z, int64_t n, cudaStream_t s,
                         const int* mask = nullptr, int64_t n_per = 0);
// Sum `groups` consecutive runs of `count` partial pairs (2 doubles per
// block) into out[2 * group], out[2 * group + 1].
cudaError_t launch_sum_pairs(const double* partials, int count, int groups, double* out,
                             cudaStream_t s);
// Record the message usp_last_error() returns on this thread (usp_api.cpp).
void set_last_error(const char* fmt, ...);
// Copy a real float32 or complex64 potential into solver storage.
cudaError_t launch_copy_bytes(void* dst, const void* src, size_t bytes, cudaStream_t s);

}  // namespace usp
