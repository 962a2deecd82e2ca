// usp_api.cpp -- the C ABI of include/usp.h: solver handles, the schedule of
// one fixed-point iteration (paper Algorithm 1, forward-eliminated operator
// of Sec. 2.1), the convergence loop and FP64 iterative refinement.
//
// Iterations are launched in CUDA graphs of `chunk` iterations.  Every
// kernel reads a device-side done flag at entry, so iterations queued after
// convergence cost only empty launches; the host reads the device state
// once per group of graph launches (the only device-to-host sync of the
// loop).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "tc_kernels.h"
#include "usp.h"

using namespace usp;

// ------------------------------------------------------------- errors ---

static thread_local std::string g_last_error;

static usp_status fail(usp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = std::string(usp_status_string(st)) + ": " + buf;
  return st;
}

void usp::set_last_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

#define CUDA_TRY(call)                                                             \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      usp_status st_ = (e_ == cudaErrorMemoryAllocation) ? USP_ERR_OOM : USP_ERR_CUDA; \
      return fail(st_, "%s failed: %s", #call, cudaGetErrorString(e_));            \
    }                                                                              \
  } while (0)

// ---------------------------------------------------- per-device init ---

static std::mutex g_init_mu;
static uint64_t g_init_mask = 0;

static usp_status ensure_device_init() {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (dev < 64 && (g_init_mask >> dev) & 1ull) return USP_OK;
  CUDA_TRY(init_twiddles());
  CUDA_TRY(plane_kernel_init());
  CUDA_TRY(cols_tma_init());
  CUDA_TRY(rows_tma_init());
  CUDA_TRY(split_init());
  CUDA_TRY(tc_cols_init());
  if (dev < 64) g_init_mask |= (1ull << dev);
  return USP_OK;
}

// ------------------------------------------------------------ solver ---

struct GraphEntry {
  const void* y;
  const void* x;
  int chunk;
  cudaGraphExec_t exec;
};

struct usp_solver {
  int ndim = 0;
  int n[3] = {1, 1, 1};
  int64_t N = 0;
  double dx = 1.0;
  usp_lsymbol sym{};
  bool vreal = false;
  double alpha = 0.0;
  double vmax = 0.0;
  usp_options opt{};
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  void* V = nullptr;
  float2* buf = nullptr;           // FP32 scratch field
  double* partials = nullptr;
  int64_t npartials = 0;
  DevState* st = nullptr;
  DevState* st_host = nullptr;     // pinned mirror
  double* hist = nullptr;
  int hist_cap = 0;
  double* red = nullptr;           // 4 doubles (device)
  double* red_host = nullptr;      // 4 doubles (pinned)
  float2* z = nullptr;             // refinement correction
  float2* yp = nullptr;            // refinement source y - A x
  double2* buf64 = nullptr;        // FP64 scratch field
  float2* hy = nullptr;            // device copies for usp_solve_host
  float2* hx = nullptr;
  std::vector<GraphEntry> graphs;
  std::vector<double> history;
  Sym<float> symf{};
  Sym<double> symd{};
  const float2* tw32 = nullptr;    // device twiddle table (fused plane pass)
  int plane_clusters = 0;          // persistent clusters of the fused plane pass
  int B = 1;                       // independent problems on this grid (batch)
  int64_t NB = 0;                  // B * N
  float4* bsym32 = nullptr;        // per-problem symbols (B > 1), device
  double* bsym64 = nullptr;
  float* balpha = nullptr;         // per-problem steps (B > 1), device
  int* bmask = nullptr;            // problems refined in the current phase, device
  int* bmask_host = nullptr;       // pinned mirror
  float2* table = nullptr;         // tabulated symbol Lhat(p) (USP_LSYM_TABLE), device
  int onchip_clusters[2] = {0, 0}; // co-resident clusters of the on-chip kernels with 8 / 16 rows per CTA
  std::vector<double> alphas;      // per problem
  std::vector<std::vector<double>> histories;   // per problem, last solve
  int num_sms = 0;
  bool maps_ok = false;            // TMA tensor maps of the scratch field
  CUtensorMap map_ax[3][2];        // [tile 32 / 16 / 8 columns][axis]: strided-axis views of s->buf
  bool split_ok = false;           // split_map encoded (grids nz x 256 x 256)
  uint32_t* ymask = nullptr;       // split layout: per rows tile, the rows where the source is nonzero
  const float2* ymask_src = nullptr;  // the source the mask was last built from
  double ymask_frac = 1.0;         // fraction of rows with a nonzero source (when counted)
  CUtensorMap split_map;           // the scratch in the split layout, 4-D (column-pass tiles)
};

// Column-tile width of the staged strided-axis passes when the options leave
// it to the library.
static constexpr int kDefaultColsTile = 8;

static bool is_pow2_in_range(int64_t v) { return v >= 2 && v <= 256 && (v & (v - 1)) == 0; }
// Axis lengths the line kernels transform: 2^k in [2, 256], and 3 * 2^k or
// 2 * 256 through their radix-3 / radix-2 outer stage.
static bool supported_length(int64_t v) { return is_pow2_in_range(v) || v == 96 || v == 192 || v == 384 || v == 512; }

static void free_graphs(usp_solver* s) {
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

// ------------------------------------------------------ TMA tensor maps ---

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool tensor_map_encoder() {
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

// The field viewed as [outer][n][inner] complex64 (8-byte elements), tiles of
// {cols, n, 1}.
static bool encode_cols_map(CUtensorMap* m, void* base, int64_t inner, int n, int64_t outer,
                            int cols) {
  if (!tensor_map_encoder()) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)n, (cuuint64_t)outer};
  const cuuint64_t strides[2] = {(cuuint64_t)inner * 8, (cuuint64_t)n * inner * 8};
  const cuuint32_t box[3] = {(cuuint32_t)cols, (cuuint32_t)n, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The scratch in the split-y layout S[k1][z][y2][kx] viewed as 4-D
// {kx 256, z nz, y2 16, k1 16} (8-byte elements; z listed before y2 so that
// a column tile lands in shared memory as [y2][z][xi]); a column-pass tile
// (k1, two kx) is the box {2, nz, 16, 1}.
static bool encode_split_map(CUtensorMap* m, void* base, int nz) {
  if (!tensor_map_encoder()) return false;
  const cuuint64_t dims[4] = {256, (cuuint64_t)nz, 16, 16};
  // S[k1][z][y2][kx]: z, y2 and k1 strides in bytes
  const cuuint64_t strides[3] = {16 * 256 * 8, 256 * 8, (cuuint64_t)nz * 16 * 256 * 8};
  const cuuint32_t box[4] = {2, (cuuint32_t)nz, 16, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static void build_maps(usp_solver* s) {
  s->split_ok = s->B == 1 && s->ndim == 3 && split_nz_ok(s->n[0]) && s->n[1] == 256 &&
                s->n[2] == 256 && encode_split_map(&s->split_map, s->buf, s->n[0]);
  s->maps_ok = false;
  if (s->ndim < 2) return;
  bool ok = true;
  for (int axis = 0; axis < s->ndim - 1 && axis < 2; ++axis) {
    if (!is_pow2_in_range(s->n[axis])) return;  // the staged kernels take 2^k <= 256
    int64_t inner = 1, outer = 1;
    for (int ax = axis + 1; ax < s->ndim; ++ax) inner *= s->n[ax];
    for (int ax = 0; ax < axis; ++ax) outer *= s->n[ax];
    ok = ok && encode_cols_map(&s->map_ax[0][axis], s->buf, inner, s->n[axis], outer * s->B, 32);
    ok = ok && encode_cols_map(&s->map_ax[1][axis], s->buf, inner, s->n[axis], outer * s->B, 16);
    ok = ok && encode_cols_map(&s->map_ax[2][axis], s->buf, inner, s->n[axis], outer * s->B, 8);
  }
  s->maps_ok = ok;
}

// ------------------------------------------------------ the schedule ---

static int64_t rows_grid_f32(const usp_solver* s) {
  const int nx = s->n[s->ndim - 1];
  const int64_t nrows = s->NB / nx;
  const int F = rows_per_block_f32(nx);
  return (nrows + F - 1) / F;
}
static int64_t rows_grid_f64(const usp_solver* s) {
  const int nx = s->n[s->ndim - 1];
  const int64_t nrows = s->NB / nx;
  const int F = rows_per_block_f64(nx);
  return (nrows + F - 1) / F;
}

// Batch descriptor for a pass: outer slabs per problem (strided-axis passes).
static Batch batch_desc(const usp_solver* s, int64_t outer_per) {
  Batch b{};
  b.count = s->B;
  b.rows_per = s->N / s->n[s->ndim - 1];
  b.outer_per = outer_per;
  b.hist_stride = s->hist_cap;
  if (s->B > 1) {
    b.sym32 = s->bsym32;
    b.sym64 = s->bsym64;
    b.alpha = s->balpha;
  }
  return b;
}

template <typename T>
static ColsArgs<T> cols_args(const usp_solver* s, int axis, int mode, int mul, int flags,
                             void* buf, const Sym<T>& sym) {
  ColsArgs<T> c{};
  c.mode = mode;
  c.mul = mul;
  c.flags = flags;
  int64_t inner = 1, outer = 1;
  for (int ax = axis + 1; ax < s->ndim; ++ax) inner *= s->n[ax];
  for (int ax = 0; ax < axis; ++ax) outer *= s->n[ax];
  c.bt = batch_desc(s, outer);
  outer *= s->B;  // problems are stacked along a new slowest axis
  c.inner = inner;
  c.outer = outer;
  const int cols = cols_per_block(s->n[axis]);
  c.inner_blocks = (inner + cols - 1) / cols;
  c.buf = buf;
  c.st = s->st;
  c.sym = sym;
  return c;
}

// A strided-axis FP32 pass: TMA-staged tiles when available, else plain.
static std::function<cudaError_t(cudaStream_t)> cols_pass_f32(usp_solver* s, int axis, int mode,
                                                              int flags) {
  auto c = cols_args<float>(s, axis, mode, MUL_LINV, flags, s->buf, s->symf);
  const int n = s->n[axis];
  if (s->opt.tc_dft && n == 256 && s->B == 1 && !(flags & F_CBLOCK) && s->maps_ok && !s->opt.no_tma) {
    // the 256-point transforms on the tensor cores (tiles of 8 columns)
    ColsTmaArgs t{};
    t.mode = mode;
    t.mul = MUL_LINV;
    t.flags = flags;
    t.inner_blocks = (c.inner + 7) / 8;
    t.tiles = t.inner_blocks * c.outer;
    t.st = s->st;
    t.tw = s->tw32;
    t.sym = s->symf;
    t.bt = c.bt;
    const int grid = (int)std::min<int64_t>(t.tiles, (int64_t)s->num_sms * 2);
    const CUtensorMap map = s->map_ax[2][axis];
    return [=](cudaStream_t st) { return launch_cols_tc(map, t, grid, st); };
  }
  if (s->maps_ok && !s->opt.no_tma) {
    // tiles of 32 / 16 / 8 columns run 1 / 2 / 4 CTAs per SM
    const int cols = s->opt.cols_tile ? s->opt.cols_tile : kDefaultColsTile;
    ColsTmaArgs t{};
    t.mode = mode;
    t.mul = MUL_LINV;
    t.flags = flags;
    t.inner_blocks = (c.inner + cols - 1) / cols;
    t.tiles = t.inner_blocks * c.outer;
    t.st = s->st;
    t.tw = s->tw32;
    t.sym = s->symf;
    t.bt = c.bt;
    const int grid = (int)std::min<int64_t>(t.tiles, (int64_t)s->num_sms * (32 / cols));
    const CUtensorMap map = s->map_ax[cols == 32 ? 0 : (cols == 16 ? 1 : 2)][axis];
    return [=](cudaStream_t st) { return launch_cols_tma(n, cols, map, t, grid, st); };
  }
  return [=](cudaStream_t st) { return launch_cols_f32(n, c, st); };
}

// One pass of an iteration: a kernel launch plus what it moves.
struct PassLaunch {
  const char* name;
  double bytes_per_point;  // algorithmic HBM bytes per grid point
  std::function<cudaError_t(cudaStream_t)> go;
};

// Kernel launches issued by this library (graph launches count their nodes).
static std::atomic<int64_t> g_launches{0};

// The passes of the pencil schedule.  y: source; xin/xout: iterate in/out
// (xin unused with F_XZERO).
//   prologue  : rows pass t = (1-V) x + y, FFT x  (once per phase)
//   iteration : column passes; rows pass inverse FFT x, Delta, update, norm,
//               and (fused) the next iteration's B x + y with its FFT x.
// A reference pass (F_REF) is prologue + columns + an unfused rows pass.
static RowsArgs<float> rows_args(usp_solver* s, const float2* y, const float2* xin,
                                 float2* xout, int flags) {
  RowsArgs<float> r{};
  r.flags = flags | (s->vreal ? F_VREAL : 0);
  r.nrows = s->NB / s->n[s->ndim - 1];
  r.bt = batch_desc(s, 1);
  r.x_in = xin;
  r.x_out = xout;
  r.y = y;
  r.V = s->V;
  r.buf = s->buf;
  r.partials = s->partials;
  r.st = s->st;
  r.hist = s->hist;
  r.alpha = (float)s->alpha;
  r.sym = s->symf;
  r.mul = MUL_LINV;
  return r;
}

static std::vector<PassLaunch> pencil_prologue(usp_solver* s, const float2* y, const float2* xin,
                                               int flags) {
  std::vector<PassLaunch> P;
  if (s->ndim == 1) return P;
  const double vb = s->vreal ? 4.0 : 8.0;
  const bool xz = (flags & F_XZERO) != 0;
  const int nx = s->n[s->ndim - 1];
  const int64_t grid = rows_grid_f32(s);
  RowsArgs<float> r = rows_args(s, y, xin, nullptr, flags);
  r.mode = R_IN_PRE | R_FWD | R_OUT_BUF;
  P.push_back({"rows_pre_fwd", 16.0 + (xz ? 0.0 : 8.0 + vb),
               [=](cudaStream_t t) { return launch_rows_f32(nx, r, grid, t); }});
  return P;
}

static std::vector<PassLaunch> pencil_passes(usp_solver* s, const float2* y, const float2* xin,
                                             float2* xout, int flags) {
  std::vector<PassLaunch> P;
  const double vb = s->vreal ? 4.0 : 8.0;
  const bool xz = (flags & F_XZERO) != 0, ref = (flags & F_REF) != 0;
  const int nd = s->ndim;
  const int nx = s->n[nd - 1];
  const int64_t grid = rows_grid_f32(s);
  RowsArgs<float> r = rows_args(s, y, xin, xout, flags);
  if (nd == 1) {
    r.mode = R_IN_PRE | R_FWD | R_MUL | R_INV | R_OUT_POST;
    P.push_back({"rows_full", 8.0 + vb + (xz ? 0.0 : 8.0) + (ref ? 0.0 : 8.0),
                 [=](cudaStream_t t) { return launch_rows_f32(nx, r, grid, t); }});
    return P;
  }
  const int cflags = flags & ~F_XZERO & ~F_REF;
  if (nd == 2) {
    // a batch's column pass walks from the last problem down: the rows pass
    // wrote it last, and the next rows pass starts at the first problem
    P.push_back({"cols0_fwd_mul_inv", 16.0,
                 cols_pass_f32(s, 0, COL_FWD_MUL_INV, cflags | (s->B > 1 ? F_REVERSE : 0))});
  } else {
    // Both y passes walk from the last z-slab down: the forward one starts
    // where the rows pass (increasing rows) stopped, and the inverse one
    // stops at the first slab, where the next rows pass starts; the parts
    // still in L2 are read first.
    P.push_back({"cols1_fwd", 16.0, cols_pass_f32(s, 1, COL_FWD, cflags | F_REVERSE)});
    P.push_back({"cols0_fwd_mul_inv", 16.0, cols_pass_f32(s, 0, COL_FWD_MUL_INV, cflags)});
    P.push_back({"cols1_inv", 16.0, cols_pass_f32(s, 1, COL_INV, cflags | F_REVERSE)});
  }
  if (ref) {
    r.mode = R_IN_BUF | R_INV | R_OUT_POST;
    P.push_back({"rows_inv_post", 8.0 + vb,
                 [=](cudaStream_t t) { return launch_rows_f32(nx, r, grid, t); }});
  } else {
    // read scratch, V, x (unless zero), y; write x, scratch
    const double bytes = 32.0 + vb + (xz ? 0.0 : 8.0);
    // bulk copies read y, V and the scratch field: 16-byte aligned sources
    const bool aligned = (((uintptr_t)y | (uintptr_t)s->V | (uintptr_t)s->buf) & 15u) == 0;
    const int64_t tile_rows = rows_tma_tile_rows(nx);
    const bool tiles_fit = tile_rows > 0 && (s->B == 1 || (r.bt.rows_per % tile_rows) == 0);
    if (!s->opt.no_tma && aligned && tiles_fit) {
      RowsTmaArgs t{};
      t.flags = r.flags;
      t.nrows = r.nrows;
      t.x_in = xin;
      t.x_out = xout;
      t.y = y;
      t.V = s->V;
      t.buf = s->buf;
      t.tw = s->tw32;
      t.twx = twiddle_x_table_f32();
      t.partials = s->partials;
      t.st = s->st;
      t.hist = s->hist;
      t.alpha = (float)s->alpha;
      t.bt = r.bt;
      const int64_t tiles = (r.nrows + tile_rows - 1) / tile_rows;
      const int tgrid = (int)std::min<int64_t>(tiles, (int64_t)s->num_sms * rows_tma_ctas_per_sm(nx));
      P.push_back({"rows_inv_post_pre_fwd", bytes,
                   [=](cudaStream_t st) { return launch_rows_tma(nx, t, tgrid, st); }});
    } else {
      r.mode = R_IN_BUF | R_INV | R_OUT_POST | R_THEN_PRE_FWD;
      P.push_back({"rows_inv_post_pre_fwd", bytes,
                   [=](cudaStream_t t) { return launch_rows_f32(nx, r, grid, t); }});
    }
  }
  return P;
}

// ---- fused two-pass schedule (grids nz x 256 x 256, fused3d_kernels.cu)

// ---- on-chip schedule (square 2-D grids n x n, n in {32, 64, 128, 256},
// onchip_kernels.cu): a whole phase of iterations per launch.

// Rows per CTA: the option, else 8 (twice the CTAs, each with half the
// values) for single problems and batches of n <= 96, 16 for the rest
// (measured, us per iteration, 16 / 8 rows: one 128^2 problem 5.97 / 5.37,
// 64 of them 16.2 / 20.4; one 64^2 3.49 / 3.05, 64 of them 4.91 / 4.13;
// one 96^2 8.6 / 6.7, 70 of them 22.8 / 21.2).
static int onchip_rows_of(const usp_solver* s, const usp_options& o) {
  if (o.onchip_rows > 0) return o.onchip_rows;
  return (s->n[0] <= 128 && (s->B == 1 || s->n[0] <= 96)) ? 8 : 16;
}
static bool onchip_available(const usp_solver* s, int rows) {
  return s->ndim == 2 && s->n[0] == s->n[1] && onchip_rows_ok(s->n[0], rows) &&
         s->onchip_clusters[rows == 8 ? 0 : 1] > 0;
}
static bool onchip_supported(const usp_solver* s) { return onchip_available(s, onchip_rows_of(s, s->opt)); }
// Schedule 3 forces the on-chip kernels, schedule 1 the pencil passes.  The
// automatic choice (0) takes on-chip where it applies unless the problems'
// clusters do not all fit on the device at once and each holds 12-16 SMs'
// worth of shared memory (n = 192, 256): there the passes keep more SMs busy
// (measured: 64 problems of 256^2, 75 us per pencil iteration against 108 us
// on chip; 70 of 192^2, 80 against 122 us; 64 of 128^2, 35 against 17 us).
static bool use_onchip(const usp_solver* s) {
  if (!onchip_supported(s)) return false;
  if (s->opt.schedule == 3) return true;
  if (s->opt.schedule != 0) return false;
  const int rows = onchip_rows_of(s, s->opt);
  return s->n[0] <= 128 || s->B <= s->onchip_clusters[rows == 8 ? 0 : 1];
}

static OnchipArgs onchip_args(usp_solver* s, const float2* y, const float2* xin, float2* xout,
                              int flags) {
  OnchipArgs a{};
  a.kind = ONCHIP_SCALAR;
  a.flags = flags | (s->vreal ? F_VREAL : 0);
  a.x_in = xin;
  a.x_out = xout;
  a.y = y;
  a.V = s->V;
  a.tw = s->tw32;
  a.st = s->st;
  a.hist = s->hist;
  a.alpha = (float)s->alpha;
  a.sym = s->symf;
  a.bt = batch_desc(s, 0);
  if (s->opt.test_wait_fault) {   // bytes that nobody sends; give up after a few thousand polls
    a.fault_tx = 8;
    a.wait_limit = 4096;
  }
  return a;
}

static cudaError_t enqueue_onchip(usp_solver* s, const float2* y, const float2* xin, float2* xout,
                                  int flags, cudaStream_t strm, bool count = true) {
  if (count) g_launches.fetch_add(1);
  return launch_onchip(s->n[0], onchip_rows_of(s, s->opt), onchip_args(s, y, xin, xout, flags), s->B, strm);
}

static bool fused_supported(const usp_solver* s) {
  return s->B == 1 && s->ndim == 3 && s->n[1] == 256 && s->n[2] == 256 && s->plane_clusters > 0 &&
         s->maps_ok;
}
// Automatic choice: the pencil schedule; schedule 2 selects the fused one
// (it bulk-copies y, so y must be 16-byte aligned; otherwise pencil).
static bool use_fused(const usp_solver* s, const float2* y) {
  return s->opt.schedule == 2 && fused_supported(s) && (((uintptr_t)y & 15u) == 0);
}

static PlaneArgs plane_args(usp_solver* s, const float2* y, const float2* xin, float2* xout,
                            int flags, int mode) {
  PlaneArgs p{};
  p.mode = mode;
  p.flags = flags | (s->vreal ? F_VREAL : 0);
  p.nz = s->n[0];
  p.x_in = xin;
  p.x_out = xout;
  p.y = y;
  p.V = s->V;
  p.buf = s->buf;
  p.tw = s->tw32;
  p.partials = s->partials;
  p.st = s->st;
  p.hist = s->hist;
  p.alpha = (float)s->alpha;
  return p;
}

static std::function<cudaError_t(cudaStream_t)> plane_pass(usp_solver* s, const PlaneArgs& p) {
  const int clusters = std::max(1, std::min(s->plane_clusters, s->n[0]));
  return [=](cudaStream_t t) { return launch_plane(p, clusters, t); };
}

static std::vector<PassLaunch> fused_prologue(usp_solver* s, const float2* y, const float2* xin,
                                              int flags) {
  const double vb = s->vreal ? 4.0 : 8.0;
  const bool xz = (flags & F_XZERO) != 0;
  PlaneArgs p = plane_args(s, y, xin, nullptr, flags & ~F_REF, PL_PRE);
  return {{"plane_pre", 16.0 + (xz ? 0.0 : 8.0 + vb), plane_pass(s, p)}};
}

static std::vector<PassLaunch> fused_passes(usp_solver* s, const float2* y, const float2* xin,
                                            float2* xout, int flags) {
  std::vector<PassLaunch> P;
  const double vb = s->vreal ? 4.0 : 8.0;
  const bool xz = (flags & F_XZERO) != 0, ref = (flags & F_REF) != 0;
  const int cflags = (flags & ~F_XZERO & ~F_REF) | F_CBLOCK;
  P.push_back({"z_fwd_mul_inv", 16.0, cols_pass_f32(s, 0, COL_FWD_MUL_INV, cflags)});
  if (ref) {
    PlaneArgs p = plane_args(s, y, xin, xout, flags, PL_POST);
    P.push_back({"plane_post", 8.0 + vb, plane_pass(s, p)});
  } else {
    PlaneArgs p = plane_args(s, y, xin, xout, flags, PL_FULL);
    P.push_back({"plane_full", 32.0 + vb + (xz ? 0.0 : 8.0), plane_pass(s, p)});
  }
  return P;
}

// ---- split-y two-pass schedule (grids nz x 256 x 256, split3d_kernels.cu)

static bool split_supported(const usp_solver* s) { return s->split_ok && s->num_sms > 0; }
// Schedule 4 selects it; the automatic choice (0) takes it wherever it
// applies (measured per iteration, split against pencil: nz = 32 48 / 78 us,
// 64 72 / 110, 128 126 / 164, 256 222 / 279).  The rows pass bulk-copies rows of y and V and the column pass
// whole tiles of the scratch, so all three must be 16-byte aligned
// (otherwise the pencil schedule runs).
static bool use_split(const usp_solver* s, const float2* y) {
  if (!split_supported(s)) return false;
  if (s->opt.schedule != 4 && !(s->opt.schedule == 0 && !s->opt.tc_dft && !s->opt.no_tma))
    return false;
  return (((uintptr_t)y | (uintptr_t)s->V | (uintptr_t)s->buf) & 15u) == 0;
}

static SplitArgs split_args(usp_solver* s, const float2* y, const float2* xin, float2* xout,
                            int flags) {
  SplitArgs a{};
  a.flags = flags | (s->vreal ? F_VREAL : 0);
  a.nz = s->n[0];
  a.x_in = xin;
  a.x_out = xout;
  a.y = y;
  a.ymask = (y && y == s->ymask_src) ? s->ymask : nullptr;
  a.V = s->V;
  a.buf = s->buf;
  a.tw = s->tw32;
  a.partials = s->partials;
  a.st = s->st;
  a.hist = s->hist;
  a.alpha = (float)s->alpha;
  return a;
}

// The split rows pass copies only the rows of the source y that hold a
// nonzero value (a point source or a beam on one face fills a few of the
// grid's rows): build the row mask of y before a phase that iterates on it.
// The mask is rebuilt at every phase start, so it always describes the
// source's current contents.  With `count`, also the fraction of rows kept.
static usp_status prepare_source_mask(usp_solver* s, const float2* y, bool count) {
  if (!use_split(s, y)) return USP_OK;
  const int nz = s->n[0];
  if (!s->ymask) CUDA_TRY(cudaMalloc(&s->ymask, sizeof(uint32_t) * (size_t)nz * 16));
  CUDA_TRY(launch_split_ymask(y, nz, s->ymask, s->stream));
  g_launches.fetch_add(1);
  s->ymask_src = y;
  if (count) {
    std::vector<uint32_t> m((size_t)nz * 16);
    CUDA_TRY(cudaMemcpyAsync(m.data(), s->ymask, sizeof(uint32_t) * m.size(), cudaMemcpyDeviceToHost,
                             s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    int64_t rows = 0;
    for (uint32_t w : m) rows += __builtin_popcount(w & 0xFFFFu);
    s->ymask_frac = (double)rows / (double)(nz * 256);
  }
  return USP_OK;
}

static std::function<cudaError_t(cudaStream_t)> split_rows_pass(usp_solver* s, int mode,
                                                                const SplitArgs& a) {
  const int grid = (int)std::min<int64_t>((int64_t)s->n[0] * 16, (int64_t)s->num_sms * 2);
  return [=](cudaStream_t t) { return launch_split_rows(mode, a, grid, t); };
}

static std::vector<PassLaunch> split_prologue(usp_solver* s, const float2* y, const float2* xin,
                                              int flags) {
  const double vb = s->vreal ? 4.0 : 8.0;
  const bool xz = (flags & F_XZERO) != 0;
  SplitArgs a = split_args(s, y, xin, nullptr, flags & ~F_REF);
  const double yb = 8.0 * (a.ymask ? s->ymask_frac : 1.0);   // source rows copied
  return {{"split_rows_pre", 8.0 + yb + (xz ? 0.0 : 8.0 + vb), split_rows_pass(s, SPLIT_PRE, a)}};
}

static std::vector<PassLaunch> split_passes(usp_solver* s, const float2* y, const float2* xin,
                                            float2* xout, int flags) {
  std::vector<PassLaunch> P;
  const double vb = s->vreal ? 4.0 : 8.0;
  const bool xz = (flags & F_XZERO) != 0, ref = (flags & F_REF) != 0;
  SplitColsArgs c{};
  c.flags = 0;
  c.buf = s->buf;
  c.tw = s->tw32;
  c.st = s->st;
  c.sym = s->symf;
  const int nz = s->n[0];
  const int cgrid = s->num_sms * split_cols_ctas_per_sm(nz);
  const CUtensorMap cmap = s->split_map;
  P.push_back({"split_cols", 16.0,
               [=](cudaStream_t t) { return launch_split_cols(nz, cmap, c, cgrid, t); }});
  SplitArgs a = split_args(s, y, xin, xout, flags);
  if (ref) P.push_back({"split_rows_post", 8.0 + vb, split_rows_pass(s, SPLIT_POST, a)});
  else {
    const double yb = 8.0 * (a.ymask ? s->ymask_frac : 1.0);   // source rows copied
    P.push_back({"split_rows_full", 24.0 + yb + vb + (xz ? 0.0 : 8.0), split_rows_pass(s, SPLIT_FULL, a)});
  }
  return P;
}

static std::vector<PassLaunch> iteration_passes(usp_solver* s, const float2* y, const float2* xin,
                                                float2* xout, int flags) {
  if (use_split(s, y)) return split_passes(s, y, xin, xout, flags);
  if (use_fused(s, y)) return fused_passes(s, y, xin, xout, flags);
  return pencil_passes(s, y, xin, xout, flags);
}

static std::vector<PassLaunch> prologue_passes(usp_solver* s, const float2* y, const float2* xin,
                                               int flags) {
  if (use_split(s, y)) return split_prologue(s, y, xin, flags);
  if (use_fused(s, y)) return fused_prologue(s, y, xin, flags);
  return pencil_prologue(s, y, xin, flags);
}

// One iteration; with `first` the phase's prologue is launched before it.
static cudaError_t enqueue_iteration(usp_solver* s, const float2* y, const float2* xin,
                                     float2* xout, int flags, cudaStream_t strm,
                                     bool count = true, bool first = false) {
  if (use_onchip(s))  // the reference pass (F_REF) or a whole phase
    return enqueue_onchip(s, y, xin, xout, flags, strm, count);
  if (first) {
    for (auto& p : prologue_passes(s, y, xin, flags)) {
      cudaError_t e = p.go(strm);
      if (e != cudaSuccess) return e;
      if (count) g_launches.fetch_add(1);
    }
  }
  for (auto& p : iteration_passes(s, y, xin, xout, flags)) {
    cudaError_t e = p.go(strm);
    if (e != cudaSuccess) return e;
    if (count) g_launches.fetch_add(1);
  }
  return cudaSuccess;
}

static_assert(sizeof(dfl2) == sizeof(double2), "the residual scratch holds 16-byte values");

// The FP64 symbol in double-float words.
static Sym<dfl> sym_df(const Sym<double>& d) {
  Sym<dfl> s{};
  s.a_re = dfl(d.a_re);
  s.a_im = dfl(d.a_im);
  s.b_re = dfl(d.b_re);
  s.b_im = dfl(d.b_im);
  s.inv_n = dfl(d.inv_n);
  for (int i = 0; i < 3; ++i) {
    s.ks[i] = dfl(d.ks[i]);
    s.n[i] = d.n[i];
  }
  s.ndim = d.ndim;
  s.table = d.table;
  return s;
}

// r = y - A x (or A x with apply_a) in T (FP64 or double-float, 16 bytes per
// complex value in s->buf64); norms into s->red[0..1].
template <typename T>
static usp_status enqueue_residual_t(usp_solver* s, const float2* x, const float2* y, float2* rout,
                                     bool apply_a, const Sym<T>& sym,
                                     cudaError_t (*rows)(int, const RowsArgs<T>&, int64_t, cudaStream_t),
                                     cudaError_t (*cols)(int, const ColsArgs<T>&, cudaStream_t)) {
  if (!s->buf64) CUDA_TRY(cudaMalloc(&s->buf64, sizeof(double2) * s->NB));
  const int vflag = s->vreal ? F_VREAL : 0;
  const int nd = s->ndim;
  const int nx = s->n[nd - 1];
  RowsArgs<T> r{};
  r.flags = F_NOSTATE | vflag | (apply_a ? F_APPLY_A : 0);
  r.nrows = s->NB / nx;
  r.bt = batch_desc(s, 1);
  r.x_in = x;
  r.y = y;
  r.V = s->V;
  r.buf = s->buf64;
  r.r_out = rout;
  r.partials = s->partials;
  r.st = s->st;
  r.sym = sym;
  r.mul = MUL_L;
  const int64_t grid = rows_grid_f64(s);   // the same row blocks for both types
  if (nd == 1) {
    r.mode = R_IN_X | R_FWD | R_MUL | R_INV | R_OUT_RESID;
    CUDA_TRY(rows(nx, r, grid, s->stream));
  } else {
    r.mode = R_IN_X | R_FWD | R_OUT_BUF;
    CUDA_TRY(rows(nx, r, grid, s->stream));
    if (nd == 2) {
      auto c = cols_args<T>(s, 0, COL_FWD_MUL_INV, MUL_L, F_NOSTATE, s->buf64, sym);
      CUDA_TRY(cols(s->n[0], c, s->stream));
    } else {
      auto c1 = cols_args<T>(s, 1, COL_FWD, MUL_L, F_NOSTATE, s->buf64, sym);
      CUDA_TRY(cols(s->n[1], c1, s->stream));
      auto c0 = cols_args<T>(s, 0, COL_FWD_MUL_INV, MUL_L, F_NOSTATE, s->buf64, sym);
      CUDA_TRY(cols(s->n[0], c0, s->stream));
      auto c2 = cols_args<T>(s, 1, COL_INV, MUL_L, F_NOSTATE, s->buf64, sym);
      CUDA_TRY(cols(s->n[1], c2, s->stream));
    }
    r.mode = R_IN_BUF | R_INV | R_OUT_RESID;
    CUDA_TRY(rows(nx, r, grid, s->stream));
  }
  // per-problem sums of the block partials (blocks never straddle problems)
  CUDA_TRY(launch_sum_pairs(s->partials, (int)(grid / s->B), s->B, s->red, s->stream));
  g_launches.fetch_add(nd == 1 ? 2 : (nd == 2 ? 4 : 6));
  return USP_OK;
}

// r = y - A x (or A x with apply_a): double-float unless the options ask
// for FP64.
static usp_status enqueue_residual64(usp_solver* s, const float2* x, const float2* y, float2* rout,
                                     bool apply_a) {
  if (s->opt.residual_fp64)
    return enqueue_residual_t<double>(s, x, y, rout, apply_a, s->symd, launch_rows_f64, launch_cols_f64);
  return enqueue_residual_t<dfl>(s, x, y, rout, apply_a, sym_df(s->symd), launch_rows_df, launch_cols_df);
}

// --------------------------------------------------------- create etc. ---

static void destroy_impl(usp_solver* s) {
  if (!s) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_graphs(s);
  cudaFree(s->V);
  cudaFree(s->buf);
  cudaFree(s->partials);
  cudaFree(s->st);
  cudaFreeHost(s->st_host);
  cudaFree(s->hist);
  cudaFree(s->red);
  cudaFreeHost(s->red_host);
  cudaFree(s->z);
  cudaFree(s->yp);
  cudaFree(s->ymask);
  cudaFree(s->buf64);
  cudaFree(s->hy);
  cudaFree(s->hx);
  cudaFree(s->bsym32);
  cudaFree(s->bsym64);
  cudaFree(s->balpha);
  cudaFree(s->bmask);
  cudaFreeHost(s->bmask_host);
  cudaFree(s->table);
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaSetDevice(cur);
  delete s;
}

// Create a solver for `count` independent problems on one grid (count == 1:
// the single-problem solver).  lsyms, alphas: host arrays of `count`.
static usp_status create_impl(const usp_grid* grid, int count, const usp_lsymbol* lsyms,
                              const void* V, int32_t V_is_real, const double* alphas,
                              void* cuda_stream, usp_solver** out) {
  if (!out) return fail(USP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !lsyms || !V || !alphas) return fail(USP_ERR_INVALID_ARG, "grid, lsym and V must be non-NULL");
  if (count < 1) return fail(USP_ERR_INVALID_ARG, "batch count must be >= 1 (got %d)", count);
  if (grid->ndim < 1 || grid->ndim > 3)
    return fail(USP_ERR_INVALID_ARG, "ndim must be 1, 2 or 3 (got %d)", grid->ndim);
  if (!(grid->dx > 0.0) || !std::isfinite(grid->dx))
    return fail(USP_ERR_INVALID_ARG, "dx must be finite and > 0");
  int64_t N = 1;
  for (int ax = 0; ax < grid->ndim; ++ax) {
    if (grid->n[ax] < 1) return fail(USP_ERR_INVALID_ARG, "axis %d has length %lld", ax, (long long)grid->n[ax]);
    if (!supported_length(grid->n[ax]))
      return fail(USP_ERR_UNSUPPORTED_SIZE,
                  "axis %d length %lld is not supported (powers of two in [2, 256], 96, 192, 384, 512)",
                  ax, (long long)grid->n[ax]);
    N *= grid->n[ax];
  }
  for (int p = 0; p < count; ++p) {
    const usp_lsymbol* lsym = lsyms + p;
    if (lsym->kind == USP_LSYM_TABLE) {
      // checked on the device after the copy (Re(Lhat + 1) > 0, finite)
      if (count != 1) return fail(USP_ERR_INVALID_ARG, "a tabulated symbol is single-problem only");
      if (!lsym->table) return fail(USP_ERR_INVALID_ARG, "USP_LSYM_TABLE needs a non-NULL table");
      if (std::isnan(alphas[p]) || std::isinf(alphas[p]) || alphas[p] > 2.0)
        return fail(USP_ERR_ALPHA_RANGE, "alpha must be finite and in (0, 2] (or <= 0 for automatic)");
      continue;
    }
    if (lsym->kind != USP_LSYM_QUADRATIC)
      return fail(USP_ERR_INVALID_ARG, "unknown symbol kind %d (problem %d)", (int)lsym->kind, p);
    const double sv[4] = {lsym->a_re, lsym->a_im, lsym->b_re, lsym->b_im};
    for (double v : sv)
      if (!std::isfinite(v)) return fail(USP_ERR_INVALID_ARG, "symbol coefficients must be finite (problem %d)", p);
    // Re(Lhat(p) + 1) > 0 on the grid: linear in |p|^2 in [0, ndim (pi/dx)^2].
    const double p2max = grid->ndim * (M_PI / grid->dx) * (M_PI / grid->dx);
    const double re0 = lsym->b_re + 1.0, re1 = lsym->a_re * p2max + lsym->b_re + 1.0;
    if (!(re0 > 0.0) || !(re1 > 0.0))
      return fail(USP_ERR_NOT_ACCRETIVE, "Re(Lhat(p)+1) <= 0 on the grid (%.3g at p=0, %.3g at |p|max; problem %d)",
                  re0, re1, p);
    if (std::isnan(alphas[p]) || std::isinf(alphas[p]) || alphas[p] > 2.0)
      return fail(USP_ERR_ALPHA_RANGE, "alpha must be finite and in (0, 2] (or <= 0 for automatic)");
  }
  if (count > 1) {
    // every block of the rows passes must hold rows of one problem
    const int nx = (int)grid->n[grid->ndim - 1];
    const int64_t rows_per = N / nx;
    const int64_t need = std::max<int64_t>(rows_per_block_f32(nx), rows_per_block_f64(nx));
    if (grid->ndim < 2 || rows_per % need != 0)
      return fail(USP_ERR_UNSUPPORTED_SIZE,
                  "a batch needs a 2-D or 3-D grid with a multiple of %lld lines per problem", (long long)need);
  }
  usp_status st0 = ensure_device_init();
  if (st0 != USP_OK) return st0;

  usp_solver* s = new usp_solver();
  s->B = count;
  s->ndim = grid->ndim;
  for (int ax = 0; ax < 3; ++ax) s->n[ax] = ax < grid->ndim ? (int)grid->n[ax] : 1;
  s->N = N;
  s->NB = N * count;
  s->dx = grid->dx;
  s->sym = lsyms[0];
  s->vreal = V_is_real != 0;
  s->user_stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&s->device);
  // symbol in both precisions (problem 0; batches use the per-problem arrays)
  const usp_lsymbol* lsym = lsyms;
  s->symd.a_re = lsym->a_re; s->symd.a_im = lsym->a_im;
  s->symd.b_re = lsym->b_re; s->symd.b_im = lsym->b_im;
  s->symd.inv_n = 1.0 / (double)N;
  s->symd.ndim = s->ndim;
  for (int ax = 0; ax < 3; ++ax) {
    s->symd.n[ax] = s->n[ax];
    s->symd.ks[ax] = 2.0 * M_PI / (s->n[ax] * grid->dx);
  }
  s->symf.a_re = (float)lsym->a_re; s->symf.a_im = (float)lsym->a_im;
  s->symf.b_re = (float)lsym->b_re; s->symf.b_im = (float)lsym->b_im;
  s->symf.inv_n = (float)(1.0 / (double)N);
  s->symf.ndim = s->ndim;
  for (int ax = 0; ax < 3; ++ax) {
    s->symf.n[ax] = s->n[ax];
    s->symf.ks[ax] = (float)s->symd.ks[ax];
  }

#define CREATE_TRY(call)                                                           \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      usp_status st_ = (e_ == cudaErrorMemoryAllocation) ? USP_ERR_OOM : USP_ERR_CUDA; \
      destroy_impl(s);                                                             \
      return fail(st_, "%s failed: %s", #call, cudaGetErrorString(e_));            \
    }                                                                              \
  } while (0)

  const int64_t NB = s->NB;
  CREATE_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  CREATE_TRY(cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming));
  const size_t esz = s->vreal ? sizeof(float) : sizeof(float2);
  const size_t vbytes = esz * (size_t)NB;
  CREATE_TRY(cudaMalloc(&s->V, vbytes));
  CREATE_TRY(cudaMalloc(&s->buf, sizeof(float2) * (size_t)NB));
  const int64_t g32 = rows_grid_f32(s), g64 = rows_grid_f64(s);
  // one per block of the rows passes, two per FP64 block, one per tile
  // (at least 8 lines) of the staged rows pass, three per statistics block
  s->npartials = std::max<int64_t>({g32, 2 * g64, NB / s->n[s->ndim - 1] / 8 + 1, 3 * 1024, 64});
  CREATE_TRY(cudaMalloc(&s->partials, sizeof(double) * s->npartials));
  CREATE_TRY(cudaMalloc(&s->st, sizeof(DevState) * count));
  CREATE_TRY(cudaMallocHost(&s->st_host, sizeof(DevState) * count));
  const size_t nred = std::max<size_t>(4, 2 * (size_t)count);
  CREATE_TRY(cudaMalloc(&s->red, nred * sizeof(double)));
  CREATE_TRY(cudaMallocHost(&s->red_host, nred * sizeof(double)));
  CREATE_TRY(cudaMemsetAsync(s->st, 0, sizeof(DevState) * count, s->stream));
  s->histories.assign(count, std::vector<double>());

  // copy V (ordered after the caller's queued work), then per-problem statistics
  CREATE_TRY(cudaEventRecord(s->ev, s->user_stream));
  CREATE_TRY(cudaStreamWaitEvent(s->stream, s->ev, 0));
  CREATE_TRY(launch_copy_bytes(s->V, V, vbytes, s->stream));
  const int nb = (int)std::min<int64_t>(1024, (N + 255) / 256);
  if (lsym->kind == USP_LSYM_TABLE) {
    CREATE_TRY(cudaMalloc(&s->table, sizeof(float2) * (size_t)N));
    CREATE_TRY(launch_copy_bytes(s->table, lsym->table, sizeof(float2) * (size_t)N, s->stream));
    CREATE_TRY(launch_table_stats(s->table, N, s->partials, nb, s->red, s->stream));
    g_launches.fetch_add(3);
    CREATE_TRY(cudaMemcpyAsync(s->red_host, s->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CREATE_TRY(cudaStreamSynchronize(s->stream));
    const double remin = s->red_host[0], bad = s->red_host[1];
    if (bad > 0) {
      destroy_impl(s);
      return fail(USP_ERR_NONFINITE, "the symbol table holds %.0f non-finite values", bad);
    }
    if (!(remin > 0.0)) {
      destroy_impl(s);
      return fail(USP_ERR_NOT_ACCRETIVE, "Re(Lhat(p)+1) = %.6g <= 0 in the symbol table", remin);
    }
    s->symf.table = s->table;
    s->symd.table = s->table;
  }
  s->alphas.assign(count, 0.0);
  for (int p = 0; p < count; ++p) {
    const void* Vp = static_cast<const char*>(s->V) + esz * (size_t)N * p;
    CREATE_TRY(launch_v_stats(Vp, s->vreal, N, s->partials, nb, s->red, s->stream));
    g_launches.fetch_add(2);
    CREATE_TRY(cudaMemcpyAsync(s->red_host, s->red, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CREATE_TRY(cudaStreamSynchronize(s->stream));
    const double vmax = s->red_host[0], astar = s->red_host[1], bad = s->red_host[2];
    if (bad > 0) {
      destroy_impl(s);
      return fail(USP_ERR_NONFINITE, "V holds %.0f non-finite values (problem %d)", bad, p);
    }
    if (!(vmax < 1.0)) {
      destroy_impl(s);
      return fail(USP_ERR_V_NOT_CONTRACTIVE, "max|V| = %.6g >= 1 (problem %d)", vmax, p);
    }
    s->vmax = std::max(s->vmax, vmax);
    s->alphas[p] = alphas[p] > 0.0 ? alphas[p] : astar;
  }
  s->alpha = s->alphas[0];
  if (count > 1) {
    std::vector<float4> h32(count);
    std::vector<double> h64(4 * (size_t)count);
    std::vector<float> ha(count);
    for (int p = 0; p < count; ++p) {
      h32[p] = make_float4((float)lsyms[p].a_re, (float)lsyms[p].a_im, (float)lsyms[p].b_re,
                           (float)lsyms[p].b_im);
      h64[4 * p] = lsyms[p].a_re;
      h64[4 * p + 1] = lsyms[p].a_im;
      h64[4 * p + 2] = lsyms[p].b_re;
      h64[4 * p + 3] = lsyms[p].b_im;
      ha[p] = (float)s->alphas[p];
    }
    CREATE_TRY(cudaMalloc(&s->bsym32, sizeof(float4) * count));
    CREATE_TRY(cudaMalloc(&s->bsym64, sizeof(double) * 4 * count));
    CREATE_TRY(cudaMalloc(&s->balpha, sizeof(float) * count));
    CREATE_TRY(cudaMalloc(&s->bmask, sizeof(int) * count));
    CREATE_TRY(cudaMallocHost(&s->bmask_host, sizeof(int) * count));
    CREATE_TRY(cudaMemcpy(s->bsym32, h32.data(), sizeof(float4) * count, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(s->bsym64, h64.data(), sizeof(double) * 4 * count, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(s->balpha, ha.data(), sizeof(float) * count, cudaMemcpyHostToDevice));
  }
  s->tw32 = twiddle_table_f32();
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  if (s->num_sms < 1) s->num_sms = 1;
  build_maps(s);
  if (count == 1 && s->ndim == 3 && s->n[1] == 256 && s->n[2] == 256)
    s->plane_clusters = plane_max_active_clusters();
  if (s->ndim == 2 && s->n[0] == s->n[1] && onchip_side(s->n[0])) {
    s->onchip_clusters[0] = onchip_clusters(s->n[0], 8, ONCHIP_SCALAR);
    s->onchip_clusters[1] = onchip_clusters(s->n[0], 16, ONCHIP_SCALAR);
  }
  *out = s;
  return USP_OK;
#undef CREATE_TRY
}

extern "C" usp_status usp_solver_create(const usp_grid* grid, const usp_lsymbol* lsym,
                                        const void* V, int32_t V_is_real, double alpha,
                                        void* cuda_stream, usp_solver** out) {
  return create_impl(grid, 1, lsym, V, V_is_real, &alpha, cuda_stream, out);
}

extern "C" usp_status usp_batch_create(const usp_grid* grid, int32_t count,
                                       const usp_lsymbol* lsyms, const void* V, int32_t V_is_real,
                                       const double* alphas, void* cuda_stream, usp_solver** out) {
  return create_impl(grid, count, lsyms, V, V_is_real, alphas, cuda_stream, out);
}

extern "C" usp_status usp_solver_set_options(usp_solver* s, const usp_options* opt) {
  if (!s || !opt) return fail(USP_ERR_INVALID_ARG, "NULL argument");
  if (opt->cols_tile != 0 && opt->cols_tile != 8 && opt->cols_tile != 16 && opt->cols_tile != 32)
    return fail(USP_ERR_INVALID_ARG, "cols_tile must be 0, 8, 16 or 32");
  if (opt->chunk < 0 || opt->max_refinements < 0 || opt->schedule < 0 || opt->schedule > 4)
    return fail(USP_ERR_INVALID_ARG, "invalid option value");
  if (opt->schedule == 2 && !fused_supported(s))
    return fail(USP_ERR_UNSUPPORTED_SIZE, "the fused schedule needs a 3-D grid nz x 256 x 256");
  if (opt->schedule == 4 && !split_supported(s))
    return fail(USP_ERR_UNSUPPORTED_SIZE,
                "the split schedule needs one 3-D problem on a grid nz x 256 x 256, nz in {32, 64, 128, 256}");
  if (opt->onchip_rows != 0 && opt->onchip_rows != 8 && opt->onchip_rows != 16)
    return fail(USP_ERR_INVALID_ARG, "onchip_rows must be 0, 8 or 16");
  if (opt->schedule == 3 && !onchip_available(s, onchip_rows_of(s, *opt)))
    return fail(USP_ERR_UNSUPPORTED_SIZE,
                "the on-chip schedule needs a 2-D grid n x n, n in {32, 64, 96, 128, 192, 256} (8 rows per CTA: "
                "n <= 128)");
  free_graphs(s);  // captured graphs follow the old schedule
  s->opt = *opt;
  return USP_OK;
}

extern "C" usp_status usp_solver_alpha(const usp_solver* s, double* alpha_out) {
  if (!s || !alpha_out) return fail(USP_ERR_INVALID_ARG, "NULL argument");
  *alpha_out = s->alpha;
  return USP_OK;
}

extern "C" void usp_solver_destroy(usp_solver* s) { destroy_impl(s); }

// -------------------------------------------------------------- solve ---

static usp_status ensure_hist(usp_solver* s, int cap) {
  if (s->hist_cap >= cap) return USP_OK;
  cudaFree(s->hist);
  s->hist = nullptr;
  s->hist_cap = 0;
  CUDA_TRY(cudaMalloc(&s->hist, sizeof(double) * (size_t)cap * s->B));
  s->hist_cap = cap;
  free_graphs(s);  // graphs captured the old pointer
  return USP_OK;
}

static usp_status get_graph(usp_solver* s, const float2* y, float2* x, int chunk,
                            cudaGraphExec_t* exec) {
  for (auto& g : s->graphs)
    if (g.y == y && g.x == x && g.chunk == chunk) {
      *exec = g.exec;
      return USP_OK;
    }
  if (s->graphs.size() >= 8) free_graphs(s);
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < chunk && e == cudaSuccess; ++i)
    e = enqueue_iteration(s, y, x, x, 0, s->stream, false);
  cudaError_t e2 = cudaStreamEndCapture(s->stream, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(USP_ERR_CUDA, "kernel launch during capture: %s", cudaGetErrorString(e));
  }
  CUDA_TRY(e2);
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, graph, 0);
  cudaGraphDestroy(graph);
  CUDA_TRY(e);
  s->graphs.push_back({y, x, chunk, ge});
  *exec = ge;
  return USP_OK;
}

static usp_status read_state(usp_solver* s) {
  CUDA_TRY(cudaMemcpyAsync(s->st_host, s->st, sizeof(DevState) * s->B, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return USP_OK;
}
static usp_status write_state(usp_solver* s) {
  CUDA_TRY(cudaMemcpyAsync(s->st, s->st_host, sizeof(DevState) * s->B, cudaMemcpyHostToDevice, s->stream));
  return USP_OK;
}

// Run iterations on (y, x) until every problem's device state says done.
static usp_status run_phase(usp_solver* s, const float2* y, float2* x, bool zero_start) {
  if (use_onchip(s)) {
    // one launch runs the phase to the end
    cudaError_t e = enqueue_onchip(s, y, x, x, zero_start ? F_XZERO : 0, s->stream);
    if (e != cudaSuccess) return fail(USP_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    usp_status st = read_state(s);
    if (st != USP_OK) return st;
    for (int p = 0; p < s->B; ++p)
      if (!s->st_host[p].done)
        return fail(USP_ERR_CUDA, "on-chip phase ended with a running problem (%d)", p);
    return USP_OK;
  }
  const int chunk = s->opt.chunk > 0 ? s->opt.chunk : 8;
  {
    usp_status st = prepare_source_mask(s, y, false);
    if (st != USP_OK) return st;
  }
  // the first iteration is launched directly (it may start from x = 0)
  {
    cudaError_t e = enqueue_iteration(s, y, x, x, zero_start ? F_XZERO : 0, s->stream, true, true);
    if (e != cudaSuccess) return fail(USP_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  }
  const int64_t passes_per_it = (int64_t)iteration_passes(s, y, x, x, 0).size();
  cudaGraphExec_t ge = nullptr;
  usp_status st = get_graph(s, y, x, chunk, &ge);
  if (st != USP_OK) return st;
  const int B = s->B;
  int launches = 1;
  std::vector<int> prev_it(B, 0);
  std::vector<double> prev_r(B, 0.0);
  // Every launched iteration either counts in a running problem's `it` or
  // finds it done, so more launched iterations than the largest remaining
  // budget (plus a chunk of slack) means the device state machine is
  // broken: stop, do not spin.
  int64_t budget = 0;
  for (int p = 0; p < B; ++p)
    if (!s->st_host[p].done)
      budget = std::max<int64_t>(budget, (int64_t)s->st_host[p].it_limit - s->st_host[p].it);
  budget += 2 * chunk + 1;
  int64_t launched = 1;
  for (;;) {
    for (int k = 0; k < launches; ++k) CUDA_TRY(cudaGraphLaunch(ge, s->stream));
    launched += (int64_t)launches * chunk;
    g_launches.fetch_add((int64_t)launches * chunk * passes_per_it);
    if ((st = read_state(s)) != USP_OK) return st;
    bool all_done = true;
    int want = 1, left_max = 1;
    for (int p = 0; p < B; ++p) {
      const DevState& h = s->st_host[p];
      if (h.done) continue;
      all_done = false;
      // Estimate the iterations left from the observed contraction rate and
      // size the next group of launches (slowest problem) to overshoot by at
      // most one chunk.
      int w = 4 * launches;
      if (prev_it[p] > 0 && h.it > prev_it[p] && h.last_r > 0 && prev_r[p] > h.last_r) {
        const double rate = std::pow(h.last_r / prev_r[p], 1.0 / (h.it - prev_it[p]));
        const double left = std::log(std::max(h.tol, 1e-300) / h.last_r) / std::log(rate);
        w = (int)std::ceil(std::max(1.0, left) / chunk);
      }
      want = std::max(want, w);
      left_max = std::max(left_max, h.it_limit - h.it);
      prev_it[p] = h.it;
      prev_r[p] = h.last_r;
    }
    if (all_done) return USP_OK;
    if (launched > budget) {
      const DevState& h = s->st_host[0];
      return fail(USP_ERR_CUDA, "device iteration state did not stop (it=%d of %d)", h.it, h.it_limit);
    }
    launches = std::min(std::max(want, 1), std::max(1, 512 / chunk));
    launches = std::min(launches, std::max(1, (left_max + chunk - 1) / chunk));
  }
}

static bool converged_state(const DevState& h, double tol) {
  return (h.status != ST_NONFINITE && h.status != ST_DIVERGED && h.status != ST_TIMEOUT) &&
         (h.it > 0 || h.ref == 0.0) && (h.last_r < tol || h.ref == 0.0);
}

// Status and message of one finished problem (prefix names it in a batch).
static usp_status problem_status(const DevState& h, double tol, bool stagnated, const char* prefix) {
  if (h.status == ST_TIMEOUT) return fail(USP_ERR_CUDA, "%sa bounded wait inside a kernel timed out (copy engine or cluster peer)", prefix);
  if (h.status == ST_NONFINITE) return fail(USP_ERR_NONFINITE, "%snon-finite value in y, x0 or an iterate", prefix);
  if (h.status == ST_DIVERGED)
    return fail(USP_ERR_DIVERGED, "%s||Delta|| grew from %.3g to %.3g (relative)", prefix, h.phase_first_r,
                h.last_r);
  if (!converged_state(h, tol))
    return fail(USP_ERR_NOT_CONVERGED, "%s%s after %d iterations, residual %.3g", prefix,
                stagnated ? "stagnated" : "iteration limit reached", h.it, h.last_r);
  return USP_OK;
}

// Solve all problems of the solver (one, or a batch sharing the passes).
// ref_norms: per problem (<= 0: automatic), or nullptr; outs, statuses: per
// problem, or nullptr.
static usp_status solve_impl(usp_solver* s, const float2* y, float2* x, int use_x0, double tol,
                             int maxit, const double* ref_norms, usp_result* outs,
                             usp_status* statuses) {
  usp_status st;
  if ((st = ensure_hist(s, maxit)) != USP_OK) return st;
  const int B = s->B;
  const bool refine = s->opt.plain == 0;
  const int max_ref = s->opt.max_refinements > 0 ? s->opt.max_refinements : 4;

  bool need_ref = false;
  for (int p = 0; p < B; ++p) {
    DevState& h = s->st_host[p];
    std::memset(&h, 0, sizeof h);
    h.it_limit = maxit;
    const double rn = ref_norms ? ref_norms[p] : 0.0;
    h.ref = rn > 0 ? rn : 0.0;
    h.tol = tol;
    need_ref = need_ref || !(rn > 0);
  }
  std::vector<int> refinements(B, 0), active(B, 1);
  std::vector<char> stagnated(B, 0);
  if (use_x0 && need_ref) {
    // ||B (L+I)^-1 y||: Delta at x = 0, no update (Algorithm 1's
    // denominator), for the problems without a given reference norm
    for (int p = 0; p < B; ++p) s->st_host[p].done = s->st_host[p].ref > 0 ? 1 : 0;
    if ((st = write_state(s)) != USP_OK) return st;
    cudaError_t e = enqueue_iteration(s, y, x, x, F_XZERO | F_REF, s->stream, true, true);
    if (e != cudaSuccess) return fail(USP_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    if ((st = read_state(s)) != USP_OK) return st;
    for (int p = 0; p < B; ++p) {
      DevState& h = s->st_host[p];
      const double rn = ref_norms ? ref_norms[p] : 0.0;
      if (rn > 0) h.done = 0;
      else if (h.done) active[p] = 0;  // non-finite y
    }
  }

  const float2* cy = y;  // source of the current phase
  float2* cx = x;        // unknown of the current phase (x, then the correction z)
  bool zero_start = !use_x0;
  std::vector<char> can_refine(B, 0);
  for (;;) {
    bool any = false;
    for (int p = 0; p < B; ++p) {
      DevState& h = s->st_host[p];
      if (!active[p] || h.it >= maxit) {
        active[p] = 0;
        h.done = 1;
        continue;
      }
      any = true;
      can_refine[p] = refine && refinements[p] < max_ref;
      h.done = 0;
      h.status = ST_RUNNING;
      h.phase_start = h.it;
      h.tol = (can_refine[p] && refinements[p] == 0) ? 8.0 * tol : tol;
      h.stall_window = can_refine[p] ? 64 : 0;
    }
    if (!any) break;
    if ((st = write_state(s)) != USP_OK) return st;
    if ((st = run_phase(s, cy, cx, zero_start)) != USP_OK) return st;
    if (cx != x) {
      // x = x_b + z for the problems of this phase
      if (B > 1) {
        for (int p = 0; p < B; ++p) s->bmask_host[p] = active[p];
        CUDA_TRY(cudaMemcpyAsync(s->bmask, s->bmask_host, sizeof(int) * B, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(launch_axpy1(x, cx, s->NB, s->stream, s->bmask, s->N));
      } else {
        CUDA_TRY(launch_axpy1(x, cx, s->NB, s->stream));
      }
      g_launches.fetch_add(1);
    }
    bool again = false;
    for (int p = 0; p < B; ++p) {
      if (!active[p]) continue;
      const DevState& h = s->st_host[p];
      const int stt = h.status;
      stagnated[p] = (stt == ST_STAGNATED);
      const bool terminal = stt == ST_NONFINITE || stt == ST_DIVERGED || stt == ST_MAXIT ||
                            stt == ST_TIMEOUT || h.last_r < tol || h.ref == 0.0 || !can_refine[p];
      if (terminal) active[p] = 0;
      else again = true;
    }
    if (!again) break;
    // Refinement: Delta(x_b + z; y) = Delta(z; y - A x_b) exactly because
    // A + B = L + I, so the same FP32 iteration continues on z with the
    // source y - A x_b formed in FP64.
    if (!s->z) CUDA_TRY(cudaMalloc(&s->z, sizeof(float2) * s->NB));
    if (!s->yp) CUDA_TRY(cudaMalloc(&s->yp, sizeof(float2) * s->NB));
    if ((st = enqueue_residual64(s, x, y, s->yp, false)) != USP_OK) return st;
    for (int p = 0; p < B; ++p)
      if (active[p]) ++refinements[p];
    cy = s->yp;
    cx = s->z;
    zero_start = true;
  }
  if ((st = read_state(s)) != USP_OK) return st;

  usp_status first_bad = USP_OK;
  std::string first_msg;
  for (int p = 0; p < B; ++p) {
    const DevState& h = s->st_host[p];
    const int nit = std::min(h.it, s->hist_cap);
    s->histories[p].assign(nit, 0.0);
    if (nit > 0)
      CUDA_TRY(cudaMemcpy(s->histories[p].data(), s->hist + (size_t)p * s->hist_cap, sizeof(double) * nit,
                          cudaMemcpyDeviceToHost));
    if (outs) {
      usp_result& o = outs[p];
      o.iterations = h.it;
      o.converged = converged_state(h, tol) ? 1 : 0;
      o.refinements = refinements[p];
      o.stagnated = stagnated[p] ? 1 : 0;
      o.final_rel_residual = h.last_r;
      o.ref_norm = h.ref;
      o.alpha = s->alphas[p];
    }
    char prefix[48] = "";
    if (B > 1) std::snprintf(prefix, sizeof prefix, "problem %d: ", p);
    const usp_status ps = problem_status(h, tol, stagnated[p] != 0, prefix);
    if (statuses) statuses[p] = ps;
    if (ps != USP_OK && first_bad == USP_OK) {
      first_bad = ps;
      first_msg = g_last_error;
    }
  }
  s->history = s->histories[0];
  if (first_bad != USP_OK) g_last_error = first_msg;
  return first_bad;
}

static usp_status check_solve_args(usp_solver* s, const void* y, void* x, double tol, int maxit) {
  if (!s) return fail(USP_ERR_INVALID_ARG, "solver is NULL");
  if (s->B > 1 && !(y && x)) return fail(USP_ERR_INVALID_ARG, "y and x must be non-NULL");
  if (!y || !x) return fail(USP_ERR_INVALID_ARG, "y and x must be non-NULL");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(USP_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (maxit < 1) return fail(USP_ERR_INVALID_ARG, "maxit must be >= 1");
  return USP_OK;
}

extern "C" usp_status usp_solve(usp_solver* s, const void* y, void* x, int32_t use_x0, double tol,
                                int32_t maxit, double ref_norm, usp_result* out) {
  usp_status st = check_solve_args(s, y, x, tol, maxit);
  if (st != USP_OK) return st;
  if (s->B > 1) return fail(USP_ERR_INVALID_ARG, "a batch solver is solved with usp_batch_solve");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) CUDA_TRY(cudaSetDevice(s->device));
  // order after the caller's queued work on its stream
  cudaError_t e = cudaEventRecord(s->ev, s->user_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev, 0);
  if (e != cudaSuccess) st = fail(USP_ERR_CUDA, "stream ordering: %s", cudaGetErrorString(e));
  if (st == USP_OK)
    st = solve_impl(s, (const float2*)y, (float2*)x, use_x0, tol, maxit, &ref_norm, out, nullptr);
  cudaStreamSynchronize(s->stream);
  if (cur != s->device) cudaSetDevice(cur);
  return st;
}

extern "C" usp_status usp_batch_solve(usp_solver* s, const void* y, void* x, int32_t use_x0,
                                      double tol, int32_t maxit, const double* ref_norms,
                                      usp_result* results, usp_status* statuses) {
  usp_status st = check_solve_args(s, y, x, tol, maxit);
  if (st != USP_OK) return st;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) CUDA_TRY(cudaSetDevice(s->device));
  cudaError_t e = cudaEventRecord(s->ev, s->user_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev, 0);
  if (e != cudaSuccess) st = fail(USP_ERR_CUDA, "stream ordering: %s", cudaGetErrorString(e));
  if (st == USP_OK)
    st = solve_impl(s, (const float2*)y, (float2*)x, use_x0, tol, maxit, ref_norms, results, statuses);
  cudaStreamSynchronize(s->stream);
  if (cur != s->device) cudaSetDevice(cur);
  return st;
}

extern "C" usp_status usp_solve_many(usp_solver* const* solvers, int32_t count,
                                     const void* const* ys, void* const* xs, int32_t use_x0,
                                     double tol, int32_t maxit, usp_result* results,
                                     usp_status* statuses) {
  if (count < 1 || !solvers || !ys || !xs) return fail(USP_ERR_INVALID_ARG, "bad argument");
  std::vector<int64_t> first(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    for (int j = 0; j < i; ++j)
      if (solvers[j] == solvers[i]) return fail(USP_ERR_INVALID_ARG, "solver %d is listed twice", i);
    usp_status st = check_solve_args(solvers[i], ys[i], xs[i], tol, maxit);
    if (st != USP_OK) return st;
    first[i + 1] = first[i] + solvers[i]->B;
  }
  // one host thread per solver: each drives its own stream and graphs, so
  // the solvers' passes run concurrently on the GPU
  std::vector<usp_status> st(count, USP_OK);
  std::vector<std::string> msg(count);
  auto run = [&](int i) {
    usp_solver* s = solvers[i];
    usp_result* r = results ? results + first[i] : nullptr;
    usp_status* ps = statuses ? statuses + first[i] : nullptr;
    if (cudaSetDevice(s->device) != cudaSuccess) {
      st[i] = fail(USP_ERR_CUDA, "cudaSetDevice(%d) failed", s->device);
    } else {
      cudaError_t e = cudaEventRecord(s->ev, s->user_stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev, 0);
      st[i] = e == cudaSuccess
                  ? solve_impl(s, (const float2*)ys[i], (float2*)xs[i], use_x0, tol, maxit,
                               nullptr, r, ps)
                  : fail(USP_ERR_CUDA, "stream ordering: %s", cudaGetErrorString(e));
      cudaStreamSynchronize(s->stream);
    }
    msg[i] = g_last_error;
  };
  int cur = 0;
  cudaGetDevice(&cur);
  std::vector<std::thread> threads;
  threads.reserve(count);
  for (int i = 1; i < count; ++i) threads.emplace_back(run, i);
  run(0);
  for (auto& t : threads) t.join();
  cudaSetDevice(cur);
  for (int i = 0; i < count; ++i)
    if (st[i] != USP_OK) {
      g_last_error = msg[i];
      return st[i];
    }
  return USP_OK;
}

extern "C" usp_status usp_batch_history(const usp_solver* s, int32_t problem, double* host_out,
                                        int32_t capacity, int32_t* n_out) {
  if (!s || !n_out) return fail(USP_ERR_INVALID_ARG, "NULL argument");
  if (problem < 0 || problem >= s->B)
    return fail(USP_ERR_INVALID_ARG, "problem %d out of range [0, %d)", problem, s->B);
  if (capacity > 0 && !host_out) return fail(USP_ERR_INVALID_ARG, "host_out is NULL");
  const std::vector<double>& h = s->histories[problem];
  const int n = (int)h.size();
  const int m = std::min(n, std::max(0, (int)capacity));
  if (m > 0) std::memcpy(host_out, h.data(), sizeof(double) * m);
  *n_out = n;
  return USP_OK;
}

extern "C" usp_status usp_solve_host(usp_solver* s, const void* y_host, void* x_host,
                                     int32_t use_x0, double tol, int32_t maxit, double ref_norm,
                                     usp_result* out) {
  usp_status st = check_solve_args(s, y_host, x_host, tol, maxit);
  if (st != USP_OK) return st;
  if (s->B > 1) return fail(USP_ERR_INVALID_ARG, "a batch solver is solved with usp_batch_solve");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) CUDA_TRY(cudaSetDevice(s->device));
  const size_t bytes = sizeof(float2) * (size_t)s->NB;
  if (!s->hy) CUDA_TRY(cudaMalloc(&s->hy, bytes));
  if (!s->hx) CUDA_TRY(cudaMalloc(&s->hx, bytes));
  CUDA_TRY(cudaMemcpyAsync(s->hy, y_host, bytes, cudaMemcpyHostToDevice, s->stream));
  if (use_x0) CUDA_TRY(cudaMemcpyAsync(s->hx, x_host, bytes, cudaMemcpyHostToDevice, s->stream));
  st = solve_impl(s, s->hy, s->hx, use_x0, tol, maxit, &ref_norm, out, nullptr);
  if (st == USP_OK || st == USP_ERR_NOT_CONVERGED) {
    const std::string keep = g_last_error;
    cudaError_t e = cudaMemcpyAsync(x_host, s->hx, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = fail(USP_ERR_CUDA, "copy back: %s", cudaGetErrorString(e));
    else g_last_error = keep;
  }
  cudaStreamSynchronize(s->stream);
  if (cur != s->device) cudaSetDevice(cur);
  return st;
}

extern "C" usp_status usp_residual_history(const usp_solver* s, double* host_out, int32_t capacity,
                                           int32_t* n_out) {
  if (!s || !n_out) return fail(USP_ERR_INVALID_ARG, "NULL argument");
  if (capacity > 0 && !host_out) return fail(USP_ERR_INVALID_ARG, "host_out is NULL");
  const int n = (int)s->history.size();
  const int m = std::min(n, std::max(0, (int)capacity));
  if (m > 0) std::memcpy(host_out, s->history.data(), sizeof(double) * m);
  *n_out = n;
  return USP_OK;
}

static usp_status residual_common(usp_solver* s, const void* x, const void* y, void* r, bool apply_a,
                                  double* rel_out) {
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) CUDA_TRY(cudaSetDevice(s->device));
  cudaError_t e = cudaEventRecord(s->ev, s->user_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev, 0);
  usp_status st = (e == cudaSuccess) ? USP_OK : fail(USP_ERR_CUDA, "stream ordering: %s", cudaGetErrorString(e));
  if (st == USP_OK) st = enqueue_residual64(s, (const float2*)x, (const float2*)y, (float2*)r, apply_a);
  if (st == USP_OK) {
    e = cudaMemcpyAsync(s->red_host, s->red, 2 * sizeof(double) * s->B, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = fail(USP_ERR_CUDA, "residual: %s", cudaGetErrorString(e));
  }
  if (st == USP_OK && rel_out) {
    double sr = 0.0, sy = 0.0;  // a batch: over all problems
    for (int p = 0; p < s->B; ++p) {
      sr += s->red_host[2 * p];
      sy += s->red_host[2 * p + 1];
    }
    const double nr = std::sqrt(sr), ny = std::sqrt(sy);
    *rel_out = ny > 0 ? nr / ny : nr;
  }
  cudaStreamSynchronize(s->stream);
  if (cur != s->device) cudaSetDevice(cur);
  return st;
}

extern "C" usp_status usp_apply_A(usp_solver* s, const void* x, void* Ax) {
  if (!s || !x || !Ax) return fail(USP_ERR_INVALID_ARG, "NULL argument");
  if (x == Ax) return fail(USP_ERR_INVALID_ARG, "Ax may not alias x");
  return residual_common(s, x, nullptr, Ax, true, nullptr);
}

extern "C" usp_status usp_residual(usp_solver* s, const void* x, const void* y, void* r,
                                   double* rel_out) {
  if (!s || !x || !y) return fail(USP_ERR_INVALID_ARG, "NULL argument");
  if (r && (r == x || r == y)) return fail(USP_ERR_INVALID_ARG, "r may not alias x or y");
  return residual_common(s, x, y, r, false, rel_out);
}

extern "C" const char* usp_status_string(usp_status st) {
  switch (st) {
    case USP_OK: return "USP_OK";
    case USP_ERR_INVALID_ARG: return "USP_ERR_INVALID_ARG";
    case USP_ERR_UNSUPPORTED_SIZE: return "USP_ERR_UNSUPPORTED_SIZE";
    case USP_ERR_V_NOT_CONTRACTIVE: return "USP_ERR_V_NOT_CONTRACTIVE";
    case USP_ERR_NOT_ACCRETIVE: return "USP_ERR_NOT_ACCRETIVE";
    case USP_ERR_ALPHA_RANGE: return "USP_ERR_ALPHA_RANGE";
    case USP_ERR_NOT_CONVERGED: return "USP_ERR_NOT_CONVERGED";
    case USP_ERR_DIVERGED: return "USP_ERR_DIVERGED";
    case USP_ERR_NONFINITE: return "USP_ERR_NONFINITE";
    case USP_ERR_CUDA: return "USP_ERR_CUDA";
    case USP_ERR_OOM: return "USP_ERR_OOM";
  }
  return "USP_ERR_UNKNOWN";
}

extern "C" const char* usp_last_error(void) { return g_last_error.c_str(); }

extern "C" int32_t usp_version(void) { return 100; }

extern "C" int64_t usp_kernel_launches(void) { return g_launches.load(); }

extern "C" usp_status usp_time_passes(usp_solver* s, const void* y, void* x, int32_t iters,
                                      usp_pass_time* out, int32_t capacity, int32_t* n_out) {
  if (!s || !y || !x || !n_out || iters < 1) return fail(USP_ERR_INVALID_ARG, "bad argument");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) CUDA_TRY(cudaSetDevice(s->device));
  usp_status st = ensure_hist(s, iters + 1);
  if (st != USP_OK) return st;
  for (int p = 0; p < s->B; ++p) {
    DevState& h = s->st_host[p];
    std::memset(&h, 0, sizeof h);
    h.it_limit = use_onchip(s) ? iters : iters + 2;  // on-chip: one launch runs them all
    h.ref = 1.0;   // fixed denominator: nothing stops the timed iterations
    h.tol = 0.0;
  }
  if ((st = write_state(s)) != USP_OK) return st;
  if ((st = prepare_source_mask(s, (const float2*)y, true)) != USP_OK) return st;
  if (use_onchip(s)) {
    // one launch of `iters` iterations; its mean per iteration
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    cudaError_t e = cudaEventRecord(e0, s->stream);
    if (e == cudaSuccess) e = enqueue_onchip(s, (const float2*)y, (const float2*)x, (float2*)x, 0, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(USP_ERR_CUDA, "timing launch: %s", cudaGetErrorString(e));
    if (capacity > 0) {
      std::memset(out[0].name, 0, sizeof out[0].name);
      std::strncpy(out[0].name, "onchip_iteration", sizeof out[0].name - 1);
      out[0].launches = 1;
      out[0].ms = ms / iters;
      out[0].bytes = 0.0;  // the fields stay on chip between iterations
    }
    *n_out = 1;
    if (cur != s->device) cudaSetDevice(cur);
    return USP_OK;
  }
  for (auto& p : prologue_passes(s, (const float2*)y, (const float2*)x, 0)) {
    cudaError_t e = p.go(s->stream);
    if (e != cudaSuccess) return fail(USP_ERR_CUDA, "prologue: %s", cudaGetErrorString(e));
    g_launches.fetch_add(1);
  }
  auto passes = iteration_passes(s, (const float2*)y, (const float2*)x, (float2*)x, 0);
  const size_t np = passes.size();
  // One untimed iteration goes first, and the timed ones are queued back to
  // back with one event between consecutive launches: each launch is then
  // already waiting when the event before it completes, so the events
  // bracket device time only, not the host's launch latency.
  std::vector<cudaEvent_t> ev((size_t)iters * np + 1, nullptr);
  usp_status res = USP_OK;
  for (auto& e : ev)
    if (res == USP_OK && cudaEventCreate(&e) != cudaSuccess) res = fail(USP_ERR_CUDA, "event create");
  std::vector<double> acc(np, 0.0);
  for (size_t k = 0; k < np && res == USP_OK; ++k) {
    if (passes[k].go(s->stream) != cudaSuccess) res = fail(USP_ERR_CUDA, "timing launch");
    g_launches.fetch_add(1);
  }
  if (res == USP_OK && cudaEventRecord(ev[0], s->stream) != cudaSuccess)
    res = fail(USP_ERR_CUDA, "timing event");
  for (int it = 0; it < iters && res == USP_OK; ++it) {
    for (size_t k = 0; k < np; ++k) {
      cudaError_t e = passes[k].go(s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(ev[(size_t)it * np + k + 1], s->stream);
      if (e != cudaSuccess) { res = fail(USP_ERR_CUDA, "timing launch: %s", cudaGetErrorString(e)); break; }
      g_launches.fetch_add(1);
    }
  }
  if (res == USP_OK) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) res = fail(USP_ERR_CUDA, "timing sync: %s", cudaGetErrorString(e));
  }
  for (int it = 0; it < iters && res == USP_OK; ++it)
    for (size_t k = 0; k < np; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[(size_t)it * np + k], ev[(size_t)it * np + k + 1]);
      acc[k] += ms;
    }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (res == USP_OK) {
    const int m = std::min<int>((int)np, std::max(0, (int)capacity));
    for (int k = 0; k < m; ++k) {
      std::memset(out[k].name, 0, sizeof out[k].name);
      std::strncpy(out[k].name, passes[k].name, sizeof out[k].name - 1);
      out[k].launches = iters;
      out[k].ms = acc[k] / iters;
      out[k].bytes = passes[k].bytes_per_point * (double)s->NB;
    }
    *n_out = (int32_t)np;
  }
  if (cur != s->device) cudaSetDevice(cur);
  return res;
}

// ------------------------------------------------------------ autotune ---

// Chosen options per (ndim, n0, n1, n2, problems, real V): the first solver of
// a shape is timed, later ones reuse the choice.
typedef std::tuple<int, int, int, int, int, int> TuneKey;
static std::map<TuneKey, usp_options> g_tuned;
static std::mutex g_tuned_mu;

extern "C" usp_status usp_autotune(usp_solver* s, const void* y, void* x, int32_t iters,
                                   usp_options* chosen) {
  if (!s || !y || !x || iters < 1) return fail(USP_ERR_INVALID_ARG, "bad argument");
  const TuneKey key{s->ndim, s->n[0], s->n[1], s->n[2], s->B, s->vreal ? 1 : 0};
  usp_options best = s->opt;
  {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      best = it->second;
      best.plain = s->opt.plain;
      best.max_refinements = s->opt.max_refinements;
      usp_status st = usp_solver_set_options(s, &best);
      if (st == USP_OK && chosen) *chosen = best;
      return st;
    }
  }
  // candidates: pass schedule x staged (TMA) or plain loads; the split and
  // on-chip schedules where the grid admits them
  std::vector<usp_options> cands;
  const int nx = s->n[s->ndim - 1];
  const bool staged = s->maps_ok || rows_tma_tile_rows(nx) > 0;
  for (int sched = 1; sched <= (fused_supported(s) ? 2 : 1); ++sched)
    for (int nt = 0; nt <= (staged ? 1 : 0); ++nt)
      for (int ct = (s->maps_ok && nt == 0 ? 8 : 16); ct <= (s->maps_ok && nt == 0 ? 32 : 16); ct *= 2) {
        usp_options o = s->opt;
        o.schedule = sched;
        o.no_tma = nt;
        o.cols_tile = ct;
        cands.push_back(o);
      }
  if (split_supported(s)) {
    usp_options o = s->opt;
    o.schedule = 4;
    o.no_tma = 0;
    o.cols_tile = 0;
    cands.push_back(o);
  }
  for (int rows = 8; rows <= 16; rows += 8)
    if (onchip_available(s, rows)) {
      usp_options o = s->opt;
      o.schedule = 3;
      o.onchip_rows = rows;
      cands.push_back(o);
    }
  const usp_options keep = s->opt;
  double best_ms = 1e300;
  for (const usp_options& o : cands) {
    usp_status st = usp_solver_set_options(s, &o);
    if (st != USP_OK) return st;
    usp_pass_time pt[16];
    int32_t np = 0;
    st = usp_time_passes(s, y, x, iters, pt, 16, &np);
    if (st != USP_OK) {
      usp_solver_set_options(s, &keep);
      return st;
    }
    double ms = 0.0;
    for (int k = 0; k < np && k < 16; ++k) ms += pt[k].ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = o;
    }
  }
  // iterations per graph launch: about 0.2 ms of GPU work between polls
  best.chunk = (int)std::min(64.0, std::max(4.0, std::round(0.2 / std::max(best_ms, 1e-6))));
  usp_status st = usp_solver_set_options(s, &best);
  if (st != USP_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned[key] = best;
  }
  if (chosen) *chosen = best;
  return USP_OK;
}
