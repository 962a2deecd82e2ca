// noalloc.cu -- usp_solve_noalloc: the plain FP32 fixed-point iteration for
// callers that cannot allocate device memory.
//
// Who needs this: a caller whose process has handed (nearly) all device
// memory to another allocator up front, or whose hot loop must not call
// cudaMalloc/cudaFree because those calls synchronise the device and can
// stall unrelated work.  Such a caller owns V, y and x but cannot let the
// library create a solver, which allocates its scratch field, reduction
// buffers and state.  This entry point instead works inside one fixed
// scratch area compiled into the library: a file-scope __device__ array of
// USP_NOALLOC_BYTES bytes (see usp.h).  CUDA may load the library's device
// code lazily, so the array may be reserved on a device only at the first
// call there (the symbol lookup loads the module); a failed reservation
// returns USP_ERR_OOM.  Once reserved, it stays until the process exits.
//
// The array's name is only a host-side stand-in in host code; its device
// address comes from cudaGetSymbolAddress, looked up once per device (with
// that device current) on the first call there and cached.  Every call uses
// the same array, so calls whose GPU work overlaps in time (two host threads,
// or two streams) race on it; the state block is rewritten at the start of
// each call, and the scratch field and partial sums are fully overwritten
// before they are read.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "usp.h"

using namespace usp;

namespace {

constexpr int64_t kMaxPoints = USP_NOALLOC_MAX_POINTS;
constexpr int kMaxIters = USP_NOALLOC_MAX_ITERS;
constexpr int64_t kPartials = 4096;  // >= rows-pass blocks and 3 x 1024 V statistics
constexpr size_t kFieldOff = 0;
constexpr size_t kPartialsOff = kFieldOff + sizeof(float2) * (size_t)kMaxPoints;
constexpr size_t kStateOff = kPartialsOff + sizeof(double) * (size_t)kPartials;
constexpr size_t kRedOff = kStateOff + 256;
constexpr size_t kHistOff = kRedOff + 256;
constexpr size_t kTotal = kHistOff + sizeof(double) * (size_t)kMaxIters;
static_assert(kTotal == USP_NOALLOC_BYTES, "usp.h states the scratch size");
static_assert(sizeof(DevState) <= 256, "state block");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kTotal];

namespace {

std::mutex g_mu;
void* g_base[64] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device: symbol lookup and the FFT twiddle tables).
usp_status scratch_base(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return USP_ERR_CUDA;
  if (dev < 0 || dev >= 64) return USP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error("usp_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? USP_ERR_OOM : USP_ERR_CUDA;
    }
    e = init_twiddles();
    if (e != cudaSuccess) {
      set_last_error("usp_solve_noalloc: twiddle set-up failed: %s", cudaGetErrorString(e));
      return USP_ERR_CUDA;
    }
    g_base[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_base[dev]);
  return USP_OK;
}

struct Ctx {
  int ndim;
  int n[3];
  int64_t N;
  bool vreal;
  const void* V;
  float2* field;
  double* partials;
  DevState* st;
  double* hist;
  float alpha;
  Sym<float> sym;
};

int64_t rows_grid(const Ctx& c) {
  const int nx = c.n[c.ndim - 1];
  const int F = rows_per_block_f32(nx);
  return (c.N / nx + F - 1) / F;
}

ColsArgs<float> cols(const Ctx& c, int axis, int mode) {
  ColsArgs<float> a{};
  a.mode = mode;
  a.mul = MUL_LINV;
  a.flags = 0;
  int64_t inner = 1, outer = 1;
  for (int ax = axis + 1; ax < c.ndim; ++ax) inner *= c.n[ax];
  for (int ax = 0; ax < axis; ++ax) outer *= c.n[ax];
  a.inner = inner;
  a.outer = outer;
  a.inner_blocks = (inner + 31) / 32;
  a.buf = c.field;
  a.st = c.st;
  a.sym = c.sym;
  return a;
}

// One iteration on the pencil schedule, launched directly (no graphs).
cudaError_t iteration(const Ctx& c, const float2* y, float2* x, int flags, cudaStream_t s) {
  const int nx = c.n[c.ndim - 1];
  RowsArgs<float> r{};
  r.flags = flags | (c.vreal ? F_VREAL : 0);
  r.nrows = c.N / nx;
  r.x_in = x;
  r.x_out = x;
  r.y = y;
  r.V = c.V;
  r.buf = c.field;
  r.partials = c.partials;
  r.st = c.st;
  r.hist = c.hist;
  r.alpha = c.alpha;
  r.sym = c.sym;
  r.mul = MUL_LINV;
  const int64_t grid = rows_grid(c);
  cudaError_t e;
  if (c.ndim == 1) {
    r.mode = R_IN_PRE | R_FWD | R_MUL | R_INV | R_OUT_POST;
    return launch_rows_f32(nx, r, grid, s);
  }
  r.mode = R_IN_PRE | R_FWD | R_OUT_BUF;
  if ((e = launch_rows_f32(nx, r, grid, s)) != cudaSuccess) return e;
  if (c.ndim == 2) {
    if ((e = launch_cols_f32(c.n[0], cols(c, 0, COL_FWD_MUL_INV), s)) != cudaSuccess) return e;
  } else {
    if ((e = launch_cols_f32(c.n[1], cols(c, 1, COL_FWD), s)) != cudaSuccess) return e;
    if ((e = launch_cols_f32(c.n[0], cols(c, 0, COL_FWD_MUL_INV), s)) != cudaSuccess) return e;
    if ((e = launch_cols_f32(c.n[1], cols(c, 1, COL_INV), s)) != cudaSuccess) return e;
  }
  r.mode = R_IN_BUF | R_INV | R_OUT_POST;
  return launch_rows_f32(nx, r, grid, s);
}

bool pow2_in_range(int64_t v) { return v >= 2 && v <= 256 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" usp_status usp_solve_noalloc(const usp_grid* grid, const usp_lsymbol* lsym,
                                        const void* V, int32_t V_is_real, double alpha,
                                        const void* y, void* x, double tol, int32_t maxit,
                                        void* cuda_stream, usp_result* out) {
  if (!grid || !lsym || !V || !y || !x) {
    set_last_error("usp_solve_noalloc: grid, lsym, V, y and x must be non-NULL");
    return USP_ERR_INVALID_ARG;
  }
  if (grid->ndim < 1 || grid->ndim > 3 || !(grid->dx > 0.0) || !std::isfinite(grid->dx)) {
    set_last_error("usp_solve_noalloc: ndim must be 1..3 and dx finite and > 0");
    return USP_ERR_INVALID_ARG;
  }
  if (!(tol >= 0.0) || !std::isfinite(tol) || maxit < 1) {
    set_last_error("usp_solve_noalloc: tol must be finite and >= 0, maxit >= 1");
    return USP_ERR_INVALID_ARG;
  }
  if (maxit > kMaxIters) {
    set_last_error("usp_solve_noalloc: maxit %d exceeds the fixed limit %d", maxit, kMaxIters);
    return USP_ERR_INVALID_ARG;
  }
  if (lsym->kind != USP_LSYM_QUADRATIC) {
    set_last_error("usp_solve_noalloc: only the quadratic symbol is supported (kind %d)", (int)lsym->kind);
    return USP_ERR_INVALID_ARG;
  }
  Ctx c{};
  c.ndim = grid->ndim;
  c.N = 1;
  for (int ax = 0; ax < 3; ++ax) {
    const int64_t n = ax < grid->ndim ? grid->n[ax] : 1;
    if (ax < grid->ndim && !pow2_in_range(n)) {
      set_last_error("usp_solve_noalloc: axis %d length %lld is not a power of two in [2, 256]",
                     ax, (long long)n);
      return USP_ERR_UNSUPPORTED_SIZE;
    }
    c.n[ax] = (int)n;
    c.N *= n;
  }
  if (c.N > kMaxPoints) {
    set_last_error("usp_solve_noalloc: the grid has %lld points; this entry point works in a "
                   "fixed scratch area for at most %lld points (use usp_solver_create)",
                   (long long)c.N, (long long)kMaxPoints);
    return USP_ERR_UNSUPPORTED_SIZE;
  }
  const double p2max = grid->ndim * (M_PI / grid->dx) * (M_PI / grid->dx);
  if (!(lsym->b_re + 1.0 > 0.0) || !(lsym->a_re * p2max + lsym->b_re + 1.0 > 0.0)) {
    set_last_error("usp_solve_noalloc: Re(Lhat(p)+1) <= 0 on the grid");
    return USP_ERR_NOT_ACCRETIVE;
  }
  if (std::isnan(alpha) || std::isinf(alpha) || alpha > 2.0) {
    set_last_error("usp_solve_noalloc: alpha must be finite and in (0, 2] (or <= 0)");
    return USP_ERR_ALPHA_RANGE;
  }
  unsigned char* base = nullptr;
  usp_status st = scratch_base(&base);
  if (st != USP_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c.vreal = V_is_real != 0;
  c.V = V;
  c.field = reinterpret_cast<float2*>(base + kFieldOff);
  c.partials = reinterpret_cast<double*>(base + kPartialsOff);
  c.st = reinterpret_cast<DevState*>(base + kStateOff);
  double* red = reinterpret_cast<double*>(base + kRedOff);
  c.hist = reinterpret_cast<double*>(base + kHistOff);
  c.sym.a_re = (float)lsym->a_re;
  c.sym.a_im = (float)lsym->a_im;
  c.sym.b_re = (float)lsym->b_re;
  c.sym.b_im = (float)lsym->b_im;
  c.sym.inv_n = (float)(1.0 / (double)c.N);
  c.sym.ndim = c.ndim;
  for (int ax = 0; ax < 3; ++ax) {
    c.sym.n[ax] = c.n[ax];
    c.sym.ks[ax] = (float)(2.0 * M_PI / (c.n[ax] * grid->dx));
  }

#define NA_TRY(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_last_error("usp_solve_noalloc: %s: %s", #call, cudaGetErrorString(e_));      \
      return USP_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

  // V statistics (validation and alpha*) in the scratch area
  const int nb = (int)std::min<int64_t>(1024, (c.N + 255) / 256);
  NA_TRY(launch_v_stats(V, c.vreal, c.N, c.partials, nb, red, s));
  double vs[3] = {0, 0, 0};
  NA_TRY(cudaMemcpyAsync(vs, red, sizeof vs, cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaStreamSynchronize(s));
  if (vs[2] > 0) {
    set_last_error("usp_solve_noalloc: V holds %.0f non-finite values", vs[2]);
    return USP_ERR_NONFINITE;
  }
  if (!(vs[0] < 1.0)) {
    set_last_error("usp_solve_noalloc: max|V| = %.6g >= 1", vs[0]);
    return USP_ERR_V_NOT_CONTRACTIVE;
  }
  const double a_used = alpha > 0.0 ? alpha : vs[1];
  c.alpha = (float)a_used;

  // the state block starts every call from zero (ticket, counters)
  DevState h;
  std::memset(&h, 0, sizeof h);
  h.it_limit = maxit;
  h.tol = tol;
  NA_TRY(cudaMemcpyAsync(c.st, &h, sizeof h, cudaMemcpyHostToDevice, s));

  NA_TRY(iteration(c, (const float2*)y, (float2*)x, F_XZERO, s));
  int batch = 4;
  int64_t launched = 1;
  for (;;) {
    NA_TRY(cudaMemcpyAsync(&h, c.st, sizeof h, cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (h.done) break;
    if (launched > (int64_t)maxit + 2 * batch + 1) {
      set_last_error("usp_solve_noalloc: device iteration state did not stop");
      return USP_ERR_CUDA;
    }
    for (int k = 0; k < batch; ++k) NA_TRY(iteration(c, (const float2*)y, (float2*)x, 0, s));
    launched += batch;
    batch = std::min(batch * 2, 64);
  }
#undef NA_TRY

  const bool converged =
      h.status != ST_NONFINITE && h.status != ST_DIVERGED && (h.last_r < tol || h.ref == 0.0);
  if (out) {
    out->iterations = h.it;
    out->converged = converged ? 1 : 0;
    out->refinements = 0;
    out->stagnated = 0;
    out->final_rel_residual = h.last_r;
    out->ref_norm = h.ref;
    out->alpha = a_used;
  }
  if (h.status == ST_NONFINITE) {
    set_last_error("usp_solve_noalloc: non-finite value in y or an iterate");
    return USP_ERR_NONFINITE;
  }
  if (h.status == ST_DIVERGED) {
    set_last_error("usp_solve_noalloc: ||Delta|| grew (relative %.3g)", h.last_r);
    return USP_ERR_DIVERGED;
  }
  if (!converged) {
    set_last_error("usp_solve_noalloc: iteration limit reached after %d iterations, residual %.3g",
                   h.it, h.last_r);
    return USP_ERR_NOT_CONVERGED;
  }
  return USP_OK;
}
