// variant_api.cpp -- runtime of the block forms of the canonical system
// (include/usp.h, "block variants"): Algorithm 1 in FP32 on an unknown of K
// components per point, one CUDA graph per group of iterations, the device
// iteration state of iteration_state.cuh.
//
// One iteration: t = B x + y (k_block_pre); forward transforms of the K
// planes (line pass, then the strided axes); (L^ + I)^-1 / N per frequency
// (k_block_mul); inverse transforms; Delta = B (u - x), x += alpha Delta,
// ||Delta|| and the stopping test (k_block_post).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "block_kernels.h"
#include "kernels.h"
#include "usp.h"

using namespace usp;

namespace {

usp_status vfail(usp_status st, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error("%s: %s", usp_status_string(st), buf);
  return st;
}

#define V_TRY(call)                                                                \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return vfail(e_ == cudaErrorMemoryAllocation ? USP_ERR_OOM : USP_ERR_CUDA,   \
                   "%s failed: %s", #call, cudaGetErrorString(e_));                \
  } while (0)

bool supported(int64_t v) {
  const bool pow2 = v >= 2 && v <= 256 && (v & (v - 1)) == 0;
  return pow2 || v == 96 || v == 192 || v == 384 || v == 512;
}

struct Graph {
  const float2* y;
  float2* x;
  int chunk;
  cudaGraphExec_t exec;
};

}  // namespace

struct usp_variant {
  int kind = 0, K = 0, ndim = 0, n[3] = {1, 1, 1};
  int64_t N = 0;
  int device = 0;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev = nullptr;
  float2 *V = nullptr, *buf = nullptr;
  DevState *st = nullptr, *st_host = nullptr;
  double *partials = nullptr, *hist = nullptr, *red = nullptr, *red_host = nullptr;
  int hist_cap = 0;
  double alpha = 0.0;
  BlockArgs base{};
  std::vector<double> history;
  std::vector<Graph> graphs;
  int schedule = 0;       // 0 automatic, 1 passes, 3 on-chip
  int onchip = 0;         // co-resident clusters of the on-chip kernel (0: unavailable)
  const float2* tw = nullptr;
};

// The on-chip kernel (onchip_kernels.cu) for square 2-D grids up to 128^2.
static bool onchip_available(const usp_variant* s) { return s->onchip > 0; }
static bool use_onchip(const usp_variant* s) {
  return onchip_available(s) && (s->schedule == 0 || s->schedule == 3);
}
static cudaError_t enqueue_onchip(usp_variant* s, const float2* y, const float2* xin, float2* xout,
                                  int flags, cudaStream_t strm) {
  OnchipArgs o{};
  o.kind = s->kind == USP_VARIANT_ANTISYMMETRIC ? ONCHIP_ANTISYMMETRIC : ONCHIP_FLUX;
  o.flags = flags;
  o.x_in = xin;
  o.x_out = xout;
  o.y = y;
  o.V = s->V;
  o.tw = s->tw;
  o.st = s->st;
  o.hist = s->hist;
  o.alpha = (float)s->alpha;
  o.sym.ndim = s->ndim;
  for (int ax = 0; ax < 3; ++ax) {
    o.sym.n[ax] = s->n[ax];
    o.sym.ks[ax] = s->base.ks[ax];
  }
  o.sym.inv_n = s->base.inv_n;
  for (int i = 0; i < 4; ++i) o.bsym[i] = s->base.sym[i];
  return launch_onchip(s->n[0], 8, o, 1, strm);
}

static void free_graphs(usp_variant* s) {
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

static void vdestroy(usp_variant* s) {
  if (!s) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_graphs(s);
  cudaFree(s->V);
  cudaFree(s->buf);
  cudaFree(s->st);
  cudaFree(s->partials);
  cudaFree(s->hist);
  cudaFree(s->red);
  cudaFreeHost(s->st_host);
  cudaFreeHost(s->red_host);
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaSetDevice(cur);
  delete s;
}

// The launches of one iteration on (y, xin -> xout).
static cudaError_t enqueue_iteration(usp_variant* s, const float2* y, const float2* xin,
                                     float2* xout, int flags, cudaStream_t strm) {
  BlockArgs a = s->base;
  a.y = y;
  a.x_in = xin;
  a.x_out = xout;
  a.flags = flags;
  cudaError_t e = launch_block_pre(a, strm);
  const int nd = s->ndim, nx = s->n[nd - 1];
  RowsArgs<float> r{};
  r.nrows = s->K * s->N / nx;
  r.buf = s->buf;
  r.st = s->st;
  const int64_t rgrid = (r.nrows + rows_per_block_f32(nx) - 1) / rows_per_block_f32(nx);
  auto cols = [&](int axis, int mode) {
    ColsArgs<float> c{};
    c.mode = mode;
    int64_t inner = 1, outer = s->K;
    for (int ax = axis + 1; ax < nd; ++ax) inner *= s->n[ax];
    for (int ax = 0; ax < axis; ++ax) outer *= s->n[ax];
    const int cpb = cols_per_block(s->n[axis]);
    c.inner = inner;
    c.outer = outer;
    c.inner_blocks = (inner + cpb - 1) / cpb;
    c.buf = s->buf;
    c.st = s->st;
    return launch_cols_f32(s->n[axis], c, strm);
  };
  r.mode = R_IN_BUF | R_FWD | R_OUT_BUF;
  if (e == cudaSuccess) e = launch_rows_f32(nx, r, rgrid, strm);
  for (int axis = nd - 2; axis >= 0 && e == cudaSuccess; --axis) e = cols(axis, COL_FWD);
  if (e == cudaSuccess) e = launch_block_mul(a, strm);
  for (int axis = 0; axis <= nd - 2 && e == cudaSuccess; ++axis) e = cols(axis, COL_INV);
  r.mode = R_IN_BUF | R_INV | R_OUT_BUF;
  if (e == cudaSuccess) e = launch_rows_f32(nx, r, rgrid, strm);
  if (e == cudaSuccess) e = launch_block_post(a, strm);
  return e;
}

extern "C" usp_status usp_variant_create(const usp_grid* grid, int32_t kind, const double* params,
                                         const void* V, double alpha, void* cuda_stream,
                                         usp_variant** out) {
  if (!out) return vfail(USP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !params || !V) return vfail(USP_ERR_INVALID_ARG, "grid, params and V must be non-NULL");
  if (kind != USP_VARIANT_ANTISYMMETRIC && kind != USP_VARIANT_FLUX_DIFFUSION)
    return vfail(USP_ERR_INVALID_ARG, "unknown variant %d", kind);
  if (grid->ndim < 1 || grid->ndim > 3) return vfail(USP_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
  if (!(grid->dx > 0.0) || !std::isfinite(grid->dx)) return vfail(USP_ERR_INVALID_ARG, "dx must be > 0");
  int64_t N = 1;
  for (int ax = 0; ax < grid->ndim; ++ax) {
    if (!supported(grid->n[ax]))
      return vfail(USP_ERR_UNSUPPORTED_SIZE, "axis %d length %lld is not supported", ax,
                   (long long)grid->n[ax]);
    N *= grid->n[ax];
  }
  const int np = kind == USP_VARIANT_ANTISYMMETRIC ? 4 : 3;
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(params[i])) return vfail(USP_ERR_INVALID_ARG, "parameters must be finite");
  if (kind == USP_VARIANT_FLUX_DIFFUSION && !(params[0] >= 1.0 && params[1] >= 1.0 && params[2] > 0.0))
    return vfail(USP_ERR_NOT_ACCRETIVE, "flux form needs alpha >= 1, beta >= 1, s > 0 (Re L >= 0)");
  if (std::isnan(alpha) || std::isinf(alpha) || alpha > 2.0)
    return vfail(USP_ERR_ALPHA_RANGE, "alpha must be finite and in (0, 2] (or <= 0 for automatic)");
  V_TRY(init_twiddles());

  usp_variant* s = new usp_variant();
  s->kind = kind;
  s->ndim = grid->ndim;
  for (int ax = 0; ax < grid->ndim; ++ax) s->n[ax] = (int)grid->n[ax];
  s->N = N;
  s->K = kind == USP_VARIANT_ANTISYMMETRIC ? 2 : 1 + grid->ndim;
  s->user_stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&s->device);
#define VC_TRY(call)                                                               \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      vdestroy(s);                                                                 \
      return vfail(e_ == cudaErrorMemoryAllocation ? USP_ERR_OOM : USP_ERR_CUDA,   \
                   "%s failed: %s", #call, cudaGetErrorString(e_));                \
    }                                                                              \
  } while (0)
  const int nb = block_grid(N);
  VC_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  VC_TRY(cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming));
  VC_TRY(cudaMalloc(&s->V, sizeof(float2) * N));
  VC_TRY(cudaMalloc(&s->buf, sizeof(float2) * N * s->K));
  VC_TRY(cudaMalloc(&s->st, sizeof(DevState)));
  VC_TRY(cudaMalloc(&s->partials, sizeof(double) * 3 * nb));
  VC_TRY(cudaMalloc(&s->red, 4 * sizeof(double)));
  VC_TRY(cudaMallocHost(&s->st_host, sizeof(DevState)));
  VC_TRY(cudaMallocHost(&s->red_host, 4 * sizeof(double)));
  VC_TRY(cudaMemsetAsync(s->st, 0, sizeof(DevState), s->stream));
  VC_TRY(cudaEventRecord(s->ev, s->user_stream));
  VC_TRY(cudaStreamWaitEvent(s->stream, s->ev, 0));
  if (kind == USP_VARIANT_ANTISYMMETRIC) {
    VC_TRY(cudaMemcpyAsync(s->V, V, sizeof(float2) * N, cudaMemcpyDeviceToDevice, s->stream));
  } else {
    const float* vp = static_cast<const float*>(V);
    VC_TRY(launch_pack2(vp, vp + N, N, s->V, s->stream));
  }
  BlockArgs& a = s->base;
  a.kind = kind == USP_VARIANT_ANTISYMMETRIC ? BLOCK_ANTISYMMETRIC : BLOCK_FLUX;
  a.K = s->K;
  a.ndim = s->ndim;
  for (int ax = 0; ax < 3; ++ax) {
    a.n[ax] = s->n[ax];
    a.ks[ax] = (float)(2.0 * M_PI / (s->n[ax] * grid->dx));
  }
  a.N = N;
  a.inv_n = (float)(1.0 / (double)N);
  for (int i = 0; i < np; ++i) a.sym[i] = (float)params[i];
  a.V = s->V;
  a.buf = s->buf;
  a.st = s->st;
  a.partials = s->partials;
  VC_TRY(launch_block_stats(a, s->partials, s->red, s->stream));
  VC_TRY(cudaMemcpyAsync(s->red_host, s->red, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  VC_TRY(cudaStreamSynchronize(s->stream));
  const double astar = s->red_host[0], vmax = s->red_host[1], bad = s->red_host[2];
  if (bad > 0) {
    vdestroy(s);
    return vfail(USP_ERR_NONFINITE, "V holds %.0f non-finite values", bad);
  }
  if (!(vmax < 1.0)) {
    vdestroy(s);
    return vfail(USP_ERR_V_NOT_CONTRACTIVE, "max ||V|| = %.6g >= 1", vmax);
  }
  s->alpha = alpha > 0.0 ? alpha : astar;
  a.alpha = (float)s->alpha;
  s->tw = twiddle_table_f32();
  if (s->ndim == 2 && s->n[0] == s->n[1] && s->n[0] <= 128 && s->tw)
    s->onchip = onchip_clusters(s->n[0], 8, kind == USP_VARIANT_ANTISYMMETRIC ? ONCHIP_ANTISYMMETRIC : ONCHIP_FLUX);
#undef VC_TRY
  *out = s;
  return USP_OK;
}

extern "C" void usp_variant_destroy(usp_variant* s) { vdestroy(s); }

extern "C" usp_status usp_variant_set_schedule(usp_variant* s, int32_t schedule) {
  if (!s) return vfail(USP_ERR_INVALID_ARG, "NULL solver");
  if (schedule != 0 && schedule != 1 && schedule != 3) return vfail(USP_ERR_INVALID_ARG, "schedule must be 0, 1 or 3");
  if (schedule == 3 && !onchip_available(s))
    return vfail(USP_ERR_UNSUPPORTED_SIZE, "the on-chip schedule needs a 2-D grid n x n, n in {32, 64, 128}");
  s->schedule = schedule;
  return USP_OK;
}

static usp_status ensure_hist(usp_variant* s, int cap) {
  if (s->hist_cap >= cap) return USP_OK;
  free_graphs(s);
  cudaFree(s->hist);
  s->hist = nullptr;
  s->hist_cap = 0;
  V_TRY(cudaMalloc(&s->hist, sizeof(double) * cap));
  s->hist_cap = cap;
  s->base.hist = s->hist;
  return USP_OK;
}

static usp_status read_state(usp_variant* s) {
  V_TRY(cudaMemcpyAsync(s->st_host, s->st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
  V_TRY(cudaStreamSynchronize(s->stream));
  return USP_OK;
}

static usp_status get_graph(usp_variant* s, const float2* y, float2* x, int chunk,
                            cudaGraphExec_t* exec) {
  for (auto& g : s->graphs)
    if (g.y == y && g.x == x && g.chunk == chunk) {
      *exec = g.exec;
      return USP_OK;
    }
  if (s->graphs.size() >= 8) free_graphs(s);
  cudaGraph_t graph = nullptr;
  V_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < chunk && e == cudaSuccess; ++i) e = enqueue_iteration(s, y, x, x, 0, s->stream);
  cudaError_t e2 = cudaStreamEndCapture(s->stream, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return vfail(USP_ERR_CUDA, "launch during capture: %s", cudaGetErrorString(e));
  }
  V_TRY(e2);
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, graph, 0);
  cudaGraphDestroy(graph);
  V_TRY(e);
  s->graphs.push_back({y, x, chunk, ge});
  *exec = ge;
  return USP_OK;
}

static usp_status vsolve(usp_variant* s, const float2* y, float2* x, int use_x0, double tol,
                         int maxit, double ref_norm, usp_result* out) {
  usp_status st = ensure_hist(s, maxit);
  if (st != USP_OK) return st;
  DevState& h = *s->st_host;
  std::memset(&h, 0, sizeof h);
  h.it_limit = maxit;
  h.ref = ref_norm > 0 ? ref_norm : 0.0;
  h.tol = tol;
  V_TRY(cudaMemcpyAsync(s->st, s->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s->stream));
  bool skip = false;
  const bool oc = use_onchip(s);
  if (use_x0 && !(ref_norm > 0)) {
    // Algorithm 1's denominator ||B (L+I)^-1 y||: Delta at x = 0, no update
    V_TRY(oc ? enqueue_onchip(s, y, x, x, F_XZERO | F_REF, s->stream)
             : enqueue_iteration(s, y, x, x, F_XZERO | F_REF, s->stream));
    if ((st = read_state(s)) != USP_OK) return st;
    skip = h.done != 0;
  }
  if (!skip && oc) {
    // one launch runs the solve to the end
    V_TRY(enqueue_onchip(s, y, x, x, use_x0 ? 0 : F_XZERO, s->stream));
    if ((st = read_state(s)) != USP_OK) return st;
    if (!h.done) return vfail(USP_ERR_CUDA, "on-chip solve ended with the state running");
  } else if (!skip) {
    V_TRY(enqueue_iteration(s, y, x, x, use_x0 ? 0 : F_XZERO, s->stream));
    const int chunk = 8;
    cudaGraphExec_t ge = nullptr;
    if ((st = get_graph(s, y, x, chunk, &ge)) != USP_OK) return st;
    int64_t launched = 1;
    int group = 1;
    for (;;) {
      if ((st = read_state(s)) != USP_OK) return st;
      if (h.done) break;
      if (launched > (int64_t)maxit + 2 * chunk + 1)
        return vfail(USP_ERR_CUDA, "device iteration state did not stop (it=%d of %d)", h.it, maxit);
      const int left = std::max(1, (h.it_limit - h.it + chunk - 1) / chunk);
      group = std::min(std::min(group * 2, 64), left);
      for (int k = 0; k < group; ++k) V_TRY(cudaGraphLaunch(ge, s->stream));
      launched += (int64_t)group * chunk;
    }
  }
  if ((st = read_state(s)) != USP_OK) return st;
  const int nit = std::min(h.it, s->hist_cap);
  s->history.assign(nit, 0.0);
  if (nit > 0) V_TRY(cudaMemcpy(s->history.data(), s->hist, sizeof(double) * nit, cudaMemcpyDeviceToHost));
  const bool converged = h.status != ST_NONFINITE && h.status != ST_DIVERGED && h.status != ST_TIMEOUT &&
                         (h.it > 0 || h.ref == 0.0) &&
                         (h.last_r < tol || h.ref == 0.0);
  if (out) {
    out->iterations = h.it;
    out->converged = converged ? 1 : 0;
    out->refinements = 0;
    out->stagnated = 0;
    out->final_rel_residual = h.last_r;
    out->ref_norm = h.ref;
    out->alpha = s->alpha;
  }
  if (h.status == ST_TIMEOUT) return vfail(USP_ERR_CUDA, "a bounded wait inside a kernel timed out");
  if (h.status == ST_NONFINITE) return vfail(USP_ERR_NONFINITE, "non-finite value in y, x0 or an iterate");
  if (h.status == ST_DIVERGED)
    return vfail(USP_ERR_DIVERGED, "||Delta|| grew from %.3g to %.3g (relative)", h.phase_first_r, h.last_r);
  if (!converged)
    return vfail(USP_ERR_NOT_CONVERGED, "iteration limit reached after %d iterations, residual %.3g", h.it,
                 h.last_r);
  return USP_OK;
}

extern "C" usp_status usp_variant_solve(usp_variant* s, const void* y, void* x, int32_t use_x0,
                                        double tol, int32_t maxit, double ref_norm,
                                        usp_result* out) {
  if (!s || !y || !x) return vfail(USP_ERR_INVALID_ARG, "NULL argument");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return vfail(USP_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (maxit < 1) return vfail(USP_ERR_INVALID_ARG, "maxit must be >= 1");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) V_TRY(cudaSetDevice(s->device));
  cudaError_t e = cudaEventRecord(s->ev, s->user_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev, 0);
  usp_status st = e == cudaSuccess ? vsolve(s, (const float2*)y, (float2*)x, use_x0, tol, maxit, ref_norm, out)
                                   : vfail(USP_ERR_CUDA, "stream ordering: %s", cudaGetErrorString(e));
  cudaStreamSynchronize(s->stream);
  if (cur != s->device) cudaSetDevice(cur);
  return st;
}

extern "C" usp_status usp_variant_history(const usp_variant* s, double* host_out, int32_t capacity,
                                          int32_t* n_out) {
  if (!s || !n_out) return vfail(USP_ERR_INVALID_ARG, "NULL argument");
  if (capacity > 0 && !host_out) return vfail(USP_ERR_INVALID_ARG, "host_out is NULL");
  const int n = (int)s->history.size();
  const int m = std::min(n, std::max(0, (int)capacity));
  if (m > 0) std::memcpy(host_out, s->history.data(), sizeof(double) * m);
  *n_out = n;
  return USP_OK;
}
