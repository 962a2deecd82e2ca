// fno_api.cpp -- runtime of the warm-start network (include/usp.h, "learned
// initial estimate"): parameters, Adam state and activations in device
// memory, the forward pass, the hand-derived backward pass and the Adam step
// as sequences of fno_kernels.cu launches on the network's own stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fno_kernels.h"
#include "kernels.h"
#include "usp.h"

using namespace usp;

namespace {

usp_status ffail(usp_status st, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error("%s: %s", usp_status_string(st), buf);
  return st;
}

#define FNO_TRY(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ffail(e_ == cudaErrorMemoryAllocation ? USP_ERR_OOM : USP_ERR_CUDA,   \
                   "%s failed: %s", #call, cudaGetErrorString(e_));                \
  } while (0)

constexpr int MAX_LAYERS = 8;

// Unit roots e^{-2 pi i k(s) n / N} for the retained mode slots s, laid out
// [n][s] (k(s) = s for s < modes/2, else N - modes + s).
std::vector<float2> mode_roots(int N, int modes) {
  std::vector<float2> t((size_t)N * modes);
  const double two_pi = 6.283185307179586476925286766559;
  for (int n = 0; n < N; ++n)
    for (int s = 0; s < modes; ++s) {
      const int k = s < modes / 2 ? s : N - modes + s;
      const long e = ((long)k * n) % N;
      t[(size_t)n * modes + s] = make_float2((float)std::cos(two_pi * e / N),
                                             (float)-std::sin(two_pi * e / N));
    }
  return t;
}

// splitmix64: the parameter initialiser's generator
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform(uint64_t& s) { return (splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

struct usp_fno {
  usp_fno_config cfg{};
  int device = 0;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev = nullptr;
  int64_t P = 0, mm = 0, nparam = 0, step = 0;
  int64_t off_P = 0, off_p = 0, off_W[MAX_LAYERS]{}, off_b[MAX_LAYERS]{}, off_R[MAX_LAYERS]{},
          off_Q = 0, off_q = 0;
  float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
  float2 *twh = nullptr, *tww = nullptr;
  float* v[MAX_LAYERS]{};   // layer inputs v_0 .. v_{L-1}
  float* z[MAX_LAYERS]{};   // pre-activations z_0 .. z_{L-1} (z_{L-1} = v_L)
  float2* X[MAX_LAYERS]{};  // retained modes of v_l
  float2 *Zm = nullptr, *G = nullptr, *xh = nullptr, *gu = nullptr;
  float *gvA = nullptr, *gvB = nullptr, *wpart = nullptr;
  double *lpart = nullptr, *dloss = nullptr, *hloss = nullptr;
};

static void fno_free(usp_fno* f) {
  if (!f) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(f->device);
  if (f->stream) cudaStreamSynchronize(f->stream);
  void* ptrs[] = {f->params, f->grads, f->am,  f->av,    f->twh,   f->tww,   f->Zm,   f->G,
                  f->xh,     f->gu,    f->gvA, f->gvB,   f->wpart, f->lpart, f->dloss};
  for (void* p : ptrs) cudaFree(p);
  for (int l = 0; l < MAX_LAYERS; ++l) {
    cudaFree(f->v[l]);
    cudaFree(f->z[l]);
    cudaFree(f->X[l]);
  }
  cudaFreeHost(f->hloss);
  if (f->ev) cudaEventDestroy(f->ev);
  if (f->stream) cudaStreamDestroy(f->stream);
  cudaSetDevice(cur);
  delete f;
}

static usp_status check_config(const usp_fno_config* c) {
  if (!c) return ffail(USP_ERR_INVALID_ARG, "config is NULL");
  if (c->h < 8 || c->h > 512 || c->w < 8 || c->w > 512)
    return ffail(USP_ERR_UNSUPPORTED_SIZE, "image %d x %d outside [8, 512]", c->h, c->w);
  if (c->c_in < 1 || c->c_in > 8) return ffail(USP_ERR_INVALID_ARG, "c_in must be in [1, 8]");
  if (c->width < 1 || c->width > 64) return ffail(USP_ERR_INVALID_ARG, "width must be in [1, 64]");
  if (c->layers < 1 || c->layers > MAX_LAYERS)
    return ffail(USP_ERR_INVALID_ARG, "layers must be in [1, %d]", MAX_LAYERS);
  const int m = c->modes;
  if (m < 2 || m > 32 || (m & (m - 1)) != 0 || m > c->h || m > c->w)
    return ffail(USP_ERR_INVALID_ARG, "modes must be a power of two in [2, 32], <= h and w");
  if (c->max_batch < 1) return ffail(USP_ERR_INVALID_ARG, "max_batch must be >= 1");
  if (fno_smem_bytes(c->h, c->w, m) > 200 * 1024)
    return ffail(USP_ERR_UNSUPPORTED_SIZE, "the spectral layer's tables exceed shared memory");
  return USP_OK;
}

extern "C" int64_t usp_fno_param_count(const usp_fno_config* c) {
  if (check_config(c) != USP_OK) return -1;
  const int64_t w = c->width, m = c->modes;
  return w * c->c_in + w + c->layers * (w * w + w + w * w * m * m * 2) + 2 * w + 2;
}

extern "C" usp_status usp_fno_create(const usp_fno_config* cfg, uint64_t seed, void* cuda_stream,
                                     usp_fno** out) {
  if (!out) return ffail(USP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  usp_status st = check_config(cfg);
  if (st != USP_OK) return st;
  usp_fno* f = new usp_fno();
  f->cfg = *cfg;
  cudaGetDevice(&f->device);
  f->user_stream = (cudaStream_t)cuda_stream;
  const int64_t w = cfg->width, L = cfg->layers, B = cfg->max_batch;
  f->P = (int64_t)cfg->h * cfg->w;
  f->mm = (int64_t)cfg->modes * cfg->modes;
  int64_t k = 0;
  f->off_P = k; k += w * cfg->c_in;
  f->off_p = k; k += w;
  for (int l = 0; l < L; ++l) {
    f->off_W[l] = k; k += w * w;
    f->off_b[l] = k; k += w;
    f->off_R[l] = k; k += w * w * f->mm * 2;
  }
  f->off_Q = k; k += 2 * w;
  f->off_q = k; k += 2;
  f->nparam = k;

#define ALLOC(ptr, bytes)                                                          \
  do {                                                                             \
    cudaError_t e_ = cudaMalloc(&(ptr), (bytes));                                  \
    if (e_ != cudaSuccess) {                                                       \
      fno_free(f);                                                                 \
      return ffail(USP_ERR_OOM, "allocating %s: %s", #ptr, cudaGetErrorString(e_)); \
    }                                                                              \
  } while (0)
  const size_t act = sizeof(float) * (size_t)(B * w * f->P);
  ALLOC(f->params, sizeof(float) * k);
  ALLOC(f->grads, sizeof(float) * k);
  ALLOC(f->am, sizeof(float) * k);
  ALLOC(f->av, sizeof(float) * k);
  ALLOC(f->twh, sizeof(float2) * cfg->h * cfg->modes);
  ALLOC(f->tww, sizeof(float2) * cfg->w * cfg->modes);
  for (int l = 0; l < L; ++l) {
    ALLOC(f->v[l], act);
    ALLOC(f->z[l], act);
    ALLOC(f->X[l], sizeof(float2) * (size_t)(B * w * f->mm));
  }
  ALLOC(f->Zm, sizeof(float2) * (size_t)(B * w * f->mm));
  ALLOC(f->G, sizeof(float2) * (size_t)(B * w * f->mm));
  ALLOC(f->xh, sizeof(float2) * (size_t)(B * f->P));
  ALLOC(f->gu, sizeof(float2) * (size_t)(B * f->P));
  ALLOC(f->gvA, act);
  ALLOC(f->gvB, act);
  ALLOC(f->wpart, sizeof(float) * fno_wgrad_partials(64, 64));
  ALLOC(f->lpart, sizeof(double) * fno_loss_partials((int)B));
  ALLOC(f->dloss, sizeof(double));
#undef ALLOC
  if (cudaMallocHost(&f->hloss, sizeof(double)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->ev, cudaEventDisableTiming) != cudaSuccess) {
    fno_free(f);
    return ffail(USP_ERR_CUDA, "stream/event/pinned allocation failed");
  }
  // unit-root tables and the seeded initial parameters
  const std::vector<float2> th = mode_roots(cfg->h, cfg->modes), tw = mode_roots(cfg->w, cfg->modes);
  std::vector<float> h((size_t)k, 0.f);
  uint64_t s = seed;
  auto fill = [&](int64_t off, int64_t n, double a) {
    for (int64_t i = 0; i < n; ++i) h[off + i] = (float)(a * (2.0 * uniform(s) - 1.0));
  };
  fill(f->off_P, w * cfg->c_in, 1.0 / std::sqrt((double)cfg->c_in));
  for (int l = 0; l < L; ++l) {
    fill(f->off_W[l], w * w, 1.0 / std::sqrt((double)w));
    fill(f->off_R[l], w * w * f->mm * 2, 1.0 / (double)(w * w));
  }
  fill(f->off_Q, 2 * w, 1.0 / std::sqrt((double)w));
  cudaError_t e = cudaMemcpy(f->twh, th.data(), sizeof(float2) * th.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->tww, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->params, h.data(), sizeof(float) * k, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(f->am, 0, sizeof(float) * k);
  if (e == cudaSuccess) e = cudaMemset(f->av, 0, sizeof(float) * k);
  if (e != cudaSuccess) {
    fno_free(f);
    return ffail(USP_ERR_CUDA, "initialising the network: %s", cudaGetErrorString(e));
  }
  *out = f;
  return USP_OK;
}

extern "C" void usp_fno_destroy(usp_fno* f) { fno_free(f); }

extern "C" usp_status usp_fno_get_params(const usp_fno* f, float* host_out, int64_t n) {
  if (!f || !host_out) return ffail(USP_ERR_INVALID_ARG, "NULL argument");
  if (n != f->nparam) return ffail(USP_ERR_INVALID_ARG, "expected %lld parameters", (long long)f->nparam);
  FNO_TRY(cudaStreamSynchronize(f->stream));
  FNO_TRY(cudaMemcpy(host_out, f->params, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return USP_OK;
}

extern "C" usp_status usp_fno_set_params(usp_fno* f, const float* host_in, int64_t n) {
  if (!f || !host_in) return ffail(USP_ERR_INVALID_ARG, "NULL argument");
  if (n != f->nparam) return ffail(USP_ERR_INVALID_ARG, "expected %lld parameters", (long long)f->nparam);
  FNO_TRY(cudaStreamSynchronize(f->stream));
  FNO_TRY(cudaMemcpy(f->params, host_in, sizeof(float) * n, cudaMemcpyHostToDevice));
  FNO_TRY(cudaMemset(f->am, 0, sizeof(float) * n));
  FNO_TRY(cudaMemset(f->av, 0, sizeof(float) * n));
  f->step = 0;
  return USP_OK;
}

// ------------------------------------------------------------ passes ---

static CStrided planar_c(const float* p, int64_t C, int64_t P) { return CStrided{p, C * P, P, 1}; }
static Strided planar(float* p, int64_t C, int64_t P) { return Strided{p, C * P, P, 1}; }

// Forward pass on a (batch x c_in x H x W, device) into f->xh, keeping every
// activation for the backward pass.
static cudaError_t forward(usp_fno* f, const float* a, int B) {
  const usp_fno_config& c = f->cfg;
  const int w = c.width, L = c.layers;
  const int64_t P = f->P;
  const float inv = 1.f / (float)P;
  cudaStream_t s = f->stream;
  cudaError_t e = fno_conv(planar_c(a, c.c_in, P), c.c_in, f->params + f->off_P, c.c_in, 1,
                           f->params + f->off_p, planar(f->v[0], w, P), w, B, P, false, s);
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    e = fno_dft2(f->v[l], (int64_t)B * w, c.h, c.w, c.modes, f->twh, f->tww, f->X[l], s);
    if (e == cudaSuccess)
      e = fno_mix(f->X[l], f->params + f->off_R[l], B, w, w, (int)f->mm, false, f->Zm, s);
    if (e == cudaSuccess)
      e = fno_conv(planar_c(f->v[l], w, P), w, f->params + f->off_W[l], w, 1,
                   f->params + f->off_b[l], planar(f->z[l], w, P), w, B, P, false, s);
    if (e == cudaSuccess)
      e = fno_idft2(f->Zm, (int64_t)B * w, c.h, c.w, c.modes, f->twh, f->tww, inv, f->z[l],
                    l + 1 < L ? f->v[l + 1] : nullptr, s);
  }
  if (e == cudaSuccess)
    e = fno_conv(planar_c(f->z[L - 1], w, P), w, f->params + f->off_Q, w, 1, f->params + f->off_q,
                 Strided{reinterpret_cast<float*>(f->xh), 2 * P, 1, 2}, 2, B, P, false, s);
  return e;
}

// Loss against x (batch x H x W complex64, device) and the backward pass
// into f->grads.
static cudaError_t backward(usp_fno* f, const float* a, const float2* x, int B) {
  const usp_fno_config& c = f->cfg;
  const int w = c.width, L = c.layers;
  const int64_t P = f->P;
  const float inv = 1.f / (float)P;
  cudaStream_t s = f->stream;
  float* g = f->grads;
  cudaError_t e = fno_loss(f->xh, x, B, P, f->lpart, f->dloss, f->gu, s);
  const CStrided gu2{reinterpret_cast<const float*>(f->gu), 2 * P, 1, 2};
  // projection: dQ, dq; gv = Q^T gu
  if (e == cudaSuccess)
    e = fno_wgrad(gu2, 2, planar_c(f->z[L - 1], w, P), w, B, P, f->wpart, g + f->off_Q,
                  g + f->off_q, s);
  float* gv = f->gvA;
  float* gn = f->gvB;
  if (e == cudaSuccess)
    e = fno_conv(gu2, 2, f->params + f->off_Q, 1, w, nullptr, planar(gv, w, P), w, B, P, false, s);
  for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
    if (l + 1 < L) e = fno_gelu_bwd(gv, f->z[l], (int64_t)B * w * P, s);   // gv -> dL/dz_l
    if (e == cudaSuccess)
      e = fno_wgrad(planar_c(gv, w, P), w, planar_c(f->v[l], w, P), w, B, P, f->wpart,
                    g + f->off_W[l], g + f->off_b[l], s);
    if (e == cudaSuccess)
      e = fno_dft2(gv, (int64_t)B * w, c.h, c.w, c.modes, f->twh, f->tww, f->G, s);
    if (e == cudaSuccess) e = fno_dR(f->G, f->X[l], B, w, w, (int)f->mm, inv, g + f->off_R[l], s);
    if (e == cudaSuccess)
      e = fno_mix(f->G, f->params + f->off_R[l], B, w, w, (int)f->mm, true, f->Zm, s);
    if (e == cudaSuccess)
      e = fno_conv(planar_c(gv, w, P), w, f->params + f->off_W[l], 1, w, nullptr,
                   planar(gn, w, P), w, B, P, false, s);
    if (e == cudaSuccess)
      e = fno_idft2(f->Zm, (int64_t)B * w, c.h, c.w, c.modes, f->twh, f->tww, inv, gn, nullptr, s);
    float* t = gv;
    gv = gn;
    gn = t;
  }
  if (e == cudaSuccess)
    e = fno_wgrad(planar_c(gv, w, P), w, planar_c(a, c.c_in, P), c.c_in, B, P, f->wpart,
                  g + f->off_P, g + f->off_p, s);
  return e;
}

static usp_status begin(usp_fno* f, const void* a, int batch, int* cur) {
  if (!f || !a) return ffail(USP_ERR_INVALID_ARG, "NULL argument");
  if (batch < 1 || batch > f->cfg.max_batch)
    return ffail(USP_ERR_INVALID_ARG, "batch %d outside [1, %d]", batch, f->cfg.max_batch);
  cudaGetDevice(cur);
  if (*cur != f->device) FNO_TRY(cudaSetDevice(f->device));
  FNO_TRY(cudaEventRecord(f->ev, f->user_stream));
  FNO_TRY(cudaStreamWaitEvent(f->stream, f->ev, 0));
  return USP_OK;
}

static usp_status finish(usp_fno* f, cudaError_t e, int cur, double* loss_out) {
  if (e == cudaSuccess && loss_out)
    e = cudaMemcpyAsync(f->hloss, f->dloss, sizeof(double), cudaMemcpyDeviceToHost, f->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
  if (cur != f->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return ffail(USP_ERR_CUDA, "network pass: %s", cudaGetErrorString(e));
  if (loss_out) *loss_out = *f->hloss;
  return USP_OK;
}

extern "C" usp_status usp_fno_predict(usp_fno* f, const float* a, int32_t batch, void* x_out) {
  if (!x_out) return ffail(USP_ERR_INVALID_ARG, "x_out is NULL");
  int cur = 0;
  usp_status st = begin(f, a, batch, &cur);
  if (st != USP_OK) return st;
  cudaError_t e = forward(f, a, batch);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x_out, f->xh, sizeof(float2) * (size_t)(batch * f->P),
                        cudaMemcpyDeviceToDevice, f->stream);
  return finish(f, e, cur, nullptr);
}

extern "C" usp_status usp_fno_gradients(usp_fno* f, const float* a, const void* x_true,
                                        int32_t batch, float* grad_host, double* loss_out) {
  if (!x_true) return ffail(USP_ERR_INVALID_ARG, "x_true is NULL");
  int cur = 0;
  usp_status st = begin(f, a, batch, &cur);
  if (st != USP_OK) return st;
  cudaError_t e = forward(f, a, batch);
  if (e == cudaSuccess) e = backward(f, a, (const float2*)x_true, batch);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, f->grads, sizeof(float) * f->nparam, cudaMemcpyDeviceToHost,
                        f->stream);
  return finish(f, e, cur, loss_out);
}

extern "C" usp_status usp_fno_train_step(usp_fno* f, const float* a, const void* x_true,
                                         int32_t batch, double lr, double* loss_out) {
  if (!x_true || !(lr > 0.0)) return ffail(USP_ERR_INVALID_ARG, "x_true NULL or lr <= 0");
  int cur = 0;
  usp_status st = begin(f, a, batch, &cur);
  if (st != USP_OK) return st;
  cudaError_t e = forward(f, a, batch);
  if (e == cudaSuccess) e = backward(f, a, (const float2*)x_true, batch);
  if (e == cudaSuccess) {
    const double b1 = 0.9, b2 = 0.999;
    const int64_t t = ++f->step;
    e = fno_adam(f->params, f->grads, f->am, f->av, f->nparam, (float)lr, (float)b1, (float)b2,
                 1e-8f, (float)(1.0 / (1.0 - std::pow(b1, (double)t))),
                 (float)(1.0 / (1.0 - std::pow(b2, (double)t))), f->stream);
  }
  return finish(f, e, cur, loss_out);
}
