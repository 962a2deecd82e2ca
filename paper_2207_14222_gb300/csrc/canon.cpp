// canon.cpp -- conversion of a physical problem to the canonical form the
// solver takes (paper Sec. 2.2 and 3.1), on the host in FP64.
//
// Helmholtz  laplacian(psi) + k^2 psi = -S :
//   kbar2, rho = centre and radius of the smallest circle enclosing the
//   values k^2(r) (the smallest-circle problem), c = i rho / norm_v so that
//   max |V| = norm_v and A is accretive for a gain-free medium;
//   V = (k^2 - kbar2)/c,  y = -S/c,  Lhat = (-|p|^2 + kbar2)/c.
// Diffusion  -D laplacian(u) + eta u = S  (scalar constant D):
//   etabar, rho = midpoint and half-range of eta, c = rho / norm_v;
//   V = (eta - etabar)/c,  y = S/c,  Lhat = (D |p|^2 + etabar)/c.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "usp.h"

namespace {

typedef std::complex<double> cd;

struct Circle {
  cd c;
  double r;
};

inline bool contains(const Circle& C, cd p) {
  return std::abs(p - C.c) <= C.r * (1.0 + 1e-12) + 1e-300;
}

Circle from2(cd a, cd b) {
  const cd c = 0.5 * (a + b);
  return {c, std::abs(a - c)};
}

// Circumcircle; for (near-)collinear points the widest pair circle.
Circle from3(cd a, cd b, cd c) {
  const double ax = a.real(), ay = a.imag(), bx = b.real(), by = b.imag();
  const double cx = c.real(), cy = c.imag();
  const double d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by));
  if (d == 0.0) {
    Circle best = from2(a, b);
    const Circle c2 = from2(a, c), c3 = from2(b, c);
    if (c2.r > best.r) best = c2;
    if (c3.r > best.r) best = c3;
    return best;
  }
  const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
  const double ux = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / d;
  const double uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d;
  const cd o(ux, uy);
  return {o, std::max({std::abs(a - o), std::abs(b - o), std::abs(c - o)})};
}

// splitmix64: a fixed-seed shuffle keeps the result reproducible.
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Welzl's randomised incremental smallest enclosing circle, expected O(n).
Circle smallest_circle(std::vector<cd>& P) {
  uint64_t seed = 0x5EED5EEDull;
  for (size_t i = P.size(); i > 1; --i) std::swap(P[i - 1], P[splitmix(seed) % i]);
  Circle C{P[0], 0.0};
  for (size_t i = 1; i < P.size(); ++i) {
    if (contains(C, P[i])) continue;
    C = {P[i], 0.0};
    for (size_t j = 0; j < i; ++j) {
      if (contains(C, P[j])) continue;
      C = from2(P[i], P[j]);
      for (size_t k = 0; k < j; ++k) {
        if (contains(C, P[k])) continue;
        C = from3(P[i], P[j], P[k]);
      }
    }
  }
  return C;
}

}  // namespace

extern "C" usp_status usp_canon_helmholtz(const double* k2, const double* S, int64_t n,
                                          double norm_v, float* V_out, float* y_out,
                                          usp_lsymbol* lsym_out, double* c_out,
                                          double* bias_out) {
  if (!k2 || !S || !V_out || !y_out || !lsym_out || n < 1) return USP_ERR_INVALID_ARG;
  if (!(norm_v > 0.0 && norm_v < 1.0)) return USP_ERR_INVALID_ARG;
  std::vector<cd> P((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    P[i] = cd(k2[2 * i], k2[2 * i + 1]);
    if (!std::isfinite(P[i].real()) || !std::isfinite(P[i].imag())) return USP_ERR_NONFINITE;
  }
  std::sort(P.begin(), P.end(), [](cd a, cd b) {
    return a.real() < b.real() || (a.real() == b.real() && a.imag() < b.imag());
  });
  P.erase(std::unique(P.begin(), P.end()), P.end());
  const Circle C = smallest_circle(P);
  const double rho = C.r;
  if (!(rho > 0.0)) return USP_ERR_INVALID_ARG;  // homogeneous medium
  const cd c(0.0, rho / norm_v);                  // c = -rho/(norm_v i)
  const cd inv_c = 1.0 / c;
  for (int64_t i = 0; i < n; ++i) {
    const cd v = (cd(k2[2 * i], k2[2 * i + 1]) - C.c) * inv_c;
    const cd yv = -cd(S[2 * i], S[2 * i + 1]) * inv_c;
    V_out[2 * i] = (float)v.real();
    V_out[2 * i + 1] = (float)v.imag();
    y_out[2 * i] = (float)yv.real();
    y_out[2 * i + 1] = (float)yv.imag();
  }
  const cd a = -inv_c, b = C.c * inv_c;
  lsym_out->a_re = a.real();
  lsym_out->a_im = a.imag();
  lsym_out->b_re = b.real();
  lsym_out->b_im = b.imag();
  lsym_out->kind = USP_LSYM_QUADRATIC;
  lsym_out->table = nullptr;
  if (c_out) {
    c_out[0] = c.real();
    c_out[1] = c.imag();
  }
  if (bias_out) {
    bias_out[0] = C.c.real();
    bias_out[1] = C.c.imag();
  }
  return USP_OK;
}

extern "C" usp_status usp_canon_diffusion(const double* eta, double D, const double* S, int64_t n,
                                          double norm_v, float* V_out, float* y_out,
                                          usp_lsymbol* lsym_out, double* c_out,
                                          double* bias_out) {
  if (!eta || !S || !V_out || !y_out || !lsym_out || n < 1) return USP_ERR_INVALID_ARG;
  if (!(norm_v > 0.0 && norm_v < 1.0) || !(D > 0.0)) return USP_ERR_INVALID_ARG;
  double lo = eta[0], hi = eta[0];
  for (int64_t i = 0; i < n; ++i) {
    if (!std::isfinite(eta[i])) return USP_ERR_NONFINITE;
    lo = std::min(lo, eta[i]);
    hi = std::max(hi, eta[i]);
  }
  const double etabar = 0.5 * (lo + hi), rho = 0.5 * (hi - lo);
  if (!(rho > 0.0)) return USP_ERR_INVALID_ARG;
  const double c = rho / norm_v;
  for (int64_t i = 0; i < n; ++i) {
    V_out[i] = (float)((eta[i] - etabar) / c);
    y_out[2 * i] = (float)(S[2 * i] / c);
    y_out[2 * i + 1] = (float)(S[2 * i + 1] / c);
  }
  lsym_out->a_re = D / c;
  lsym_out->a_im = 0.0;
  lsym_out->b_re = etabar / c;
  lsym_out->b_im = 0.0;
  lsym_out->kind = USP_LSYM_QUADRATIC;
  lsym_out->table = nullptr;
  if (c_out) {
    c_out[0] = c;
    c_out[1] = 0.0;
  }
  if (bias_out) {
    bias_out[0] = etabar;
    bias_out[1] = 0.0;
  }
  return USP_OK;
}

// Antisymmetrised form (Sec. 2.2, Eq. antisymmetrised) of laplacian psi +
// k^2 psi = -S with the adjoint source S_adj (NULL: 0):
//   kbar2, rho as above, c = rho / norm_v (real), v = (k^2 - kbar2)/c,
//   l = (-|p|^2 + kbar2)/c  (params = a_re, a_im, b_re, b_im of l),
//   y = [S_adj / c ; -S / c]  (= [-y0' ; y0] / c with y0 = -S).
extern "C" usp_status usp_canon_antisymmetric(const double* k2, const double* S,
                                              const double* S_adj, int64_t n, double norm_v,
                                              float* v_out, float* y_out, double* params_out,
                                              double* c_out) {
  if (!k2 || !S || !v_out || !y_out || !params_out || n < 1) return USP_ERR_INVALID_ARG;
  if (!(norm_v > 0.0 && norm_v < 1.0)) return USP_ERR_INVALID_ARG;
  std::vector<cd> P((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    P[i] = cd(k2[2 * i], k2[2 * i + 1]);
    if (!std::isfinite(P[i].real()) || !std::isfinite(P[i].imag())) return USP_ERR_NONFINITE;
  }
  std::sort(P.begin(), P.end(), [](cd a, cd b) {
    return a.real() < b.real() || (a.real() == b.real() && a.imag() < b.imag());
  });
  P.erase(std::unique(P.begin(), P.end()), P.end());
  const Circle C = smallest_circle(P);
  if (!(C.r > 0.0)) return USP_ERR_INVALID_ARG;  // homogeneous medium
  const double c = C.r / norm_v;
  for (int64_t i = 0; i < n; ++i) {
    const cd v = (cd(k2[2 * i], k2[2 * i + 1]) - C.c) / c;
    v_out[2 * i] = (float)v.real();
    v_out[2 * i + 1] = (float)v.imag();
    const cd ya = S_adj ? cd(S_adj[2 * i], S_adj[2 * i + 1]) / c : cd(0.0, 0.0);
    const cd y1 = -cd(S[2 * i], S[2 * i + 1]) / c;
    y_out[2 * i] = (float)ya.real();
    y_out[2 * i + 1] = (float)ya.imag();
    y_out[2 * (n + i)] = (float)y1.real();
    y_out[2 * (n + i) + 1] = (float)y1.imag();
  }
  params_out[0] = -1.0 / c;
  params_out[1] = 0.0;
  params_out[2] = C.c.real() / c;
  params_out[3] = C.c.imag() / c;
  if (c_out) c_out[0] = c;
  return USP_OK;
}

// Flux form of steady diffusion -div(D grad u) + eta u = S (Sec. 3.2, Eq.
// diffusion-equation-matrix-form, d/dt = 0, scalar D(r) > 0): etabar,
// Dinvbar = midpoints of the ranges of eta and 1/D, r_eta, r_D their
// half-ranges; C = diag(c_u, c_J I) with c_u = r_eta / norm_v, c_J = r_D /
// norm_v (a block with zero range takes the other's scale);
//   V planes: Vu = (eta - etabar)/c_u, VJ = (1/D - Dinvbar)/c_J;
//   params = (etabar/c_u + 1, Dinvbar/c_J + 1, 1/sqrt(c_u c_J));
//   y = [S / sqrt(c_u); 0 (ndim planes)];  scales = (c_u, c_J).
extern "C" usp_status usp_canon_flux_diffusion(const double* eta, const double* D,
                                               const double* S, int64_t n, int32_t ndim,
                                               double norm_v, float* V_out, float* y_out,
                                               double* params_out, double* scales_out) {
  if (!eta || !D || !S || !V_out || !y_out || !params_out || n < 1 || ndim < 1 || ndim > 3)
    return USP_ERR_INVALID_ARG;
  if (!(norm_v > 0.0 && norm_v < 1.0)) return USP_ERR_INVALID_ARG;
  double e0 = eta[0], e1 = eta[0], d0 = 1.0 / D[0], d1 = 1.0 / D[0];
  for (int64_t i = 0; i < n; ++i) {
    if (!std::isfinite(eta[i]) || !std::isfinite(D[i]) || !std::isfinite(S[i])) return USP_ERR_NONFINITE;
    if (eta[i] < 0.0 || !(D[i] > 0.0)) return USP_ERR_INVALID_ARG;
    e0 = std::min(e0, eta[i]);
    e1 = std::max(e1, eta[i]);
    d0 = std::min(d0, 1.0 / D[i]);
    d1 = std::max(d1, 1.0 / D[i]);
  }
  const double etabar = 0.5 * (e0 + e1), r_eta = 0.5 * (e1 - e0);
  const double dbar = 0.5 * (d0 + d1), r_d = 0.5 * (d1 - d0);
  if (!(r_eta > 0.0) && !(r_d > 0.0)) return USP_ERR_INVALID_ARG;  // homogeneous
  const double c_u = (r_eta > 0.0 ? r_eta : r_d) / norm_v;
  const double c_J = (r_d > 0.0 ? r_d : r_eta) / norm_v;
  const double su = std::sqrt(c_u);
  for (int64_t i = 0; i < n; ++i) {
    V_out[i] = (float)((eta[i] - etabar) / c_u);
    V_out[n + i] = (float)((1.0 / D[i] - dbar) / c_J);
  }
  for (int64_t i = 0; i < (1 + ndim) * n; ++i) y_out[2 * i] = y_out[2 * i + 1] = 0.f;
  for (int64_t i = 0; i < n; ++i) y_out[2 * i] = (float)(S[i] / su);
  params_out[0] = etabar / c_u + 1.0;
  params_out[1] = dbar / c_J + 1.0;
  params_out[2] = 1.0 / std::sqrt(c_u * c_J);
  if (scales_out) {
    scales_out[0] = c_u;
    scales_out[1] = c_J;
  }
  return USP_OK;
}
