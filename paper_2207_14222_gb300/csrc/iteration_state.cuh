// iteration_state.cuh -- device-side bookkeeping of Algorithm 1's
// convergence test, shared by every kernel that finishes an iteration.
#pragma once

#include "kernels.h"

namespace usp {

// Iteration bookkeeping after ||Delta||^2 is known (Algorithm 1's test).
// hist may be nullptr (a replica of the state that keeps no history).
__device__ __forceinline__ void finalize_iteration(DevState* st, double* hist, double sumsq, int flags) {
  const double nrm = sqrt(sumsq);
  if (flags & F_REF) {
    st->ref = nrm;
    if (!isfinite(nrm)) {
      st->status = ST_NONFINITE;
      st->done = 1;
    }
    return;
  }
  if (st->it >= st->it_limit) {  // never write past the history buffer
    st->status = ST_MAXIT;
    st->done = 1;
    return;
  }
  st->sumsq = sumsq;
  if (!isfinite(nrm)) {
    st->last_r = nrm;
    st->status = ST_NONFINITE;
    st->done = 1;
    return;
  }
  double ref = st->ref;
  if (ref <= 0.0) {  // x0 = 0: Delta_1 = B (L+I)^-1 y, the reference itself
    ref = nrm;
    st->ref = nrm;
  }
  const double r = ref > 0.0 ? nrm / ref : 0.0;
  const int it = st->it;
  if (hist) hist[it] = r;
  st->it = it + 1;
  st->last_r = r;
  if (it == st->phase_start) {
    st->phase_first_r = r;
    st->best_r = r;
    st->best_it = it + 1;
  }
  if (r < st->tol || ref == 0.0) {
    st->status = ST_CONVERGED;
    st->done = 1;
    return;
  }
  if (it > st->phase_start && r > 4.0 * st->phase_first_r) {
    st->status = ST_DIVERGED;
    st->done = 1;
    return;
  }
  if (it + 1 >= st->it_limit) {
    st->status = ST_MAXIT;
    st->done = 1;
    return;
  }
  if (st->stall_window > 0) {
    if (r < st->best_r * (1.0 - 1e-3)) {
      st->best_r = r;
      st->best_it = it + 1;
    } else if (it + 1 - st->best_it >= st->stall_window) {
      st->status = ST_STAGNATED;
      st->done = 1;
    }
  }
}

// The symbol of problem p (batch) or the scalar one.
__device__ __forceinline__ Sym<float> problem_sym(const Sym<float>& s, const Batch& b, int p) {
  Sym<float> r = s;
  if (b.sym32) {
    const float4 c = b.sym32[p];
    r.a_re = c.x;
    r.a_im = c.y;
    r.b_re = c.z;
    r.b_im = c.w;
  }
  return r;
}
__device__ __forceinline__ Sym<double> problem_sym(const Sym<double>& s, const Batch& b, int p) {
  Sym<double> r = s;
  if (b.sym64) {
    r.a_re = b.sym64[4 * p];
    r.a_im = b.sym64[4 * p + 1];
    r.b_re = b.sym64[4 * p + 2];
    r.b_im = b.sym64[4 * p + 3];
  }
  return r;
}

}  // namespace usp
