// dfloat.cuh -- double-float arithmetic: a real number held as the unevaluated
// sum hi + lo of two FP32 values with |lo| <= ulp(hi)/2 (a 48-bit
// significand), for the refinement residual y - A x.
//
// The operations are built from the error-free transformations of
// floating-point arithmetic: the exact sum a + b = s + e of Knuth's
// two-sum, the same with |a| >= |b| known in advance (Dekker's fast
// two-sum), and the exact product a b = p + e with e from one fused
// multiply-add.  Addition adds the high words exactly, folds in the low
// words and renormalises; its absolute error is a few units of 2^-48
// (|a| + |b|), which is what a transform's normwise error analysis needs
// (the relative error of a sum that cancels can be larger; no step here
// depends on one).  Multiplication forms the exact product of the high
// words and the two cross terms by fused multiply-adds.
//
// Every primitive uses the rounded intrinsics (__fadd_rn, __fmul_rn,
// __fmaf_rn), which the compiler neither contracts into fused operations nor
// reorders, so the error terms are exact as written.
//
// Why: the GPU's FP64 rate is about 1/64 of its FP32 rate, so the residual's
// transforms in double-float (about ten FP32 operations per FP64 operation)
// run several times faster than in FP64, at an accuracy (2^-48 per
// operation) far beyond what the refinement needs.
#pragma once

#include <cuda_runtime.h>

#include "fft_core.cuh"
#include "kernels.h"

namespace usp {

template <> struct cplx_of<dfl> { typedef dfl2 type; };

// s + e = a + b exactly (two-sum, no condition on the magnitudes).
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// p + e = a b exactly (barring underflow).
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return dfl(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a / b: the float quotient of the high words, corrected once by the
// remainder a - q b.
__device__ __forceinline__ dfl quot(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfl r = a - b * dfl(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}

// Per-problem symbol of a batch (coefficients held in FP64 on the device).
__device__ __forceinline__ Sym<dfl> problem_sym(const Sym<dfl>& s, const Batch& b, int p) {
  Sym<dfl> r = s;
  if (b.sym64) {
    r.a_re = dfl(b.sym64[4 * p]);
    r.a_im = dfl(b.sym64[4 * p + 1]);
    r.b_re = dfl(b.sym64[4 * p + 2]);
    r.b_im = dfl(b.sym64[4 * p + 3]);
  }
  return r;
}

}  // namespace usp
