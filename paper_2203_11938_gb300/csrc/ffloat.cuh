// Float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48
// significant bits.  GB300 issues FP64 arithmetic at a small fraction of its FP32 rate, so
// the FP32 mode's CG keeps its dot-product sums, its scalars (r.z, alpha, the stopping
// threshold) and its solution accumulator in this form, and turns to FP64 only once per
// solve (the solution vector and the diagnostic copies of the scalars).
//
// Addition: Knuth's two-sum of the high parts, the low parts added to its error, then a
// fast two-sum renormalisation (Dekker 1971; the "sloppy" double-double addition of Hida,
// Li and Bailey).  Product with a float: Dekker's exact product, its error term taken with
// one fused multiply-add.  The explicit round-to-nearest intrinsics keep the compiler from
// contracting or reassociating the error terms away.
#pragma once

#include <cuda_runtime.h>

namespace cloth {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
  const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, t);
  return {hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

// a * x for a float-float a and a float x
__device__ __forceinline__ FF ff_mul(FF a, float x) {
  const float p = __fmul_rn(a.hi, x);
  const float e = __fmaf_rn(a.hi, x, -p);  // exact: a.hi * x = p + e
  const float t = __fmaf_rn(a.lo, x, e);
  const float hi = __fadd_rn(p, t);
  return {hi, __fsub_rn(t, __fsub_rn(hi, p))};
}

// nearest float-float of a double (hi is the double rounded to float)
__host__ __device__ __forceinline__ FF ff_from_double(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }

// a / b: float quotient, its remainder a - q1 b formed in float-float, one correction term
// (the double-double division of Hida, Li and Bailey, carried out on float pairs).  The
// two partial quotients come from the fast float division (within 2 ulp): the remainder
// is formed from the q1 actually taken, so the result keeps about 44 bits (relative error
// <= 6.5e-14 in an emulation over 20,000 quotients, against 1.6e-14 with correctly rounded
// partial quotients); it sits on the per-iteration serial chain of every CG solve.
__device__ __forceinline__ FF ff_div(FF a, FF b) {
  const float q1 = __fdividef(a.hi, b.hi);
  const FF r = ff_add(a, ff_neg(ff_mul(b, q1)));
  const float q2 = __fdividef(r.hi, b.hi);
  const float hi = __fadd_rn(q1, q2);
  return {hi, __fsub_rn(q2, __fsub_rn(hi, q1))};
}

// a <= b for normalised pairs
__device__ __forceinline__ bool ff_le(FF a, FF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

__device__ __forceinline__ FF ff_warp_sum(FF x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const FF y = {__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)};
    x = ff_add(x, y);
  }
  return x;
}

}  // namespace cloth
