// FP64 reciprocal for the pivots of the coarse factorisations.
//
// An FP64 division is a chain of dependent FP64 instructions, and on this GPU
// each FP64 warp instruction holds its sub-partition's FP64 unit for about
// 64 cycles, so a pivot's reciprocal is formed from the hardware estimate
// (rcp.approx.ftz.f64, on the special-function unit) and one step of
// Halley's method for f(x) = 1/x - d: with e = 1 - d x0,
//   x1 = x0 + x0 (e + e^2),
// whose relative error is of order e^3 (Halley's iteration converges
// cubically).  Three FMAs replace the division; tests/test_gpu_rcp64.py holds
// the result to IEEE 1/d over random values of many binades.  Subnormal
// inputs flush to zero (the estimate is .ftz): a pivot that small is
// reported as singular before it gets here.
#pragma once

namespace cams {

__device__ __forceinline__ double rcp_halley(double d) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
  const double e = fma(-d, x, 1.0);
  return fma(x, fma(e, e, e), x);
}

}  // namespace cams
