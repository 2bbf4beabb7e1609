// fp64.cuh - FP64 helpers shared by the line-solve kernels (internal).
#pragma once

#include <cuda_runtime.h>

namespace mgs {

// 1 / v by Newton-Raphson iteration r <- r + r (1 - v r) from the hardware's
// single-precision approximate reciprocal (relative error below 2^-22, squared
// by each step: two steps reach double precision, within an ulp of 1/v).
// Values whose seed would leave the single-precision range take an IEEE
// division instead.
__device__ __forceinline__ double rcp64(double v) {
    const int e = (__double2hiint(v) >> 20) & 0x7ff;   // biased exponent
    if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / v;
    float s;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(__double2float_rn(v)));
    double r = (double)s;
    r = __fma_rn(r, __fma_rn(-v, r, 1.0), r);
    return __fma_rn(r, __fma_rn(-v, r, 1.0), r);
}

}  // namespace mgs
