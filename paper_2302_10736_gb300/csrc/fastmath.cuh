// fastmath.cuh - FP64 reciprocal with few FP64-pipe instructions, and sign
// flips on the integer pipe (the GB300 FP64 pipe is the binding resource of
// this library; the sine and cosine are in isincos.cuh).
//
// rcp: the hardware's approximate reciprocal refined by two Newton-Raphson
// steps y <- y + y (1 - v y) (quadratic convergence from ~23 correct bits);
// 4 FMAs.  Zero or subnormal v is not supported (flushed).
#pragma once

#include <cstdint>

namespace pf {

// -x by flipping the sign bit on the integer pipe (exact, and no FP64 instruction)
__device__ __forceinline__ double neg(double x)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// x or -x, chosen per thread without a branch (sign bit on the integer pipe)
__device__ __forceinline__ double neg_if(double x, bool flip)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (flip ? (long long)0x8000000000000000ULL : 0LL));
}

__device__ __forceinline__ double fast_rcp(double v)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(v));
    double e = fma(-v, y, 1.0);
    y = fma(y, e, y);
    e = fma(-v, y, 1.0);
    return fma(y, e, y);
}

}  // namespace pf
