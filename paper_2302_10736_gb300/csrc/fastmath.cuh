// fastmath.cuh - FP64 sine/cosine and reciprocal with few FP64-pipe
// instructions, for the phasor step (the GB300 FP64 pipe is the binding
// resource of this library).
//
// sincos: table-driven method (Gal 1986; Tang 1990) with Cody-Waite additive
// range reduction (Cody & Waite 1980):
//   x = k * (2 pi / N) + r,  k = nearest integer to x N / (2 pi),  |r| <= pi/N,
//   cos x = cos(a_k) cos r - sin(a_k) sin r,  sin x = sin(a_k) cos r + cos(a_k) sin r,
// with N = 256, a table of (cos a_k, sin a_k), a_k = 2 pi k / N, and the Taylor
// polynomials of sin r (to r^5) and cos r - 1 (to r^6) whose truncation errors
// are below 2e-18 for |r| <= pi/256.  2 pi / N is split as C1 + C2, C1 with 33
// significant bits so k C1 is exact for |k| < 2^20.  |x| >= 2^16 (and NaN,
// inf) falls back to the library sincos.  Error: a few ulp (checked against
// the library in the GPU tests).  15 FP64 instructions on the fast path.
//
// rcp: the hardware's approximate reciprocal refined by two Newton-Raphson
// steps y <- y + y (1 - v y) (quadratic convergence from ~23 correct bits);
// 4 FMAs.  Zero or subnormal v is not supported (flushed).
#pragma once

#include <cstdint>

namespace pf {

// table size; `tab` below holds (cos, sin)(2 pi k / 256), k = 0..255
constexpr int kTrigN = 256;
// copies of the table in global memory: every CTA of a launch copies one into
// shared memory at its start, and kTrigCopies copies spread those reads over
// many L2 lines instead of 32
constexpr int kTrigCopies = 64;

__device__ __forceinline__ void fast_sincos(double x, const double2 *__restrict__ tab, double *s_out,
                                            double *c_out)
{
    const int hi = __double2hiint(x);
    if ((hi & 0x7fffffff) >= 0x40f00000) {   // |x| >= 2^16, inf or NaN
        sincos(x, s_out, c_out);
        return;
    }
    const double kInvStep = 0x1.45f306dc9c883p+5;   // 256 / (2 pi)
    const double kShift = 0x1.8p52;                 // 1.5 * 2^52: rounds to an integer in the low bits
    const double kC1 = 0x1.921fb544p-6;             // 2 pi / 256, first 33 bits
    const double kC2 = 0x1.0b4611a626331p-40;       // 2 pi / 256 - kC1
    const double t = fma(x, kInvStep, kShift);
    const int k = __double2loint(t);                // nearest integer (two's complement low bits)
    const double kd = t - kShift;
    double r = fma(-kd, kC1, x);
    r = fma(-kd, kC2, r);
    const double r2 = r * r;
    // sin r = r + r^3 (-1/6 + r^2 / 120)
    const double ps = fma(r2, 1.0 / 120.0, -1.0 / 6.0);
    const double sr = fma(r * r2, ps, r);
    // cos r - 1 = r^2 (-1/2 + r^2 (1/24 - r^2 / 720))
    const double pc = fma(r2, -1.0 / 720.0, 1.0 / 24.0);
    const double cm1 = r2 * fma(r2, pc, -0.5);
    const double2 a = tab[k & (kTrigN - 1)];
    *c_out = fma(a.x, cm1, fma(-a.y, sr, a.x));
    *s_out = fma(a.y, cm1, fma(a.x, sr, a.y));
}

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
