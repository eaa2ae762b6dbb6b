// isincos.cuh - sine and cosine of an FP64 angle computed on the integer
// pipe, for the phasor step U = e^{j theta} (Sec. IV-B.1 step 1).
//
// On GB300 the FP64 pipe issues about 2 thread-operations per cycle per SM,
// the integer pipes 64 each, so a sine/cosine written as fixed-point integer
// arithmetic costs a fraction of the FP64 issue time of a floating-point one
// and leaves the FP64 pipe to the method's own products.  The method:
//
//   1. Exact reduction to turns (Payne & Hanek 1983): x = m 2^(e-1075) with
//      the 53-bit significand m, and phi = frac(x / (2 pi)) as a 64-bit
//      fixed-point fraction of a turn, from the product of m with the first
//      128 bits of 1/(2 pi) (floor(2^129 / pi)).  |x| < 2^16 keeps every bit
//      of phi that matters inside that product; |x| < 4 needs only its upper
//      64 bits (phi then within one unit of its last place).
//   2. Table method (Tang 1990): the nearest of 256 points a_k = 2 pi k / 256,
//      k = round(256 phi), leaves rho = x - a_k with |rho| <= pi / 256; k's top
//      two bits select the quadrant and its low six bits one of 64 entries
//      (cos a_j, sin a_j) of the first quadrant, held as 62-bit fractions.
//   3. Taylor polynomials of sin rho (to rho^7) and 1 - cos rho (to rho^6) in
//      fixed point; the first omitted terms are below 2e-20; the products
//      feeding the three smallest terms use 32-bit multiplies.
//   4. cos(a_j + rho), sin(a_j + rho) by the angle-addition formulas, the
//      quadrant by swapping and negating, and each result rounded once to the
//      nearest double (leading-zero count, shift, round half up).
//
// Every product is the high word of a 64 x 64-bit product.  The truncation
// errors of the fixed-point steps are below 2^-60 in absolute value, so the
// results are within one rounding of the exact sine and cosine (checked
// against the library's sincos in the GPU tests).  |x| >= 2^16, inf and NaN
// take the library sincos.  The constants are bits of 1/(2 pi), 2 pi and
// reciprocal factorials (checked by a CPU test that recomputes them from
// Machin's formula).
#pragma once

#include <cstdint>

#ifndef __CUDACC__
#include <cstring>
#endif

namespace pf {

// entries of the first-quadrant table (cos, sin)(2 pi j / 256), j = 0 .. 63,
// each a fraction scaled by 2^62
constexpr int kITrigN = 64;
// copies of the table in global memory (CTAs spread their reads over them)
constexpr int kITrigCopies = 64;

struct alignas(16) ITrig {
    uint64_t c, s;
};

// round(2^62 cos(2 pi j / 256)), round(2^62 sin(2 pi j / 256)), j = 0 .. 63
// (checked by a CPU test that recomputes them from a Taylor series in exact
// integer arithmetic)
constexpr ITrig kITrigTable[kITrigN] = {
    {0x4000000000000000ull, 0x0000000000000000ull},
    {0x3ffb10c1099a1976ull, 0x0192155f7a3667e0ull},
    {0x3fec43c6f2dafbc7ull, 0x0323ecbe21bb027dull},
    {0x3fd39b5a0310742aull, 0x04b54824b3867d73ull},
    {0x3fb11b47a24a4b3cull, 0x0645e9af0a6d0af8ull},
    {0x3f84c8e1c33fa68full, 0x07d59395aa5cc38dull},
    {0x3f4eaafe114a2d43ull, 0x0964083747309d11ull},
    {0x3f0ec9f4e297526bull, 0x0af10a22459fe32aull},
    {0x3ec52f9feeb96056ull, 0x0c7c5c1e34d3055bull},
    {0x3e71e758c9cb118aull, 0x0e05c1353f27b17eull},
    {0x3e14fdf72461ae55ull, 0x0f8cfcbd90af8d58ull},
    {0x3dae81ced092c67aull, 0x1111d262b1f67761ull},
    {0x3d3e82ad8c5bb4bbull, 0x1294062ed59f05a9ull},
    {0x3cc511d891c223ddull, 0x14135c9417660143ull},
    {0x3c424209ed0dc97full, 0x158f9a75ab1fdcfeull},
    {0x3bb6276d998478c2ull, 0x17088530fa459eafull},
    {0x3b20d79e651a8c51ull, 0x187de2a6aea962d2ull},
    {0x3a8269a29b927359ull, 0x19ef7943a8ed8a2eull},
    {0x39daf5e8798ee5e2ull, 0x1b5d1009e15cc02bull},
    {0x392a96426823e9edull, 0x1cc66e9931c45e17ull},
    {0x387165e3017b61a4ull, 0x1e2b5d3806f63b1eull},
    {0x37af8158df2a533full, 0x1f8ba4dbf89ab9fbull},
    {0x36e5068a32dc7b22ull, 0x20e70f3245ffdb2dull},
    {0x361214b02a03ff37ull, 0x223d66a836964508ull},
    {0x3536cc521d434606ull, 0x238e76735cd190d9ull},
    {0x34534f408c4f03bbull, 0x24da0a99ba25bd51ull},
    {0x3367c08fe70e8168ull, 0x261feff9c2e069c2ull},
    {0x3274449324c7f69full, 0x275ff45240a17279ull},
    {0x317900d62a2e816aull, 0x2899e64a123bac30ull},
    {0x30761c17ff2edba4ull, 0x29cd9577c7cbd228ull},
    {0x2f6bbe44d55f5dbcull, 0x2afad26919d93f45ull},
    {0x2e5a106fdfff2c87ull, 0x2c216eaa3a59bdb7ull},
    {0x2d413cccfe779921ull, 0x2d413cccfe779921ull},
    {0x2c216eaa3a59bdb7ull, 0x2e5a106fdfff2c87ull},
    {0x2afad26919d93f45ull, 0x2f6bbe44d55f5dbcull},
    {0x29cd9577c7cbd228ull, 0x30761c17ff2edba4ull},
    {0x2899e64a123bac30ull, 0x317900d62a2e816aull},
    {0x275ff45240a17279ull, 0x3274449324c7f69full},
    {0x261feff9c2e069c2ull, 0x3367c08fe70e8168ull},
    {0x24da0a99ba25bd51ull, 0x34534f408c4f03bbull},
    {0x238e76735cd190d9ull, 0x3536cc521d434606ull},
    {0x223d66a836964508ull, 0x361214b02a03ff37ull},
    {0x20e70f3245ffdb2dull, 0x36e5068a32dc7b22ull},
    {0x1f8ba4dbf89ab9fbull, 0x37af8158df2a533full},
    {0x1e2b5d3806f63b1eull, 0x387165e3017b61a4ull},
    {0x1cc66e9931c45e17ull, 0x392a96426823e9edull},
    {0x1b5d1009e15cc02bull, 0x39daf5e8798ee5e2ull},
    {0x19ef7943a8ed8a2eull, 0x3a8269a29b927359ull},
    {0x187de2a6aea962d2ull, 0x3b20d79e651a8c51ull},
    {0x17088530fa459eafull, 0x3bb6276d998478c2ull},
    {0x158f9a75ab1fdcfeull, 0x3c424209ed0dc97full},
    {0x14135c9417660143ull, 0x3cc511d891c223ddull},
    {0x1294062ed59f05a9ull, 0x3d3e82ad8c5bb4bbull},
    {0x1111d262b1f67761ull, 0x3dae81ced092c67aull},
    {0x0f8cfcbd90af8d58ull, 0x3e14fdf72461ae55ull},
    {0x0e05c1353f27b17eull, 0x3e71e758c9cb118aull},
    {0x0c7c5c1e34d3055bull, 0x3ec52f9feeb96056ull},
    {0x0af10a22459fe32aull, 0x3f0ec9f4e297526bull},
    {0x0964083747309d11ull, 0x3f4eaafe114a2d43ull},
    {0x07d59395aa5cc38dull, 0x3f84c8e1c33fa68full},
    {0x0645e9af0a6d0af8ull, 0x3fb11b47a24a4b3cull},
    {0x04b54824b3867d73ull, 0x3fd39b5a0310742aull},
    {0x0323ecbe21bb027dull, 0x3fec43c6f2dafbc7ull},
    {0x0192155f7a3667e0ull, 0x3ffb10c1099a1976ull},
};

namespace isc {
// floor(2^129 / pi) = floor(2^130 / (2 pi)): the first 128 bits of 1/(2 pi)
constexpr uint64_t kInv2PiHi = 0xa2f9836e4e441529ull;
constexpr uint64_t kInv2PiLo = 0xfc2757d1f534ddc0ull;
// round(2 pi 2^61)
constexpr uint64_t kTwoPi61 = 0xc90fdaa22168c235ull;
// round(2^64 / n) and round(2^54 / n)
constexpr uint64_t kInv6 = 0x2aaaaaaaaaaaaaabull;
constexpr uint64_t kInv24 = 0x0aaaaaaaaaaaaaabull;
constexpr uint64_t kInv120 = 0x0222222222222222ull;
constexpr uint64_t kInv720_54 = 0x16c16c16c16cull;
constexpr uint64_t kInv5040_54 = 0x034034034034ull;
}  // namespace isc

__host__ __device__ __forceinline__ uint64_t u64_mulhi(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ uint64_t dbl_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
#endif
}

__host__ __device__ __forceinline__ double bits_dbl(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

__host__ __device__ __forceinline__ int clz64(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)u);
#else
    return u ? __builtin_clzll(u) : 64;
#endif
}

// a b 2^-64 from the upper 32 bits of a (a < 2^62) and of b 2^-sb (below 2^32):
// one 32 x 32-bit product, for the polynomial terms that need few bits (the
// truncations are below 2^-29 of the product)
__host__ __device__ __forceinline__ uint64_t mulhi_short(uint64_t a, uint64_t b, int sb)
{
    return ((uint64_t)(uint32_t)(a >> 32) * (uint64_t)(uint32_t)(b >> sb)) >> (32 - sb);
}

// v 2^-62 as the nearest double (ties rounded up in magnitude), |v| <= 2^63
__host__ __device__ __forceinline__ double q62_to_double(int64_t v)
{
    const uint64_t sg = (uint64_t)v & 0x8000000000000000ull;
    const uint64_t u = sg ? 0ull - (uint64_t)v : (uint64_t)v;
    const int lz = clz64(u) & 63;   // u = 0 is handled by the select below
    const uint64_t un = u << lz;
    const uint64_t mant = (un >> 11) + ((un >> 10) & 1ull);
    // the significand's leading bit adds one to the exponent field
    const uint64_t bits = ((uint64_t)(1023 - lz) << 52) + mant;
    return bits_dbl(u ? (bits | sg) : 0ull);
}

// cos x and sin x for |x| < 2^16 (finite) as fractions scaled by 2^62 (|.| <= 2^62);
// tab: the 64-entry first-quadrant table
__host__ __device__ __forceinline__ void int_sincos_fix(double x, const ITrig *tab, int64_t *c_out, int64_t *s_out)
{
    using namespace isc;
    const uint64_t bits = dbl_bits(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    const uint64_t m = (bits & 0x000fffffffffffffull) | (e ? (1ull << 52) : 0ull);
    // m C, C = floor(2^129 / pi): its words above 2^64 (the lowest word only
    // holds bits far below the 64 fraction bits kept).  For |x| < 4 the
    // product with C's lowest word (below 2^53) moves the fraction of a turn
    // by less than one unit of its last place (2^-64) and is left out.
    const uint64_t L1 = m * kInv2PiHi;
    const uint64_t H1 = u64_mulhi(m, kInv2PiHi);
    uint64_t P1 = L1, P2 = H1;
    if (e > 1024) {
        const uint64_t H0 = u64_mulhi(m, kInv2PiLo);
        P1 = L1 + H0;
        P2 = H1 + (P1 < L1 ? 1ull : 0ull);
    }
    // x / (2 pi) = m C 2^(e - 1205): the fraction of a turn is bits
    // [s, s + 64) of (P2, P1) with s = 1077 - e (>= 39 for |x| < 2^16)
    int s = 1077 - (e ? e : 1);
    s = s > 127 ? 127 : s;
    const uint64_t lo = (P1 >> (s & 63)) | (P2 << ((64 - s) & 63));
    const uint64_t hi = P2 >> ((s - 64) & 63);
    uint64_t phi = s < 64 ? lo : hi;
    if (bits >> 63) phi = 0ull - phi;
    // nearest table point: k = round(256 phi) mod 256, rho = 2 pi r 2^-64
    const int64_t r = (int64_t)(phi << 8) >> 8;
    const uint32_t k = (uint32_t)((phi - (uint64_t)r) >> 56);
    const bool rneg = r < 0;
    const uint64_t u = rneg ? 0ull - (uint64_t)r : (uint64_t)r;   // <= 2^55
    const uint64_t X = u64_mulhi(u << 8, kTwoPi61);                // |rho| 2^69
    const uint64_t A = u64_mulhi(X, X);                            // rho^2 2^74
    // |sin rho| = |rho| (1 - rho^2 (1/6 - rho^2 (1/120 - rho^2 / 5040)))
    // (A < 2^62; the terms rho^7 / 5040, rho^5 / 120 and rho^6 / 720 need 6,
    // 25 and 16 significant bits of their products: 32-bit products suffice)
    const uint64_t p3 = kInv120 - mulhi_short(A, kInv5040_54, 10);  // 2^64
    const uint64_t p2 = kInv6 - (mulhi_short(A, p3, 26) >> 10);     // 2^64
    const uint64_t sr = X - (u64_mulhi(X, u64_mulhi(A, p2)) >> 10);   // |sin rho| 2^69
    // 1 - cos rho = rho^2 (1/2 - rho^2 (1/24 - rho^2 / 720))
    const uint64_t q2 = kInv24 - mulhi_short(A, kInv720_54, 13);    // 2^64
    const uint64_t q1 = (1ull << 63) - (u64_mulhi(A, q2) >> 10);   // 2^64
    const uint64_t cm = u64_mulhi(A, q1);                          // (1 - cos rho) 2^74
    const ITrig t = tab[k & (kITrigN - 1)];                        // 2^62
    const int64_t c_cm = (int64_t)(u64_mulhi(t.c, cm) >> 10);      // 2^62
    const int64_t s_cm = (int64_t)(u64_mulhi(t.s, cm) >> 10);
    const int64_t c_sr = (int64_t)(u64_mulhi(t.c, sr) >> 5);       // 2^62
    const int64_t s_sr = (int64_t)(u64_mulhi(t.s, sr) >> 5);
    // cos(a_j + rho) = c (1 - (1 - cos rho)) - s sin rho, sin(a_j + rho) = s (...) + c sin rho
    const int64_t C = ((int64_t)t.c - c_cm) + (rneg ? s_sr : -s_sr);
    const int64_t S = ((int64_t)t.s - s_cm) + (rneg ? -c_sr : c_sr);
    // quadrant q = k >> 6: rotate by q quarter turns
    const uint32_t q = (k >> 6) & 3u;
    int64_t cq = (q & 1u) ? -S : C;
    int64_t sq = (q & 1u) ? C : S;
    if (q & 2u) {
        cq = -cq;
        sq = -sq;
    }
    *c_out = cq;
    *s_out = sq;
}

// sin x and cos x for |x| < 2^16 (finite), each rounded once to the nearest double
__host__ __device__ __forceinline__ void int_sincos_core(double x, const ITrig *tab, double *s_out, double *c_out)
{
    int64_t cq, sq;
    int_sincos_fix(x, tab, &cq, &sq);
    *c_out = q62_to_double(cq);
    *s_out = q62_to_double(sq);
}

#ifdef __CUDACC__
// the library sincos for |x| >= 2^16, inf and NaN
__device__ __forceinline__ void int_sincos(double x, const ITrig *tab, double *s_out, double *c_out)
{
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40f00000) {
        sincos(x, s_out, c_out);
        return;
    }
    int_sincos_core(x, tab, s_out, c_out);
}
#endif

}  // namespace pf
