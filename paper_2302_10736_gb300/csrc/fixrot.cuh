// fixrot.cuh - the angle-difference product of the element-wise method and
// its coupling product,
//     E_t = V_o conj(U_q) = v_o e^{j (theta_o - theta_q)},   G_t = conj(Yc_t) E_t   (Eqs. 5-6),
// in 64-bit fixed point on the integer pipe.
//
// On GB300 an FP64 operation costs as much issue time of the SM's FP64 pipe as
// about two 64-bit integer multiply-highs cost of its integer pipes, and the
// element-wise evaluation is bound by the FP64 pipe.  The complex product E_t
// (4 FP64 operations per terminal, plus 2 per bus for V = v U) therefore runs
// on the integer pipes, from the phasor step's fixed-point sine and cosine:
//
//   * U = (C, S) = 2^62 (cos theta, sin theta) as signed 64-bit integers
//     (isincos.cuh, before its final rounding);
//   * V_o in block floating point: A = floor(M C / 2^64), floor(M S / 2^64) with
//     M = 2^10 times the 53-bit significand of v_o, so that V_o = A 2^(e - 1083)
//     with e the biased exponent of v_o, |A| < 2^61;
//   * B = A conj(U_q) by three signed multiply-highs (Gauss's complex product):
//     E = B 2^(e - 1081), |B| < 2^60;
//   * Yc_t in block floating point (its larger component exact, per-terminal
//     exponent, formed at setup) and G = conj(Yc) B by three more;
//   * each component of G (or of E) rounded once to the nearest double (ties
//     away from zero) by a leading-zero count and a shift.
//
// The truncations leave an absolute error below 2^-56 |v_o| = 2^-56 |E| in
// each component of E before its rounding, and about 2^-53 |G| in each
// component of G, so that after its rounding each component of G is within
// 2^-52 |G| (the FP64 products they replace round four times at 2^-53).
// Angles that are not finite, v_o with a biased exponent outside
// [kFixExpMin, kFixExpMax] (zero, subnormal, or beyond 2^957 in magnitude),
// and Yc or products outside the range take FP64 products instead
// (fix_E_slow, fix_G): IEEE semantics, NaN propagation included.  The same
// functions compiled for the host are checked against 50-digit products by a
// CPU test.
#pragma once

#include <cstdint>

#include "isincos.cuh"

namespace pf {

// marker of a fixed-point value that is not representable (non-finite angle,
// or v outside the fixed-point exponent range)
constexpr int64_t kFixNaN = (int64_t)0x8000000000000000ull;
constexpr int kFixExpMin = 64, kFixExpMax = 1980;

__host__ __device__ __forceinline__ int64_t s64_mulhi(int64_t a, int64_t b)
{
#ifdef __CUDA_ARCH__
    return __mul64hi((long long)a, (long long)b);
#else
    return (int64_t)(((__int128)a * b) >> 64);
#endif
}

// x 2^(e1 - 1085) as the nearest double (ties away from zero), |x| < 2^63;
// the caller keeps the result normal (e1 - 63 >= 1, e1 <= 2046)
__host__ __device__ __forceinline__ double fix_to_double(int64_t x, int e1)
{
    const uint64_t sg = (uint64_t)x & 0x8000000000000000ull;
    const uint64_t u = sg ? 0ull - (uint64_t)x : (uint64_t)x;
    const int lz = clz64(u) & 63;   // u = 0 is handled by the select below
    const uint64_t un = u << lz;
    const uint64_t mant = (un >> 11) + ((un >> 10) & 1ull);
    // the significand's leading bit adds one to the exponent field
    const uint64_t bits = ((uint64_t)(e1 - lz) << 52) + mant;
    return bits_dbl(u ? (bits | sg) : 0ull);
}

// biased exponent of v
__host__ __device__ __forceinline__ int fix_vexp(double v) { return (int)((dbl_bits(v) >> 52) & 0x7ff); }

// V = v (C, S) 2^-62 in block floating point: (*ar, *ai) 2^(fix_vexp(v) - 1083);
// *ar = kFixNaN if C is the marker or v is outside the exponent range
__host__ __device__ __forceinline__ void fix_phasor(int64_t C, int64_t S, double v, int64_t *ar, int64_t *ai)
{
    const uint64_t bits = dbl_bits(v);
    const int ev = (int)((bits >> 52) & 0x7ff);
    if (C == kFixNaN || ev < kFixExpMin || ev > kFixExpMax) {
        *ar = kFixNaN;
        *ai = 0;
        return;
    }
    const int64_t M = (int64_t)(((bits & 0x000fffffffffffffull) | (1ull << 52)) << 10);   // [2^62, 2^63)
    int64_t r = s64_mulhi(C, M), i = s64_mulhi(S, M);
    if (bits >> 63) {
        r = -r;
        i = -i;
    }
    *ar = r;
    *ai = i;
}

// cos and sin (2^62-scaled, or the marker) as doubles: NaN for the marker
__host__ __device__ __forceinline__ double fix_q62_or_nan(int64_t x)
{
    return x == kFixNaN ? bits_dbl(0x7ff8000000000000ull) : q62_to_double(x);
}

// E = v_o (c_o + j s_o) conj(c_q + j s_q) by FP64 products (the values the
// fixed-point form does not represent)
__host__ __device__ __forceinline__ void fix_E_slow(double vo, int64_t Co, int64_t So, int64_t Cq, int64_t Sq,
                                                    double *er, double *ei)
{
    const double co = fix_q62_or_nan(Co), so = Co == kFixNaN ? co : q62_to_double(So);
    const double cq = fix_q62_or_nan(Cq), sq = Cq == kFixNaN ? cq : q62_to_double(Sq);
    const double Vr = vo * co, Vi = vo * so;
    *er = fma(Vr, cq, Vi * sq);
    *ei = fma(Vi, cq, -Vr * sq);
}

// E = V_o conj(U_q) in fixed point: (Ar, Ai) = fix_phasor(Co, So, vo) and
// (Cq, Sq) = U_q, neither the marker
__host__ __device__ __forceinline__ void fix_E_fast(int64_t Ar, int64_t Ai, double vo, int64_t Cq, int64_t Sq,
                                                    double *er, double *ei)
{
    const int64_t br = s64_mulhi(Ar, Cq) + s64_mulhi(Ai, Sq);
    const int64_t bi = s64_mulhi(Ai, Cq) - s64_mulhi(Ar, Sq);
    const int e1 = fix_vexp(vo) + 4;   // E = B 2^(e - 1081)
    *er = fix_to_double(br, e1);
    *ei = fix_to_double(bi, e1);
}

// E = V_o conj(U_q): (Ar, Ai) = fix_phasor(Co, So, vo), (Cq, Sq) = U_q
__host__ __device__ __forceinline__ void fix_E(int64_t Ar, int64_t Ai, double vo, int64_t Co, int64_t So, int64_t Cq,
                                               int64_t Sq, double *er, double *ei)
{
    if (Ar == kFixNaN || Cq == kFixNaN)
        fix_E_slow(vo, Co, So, Cq, Sq, er, ei);
    else
        fix_E_fast(Ar, Ai, vo, Cq, Sq, er, ei);
}

// A complex constant y = (yr, yi) (a coupling constant Yc, a Ybus value) in
// block floating point: (*fr, *fi) 2^(e - 1084) with e the larger biased
// exponent of yr, yi (the larger component exact, in [2^61, 2^62), so that the
// sums of components in fix_mul stay below 2^63); returns e, or 0 if y is
// zero, subnormal, non-finite or beyond the exponent range (the kernels then
// multiply in FP64).  Setup arithmetic.
__host__ __device__ __forceinline__ int fix_block(double yr, double yi, int64_t *fr, int64_t *fi)
{
    const int er = fix_vexp(yr), ei = fix_vexp(yi);
    const int e = er > ei ? er : ei;
    if (e < kFixExpMin || e > kFixExpMax) {
        *fr = 0;
        *fi = 0;
        return 0;
    }
    const double sc = bits_dbl((uint64_t)(1084 - e + 1023) << 52);   // 2^(1084 - e), exact products
#ifdef __CUDA_ARCH__
    *fr = __double2ll_rn(yr * sc);
    *fi = __double2ll_rn(yi * sc);
#else
    *fr = (int64_t)llrint(yr * sc);
    *fi = (int64_t)llrint(yi * sc);
#endif
    return e;
}

// a conj(b) 2^-64 and a b 2^-64 of two fixed-point complex numbers by three
// multiply-highs each (Gauss's product: k1 = br (ar + ai), then a conj(b) =
// (k1 - ai (br - bi), k1 - ar (br + bi)) and a b = (k1 - ai (br + bi),
// k1 + ar (bi - br))); every component sum of a and of b must stay below 2^63
// in magnitude, and each result component is within 2 units of the exact one
__host__ __device__ __forceinline__ void fix_mul_conj(int64_t ar, int64_t ai, int64_t br, int64_t bi, int64_t *r,
                                                      int64_t *i)
{
    const int64_t k1 = s64_mulhi(br, ar + ai);
    *r = k1 - s64_mulhi(ai, br - bi);
    *i = k1 - s64_mulhi(ar, br + bi);
}
__host__ __device__ __forceinline__ void fix_mul(int64_t ar, int64_t ai, int64_t br, int64_t bi, int64_t *r,
                                                 int64_t *i)
{
    const int64_t k1 = s64_mulhi(br, ar + ai);
    *r = k1 - s64_mulhi(ai, br + bi);
    *i = k1 + s64_mulhi(ar, bi - br);
}

// G = conj(Yc) V_o conj(U_q) (= dS_t/dv_q) entirely in fixed point: (Ar, Ai) =
// fix_phasor(Co, So, vo) and (Cq, Sq) = U_q not the marker, (Yr, Yi, ey) =
// fix_block(Yc) with ey != 0.  Returns false (nothing written) when the
// product's exponent leaves the range of normal doubles.
__host__ __device__ __forceinline__ bool fix_G_fast(int64_t Ar, int64_t Ai, double vo, int64_t Cq, int64_t Sq,
                                                    int64_t Yr, int64_t Yi, int ey, double *gr, double *gi)
{
    const int e1 = ey + fix_vexp(vo) - 1016;   // G = g 2^(ey + e_o - 2101), |g| < 2^58
    if (e1 < 64 || e1 > 2046) return false;
    int64_t br, bi, g_r, g_i;
    fix_mul_conj(Ar, Ai, Cq, Sq, &br, &bi);   // E = B 2^(e_o - 1081)
    fix_mul_conj(br, bi, Yr, Yi, &g_r, &g_i);   // conj(Yc) E
    *gr = fix_to_double(g_r, e1);
    *gi = fix_to_double(g_i, e1);
    return true;
}

// The Ybus method's products for entry (i, j) in fixed point (Eqs. 3-4):
// YU = Y_ij U_j (|yu| < 2^61, YU = yu 2^(ey - 1082)) and dS_i/dv_j =
// V_i conj(YU), from (Yr, Yi, ey) = fix_block(Y_ij) with ey != 0, (C, S) = U_j
// and (Ar, Ai) = fix_phasor of V_i, neither the marker.  Returns false
// (nothing written) when dS_i/dv_j's exponent leaves the range of normal
// doubles.
__host__ __device__ __forceinline__ bool fix_ybus_entry(int64_t Yr, int64_t Yi, int ey, int64_t C, int64_t S,
                                                        int64_t Ar, int64_t Ai, double vi, double *yur,
                                                        double *yui, double *svr, double *svi)
{
    const int e1 = ey + fix_vexp(vi) - 1016;   // dS/dv = sv 2^(ey + e_i - 2101), |sv| < 2^58
    if (e1 < 64 || e1 > 2046) return false;
    int64_t ur, ui, sr, si;
    fix_mul(Yr, Yi, C, S, &ur, &ui);
    fix_mul_conj(Ar, Ai, ur, ui, &sr, &si);
    *yur = fix_to_double(ur, ey + 3);
    *yui = fix_to_double(ui, ey + 3);
    *svr = fix_to_double(sr, e1);
    *svi = fix_to_double(si, e1);
    return true;
}

// Y_ij U_j alone (the injections): yu 2^(ey - 1082) rounded to doubles
__host__ __device__ __forceinline__ void fix_ybus_yu(int64_t Yr, int64_t Yi, int ey, int64_t C, int64_t S,
                                                     double *yur, double *yui)
{
    int64_t ur, ui;
    fix_mul(Yr, Yi, C, S, &ur, &ui);
    *yur = fix_to_double(ur, ey + 3);
    *yui = fix_to_double(ui, ey + 3);
}

// G = conj(Yc) E: the fixed-point product where it applies, else E (fixed
// point or FP64 products) and conj(Yc) E in FP64
__host__ __device__ __forceinline__ void fix_G(int64_t Ar, int64_t Ai, double vo, int64_t Co, int64_t So, int64_t Cq,
                                               int64_t Sq, int64_t Yr, int64_t Yi, int ey, double ycr, double yci,
                                               double *gr, double *gi)
{
    if (Ar != kFixNaN && Cq != kFixNaN && ey != 0 && fix_G_fast(Ar, Ai, vo, Cq, Sq, Yr, Yi, ey, gr, gi)) return;
    double er, ei;
    fix_E(Ar, Ai, vo, Co, So, Cq, Sq, &er, &ei);
    *gr = fma(ycr, er, yci * ei);
    *gi = fma(ycr, ei, -yci * er);
}

// 2 v, exact: the exponent field incremented on the integer pipe (zero,
// subnormal, huge and non-finite v by an FP64 addition)
__host__ __device__ __forceinline__ double fix_twice(double v)
{
    const uint64_t bits = dbl_bits(v);
    const uint64_t e = (bits >> 52) & 0x7ff;
    return (e == 0 || e >= 0x7fe) ? v + v : bits_dbl(bits + (1ull << 52));
}

#ifdef __CUDACC__
// cos and sin of x, 2^62-scaled (library sincos for |x| >= 2^16, scaled and
// rounded; kFixNaN for inf and NaN)
__device__ __forceinline__ void int_sincos_q62(double x, const ITrig *tab, int64_t *c_out, int64_t *s_out)
{
    const int hi = __double2hiint(x) & 0x7fffffff;
    if (hi >= 0x40f00000) {
        if (hi >= 0x7ff00000) {
            *c_out = kFixNaN;
            *s_out = kFixNaN;
            return;
        }
        double s, c;
        sincos(x, &s, &c);
        *c_out = __double2ll_rn(c * 0x1p62);
        *s_out = __double2ll_rn(s * 0x1p62);
        return;
    }
    int_sincos_fix(x, tab, c_out, s_out);
}
#endif

}  // namespace pf
