// Host build of the fixed-point angle-difference product (fixrot.cuh) for a
// CPU test.  Reads lines on stdin:
//   "E vo tho thq"  -> prints "er ei" (E = vo e^{j(tho - thq)}, |angles| < 2^16 or not finite)
//   "G vo tho thq yr yi" -> prints "gr gi" (G = conj(yr + j yi) E, fixed point where it applies)
//   "D x e1"        -> prints the bits of fix_to_double(x, e1) in hex
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#define __host__
#define __device__
#define __forceinline__ inline
#include "fixrot.cuh"

static void sincos_fix_host(double x, int64_t *c, int64_t *s)
{
    if (!std::isfinite(x)) {
        *c = *s = pf::kFixNaN;
        return;
    }
    pf::int_sincos_fix(x, pf::kITrigTable, c, s);
}

int main()
{
    char mode[8];
    while (std::scanf("%7s", mode) == 1) {
        if (std::strcmp(mode, "E") == 0) {
            double vo, tho, thq;
            if (std::scanf("%lf %lf %lf", &vo, &tho, &thq) != 3) return 1;
            int64_t Co, So, Cq, Sq, Ar, Ai;
            sincos_fix_host(tho, &Co, &So);
            sincos_fix_host(thq, &Cq, &Sq);
            pf::fix_phasor(Co, So, vo, &Ar, &Ai);
            double er, ei;
            pf::fix_E(Ar, Ai, vo, Co, So, Cq, Sq, &er, &ei);
            std::printf("%.17g %.17g\n", er, ei);
        } else if (std::strcmp(mode, "G") == 0) {
            double vo, tho, thq, yr, yi;
            if (std::scanf("%lf %lf %lf %lf %lf", &vo, &tho, &thq, &yr, &yi) != 5) return 1;
            int64_t Co, So, Cq, Sq, Ar, Ai, Yr, Yi;
            sincos_fix_host(tho, &Co, &So);
            sincos_fix_host(thq, &Cq, &Sq);
            pf::fix_phasor(Co, So, vo, &Ar, &Ai);
            const int ey = pf::fix_block(yr, yi, &Yr, &Yi);
            double gr, gi;
            pf::fix_G(Ar, Ai, vo, Co, So, Cq, Sq, Yr, Yi, ey, yr, yi, &gr, &gi);
            std::printf("%.17g %.17g\n", gr, gi);
        } else if (std::strcmp(mode, "D") == 0) {
            long long x;
            int e1;
            if (std::scanf("%lld %d", &x, &e1) != 2) return 1;
            const double d = pf::fix_to_double((int64_t)x, e1);
            unsigned long long u;
            std::memcpy(&u, &d, 8);
            std::printf("%016llx\n", u);
        } else {
            return 1;
        }
    }
    return 0;
}
