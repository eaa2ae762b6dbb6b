// Host build of the integer-pipe sine/cosine (isincos.cuh) for a CPU test:
// reads angles (one per line) on stdin and prints "sin cos" with 17 digits.
#include <cstdio>
#include <cstdlib>

#define __host__
#define __device__
#define __forceinline__ inline
#include "isincos.cuh"

int main()
{
    double x;
    while (std::scanf("%lf", &x) == 1) {
        double s, c;
        pf::int_sincos_core(x, pf::kITrigTable, &s, &c);
        std::printf("%.17g %.17g\n", s, c);
    }
    return 0;
}
