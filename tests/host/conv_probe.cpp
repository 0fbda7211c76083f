// Host-side check of the integer FP64 <-> FP32 conversions (hg_internal.cuh):
// for each input line "d <hex of a double>" prints the bits of d2f(x); for
// "f <hex of a float>" the bits of f2d(x).
#include <inttypes.h>
#include <stdio.h>
#include <string.h>

#include "hg_internal.cuh"

int main()
{
    char kind[4];
    unsigned long long v;
    while (scanf("%3s %llx", kind, &v) == 2) {
        if (kind[0] == 'd') {
            const float r = hg::d2f(hg::double_of(v));
            printf("%08x\n", hg::bits_of(r));
        } else {
            const double r = hg::f2d(hg::float_of((unsigned int)v));
            printf("%016llx\n", hg::bits_of(r));
        }
    }
    return 0;
}
