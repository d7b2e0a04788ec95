// Host check of fqsl::bits::narrow_exact: for float bit patterns of every
// exponent (every 127th mantissa and the edge mantissas), narrowing the
// exactly widened double gives back the same float, bit for bit (NaN: a NaN).
// Prints the number of patterns checked and of mismatches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "bits.cuh"

static int check(unsigned u)
{
    float f;
    memcpy(&f, &u, 4);
    const float g = fqsl::bits::narrow_exact((double)f);
    if (isnan(f)) return isnan(g) ? 0 : 1;
    unsigned v;
    memcpy(&v, &g, 4);
    return v == u ? 0 : 1;
}

int main()
{
    long long n = 0, bad = 0;
    const unsigned edges[] = {0u, 1u, 2u, 3u, 0x400000u, 0x7ffffeu, 0x7fffffu};
    for (unsigned s = 0; s < 2; s++)
        for (unsigned e = 0; e < 256; e++) {
            for (unsigned m = 0; m < 0x800000u; m += 127u) {
                bad += check((s << 31) | (e << 23) | m);
                n++;
            }
            for (unsigned m : edges) {
                bad += check((s << 31) | (e << 23) | m);
                n++;
            }
        }
    printf("%lld %lld\n", n, bad);
    return bad != 0;
}
