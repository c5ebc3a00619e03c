/* Host check of the quotient from a reciprocal used by the FP64 substitution
 * chains of the tile kernels: q = RN(a r) with r = RN(1 / d), then one
 * correction RN(q + RN(a - q d) r) with fused multiply-adds (Markstein's
 * theorem), a zero quotient keeping the sign of q.  Counts the pairs (a, d)
 * whose result differs, bit for bit, from the IEEE quotient a / d.
 * Compiled with -ffp-contract=off so that only the written fma() calls fuse.
 *
 * usage: div_rcp_check <random pairs>; prints "pairs <n> mismatches <m>". */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static uint64_t st[2] = {0x9E3779B97F4A7C15ull, 0xD1B54A32D192ED03ull};
static uint64_t next(void) { /* xorshift128+ */
    uint64_t s1 = st[0];
    const uint64_t s0 = st[1];
    st[0] = s0;
    s1 ^= s1 << 23;
    st[1] = s1 ^ s0 ^ (s1 >> 17) ^ (s0 >> 26);
    return st[1] + s0;
}
static uint64_t bits(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }
static double from_bits(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }
/* random normal double with exponent in [emin, emax] and a random sign */
static double rnd(int emin, int emax) {
    const uint64_t m = next() & ((1ull << 52) - 1);
    const int e = emin + (int)(next() % (uint64_t)(emax - emin + 1));
    return from_bits(((uint64_t)(e + 1023) << 52) | m | ((next() & 1) << 63));
}
static double div_rcp(double a, double d, double r) {
    const double q = a * r;
    const double q1 = fma(fma(-q, d, a), r, q);
    return (bits(q) << 1) == 0 ? q : q1;
}
static long n, bad;
static void check(double a, double d) {
    const double r = 1.0 / d;
    ++n;
    if (bits(div_rcp(a, d, r)) != bits(a / d)) {
        if (bad < 5) fprintf(stderr, "mismatch a=%a d=%a\n", a, d);
        ++bad;
    }
}
int main(int argc, char **argv) {
    const long pairs = argc > 1 ? atol(argv[1]) : 10000000;
    for (long i = 0; i < pairs; ++i) {
        double a = rnd(-60, 60), d = rnd(-30, 30);
        /* significands close to 2 (1/d and a/d near a binade edge) */
        if ((i & 3) == 0) d = from_bits(bits(d) | 0x000FFFFFFFFFFF00ull);
        if ((i & 7) == 1) a = from_bits(bits(a) | 0x000FFFFFFFFFFF00ull);
        check(a, d);
    }
    /* integer quotients and remainders (the integer-exact Cholesky tests) */
    for (long a = -400; a <= 400; ++a)
        for (long d = 1; d <= 400; ++d) check((double)a, (double)d);
    /* pivots that are square roots of integers */
    for (long k = 1; k < 200000; ++k)
        for (int j = -3; j <= 3; ++j) check((double)(7 * k + j) * 0.5, sqrt((double)k));
    /* signed zeros and exact quotients */
    check(0.0, 3.0); check(-0.0, 3.0); check(0.0, -3.0); check(-0.0, -3.0);
    check(6.0, 3.0); check(-1.0, 0.5); check(1.0, 3.0);
    printf("pairs %ld mismatches %ld\n", n, bad);
    return 0;
}
