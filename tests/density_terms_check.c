/* Host check of the identity the binary64 sweep's density sum relies on.
 *
 * The sweep sums a site's Q pulled binary64 values exactly in a 64-bit
 * fixed-point integer whose unit is 2^(emax - 1075 - GB), emax the largest
 * biased exponent among them and GB = 10 - ceil(log2 Q) guard bits.  Two ways
 * of rounding each term to that unit are compared here:
 *
 *   A (definition): sign(v) * floor(|v| / unit + 1/2), summed;
 *   B (the sweep's form): t = (mantissa << (GB + 1)) >> rs, complemented for a
 *     negative value, summed in four partials together with the count of odd
 *     t; each partial's (sum t + #odd) is even and its half is the partial's
 *     rounded sum.
 *
 * Exit status 0 when every case agrees bit for bit.  Usage: prog [cases] */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static uint64_t state = 0x243f6a8885a308d3ull;
static uint64_t next(void)
{
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static int ceil_log2(int q)
{
    int r = 0;
    while ((1 << r) < q) ++r;
    return r;
}

static uint64_t bits(double v)
{
    uint64_t b;
    memcpy(&b, &v, 8);
    return b;
}

/* A: each term rounded to the unit, ties away from zero. */
static long long term_a(double v, int emax, int gb)
{
    uint64_t b = bits(v);
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0; /* zero or subnormal: below any unit used (emax >= 64) */
    uint64_t m = (b & 0xfffffffffffffull) | (1ull << 52);
    int rs = emax - e; /* |v| / unit = m * 2^(gb - rs) */
    long long t;
    if (rs <= gb) t = (long long)(m << (gb - rs));
    else if (rs - gb > 60) t = 0;
    else {
        int sh = rs - gb;
        t = (long long)((m + (1ull << (sh - 1))) >> sh);
    }
    return (b >> 63) ? -t : t;
}

/* B: doubled resolution, sign by complement. */
static long long term_b(double v, int emax, int gb)
{
    uint64_t b = bits(v);
    int32_t hi = (int32_t)(b >> 32);
    int e = (hi >> 20) & 0x7ff;
    uint64_t m = ((b & 0xfffffffffffffull) | (1ull << 52)) << (gb + 1);
    int rs = emax - e;
    uint64_t r = rs >= 64 ? 0 : m >> rs;
    return (long long)r ^ (long long)(hi >> 31);
}

int main(int argc, char** argv)
{
    long cases = argc > 1 ? atol(argv[1]) : 200000;
    static const int qs[8] = {5, 9, 13, 19, 25, 81, 111, 169};
    long checked = 0, bad = 0;
    for (long it = 0; it < cases; ++it) {
        int q = qs[it % 8];
        int gb = 10 - ceil_log2(q);
        int n = (it % 3) ? q : 1 + (int)(next() % (uint64_t)q);
        double v[169];
        double scale = ldexp(1.0, (int)(next() % 200) - 100);
        for (int k = 0; k < n; ++k) {
            int kind = (int)(next() % 16);
            double x;
            if (kind == 0) x = 0.0;
            else if (kind == 1) x = -0.0;
            else if (kind == 2) /* few mantissa bits: exact ties are common */
                x = ldexp((double)((int64_t)(next() % 64) - 32), (int)(next() % 60) - 40) * scale;
            else if (kind == 3) x = ldexp((double)(next() >> 11), -1074); /* tiny */
            else x = ((double)(next() >> 11) * 0x1p-53 - 0.5) * ldexp(scale, (int)(next() % 40) - 20);
            v[k] = x;
        }
        int emax = 0;
        for (int k = 0; k < n; ++k) {
            int e = (int)((bits(v[k]) >> 52) & 0x7ff);
            if (e > emax) emax = e;
        }
        if (emax == 0x7ff || emax < 64) continue; /* the sweep sums these in binary64 */
        long long sa = 0;
        for (int k = 0; k < n; ++k) sa += term_a(v[k], emax, gb);
        long long part[4] = {0, 0, 0, 0};
        int odd[4] = {0, 0, 0, 0};
        for (int k = 0; k < n; ++k) {
            long long t = term_b(v[k], emax, gb);
            part[k % 4] += t;
            odd[k % 4] += (int)(t & 1);
        }
        long long sb = 0;
        for (int j = 0; j < 4; ++j) {
            long long w = part[j] + odd[j];
            if (w & 1) {
                printf("odd partial: q=%d n=%d\n", q, n);
                return 2;
            }
            sb += w >> 1;
        }
        ++checked;
        if (sa != sb) {
            if (bad < 5) printf("mismatch: q=%d n=%d emax=%d A=%lld B=%lld\n", q, n, emax, sa, sb);
            ++bad;
        }
    }
    printf("checked %ld mismatches %ld\n", checked, bad);
    return bad != 0;
}
