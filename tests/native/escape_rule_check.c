/* The two-float decisions for large escapes, restated in C with the same
 * float operations as the device helpers quant_big and dequant_big
 * (csrc/common.cuh), checked against the double-precision rules they stand
 * for: q = rint(fl64(c / w)) and fl32(fl64(q * w)).  Inputs crowd the
 * rounding boundaries: half-integer quotients and their float neighbours,
 * near-ties, products placed on float midpoints or one double ulp beside
 * them, widths outside the split range, huge q.  Build without contraction
 * (-ffp-contract=off) so every operation rounds once, as the __*_rn
 * intrinsics do.  Prints the counts; exits 1 on any mismatch.
 * Usage: escape_rule_check [cases per width] */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct { float hi, lo; } Split;

static Split split_width(double w) {
    Split s = {0.f, 0.f};
    if (w >= 0x1p-60 && w <= 0x1p60) {
        s.hi = (float)w;
        s.lo = (float)(w - (double)s.hi);
    }
    return s;
}

static long fallback_q, fallback_d;

static int quant_big(float c, Split ws, double w, int32_t* qo) {
    const float q0 = c / ws.hi;
    if (fabsf(q0) < 0x1p21f) {
        const float r = fmaf(-q0, ws.hi, c);
        const float r2 = fmaf(-q0, ws.lo, r);
        const float q1 = r2 / ws.hi;
        const float k0 = rintf(q0);
        const float f = (q0 - k0) + q1;
        const float n = rintf(f);
        const float g = f - n;
        if (fabsf(g) < 0.5f - 0x1p-16f) {
            *qo = (int32_t)k0 + (int32_t)n;
            return 1;
        }
    }
    ++fallback_q;
    const double qd = rint((double)c / w);
    if (fabs(qd) > 2147483647.0) return 0;
    *qo = (int32_t)qd;
    return 1;
}

static float bits_to_float(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t float_to_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

static float dequant_big(int32_t q, Split ws, double w) {
    if (q > -(1 << 24) && q < (1 << 24)) {
        const float qf = (float)q;
        const float p0 = qf * ws.hi;
        const float e0 = fmaf(qf, ws.hi, -p0);
        const float s = fmaf(qf, ws.lo, e0);
        const float f = p0 + s;
        const float bb = f - p0;
        const float err = (p0 - (f - bb)) + (s - bb);
        const uint32_t b = float_to_bits(f);
        const uint32_t ex = (b >> 23) & 0xFFu;
        if (ex >= 64u && ex < 255u && (b & 0x7FFFFFu) != 0u) {
            const float lim = bits_to_float((ex - 24u) << 23) * (1.f - 0x1p-15f);
            if (fabsf(err) < lim) return f;
        }
    }
    ++fallback_d;
    return (float)((double)q * w);
}

static uint64_t state = 88172645463325252ull;
static uint64_t next_u64(void) {   /* xorshift64 */
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return state;
}
static double unit(void) { return (double)(next_u64() >> 11) * 0x1p-53; }

int main(int argc, char** argv) {
    const long per = argc > 1 ? atol(argv[1]) : 1000000;
    const double widths[] = {1.0, 0x1p-10, 0.1, 3.7e-3, 1e-7, 123.456, 0x1p-70, 0x1p70,
                             3.0 * 0x1p-22, 1.0 / 3.0, 1e-12, 7e5};
    long nq = 0, bad_q = 0, nd = 0, bad_d = 0;
    for (int wi = 0; wi < 12; ++wi) {
        const double w = widths[wi];
        const Split ws = split_width(w);
        for (long i = 0; i < per; ++i) {
            const int64_t k = 4200 + (int64_t)(unit() * ((1 << 21) - 4200));
            double t;
            switch (i % 4) {
                case 0: t = (double)k + 0.5; break;                                 /* ties */
                case 1: t = (double)k + unit(); break;                              /* random */
                case 2: t = (double)k + 0.5 + (unit() - 0.5) * 1e-6 * (double)k; break;   /* near */
                default: t = 4200.0 + unit() * 3e9; break;                          /* large */
            }
            float c = (float)(t * w);
            const int step = (int)(next_u64() % 7) - 3;   /* float neighbours */
            for (int j = 0; j < abs(step); ++j) c = nextafterf(c, step > 0 ? INFINITY : -INFINITY);
            if (next_u64() & 1) c = -c;
            if (!(fabs((double)c / w) >= 4200.0)) continue;
            int32_t q = 0;
            const int ok = quant_big(c, ws, w, &q);
            const double ref = rint((double)c / w);
            const int ok_ref = fabs(ref) <= 2147483647.0;
            ++nq;
            if (ok != ok_ref || (ok && q != (int32_t)ref)) {
                if (bad_q < 5) printf("quotient mismatch: c=%a w=%a q=%d ref=%.1f\n", c, w, q, ref);
                ++bad_q;
            }
        }
        for (long i = 0; i < per; ++i) {
            int64_t q;
            switch (i % 3) {
                case 0: q = 4096 + (int64_t)(unit() * ((1 << 24) - 4096)); break;
                case 1: q = (int64_t)(unit() * 2147483647.0); break;
                default: q = 4096 + (int64_t)(next_u64() % 100000); break;
            }
            if (next_u64() & 1) q = -q;
            double ww = w;
            if (i % 5 == 0) {   /* a width that puts q * w on a float midpoint */
                const float f = (float)(1.0 + unit()) * 1024.f;
                const double mid = (double)f + (double)(nextafterf(f, INFINITY) - f) / 2;
                ww = mid / (double)q;
                const int sh = (int)(next_u64() % 3) - 1;
                if (sh) ww = nextafter(ww, sh > 0 ? INFINITY : -INFINITY);
            }
            const float got = dequant_big((int32_t)q, split_width(ww), ww);
            const float ref = (float)((double)q * ww);
            ++nd;
            if (float_to_bits(got) != float_to_bits(ref)) {
                if (bad_d < 5) printf("product mismatch: q=%lld w=%a got=%a ref=%a\n", (long long)q, ww, got, ref);
                ++bad_d;
            }
        }
    }
    printf("quotients %ld mismatches %ld double fallbacks %ld\n", nq, bad_q, fallback_q);
    printf("products %ld mismatches %ld double fallbacks %ld\n", nd, bad_d, fallback_d);
    return (bad_q || bad_d) ? 1 : 0;
}
