// Host check of the integer-pipe TwoSum error term (mp_eft_int.cuh) against the
// host's binary64 arithmetic: for every pair the function accepts (bad == 0) its
// result must equal e = (a - (s - v)) + (b - v), v = s - a, s = a + b bit for
// bit (Algorithm 2); inside the documented domain it must accept.  Both forms:
// the default one and the one that also packs subnormal error terms.
//   usage: eft_int_check <pairs> <seed>     exit 0 = pass
#define __host__
#define __device__
#define __forceinline__ inline
#include "../paper_2603_14926_gb300/csrc/mp_eft_int.cuh"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

static uint64_t bits(double x) { uint64_t u; std::memcpy(&u, &x, 8); return u; }
static double dbl(uint64_t u) { double x; std::memcpy(&x, &u, 8); return x; }

static uint64_t state;
static uint64_t next()  // splitmix64
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double make(int e, uint64_t frac, bool neg) { return dbl((neg ? 1ull << 63 : 0) | ((uint64_t)e << 52) | frac); }

static double random_frac_double(int emin, int emax)
{
    uint64_t f = next() & ((1ull << 52) - 1);
    switch (next() % 6) {
    case 0: f = 0; break;                                  // power of two
    case 1: f = (1ull << 52) - 1; break;                   // all ones
    case 2: f &= ~((1ull << (next() % 52)) - 1); break;    // trailing zeros
    default: break;
    }
    return make(emin + (int)(next() % (uint64_t)(emax - emin + 1)), f, next() & 1);
}

static long checked = 0, accepted = 0, wrong = 0, refused_in_domain = 0;
static long schecked = 0, saccepted = 0, swrong = 0, srefused = 0;
static long pchecked = 0, paccepted = 0, pwrong = 0, prefused = 0;

// TwoProd error term against the host's correctly rounded fma
static void check_prod(double a, double b, bool in_domain)
{
    volatile double p = a * b;
    const double e = std::fma(a, b, -p);
    uint32_t bad = 0;
    const uint64_t got = mp::eft_int::two_prod_err(bits(a), bits(b), bits(p), bad);
    pchecked++;
    if (bad) {
        if (in_domain) {
            if (prefused < 5) std::printf("product refused in domain: a=%a b=%a\n", a, b);
            prefused++;
        }
        return;
    }
    paccepted++;
    if (got != bits(e)) {
        if (pwrong < 10) std::printf("product wrong: a=%a b=%a  got %a  want %a\n", a, b, dbl(got), e);
        pwrong++;
    }
}

static void check(double a, double b, bool in_domain)
{
    volatile double s = a + b;
    volatile double v = s - a;
    volatile double t = s - v;
    volatile double x = a - t, y = b - v;
    const double e = x + y;
    uint32_t bad = 0;
    const uint64_t got = mp::eft_int::two_sum_err(bits(a), bits(b), bits(s), bad);
    checked++;
    if (bad) {
        if (in_domain) {
            if (refused_in_domain < 5) std::printf("refused in domain: a=%a b=%a\n", a, b);
            refused_in_domain++;
        }
        return;
    }
    accepted++;
    if (got != bits(e)) {
        if (wrong < 10) std::printf("wrong: a=%a b=%a  got %a  want %a\n", a, b, dbl(got), e);
        wrong++;
    }
}

// The variant that also packs subnormal error terms: its domain is only "both
// exponents <= 2045" (tiny and subnormal operands included).
static void check_sub(double a, double b)
{
    volatile double s = a + b;
    volatile double v = s - a;
    volatile double t = s - v;
    volatile double x = a - t, y = b - v;
    const double e = x + y;
    uint32_t bad = 0;
    const uint64_t got = mp::eft_int::two_sum_err<true>(bits(a), bits(b), bits(s), bad);
    const bool in_domain = ((bits(a) >> 52) & 0x7FF) <= 2045 && ((bits(b) >> 52) & 0x7FF) <= 2045;
    schecked++;
    if (bad) {
        if (in_domain) {
            if (srefused < 5) std::printf("subnormal variant refused in domain: a=%a b=%a\n", a, b);
            srefused++;
        }
        return;
    }
    saccepted++;
    if (got != bits(e)) {
        if (swrong < 10) std::printf("subnormal variant wrong: a=%a b=%a  got %a  want %a\n", a, b, dbl(got), e);
        swrong++;
    }
}

int main(int argc, char **argv)
{
    const long pairs = argc > 1 ? std::atol(argv[1]) : 1000000;
    state = argc > 2 ? std::strtoull(argv[2], nullptr, 10) : 1;
    const double special[] = {0.0, -0.0, 1.0, -1.0, 3.0, 0x1p-1022, -0x1p-1022, 0x1p-1074, 0x1.8p-1030,
                              0x1.fffffffffffffp+1023, -0x1.fffffffffffffp+1022, 0x1p+1023, INFINITY, -INFINITY,
                              NAN, 0x1p-960, 0x1.0000000000001p-960};
    for (double a : special)
        for (double b : special) {
            check(a, b, false);
            check_sub(a, b);
            check_prod(a, b, false);
        }
    for (long i = 0; i < pairs; i++) {
        const int mode = (int)(next() % 10);
        double a = random_frac_double(64, 2045), b;
        const int ea = (int)((bits(a) >> 52) & 0x7FF);
        bool dom = true;
        if (mode < 5) {  // exponent gap 0..70
            const int gap = (int)(next() % 71);
            int eb = ea - gap;
            if (eb < 64) eb = 64;
            b = make(eb, next() & ((1ull << 52) - 1), next() & 1);
            if (next() & 1) b = dbl(bits(b) & ~((1ull << (next() % 53)) - 1));
        } else if (mode == 5) {  // near cancellation: -a moved by a few ulps
            b = dbl((bits(a) ^ (1ull << 63)) + (uint64_t)((int64_t)(next() % 9) - 4));
        } else if (mode == 6) {  // zeros
            b = (next() & 1) ? -0.0 : 0.0;
            if (next() % 4 == 0) a = (next() & 1) ? -0.0 : 0.0;
        } else if (mode == 7) {  // tiny and subnormal operands: outside the guaranteed domain
            a = random_frac_double(0, 70);
            b = random_frac_double(0, 70);
            dom = false;
        } else {
            b = random_frac_double(64, 2045);
        }
        if (next() & 1) { const double t = a; a = b; b = t; }
        // the domain: biased exponents <= 2045 and a normal (or zero) error term
        if (((bits(a) >> 52) & 0x7FF) > 2045 || ((bits(b) >> 52) & 0x7FF) > 2045) dom = false;
        if (dom) {
            volatile double s = a + b;
            volatile double v = s - a;
            const double e = (a - (s - v)) + (b - v);
            if (e != 0 && std::fabs(e) < 0x1p-1022) dom = false;
        }
        check(a, b, dom);
        check_sub(a, b);
        if (mode == 7) {  // the subnormal range proper: both operands below 2^-1000, gaps 0..60
            const double c = random_frac_double(0, 22);
            const double d = random_frac_double(0, 22);
            check_sub(c, d);
            check_sub(c, -d);
        }
        // products: exponents spread around the range, ties and zeros included
        {
            double c = random_frac_double(1, 2046), d;
            const int ec = (int)((bits(c) >> 52) & 0x7FF);
            int ed = 2046 - ec + (int)(next() % 1200) - 600;  // product exponent around the middle of the range
            if (ed < 1) ed = 1;
            if (ed > 2046) ed = 2046;
            d = make(ed, next() & ((1ull << 52) - 1), next() & 1);
            if (next() % 8 == 0) d = dbl(bits(d) & ~((1ull << (next() % 53)) - 1));
            if (next() % 16 == 0) d = (next() & 1) ? -0.0 : 0.0;
            if (next() % 32 == 0) c = random_frac_double(0, 3);  // subnormal and tiny operands
            volatile double p = c * d;
            const double e = std::fma(c, d, -p);
            const int pc = (int)((bits(c) >> 52) & 0x7FF), pd = (int)((bits(d) >> 52) & 0x7FF);
            // domain: both operands normal with a finite normal product whose unit 2^(Ea+Eb-2150) is
            // normal (so any nonzero error is normal too), or a zero operand
            const bool pdom = (pc >= 1 && pd >= 1 && pc + pd >= 1128 && std::isfinite(p) &&
                               std::fabs(p) >= 0x1p-1022) || c == 0 || d == 0;
            check_prod(c, d, pdom);
        }
    }
    std::printf("checked %ld accepted %ld wrong %ld refused-in-domain %ld\n", checked, accepted, wrong, refused_in_domain);
    std::printf("products: checked %ld accepted %ld wrong %ld refused-in-domain %ld\n", pchecked, paccepted, pwrong,
                prefused);
    std::printf("subnormal variant: checked %ld accepted %ld wrong %ld refused-in-domain %ld\n", schecked, saccepted,
                swrong, srefused);
    return (wrong || refused_in_domain || pwrong || prefused || swrong || srefused) ? 1 : 0;
}
